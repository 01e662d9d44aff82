// hx_histogram.cu -- 256-bin byte histogram and exclusive scan of the bins.
//
// The histogram is a reduce over a 256-entry collection (Sec. 3.2, 3.3).
// Each CTA keeps private bins in shared memory (a collection constant of a
// block-level fork placed in shared memory, with an extra dimension for the
// thread-level fork, as Sec. 4.4 describes), replicated per slot so that a
// warp's 32 increments always hit 32 different banks.  CTAs then add their
// bins into one of kHiReplicas copies of the bins in the workspace with
// integer atomics (exact and order independent), and the last CTA to arrive
// adds the copies, publishes the bins and runs the exclusive scan (a
// sequential fold over 256 entries, done as a warp-shuffle scan).
#include "hx_internal.cuh"

namespace hx {

template <int THREADS>
__global__ void __launch_bounds__(THREADS)
histogram_kernel(const uint8_t *__restrict__ v, int64_t n, int head, int64_t nvec, int tail,
                 WsSlot *ws, uint32_t *d_bins, uint32_t *d_scan) {
    extern __shared__ __align__(16) unsigned int sh[];   // kHiSmemBytes of counters
    __shared__ unsigned int wtot[kHiBins / kWarp];
    __shared__ bool is_last;
    static_assert(THREADS >= kHiBins, "the finish maps one thread to one bin");
    hist_zero(sh);
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (!HX_CHECK(head + 16 * nvec + tail == n && head < 16 && tail < 16, kChkHistSplit, n, nvec)) nvec = 0;
    const unsigned int slot = hist_slot_offset();
    hist_count_strided(sh, slot, reinterpret_cast<const uint4 *>(v + head),
                       (int64_t)blockIdx.x * THREADS + threadIdx.x, (int64_t)gridDim.x * THREADS, nvec);
    if (blockIdx.x == 0) {   // unaligned head and ragged tail bytes
        if (threadIdx.x < head) hist_count_byte(sh, slot, v[threadIdx.x]);
        if (threadIdx.x < tail) hist_count_byte(sh, slot, v[n - tail + threadIdx.x]);
    }
    __syncthreads();
    if (hist_merge(sh, ws->hi_bins[blockIdx.x % kHiReplicas])) __threadfence();   // only threads that wrote bins
    __syncthreads();
    if (threadIdx.x == 0) is_last = atomicAdd(&ws->hi_ticket, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!is_last || threadIdx.x >= kHiBins) return;
    __threadfence();
    // Final, one thread per bin (the first kHiBins threads): add the copies
    // that CTAs used (reading them from L2, where the atomics were performed)
    // and zero them, publish the bins, exclusive scan over the kHiBins / 32
    // warp totals, reset the ticket.
    const int used = gridDim.x < kHiReplicas ? (int)gridDim.x : kHiReplicas;
    unsigned int part[kHiReplicas];
#pragma unroll
    for (int r = 0; r < kHiReplicas; ++r) part[r] = r < used ? __ldcg(&ws->hi_bins[r][threadIdx.x]) : 0u;
    unsigned int c = 0u;
#pragma unroll
    for (int r = 0; r < kHiReplicas; ++r) {
        c += part[r];
        if (r < used) ws->hi_bins[r][threadIdx.x] = 0u;
    }
    d_bins[threadIdx.x] = c;
    unsigned int incl = c;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned int t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
    }
    if (lane == 31) wtot[warp] = incl;
    // a barrier of the kHiBins threads still running (named barrier 1)
    asm volatile("bar.sync 1, %0;" ::"n"(kHiBins) : "memory");
    unsigned int before = 0u;
#pragma unroll
    for (int w = 0; w < kHiBins / kWarp - 1; ++w)
        if (w < warp) before += wtot[w];
    if (d_scan) d_scan[threadIdx.x] = before + incl - c;
    if (threadIdx.x == 0) ws->hi_ticket = 0u;
}

// Opt the kernels into 64 KiB of dynamic shared memory and record how many
// CTAs of each width fit on an SM (called once per context).
hx_status histogram_setup(hx_ctx *ctx) {
    const int widths[3] = {256, 512, 1024};
    void *fns[3] = {(void *)histogram_kernel<256>, (void *)histogram_kernel<512>, (void *)histogram_kernel<1024>};
    for (int i = 0; i < 3; ++i) {
        cudaError_t e = cudaFuncSetAttribute(fns[i], cudaFuncAttributeMaxDynamicSharedMemorySize, kHiSmemBytes);
        int occ = 0;
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fns[i], widths[i], kHiSmemBytes);
        if (e != cudaSuccess) return cuda_fail(e, "hx_create: histogram kernel set-up");
        ctx->hist_ctas_per_sm[i] = occ > 0 ? occ : 1;
    }
    return HX_OK;
}

HX_CHECKS_READER(checks_histogram)

}  // namespace hx

extern "C" hx_status hx_histogram(hx_ctx *ctx, const uint8_t *v, int64_t n, uint32_t *d_bins,
                                  uint32_t *d_excl_scan, hx_stream_t stream) {
    using namespace hx;
    if (!ctx) return fail(HX_ERR_INVALID, "hx_histogram: ctx is NULL");
    if (n < 0 || n > HX_HISTOGRAM_MAX_N) return fail(HX_ERR_INVALID, "hx_histogram: n out of range");
    if (!d_bins) return fail(HX_ERR_INVALID, "hx_histogram: d_bins is NULL");
    if (n > 0 && !v) return fail(HX_ERR_INVALID, "hx_histogram: v is NULL");
    if ((((uintptr_t)d_bins | (uintptr_t)d_excl_scan) & 3u) != 0)
        return fail(HX_ERR_INVALID, "hx_histogram: bins must be 4-byte aligned");
    DeviceGuard g(ctx->device);
    WsSlot *ws = nullptr;
    hx_status st = slot_for(ctx, stream, &ws);
    if (st != HX_OK) return st;
    if (take_injected_failure(ctx)) return fail(HX_ERR_CUDA, "hx_histogram: injected launch failure (test hook)");
    int head = (int)((16 - ((uintptr_t)v & 15u)) & 15u);
    if (head > n) head = (int)n;
    const int64_t nvec = (n - head) / 16;
    const int tail = (int)((n - head) % 16);
    const int threads = ctx->tune.hist_threads[size_class(n)];
    const int wi = threads == 256 ? 0 : (threads == 512 ? 1 : 2);
    const int64_t want = (nvec + 2 * threads - 1) / (2 * threads);
    const int64_t cap = (int64_t)ctx->num_sms * ctx->hist_ctas_per_sm[wi];
    const int grid = (int)(want < 1 ? 1 : (want > cap ? cap : want));
    cudaStream_t s = (cudaStream_t)stream;
    if (wi == 0) histogram_kernel<256><<<grid, 256, kHiSmemBytes, s>>>(v, n, head, nvec, tail, ws, d_bins, d_excl_scan);
    else if (wi == 1) histogram_kernel<512><<<grid, 512, kHiSmemBytes, s>>>(v, n, head, nvec, tail, ws, d_bins, d_excl_scan);
    else histogram_kernel<1024><<<grid, 1024, kHiSmemBytes, s>>>(v, n, head, nvec, tail, ws, d_bins, d_excl_scan);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "hx_histogram: launch");
    return HX_OK;
}
