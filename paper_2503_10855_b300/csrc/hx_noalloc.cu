// hx_noalloc.cu -- map->reduce for callers that may not allocate device memory.
//
// Some callers cannot call cudaMalloc: a plugin whose host application owns
// all device memory through its own pool, or latency-critical code that
// cannot afford an allocation (cudaFree, and sometimes cudaMalloc, can
// synchronise the whole device).  Such a caller cannot even create an
// hx_ctx, because hx_create allocates the workspace.  This file gives it one
// entry point that allocates nothing: the scratch the reduction needs (the
// per-tile partials and the arrival ticket) lives in a file-scope __device__
// array that the CUDA module holds on every device that loads this library,
// until the process exits.  The computation is exactly hx_map_reduce's with
// the built-in default tuning (same tile plan, same fold order: the last
// warp to arrive evaluates the canonical partial fold that hx_map_reduce's
// second launch evaluates with a whole CTA), so the results are the same.
#include <mutex>

#include "hx_internal.cuh"

namespace {

struct NoAllocScratch {
    float2 partial[HX_NOALLOC_MAX_TILES];
    unsigned int ticket;
    unsigned int pad[63];
};
static_assert(hx::kMrMaxTiles == HX_NOALLOC_MAX_TILES, "scratch must hold every tile partial of the plan");

// The scratch itself.  In host code this name is only a stand-in for the
// device object: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) NoAllocScratch g_scratch;

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
NoAllocScratch *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch on `dev` (which must be current), looked up
// once per device.
hx_status scratch_for_device(int dev, NoAllocScratch **out) {
    if (dev < 0 || dev >= kMaxDevices) return hx::fail(HX_ERR_INVALID, "hx_map_reduce_noalloc: device index too large");
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
        if (e != cudaSuccess) return hx::cuda_fail(e, "hx_map_reduce_noalloc: cudaGetSymbolAddress");
        g_scratch_ptr[dev] = static_cast<NoAllocScratch *>(p);
    }
    *out = g_scratch_ptr[dev];
    return HX_OK;
}

__global__ void __launch_bounds__(hx::kMrWarpsPerCta * hx::kWarp)
map_reduce_noalloc_kernel(const float *__restrict__ x, const float *__restrict__ y, float *__restrict__ out, float a,
                          hx::MrPlan p, bool aligned, NoAllocScratch *scratch, float *d_sum, double *d_sum64) {
    const int64_t tile = (int64_t)blockIdx.x * hx::kMrWarpsPerCta + (threadIdx.x >> 5);
    if (tile >= p.tiles) return;
    if (!HX_CHECK(tile < HX_NOALLOC_MAX_TILES, hx::kChkNoAllocTile, tile, HX_NOALLOC_MAX_TILES)) return;
    hx::mr_warp_item(x, y, out, a, p, tile, aligned, scratch->partial, &scratch->ticket, d_sum, d_sum64);
}

__global__ void map_reduce_noalloc_empty_kernel(float *d_sum, double *d_sum64) {
    *d_sum = 0.0f;
    if (d_sum64) *d_sum64 = 0.0;
}

}  // namespace

namespace hx {
HX_CHECKS_READER(checks_noalloc)
}  // namespace hx

extern "C" hx_status hx_map_reduce_noalloc(const float *x, const float *y, float *out, float a, int64_t n,
                                           float *d_sum, double *d_sum64, hx_stream_t stream) {
    using namespace hx;
    if (n < 0 || n > HX_MAP_REDUCE_NOALLOC_MAX_N)
        return fail(HX_ERR_INVALID, "hx_map_reduce_noalloc: n must be in [0, HX_MAP_REDUCE_NOALLOC_MAX_N]");
    if (!d_sum) return fail(HX_ERR_INVALID, "hx_map_reduce_noalloc: d_sum is NULL");
    if (n > 0 && (!x || !y)) return fail(HX_ERR_INVALID, "hx_map_reduce_noalloc: x or y is NULL");
    if ((((uintptr_t)x | (uintptr_t)y | (uintptr_t)out) & 3u) != 0)
        return fail(HX_ERR_INVALID, "hx_map_reduce_noalloc: fp32 buffers must be 4-byte aligned");
    const size_t bytes = (size_t)n * sizeof(float);
    auto overlaps = [](const void *p, const void *q, size_t len) {
        return (uintptr_t)p < (uintptr_t)q + len && (uintptr_t)q < (uintptr_t)p + len;
    };
    if (out && n > 0 && (overlaps(out, x, bytes) || overlaps(out, y, bytes)))
        return fail(HX_ERR_INVALID, "hx_map_reduce_noalloc: out overlaps an input");
    const MrPlan p = mr_plan(n > 0 ? n : 1);   // the built-in default tile plan
    if (n > 0 && p.tiles > HX_NOALLOC_MAX_TILES)
        return fail(HX_ERR_INVALID, "hx_map_reduce_noalloc: n needs more tile partials than the scratch holds");
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "hx_map_reduce_noalloc: cudaGetDevice");
    if (n == 0) {
        map_reduce_noalloc_empty_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(d_sum, d_sum64);
    } else {
        NoAllocScratch *scratch = nullptr;
        hx_status st = scratch_for_device(dev, &scratch);
        if (st != HX_OK) return st;
        // The scratch keeps the previous call's contents; only the ticket has
        // to start at zero (every tile partial is written before it is read).
        e = cudaMemsetAsync(&scratch->ticket, 0, sizeof(unsigned int), (cudaStream_t)stream);
        if (e != cudaSuccess) return cuda_fail(e, "hx_map_reduce_noalloc: clearing the ticket");
        const bool aligned = (((uintptr_t)x | (uintptr_t)y | (uintptr_t)out) & 15u) == 0;
        const unsigned grid = (unsigned)((p.tiles + kMrWarpsPerCta - 1) / kMrWarpsPerCta);
        map_reduce_noalloc_kernel<<<grid, kMrWarpsPerCta * kWarp, 0, (cudaStream_t)stream>>>(
            x, y, out, a, p, aligned, scratch, d_sum, d_sum64);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "hx_map_reduce_noalloc: launch");
    return HX_OK;
}
