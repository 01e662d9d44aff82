// hx_stencil.cu -- clamp-to-edge 5-point Jacobi sweeps fused with a max
// residual reduce.
//
// One sweep is a 2-D fork over the grid (Sec. 3.3) tiled into warp blocks of
// R rows x 128 columns (R tuned per size class), stacked kStWarps to a CTA; a warp loads its rows and halo columns up front
// into registers and takes horizontal neighbours from the adjacent lanes, so
// each input point is read from memory about once per sweep.  The max of
// |u' - u| is the fused reduction (loop fusion, Sec. 5.1; max reduction tree,
// Sec. 5.2): warp shuffle max, a shared-memory max over the CTA's warps, one
// atomic max per CTA into the workspace (max is exact and order
// independent), and the last CTA to arrive publishes it.  Sweeps form a
// sequential loop (Sec. 4.4 rule 1): one launch each, chained with
// programmatic dependent launch so that a sweep's CTAs are already resident
// when the previous sweep drains.
#include "hx_internal.cuh"

namespace hx {

// A CTA covers one 128-column (or 32-column) strip and kStWarps warp blocks
// stacked vertically; CTAs run row band by row band.  The CTA folds its
// warps' maxima in shared memory and publishes once: one atomic max and one
// arrival ticket per CTA, the last CTA writes the residual.
template <bool VEC, int R>
__global__ void __launch_bounds__(kStWarps * kWarp)
stencil_kernel(const float *__restrict__ src, float *__restrict__ dst, int nx, int ny,
               WsSlot *ws, float *d_resid_t) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    __shared__ float wmax[kStWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c_begin = blockIdx.x * 128;
    const int r_begin = (blockIdx.y * kStWarps + warp) * R;
    float m = 0.0f;
    if (r_begin < ny) {
        m = VEC ? stencil_block_vec<R>(src, dst, nx, ny, c_begin, r_begin)
                : stencil_block_scalar<R>(src, dst, nx, ny, c_begin, r_begin);
    }
    m = warp_max(m);
    if (lane == 0) wmax[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float bm = wmax[0];
        for (int i = 1; i < kStWarps; ++i) bm = fmaxf(bm, wmax[i]);
        atomicMax(&ws->st_max_bits, __float_as_uint(bm));
        __threadfence();
        if (atomicAdd(&ws->st_ticket, 1u) == gridDim.x * gridDim.y - 1) {
            __threadfence();
            *d_resid_t = __uint_as_float(atomicExch(&ws->st_max_bits, 0u));
            ws->st_ticket = 0u;
        }
    }
}

}  // namespace hx

extern "C" hx_status hx_stencil2d(hx_ctx *ctx, float *u0, float *u1, int32_t nx, int32_t ny,
                                  int32_t iters, float *d_resid, int32_t *result_in_u1,
                                  hx_stream_t stream) {
    using namespace hx;
    if (!ctx) return fail(HX_ERR_INVALID, "hx_stencil2d: ctx is NULL");
    if (nx < 1 || ny < 1 || nx > 65536 || ny > 65536 || (int64_t)nx * ny > ((int64_t)1 << 31))
        return fail(HX_ERR_INVALID, "hx_stencil2d: grid size out of range");
    if (iters < 0 || iters > (1 << 20)) return fail(HX_ERR_INVALID, "hx_stencil2d: iters out of range");
    if (!u0 || !u1) return fail(HX_ERR_INVALID, "hx_stencil2d: grid pointer is NULL");
    if (iters > 0 && !d_resid) return fail(HX_ERR_INVALID, "hx_stencil2d: d_resid is NULL");
    if ((((uintptr_t)u0 | (uintptr_t)u1) & 3u) != 0)
        return fail(HX_ERR_INVALID, "hx_stencil2d: grids must be 4-byte aligned");
    const size_t bytes = (size_t)nx * ny * sizeof(float);
    if ((uintptr_t)u0 < (uintptr_t)u1 + bytes && (uintptr_t)u1 < (uintptr_t)u0 + bytes)
        return fail(HX_ERR_INVALID, "hx_stencil2d: u0 and u1 overlap");
    if (result_in_u1) *result_in_u1 = iters & 1;
    if (iters == 0) return HX_OK;
    DeviceGuard g(ctx->device);
    WsSlot *ws = nullptr;
    hx_status st = slot_for(ctx, stream, &ws);
    if (st != HX_OK) return st;

    const bool vec = (nx % 4 == 0) && ((((uintptr_t)u0 | (uintptr_t)u1) & 15u) == 0);
    const int width = 128;   // both paths: 32 lanes x 4 columns
    const int rows = ctx->tune.stencil_rows[size_class((int64_t)nx * ny)];
    dim3 grid((nx + width - 1) / width, (ny + kStWarps * rows - 1) / (kStWarps * rows));
    using KernelFn = void (*)(const float *, float *, int, int, WsSlot *, float *);
    KernelFn fn;
    if (rows == 4) fn = vec ? stencil_kernel<true, 4> : stencil_kernel<false, 4>;
    else if (rows == 16) fn = vec ? stencil_kernel<true, 16> : stencil_kernel<false, 16>;
    else fn = vec ? stencil_kernel<true, 8> : stencil_kernel<false, 8>;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(kStWarps * kWarp);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = (cudaStream_t)stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    for (int t = 0; t < iters; ++t) {
        const float *src = (t & 1) ? u1 : u0;
        float *dst = (t & 1) ? u0 : u1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, fn, src, dst, (int)nx, (int)ny, ws, d_resid + t);
        if (e != cudaSuccess) return cuda_fail(e, "hx_stencil2d: launch");
    }
    return HX_OK;
}
