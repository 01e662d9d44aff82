// hx_stencil.cu -- clamp-to-edge 5-point Jacobi sweeps fused with a max
// residual reduce.
//
// One sweep is a 2-D fork over the grid (Sec. 3.3) tiled into warp blocks of
// R rows x 128 columns (R tuned per size class), stacked kStWarps to a CTA;
// a warp loads its rows and halo columns up front into registers and takes
// horizontal neighbours from the adjacent lanes, so each input point is read
// from memory about once per sweep.  The max of |u' - u| is the fused
// reduction (loop fusion, Sec. 5.1; max reduction tree, Sec. 5.2): warp
// shuffle max, a shared-memory max over the CTA's warps, then one partial per
// CTA, folded for a run of sweeps by a small residual kernel (max is exact
// and order independent); grids with more CTAs than the workspace holds use
// one atomic max per CTA and let the last CTA to arrive publish it instead.
// Sweeps form a sequential loop (Sec. 4.4 rule 1): one launch each, chained
// with programmatic dependent launch so that a sweep's CTAs are already
// resident when the previous sweep drains.
#include "hx_internal.cuh"

namespace hx {

// A CTA covers one 128-column strip and kStWarps warp blocks stacked
// vertically; CTAs run row band by row band.  The CTA folds its warps' maxima
// in shared memory and publishes once.  PART: it stores its maximum at
// part[cta] and a residual kernel reduces the sweep's partials later (no
// same-address atomics in the sweep: at 2048^2 those cost 30 % of a sweep);
// otherwise one atomic max and one arrival ticket per CTA, and the last CTA
// writes the residual.
template <bool VEC, int R, bool PART>
__global__ void __launch_bounds__(kStWarps * kWarp)
stencil_kernel(const float *__restrict__ src, float *__restrict__ dst, int nx, int ny,
               WsSlot *ws, float *d_resid_t, float *part) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    __shared__ float wmax[kStWarps];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c_begin = blockIdx.x * 128;
    const int r_begin = (blockIdx.y * kStWarps + warp) * R;
    float m = 0.0f;
    if (r_begin < ny && HX_CHECK(c_begin < nx, kChkStencilBlock, c_begin, r_begin)) {
        m = VEC ? stencil_block_vec<R>(src, dst, nx, ny, c_begin, r_begin)
                : stencil_block_scalar<R>(src, dst, nx, ny, c_begin, r_begin);
    }
    m = warp_max(m);
    if (lane == 0) wmax[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        float bm = wmax[0];
        for (int i = 1; i < kStWarps; ++i) bm = fmaxf(bm, wmax[i]);
        if (PART) {
            part[blockIdx.y * gridDim.x + blockIdx.x] = bm;
            return;
        }
        atomicMax(&ws->st_max_bits, __float_as_uint(bm));
        __threadfence();
        if (atomicAdd(&ws->st_ticket, 1u) == gridDim.x * gridDim.y - 1) {
            __threadfence();
            *d_resid_t = __uint_as_float(atomicExch(&ws->st_max_bits, 0u));
            ws->st_ticket = 0u;
        }
    }
}

// Residuals of a run of sweeps: CTA t folds the p partial maxima of sweep
// t (max is exact, so the order does not matter) into resid[t].
__global__ void __launch_bounds__(256) stencil_resid_kernel(const float *__restrict__ part, int p, float *resid) {
    __shared__ float wmax[256 / kWarp];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const float *q = part + (size_t)blockIdx.x * p;
    float m = 0.0f;
    for (int i = threadIdx.x; i < p; i += 256) m = fmaxf(m, __ldcg(q + i));
    m = warp_max(m);
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < 256 / kWarp; ++w) m = fmaxf(m, wmax[w]);
        resid[blockIdx.x] = m;
    }
}

HX_CHECKS_READER(checks_stencil)

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
    if (take_injected_failure(ctx)) return fail(HX_ERR_CUDA, "hx_stencil2d: injected launch failure (test hook)");

    const bool vec = (nx % 4 == 0) && ((((uintptr_t)u0 | (uintptr_t)u1) & 15u) == 0);
    const int width = 128;   // both paths: 32 lanes x 4 columns
    const int rows = ctx->tune.stencil_rows[size_class((int64_t)nx * ny)];
    dim3 grid((nx + width - 1) / width, (ny + kStWarps * rows - 1) / (kStWarps * rows));
    // Partial maxima per sweep go to the stream's nest workspace (free while
    // this call runs: calls on one stream are serial), up to kStPartCap per
    // run of sweeps; grids with more CTAs than that use the atomic path.
    const int64_t p = (int64_t)grid.x * grid.y;
    const bool use_part = p <= kStPartCap;
    float *part = reinterpret_cast<float *>(ctx->nest_ws[ws - ctx->ws].part);
    using KernelFn = void (*)(const float *, float *, int, int, WsSlot *, float *, float *);
    KernelFn fn;
    if (use_part) {
        if (rows == 4) fn = vec ? stencil_kernel<true, 4, true> : stencil_kernel<false, 4, true>;
        else if (rows == 16) fn = vec ? stencil_kernel<true, 16, true> : stencil_kernel<false, 16, true>;
        else fn = vec ? stencil_kernel<true, 8, true> : stencil_kernel<false, 8, true>;
    } else {
        if (rows == 4) fn = vec ? stencil_kernel<true, 4, false> : stencil_kernel<false, 4, false>;
        else if (rows == 16) fn = vec ? stencil_kernel<true, 16, false> : stencil_kernel<false, 16, false>;
        else fn = vec ? stencil_kernel<true, 8, false> : stencil_kernel<false, 8, false>;
    }
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
    const int per_run = use_part ? (int)(kStPartCap / p) : iters;
    for (int t0 = 0; t0 < iters; t0 += per_run) {
        const int t1 = t0 + per_run < iters ? t0 + per_run : iters;
        for (int t = t0; t < t1; ++t) {
            const float *src = (t & 1) ? u1 : u0;
            float *dst = (t & 1) ? u0 : u1;
            cudaError_t e = cudaLaunchKernelEx(&cfg, fn, src, dst, (int)nx, (int)ny, ws, d_resid + t,
                                               part + (size_t)(t - t0) * p);
            if (e != cudaSuccess) return cuda_fail(e, "hx_stencil2d: launch");
        }
        if (use_part) {
            cudaLaunchConfig_t rc = cfg;
            rc.gridDim = dim3((unsigned)(t1 - t0));
            rc.blockDim = dim3(256);
            cudaError_t e = cudaLaunchKernelEx(&rc, stencil_resid_kernel, (const float *)part, (int)p, d_resid + t0);
            if (e != cudaSuccess) return cuda_fail(e, "hx_stencil2d: residual launch");
        }
    }
    return HX_OK;
}
