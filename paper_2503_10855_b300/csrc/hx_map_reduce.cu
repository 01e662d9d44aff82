// hx_map_reduce.cu -- fused map -> sum reduce (one fork of factor n).
//
// Lowering: the fork is chunked into tiles of consecutive elements (the
// fork-chunk of Sec. 2.2), each tile's partial starts from the identity
// (monoid-reassociate, Sec. 5.2), and the tile partials are combined by a
// second level (fork-fission into a producer and a consumer, Sec. 5.2).  On
// the GPU the producer is one launch in which every warp stores one tile
// partial (no fence, no same-address atomic), and the consumer is a
// one-CTA launch chained with programmatic dependent launch that folds the
// partials in the fixed order of mr_final_cta.  Inside a tile the leaf
// reduction is a per-lane compensated fold, then a warp-shuffle butterfly,
// the warp reductions of Sec. 4.4.
#include "hx_internal.cuh"

namespace hx {

// One warp per tile, kMrWarpsPerCta tiles per CTA; no block-level barrier.
// A warp only stores its tile partial; map_reduce_final_kernel folds them.
// Three load groups per operand in flight (124 registers, 8 CTAs of two
// warps per SM): measured on B300 against two groups at 6 or 7 CTAs of four
// warps per SM, it is the fastest from 2^22 to 2^28 elements.
__global__ void __launch_bounds__(kMrWarpsPerCta * kWarp)
map_reduce_kernel(const float *__restrict__ x, const float *__restrict__ y, float *__restrict__ out,
                  float a, MrPlan p, bool aligned, WsSlot *ws) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const int64_t tile = (int64_t)blockIdx.x * kMrWarpsPerCta + (threadIdx.x >> 5);
    if (tile >= p.tiles) return;
    if (!HX_CHECK(tile * p.tile_elems < p.n, kChkMapTile, tile, p.n)) return;
    if (!HX_CHECK(tile < kMrMaxTiles, kChkMapPartial, tile, kMrMaxTiles)) return;
    const ff part = mr_tile<3>(x, y, out, a, p, tile, aligned, threadIdx.x & 31);
    if ((threadIdx.x & 31) == 0) st_keep2(ws->mr_partial + tile, make_float2(part.hi, part.lo));
}

// The consumer level of the tree: one CTA of kMrFoldLanes threads, launched
// after the producer has finished (programmatic dependent launch).
__global__ void __launch_bounds__(kMrFoldLanes) map_reduce_final_kernel(const float2 *partials, int64_t tiles,
                                                                        float *d_sum, double *d_sum64) {
    __shared__ ff red[kMrFoldLanes];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    if (!HX_CHECK(tiles <= kMrMaxTiles, kChkMapFold, tiles, kMrMaxTiles)) return;
    const ff sf = mr_final_cta(partials, tiles, red);
    if (threadIdx.x == 0) {
        const double s = ff_to_double(sf);
        *d_sum = (float)s;
        if (d_sum64) *d_sum64 = s;
    }
}

__global__ void map_reduce_empty_kernel(float *d_sum, double *d_sum64) {
    *d_sum = 0.0f;
    if (d_sum64) *d_sum64 = 0.0;
}

static bool overlaps(const void *a, size_t abytes, const void *b, size_t bbytes) {
    const uintptr_t pa = (uintptr_t)a, pb = (uintptr_t)b;
    return pa < pb + bbytes && pb < pa + abytes;
}

HX_CHECKS_READER(checks_map_reduce)

}  // namespace hx

extern "C" hx_status hx_map_reduce(hx_ctx *ctx, const float *x, const float *y, float *out, float a,
                                   int64_t n, float *d_sum, double *d_sum64, hx_stream_t stream) {
    using namespace hx;
    if (!ctx) return fail(HX_ERR_INVALID, "hx_map_reduce: ctx is NULL");
    if (n < 0 || n > HX_MAP_REDUCE_MAX_N) return fail(HX_ERR_INVALID, "hx_map_reduce: n out of range");
    if (!d_sum) return fail(HX_ERR_INVALID, "hx_map_reduce: d_sum is NULL");
    if (n > 0 && (!x || !y)) return fail(HX_ERR_INVALID, "hx_map_reduce: x or y is NULL");
    if ((((uintptr_t)x | (uintptr_t)y | (uintptr_t)out) & 3u) != 0)
        return fail(HX_ERR_INVALID, "hx_map_reduce: fp32 buffers must be 4-byte aligned");
    const size_t bytes = (size_t)n * sizeof(float);
    if (out && n > 0 && (overlaps(out, bytes, x, bytes) || overlaps(out, bytes, y, bytes)))
        return fail(HX_ERR_INVALID, "hx_map_reduce: out overlaps an input");
    DeviceGuard g(ctx->device);
    WsSlot *ws = nullptr;
    hx_status st = slot_for(ctx, stream, &ws);
    if (st != HX_OK) return st;
    if (take_injected_failure(ctx)) return fail(HX_ERR_CUDA, "hx_map_reduce: injected launch failure (test hook)");
    if (n == 0) {
        map_reduce_empty_kernel<<<1, 1, 0, (cudaStream_t)stream>>>(d_sum, d_sum64);
    } else {
        const MrPlan p = mr_plan(n, ctx->tune.map_vecs[size_class(n)]);
        const bool aligned = (((uintptr_t)x | (uintptr_t)y | (uintptr_t)out) & 15u) == 0;
        const unsigned grid = (unsigned)((p.tiles + kMrWarpsPerCta - 1) / kMrWarpsPerCta);
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[0].val.programmaticStreamSerializationAllowed = 1;
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(grid);
        cfg.blockDim = dim3(kMrWarpsPerCta * kWarp);
        cfg.stream = (cudaStream_t)stream;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        cudaError_t e = cudaLaunchKernelEx(&cfg, map_reduce_kernel, x, y, out, a, p, aligned, ws);
        if (e == cudaSuccess) {
            cfg.gridDim = dim3(1);
            cfg.blockDim = dim3(kMrFoldLanes);
            e = cudaLaunchKernelEx(&cfg, map_reduce_final_kernel, (const float2 *)ws->mr_partial, p.tiles, d_sum,
                                   d_sum64);
        }
        if (e != cudaSuccess) return cuda_fail(e, "hx_map_reduce: launch");
        return HX_OK;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "hx_map_reduce: launch");
    return HX_OK;
}
