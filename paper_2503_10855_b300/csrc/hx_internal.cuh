// hx_internal.cuh -- device building blocks of libhx shared by the standalone
// kernels and the batched persistent kernel.  Each nest is written once, as a
// per-tile device function; a standalone launch runs one tile per CTA and the
// batched kernel runs the same functions on work items, so an instance gives
// bit-identical results alone and inside a batch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdio>
#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "../../include/hx.h"

namespace hx {

// ---------------------------------------------------------------- checks
// In the library's debug build (HX_DEBUG_CHECKS, libhx_debug.so) kernels
// check the index ranges of their work items before using them.  A failed
// check records (code, a, b) -- the first failure only -- and the work item
// is skipped; nothing traps.  The record is per translation unit (the
// library is built without relocatable device code); each kernel file
// defines a reader with HX_CHECKS_READER and hx_debug_checks() asks them
// all.  In the release build HX_CHECK is the constant true.
#ifdef HX_DEBUG_CHECKS
static __device__ unsigned long long g_check_rec[3];
__device__ __forceinline__ bool check_ok(bool ok, int code, long long a, long long b) {
    if (ok) return true;
    if (atomicCAS(&g_check_rec[0], 0ull, (unsigned long long)code) == 0ull) {
        g_check_rec[1] = (unsigned long long)a;
        g_check_rec[2] = (unsigned long long)b;
    }
    return false;
}
#define HX_CHECK(cond, code, a, b) ::hx::check_ok((cond), (code), (long long)(a), (long long)(b))
#define HX_CHECKS_READER(name)                                                                          \
    hx_status name(int32_t *code, int64_t *a, int64_t *b) {                                             \
        unsigned long long r[3] = {0, 0, 0};                                                            \
        cudaError_t e = cudaMemcpyFromSymbol(r, g_check_rec, sizeof r);                                 \
        if (e == cudaSuccess && r[0] != 0) {                                                            \
            const unsigned long long z[3] = {0, 0, 0};                                                  \
            e = cudaMemcpyToSymbol(g_check_rec, z, sizeof z);                                           \
        }                                                                                               \
        if (e != cudaSuccess) return cuda_fail(e, "hx_debug_checks");                                   \
        *code = (int32_t)r[0];                                                                          \
        *a = (int64_t)r[1];                                                                             \
        *b = (int64_t)r[2];                                                                             \
        return HX_OK;                                                                                   \
    }
#else
#define HX_CHECK(cond, code, a, b) true
#define HX_CHECKS_READER(name)                                                                          \
    hx_status name(int32_t *code, int64_t *a, int64_t *b) {                                             \
        *code = 0;                                                                                      \
        *a = 0;                                                                                         \
        *b = 0;                                                                                         \
        return HX_OK;                                                                                   \
    }
#endif
// Check codes (a, b): the values compared.
enum : int {
    kChkMapTile = 1,        // map->reduce tile start past n (tile, n)
    kChkMapPartial = 2,     // tile partial index past the workspace (tile, capacity)
    kChkMapFold = 3,        // tile count of a fold past the workspace (tiles, capacity)
    kChkStencilBlock = 4,   // stencil warp block origin outside the grid (column, row)
    kChkHistSplit = 5,      // histogram head + vectors + tail != n (n, vectors)
    kChkBatchInst = 6,      // batch work item mapped to no instance (instance, count)
    kChkBatchRun = 7,       // batch run past its instance's tiles (last tile, tiles)
    kChkBatchStencil = 8,   // batch stencil block outside its grid (column, row)
    kChkSradTile = 9,       // SRAD region tile index out of range (tile, tiles)
    kChkNoAllocTile = 10,   // no-allocation call's tile past its scratch (tile, capacity)
    // 11 nest chunk partial, 12 nest group partial, 13 nest arrival ticket:
    // checked inside the generated nest kernels (same meaning: index, capacity)
};

// ---------------------------------------------------------------- constants
constexpr int kWarp = 32;

// map->reduce tile plan: a tile is owned by ONE warp; lane l of the tile owns
// the float4 vectors l, l + 32, l + 64, ... (coalesced per step).  Warps work
// independently (no block barriers); the plan (vectors per lane) is a
// function of n only.
constexpr int kMrMinVecs = 4;        // vectors per lane in the smallest tile (one load round)
constexpr int kMrUnroll = 4;         // loads in flight per operand per lane
constexpr int kMrMaxTiles = 4096;    // tile partials per instance (workspace)
// standalone launch: tiles (warps) per CTA.  Two: the grid's CTAs spread
// over the SMs more evenly than with four (2^20 elements, 2048 tiles: 1024
// CTAs, 6-7 per SM, against 512 CTAs, 3-4 per SM); measured on B300, back to
// back, 1-2 % faster from 2^20 to 2^28 than four warps, and eight slower.
constexpr int kMrWarpsPerCta = 2;

// stencil: one warp owns a block of R rows x 128 columns (R tuned per size
// class; kStRows is the default).
constexpr int kStRows = 8;
constexpr int kStWarps = 4;          // warps per CTA, stacked vertically
constexpr int kBatchStRows = 8;      // rows per warp block inside the batched kernel

// histogram: 256 bins; per-CTA shared counters replicated per slot (below).
constexpr int kHiBins = 256;

// ---------------------------------------------------------------- workspace
// The histogram's CTA totals go into kHiReplicas copies of the 256 bins, CTA
// c into copy c mod kHiReplicas, and the last CTA adds the copies.  One copy
// is 1 KiB, 8 lines of L2, whose atomics the L2 performs one after another:
// with a single copy the 256 atomics of each of several hundred CTAs queue on
// those 8 lines (measured on B300: 8 copies take a 2^24-byte call from 11.7
// to 8.9 us and a 2^22-byte one from 7.7 to 6.4 us, 512-thread CTAs; 32 or
// 64 copies are no faster, and 2^26 bytes and more are unchanged).
constexpr int kHiReplicas = 8;

// One slot per stream.  Tickets count arriving tiles; the last arrival does
// the final combine and resets its ticket and accumulators to zero, so a slot
// is clean again when a call's stream work completes.
struct WsSlot {
    float2 mr_partial[kMrMaxTiles];   // (hi, lo) tile partials
    unsigned int hi_bins[kHiReplicas][kHiBins];   // zero between calls
    unsigned int st_ticket;
    unsigned int st_max_bits;   // running max |u'-u| as float bits (>= 0)
    unsigned int hi_ticket;
    unsigned int pad[61];
};
static_assert(sizeof(WsSlot) % 256 == 0, "slot alignment");

// Per-stream workspace of the generic fork-join nests: chunk partials (one
// per chunk), group partials (one per 32 chunks of a segment) and arrival
// tickets, which are zero between calls.  A chunk plan keeps segments x
// chunks <= kNestCap; with more than 32 chunks per segment there are fewer
// than kNestCap / 32 segments, which bounds the group arrays.
constexpr int kNestCap = 65536;
constexpr int kNestTick = kNestCap / 2;
constexpr int kNestCap2 = 4096;
constexpr int kNestTick2 = 2048;
struct NestWs {
    float4 part[kNestCap];
    float4 part2[kNestCap2];
    unsigned int tick[kNestTick];
    unsigned int tick2[kNestTick2];
};
// A run of Jacobi sweeps stores one partial maximum per CTA and sweep in
// NestWs::part (as floats) before a residual kernel folds them.
constexpr int64_t kStPartCap = 4 * (int64_t)kNestCap;

// ---------------------------------------------------------------- plans
struct MrPlan {
    int64_t n;
    int vecs_per_thread;   // float4 vectors per lane, multiple of kMrUnroll
    int64_t tile_elems;    // 32 * 4 * vecs_per_thread
    int64_t tiles;
};

// vecs_pref: preferred float4 vectors per lane (the tuned value for n's size
// class); raised when n would otherwise need more than kMrMaxTiles tiles.
__host__ __device__ inline MrPlan mr_plan(int64_t n, int vecs_pref = kMrMinVecs) {
    MrPlan p;
    p.n = n;
    const int64_t per_vec_row = (int64_t)kWarp * 4;
    int64_t need = (n + per_vec_row * kMrMaxTiles - 1) / (per_vec_row * kMrMaxTiles);
    if (need < vecs_pref) need = vecs_pref;
    int64_t v = need < kMrMinVecs ? kMrMinVecs : need;
    v = (v + kMrUnroll - 1) / kMrUnroll * kMrUnroll;
    p.vecs_per_thread = (int)v;
    p.tile_elems = per_vec_row * v;
    p.tiles = (n + p.tile_elems - 1) / p.tile_elems;
    return p;
}

// ---------------------------------------------------------------- loads
__device__ __forceinline__ float4 ld_stream4(const float4 *p) {
    float4 v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ uint4 ld_stream_u4(const uint4 *p) {
    uint4 v;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "l"(p));
    return v;
}
__device__ __forceinline__ void st_stream4(float4 *p, float4 v) {
    asm volatile("st.global.cs.v4.f32 [%0], {%1,%2,%3,%4};"
                 :: "l"(p), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w) : "memory");
}
// Store of a tile partial, which the final combine reads back after the
// streams of the same launch have passed through L2: written with L2
// evict-last priority so those streams do not push it out to DRAM.
__device__ __forceinline__ void st_keep2(float2 *p, float2 v) {
    uint64_t pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("st.global.L2::cache_hint.v2.f32 [%0], {%1,%2}, %3;"
                 :: "l"(p), "f"(v.x), "f"(v.y), "l"(pol) : "memory");
}

// ---------------------------------------------------------------- trees
// Sums are carried as unevaluated pairs hi + lo of fp32 numbers (the
// "double-float" representation): TwoSum (Knuth) yields the exact rounding
// error of an fp32 addition, so a pair holds about 48 significant bits while
// using only the fp32 pipes (B300's fp64 rate is a small fraction of its
// fp32 rate).  TwoSum's error term is exact whichever operand comes first,
// so ff_add is commutative bit for bit and a butterfly leaves the same value
// in every lane: the combination order, and hence the result, is fixed.
struct ff {
    float hi, lo;
};

__device__ __forceinline__ ff two_sum(float a, float b) {
    const float s = a + b;
    const float bb = s - a;
    const float e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
// Renormalise (s, e) with |e| small against s: hi = fl(s + e), lo = the rest.
// A running value s that is not finite (an infinite operand, an fp32
// overflow, a NaN) is kept as it is with lo = 0: its error term is inf - inf
// = NaN and must not reach hi, so that a sum meeting +inf stays +inf, as a
// left fold gives (Sec. 3.3).  Applied to a pair it already normalised, it
// returns the pair unchanged.
__device__ __forceinline__ ff ff_settle(float s, float e) {
    const float h = s + e;
    const bool fin = fabsf(s) <= 3.402823466e38f;   // false for +-inf and NaN
    return {fin ? h : s, fin ? e - (h - s) : 0.0f};
}
__device__ __forceinline__ ff ff_add(ff a, ff b) {
    const ff s = two_sum(a.hi, b.hi);
    return ff_settle(s.hi, s.lo + (a.lo + b.lo));
}
__device__ __forceinline__ ff ff_add_f(ff a, float b) {
    const ff s = two_sum(a.hi, b);
    return ff_settle(s.hi, s.lo + a.lo);
}
// Cascaded summation (Ogita, Rump and Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 2005, Algorithm Sum2): p takes the plain
// fp32 sum and c collects the exact TwoSum errors, without renormalising
// each step; ff_settle renormalises the pair once per group of values.
__device__ __forceinline__ void sum2_step(float &p, float &c, float v) {
    const ff s = two_sum(p, v);
    p = s.hi;
    c += s.lo;
}
__device__ __forceinline__ ff ff_shfl_xor(ff v, int off) {
    return {__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off)};
}
__device__ __forceinline__ ff warp_sum(ff v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = ff_add(v, ff_shfl_xor(v, off));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// The exact value hi + lo of a pair (fits a double: the two parts span at
// most 48 bits).
__device__ __forceinline__ double ff_to_double(ff v) { return (double)v.hi + (double)v.lo; }

// ---------------------------------------------------------------- map->reduce
// Sum of out[e] over the elements of tile `tile` owned by this thread, in the
// fixed order (vector u ascending, then lane j = 0..3 within the vector),
// storing out[e] = fmaf(a, x[e], y[e]) when out != nullptr.  The values of
// each group of kMrUnroll vectors (16 elements) fold by Sum2 steps into the
// running pair, which ff_settle renormalises after the group (and after a
// ragged tile's last element).  The vector path (aligned, full tile) and the
// element path produce the same sequence of operations.
// GROUPS (2 or 3): groups of kMrUnroll vectors per operand in flight on the
// aligned full-tile path.  The fold order does not depend on it, so the
// standalone kernel (3 groups, 120 registers) and the batched kernel (2
// groups, inside its 128-register budget) give the same bits.
//
// PF > 0 (whole-warp calls, nthreads == 32): each load of a group also
// prefetches into L2 the group PF groups further on, lanes 0..15 one line
// each of its 4 vectors x 512 bytes per operand, so that later groups' loads
// find their lines in L2.  Vector u of the next tile is vector V + u of this
// one (tiles are consecutive), so pf_vecs = 2V lets the last groups prefetch
// the next tile's first ones; pf_vecs = V (the default) stays in the tile.
// A prefetch changes no result.
template <int GROUPS = 2, int PF = 0>
__device__ __forceinline__ ff mr_thread_partial(const float *__restrict__ x,
                                                   const float *__restrict__ y,
                                                   float *__restrict__ out, float a,
                                                   const MrPlan &p, int64_t tile,
                                                   bool aligned, int t, int nthreads, int pf_vecs = 0) {
    static_assert(GROUPS == 2 || GROUPS == 3, "two or three load groups");
    const int64_t base = tile * p.tile_elems;
    ff acc = {0.0f, 0.0f};
    const bool full = base + p.tile_elems <= p.n;
    if (full && aligned) {
        // GROUPS groups of kMrUnroll vectors per operand in flight: the loads
        // of groups g + 1 .. g + GROUPS - 1 are issued before group g is
        // computed.
        const float4 *x4 = reinterpret_cast<const float4 *>(x + base);
        const float4 *y4 = reinterpret_cast<const float4 *>(y + base);
        float4 *o4 = reinterpret_cast<float4 *>(out + base);
        float4 xa[kMrUnroll], ya[kMrUnroll], xb[kMrUnroll], yb[kMrUnroll];
        auto load = [&](float4 *xv, float4 *yv, int u0) {
            if constexpr (PF > 0) {
                const int up = u0 + PF * kMrUnroll + (t >> 2);
                if (t < 4 * kMrUnroll && up < (pf_vecs > 0 ? pf_vecs : p.vecs_per_thread)) {
                    const int64_t vp = (int64_t)up * kWarp + (t & 3) * 8;
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(x4 + vp));
                    asm volatile("prefetch.global.L2 [%0];" ::"l"(y4 + vp));
                }
            }
#pragma unroll
            for (int k = 0; k < kMrUnroll; ++k) {
                const int64_t vi = (int64_t)(u0 + k) * nthreads + t;
                xv[k] = ld_stream4(x4 + vi);
                yv[k] = ld_stream4(y4 + vi);
            }
        };
        auto consume = [&](const float4 *xv, const float4 *yv, int u0) {
            float sp = acc.hi, sc = acc.lo;
#pragma unroll
            for (int k = 0; k < kMrUnroll; ++k) {
                float4 o;
                o.x = fmaf(a, xv[k].x, yv[k].x);
                o.y = fmaf(a, xv[k].y, yv[k].y);
                o.z = fmaf(a, xv[k].z, yv[k].z);
                o.w = fmaf(a, xv[k].w, yv[k].w);
                if (out) st_stream4(o4 + (int64_t)(u0 + k) * nthreads + t, o);
                sum2_step(sp, sc, o.x);
                sum2_step(sp, sc, o.y);
                sum2_step(sp, sc, o.z);
                sum2_step(sp, sc, o.w);
            }
            acc = ff_settle(sp, sc);
        };
        const int V = p.vecs_per_thread;
        constexpr int U = kMrUnroll;
        if constexpr (GROUPS == 2) {
            load(xa, ya, 0);
            for (int u0 = 0; u0 < V; u0 += 2 * U) {
                if (u0 + U < V) load(xb, yb, u0 + U);
                consume(xa, ya, u0);
                if (u0 + U >= V) break;
                if (u0 + 2 * U < V) load(xa, ya, u0 + 2 * U);
                consume(xb, yb, u0 + U);
            }
        } else {
            float4 xc[kMrUnroll], yc[kMrUnroll];
            load(xa, ya, 0);
            if (U < V) load(xb, yb, U);
            for (int u0 = 0; u0 < V; u0 += 3 * U) {
                if (u0 + 2 * U < V) load(xc, yc, u0 + 2 * U);
                consume(xa, ya, u0);
                if (u0 + U >= V) break;
                if (u0 + 3 * U < V) load(xa, ya, u0 + 3 * U);
                consume(xb, yb, u0 + U);
                if (u0 + 2 * U >= V) break;
                if (u0 + 4 * U < V) load(xb, yb, u0 + 4 * U);
                consume(xc, yc, u0 + 2 * U);
            }
        }
    } else {
        float sp = 0.0f, sc = 0.0f;
        for (int u = 0; u < p.vecs_per_thread; ++u) {
            const int64_t e0 = base + ((int64_t)u * nthreads + t) * 4;
            if (e0 >= p.n) break;   // later vectors of this thread are past n too
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int64_t e = e0 + j;
                if (e < p.n) {
                    const float o = fmaf(a, __ldg(x + e), __ldg(y + e));
                    if (out) out[e] = o;
                    sum2_step(sp, sc, o);
                }
            }
            if (u % kMrUnroll == kMrUnroll - 1) {
                acc = ff_settle(sp, sc);
                sp = acc.hi;
                sc = acc.lo;
            }
        }
        acc = ff_settle(sp, sc);
    }
    return acc;
}

// Partial of one map->reduce tile, computed by one whole warp (lane = its
// lane index); the same value in every lane.
template <int GROUPS = 2, int PF = 0>
__device__ __forceinline__ ff mr_tile(const float *__restrict__ x, const float *__restrict__ y,
                                      float *__restrict__ out, float a, const MrPlan &p, int64_t tile,
                                      bool aligned, int lane, int pf_vecs = 0) {
    return warp_sum(mr_thread_partial<GROUPS, PF>(x, y, out, a, p, tile, aligned, lane, kWarp, pf_vecs));
}

// Final combine of `tiles` tile partials in one fixed order, the same
// whether one warp or one CTA of 256 threads evaluates it.  There are 256
// virtual lanes; virtual lane v folds partials v, v + 256, v + 512, ... in
// order.  The 256 values are then combined by a butterfly whose levels pair
// lanes at distance 128, 64 and 32, then 16, 8, 4, 2 and 1 (a warp
// butterfly).  ff_add is commutative bit for bit, so both lanes of a pair get
// the same value, and the result is in every lane.
constexpr int kMrFoldLanes = 256;

// One warp: lane l plays virtual lanes l + 32 w, w = 0..7, as eight
// independent chains; the loads of two blocks of 256 partials (16 per lane)
// are issued before they are folded.
__device__ __forceinline__ ff mr_final(const float2 *partials, int64_t tiles, int lane) {
    ff acc[8];
#pragma unroll
    for (int w = 0; w < 8; ++w) acc[w] = ff{0.0f, 0.0f};
    for (int64_t b0 = 0; b0 < tiles; b0 += 2 * kMrFoldLanes) {
        float2 q[2][8];
#pragma unroll
        for (int bb = 0; bb < 2; ++bb)
#pragma unroll
            for (int w = 0; w < 8; ++w) {
                const int64_t i = b0 + bb * kMrFoldLanes + 32 * w + lane;
                q[bb][w] = i < tiles ? __ldcg(partials + i) : make_float2(0.0f, 0.0f);
            }
#pragma unroll
        for (int bb = 0; bb < 2; ++bb)
#pragma unroll
            for (int w = 0; w < 8; ++w)
                if (b0 + bb * kMrFoldLanes + 32 * w + lane < tiles) acc[w] = ff_add(acc[w], ff{q[bb][w].x, q[bb][w].y});
    }
#pragma unroll
    for (int d = 4; d >= 1; d >>= 1) {   // virtual distances 128, 64, 32
        ff t[8];
#pragma unroll
        for (int w = 0; w < 8; ++w) t[w] = ff_add(acc[w], acc[w ^ d]);
#pragma unroll
        for (int w = 0; w < 8; ++w) acc[w] = t[w];
    }
    return warp_sum(acc[0]);
}

// One CTA of kMrFoldLanes threads: thread v is virtual lane v (all its
// partials' loads in flight at once for up to 4096 tiles); red: shared
// scratch of kMrFoldLanes pairs.  Call from every thread of the CTA.
__device__ __forceinline__ ff mr_final_cta(const float2 *partials, int64_t tiles, ff *red) {
    const int v = threadIdx.x;
    ff acc = {0.0f, 0.0f};
    for (int64_t i0 = v; i0 < tiles; i0 += (int64_t)kMrFoldLanes * 16) {
        float2 q[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const int64_t i = i0 + (int64_t)k * kMrFoldLanes;
            q[k] = i < tiles ? __ldcg(partials + i) : make_float2(0.0f, 0.0f);
        }
#pragma unroll
        for (int k = 0; k < 16; ++k)
            if (i0 + (int64_t)k * kMrFoldLanes < tiles) acc = ff_add(acc, ff{q[k].x, q[k].y});
    }
#pragma unroll
    for (int d = 128; d >= 32; d >>= 1) {
        red[v] = acc;
        __syncthreads();
        acc = ff_add(acc, red[v ^ d]);
        __syncthreads();
    }
    return warp_sum(acc);
}

// One warp-tile of a map->reduce instance, end to end: tile partial, arrival
// ticket, and the final combine when this warp is the last to arrive.
__device__ __forceinline__ void mr_warp_item(const float *__restrict__ x, const float *__restrict__ y,
                                             float *__restrict__ out, float a, const MrPlan &p, int64_t tile,
                                             bool aligned, float2 *partials, unsigned int *ticket,
                                             float *d_sum, double *d_sum64) {
    const int lane = threadIdx.x & 31;
    const ff part = mr_tile(x, y, out, a, p, tile, aligned, lane);
    unsigned int prev = 0u;
    if (lane == 0) {
        st_keep2(partials + tile, make_float2(part.hi, part.lo));
        __threadfence();
        prev = atomicAdd(ticket, 1u);
    }
    prev = __shfl_sync(0xffffffffu, prev, 0);
    if (prev != (unsigned int)(p.tiles - 1)) return;
    __threadfence();
    const ff sf = mr_final(partials, p.tiles, lane);
    if (lane == 0) {
        const double s = ff_to_double(sf);
        *d_sum = (float)s;
        if (d_sum64) *d_sum64 = s;
        *ticket = 0u;
    }
}

// ---------------------------------------------------------------- stencil
__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Grid loads.  A launch that only reads its source grid loads it through the
// read-only path (__ldg); a launch that runs several sweeps writes the grids
// it later reads, so it loads through L2 only (CG: ld.global.cg, coherent
// across SMs).  The values are the same either way.
template <bool CG, typename T>
__device__ __forceinline__ T grid_ld(const T *p) {
    if constexpr (CG) return __ldcg(p);
    else return __ldg(p);
}

__device__ __forceinline__ float jacobi_point(float n, float s, float w, float e) {
    const float ns = n + s;
    const float we = w + e;
    return 0.25f * (ns + we);
}

// One warp updates a block of R rows [r_begin, r_begin + R) x 128 columns
// [c_begin, c_begin + 128) (vector path: nx % 4 == 0 and 16-byte aligned
// rows; each lane owns 4 consecutive columns).  All R + 2 input rows and the
// two halo columns are loaded before any arithmetic, so a warp has its whole
// block in flight at once; vertical neighbours come from registers and
// horizontal ones from the neighbouring lanes.  Rows past ny are clamped on
// load and not stored.  Returns the lane's max |u' - u|.
template <int R, bool CG = false>
__device__ __forceinline__ float stencil_block_vec(const float *__restrict__ src, float *__restrict__ dst,
                                                   int nx, int ny, int c_begin, int r_begin) {
    const int lane = threadIdx.x & 31;
    const int c0 = c_begin + lane * 4;
    const bool valid = c0 < nx;
    const int cl = valid ? c0 : 0;   // keep inactive lanes' loads in bounds
    float4 rows[R + 2];
#pragma unroll
    for (int k = 0; k < R + 2; ++k) {
        const int r = clampi(r_begin - 1 + k, 0, ny - 1);
        rows[k] = grid_ld<CG>(reinterpret_cast<const float4 *>(src + (size_t)r * nx + cl));
    }
    // halo columns: lane 0 needs column c0 - 1, lane 31 column c0 + 4
    const bool need_left = (lane == 0) && valid && c0 > 0;
    const bool need_right = (lane == 31) && (c0 + 4 < nx);
    const int hc = need_left ? c0 - 1 : (need_right ? c0 + 4 : 0);
    float halo[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int r = min(r_begin + k, ny - 1);
        halo[k] = (need_left || need_right) ? grid_ld<CG>(src + (size_t)r * nx + hc) : 0.0f;
    }
    float m = 0.0f;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const float4 up = rows[k], cur = rows[k + 1], dn = rows[k + 2];
        float left = __shfl_up_sync(0xffffffffu, cur.w, 1);
        float right = __shfl_down_sync(0xffffffffu, cur.x, 1);
        if (lane == 0) left = need_left ? halo[k] : cur.x;
        if (c0 + 4 >= nx) right = cur.w;
        else if (lane == 31) right = halo[k];
        float4 o;
        o.x = jacobi_point(up.x, dn.x, left, cur.y);
        o.y = jacobi_point(up.y, dn.y, cur.x, cur.z);
        o.z = jacobi_point(up.z, dn.z, cur.y, cur.w);
        o.w = jacobi_point(up.w, dn.w, cur.z, right);
        const int r = r_begin + k;
        if (valid && r < ny) {
            *reinterpret_cast<float4 *>(dst + (size_t)r * nx + c0) = o;
            m = fmaxf(m, fmaxf(fmaxf(fabsf(o.x - cur.x), fabsf(o.y - cur.y)),
                               fmaxf(fabsf(o.z - cur.z), fabsf(o.w - cur.w))));
        }
    }
    return m;
}

// Element path for any nx and alignment: each lane owns 4 consecutive
// columns read with 4 scalar loads per row (the warp still covers 128
// columns and keeps as many bytes in flight as the vector path; L1 serves
// the neighbouring words of each sector).  Every column index is clamped to
// [0, nx-1] when loading, which makes the clamp-to-edge rule automatic:
// past the last column a lane just re-reads column nx-1.  Same arithmetic per
// point as the vector path.
template <int R, bool CG = false>
__device__ __forceinline__ float stencil_block_scalar(const float *__restrict__ src, float *__restrict__ dst,
                                                      int nx, int ny, int c_begin, int r_begin) {
    const int lane = threadIdx.x & 31;
    const int c0 = c_begin + lane * 4;
    int cc[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) cc[j] = min(c0 + j, nx - 1);
    float rows[R + 2][4];
#pragma unroll
    for (int k = 0; k < R + 2; ++k) {
        const float *row = src + (size_t)clampi(r_begin - 1 + k, 0, ny - 1) * nx;
#pragma unroll
        for (int j = 0; j < 4; ++j) rows[k][j] = grid_ld<CG>(row + cc[j]);
    }
    const int hc = (lane == 0) ? max(c0 - 1, 0) : min(c0 + 4, nx - 1);
    float halo[R];
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const int r = min(r_begin + k, ny - 1);
        halo[k] = (lane == 0 || lane == 31) ? grid_ld<CG>(src + (size_t)r * nx + hc) : 0.0f;
    }
    float m = 0.0f;
#pragma unroll
    for (int k = 0; k < R; ++k) {
        const float *up = rows[k], *cur = rows[k + 1], *dn = rows[k + 2];
        float left = __shfl_up_sync(0xffffffffu, cur[3], 1);
        float right = __shfl_down_sync(0xffffffffu, cur[0], 1);
        if (lane == 0) left = halo[k];
        if (lane == 31) right = halo[k];
        float o[4];
        o[0] = jacobi_point(up[0], dn[0], left, cur[1]);
        o[1] = jacobi_point(up[1], dn[1], cur[0], cur[2]);
        o[2] = jacobi_point(up[2], dn[2], cur[1], cur[3]);
        o[3] = jacobi_point(up[3], dn[3], cur[2], right);
        const int r = r_begin + k;
        if (r < ny) {
            float *drow = dst + (size_t)r * nx;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (c0 + j < nx) {
                    drow[c0 + j] = o[j];
                    m = fmaxf(m, fabsf(o[j] - cur[j]));
                }
            }
        }
    }
    return m;
}

// Element path of a launch that runs several sweeps, whose grids are read
// through L2 only (grid_ld<true>): the warp still covers 128 columns, but
// lane l owns columns c_begin + l + 32 k (k = 0..3), so each load
// instruction reads 32 consecutive floats and no sector is requested twice
// (the layout of stencil_block_scalar, 4 consecutive columns per lane, has
// its 4 loads per row touch the same sectors, which L1 serves on the read-only
// path but L2 would see four times).  Horizontal neighbours come from the
// neighbouring lanes, across 32-column groups from lane 31 / lane 0 of the
// neighbouring group, and at the warp's edges from halo loads.  Every point
// has the operands it has in stencil_block_scalar (indices clamped on load),
// so the results are the same bits.
template <int R>
__device__ __forceinline__ float stencil_block_strided(const float *__restrict__ src, float *__restrict__ dst,
                                                       int nx, int ny, int c_begin, int r_begin) {
    const int lane = threadIdx.x & 31;
    int cc[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) cc[k] = min(c_begin + lane + 32 * k, nx - 1);
    float rows[R + 2][4];
#pragma unroll
    for (int kr = 0; kr < R + 2; ++kr) {
        const float *row = src + (size_t)clampi(r_begin - 1 + kr, 0, ny - 1) * nx;
#pragma unroll
        for (int k = 0; k < 4; ++k) rows[kr][k] = grid_ld<true>(row + cc[k]);
    }
    const int hc = (lane == 0) ? max(c_begin - 1, 0) : min(c_begin + 128, nx - 1);
    float halo[R];
#pragma unroll
    for (int kr = 0; kr < R; ++kr) {
        const int r = min(r_begin + kr, ny - 1);
        halo[kr] = (lane == 0 || lane == 31) ? grid_ld<true>(src + (size_t)r * nx + hc) : 0.0f;
    }
    float m = 0.0f;
#pragma unroll
    for (int kr = 0; kr < R; ++kr) {
        const float *up = rows[kr], *cur = rows[kr + 1], *dn = rows[kr + 2];
        float o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float left = __shfl_up_sync(0xffffffffu, cur[k], 1);
            float right = __shfl_down_sync(0xffffffffu, cur[k], 1);
            const float from31 = __shfl_sync(0xffffffffu, cur[k > 0 ? k - 1 : 0], 31);   // column c - 1 for lane 0
            const float from0 = __shfl_sync(0xffffffffu, cur[k < 3 ? k + 1 : 3], 0);     // column c + 1 for lane 31
            if (lane == 0) left = (k == 0) ? halo[kr] : from31;
            if (lane == 31) right = (k == 3) ? halo[kr] : from0;
            o[k] = jacobi_point(up[k], dn[k], left, right);
        }
        const int r = r_begin + kr;
        if (r < ny) {
            float *drow = dst + (size_t)r * nx;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int c = c_begin + lane + 32 * k;
                if (c < nx) {
                    drow[c] = o[k];
                    m = fmaxf(m, fabsf(o[k] - cur[k]));
                }
            }
        }
    }
    return m;
}

// ---------------------------------------------------------------- histogram
// Shared counters are laid out [bin][slot], 256 bins x 64 slots of uint32
// (64 KiB, dynamic shared memory).  A thread owns slot (lane + 32 * (warp &
// 1)): one warp-wide increment touches 32 different banks whatever the data,
// and neighbouring warps share no counter.  A bin row is 256 bytes, so the
// byte offset of bin b in a thread's slot is (b << 8) | slot_offset, with
// slot_offset < 256: one prmt builds it straight from the loaded word (byte k
// of the word into bits 8-15, the slot offset into bits 0-7), and the shared
// atomic adds the array base as an immediate.  Two instructions per byte.
constexpr int kHiSlots = 64;
constexpr int kHiSmemBytes = kHiBins * kHiSlots * 4;

__device__ __forceinline__ unsigned int hist_slot_offset() {
    return ((threadIdx.x & 31u) << 2) | (((threadIdx.x >> 5) & 1u) << 7);
}
__device__ __forceinline__ void hist_inc(unsigned int *sh, unsigned int byte_off) {
    atomicAdd(reinterpret_cast<unsigned int *>(reinterpret_cast<char *>(sh) + byte_off), 1u);
}
__device__ __forceinline__ void hist_count_word(unsigned int *sh, unsigned int slot, unsigned int w) {
    hist_inc(sh, __byte_perm(w, slot, 0x5504u));
    hist_inc(sh, __byte_perm(w, slot, 0x5514u));
    hist_inc(sh, __byte_perm(w, slot, 0x5524u));
    hist_inc(sh, __byte_perm(w, slot, 0x5534u));
}
__device__ __forceinline__ void hist_count_vec(unsigned int *sh, unsigned int slot, const uint4 &w) {
    hist_count_word(sh, slot, w.x);
    hist_count_word(sh, slot, w.y);
    hist_count_word(sh, slot, w.z);
    hist_count_word(sh, slot, w.w);
}
__device__ __forceinline__ void hist_count_byte(unsigned int *sh, unsigned int slot, unsigned int b) {
    hist_inc(sh, (b << 8) | slot);
}
// Zero the counters (all threads of the CTA; a barrier must follow).
__device__ __forceinline__ void hist_zero(unsigned int *sh) {
    uint4 *s4 = reinterpret_cast<uint4 *>(sh);
    for (int i = threadIdx.x; i < kHiSmemBytes / 16; i += blockDim.x) s4[i] = make_uint4(0, 0, 0, 0);
}
// Fold the 64 slots of each bin (rotated start: conflict-free) and add the
// non-zero totals into bins_out with integer atomics (exact, any order).
// Called after a barrier; returns whether this thread issued an atomic.
__device__ __forceinline__ bool hist_merge(const unsigned int *sh, unsigned int *bins_out) {
    bool wrote = false;
    for (int b = threadIdx.x; b < kHiBins; b += blockDim.x) {
        unsigned int c = 0u;
#pragma unroll 8
        for (int k = 0; k < kHiSlots; ++k) c += sh[b * kHiSlots + ((k + b) & (kHiSlots - 1))];
        if (c) {
            atomicAdd(bins_out + b, c);
            wrote = true;
        }
    }
    return wrote;
}

// Count the 16-byte vectors v4[first], v4[first + stride], ... below nvec into
// the shared counters, keeping the next D vectors' loads in flight while the
// current D are counted.  The standalone histogram runs wide CTAs at several
// per SM and keeps D = 2; the batch counts a chunk with one 256-thread CTA
// and needs a deeper pipeline for the same bytes in flight per SM.
template <int D = 2>
__device__ __forceinline__ void hist_count_strided(unsigned int *sh, unsigned int slot,
                                                   const uint4 *__restrict__ v4, int64_t first, int64_t stride,
                                                   int64_t nvec) {
    int64_t i = first;
    uint4 a[D];
#pragma unroll
    for (int d = 0; d < D; ++d) {
        a[d] = make_uint4(0, 0, 0, 0);
        if (i + d * stride < nvec) a[d] = ld_stream_u4(v4 + i + d * stride);
    }
    while (i < nvec) {
        const int64_t j = i + D * stride;
        uint4 b[D];
#pragma unroll
        for (int d = 0; d < D; ++d) {
            b[d] = make_uint4(0, 0, 0, 0);
            if (j + d * stride < nvec) b[d] = ld_stream_u4(v4 + j + d * stride);
        }
#pragma unroll
        for (int d = 0; d < D; ++d)
            if (d == 0 || i + d * stride < nvec) hist_count_vec(sh, slot, a[d]);
#pragma unroll
        for (int d = 0; d < D; ++d) a[d] = b[d];
        i = j;
    }
}

// ---------------------------------------------------------------- host side
}  // namespace hx

extern "C" void hx_batch_free(hx_batch *batch);

struct hx_ctx {
    int device = 0;
    int num_sms = 0;
    size_t hbm_budget = 0;
    hx::WsSlot *ws = nullptr;   // HX_MAX_STREAMS slots
    hx::NestWs *nest_ws = nullptr;  // HX_MAX_STREAMS slots, same index as ws
    hx_stream_t slot_stream[HX_MAX_STREAMS] = {};
    bool slot_used[HX_MAX_STREAMS] = {};
    std::mutex slot_mu;                  // a server's thread and the caller's may both take slots
    hx_tune_table tune = {};             // per-size-class choices (see hx.h)
    int hist_ctas_per_sm[3] = {1, 1, 1}; // resident CTAs per SM for widths 256, 512, 1024
    int batch_ctas_per_sm[2][2] = {{1, 1}, {1, 1}};   // batched kernel [one sweep / several][without / with histogram counters]
    // test hook: after `inject_after` more launching calls, `inject_count`
    // calls fail before launching
    mutable std::mutex inject_mu;
    mutable int inject_after = 0;
    mutable int inject_count = 0;
    // hx_batch_submit bookkeeping: ticket -> (plan, completion event)
    uint64_t next_ticket = 1;
    std::map<uint64_t, std::pair<hx_batch *, cudaEvent_t>> pending;
};

namespace hx {
hx_status fail(hx_status st, const std::string &msg);
hx_status cuda_fail(cudaError_t e, const char *what);
hx_status slot_for(hx_ctx *ctx, hx_stream_t stream, WsSlot **slot);
// Frees the slot of a stream that will not be used again (its work has
// completed; a server calls this for its own stream when it is destroyed).
void release_slot(hx_ctx *ctx, hx_stream_t stream);
hx_status histogram_setup(hx_ctx *ctx);
// Size class of a problem size: floor(log2(n)) clamped to the table, 0 for n <= 1.
inline int size_class(int64_t n) {
    int c = 0;
    while (c + 1 < HX_TUNE_CLASSES && ((int64_t)1 << (c + 1)) <= n) ++c;
    return c;
}
hx_status batch_setup(hx_ctx *ctx);
// Readers of each kernel file's check record (see HX_CHECKS_READER).
hx_status checks_map_reduce(int32_t *code, int64_t *a, int64_t *b);
hx_status checks_stencil(int32_t *code, int64_t *a, int64_t *b);
hx_status checks_histogram(int32_t *code, int64_t *a, int64_t *b);
hx_status checks_batch(int32_t *code, int64_t *a, int64_t *b);
hx_status checks_srad(int32_t *code, int64_t *a, int64_t *b);
hx_status checks_noalloc(int32_t *code, int64_t *a, int64_t *b);
hx_status checks_nest(int32_t *code, int64_t *a, int64_t *b);   // every loaded generated nest kernel

// Consumes one injected launch failure (hx_debug_inject_launch_failures):
// true when the calling entry point must fail with HX_ERR_CUDA before it
// launches anything.
inline bool take_injected_failure(const hx_ctx *ctx) {
    std::lock_guard<std::mutex> lk(ctx->inject_mu);
    if (ctx->inject_count <= 0) return false;
    if (ctx->inject_after > 0) {
        --ctx->inject_after;
        return false;
    }
    --ctx->inject_count;
    return true;
}

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
            changed = cudaSetDevice(dev) == cudaSuccess;
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};
}  // namespace hx
