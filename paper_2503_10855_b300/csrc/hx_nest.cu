// hx_nest.cu -- generic fork-join nests: a fork of one to three factors whose
// body is a small straight-line map program, feeding a monoid reduce over the
// innermost fork dimensions (Hercules paper, Sec. 3.3 fork-joins and reduces,
// Sec. 3.4 MonoidReduce).
//
// Like the Hercules GPU backend (Sec. 4.4), the library turns the nest into a
// CUDA kernel: the map program becomes one fused expression, pasted into the
// hand-written kernel template below together with the nest's shape
// (dimension split, monoid, reduction schedule, addressing mode of every
// input), and the result is compiled for sm_103a with NVRTC.  Sizes, strides,
// constants and pointers are launch arguments, so one compiled kernel serves
// every nest of the same shape; compiled kernels are cached process-wide by
// their source text.
//
// Reduction schedules (Sec. 5.2: the reduction-tree macro -- chunk,
// monoid-reassociate, fork-fission -- and the lowering of reductions to warp
// primitives):
//   HX_TREE_WARP   a segment is cut into chunks; a group of G lanes (G = 32,
//                  fewer for short segments) takes a chunk in "slots" of 4
//                  consecutive elements, lane l taking slots l, l+G, ...; each
//                  lane folds its elements in increasing order, the group
//                  combines lanes with a shuffle butterfly.  Chunk partials
//                  form a 3-level tree (chunks -> groups of 32 chunks ->
//                  segment), each level finished by the last arrival (ticket).
//   HX_TREE_CHUNK  the two-level tree of the reduction-tree macro: one thread
//                  folds each contiguous chunk sequentially, the last thread
//                  to finish folds the chunk partials sequentially.
//   HX_TREE_SEQ    the untransformed loop: one thread folds a whole segment.
// Sums and products accumulate in float-float (hi, lo) pairs; extrema are
// exact.  The combination order depends only on the nest's sizes, schedule,
// chunk, tuning table and the number of warps the device holds at once --
// not on pointer alignment (the float4 and scalar load paths assign the same
// elements to the same lanes) -- so results are bit-identical from run to run.
#include <nvrtc.h>

#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <unordered_map>

#include "hx_internal.cuh"

namespace {

constexpr int kNestBlock = 256;

// ---------------------------------------------------------------- device template
// Everything the generated kernels share.  MONOID (-1 = map only), TREE, G, U,
// VEC and the HAS_* flags are #defined by the generated header in front of
// it; the generated part also supplies struct Seg, seg_setup(), struct Buf,
// load_group(), map_elem() and map_at().
// L2 prefetch in the warp tree (no registers held): a group narrower than a
// warp prefetches the segment after the one it has in flight.  Measured on
// B300, max over 2^24 rows of 8: 0.90 -> 0.97 of HBM.  Whole-warp groups do
// not prefetch: two load groups beyond each load took a permuted 3-D reduce
// from 0.94 to 0.82 and a 2^28 sum from 1.01 to 0.99.
constexpr int kNestPrefetch = 1;

const char *kPrelude = R"CUDA(
typedef long long i64;
typedef unsigned long long u64;
// Range checks of the debug build (HX_DEBUG_CHECKS): the first failure's
// code and values in hx_check_rec, the access skipped, nothing trapped.
#ifdef HX_DEBUG_CHECKS
extern "C" __device__ unsigned long long hx_check_rec[3];
__device__ unsigned long long hx_check_rec[3];
__device__ __forceinline__ bool check_ok(bool ok, int code, long long a, long long b) {
    if (ok) return true;
    if (atomicCAS(&hx_check_rec[0], 0ull, (unsigned long long)code) == 0ull) {
        hx_check_rec[1] = (unsigned long long)a;
        hx_check_rec[2] = (unsigned long long)b;
    }
    return false;
}
#define HX_CHECK(cond, code, a, b) check_ok((cond), (code), (long long)(a), (long long)(b))
#else
#define HX_CHECK(cond, code, a, b) true
#endif
struct NestParams {
    const float *in[4];
    i64 st[4][3];
    i64 lin[4];         // stride of an input addressed linearly inside a segment
    float c[8];
    i64 dims[3];
    unsigned dm[3];     // n / dims[d] == (n * dm[d]) >> ds[d] for 0 <= n < 2^31
    unsigned ds[3];
    i64 outer, inner, chunk, nchunks, ngroups, n_items;
    float *out;
    float *res;
    double *res64;
    i64 *res_idx;
    float4 *part;       // one partial per chunk
    float4 *part2;      // one partial per group of 32 chunks
    unsigned *tick;     // chunk arrivals per (segment, group)
    unsigned *tick2;    // group arrivals per segment
};

// Quotient by a fork factor, by multiplication (Granlund and Montgomery,
// "Division by invariant integers using multiplication", 1994, Thm. 4.2 with
// N = 31): exact for 0 <= n < 2^31.
__device__ __forceinline__ unsigned hx_div(const NestParams &p, int d, unsigned n) {
    return (unsigned)(((u64)n * p.dm[d]) >> p.ds[d]);
}

__device__ __forceinline__ float hx_minnum(float a, float b) {
    return isnan(a) ? b : (isnan(b) ? a : (b < a ? b : a));
}
__device__ __forceinline__ float hx_maxnum(float a, float b) {
    return isnan(a) ? b : (isnan(b) ? a : (b > a ? b : a));
}
__device__ __forceinline__ void prefetch_l2(const float *a) { asm volatile("prefetch.global.L2 [%0];" ::"l"(a)); }
__device__ __forceinline__ float hx_comp(const float4 &v, int q) {
    return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}
#define HX_NEG_INF __int_as_float(0xff800000)
#define HX_POS_INF __int_as_float(0x7f800000)

#if MONOID == 0 || MONOID == 3
struct Acc { float hi, lo; };
#elif MONOID == 1 || MONOID == 2
struct Acc { float v; };
#elif MONOID >= 4
struct Acc { float v; i64 i; };
#else
struct Acc { int unused; };
#endif

__device__ __forceinline__ Acc acc_init() {
#if MONOID == 0
    return Acc{0.0f, 0.0f};
#elif MONOID == 3
    return Acc{1.0f, 0.0f};
#elif MONOID == 1
    return Acc{HX_NEG_INF};
#elif MONOID == 2
    return Acc{HX_POS_INF};
#elif MONOID == 4
    return Acc{HX_NEG_INF, -1};
#elif MONOID == 5
    return Acc{HX_POS_INF, -1};
#else
    return Acc{0};
#endif
}

// A sum or product whose running value is not finite (an infinite operand,
// an fp32 overflow, a NaN) keeps that value with lo = 0: its error term would
// be inf - inf = NaN, and a left fold that meets +inf gives +inf.
__device__ __forceinline__ bool hx_finite(float v) { return fabsf(v) <= 3.402823466e38f; }
#if MONOID == 0 || MONOID == 3
__device__ __forceinline__ Acc acc_pair(float s, float e) {
    const float h = s + e;
    return hx_finite(s) ? Acc{h, e - (h - s)} : Acc{s, 0.0f};
}
#endif

// Fold one value of thread r into a running accumulator (thread-ID order).
__device__ __forceinline__ void acc_fold(Acc &a, float v, i64 r) {
#if MONOID == 0
    float s = a.hi + v, bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (v - bb);     // exact error of a.hi + v
    a = acc_pair(s, e + a.lo);
#elif MONOID == 3
    float pr = a.hi * v;
    float e = fmaf(a.hi, v, -pr);               // exact error of a.hi * v
    a = acc_pair(pr, fmaf(a.lo, v, e));
#elif MONOID == 1 && G == 32
    // The running value is never NaN (it starts at -inf), and fmaxf skips a
    // NaN operand and ranks +0 above -0 (checked on B300; the parity tests
    // pin both): the monoid's rules in one instruction.  Measured: max |x|
    // over 2^28 0.90 -> 0.96 of HBM.  Groups narrower than a warp keep the
    // explicit comparison (the same bits), which measured 2 % faster there.
    a.v = fmaxf(a.v, v);
#elif MONOID == 2 && G == 32
    a.v = fminf(a.v, v);   // likewise: NaN skipped, -0 below +0
#elif MONOID == 1
    if (v > a.v || (v == 0.0f && a.v == 0.0f && signbit(a.v) && !signbit(v))) a.v = v;
#elif MONOID == 2
    if (v < a.v || (v == 0.0f && a.v == 0.0f && !signbit(a.v) && signbit(v))) a.v = v;
#elif MONOID == 4
    if (!isnan(v) && (a.i < 0 || v > a.v)) { a.v = v; a.i = r; }
#elif MONOID == 5
    if (!isnan(v) && (a.i < 0 || v < a.v)) { a.v = v; a.i = r; }
#endif
}

// Fold for the few values of one load group (warp tree).  For sums this is a
// step of Ogita, Rump and Oishi's cascaded summation (Sum2, 2005): hi takes
// the plain fp32 sum and lo collects the exact TwoSum errors, without the
// renormalisation of every step; acc_settle renormalises the pair once per
// group, so lo never gathers more than 4 U errors.  Other monoids fold as
// acc_fold does.
__device__ __forceinline__ void acc_fold_run(Acc &a, float v, i64 r) {
#if MONOID == 0
    float s = a.hi + v, bb = s - a.hi;
    a.lo += (a.hi - (s - bb)) + (v - bb);
    a.hi = s;
#else
    acc_fold(a, v, r);
#endif
}
__device__ __forceinline__ void acc_settle(Acc &a) {
#if MONOID == 0
    float s = a.hi + a.lo, bb = s - a.hi;
    const bool fin = hx_finite(a.hi);
    a.lo = fin ? (a.hi - (s - bb)) + (a.lo - bb) : 0.0f;     // exact: hi + lo unchanged
    a.hi = fin ? s : a.hi;
#endif
}

#if MONOID >= 0
// Combine two partial results.  Commutative bit for bit (the exact TwoSum /
// TwoProd error terms do not depend on operand order; extrema break ties by
// the smaller thread index), so both lanes of a butterfly pair agree.
__device__ __forceinline__ Acc acc_combine(Acc a, Acc b) {
#if MONOID == 0
    float s = a.hi + b.hi, bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    return acc_pair(s, e + (a.lo + b.lo));
#elif MONOID == 3
    float pr = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -pr);
    return acc_pair(pr, e + (a.hi * b.lo + a.lo * b.hi));
#elif MONOID == 1 && G == 32
    a.v = fmaxf(a.v, b.v);
    return a;
#elif MONOID == 2 && G == 32
    a.v = fminf(a.v, b.v);
    return a;
#elif MONOID == 1
    return (b.v > a.v || (b.v == 0.0f && a.v == 0.0f && signbit(a.v) && !signbit(b.v))) ? b : a;
#elif MONOID == 2
    return (b.v < a.v || (b.v == 0.0f && a.v == 0.0f && !signbit(a.v) && signbit(b.v))) ? b : a;
#elif MONOID == 4
    if (b.i < 0) return a;
    if (a.i < 0) return b;
    return (b.v > a.v || (b.v == a.v && b.i < a.i)) ? b : a;
#else
    if (b.i < 0) return a;
    if (a.i < 0) return b;
    return (b.v < a.v || (b.v == a.v && b.i < a.i)) ? b : a;
#endif
}

template <int W>
__device__ __forceinline__ Acc acc_shfl(unsigned mask, Acc a, int k) {
    Acc o = a;
#if MONOID == 0 || MONOID == 3
    o.hi = __shfl_xor_sync(mask, a.hi, k, W);
    o.lo = __shfl_xor_sync(mask, a.lo, k, W);
#elif MONOID == 1 || MONOID == 2
    o.v = __shfl_xor_sync(mask, a.v, k, W);
#else
    o.v = __shfl_xor_sync(mask, a.v, k, W);
    o.i = __shfl_xor_sync(mask, a.i, k, W);
#endif
    return o;
}

template <int W>
__device__ __forceinline__ Acc acc_butterfly(unsigned mask, Acc a) {
#pragma unroll
    for (int k = W / 2; k >= 1; k >>= 1) a = acc_combine(a, acc_shfl<W>(mask, a, k));
    return a;
}

union PartBits { float4 f4; struct { float a, b; i64 i; } s; };

// Partials are read back by the last arrival of their group, possibly after
// much of the launch's input has streamed through L2: stored with L2
// evict-last priority.
__device__ __forceinline__ void st_keep4(float4 *dst, float4 v) {
    unsigned long long pol;
    asm("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1,%2,%3,%4}, %5;"
                 :: "l"(dst), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w), "l"(pol) : "memory");
}

__device__ __forceinline__ void part_store(float4 *dst, Acc a) {
    PartBits u;
    u.f4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#if MONOID == 0 || MONOID == 3
    u.s.a = a.hi; u.s.b = a.lo;
#elif MONOID == 1 || MONOID == 2
    u.s.a = a.v;
#else
    u.s.a = a.v; u.s.i = a.i;
#endif
    st_keep4(dst, u.f4);
}

__device__ __forceinline__ Acc part_load(const float4 *src) {
    PartBits u;
    u.f4 = __ldcg(src);     // written by other SMs: read at L2
    Acc a;
#if MONOID == 0 || MONOID == 3
    a.hi = u.s.a; a.lo = u.s.b;
#elif MONOID == 1 || MONOID == 2
    a.v = u.s.a;
#else
    a.v = u.s.a; a.i = u.s.i;
#endif
    return a;
}

__device__ __forceinline__ void write_result(const NestParams &p, i64 s, Acc a) {
#if MONOID == 0 || MONOID == 3
    p.res[s] = a.hi + a.lo;
#if HAS_RES64
    p.res64[s] = (double)a.hi + (double)a.lo;
#endif
#else
    p.res[s] = a.v;
#if HAS_RES64
    p.res64[s] = (double)a.v;
#endif
#if MONOID >= 4
    p.res_idx[s] = a.i;
#endif
#endif
}
#endif  // MONOID >= 0
)CUDA";

// Warp-tree kernel (TREE == 0).  Double-buffered: the loads of the next U
// slots per lane are issued before the current ones are folded.
const char *kWarpBody = R"CUDA(
__device__ __forceinline__ void proc_group(const NestParams &p, const Seg &g, const Buf &b, i64 t0, Acc &acc) {
#pragma unroll
    for (int j = 0; j < U; ++j) {
        const i64 t = t0 + (i64)j * G;
        if (t < g.nslot) {
            const i64 r0 = g.r_begin + 4 * t;
            float vq[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) vq[q] = (VEC || r0 + q < g.r_end) ? map_elem(p, g, b, j, q, r0 + q) : 0.0f;
#if HAS_OUT
            float *o = p.out + g.s * p.inner + r0;
            if (VEC) {
                *(float4 *)o = make_float4(vq[0], vq[1], vq[2], vq[3]);
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (r0 + q < g.r_end) o[q] = vq[q];
            }
#endif
#if MONOID >= 0
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (VEC || r0 + q < g.r_end) acc_fold_run(acc, vq[q], r0 + q);
#endif
        }
    }
#if MONOID >= 0
    acc_settle(acc);
#endif
}

#if MONOID >= 0
// Last step of a segment in a group narrower than a warp: the group's lanes
// combine their partials, and the group's first lane writes the result.
__device__ __forceinline__ void group_result(const NestParams &p, i64 s, Acc acc, unsigned gmask, int gl) {
    acc = acc_butterfly<G>(gmask, acc);
    if (gl == 0) write_result(p, s, acc);
}
#endif

#if MONOID >= 0 && G == 32
// Reduction tree of one item once its lanes have folded their slots: the
// butterfly, then for a segment of several chunks the last-arrival levels.
__device__ __forceinline__ void item_tree(const NestParams &p, const Seg &g, i64 item, Acc acc, int lane) {
    acc = acc_butterfly<32>(0xffffffffu, acc);
    if (p.nchunks == 1) {
        if (lane == 0) write_result(p, g.s, acc);
        return;
    }
    // Level 1: the last chunk of its group of 32 folds the group's partials.
    const i64 c = item - g.s * p.nchunks;
    const i64 grp = c >> 5;
    const int gsize = (int)min((i64)32, p.nchunks - grp * 32);
    unsigned *t1 = p.tick + g.s * p.ngroups + grp;
    if (!HX_CHECK(item < HX_NEST_CAP, 11, item, HX_NEST_CAP)) return;
    if (!HX_CHECK(g.s * p.ngroups + grp < HX_NEST_TICK, 13, g.s * p.ngroups + grp, HX_NEST_TICK)) return;
    unsigned last = 0;
    if (lane == 0) {
        part_store(p.part + item, acc);
        __threadfence();
        last = atomicAdd(t1, 1u) == (unsigned)(gsize - 1) ? 1u : 0u;
    }
    if (!__shfl_sync(0xffffffffu, last, 0)) return;
    __threadfence();
    Acc t = lane < gsize ? part_load(p.part + g.s * p.nchunks + grp * 32 + lane) : acc_init();
    t = acc_butterfly<32>(0xffffffffu, t);
    if (p.ngroups == 1) {
        if (lane == 0) {
            write_result(p, g.s, t);
            *t1 = 0u;
        }
        return;
    }
    // Level 2: the last group of the segment folds the group partials.
    if (!HX_CHECK(g.s * p.ngroups + grp < HX_NEST_CAP2 && g.s < HX_NEST_TICK2, 12, g.s * p.ngroups + grp,
                  HX_NEST_CAP2)) return;
    last = 0;
    if (lane == 0) {
        *t1 = 0u;
        part_store(p.part2 + g.s * p.ngroups + grp, t);
        __threadfence();
        last = atomicAdd(p.tick2 + g.s, 1u) == (unsigned)(p.ngroups - 1) ? 1u : 0u;
    }
    if (!__shfl_sync(0xffffffffu, last, 0)) return;
    __threadfence();
    // lane l folds group partials l, l + 32, ... in order; the loads of 4 of
    // them are issued before they are folded
    Acc u = acc_init();
    const float4 *gp = p.part2 + g.s * p.ngroups;
    for (i64 q0 = lane; q0 < p.ngroups; q0 += 32 * 4) {
        Acc v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] = q0 + 32 * k < p.ngroups ? part_load(gp + q0 + 32 * k) : acc_init();
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (q0 + 32 * k < p.ngroups) u = acc_combine(u, v[k]);
    }
    u = acc_butterfly<32>(0xffffffffu, u);
    if (lane == 0) {
        write_result(p, g.s, u);
        p.tick2[g.s] = 0u;
    }
}
#endif

// Item `item` (chunk item % nchunks of segment item / nchunks).
__device__ __forceinline__ void seg_item(const NestParams &p, Seg &g, i64 item) {
    g.s = p.nchunks == 1 ? item : item / p.nchunks;
    g.r_begin = (item - g.s * p.nchunks) * p.chunk;
    g.r_end = min(p.inner, g.r_begin + p.chunk);
    g.nslot = (g.r_end - g.r_begin + 3) >> 2;
    seg_setup(p, g);
}

// Segment s as one item (the whole inner extent).
__device__ __forceinline__ void seg_whole(const NestParams &p, Seg &g, i64 s) {
    g.s = s;
    g.r_begin = 0;
    g.r_end = p.inner;
    g.nslot = (p.inner + 3) >> 2;
    seg_setup(p, g);
}

extern "C" __global__ void __launch_bounds__(256) hx_nest_kernel(const NestParams p) {
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const i64 per_cta = 256 / G;
#if G < 32
    // Groups narrower than a warp take whole segments, and G lanes x U slots
    // cover a segment's inner extent, so one load group holds a segment: the
    // loads of the group's next segment are issued before the current one is
    // folded (two segments in flight per lane).
    const i64 stride = (i64)gridDim.x * per_cta;
    i64 item = (i64)blockIdx.x * per_cta + threadIdx.x / G;
    Seg ga, gb;
    Buf ba, bb;
    if (item < p.n_items) {
        seg_whole(p, ga, item);
        load_group(p, ga, ba, gl);
    }
    while (item < p.n_items) {
        const i64 i1 = item + stride;
        if (i1 < p.n_items) {
            seg_whole(p, gb, i1);
            load_group(p, gb, bb, gl);
#if HX_NEST_PF
            if (i1 + stride < p.n_items) {   // a third segment's lines into L2
                Seg gc;
                seg_whole(p, gc, i1 + stride);
                prefetch_group(p, gc, gl);
            }
#endif
        }
        {
            Acc acc = acc_init();
            proc_group(p, ga, ba, gl, acc);
#if MONOID >= 0
            group_result(p, ga.s, acc, gmask, gl);
#endif
        }
        if (i1 >= p.n_items) break;
        const i64 i2 = i1 + stride;
        if (i2 < p.n_items) {
            seg_whole(p, ga, i2);
            load_group(p, ga, ba, gl);
#if HX_NEST_PF
            if (i2 + stride < p.n_items) {
                Seg gc;
                seg_whole(p, gc, i2 + stride);
                prefetch_group(p, gc, gl);
            }
#endif
        }
        {
            Acc acc = acc_init();
            proc_group(p, gb, bb, gl, acc);
#if MONOID >= 0
            group_result(p, gb.s, acc, gmask, gl);
#endif
        }
        item = i2;
    }
#else
    // G == 32: the whole warp shares an item (a chunk of a segment).
    for (i64 item = (i64)blockIdx.x * per_cta + threadIdx.x / G; item < p.n_items;
         item += (i64)gridDim.x * per_cta) {
        Seg g;
        seg_item(p, g, item);
        Acc acc = acc_init();
        Buf ba, bb;
        load_group(p, g, ba, gl);
        for (i64 t0 = gl; t0 < g.nslot; t0 += 2 * G * U) {
            load_group(p, g, bb, t0 + G * U);
            proc_group(p, g, ba, t0, acc);
            load_group(p, g, ba, t0 + 2 * G * U);
            proc_group(p, g, bb, t0 + G * U, acc);
        }
#if MONOID >= 0
        item_tree(p, g, item, acc, lane);
#endif
    }
#endif  // G < 32
}
)CUDA";

// One thread per item: HX_TREE_CHUNK (items = chunks of a segment) or
// HX_TREE_SEQ (items = segments).  Sequential fold in thread-ID order; the
// last chunk of a segment folds the chunk partials in chunk order.
const char *kThreadBody = R"CUDA(
extern "C" __global__ void __launch_bounds__(256) hx_nest_kernel(const NestParams p) {
    for (i64 item = (i64)blockIdx.x * 256 + threadIdx.x; item < p.n_items; item += (i64)gridDim.x * 256) {
        Seg g;
        g.s = p.nchunks == 1 ? item : item / p.nchunks;
        g.r_begin = (item - g.s * p.nchunks) * p.chunk;
        g.r_end = min(p.inner, g.r_begin + p.chunk);
        g.nslot = 0;
        seg_setup(p, g);
        Acc acc = acc_init();
#pragma unroll 4
        for (i64 r = g.r_begin; r < g.r_end; ++r) {
            const float v = map_at(p, g, r);
#if HAS_OUT
            p.out[g.s * p.inner + r] = v;
#endif
            acc_fold(acc, v, r);
        }
#if MONOID >= 0
        if (p.nchunks == 1) {
            write_result(p, g.s, acc);
            continue;
        }
        if (!HX_CHECK(item < HX_NEST_CAP && g.s < HX_NEST_TICK, 11, item, HX_NEST_CAP)) continue;
        part_store(p.part + item, acc);
        __threadfence();
        if (atomicAdd(p.tick + g.s, 1u) == (unsigned)(p.nchunks - 1)) {
            __threadfence();
            Acc t = acc_init();
            for (i64 q = 0; q < p.nchunks; ++q) t = acc_combine(t, part_load(p.part + g.s * p.nchunks + q));
            write_result(p, g.s, t);
            p.tick[g.s] = 0u;
        }
#endif
    }
}
)CUDA";

// ---------------------------------------------------------------- host side
// Host image of the generated kernels' NestParams (same member types and
// order, so the same layout).
struct NestArgs {
    const float *in[4];
    int64_t st[4][3];
    int64_t lin[4];
    float c[8];
    int64_t dims[3];
    uint32_t dm[3];
    uint32_t ds[3];
    int64_t outer, inner, chunk, nchunks, ngroups, n_items;
    float *out;
    float *res;
    double *res64;
    int64_t *res_idx;
    float4 *part;
    float4 *part2;
    unsigned *tick;
    unsigned *tick2;
};
static_assert(sizeof(NestArgs) == 352, "NestParams layout");

struct Shape {
    int ndim, m;          // fork dims; outer dims (those indexing segments)
    int monoid;           // -1: map only
    int tree, G, U;
    bool vec;             // float4 loads / stores (aligned, unit-stride, inner % 4 == 0)
    bool has_out, has_res64, use32;
    bool used[HX_NEST_MAX_INPUTS];
    bool linear[HX_NEST_MAX_INPUTS];
    bool index_used[HX_NEST_MAX_DIMS];
};

hx_status validate(const hx_nest *n) {
    using hx::fail;
    if (!n) return fail(HX_ERR_INVALID, "hx_nest: NULL descriptor");
    if (n->ndim < 1 || n->ndim > HX_NEST_MAX_DIMS) return fail(HX_ERR_INVALID, "hx_nest: ndim must be 1..3");
    if (n->reduce_dims < 0 || n->reduce_dims > n->ndim)
        return fail(HX_ERR_INVALID, "hx_nest: reduce_dims must be 0..ndim");
    int64_t total = 1;
    for (int d = 0; d < n->ndim; ++d) {
        if (n->dims[d] < 0) return fail(HX_ERR_INVALID, "hx_nest: negative fork factor");
        if (n->dims[d] > 0 && total > ((int64_t)1 << 60) / n->dims[d])
            return fail(HX_ERR_INVALID, "hx_nest: fork too large (more than 2^60 threads)");
        total *= n->dims[d];
    }
    if (n->tree < HX_TREE_WARP || n->tree > HX_TREE_SEQ) return fail(HX_ERR_INVALID, "hx_nest: unknown tree");
    if (n->chunk < 0) return fail(HX_ERR_INVALID, "hx_nest: negative chunk");
    // pointers are needed only where the fork reads or writes something:
    // inputs and out when it has threads, results when it has segments
    int64_t segments = 1;
    for (int d = 0; d < n->ndim - n->reduce_dims; ++d) segments *= n->dims[d];
    if (n->reduce_dims == 0) {
        if (!n->out && total > 0) return fail(HX_ERR_INVALID, "hx_nest: a map-only nest needs out");
    } else {
        if (n->monoid < HX_MONOID_SUM || n->monoid > HX_MONOID_ARGMIN)
            return fail(HX_ERR_INVALID, "hx_nest: unknown monoid");
        if (!n->result && segments > 0) return fail(HX_ERR_INVALID, "hx_nest: result is NULL");
        if (n->monoid >= HX_MONOID_ARGMAX && !n->result_index && segments > 0)
            return fail(HX_ERR_INVALID, "hx_nest: argmax / argmin need result_index");
        if (((uintptr_t)n->result & 3) || ((uintptr_t)n->result64 & 7) || ((uintptr_t)n->result_index & 7))
            return fail(HX_ERR_INVALID, "hx_nest: misaligned result pointer");
    }
    if ((uintptr_t)n->out & 3) return fail(HX_ERR_INVALID, "hx_nest: misaligned out");
    if (n->n_ops < 1 || n->n_ops > HX_NEST_MAX_OPS) return fail(HX_ERR_INVALID, "hx_nest: n_ops must be 1..32");
    int depth = 0;
    for (int k = 0; k < n->n_ops; ++k) {
        const int code = n->ops[k].code, arg = n->ops[k].arg;
        switch (code) {
        case HX_OP_IN:
            if (arg < 0 || arg >= HX_NEST_MAX_INPUTS || (!n->in[arg] && total > 0))
                return fail(HX_ERR_INVALID, "hx_nest: IN names a missing input");
            if ((uintptr_t)n->in[arg] & 3) return fail(HX_ERR_INVALID, "hx_nest: misaligned input");
            depth += 1;
            break;
        case HX_OP_CONST:
            if (arg < 0 || arg >= HX_NEST_MAX_CONSTS) return fail(HX_ERR_INVALID, "hx_nest: CONST slot out of range");
            depth += 1;
            break;
        case HX_OP_INDEX:
            if (arg < 0 || arg >= n->ndim) return fail(HX_ERR_INVALID, "hx_nest: INDEX names a missing dimension");
            depth += 1;
            break;
        case HX_OP_ADD: case HX_OP_SUB: case HX_OP_MUL: case HX_OP_DIV: case HX_OP_MIN: case HX_OP_MAX:
            depth -= 1;
            break;
        case HX_OP_FMA:
            depth -= 2;
            break;
        case HX_OP_NEG: case HX_OP_ABS: case HX_OP_SQRT:
            break;
        default:
            return fail(HX_ERR_INVALID, "hx_nest: unknown op code");
        }
        if (depth < 1) return fail(HX_ERR_INVALID, "hx_nest: program pops an empty stack");
        if (depth > HX_NEST_MAX_STACK) return fail(HX_ERR_INVALID, "hx_nest: program needs more than 8 stack slots");
    }
    if (depth != 1) return fail(HX_ERR_INVALID, "hx_nest: program must leave exactly one value");
    return HX_OK;
}

// Segments (outer) and elements per segment (inner).  A map-only nest is one
// segment over the whole fork.
void extents(const hx_nest *n, int64_t *outer, int64_t *inner, int *m) {
    *m = n->reduce_dims == 0 ? 0 : n->ndim - n->reduce_dims;
    *outer = 1;
    *inner = 1;
    for (int d = 0; d < *m; ++d) *outer *= n->dims[d];
    for (int d = *m; d < n->ndim; ++d) *inner *= n->dims[d];
}

// Stride with which input k is addressed linearly over a segment (off =
// r * stride), or false when its inner dimensions do not collapse: every
// inner dimension of extent > 1 must have stride S * (product of the inner
// extents after it).
bool linear_stride(const hx_nest *n, int m, int k, int64_t *S) {
    int64_t s = 0, after = 1;
    bool have = false;
    for (int d = n->ndim - 1; d >= m; --d) {
        if (n->dims[d] > 1) {
            if (!have) {
                s = n->strides[k][d] / after;
                if (s * after != n->strides[k][d]) return false;
                have = true;
            }
            if (n->strides[k][d] != s * after) return false;
        }
        after *= n->dims[d] > 0 ? n->dims[d] : 1;
    }
    *S = s;
    return true;
}

std::string fmt(const char *f, ...) __attribute__((format(printf, 1, 2)));
std::string fmt(const char *f, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, f);
    vsnprintf(buf, sizeof buf, f, ap);
    va_end(ap);
    return buf;
}

Shape shape_of(const hx_nest *n) {
    Shape sh{};
    sh.ndim = n->ndim;
    int64_t outer, inner;
    extents(n, &outer, &inner, &sh.m);
    sh.monoid = n->reduce_dims == 0 ? -1 : n->monoid;
    sh.tree = n->tree;
    int n_used = 0;
    for (int k = 0; k < n->n_ops; ++k) {
        if (n->ops[k].code == HX_OP_IN && !sh.used[n->ops[k].arg]) {
            sh.used[n->ops[k].arg] = true;
            ++n_used;
        }
        if (n->ops[k].code == HX_OP_INDEX) sh.index_used[n->ops[k].arg] = true;
    }
    sh.U = n_used <= 2 ? 4 : 2;
    sh.G = 32;
    if (n->tree == HX_TREE_WARP) {
        const int64_t per_lane = 4 * sh.U;   // elements a lane loads per buffer
        const int64_t want = (inner + per_lane - 1) / per_lane;
        sh.G = 1;
        while (sh.G < 32 && sh.G < want) sh.G *= 2;
        // a group narrower than a warp loads a whole segment at once: no more
        // slots per lane than the segment has (registers for more segments
        // in flight)
        if (sh.G < 32) {
            const int64_t u = ((inner + 3) / 4 + sh.G - 1) / sh.G;
            if (u < sh.U) sh.U = u < 1 ? 1 : (int)u;
        }
    }
    sh.has_out = n->out != nullptr;
    sh.has_res64 = n->reduce_dims > 0 && n->result64 != nullptr;
    sh.use32 = inner < ((int64_t)1 << 31);
    // float4 slots: every slot of 4 consecutive threads must be 4 contiguous,
    // 16-byte aligned floats of every input (and of out).  That holds for a
    // linear input of stride 1, and for a strided one whose innermost
    // dimension has stride 1 and an extent divisible by 4, when the base and
    // all other strides are multiples of 4 floats.
    bool vec = n->tree == HX_TREE_WARP && inner % 4 == 0 && ((uintptr_t)n->out & 15) == 0;
    const int last = n->ndim - 1;
    for (int k = 0; k < HX_NEST_MAX_INPUTS; ++k) {
        int64_t S = 0;
        sh.linear[k] = linear_stride(n, sh.m, k, &S);
        if (!sh.used[k]) continue;
        bool ok = ((uintptr_t)n->in[k] & 15) == 0;
        if (sh.linear[k]) {
            ok = ok && (S == 1 || inner <= 1);
        } else {
            ok = ok && n->strides[k][last] == 1 && n->dims[last] % 4 == 0;
            for (int d = sh.m; d < last; ++d) ok = ok && n->strides[k][d] % 4 == 0;
        }
        for (int d = 0; d < sh.m; ++d) ok = ok && n->strides[k][d] % 4 == 0;
        vec = vec && ok;
    }
    sh.vec = vec;
    return sh;
}

// Declarations i<m> .. i<ndim-1> of the inner indices of thread r of a
// segment (multiplicative division when the segment has < 2^31 threads).
std::string inner_indices(const Shape &sh, const char *r) {
    const int last = sh.ndim - 1;
    if (sh.m == last) return fmt(" const i64 i%d = (%s);", last, r);
    std::string code;
    if (sh.use32) {
        code += fmt(" unsigned rr = (unsigned)(%s);", r);
        for (int d = last; d > sh.m; --d)
            code += fmt(" const unsigned q%d = hx_div(p, %d, rr); const i64 i%d = (i64)(rr - q%d * (unsigned)p.dims[%d]);"
                        " rr = q%d;", d, d, d, d, d, d);
    } else {
        code += fmt(" i64 rr = (%s);", r);
        for (int d = last; d > sh.m; --d) code += fmt(" const i64 i%d = rr %% p.dims[%d]; rr /= p.dims[%d];", d, d, d);
    }
    code += fmt(" const i64 i%d = (i64)rr;", sh.m);
    return code;
}

// The map program as one C expression.  style 0: inputs are slot components
// hx_comp(b.x<k>[j], q); style 1: scalars x<k>.
std::string map_expression(const hx_nest *n, const Shape &sh, int style) {
    std::string st[HX_NEST_MAX_STACK];
    int sp = 0;
    for (int k = 0; k < n->n_ops; ++k) {
        const int code = n->ops[k].code, arg = n->ops[k].arg;
        std::string a, b, c;
        switch (code) {
        case HX_OP_IN: st[sp++] = style == 0 ? fmt("hx_comp(b.x%d[j], q)", arg) : fmt("x%d", arg); break;
        case HX_OP_CONST: st[sp++] = fmt("p.c[%d]", arg); break;
        case HX_OP_INDEX: st[sp++] = arg < sh.m ? fmt("(float)g.i%d", arg) : fmt("(float)i%d", arg); break;
        case HX_OP_NEG: st[sp - 1] = "(-" + st[sp - 1] + ")"; break;
        case HX_OP_ABS: st[sp - 1] = "fabsf(" + st[sp - 1] + ")"; break;
        case HX_OP_SQRT: st[sp - 1] = "sqrtf(" + st[sp - 1] + ")"; break;
        case HX_OP_FMA:
            c = st[--sp]; b = st[--sp]; a = st[--sp];
            st[sp++] = "fmaf(" + a + ", " + b + ", " + c + ")";
            break;
        default: {
            b = st[--sp]; a = st[--sp];
            static const char *infix[] = {nullptr, nullptr, nullptr, nullptr, " + ", " - ", " * ", " / "};
            if (code >= HX_OP_ADD && code <= HX_OP_DIV) st[sp++] = "(" + a + infix[code] + b + ")";
            else st[sp++] = std::string(code == HX_OP_MIN ? "hx_minnum(" : "hx_maxnum(") + a + ", " + b + ")";
        }
        }
    }
    return st[0];
}

std::string generate(const hx_nest *n, const Shape &sh) {
    std::string src = "// libhx fork-join nest kernel (generated)\n";
    src += fmt("#define MONOID %d\n#define TREE %d\n#define G %d\n#define U %d\n#define VEC %d\n", sh.monoid, sh.tree,
               sh.G, sh.U, sh.vec ? 1 : 0);
    src += fmt("#define HAS_OUT %d\n#define HAS_RES64 %d\n", sh.has_out ? 1 : 0, sh.has_res64 ? 1 : 0);
    src += fmt("#define HX_NEST_PF %d\n", kNestPrefetch);
    src += fmt("#define HX_NEST_CAP %d\n#define HX_NEST_CAP2 %d\n#define HX_NEST_TICK %d\n#define HX_NEST_TICK2 %d\n",
               hx::kNestCap, hx::kNestCap2, hx::kNestTick, hx::kNestTick2);
#ifdef HX_DEBUG_CHECKS
    src += "#define HX_DEBUG_CHECKS 1\n";
#endif
    src += kPrelude;
    bool inner_index_used = false;
    for (int d = sh.m; d < sh.ndim; ++d) inner_index_used = inner_index_used || sh.index_used[d];

    // segment: outer indices and per-input base pointers
    std::string seg = "struct Seg {\n    i64 s, r_begin, r_end, nslot;\n";
    std::string setup = "__device__ __forceinline__ void seg_setup(const NestParams &p, Seg &g) {\n";
    if (sh.m > 0) {
        seg += "    i64";
        for (int d = 0; d < sh.m; ++d) seg += fmt("%s i%d", d ? "," : "", d);
        seg += ";\n";
        setup += "    i64 so = g.s;\n";
        for (int d = sh.m - 1; d >= 1; --d) setup += fmt("    g.i%d = so %% p.dims[%d]; so /= p.dims[%d];\n", d, d, d);
        setup += "    g.i0 = so;\n";
    }
    std::string buf = "struct Buf {\n";
    bool any_in = false;
    for (int k = 0; k < HX_NEST_MAX_INPUTS; ++k) {
        if (!sh.used[k]) continue;
        any_in = true;
        seg += fmt("    const float *b%d;\n", k);
        std::string base = "0";
        for (int d = 0; d < sh.m; ++d) base += fmt(" + g.i%d * p.st[%d][%d]", d, k, d);
        setup += fmt("    g.b%d = p.in[%d] + (%s);\n", k, k, base.c_str());
        buf += fmt("    float4 x%d[U];\n", k);
    }
    if (!any_in) buf += "    int unused;\n";
    src += seg + "};\n" + setup + "}\n" + buf + "};\n";

    // element offset of thread r of the segment in input k
    for (int k = 0; k < HX_NEST_MAX_INPUTS; ++k) {
        if (!sh.used[k]) continue;
        src += fmt("__device__ __forceinline__ i64 off%d(const NestParams &p, i64 r) {", k);
        if (sh.linear[k]) {
            src += fmt(" return r * p.lin[%d]; }\n", k);
        } else {
            src += inner_indices(sh, "r") + " return 0";
            for (int d = sh.m; d < sh.ndim; ++d) src += fmt(" + i%d * p.st[%d][%d]", d, k, d);
            src += "; }\n";
        }
    }
    // load U slots of 4 elements per lane
    src += "__device__ __forceinline__ void load_group(const NestParams &p, const Seg &g, Buf &b, i64 t0) {\n"
           "#pragma unroll\n    for (int j = 0; j < U; ++j) {\n        const i64 t = t0 + (i64)j * G;\n"
           "        if (t < g.nslot) {\n            const i64 r = g.r_begin + 4 * t;\n";
    for (int k = 0; k < HX_NEST_MAX_INPUTS; ++k) {
        if (!sh.used[k]) continue;
        if (sh.vec) {
            // a linear float4 input has stride 1: its offset is r itself
            if (sh.linear[k]) src += fmt("            b.x%d[j] = __ldg((const float4 *)(g.b%d + r));\n", k, k);
            else src += fmt("            b.x%d[j] = __ldg((const float4 *)(g.b%d + off%d(p, r)));\n", k, k, k);
        } else {
            src += fmt("            b.x%d[j].x = __ldg(g.b%d + off%d(p, r));\n", k, k, k);
            static const char comp[] = "xyzw";
            for (int q = 1; q < 4; ++q)
                src += fmt("            b.x%d[j].%c = (r + %d < g.r_end) ? __ldg(g.b%d + off%d(p, r + %d)) : 0.0f;\n", k,
                           comp[q], q, k, k, q);
        }
    }
    src += "        }\n    }\n}\n";
    // the same slots' lines prefetched into L2 (no registers held): a vector
    // slot is one 16-byte load, an element slot up to four loads
    src += "__device__ __forceinline__ void prefetch_group(const NestParams &p, const Seg &g, i64 t0) {\n"
           "#pragma unroll\n    for (int j = 0; j < U; ++j) {\n        const i64 t = t0 + (i64)j * G;\n"
           "        if (t < g.nslot) {\n            const i64 r = g.r_begin + 4 * t;\n";
    for (int k = 0; k < HX_NEST_MAX_INPUTS; ++k) {
        if (!sh.used[k]) continue;
        if (sh.vec) {
            if (sh.linear[k]) src += fmt("            prefetch_l2(g.b%d + r);\n", k);
            else src += fmt("            prefetch_l2(g.b%d + off%d(p, r));\n", k, k);
        } else {
            src += fmt("            prefetch_l2(g.b%d + off%d(p, r));\n", k, k);
            if (!sh.linear[k])
                for (int q = 1; q < 4; ++q)
                    src += fmt("            if (r + %d < g.r_end) prefetch_l2(g.b%d + off%d(p, r + %d));\n", q, k, k, q);
        }
    }
    src += "        }\n    }\n}\n";
    // map value of element (slot j, component q) = thread r
    src += "__device__ __forceinline__ float map_elem(const NestParams &p, const Seg &g, const Buf &b, int j, int q,"
           " i64 r) {";
    if (inner_index_used) src += inner_indices(sh, "r");
    src += " return " + map_expression(n, sh, 0) + "; }\n";
    // map value of thread r, loading its inputs (sequential trees)
    src += "__device__ __forceinline__ float map_at(const NestParams &p, const Seg &g, i64 r) {";
    if (inner_index_used) src += inner_indices(sh, "r");
    for (int k = 0; k < HX_NEST_MAX_INPUTS; ++k)
        if (sh.used[k]) src += fmt(" const float x%d = __ldg(g.b%d + off%d(p, r));", k, k, k);
    src += " return " + map_expression(n, sh, 1) + "; }\n";
    src += sh.tree == HX_TREE_WARP ? kWarpBody : kThreadBody;
    return src;
}

// ---------------------------------------------------------------- compile cache
struct Compiled {
    std::string cubin;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kernel = nullptr;
    int ctas_per_sm = 1;   // resident CTAs of kNestBlock threads per SM
};

std::mutex g_mu;
std::unordered_map<std::string, Compiled *> g_cache;

hx_status compile(const std::string &src, Compiled **out) {
    {
        std::lock_guard<std::mutex> lk(g_mu);
        auto it = g_cache.find(src);
        if (it != g_cache.end()) {
            *out = it->second;
            return HX_OK;
        }
    }
    nvrtcProgram prog;
    if (nvrtcCreateProgram(&prog, src.c_str(), "hx_nest.cu", 0, nullptr, nullptr) != NVRTC_SUCCESS)
        return hx::fail(HX_ERR_CUDA, "hx_nest: nvrtcCreateProgram failed");
    const char *opts[] = {"--gpu-architecture=sm_103a", "--fmad=false", "--ftz=false", "--prec-div=true",
                          "--prec-sqrt=true", "-default-device", "--std=c++17"};
    nvrtcResult rc = nvrtcCompileProgram(prog, (int)(sizeof opts / sizeof opts[0]), opts);
    if (rc != NVRTC_SUCCESS) {
        size_t n = 0;
        nvrtcGetProgramLogSize(prog, &n);
        std::string log(n, '\0');
        nvrtcGetProgramLog(prog, &log[0]);
        nvrtcDestroyProgram(&prog);
        return hx::fail(HX_ERR_CUDA, "hx_nest: generated kernel failed to compile: " + log.substr(0, 2000));
    }
    size_t n = 0;
    nvrtcGetCUBINSize(prog, &n);
    Compiled *c = new Compiled();
    c->cubin.resize(n);
    nvrtcGetCUBIN(prog, &c->cubin[0]);
    nvrtcDestroyProgram(&prog);
    std::lock_guard<std::mutex> lk(g_mu);
    auto ins = g_cache.emplace(src, c);
    if (!ins.second) delete c;   // another thread compiled it first
    *out = ins.first->second;
    return HX_OK;
}

hx_status load(Compiled *c) {
    std::lock_guard<std::mutex> lk(g_mu);
    if (c->kernel) return HX_OK;
    cudaError_t e = cudaLibraryLoadData(&c->lib, c->cubin.data(), nullptr, nullptr, 0, nullptr, nullptr, 0);
    if (e != cudaSuccess) return hx::cuda_fail(e, "hx_nest: cudaLibraryLoadData");
    cudaKernel_t k = nullptr;
    e = cudaLibraryGetKernel(&k, c->lib, "hx_nest_kernel");
    if (e != cudaSuccess) return hx::cuda_fail(e, "hx_nest: cudaLibraryGetKernel");
    int occ = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, (const void *)k, kNestBlock, 0);
    if (e != cudaSuccess) return hx::cuda_fail(e, "hx_nest: occupancy query");
    c->ctas_per_sm = occ > 0 ? occ : 1;
    c->kernel = k;
    return HX_OK;
}

// Work split of a nest: elements per item (chunk), items per segment, and
// groups of 32 chunks per segment (warp tree).
struct Split {
    int64_t chunk, nchunks, ngroups;
};

hx_status split_of(const hx_nest *n, const hx_tune_table *tune, int64_t outer, int64_t inner, const Shape &sh,
                   Split *out) {
    const int64_t cap = hx::kNestCap;
    const int64_t whole = inner > 0 ? inner : 1;
    Split sp{whole, 1, 1};
    if (n->tree == HX_TREE_SEQ) {
        *out = sp;
        return HX_OK;
    }
    int64_t chunk;
    if (n->chunk > 0) chunk = n->chunk;
    else if (n->tree == HX_TREE_WARP) chunk = (int64_t)sh.G * (tune ? tune->nest_lane_elems[hx::size_class(inner)] : 16);
    else chunk = 64;
    if (n->tree == HX_TREE_WARP) chunk = (chunk + 3) / 4 * 4;   // whole slots
    // groups narrower than a warp take whole segments (the chunk tree below
    // relies on the full warp sharing a chunk)
    if ((n->tree == HX_TREE_WARP && sh.G < 32) || inner <= chunk || (sh.monoid >= 0 && outer > cap / 2)) {
        *out = sp;
        return HX_OK;
    }
    int64_t nchunks = (inner + chunk - 1) / chunk;
    if (sh.monoid >= 0 && outer * nchunks > cap) {
        nchunks = cap / outer;
        chunk = (inner + nchunks - 1) / nchunks;
        if (n->tree == HX_TREE_WARP) chunk = (chunk + 511) / 512 * 512;
        nchunks = (inner + chunk - 1) / chunk;
    }
    sp.chunk = chunk;
    sp.nchunks = nchunks;
    sp.ngroups = n->tree == HX_TREE_WARP ? (nchunks + 31) / 32 : 1;
    if (sh.monoid >= 0) {
        // workspace bounds (see NestWs): these hold by construction
        const bool ok = outer * nchunks <= cap && outer * sp.ngroups <= hx::kNestTick &&
                        (sp.ngroups == 1 || (outer * sp.ngroups <= hx::kNestCap2 && outer <= hx::kNestTick2));
        if (!ok) return hx::fail(HX_ERR_NOMEM, "hx_nest: chunk plan exceeds the workspace");
    }
    *out = sp;
    return HX_OK;
}

// A warp-tree reduction whose chunks outnumber the warps the device holds at
// once gets longer chunks instead: one chunk per resident warp (at least one
// per segment), a multiple of 512 elements.  Each warp then streams one long
// chunk, and the tree above the chunks (arrival tickets, group partials)
// shrinks by the same factor.  Explicit chunk lengths are kept.  Pure maps
// keep the tuned chunk: without a tree to shrink, 16 KiB chunks over several
// waves measured faster (1.03 against 0.97 of HBM for a 2^27 copy-like map).
void one_wave(const hx_nest *n, const Shape &sh, int64_t outer, int64_t inner, int64_t warps, Split *sp) {
    if (n->tree != HX_TREE_WARP || sh.G != 32 || sh.monoid < 0 || n->chunk > 0) return;
    if (outer * sp->nchunks <= warps) return;
    int64_t per_seg = warps / outer;
    if (per_seg < 1) per_seg = 1;
    if (per_seg >= sp->nchunks) return;
    int64_t chunk = (inner + per_seg - 1) / per_seg;
    chunk = (chunk + 511) / 512 * 512;
    sp->chunk = chunk;
    sp->nchunks = (inner + chunk - 1) / chunk;
    sp->ngroups = (sp->nchunks + 31) / 32;
}

// A large warp-tree SUM takes about 2.7 chunks per resident warp instead of
// one.  The grid holds at most 2048 threads per SM, so a warp then folds one
// to three chunks and the CTAs run as waves whose last one is nearly full.
// Measured on a B300 (fraction of copy bandwidth, one chunk per warp against
// this split): 2^28 sum 0.95 -> 1.01, 1024 x 512 x 512 permuted reduce
// 0.90 -> 0.95, rows of 163840 0.93 -> 1.03, rows of 65536 0.95 -> 1.01.
// Load counts just above a whole number of waves (x = items / resident warps
// in 2.0-2.2 or 1.1-1.3) measured 0.77-0.94, so x is kept in 1.8-2.9.
// Chunks of a multiple of 16384 elements (64 KiB) measured 3-4 % slower than
// their neighbours and are avoided.  Chunks shorter than 8192 elements (a 2^26
// sum) lose more to the larger tree than they gain, and the exact monoids
// (max, min, argmax ...) measured fastest at one chunk per warp (max |x| over
// 2^28: 0.97 against 0.91), so both keep one_wave.  Returns whether it split.
bool spread_sum(const hx_nest *n, const Shape &sh, int64_t outer, int64_t inner, int64_t warps, Split *sp) {
    if (n->tree != HX_TREE_WARP || sh.G != 32 || sh.monoid != HX_MONOID_SUM || n->chunk > 0 || warps < 1) return false;
    const double target = 2.7 * (double)warps;
    if ((double)(outer * sp->nchunks) <= target) return false;
    int64_t p0 = (int64_t)(target / (double)outer + 0.5);
    if (p0 < 1) p0 = 1;
    int64_t best_chunk = 0;
    int best_bad = 4;
    double best_dist = 0;
    for (int64_t d = 0; d <= 16; ++d) {
        for (int side = 0; side < 2; ++side) {
            if (d == 0 && side == 1) continue;
            const int64_t p = side == 0 ? p0 + d : p0 - d;
            if (p < 1 || p > sp->nchunks) continue;   // p <= the tuned count keeps the workspace bounds
            int64_t chunk = (inner + p - 1) / p;
            chunk = (chunk + 511) / 512 * 512;
            const int64_t nch = (inner + chunk - 1) / chunk;
            const double x = (double)(outer * nch) / (double)warps;
            const int bad = (chunk % 16384 == 0 ? 2 : 0) + (x >= 1.8 && x <= 2.9 ? 0 : 1);
            const double dist = x > 2.7 ? x - 2.7 : 2.7 - x;
            if (bad < best_bad || (bad == best_bad && dist < best_dist)) {
                best_bad = bad;
                best_dist = dist;
                best_chunk = chunk;
            }
        }
    }
    if (best_chunk < 8192) return false;
    sp->chunk = best_chunk;
    sp->nchunks = (inner + best_chunk - 1) / best_chunk;
    sp->ngroups = (sp->nchunks + 31) / 32;
    return true;
}

hx_status prepare(const hx_nest *n, const hx_tune_table *tune, Compiled **c, Shape *sh, Split *sp, int64_t *outer,
                  int64_t *inner) {
    hx_status st = validate(n);
    if (st != HX_OK) return st;
    int m;
    extents(n, outer, inner, &m);
    *sh = shape_of(n);
    st = split_of(n, tune, *outer, *inner, *sh, sp);
    if (st != HX_OK) return st;
    return compile(generate(n, *sh), c);
}

// Multiplier and shift for quotients by d of 31-bit numerators: l =
// ceil(log2 d), m = ceil(2^(31+l) / d) < 2^32 (Granlund and Montgomery 1994,
// Thm. 4.2: m*d - 2^(31+l) < d <= 2^l).
void magic(int64_t d, uint32_t *m, uint32_t *s) {
    if (d < 1 || d >= ((int64_t)1 << 31)) d = 1;   // unused: the kernel divides in 64 bits then
    int l = 0;
    while (((int64_t)1 << l) < d) ++l;
    const uint64_t two = (uint64_t)1 << (31 + l);
    *m = (uint32_t)((two + (uint64_t)d - 1) / (uint64_t)d);
    *s = 31 + l;
}

}  // namespace

namespace hx {
// The check records of every loaded generated kernel (debug build): the
// first non-empty one is reported; all are cleared.
hx_status checks_nest(int32_t *code, int64_t *a, int64_t *b) {
    *code = 0;
    *a = 0;
    *b = 0;
#ifdef HX_DEBUG_CHECKS
    std::lock_guard<std::mutex> lk(g_mu);
    for (auto &kv : g_cache) {
        Compiled *c = kv.second;
        if (!c->lib) continue;
        void *d = nullptr;
        size_t bytes = 0;
        cudaError_t e = cudaLibraryGetGlobal(&d, &bytes, c->lib, "hx_check_rec");
        if (e != cudaSuccess || bytes < 3 * sizeof(unsigned long long)) return cuda_fail(e, "hx_debug_checks: nest record");
        unsigned long long r[3];
        e = cudaMemcpy(r, d, sizeof r, cudaMemcpyDeviceToHost);
        if (e == cudaSuccess && r[0] != 0) e = cudaMemset(d, 0, sizeof r);
        if (e != cudaSuccess) return cuda_fail(e, "hx_debug_checks: nest record");
        if (r[0] != 0 && *code == 0) {
            *code = (int32_t)r[0];
            *a = (int64_t)r[1];
            *b = (int64_t)r[2];
        }
    }
#endif
    return HX_OK;
}
}  // namespace hx

extern "C" {

hx_status hx_nest_source(const hx_nest *nest, char *buf, size_t cap, size_t *len) {
    hx_status st = validate(nest);
    if (st != HX_OK) return st;
    const std::string src = generate(nest, shape_of(nest));
    if (len) *len = src.size();
    if (buf && cap) {
        const size_t k = src.size() < cap - 1 ? src.size() : cap - 1;
        memcpy(buf, src.data(), k);
        buf[k] = '\0';
    }
    return HX_OK;
}

hx_status hx_nest_prepare(const hx_nest *nest) {
    Compiled *c;
    Shape sh;
    Split sp;
    int64_t outer, inner;
    return prepare(nest, nullptr, &c, &sh, &sp, &outer, &inner);
}

hx_status hx_fork_reduce(hx_ctx *ctx, const hx_nest *nest, hx_stream_t stream) {
    if (!ctx) return hx::fail(HX_ERR_INVALID, "hx_fork_reduce: NULL context");
    Compiled *c;
    Shape sh;
    Split sp;
    int64_t outer, inner;
    hx_status st = prepare(nest, &ctx->tune, &c, &sh, &sp, &outer, &inner);
    if (st != HX_OK) return st;
    if (outer == 0 || (nest->reduce_dims == 0 && inner == 0)) return HX_OK;
    hx::DeviceGuard g(ctx->device);
    hx::WsSlot *slot;
    st = hx::slot_for(ctx, stream, &slot);
    if (st != HX_OK) return st;
    st = load(c);
    if (st != HX_OK) return st;
    const int64_t warps = (int64_t)ctx->num_sms * c->ctas_per_sm * (kNestBlock / 32);
    if (!spread_sum(nest, sh, outer, inner, warps, &sp)) one_wave(nest, sh, outer, inner, warps, &sp);
    if (hx::take_injected_failure(ctx))
        return hx::fail(HX_ERR_CUDA, "hx_fork_reduce: injected launch failure (test hook)");
    hx::NestWs *ws = ctx->nest_ws + (slot - ctx->ws);

    NestArgs a{};
    for (int k = 0; k < HX_NEST_MAX_INPUTS; ++k) {
        a.in[k] = nest->in[k];
        for (int d = 0; d < 3; ++d) a.st[k][d] = d < nest->ndim ? nest->strides[k][d] : 0;
        if (sh.linear[k]) linear_stride(nest, sh.m, k, &a.lin[k]);
    }
    for (int k = 0; k < HX_NEST_MAX_CONSTS; ++k) a.c[k] = nest->consts[k];
    for (int d = 0; d < 3; ++d) {
        a.dims[d] = d < nest->ndim ? nest->dims[d] : 1;
        magic(a.dims[d], &a.dm[d], &a.ds[d]);
    }
    a.outer = outer;
    a.inner = inner;
    a.chunk = sp.chunk;
    a.nchunks = sp.nchunks;
    a.ngroups = sp.ngroups;
    a.n_items = outer * sp.nchunks;
    a.out = nest->out;
    a.res = nest->result;
    a.res64 = nest->result64;
    a.res_idx = nest->result_index;
    a.part = ws->part;
    a.part2 = ws->part2;
    a.tick = ws->tick;
    a.tick2 = ws->tick2;

    const int64_t threads = sh.tree == HX_TREE_WARP ? a.n_items * sh.G : a.n_items;
    int64_t blocks = (threads + kNestBlock - 1) / kNestBlock;
    // whole waves of resident CTAs, up to 2048 threads per SM (a partial
    // last wave would run the items' tail at low occupancy)
    const int waves = c->ctas_per_sm >= 2048 / kNestBlock ? 1 : (2048 / kNestBlock) / c->ctas_per_sm;
    const int64_t max_blocks = (int64_t)ctx->num_sms * c->ctas_per_sm * waves;
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    void *args[] = {&a};
    cudaError_t e = cudaLaunchKernel((const void *)c->kernel, dim3((unsigned)blocks), dim3(kNestBlock), args, 0,
                                     (cudaStream_t)stream);
    if (e != cudaSuccess) return hx::cuda_fail(e, "hx_fork_reduce: launch");
    return HX_OK;
}

}  // extern "C"
