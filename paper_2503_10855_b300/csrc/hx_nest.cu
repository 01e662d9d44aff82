// hx_nest.cu -- generic fork-join nests: a fork of one to three factors whose
// body is a small straight-line map program, feeding a monoid reduce over the
// innermost fork dimensions (Hercules paper, Sec. 3.3 fork-joins and reduces,
// Sec. 3.4 MonoidReduce).
//
// Like the Hercules GPU backend (Sec. 4.4), the library turns the nest into a
// CUDA kernel: the map program becomes one fused expression, pasted into the
// hand-written kernel template below together with the nest's shape
// (dimension counts, monoid, reduction schedule, addressing mode of every
// input), and the result is compiled for sm_103a with NVRTC.  Sizes, strides,
// constants and pointers are launch arguments, so one compiled kernel serves
// every nest of the same shape; compiled kernels are cached process-wide by
// their source text.
//
// Reduction schedules (Sec. 5.2, the reduction-tree macro and warp reductions):
//   HX_TREE_WARP   chunks of a segment go to groups of G lanes (G = 32, or the
//                  next power of two >= the segment length when that is below
//                  32); lanes stride through the chunk, fold their elements
//                  in order, combine with a shuffle butterfly; chunk partials
//                  are combined by the group that arrives last (ticket).
//   HX_TREE_CHUNK  the two-level tree of the reduction-tree macro: one thread
//                  folds each contiguous chunk sequentially, the last thread
//                  to finish folds the chunk partials sequentially.
//   HX_TREE_SEQ    the untransformed loop: one thread folds a whole segment.
// Sums and products accumulate in float-float (hi, lo) pairs; extrema are
// exact.  The combination order depends only on the nest's sizes, schedule
// and chunk, so results are bit-identical from run to run.
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
constexpr int kNestU = 8;   // elements per lane in flight (warp tree)

// ---------------------------------------------------------------- device template
// Everything the generated kernels share.  MONOID (-1 = map only), TREE, G and
// the HAS_* flags are #defined by the generated header in front of it.
const char *kPrelude = R"CUDA(
typedef long long i64;
struct NestParams {
    const float *in[4];
    i64 st[4][3];
    i64 lin[4];     // stride of an input addressed linearly inside a segment
    float c[8];
    i64 dims[3];
    i64 outer, inner, chunk, nchunks, n_items;
    float *out;
    float *res;
    double *res64;
    i64 *res_idx;
    float4 *part;
    unsigned *tick;
};

__device__ __forceinline__ float hx_minnum(float a, float b) {
    return isnan(a) ? b : (isnan(b) ? a : (b < a ? b : a));
}
__device__ __forceinline__ float hx_maxnum(float a, float b) {
    return isnan(a) ? b : (isnan(b) ? a : (b > a ? b : a));
}
#define HX_NEG_INF __int_as_float(0xff800000)
#define HX_POS_INF __int_as_float(0x7f800000)

#if MONOID == 0 || MONOID == 3
struct Acc { float hi, lo; };
#elif MONOID == 1 || MONOID == 2
struct Acc { float v; };
#elif MONOID >= 4
struct Acc { float v; i64 i; };
#endif

#if MONOID >= 0
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
#else
    return Acc{HX_POS_INF, -1};
#endif
}

// Fold one value of thread r into a running accumulator (thread-ID order).
__device__ __forceinline__ void acc_fold(Acc &a, float v, i64 r) {
#if MONOID == 0
    float s = a.hi + v, bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (v - bb);     // exact error of a.hi + v
    e = e + a.lo;
    float h = s + e;
    a.lo = e - (h - s);
    a.hi = h;
#elif MONOID == 3
    float pr = a.hi * v;
    float e = fmaf(a.hi, v, -pr);               // exact error of a.hi * v
    e = fmaf(a.lo, v, e);
    float h = pr + e;
    a.lo = e - (h - pr);
    a.hi = h;
#elif MONOID == 1
    if (v > a.v || (v == 0.0f && a.v == 0.0f && signbit(a.v) && !signbit(v))) a.v = v;
#elif MONOID == 2
    if (v < a.v || (v == 0.0f && a.v == 0.0f && !signbit(a.v) && signbit(v))) a.v = v;
#elif MONOID == 4
    if (!isnan(v) && (a.i < 0 || v > a.v)) { a.v = v; a.i = r; }
#else
    if (!isnan(v) && (a.i < 0 || v < a.v)) { a.v = v; a.i = r; }
#endif
}

// Combine two partial results.  Commutative bit for bit (the exact TwoSum /
// TwoProd error terms do not depend on operand order; extrema break ties by
// the smaller thread index), so both lanes of a butterfly pair agree.
__device__ __forceinline__ Acc acc_combine(Acc a, Acc b) {
#if MONOID == 0
    float s = a.hi + b.hi, bb = s - a.hi;
    float e = (a.hi - (s - bb)) + (b.hi - bb);
    e = e + (a.lo + b.lo);
    float h = s + e;
    return Acc{h, e - (h - s)};
#elif MONOID == 3
    float pr = a.hi * b.hi;
    float e = fmaf(a.hi, b.hi, -pr);
    e = e + (a.hi * b.lo + a.lo * b.hi);
    float h = pr + e;
    return Acc{h, e - (h - pr)};
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

__device__ __forceinline__ Acc acc_shfl(unsigned mask, Acc a, int k) {
    Acc o = a;
#if MONOID == 0 || MONOID == 3
    o.hi = __shfl_xor_sync(mask, a.hi, k, G);
    o.lo = __shfl_xor_sync(mask, a.lo, k, G);
#elif MONOID == 1 || MONOID == 2
    o.v = __shfl_xor_sync(mask, a.v, k, G);
#else
    o.v = __shfl_xor_sync(mask, a.v, k, G);
    o.i = __shfl_xor_sync(mask, a.i, k, G);
#endif
    return o;
}

union PartBits { float4 f4; struct { float a, b; i64 i; } s; };

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
    *dst = u.f4;
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

// Chunk partial of item (s, c); the last chunk of segment s to arrive folds
// all of the segment's partials in chunk order.  Called by one thread.
__device__ __forceinline__ bool publish_partial(const NestParams &p, i64 s, i64 item, Acc a) {
    part_store(p.part + item, a);
    __threadfence();
    return atomicAdd(p.tick + s, 1u) == (unsigned)(p.nchunks - 1);
}
#endif  // MONOID >= 0
)CUDA";

// The kernel bodies.  OUTER_SETUP(s), LOAD(j, r) / MAP(j, r) and the
// per-element index setup INNER_IDX(r) are generated per nest.
const char *kWarpBody = R"CUDA(
extern "C" __global__ void __launch_bounds__(256) hx_nest_kernel(const NestParams p) {
    const int lane = threadIdx.x & 31;
    const int gl = lane & (G - 1);
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const i64 per_cta = 256 / G;
    for (i64 item = (i64)blockIdx.x * per_cta + threadIdx.x / G; item < p.n_items;
         item += (i64)gridDim.x * per_cta) {
        const i64 s = item / p.nchunks;
        const i64 r_begin = (item - s * p.nchunks) * p.chunk;
        const i64 r_end = min(p.inner, r_begin + p.chunk);
        OUTER_SETUP
#if MONOID >= 0
        Acc acc = acc_init();
#endif
        for (i64 r0 = r_begin + gl; r0 < r_end; r0 += (i64)G * U) {
            LOAD_DECL
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const i64 r = r0 + (i64)j * G;
                if (r < r_end) {
                    LOAD_BODY
                }
            }
#pragma unroll
            for (int j = 0; j < U; ++j) {
                const i64 r = r0 + (i64)j * G;
                if (r < r_end) {
                    MAP_BODY
#if HAS_OUT
                    p.out[s * p.inner + r] = v;
#endif
#if MONOID >= 0
                    acc_fold(acc, v, r);
#endif
                }
            }
        }
#if MONOID >= 0
#pragma unroll
        for (int k = G / 2; k >= 1; k >>= 1) acc = acc_combine(acc, acc_shfl(gmask, acc, k));
        if (p.nchunks == 1) {
            if (gl == 0) write_result(p, s, acc);
        } else {
            // nchunks > 1 only with G == 32: the whole warp shares the item
            unsigned last = 0;
            if (lane == 0) last = publish_partial(p, s, item, acc) ? 1u : 0u;
            last = __shfl_sync(0xffffffffu, last, 0);
            if (last) {
                __threadfence();
                Acc t = acc_init();
                for (i64 q = lane; q < p.nchunks; q += 32) t = acc_combine(t, part_load(p.part + s * p.nchunks + q));
#pragma unroll
                for (int k = 16; k >= 1; k >>= 1) t = acc_combine(t, acc_shfl(0xffffffffu, t, k));
                if (lane == 0) {
                    write_result(p, s, t);
                    p.tick[s] = 0u;
                }
            }
        }
#endif
    }
}
)CUDA";

const char *kThreadBody = R"CUDA(
// One thread per item: HX_TREE_CHUNK (items = chunks) or HX_TREE_SEQ (items =
// segments, nchunks == 1).  Sequential fold in thread-ID order.
extern "C" __global__ void __launch_bounds__(256) hx_nest_kernel(const NestParams p) {
    for (i64 item = (i64)blockIdx.x * 256 + threadIdx.x; item < p.n_items; item += (i64)gridDim.x * 256) {
        const i64 s = item / p.nchunks;
        const i64 r_begin = (item - s * p.nchunks) * p.chunk;
        const i64 r_end = min(p.inner, r_begin + p.chunk);
        OUTER_SETUP
#if MONOID >= 0
        Acc acc = acc_init();
#endif
        for (i64 r = r_begin; r < r_end; ++r) {
            const int j = 0;
            LOAD_DECL
            LOAD_BODY
            MAP_BODY
#if HAS_OUT
            p.out[s * p.inner + r] = v;
#endif
#if MONOID >= 0
            acc_fold(acc, v, r);
#endif
        }
#if MONOID >= 0
        if (p.nchunks == 1) {
            write_result(p, s, acc);
        } else if (publish_partial(p, s, item, acc)) {
            __threadfence();
            Acc t = acc_init();
            for (i64 q = 0; q < p.nchunks; ++q) t = acc_combine(t, part_load(p.part + s * p.nchunks + q));
            write_result(p, s, t);
            p.tick[s] = 0u;
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
    int64_t outer, inner, chunk, nchunks, n_items;
    float *out;
    float *res;
    double *res64;
    int64_t *res_idx;
    float4 *part;
    unsigned *tick;
};
static_assert(sizeof(NestArgs) == 304, "NestParams layout");

struct Shape {
    int ndim, m;          // fork dims; dims addressed per segment (outer)
    int monoid;           // -1: map only
    int tree, G, U;
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

Shape shape_of(const hx_nest *n) {
    Shape sh{};
    sh.ndim = n->ndim;
    int64_t outer, inner;
    extents(n, &outer, &inner, &sh.m);
    sh.monoid = n->reduce_dims == 0 ? -1 : n->monoid;
    sh.tree = n->tree;
    sh.U = kNestU;
    sh.G = 32;
    if (n->tree == HX_TREE_WARP && inner < 32) {
        sh.G = 1;
        while (sh.G < inner) sh.G *= 2;
    }
    sh.has_out = n->out != nullptr;
    sh.has_res64 = n->reduce_dims > 0 && n->result64 != nullptr;
    sh.use32 = inner < ((int64_t)1 << 31);
    for (int k = 0; k < n->n_ops; ++k) {
        if (n->ops[k].code == HX_OP_IN) sh.used[n->ops[k].arg] = true;
        if (n->ops[k].code == HX_OP_INDEX) sh.index_used[n->ops[k].arg] = true;
    }
    for (int k = 0; k < HX_NEST_MAX_INPUTS; ++k) {
        int64_t S;
        sh.linear[k] = linear_stride(n, sh.m, k, &S);
    }
    return sh;
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

// The map program as one C expression over x<k>[j] (loaded inputs), p.c[k]
// and the fork indices i<d>.
std::string map_expression(const hx_nest *n) {
    std::string st[HX_NEST_MAX_STACK];
    int sp = 0;
    for (int k = 0; k < n->n_ops; ++k) {
        const int code = n->ops[k].code, arg = n->ops[k].arg;
        std::string a, b, c;
        switch (code) {
        case HX_OP_IN: st[sp++] = fmt("x%d[j]", arg); break;
        case HX_OP_CONST: st[sp++] = fmt("p.c[%d]", arg); break;
        case HX_OP_INDEX: st[sp++] = fmt("(float)i%d", arg); break;
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

// Index of dimension d inside the segment, from r (the segment-local thread
// index), for the inner dims [m, ndim).
std::string inner_indices(const Shape &sh, bool need[HX_NEST_MAX_DIMS]) {
    std::string code;
    const int last = sh.ndim - 1;
    bool any = false;
    for (int d = sh.m; d <= last; ++d) any = any || need[d];
    if (!any) return code;
    if (sh.m == last) return fmt("const i64 i%d = r;", last);
    const char *ty = sh.use32 ? "unsigned" : "i64";
    code += fmt("%s rr = (%s)r;", ty, ty);
    for (int d = last; d > sh.m; --d) {
        code += fmt(" const i64 i%d = (i64)(rr %% (%s)p.dims[%d]); rr /= (%s)p.dims[%d];", d, ty, d, ty, d);
    }
    code += fmt(" const i64 i%d = (i64)rr;", sh.m);
    return code;
}

std::string generate(const hx_nest *n, const Shape &sh) {
    std::string src = "// libhx fork-join nest kernel (generated)\n";
    src += fmt("#define MONOID %d\n#define TREE %d\n#define G %d\n#define U %d\n", sh.monoid, sh.tree, sh.G,
               sh.tree == HX_TREE_WARP ? sh.U : 1);
    src += fmt("#define HAS_OUT %d\n#define HAS_RES64 %d\n", sh.has_out ? 1 : 0, sh.has_res64 ? 1 : 0);
    // outer indices and per-input segment base offsets
    std::string outer = "";
    if (sh.m > 0) {
        outer += "i64 so = s;";
        for (int d = sh.m - 1; d >= 1; --d)
            outer += fmt(" const i64 i%d = so %% p.dims[%d]; so /= p.dims[%d];", d, d, d);
        outer += " const i64 i0 = so;";
    }
    bool need_inner[HX_NEST_MAX_DIMS] = {};
    for (int d = sh.m; d < sh.ndim; ++d) need_inner[d] = sh.index_used[d];
    std::string load_decl, load_body;
    for (int k = 0; k < HX_NEST_MAX_INPUTS; ++k) {
        if (!sh.used[k]) continue;
        std::string base = "0";
        for (int d = 0; d < sh.m; ++d) base += fmt(" + i%d * p.st[%d][%d]", d, k, d);
        outer += fmt(" const float *b%d = p.in[%d] + (%s);", k, k, base.c_str());
        load_decl += fmt(" float x%d[U];", k);
        if (!sh.linear[k])
            for (int d = sh.m; d < sh.ndim; ++d) need_inner[d] = true;
    }
    // loads: linear inputs use r directly, the others the inner indices
    bool lin_need[HX_NEST_MAX_DIMS] = {};
    bool any_nonlin = false;
    for (int k = 0; k < HX_NEST_MAX_INPUTS; ++k)
        if (sh.used[k] && !sh.linear[k]) any_nonlin = true;
    if (any_nonlin) {
        for (int d = sh.m; d < sh.ndim; ++d) lin_need[d] = true;
        load_body += "{ " + inner_indices(sh, lin_need);
    } else {
        load_body += "{";
    }
    for (int k = 0; k < HX_NEST_MAX_INPUTS; ++k) {
        if (!sh.used[k]) continue;
        std::string off;
        if (sh.linear[k]) {
            off = fmt("r * p.lin[%d]", k);
        } else {
            off = "0";
            for (int d = sh.m; d < sh.ndim; ++d) off += fmt(" + i%d * p.st[%d][%d]", d, k, d);
        }
        load_body += fmt(" x%d[j] = __ldg(b%d + (%s));", k, k, off.c_str());
    }
    load_body += " }";
    bool idx_need[HX_NEST_MAX_DIMS] = {};
    for (int d = sh.m; d < sh.ndim; ++d) idx_need[d] = sh.index_used[d];
    std::string map_body = inner_indices(sh, idx_need) + " const float v = " + map_expression(n) + ";";
    if (load_decl.empty()) load_decl = " ";
    src += "#define OUTER_SETUP " + (outer.empty() ? std::string(" ") : outer) + "\n";
    src += "#define LOAD_DECL" + load_decl + "\n";
    src += "#define LOAD_BODY " + load_body + "\n";
    src += "#define MAP_BODY " + map_body + "\n";
    src += kPrelude;
    src += sh.tree == HX_TREE_WARP ? kWarpBody : kThreadBody;
    return src;
}

// ---------------------------------------------------------------- compile cache
struct Compiled {
    std::string cubin;
    cudaLibrary_t lib = nullptr;
    cudaKernel_t kernel = nullptr;
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
    e = cudaLibraryGetKernel(&c->kernel, c->lib, "hx_nest_kernel");
    if (e != cudaSuccess) return hx::cuda_fail(e, "hx_nest: cudaLibraryGetKernel");
    return HX_OK;
}

// Work split of a nest: elements per item and items per segment.
struct Split {
    int64_t chunk, nchunks;
};

Split split_of(const hx_nest *n, const hx_tune_table *tune, int64_t outer, int64_t inner, const Shape &sh) {
    const int64_t cap = hx::kNestCap;
    int64_t chunk;
    if (n->tree == HX_TREE_SEQ) return Split{inner > 0 ? inner : 1, 1};
    // sub-warp groups (segments shorter than 32) take a whole segment each:
    // the ticket path below assumes the full warp shares a chunk
    if (n->tree == HX_TREE_WARP && sh.G < 32) return Split{inner > 0 ? inner : 1, 1};
    if (n->chunk > 0) {
        chunk = n->chunk;
    } else if (n->tree == HX_TREE_WARP) {
        chunk = (int64_t)sh.G * (tune ? tune->nest_lane_elems[hx::size_class(inner)] : 16);
    } else {
        chunk = 64;
    }
    if (inner <= chunk || (sh.monoid >= 0 && outer > cap / 2)) return Split{inner > 0 ? inner : 1, 1};
    int64_t nchunks = (inner + chunk - 1) / chunk;
    if (sh.monoid >= 0 && outer * nchunks > cap) {
        nchunks = cap / outer;
        chunk = (inner + nchunks - 1) / nchunks;
        if (n->tree == HX_TREE_WARP) chunk = (chunk + 32 * kNestU - 1) / (32 * kNestU) * (32 * kNestU);
        nchunks = (inner + chunk - 1) / chunk;
    }
    return Split{chunk, nchunks};
}

hx_status prepare(const hx_nest *n, const hx_tune_table *tune, Compiled **c, Shape *sh, Split *sp, int64_t *outer,
                  int64_t *inner) {
    hx_status st = validate(n);
    if (st != HX_OK) return st;
    int m;
    extents(n, outer, inner, &m);
    *sh = shape_of(n);
    *sp = split_of(n, tune, *outer, *inner, *sh);
    return compile(generate(n, *sh), c);
}

}  // namespace

extern "C" {

hx_status hx_nest_source(const hx_nest *nest, char *buf, size_t cap, size_t *len) {
    hx_status st = validate(nest);
    if (st != HX_OK) return st;
    int64_t outer, inner;
    int m;
    extents(nest, &outer, &inner, &m);
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
    hx::NestWs *ws = ctx->nest_ws + (slot - ctx->ws);

    NestArgs a{};
    for (int k = 0; k < HX_NEST_MAX_INPUTS; ++k) {
        a.in[k] = nest->in[k];
        for (int d = 0; d < 3; ++d) a.st[k][d] = d < nest->ndim ? nest->strides[k][d] : 0;
        if (sh.linear[k]) linear_stride(nest, sh.m, k, &a.lin[k]);
    }
    for (int k = 0; k < HX_NEST_MAX_CONSTS; ++k) a.c[k] = nest->consts[k];
    for (int d = 0; d < 3; ++d) a.dims[d] = d < nest->ndim ? nest->dims[d] : 1;
    a.outer = outer;
    a.inner = inner;
    a.chunk = sp.chunk;
    a.nchunks = sp.nchunks;
    a.n_items = outer * sp.nchunks;
    a.out = nest->out;
    a.res = nest->result;
    a.res64 = nest->result64;
    a.res_idx = nest->result_index;
    a.part = ws->part;
    a.tick = ws->tick;

    int64_t threads;
    if (sh.tree == HX_TREE_WARP) threads = a.n_items * sh.G;
    else threads = a.n_items;
    int64_t blocks = (threads + kNestBlock - 1) / kNestBlock;
    const int64_t max_blocks = (int64_t)ctx->num_sms * (2048 / kNestBlock);
    if (blocks > max_blocks) blocks = max_blocks;
    if (blocks < 1) blocks = 1;
    void *args[] = {&a};
    cudaError_t e = cudaLaunchKernel((const void *)c->kernel, dim3((unsigned)blocks), dim3(kNestBlock), args, 0,
                                     (cudaStream_t)stream);
    if (e != cudaSuccess) return hx::cuda_fail(e, "hx_fork_reduce: launch");
    return HX_OK;
}

}  // extern "C"
