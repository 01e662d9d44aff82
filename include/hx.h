/*
 * hx.h -- C ABI of libhx, the sm_103a (B300) implementation of the
 * data-parallel hot path that Hercules produces for fork-join loop nests
 * with associative reductions (Hercules paper, Sec. 3.3 fork-joins, Sec. 3.4
 * reduce attributes, Sec. 4.4 GPU lowering).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Pointers named d_* or documented as "device" are device pointers that
 *    the CALLER allocates and owns.  Nothing here frees or retains them
 *    beyond the call's stream work.
 *  - Every compute call is asynchronous on `stream` (a cudaStream_t; NULL is
 *    the legacy default stream).  Results are valid once that stream's work
 *    has completed.  Host-side argument checks happen before any launch.
 *  - A context (hx_ctx) owns the device workspace that the reductions need
 *    (per-tile partials, arrival tickets), allocated once by hx_create, the
 *    way a Hercules runner owns the backing memory of a call (Sec. 4.2 last
 *    paragraph, Sec. 4.6).  The workspace is split into per-stream slots:
 *    calls on the same stream share a slot (ordered by the stream), calls on
 *    different streams use different slots, up to HX_MAX_STREAMS streams per
 *    context.  A context is not thread-safe: serialise host calls on it.
 *  - Reductions are deterministic: the combination order is a function of
 *    the problem size and the context's tuning table alone (never of timing,
 *    grid size or batching), so a result is bit-identical across runs and
 *    between a standalone call and the same instance inside a batch planned
 *    on the same context.
 *  - Errors: every call returns an hx_status.  HX_ERR_INVALID = bad argument
 *    (nothing launched); HX_ERR_CUDA = a CUDA call failed; HX_ERR_NOMEM = a
 *    workspace, budget or capacity limit was exceeded.  hx_last_error()
 *    returns a message for the calling thread's last failure.  No C++
 *    exception crosses this boundary.
 */
#ifndef HX_H
#define HX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum hx_status {
    HX_OK = 0,
    HX_ERR_INVALID = 1,
    HX_ERR_CUDA = 2,
    HX_ERR_NOMEM = 3,
    HX_ERR_TIMEOUT = 4,
    HX_ERR_BUSY = 5
} hx_status;

typedef struct hx_ctx hx_ctx;
typedef struct CUstream_st *hx_stream_t; /* identical to cudaStream_t */

#define HX_MAX_STREAMS 16
/* Largest element count of one map->reduce instance (tile partials must fit
 * the per-stream workspace). */
#define HX_MAP_REDUCE_MAX_N ((int64_t)1 << 34)
/* Largest byte count of one histogram: counts are uint32. */
#define HX_HISTOGRAM_MAX_N ((int64_t)0xFFFFFFFF)

/* Library version, (major << 16) | minor. */
int hx_version(void);

/* Message for the calling thread's most recent failed call ("" if none). */
const char *hx_last_error(void);

/* Create a context on CUDA device `device`.  hbm_budget_bytes bounds the
 * device memory that batched and served work may hold resident (0 = no
 * limit).  Allocates the workspace (about 1 MiB) on that device.
 * Returns HX_ERR_INVALID for a bad device or NULL out. */
hx_status hx_create(hx_ctx **out, int device, size_t hbm_budget_bytes);

/* Release the context's workspace.  The caller must first make sure no
 * stream work issued through it is still running.  NULL is accepted. */
void hx_destroy(hx_ctx *ctx);

/* Test hook for failure handling without a GPU fault: of the calls on this
 * context that would launch device work (hx_map_reduce, hx_stencil2d,
 * hx_histogram, each round of a batch launch or served step,
 * hx_fork_reduce, hx_srad), the next `after` run normally and the `count`
 * after those fail with HX_ERR_CUDA ("injected launch failure") before
 * launching anything.  The context stays usable; a server fails every
 * request that had work in the failed step and recycles its workspace.
 * count == 0 clears the hook; negative arguments are HX_ERR_INVALID. */
hx_status hx_debug_inject_launch_failures(hx_ctx *ctx, int32_t after, int32_t count);

/* Device-side range checks (the library's debug build, libhx_debug.so,
 * compiled with HX_DEBUG_CHECKS).  Its kernels check the index ranges of
 * their work items (tile starts against n, partial indices against the
 * workspace, batch runs against their instance, stencil blocks against the
 * grid, ...) before using them; a failed check skips the work item (the
 * results are then wrong) and records its code and two values, the first
 * failure per kernel file only.  Nothing traps.  This call synchronises the
 * device, then reports and clears the records:
 *   enabled  1 in the debug build, 0 in the release build (whose kernels
 *            check nothing; code, a and b are then 0).
 *   code     0 when no check failed, else the first failure's code
 *            (1 map tile start, 2 map partial index, 3 map fold length,
 *            4 stencil block, 5 histogram split, 6 batch instance, 7 batch
 *            run, 8 batch stencil block, 9 SRAD region tile, 10 no-alloc
 *            tile, 11 nest chunk partial, 12 nest group partial, 13 nest
 *            arrival ticket) and the values it compared in a and b.
 * All pointers must be non-NULL (HX_ERR_INVALID otherwise). */
hx_status hx_debug_checks(int32_t *enabled, int32_t *code, int64_t *a, int64_t *b);

/* ------------------------------------------------------------------ map->reduce
 * One fork of factor n (Sec. 3.3): thread i computes
 *     out[i] = fmaf(a, x[i], y[i])            (one rounding, fp32)
 * and a sum reduce folds the out[i] into s.  The sum is reassociated as the
 * MonoidReduce attribute allows (Sec. 3.4) into the reduction tree of
 * Sec. 5.2: each tile of consecutive elements belongs to one warp and is
 * summed in a fixed order (each lane folds its own elements, then a fixed
 * shuffle butterfly), and a second launch on `stream`, chained by
 * programmatic dependent launch, folds the tile partials in a fixed order
 * (256 virtual lanes, each folding every 256th partial, then a butterfly;
 * the batched kernel folds an instance's partials in the same order, so an
 * instance gives the same bits alone and in a batch).  Partial sums are
 * carried as compensated
 * (hi, lo) pairs of fp32 numbers, about 48 significant bits.  The map and
 * the reduce are fused: out is written in the same pass (loop fusion,
 * Sec. 5.1).
 * Non-finite values: the pairs have fp32's exponent range.  A sum over
 * values that include +-inf is +-inf (NaN when both infinities or a NaN
 * occur), and a sum beyond fp32's range is +-inf in d_sum and in d_sum64
 * alike.  A running sum that overflows although the exact sum would come
 * back into range (cancellation after an overflow) is not defined.
 *
 *   x, y     device, n fp32 each, read-only.  Any alignment (16-byte
 *            aligned buffers take the vector path; results are identical).
 *   out      device, n fp32, or NULL to skip storing the map result.
 *   d_sum    device, 1 fp32: s rounded to fp32.  Required.
 *   d_sum64  device, 1 fp64: hi + lo of the final pair, or NULL.
 *   n        0 <= n <= HX_MAP_REDUCE_MAX_N; n == 0 gives s = 0.
 */
hx_status hx_map_reduce(hx_ctx *ctx, const float *x, const float *y, float *out,
                        float a, int64_t n, float *d_sum, double *d_sum64,
                        hx_stream_t stream);

/* ------------------------------------------------------------------ map->reduce, no allocation
 * The paper has no counterpart to this entry point; it exists for callers
 * that may not allocate device memory -- for example a plugin whose host
 * application owns all device memory through its own pool, or
 * latency-critical code that cannot afford cudaMalloc/cudaFree (which can
 * synchronise the device).  Such callers cannot use hx_create either,
 * because a context allocates its workspace.
 *
 * Computes exactly what hx_map_reduce computes with the built-in default
 * tuning table (same tile plan and fold order, so the same results; here
 * the warp that finishes last folds the tile partials, in one launch),
 * without a context and without allocating:
 * the reduction's scratch (HX_NOALLOC_MAX_TILES tile partials plus an
 * arrival ticket, about 33 KiB) is a static device array of this library,
 * held on every GPU that loads the library until the process exits.
 *   - Arguments, layout and alignment rules are those of hx_map_reduce;
 *     the caller still allocates and owns x, y, out, d_sum and d_sum64.
 *   - n must be in [0, HX_MAP_REDUCE_NOALLOC_MAX_N]; larger n returns
 *     HX_ERR_INVALID with a message.
 *   - Runs on the calling thread's current device.  The first call on a
 *     device looks up the scratch's device address (cudaGetSymbolAddress)
 *     and keeps it for the life of the process; make that first call
 *     before any stream capture begins.  cudaDeviceReset (or destroying
 *     and re-creating the device's primary context) unloads the library's
 *     device module and invalidates that address: after it, do not call
 *     this entry point on that device again in the same process.
 *   - Every call shares the one scratch array, which keeps the last call's
 *     contents; each call clears the arrival ticket on `stream` before its
 *     kernel.  Calls whose work overlaps on the GPU (different streams, or
 *     several host threads) race on the scratch and give wrong sums:
 *     serialise them.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine. */
#define HX_NOALLOC_MAX_TILES 4096
#define HX_MAP_REDUCE_NOALLOC_MAX_N ((int64_t)1 << 31)
hx_status hx_map_reduce_noalloc(const float *x, const float *y, float *out, float a, int64_t n,
                                float *d_sum, double *d_sum64, hx_stream_t stream);

/* ------------------------------------------------------------------ stencil
 * `iters` sweeps of the clamp-to-edge 5-point Jacobi update over a row-major
 * grid of ny rows by nx columns (element (i, j) at [i*nx + j]):
 *     u'[i][j] = 0.25f * ((u[i-1][j] + u[i+1][j]) + (u[i][j-1] + u[i][j+1]))
 * with out-of-range rows/columns clamped to the nearest edge, each rounded
 * in fp32 in exactly that order; fused with a max reduce of |u' - u| per
 * sweep (the max-gradient reduction of Sec. 5.2; max is exact, so the
 * residual is order independent).  Sweep t reads one buffer and writes the
 * other (u0 -> u1 -> u0 ...); sweeps are a sequential loop (Sec. 4.4 rule 1)
 * issued as back-to-back launches with programmatic dependent launch.
 *
 *   u0       device, nx*ny fp32: input grid; overwritten when iters >= 2.
 *   u1       device, nx*ny fp32: second buffer; must not overlap u0.
 *   d_resid  device, iters fp32: resid[t] = max |u_{t+1} - u_t|; may be NULL
 *            only when iters == 0.
 *   result_in_u1  host int32 out (may be NULL): 1 if the final grid is in
 *            u1 (iters odd), 0 if it is in u0.
 *   1 <= nx, ny <= 65536, nx*ny <= 2^31, 0 <= iters <= 1<<20.
 */
hx_status hx_stencil2d(hx_ctx *ctx, float *u0, float *u1, int32_t nx, int32_t ny,
                       int32_t iters, float *d_resid, int32_t *result_in_u1,
                       hx_stream_t stream);

/* ------------------------------------------------------------------ histogram
 * 256-bin byte histogram, a reduce over a 256-entry collection (Sec. 3.2
 * collections, Sec. 3.3 reduce; the per-thread private bins are what the
 * ParallelReduce/MonoidReduce attributes of Sec. 3.4 license), followed by
 * an exclusive prefix sum over the bins: scan[0] = 0,
 * scan[k] = bins[0] + ... + bins[k-1].  Integer and exact.
 *
 *   v            device, n bytes, any alignment.
 *   d_bins       device, 256 uint32 (overwritten, need not be zeroed).
 *   d_excl_scan  device, 256 uint32, or NULL to skip the scan.
 *   0 <= n <= HX_HISTOGRAM_MAX_N.
 */
hx_status hx_histogram(hx_ctx *ctx, const uint8_t *v, int64_t n, uint32_t *d_bins,
                       uint32_t *d_excl_scan, hx_stream_t stream);

/* ------------------------------------------------------------------ SRAD-style fused nest
 * Speckle reducing anisotropic diffusion, iterated: per iteration a reduce
 * (the speckle scale q0^2 = var/mean^2 of a region of interest) feeds two
 * stencil fork-joins (diffusion coefficient, then flux update).  The paper's
 * SRAD schedule fuses the two large loops (Sec. 5.1) and builds a GPU-only
 * reduction tree for the large sum (Sec. 5.2).  The arithmetic is the
 * published SRAD scheme; with clamp-to-edge neighbours and Jc = J[i][j]:
 *   dN = J[i-1][j]-Jc, dS = J[i+1][j]-Jc, dW = J[i][j-1]-Jc, dE = J[i][j+1]-Jc
 *   G2 = ((dN*dN + dS*dS) + (dW*dW + dE*dE)) / (Jc*Jc),
 *   L = ((dN + dS) + (dW + dE)) / Jc,
 *   qsq = (0.5*G2 - 0.0625*L*L) / ((1 + 0.25*L)^2),
 *   c = clamp(1 / (1 + (qsq - q0sq) / (q0sq*(1 + q0sq))), 0, 1),
 *   J' = Jc + (0.25*lambda) * ((c[i][j]*dN + c[i+1][j]*dS) + (c[i][j]*dW + c[i][j+1]*dE)),
 * in fp32 with the coefficient multiplied through by Jc^2 den^2, in which
 * Jc^2 cancels: with S1 = (dN + dS) + (dW + dE), S2 = the sum of the d^2,
 * E = Jc + 0.25*S1 (the mean of the four neighbours) and iq =
 * 1/(q0sq*(1 + q0sq)) once per iteration,
 *   c = clamp(E^2 / (E^2 + (0.5*S2 - 0.0625*S1^2 - q0sq*E^2) * iq), 0, 1),
 * each a*b + c of it and of the update one fused multiply-add:
 * algebraically the expression above, one division per pixel instead of
 * five, rounded differently.  For an image with values in [m, M] (diffusion
 * keeps every iterate there) and lambda <= 1, the result after T iterations
 * is within T * (1 + 0.25*lambda*(132 + 24*M/m)) * 2^-24 (at most 1e-5) of
 * M from an fp64 evaluation of the expression above, to first order.
 * q0sq is formed in double from float-float region sums (R1 = sum J,
 * R2 = sum J^2 over rows [r0, r1) x cols [c0, c1); mean = R1/N,
 * var = R2/N - mean^2) and rounded to fp32 once.
 *
 *   J0, J1   device, ny x nx fp32 row-major; J0 holds the input image
 *            (nonzero intensities: the scheme divides by J).  Iterations
 *            ping-pong J0 -> J1 -> J0 ...; *result_in_J1 (host, nullable)
 *            is 1 when the result is in J1 (iters odd).
 *   C        device scratch, ny x nx fp32, used by the unfused path only
 *            (may be NULL when fused != 0).
 *   d_q0sq   device, iters floats: the speckle scale each iteration used.
 *   fused    1: one kernel per iteration (coefficients recomputed in shared
 *            memory per tile, the next iteration's region sums accumulated by
 *            the same pass); 0: region reduce, coefficient and update as
 *            three kernels per iteration.  Both give bit-identical results.
 *   1 <= nx, ny <= 65536, nx*ny <= 2^31; the region must be non-empty and
 *   inside the image and span at most 65536 tiles of 32 x 128 pixels.
 * A homogeneous region (q0sq == 0) makes the coefficient 0/0: the image
 * becomes NaN, as the formula says. */
hx_status hx_srad(hx_ctx *ctx, float *J0, float *J1, float *C, int32_t nx, int32_t ny, int32_t iters,
                  float lambda, int32_t r0, int32_t r1, int32_t c0, int32_t c1, float *d_q0sq,
                  int32_t fused, int32_t *result_in_J1, hx_stream_t stream);

/* ------------------------------------------------------------------ generic nests
 * A fork-join nest in general form (Sec. 3.3): a fork of factors
 * dims[0..ndim) (dimension 0 outermost, 1 <= ndim <= 3) whose threads each
 * evaluate a small map program, and a reduce that folds the innermost
 * `reduce_dims` dimensions under a monoid (the MonoidReduce attribute of
 * Sec. 3.4).  Thread (i0, i1, i2) has flat ID f = (i0*dims[1] + i1)*dims[2]
 * + i2.  The outer ndim - reduce_dims dimensions index independent
 * "segments": with O = product of the outer factors and I = product of the
 * reduced ones, segment s is threads s*I .. s*I + I - 1 and yields one
 * result.  reduce_dims == 0 is a pure map (a fork with no reduce).
 *
 * The map program is postfix over single-precision values; every operation
 * rounds once to fp32 (IEEE add, sub, mul, div, sqrt, fma; no contraction):
 *   HX_OP_IN k     push in[k][sum_d i_d * strides[k][d]]  (element strides,
 *                  any sign; 0 broadcasts along that dimension)
 *   HX_OP_CONST k  push consts[k]          HX_OP_INDEX d  push (float)i_d
 *   HX_OP_ADD / SUB / MUL / DIV  pop b, pop a, push a op b
 *   HX_OP_FMA      pop c, b, a, push fmaf(a, b, c)
 *   HX_OP_NEG / ABS / SQRT       pop a, push -a, |a|, sqrt(a)
 *   HX_OP_MIN / MAX  pop b, pop a, push the smaller / larger (a NaN
 *                  operand yields the other operand)
 * At most 32 ops and 8 stack slots; the program must leave one value.
 *
 * Monoids (results per segment):
 *   SUM, PROD   float-float accumulation; result = the pair rounded to
 *               fp32, result64 = hi + lo in double.  Against an exact
 *               left fold the error is far below fp32 rounding.  The pair
 *               has fp32's exponent range: a segment holding +-inf gives
 *               +-inf (NaN when it holds both, or a NaN, or inf * 0), and a
 *               sum or product beyond fp32's range gives +-inf in result
 *               and in result64.  Partial results that leave fp32's range
 *               although the exact value would not (cancellation after an
 *               overflow) are not defined.
 *   MAX, MIN    exact; NaN values are skipped; +0 beats -0 for MAX and -0
 *               beats +0 for MIN; an empty segment gives -inf / +inf.
 *   ARGMAX, ARGMIN  the first thread (in thread-ID order) holding the
 *               largest / smallest non-NaN value: result = that value,
 *               result_index = its position r inside the segment (0..I-1);
 *               (-inf / +inf, -1) when the segment is empty or all NaN.
 * Every result is deterministic: the combination order depends only on the
 * sizes, the tree, the chunk, the tuning table and, for HX_TREE_WARP with
 * chunk 0, how many warps the device holds at once.  (A large reduction gets
 * longer chunks than the tuning table's: about 2.7 per resident warp for SUM,
 * one per resident warp for the other monoids.)
 *
 * Reduction schedule (`tree`), after the paper's reduction-tree schedule
 * (Sec. 5.2: chunk, reassociate the monoid, fission) and its lowering of
 * reductions to warp primitives (Sec. 4.4):
 *   HX_TREE_WARP   chunks of `chunk` elements per group of lanes, shuffle
 *                  butterfly inside the group, chunk partials combined by
 *                  the last group to arrive (default; chunk 0 = tuned).
 *   HX_TREE_CHUNK  one thread per contiguous chunk (default 64 elements),
 *                  sequential fold; the last thread folds the partials.
 *   HX_TREE_SEQ    one thread folds a whole segment (the loop as written).
 *
 * The library generates the kernel for a nest's shape (program, monoid,
 * tree, dimension split, addressing mode of each input) from its own
 * template and compiles it for sm_103a with NVRTC on first use (a fraction
 * of a second); kernels are cached for the life of the process.
 *
 *   in[k]      device float pointers (4-byte aligned) of the inputs the
 *              program reads; strides[k][d] in elements.
 *   out        device, O*I floats at flat IDs, or NULL; required when
 *              reduce_dims == 0.  It may alias an input only if both have
 *              the same layout.
 *   result     device, O floats (required when reduce_dims > 0).
 *   result64   device, O doubles, or NULL.
 *   result_index  device, O int64 (required for ARGMAX / ARGMIN).
 * A pointer the nest never touches may be NULL: inputs and out when the
 * fork has no threads, the results when it has no segments (O == 0).
 * Errors: HX_ERR_INVALID for a malformed descriptor (nothing launched);
 * HX_ERR_CUDA with the compiler log in hx_last_error() if the generated
 * kernel fails to compile.  O*I <= 2^60. */
#define HX_NEST_MAX_DIMS 3
#define HX_NEST_MAX_OPS 32
#define HX_NEST_MAX_INPUTS 4
#define HX_NEST_MAX_CONSTS 8
#define HX_NEST_MAX_STACK 8

typedef enum hx_nest_opcode {
    HX_OP_IN = 1, HX_OP_CONST = 2, HX_OP_INDEX = 3,
    HX_OP_ADD = 4, HX_OP_SUB = 5, HX_OP_MUL = 6, HX_OP_DIV = 7, HX_OP_FMA = 8,
    HX_OP_NEG = 9, HX_OP_ABS = 10, HX_OP_MIN = 11, HX_OP_MAX = 12, HX_OP_SQRT = 13
} hx_nest_opcode;

typedef enum hx_monoid {
    HX_MONOID_SUM = 0, HX_MONOID_MAX = 1, HX_MONOID_MIN = 2, HX_MONOID_PROD = 3,
    HX_MONOID_ARGMAX = 4, HX_MONOID_ARGMIN = 5
} hx_monoid;

typedef enum hx_tree { HX_TREE_WARP = 0, HX_TREE_CHUNK = 1, HX_TREE_SEQ = 2 } hx_tree;

typedef struct hx_nest_op {
    int32_t code;   /* hx_nest_opcode */
    int32_t arg;    /* input slot, constant slot or dimension */
} hx_nest_op;

typedef struct hx_nest {
    int32_t ndim;
    int32_t reduce_dims;
    int32_t monoid;                 /* hx_monoid, ignored when reduce_dims == 0 */
    int32_t tree;                   /* hx_tree */
    int64_t dims[HX_NEST_MAX_DIMS];
    int64_t chunk;                  /* elements per chunk, 0 = default / tuned */
    int32_t n_ops;
    int32_t pad_;
    hx_nest_op ops[HX_NEST_MAX_OPS];
    float consts[HX_NEST_MAX_CONSTS];
    const float *in[HX_NEST_MAX_INPUTS];
    int64_t strides[HX_NEST_MAX_INPUTS][HX_NEST_MAX_DIMS];
    float *out;
    float *result;
    double *result64;
    int64_t *result_index;
} hx_nest;

/* Run the nest on `stream` (asynchronous; uses the stream's workspace slot). */
hx_status hx_fork_reduce(hx_ctx *ctx, const hx_nest *nest, hx_stream_t stream);

/* Validate the nest and compile its kernel now (no device needed), so that
 * the first hx_fork_reduce does not pay for compilation. */
hx_status hx_nest_prepare(const hx_nest *nest);

/* The CUDA source generated for the nest's shape (for inspection): copies
 * at most cap-1 bytes plus a terminating NUL into buf (if buf and cap are
 * non-zero) and stores the full length in *len (if len is non-NULL). */
hx_status hx_nest_source(const hx_nest *nest, char *buf, size_t cap, size_t *len);

/* ------------------------------------------------------------------ tuning
 * The paper leaves tile, chunk and vector choices to a hand-written schedule
 * per target (Sec. 2.2: fork-chunk, fork-tile, fork-reshape; Sec. 5.2: the
 * reduction-tree and multicore schedules).  Here an autotuner measures the
 * candidates on the device and keeps, per size class, the fastest:
 *   map_vecs[c]      float4 vectors per lane in one map->reduce tile, for
 *                    n in class c (a multiple of 4; raised automatically so
 *                    that an instance never has more than 4096 tiles).  This
 *                    choice fixes the summation tree, so it changes the sum's
 *                    rounding (still within tolerance, still deterministic);
 *                    a standalone call and a batch planned with the same
 *                    table give identical results.
 *   hist_threads[c]  histogram CTA width (256, 512 or 1024), n in class c.
 *   stencil_rows[c]  rows per warp block of a standalone sweep (4, 8 or
 *                    16), class of nx*ny; results do not depend on it.
 *   nest_lane_elems[c]  elements per lane of one warp-tree chunk of a
 *                    generic nest whose segments hold n elements, n in class
 *                    c (a multiple of 8 in [8, 512]; raised automatically so
 *                    that a nest never needs more than 65536 chunk partials).
 *                    Like map_vecs it fixes the summation tree.
 *   batch_map_run, batch_stencil_run: tiles per warp run in batches.
 * Size class c holds sizes in [2^c, 2^(c+1)); sizes 0 and 1 are class 0.
 * A context starts from the built-in defaults, or from the JSON file named
 * by the environment variable HX_TUNE_FILE when it is set. */
#define HX_TUNE_CLASSES 40
typedef struct hx_tune_table {
    int32_t map_vecs[HX_TUNE_CLASSES];
    int32_t hist_threads[HX_TUNE_CLASSES];
    int32_t stencil_rows[HX_TUNE_CLASSES];
    int32_t nest_lane_elems[HX_TUNE_CLASSES];
    int32_t batch_map_run;
    int32_t batch_stencil_run;
} hx_tune_table;

/* Built-in defaults (host only, no device needed). */
void hx_tune_table_default(hx_tune_table *t);
/* HX_OK if every entry is one of the allowed values, else HX_ERR_INVALID. */
hx_status hx_tune_table_check(const hx_tune_table *t);
/* Write / read a table as JSON (host only).  Read validates the result. */
hx_status hx_tune_table_save(const hx_tune_table *t, const char *path);
hx_status hx_tune_table_load(hx_tune_table *t, const char *path);

/* Copy the context's table out / replace it (validated).  Batches planned
 * earlier keep the plans they were made with. */
hx_status hx_tune_get(const hx_ctx *ctx, hx_tune_table *out);
hx_status hx_tune_set(hx_ctx *ctx, const hx_tune_table *t);

/* Measure the candidates for every size class up to 2^max_log2 elements
 * (10 <= max_log2 <= 30) on this context's device and store the fastest in
 * the context's table.  Allocates and frees about 3.5 GiB of temporary
 * device memory, synchronises `stream`, takes a few seconds. */
hx_status hx_autotune(hx_ctx *ctx, int32_t max_log2, hx_stream_t stream);

/* ------------------------------------------------------------------ batches
 * Many independent nest instances in one persistent launch.  The Hercules
 * host backend runs independent calls and the iterations of parallel
 * fork-joins as concurrent tasks (Sec. 4.5, the AsyncCall attribute of
 * Sec. 3.4); here the instances become one device work-list of
 * (instance, tile) items that resident CTAs pull from an atomic counter.
 * Every item runs the same tile code as the standalone calls above and the
 * tile plan of an instance depends only on its own sizes, so each result is
 * bit-identical to the standalone call's.  Work items only store partial
 * results; a second launch chained after the batched one runs the final
 * combine of every instance the launch completed (no CTA ever waits for
 * another).
 *
 * A stencil task with iters > 1 runs all its sweeps inside the same
 * persistent launch (the sequential outer loop of Sec. 4.4 rule 1 kept on
 * the device): a block of sweep s of an instance waits until it and its
 * north, south, west and east neighbouring blocks have finished sweep s - 1,
 * so an instance's sweeps overlap as a wavefront.  Items are taken in an
 * order in which every wait is for items already taken, and the launch never
 * has more CTAs than the device holds at once, so every wait ends; each
 * wait is also
 * bounded in time (1 s): if one runs out, the launch records HX_ERR_TIMEOUT
 * (hx_batch_status, hx_batch_query) and its results are not valid.  With
 * HX_BATCH_ROUNDS, above 255 sweeps, or by default when the stencil tasks
 * with iters > 1 move more than 512 MiB per sweep (8 bytes per grid point),
 * the plan runs as rounds instead:
 * round r runs sweep r of every stencil instance that has one (plus, in
 * round 0, all map->reduce and histogram instances), one launch per round.
 *
 * Pointer, size and alignment rules of each task kind are those of the
 * matching standalone call.  Instances of one batch must not write
 * overlapping memory.  An instance's sweep count is capped at 4096. */
typedef enum hx_task_kind {
    HX_TASK_MAP_REDUCE = 0,
    HX_TASK_STENCIL2D = 1,
    HX_TASK_HISTOGRAM = 2
} hx_task_kind;

typedef struct hx_task {
    int32_t kind; /* hx_task_kind */
    int32_t reserved;
    union {
        struct { const float *x; const float *y; float *out; float *sum; double *sum64;
                 float a; int32_t pad; int64_t n; } mr;          /* out, sum64 nullable */
        struct { float *u0; float *u1; float *resid;
                 int32_t nx; int32_t ny; int32_t iters; int32_t pad; } st;
        struct { const uint8_t *v; uint32_t *bins; uint32_t *scan; int64_t n; } hi; /* scan nullable */
    } u;
} hx_task;

typedef struct hx_batch hx_batch;

/* Validate `tasks` and build their device work-list and workspace
 * (allocates device memory; must not be called during stream capture).
 * The tasks' buffers are bound to the plan: launching it again re-runs the
 * same instances on the same buffers.  *out_rounds (nullable) receives the
 * number of launches one hx_batch_launch issues. */
hx_status hx_batch_plan(hx_ctx *ctx, const hx_task *tasks, int32_t n_tasks, hx_batch **out,
                        int32_t *out_rounds);

/* hx_batch_plan with flags: 0 (the default schedule: every sweep in one
 * launch when the stencil tasks with iters > 1 move at most 512 MiB per
 * sweep, else rounds),
 * HX_BATCH_ROUNDS (one launch per sweep) or HX_BATCH_ONE_LAUNCH (every sweep
 * in one launch, whatever the task count; at most 255 sweeps).  All give the
 * same results; HX_ERR_INVALID for unknown or conflicting flags. */
#define HX_BATCH_ROUNDS 1
#define HX_BATCH_ONE_LAUNCH 2
hx_status hx_batch_plan_ex(hx_ctx *ctx, const hx_task *tasks, int32_t n_tasks, int32_t flags, hx_batch **out,
                           int32_t *out_rounds);

/* Run a planned batch on `stream`: one persistent launch per round, no host
 * synchronisation, no allocation (may be captured in a CUDA graph).  A plan
 * must not run on two streams at once. */
hx_status hx_batch_launch(hx_batch *batch, hx_stream_t stream);

/* Free a plan.  Its launches must have completed. */
void hx_batch_free(hx_batch *batch);

/* A text description of a plan, one line per instance: its kind and sizes,
 * tile plan or blocks per sweep, run length, load path and schedule (a
 * stand-in for the IR debugger of the paper's tool chain, which draws its
 * programs as graphs).  Writes at most len bytes including the terminating
 * NUL (buf may be NULL when len is 0); *needed (nullable) receives the size
 * the whole text needs.  Setting the environment variable HX_DUMP_PLAN=1
 * prints every new plan's description to stderr.  Host only. */
hx_status hx_batch_describe(const hx_batch *batch, char *buf, size_t len, size_t *needed);

/* After the plan's launches have completed (the caller synchronised their
 * stream): HX_ERR_TIMEOUT if a wait between two sweeps of an instance ran
 * out of time in any of them since the last call (their results are then not
 * valid), else HX_OK.  Reads and clears a word of host memory; no CUDA call. */
hx_status hx_batch_status(hx_batch *batch);

/* Test hook for the bounded waits, without a GPU fault: the waits of task
 * `task`'s later sweeps can never be satisfied (they expect one block more
 * than the sweep has), and every wait of the plan gives up after
 * wait_limit_ns nanoseconds instead of 1 s.  A launch of the plan then ends
 * by itself with HX_ERR_TIMEOUT recorded.  Meant for a plan whose task
 * `task` is a stencil with iters > 1; other plans are unaffected.  Returns
 * HX_ERR_INVALID for a bad task index or a negative limit. */
hx_status hx_debug_batch_stall(hx_batch *batch, int32_t task, int64_t wait_limit_ns);

/* Plan, launch on `stream` and record completion in one call; *ticket_out
 * identifies the submission for hx_batch_query.  The plan is released when
 * a query sees it complete (or at hx_destroy). */
hx_status hx_batch_submit(hx_ctx *ctx, const hx_task *tasks, int32_t n_tasks, hx_stream_t stream,
                          uint64_t *ticket_out);

/* HX_OK when the submission's device work has completed, HX_ERR_BUSY while
 * it is pending, HX_ERR_INVALID for an unknown ticket (including one already
 * reported complete), HX_ERR_TIMEOUT when it completed but a wait between
 * sweeps ran out of time (see hx_batch_status). */
hx_status hx_batch_query(hx_ctx *ctx, uint64_t ticket);

/* ------------------------------------------------------------------ serving
 * A request loop over the same nests.  Requests (hx_task, buffers already
 * on the device) arrive at any time; the server admits them in arrival order
 * while the summed device footprint of admitted, unfinished requests stays
 * within a budget (the footprint is a closed form of the request's sizes,
 * as Hercules sizes a call's backing memory from its dynamic constants,
 * Sec. 4.2 and 4.6), and runs them in one of two modes:
 *
 *   HX_SERVE_CONTINUOUS  continuous batching: a scheduler thread repeatedly
 *       forms a step out of every admitted request's next slice of work (up
 *       to step_quantum_bytes of tiles of a map->reduce or histogram, or of
 *       the current sweep of a stencil) and runs the step as one launch of
 *       the batched kernel (plus its final-combine launch); up to
 *       max_steps_in_flight steps are queued on the device, so requests that
 *       arrive while a step runs join the next one and their work overlaps
 *       with the requests already running.  At low load -- at most
 *       direct_max requests waiting, none started -- each of them is issued
 *       as its standalone call instead (no step to build and upload).  Each
 *       request computes exactly what its standalone call computes (same
 *       tile plans, same device code), so its results do not depend on what
 *       it was batched with or on which path it took.
 *   HX_SERVE_PER_LAUNCH  the baseline: every admitted request is issued as
 *       its own standalone call(s), in arrival order, on one stream.
 *
 * A completion thread watches the device and retires each request when the
 * launch carrying its last piece of work has finished; latency = completion
 * time - arrival time (host steady clock).  While a server runs, its context
 * must not be used from other threads.  The caller keeps every request's
 * buffers alive and untouched until the request completes. */
typedef enum hx_serve_mode { HX_SERVE_CONTINUOUS = 0, HX_SERVE_PER_LAUNCH = 1 } hx_serve_mode;

/* Completion callback: called once per request, from the server's completion
 * thread and without the server's lock held (it may call hx_server_poll or
 * hx_server_submit), after the request has completed (status HX_OK) or
 * failed (HX_ERR_CUDA); latency_s as hx_server_poll reports it (for a
 * failed request, the time until it failed).  Callbacks run in completion
 * order, one at a time; a callback must not call hx_server_drain,
 * hx_server_run_trace or hx_server_destroy. */
typedef void (*hx_server_done_fn)(void *user, uint64_t req_id, hx_status status, double latency_s);

typedef struct hx_server_config {
    int32_t mode;                 /* hx_serve_mode */
    int32_t max_inflight;         /* admitted, unfinished requests at most (0: 4096; at most 16384;
                                   * continuous mode keeps 49 KiB of device workspace per slot) */
    size_t hbm_budget_bytes;      /* admission budget (0: the context's budget; 0 there too: unlimited).
                                   * A request larger than the budget is admitted only when nothing else
                                   * is in flight. */
    int32_t max_steps_in_flight;  /* continuous mode: steps queued on the device (0: 4) */
    int32_t max_step_requests;    /* continuous mode: requests per step at most (0: 4096) */
    size_t step_quantum_bytes;    /* continuous mode: each step aims at step_target_bytes of traffic
                                   * shared by its requests; a request's slice is that share, but at
                                   * least step_quantum_bytes (0: 32 MiB).  Larger requests are spread
                                   * over several steps. */
    size_t step_target_bytes;     /* continuous mode (0: 512 MiB) */
    hx_server_done_fn on_done;    /* completion callback, or NULL */
    void *on_done_user;           /* passed to on_done */
    int32_t direct_max;           /* continuous mode: when at most this many admitted requests are
                                   * waiting to start and none has started, each runs as its own
                                   * standalone call instead of a batched step -- the shorter path at
                                   * low load (0: 4; -1: always batch; at most 65536) */
    int64_t direct_sweep_bytes;   /* continuous mode: a stencil request that has not started and whose
                                   * sweep moves at least this many bytes (8 per grid point) runs as its
                                   * standalone call even while other requests wait.  Its sweeps are
                                   * large enough to fill the device alone, and in batched steps it
                                   * would advance one sweep per step.  (0: 16 MiB; -1: never) */
    int32_t max_step_sweeps;      /* continuous mode: a stencil request at a sweep boundary whose sweep
                                   * moves less than direct_sweep_bytes (16 MiB when that is -1) runs up
                                   * to this many of its remaining sweeps inside one batched step, one
                                   * after another on the device (0: 128, the most; 1: one sweep per
                                   * step) */
    int32_t pad_;
} hx_server_config;

typedef struct hx_server_stats {
    int64_t submitted, admitted, completed;
    int64_t launches;             /* batched steps (continuous) or request launches (per-launch) */
    int64_t failed;               /* requests whose launch failed */
    size_t footprint_in_flight;   /* bytes currently admitted */
    size_t peak_footprint;        /* most bytes admitted at once */
} hx_server_stats;

typedef struct hx_server hx_server;

/* Start a server (its threads, its stream and, in continuous mode, one
 * descriptor staging buffer per queued step plus 49 KiB of workspace per
 * in-flight slot) on ctx's device. */
hx_status hx_server_create(hx_ctx *ctx, const hx_server_config *cfg, hx_server **out);

/* Wait for in-flight work, stop the threads, free the server. */
void hx_server_destroy(hx_server *s);

/* Submit one request now (thread-safe).  The task is validated as its
 * standalone call would be; *req_id identifies it for hx_server_poll. */
hx_status hx_server_submit(hx_server *s, const hx_task *task, uint64_t *req_id);

/* HX_OK when the request has completed (its latency in *latency_s, may be
 * NULL), HX_ERR_BUSY while pending, HX_ERR_CUDA if its launch failed,
 * HX_ERR_INVALID for an unknown id. */
hx_status hx_server_poll(hx_server *s, uint64_t req_id, double *latency_s);

/* The server's timeline (no profiler needed): one record per step it issued
 * -- a batched step, or a request's standalone call (low-load path and
 * per-launch mode) -- for the first 65536 steps, in issue order.  Times are
 * seconds since hx_server_create: when the step was issued, and when the
 * completion thread saw it finish (-1 while pending).  Copies at most max
 * records into out; *n receives how many there are. */
typedef struct hx_server_step_record {
    double issue_s;
    double done_s;
    int32_t requests;   /* requests with work (or an output) in the step */
    int32_t direct;     /* 1: one request's standalone call; 0: a batched step */
} hx_server_step_record;
hx_status hx_server_get_timeline(hx_server *s, hx_server_step_record *out, int32_t max, int32_t *n);

/* Test hook (continuous mode): the next batched step that runs several
 * sweeps of a request gets one such request whose waits between sweeps can
 * never be satisfied, and every wait of that step gives up after
 * wait_limit_ns nanoseconds.  The step ends by itself; every request with
 * work in it completes with HX_ERR_TIMEOUT (hx_server_poll), and
 * hx_server_drain reports the failure.  One-shot.  HX_ERR_INVALID for a
 * negative limit or a per-launch server. */
hx_status hx_debug_server_stall(hx_server *s, int64_t wait_limit_ns);

/* Block until every submitted request has completed (and, with on_done,
 * been reported), at most timeout_s seconds (HX_ERR_TIMEOUT otherwise).  HX_ERR_CUDA when a request completed
 * with a failed launch since the previous drain returned (hx_server_poll
 * tells which); HX_OK otherwise. */
hx_status hx_server_drain(hx_server *s, double timeout_s);

hx_status hx_server_get_stats(hx_server *s, hx_server_stats *out);

/* Open-loop replay: submit tasks[i] at start + arrival_s[i] (arrival_s
 * non-decreasing, seconds), pacing from the calling thread, then drain.
 * latency_s[i] (required) = completion - scheduled arrival of request i;
 * *makespan_s (nullable) = last completion - start.  Fails with
 * HX_ERR_TIMEOUT if the requests have not completed timeout_s seconds after
 * the last arrival. */
hx_status hx_server_run_trace(hx_server *s, const hx_task *tasks, const double *arrival_s, int32_t n,
                              double timeout_s, double *latency_s, double *makespan_s);

#ifdef __cplusplus
}
#endif
#endif /* HX_H */
