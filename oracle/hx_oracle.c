/*
 * hx_oracle.c -- sequential CPU oracle for the fork-join hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file: only the test-suite, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or constant with the CUDA
 * path.
 *
 * Semantics (Hercules paper, Sec. 3.3, "Representing Parallelism with
 * Fork-Joins"): a fork with factors (f0, f1, ...) spawns an n-D grid of
 * threads; a reduce node starts from its init value and folds one value per
 * thread, in increasing order of thread ID, with dimension 0 outermost.  Work
 * outside a reduction cycle is independent per thread.  Every nest below is
 * that rule written out as plain nested loops: the fork grid is walked in
 * lexicographic order and each reduction is a left fold in that order.  No
 * blocking, no reassociation, no fusion beyond what each definition states.
 *
 * Floating point: double precision unless a function says otherwise.  Build
 * with -ffp-contract=off so that a*b+c is two roundings exactly as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------------------
 * Map -> sum reduce.
 *
 * One fork of factor n.  Thread i computes out[i] = a*x[i] + y[i] (the map,
 * parallel), and a reduce node with init 0 folds s = s + out[i] for
 * i = 0, 1, ..., n-1 (Sec. 3.3 order).  Fusing the map into the reduce's
 * producer is the loop fusion of Sec. 5.1 (SRAD) and changes nothing here.
 *
 * out may be NULL (the map result is then only consumed by the reduce).
 */
void hxo_map_reduce_f64(const float *x, const float *y, double a, int64_t n,
                        double *out, double *sum)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double v = a * (double)x[i] + (double)y[i];
        if (out) out[i] = v;
        s = s + v;
    }
    *sum = s;
}

/* ---------------------------------------------------------------------------
 * Generic monoid reduce over one fork (the MonoidReduce attribute of
 * Sec. 3.4 licenses reassociating these; the oracle never does).
 *   op 0: sum  (init 0)        op 1: max  (init -inf)
 *   op 2: min  (init +inf)     op 3: product (init 1)
 * The map feeding it is out[i] = a*x[i] + y[i] as above (y may be NULL,
 * meaning 0).
 */
int hxo_monoid_reduce_f64(int op, const float *x, const float *y, double a,
                          int64_t n, double *result)
{
    double acc;
    switch (op) {
    case 0: acc = 0.0; break;
    case 1: acc = -INFINITY; break;
    case 2: acc = INFINITY; break;
    case 3: acc = 1.0; break;
    default: return 1;
    }
    for (int64_t i = 0; i < n; ++i) {
        double v = a * (double)x[i] + (y ? (double)y[i] : 0.0);
        switch (op) {
        case 0: acc = acc + v; break;
        case 1: acc = (v > acc) ? v : acc; break;
        case 2: acc = (v < acc) ? v : acc; break;
        case 3: acc = acc * v; break;
        }
    }
    *result = acc;
    return 0;
}

/* ---------------------------------------------------------------------------
 * 2-D 5-point Jacobi sweep with clamp-to-edge boundary, iterated.
 *
 * Grid u is row-major, ny rows by nx columns, u[i][j] at u[i*nx + j].
 * One iteration is a 2-D fork of factors (ny, nx).  Thread (i, j) computes
 *     u'[i][j] = 0.25 * ((u[i-1][j] + u[i+1][j]) + (u[i][j-1] + u[i][j+1]))
 * where a row index is clamped to [0, ny-1] and a column index to [0, nx-1],
 * and a max reduce (init 0) folds |u'[i][j] - u[i][j]| in lexicographic
 * (i, j) order into resid[t].  The iterations form a sequential outer loop
 * (its body carries u), the case Sec. 4.4 rule 1 keeps sequential.
 *
 * u_out receives the grid after `iters` iterations (u0 itself when
 * iters == 0).  Returns 0, or 1 when the scratch allocation fails.
 */
static int64_t clampi(int64_t v, int64_t lo, int64_t hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

int hxo_jacobi_f64(const double *u0, int32_t nx, int32_t ny, int32_t iters,
                   double *u_out, double *resid)
{
    size_t npts = (size_t)nx * (size_t)ny;
    double *cur = (double *)malloc(npts * sizeof(double));
    double *nxt = (double *)malloc(npts * sizeof(double));
    if (!cur || !nxt) { free(cur); free(nxt); return 1; }
    memcpy(cur, u0, npts * sizeof(double));
    for (int32_t t = 0; t < iters; ++t) {
        double r = 0.0;
        for (int64_t i = 0; i < ny; ++i) {
            for (int64_t j = 0; j < nx; ++j) {
                double north = cur[clampi(i - 1, 0, ny - 1) * nx + j];
                double south = cur[clampi(i + 1, 0, ny - 1) * nx + j];
                double west  = cur[i * nx + clampi(j - 1, 0, nx - 1)];
                double east  = cur[i * nx + clampi(j + 1, 0, nx - 1)];
                double v = 0.25 * ((north + south) + (west + east));
                nxt[i * nx + j] = v;
                double d = fabs(v - cur[i * nx + j]);
                r = (d > r) ? d : r;
            }
        }
        resid[t] = r;
        double *tmp = cur; cur = nxt; nxt = tmp;
    }
    memcpy(u_out, cur, npts * sizeof(double));
    free(cur);
    free(nxt);
    return 0;
}

/* Same nest evaluated in single precision, every operation rounded to fp32
 * in the order written above ((N+S)+(W+E), then *0.25, then |u'-u|). */
int hxo_jacobi_f32(const float *u0, int32_t nx, int32_t ny, int32_t iters,
                   float *u_out, float *resid)
{
    size_t npts = (size_t)nx * (size_t)ny;
    float *cur = (float *)malloc(npts * sizeof(float));
    float *nxt = (float *)malloc(npts * sizeof(float));
    if (!cur || !nxt) { free(cur); free(nxt); return 1; }
    memcpy(cur, u0, npts * sizeof(float));
    for (int32_t t = 0; t < iters; ++t) {
        float r = 0.0f;
        for (int64_t i = 0; i < ny; ++i) {
            for (int64_t j = 0; j < nx; ++j) {
                float north = cur[clampi(i - 1, 0, ny - 1) * nx + j];
                float south = cur[clampi(i + 1, 0, ny - 1) * nx + j];
                float west  = cur[i * nx + clampi(j - 1, 0, nx - 1)];
                float east  = cur[i * nx + clampi(j + 1, 0, nx - 1)];
                float ns = north + south;
                float we = west + east;
                float v = 0.25f * (ns + we);
                nxt[i * nx + j] = v;
                float d = fabsf(v - cur[i * nx + j]);
                r = (d > r) ? d : r;
            }
        }
        resid[t] = r;
        float *tmp = cur; cur = nxt; nxt = tmp;
    }
    memcpy(u_out, cur, npts * sizeof(float));
    free(cur);
    free(nxt);
    return 0;
}

/* ---------------------------------------------------------------------------
 * Byte histogram followed by an exclusive prefix sum over the bins.
 *
 * The histogram is a reduce over a 256-entry collection (Sec. 3.2
 * collections, Sec. 3.3 reduce): init all zeros (the implicit zero
 * initialisation of arrays, Sec. 2.1), then for i = 0..n-1 in order,
 * bins[v[i]] = bins[v[i]] + 1.  The scan is a second, sequential fold over
 * the bins: scan[0] = 0, scan[k] = scan[k-1] + bins[k-1].
 * Counts are uint32; callers keep n below 2^32.
 */
void hxo_histogram_u8(const uint8_t *v, int64_t n, uint32_t *bins,
                      uint32_t *excl_scan)
{
    for (int k = 0; k < 256; ++k) bins[k] = 0u;
    for (int64_t i = 0; i < n; ++i) bins[v[i]] = bins[v[i]] + 1u;
    if (excl_scan) {
        uint32_t run = 0u;
        for (int k = 0; k < 256; ++k) {
            excl_scan[k] = run;
            run = run + bins[k];
        }
    }
}

/* ---------------------------------------------------------------------------
 * Generic fork-join nest: a fork of up to three factors whose body is a small
 * straight-line map program, feeding a reduce over the innermost
 * `reduce_dims` fork dimensions under one of six monoids.
 *
 * Fork (Sec. 3.3): factors dims[0..ndim), dimension 0 outermost; thread
 * (i0, i1, i2) has the flat ID f = (i0*dims[1] + i1)*dims[2] + i2 (missing
 * dimensions dropped).  The outer m = ndim - reduce_dims dimensions index the
 * independent reductions ("segments"); the inner ones are folded.  With
 * O = dims[0]*...*dims[m-1] and I = dims[m]*...*dims[ndim-1], segment s holds
 * the threads s*I .. s*I + I - 1, and the reduce of segment s starts at the
 * monoid's identity and folds the segment's values for r = 0, 1, ..., I-1:
 * the increasing thread-ID order of Sec. 3.3.  reduce_dims == 0 means no
 * reduce: only the map values are produced.
 *
 * Map program: a postfix (stack) program over single-precision values, every
 * operation rounded to fp32 as IEEE 754 single does it (the C float
 * operators, sqrtf and fmaf are correctly rounded):
 *   1 IN k     push in[k][sum_d i_d*strides[k*3+d]]    (element strides)
 *   2 CONST k  push consts[k]
 *   3 INDEX d  push (float)i_d
 *   4 ADD  5 SUB  6 MUL  7 DIV    pop b, pop a, push a op b
 *   8 FMA      pop c, b, a, push fmaf(a, b, c) (one rounding)
 *   9 NEG  10 ABS  13 SQRT        pop a, push -a / fabsf(a) / sqrtf(a)
 *  11 MIN  12 MAX                 pop b, pop a, push the smaller / larger
 *                                 (a NaN operand yields the other one)
 * The program must leave exactly one value; the stack holds at most 8.
 *
 * Monoids (Sec. 3.4 MonoidReduce), folded left in thread-ID order:
 *   0 sum   acc = acc + v in double, init 0
 *   1 max   acc = v if v > acc, init -inf (NaN never taken; equal values keep
 *           the earlier one except that +0 replaces -0)
 *   2 min   acc = v if v < acc, init +inf (-0 replaces +0)
 *   3 prod  acc = acc * v in double, init 1
 *   4 argmax, 5 argmin: (value, index) of the first thread, in thread-ID
 *           order, whose value is the largest / smallest non-NaN value;
 *           index = r, the position inside the segment; init (-inf / +inf,
 *           -1), and index -1 remains when every value is NaN or I == 0.
 * result[s] is the folded value (sum and prod as double, the rest exactly
 * the fp32 value widened); result_index[s] the index for argmax / argmin.
 *
 * out (nullable) receives every thread's map value at its flat ID.  Returns 0,
 * or 1 for a malformed program or arguments.
 */
#define HXO_MAX_STACK 8

static int hxo_eval(int n_ops, const int32_t *ops, const float *consts,
                    const float *const *in, const int64_t *strides,
                    const int64_t *idx, int ndim, float *value)
{
    float st[HXO_MAX_STACK];
    int sp = 0;
    for (int k = 0; k < n_ops; ++k) {
        int code = ops[2 * k], arg = ops[2 * k + 1];
        float a, b, c;
        switch (code) {
        case 1: {
            int64_t off = 0;
            for (int d = 0; d < ndim; ++d) off += idx[d] * strides[arg * 3 + d];
            if (sp >= HXO_MAX_STACK) return 1;
            st[sp++] = in[arg][off];
            break;
        }
        case 2:
            if (sp >= HXO_MAX_STACK) return 1;
            st[sp++] = consts[arg];
            break;
        case 3:
            if (sp >= HXO_MAX_STACK || arg < 0 || arg >= ndim) return 1;
            st[sp++] = (float)idx[arg];
            break;
        case 4: case 5: case 6: case 7: case 11: case 12:
            if (sp < 2) return 1;
            b = st[--sp];
            a = st[--sp];
            if (code == 4) st[sp++] = a + b;
            else if (code == 5) st[sp++] = a - b;
            else if (code == 6) st[sp++] = a * b;
            else if (code == 7) st[sp++] = a / b;
            else if (code == 11) st[sp++] = isnan(a) ? b : (isnan(b) ? a : (b < a ? b : a));
            else st[sp++] = isnan(a) ? b : (isnan(b) ? a : (b > a ? b : a));
            break;
        case 8:
            if (sp < 3) return 1;
            c = st[--sp];
            b = st[--sp];
            a = st[--sp];
            st[sp++] = fmaf(a, b, c);
            break;
        case 9: case 10: case 13:
            if (sp < 1) return 1;
            a = st[--sp];
            st[sp++] = code == 9 ? -a : (code == 10 ? fabsf(a) : sqrtf(a));
            break;
        default:
            return 1;
        }
    }
    if (sp != 1) return 1;
    *value = st[0];
    return 0;
}

int hxo_fork_reduce(int ndim, const int64_t *dims, int reduce_dims, int monoid,
                    int n_ops, const int32_t *ops, const float *consts,
                    int n_in, const float *const *in, const int64_t *strides,
                    float *out, double *result, int64_t *result_index)
{
    if (ndim < 1 || ndim > 3 || reduce_dims < 0 || reduce_dims > ndim) return 1;
    if (reduce_dims > 0 && (monoid < 0 || monoid > 5 || !result)) return 1;
    if (reduce_dims > 0 && monoid >= 4 && !result_index) return 1;
    for (int d = 0; d < ndim; ++d)
        if (dims[d] < 0) return 1;
    /* the program must be well formed even when the fork is empty */
    int depth = 0;
    for (int k = 0; k < n_ops; ++k) {
        int code = ops[2 * k], arg = ops[2 * k + 1];
        if (code == 1 && (arg < 0 || arg >= n_in || !in[arg])) return 1;
        if (code == 2 && (arg < 0 || arg >= 8)) return 1;
        if (code == 3 && (arg < 0 || arg >= ndim)) return 1;
        if (code >= 1 && code <= 3) depth += 1;
        else if ((code >= 4 && code <= 7) || code == 11 || code == 12) depth -= 1;
        else if (code == 8) depth -= 2;
        else if (code != 9 && code != 10 && code != 13) return 1;
        if (depth < 1 || depth > HXO_MAX_STACK) return 1;
    }
    if (depth != 1) return 1;
    int m = ndim - reduce_dims;
    int64_t outer = 1, inner = 1;
    for (int d = 0; d < m; ++d) outer *= dims[d];
    for (int d = m; d < ndim; ++d) inner *= dims[d];
    for (int64_t s = 0; s < outer; ++s) {
        double acc = 0.0;
        float best = 0.0f;
        int64_t best_i = -1;
        switch (monoid) {
        case 0: acc = 0.0; break;
        case 1: case 4: best = -INFINITY; break;
        case 2: case 5: best = INFINITY; break;
        case 3: acc = 1.0; break;
        }
        for (int64_t r = 0; r < inner; ++r) {
            int64_t f = s * inner + r, rem = f, idx[3] = {0, 0, 0};
            for (int d = ndim - 1; d >= 0; --d) {
                idx[d] = rem % dims[d];
                rem /= dims[d];
            }
            float v;
            if (hxo_eval(n_ops, ops, consts, in, strides, idx, ndim, &v)) return 1;
            if (out) out[f] = v;
            if (reduce_dims == 0) continue;
            switch (monoid) {
            case 0: acc = acc + (double)v; break;
            case 3: acc = acc * (double)v; break;
            case 1:
                if (v > best || (v == 0.0f && best == 0.0f && signbit(best) && !signbit(v))) best = v;
                break;
            case 2:
                if (v < best || (v == 0.0f && best == 0.0f && !signbit(best) && signbit(v))) best = v;
                break;
            case 4:
                if (!isnan(v) && (best_i < 0 || v > best)) { best = v; best_i = r; }
                break;
            case 5:
                if (!isnan(v) && (best_i < 0 || v < best)) { best = v; best_i = r; }
                break;
            }
        }
        if (reduce_dims == 0) continue;
        result[s] = (monoid == 0 || monoid == 3) ? acc : (double)best;
        if (monoid >= 4) result_index[s] = best_i;
    }
    return 0;
}

/* ---------------------------------------------------------------------------
 * SRAD-style fused nest: speckle reducing anisotropic diffusion, iterated.
 *
 * The paper evaluates SRAD (Sec. 6), whose GPU schedule fuses two large loops
 * and turns a large sum reduction into a 3-layer reduction tree (Sec. 5.1,
 * Sec. 5.2).  It does not print SRAD's arithmetic; the steps below are the
 * published SRAD scheme (Yu and Acton, "Speckle reducing anisotropic
 * diffusion", IEEE TIP 2002), written as one outer sequential loop with
 * three fork-joins per iteration:
 *
 *  1. reduce: over the region of interest rows [r0, r1) x cols [c0, c1), in
 *     row-major order, S1 = sum J, S2 = sum J^2 (double); with N pixels,
 *     mean = S1/N, var = S2/N - mean^2, q0sq = var / mean^2 (the speckle
 *     scale of iteration t);
 *  2. fork over pixels: with clamp-to-edge neighbours and Jc = J[i][j],
 *     dN = J[i-1][j] - Jc, dS = J[i+1][j] - Jc, dW = J[i][j-1] - Jc,
 *     dE = J[i][j+1] - Jc,
 *     G2 = ((dN*dN + dS*dS) + (dW*dW + dE*dE)) / (Jc*Jc)
 *     L  = ((dN + dS) + (dW + dE)) / Jc
 *     num = 0.5*G2 - 0.0625*(L*L),  den = 1 + 0.25*L,  qsq = num / (den*den)
 *     c = 1 / (1 + (qsq - q0sq) / (q0sq * (1 + q0sq))), clamped to [0, 1]
 *     (a NaN c stays NaN);
 *  3. fork over pixels: D = (c[i][j]*dN + c[i+1][j]*dS) + (c[i][j]*dW +
 *     c[i][j+1]*dE) (neighbour indices clamped), J'[i][j] = Jc + (0.25*lambda)*D.
 *
 * Parity: conservation, symmetry, the maximum principle, the Jacobi limit,
 * the ROI statistics and a checkerboard closed form for qsq pin this nest;
 * the mapping from qsq to c is pinned by values worked by hand from the
 * published coefficient on checkerboard images with a separate region of
 * interest (the test suite's golden file for the SRAD coefficient).
 *
 * Intensities must be nonzero (the scheme divides by J); a homogeneous ROI
 * (q0sq == 0) makes the coefficient 0/0 and the result NaN, as the formula
 * says.  q0sq_out[t] receives iteration t's speckle scale.  The f32 variant
 * (below) evaluates the same expressions in single precision.
 * Returns 0, or 1 for bad arguments / failed scratch allocation.
 */
#define HXO_SRAD_BODY(T, HALF, SIXTEENTH, QUARTER, ONE, ZERO)                         \
    size_t npts = (size_t)nx * (size_t)ny;                                            \
    if (nx < 1 || ny < 1 || r0 < 0 || r1 > ny || r0 >= r1 || c0 < 0 || c1 > nx ||     \
        c0 >= c1 || iters < 0)                                                         \
        return 1;                                                                      \
    T *cur = (T *)malloc(npts * sizeof(T));                                           \
    T *nxt = (T *)malloc(npts * sizeof(T));                                           \
    T *cc = (T *)malloc(npts * sizeof(T));                                            \
    if (!cur || !nxt || !cc) { free(cur); free(nxt); free(cc); return 1; }            \
    memcpy(cur, J0, npts * sizeof(T));                                                \
    const T k = QUARTER * lambda;                                                     \
    for (int32_t t = 0; t < iters; ++t) {                                             \
        double s1 = 0.0, s2 = 0.0;                                                    \
        for (int64_t i = r0; i < r1; i++)                                             \
            for (int64_t j = c0; j < c1; ++j) {                                       \
                double v = (double)cur[i * nx + j];                                   \
                s1 = s1 + v;                                                          \
                s2 = s2 + v * v;                                                      \
            }                                                                         \
        double npix = (double)(r1 - r0) * (double)(c1 - c0);                          \
        double mean = s1 / npix;                                                      \
        double var = s2 / npix - mean * mean;                                         \
        const T q0sq = (T)(var / (mean * mean));                                      \
        q0sq_out[t] = q0sq;                                                           \
        for (int64_t i = 0; i < ny; ++i)                                              \
            for (int64_t j = 0; j < nx; ++j) {                                        \
                T Jc = cur[i * nx + j];                                               \
                T dN = cur[clampi(i - 1, 0, ny - 1) * nx + j] - Jc;                   \
                T dS = cur[clampi(i + 1, 0, ny - 1) * nx + j] - Jc;                   \
                T dW = cur[i * nx + clampi(j - 1, 0, nx - 1)] - Jc;                   \
                T dE = cur[i * nx + clampi(j + 1, 0, nx - 1)] - Jc;                   \
                T G2 = ((dN * dN + dS * dS) + (dW * dW + dE * dE)) / (Jc * Jc);       \
                T L = ((dN + dS) + (dW + dE)) / Jc;                                   \
                T num = HALF * G2 - SIXTEENTH * (L * L);                              \
                T den = ONE + QUARTER * L;                                            \
                T qsq = num / (den * den);                                            \
                T c = ONE / (ONE + (qsq - q0sq) / (q0sq * (ONE + q0sq)));             \
                if (c < ZERO) c = ZERO;                                               \
                else if (c > ONE) c = ONE;                                            \
                cc[i * nx + j] = c;                                                   \
            }                                                                         \
        for (int64_t i = 0; i < ny; ++i)                                              \
            for (int64_t j = 0; j < nx; ++j) {                                        \
                T Jc = cur[i * nx + j];                                               \
                int64_t is = clampi(i + 1, 0, ny - 1), je = clampi(j + 1, 0, nx - 1); \
                T dN = cur[clampi(i - 1, 0, ny - 1) * nx + j] - Jc;                   \
                T dS = cur[is * nx + j] - Jc;                                         \
                T dW = cur[i * nx + clampi(j - 1, 0, nx - 1)] - Jc;                   \
                T dE = cur[i * nx + je] - Jc;                                         \
                T cN = cc[i * nx + j], cS = cc[is * nx + j];                          \
                T cW = cc[i * nx + j], cE = cc[i * nx + je];                          \
                T D = (cN * dN + cS * dS) + (cW * dW + cE * dE);                      \
                nxt[i * nx + j] = Jc + k * D;                                         \
            }                                                                         \
        T *tmp = cur; cur = nxt; nxt = tmp;                                           \
    }                                                                                 \
    memcpy(J_out, cur, npts * sizeof(T));                                             \
    free(cur); free(nxt); free(cc);                                                   \
    return 0;

int hxo_srad_f64(const double *J0, int32_t nx, int32_t ny, int32_t iters, double lambda,
                 int32_t r0, int32_t r1, int32_t c0, int32_t c1, double *J_out, double *q0sq_out)
{
    HXO_SRAD_BODY(double, 0.5, 0.0625, 0.25, 1.0, 0.0)
}

/* Single precision: the same nest, literally, with every operation of steps
 * 2 and 3 rounded to fp32 in the order written above (five divisions per
 * pixel); the ROI statistics are the double sums of the fp32 values, and
 * q0sq is rounded to fp32 once. */
int hxo_srad_f32(const float *J0, int32_t nx, int32_t ny, int32_t iters, float lambda,
                 int32_t r0, int32_t r1, int32_t c0, int32_t c1, float *J_out, float *q0sq_out)
{
    HXO_SRAD_BODY(float, 0.5f, 0.0625f, 0.25f, 1.0f, 0.0f)
}
