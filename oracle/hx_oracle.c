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
