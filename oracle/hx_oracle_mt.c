/*
 * hx_oracle_mt.c -- TEST AND BENCHMARK INFRASTRUCTURE ONLY.
 *
 * The host (multicore) schedule of three of the oracle's nests, timed by the
 * benchmark as context for the single-thread oracle: the fork is split into
 * T contiguous chunks, one POSIX thread per chunk (the fork-chunk of
 * Sec. 2.2 run by the host backend's concurrent tasks, Sec. 4.5), and each
 * reduce is reassociated per chunk (monoid-reassociate, Sec. 5.2): chunk
 * partials start from the identity and are folded in chunk order at the
 * join.  Integer and max reductions give the sequential oracle's results
 * exactly; the fp64 sum differs from the sequential fold only by rounding.
 *
 * Nothing here is used to check the GPU: parity is against hx_oracle.c.
 * The tests compare these functions with the sequential oracle.
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define HXO_MT_MAX_THREADS 256

static int64_t chunk_lo(int64_t n, int t, int T) { return n * t / T; }

/* ------------------------------------------------------------ map->reduce */
typedef struct {
    const float *x, *y;
    double a, *out, sum;
    int64_t lo, hi;
} mr_job;

static void *mr_run(void *arg)
{
    mr_job *j = (mr_job *)arg;
    double s = 0.0;
    for (int64_t i = j->lo; i < j->hi; ++i) {
        double v = j->a * (double)j->x[i] + (double)j->y[i];
        if (j->out) j->out[i] = v;
        s = s + v;
    }
    j->sum = s;
    return NULL;
}

/* out[i] = a*x[i] + y[i] (fp64; out may be NULL), *sum = the chunk sums of
 * T contiguous chunks folded in chunk order.  Returns 0, or 1 on a bad
 * thread count or a failed thread start. */
int hxo_mt_map_reduce_f64(const float *x, const float *y, double a, int64_t n, double *out, double *sum,
                          int threads)
{
    if (threads < 1 || threads > HXO_MT_MAX_THREADS || n < 0) return 1;
    mr_job jobs[HXO_MT_MAX_THREADS];
    pthread_t tid[HXO_MT_MAX_THREADS];
    int started = 0, rc = 0;
    for (int t = 0; t < threads; ++t) {
        jobs[t] = (mr_job){x, y, a, out, 0.0, chunk_lo(n, t, threads), chunk_lo(n, t + 1, threads)};
        if (pthread_create(&tid[t], NULL, mr_run, &jobs[t]) != 0) { rc = 1; break; }
        ++started;
    }
    for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    if (rc) return rc;
    double s = 0.0;
    for (int t = 0; t < threads; ++t) s = s + jobs[t].sum;
    *sum = s;
    return 0;
}

/* ------------------------------------------------------------ histogram */
typedef struct {
    const uint8_t *v;
    int64_t lo, hi;
    uint32_t bins[256];
} hi_job;

static void *hi_run(void *arg)
{
    hi_job *j = (hi_job *)arg;
    memset(j->bins, 0, sizeof j->bins);
    for (int64_t i = j->lo; i < j->hi; ++i) j->bins[j->v[i]] += 1u;
    return NULL;
}

/* Bins of the bytes of v (per-chunk bins added at the join) and their
 * exclusive scan (excl_scan may be NULL).  Returns 0 or 1 as above. */
int hxo_mt_histogram_u8(const uint8_t *v, int64_t n, uint32_t *bins, uint32_t *excl_scan, int threads)
{
    if (threads < 1 || threads > HXO_MT_MAX_THREADS || n < 0) return 1;
    hi_job *jobs = (hi_job *)malloc(sizeof(hi_job) * (size_t)threads);
    if (!jobs) return 1;
    pthread_t tid[HXO_MT_MAX_THREADS];
    int started = 0, rc = 0;
    for (int t = 0; t < threads; ++t) {
        jobs[t].v = v;
        jobs[t].lo = chunk_lo(n, t, threads);
        jobs[t].hi = chunk_lo(n, t + 1, threads);
        if (pthread_create(&tid[t], NULL, hi_run, &jobs[t]) != 0) { rc = 1; break; }
        ++started;
    }
    for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    if (!rc) {
        for (int k = 0; k < 256; ++k) {
            uint32_t c = 0u;
            for (int t = 0; t < threads; ++t) c += jobs[t].bins[k];
            bins[k] = c;
        }
        if (excl_scan) {
            uint32_t run = 0u;
            for (int k = 0; k < 256; ++k) {
                excl_scan[k] = run;
                run += bins[k];
            }
        }
    }
    free(jobs);
    return rc;
}

/* ------------------------------------------------------------ Jacobi */
typedef struct {
    const double *cur;
    double *nxt;
    int64_t nx, ny, lo, hi;
    double resid;                  /* this slab's maximum |u' - u| */
} st_job;

static int64_t clampi(int64_t v, int64_t lo, int64_t hi) { return v < lo ? lo : (v > hi ? hi : v); }

static void *st_run(void *arg)
{
    st_job *j = (st_job *)arg;
    const int64_t nx = j->nx, ny = j->ny;
    const double *cur = j->cur;
    double r = 0.0;
    for (int64_t i = j->lo; i < j->hi; ++i) {
        for (int64_t c = 0; c < nx; ++c) {
            double north = cur[clampi(i - 1, 0, ny - 1) * nx + c];
            double south = cur[clampi(i + 1, 0, ny - 1) * nx + c];
            double west = cur[i * nx + clampi(c - 1, 0, nx - 1)];
            double east = cur[i * nx + clampi(c + 1, 0, nx - 1)];
            double v = 0.25 * ((north + south) + (west + east));
            j->nxt[i * nx + c] = v;
            double d = fabs(v - cur[i * nx + c]);
            r = (d > r) ? d : r;
        }
    }
    j->resid = r;
    return NULL;
}

/* The clamp-to-edge Jacobi sweeps of hxo_jacobi_f64, each sweep a fork of
 * T threads over contiguous row slabs joined before the next sweep; the
 * residual of a sweep is the maximum of the slabs' maxima (exact).
 * Returns 0, or 1 on a bad argument or a failed allocation or thread
 * start. */
int hxo_mt_jacobi_f64(const double *u0, int32_t nx, int32_t ny, int32_t iters, double *u_out, double *resid,
                      int threads)
{
    if (threads < 1 || threads > HXO_MT_MAX_THREADS || nx < 1 || ny < 1 || iters < 0) return 1;
    if (threads > ny) threads = ny;
    size_t npts = (size_t)nx * (size_t)ny;
    double *cur = (double *)malloc(npts * sizeof(double));
    double *nxt = (double *)malloc(npts * sizeof(double));
    if (!cur || !nxt) { free(cur); free(nxt); return 1; }
    memcpy(cur, u0, npts * sizeof(double));
    st_job jobs[HXO_MT_MAX_THREADS];
    pthread_t tid[HXO_MT_MAX_THREADS];
    int rc = 0;
    for (int32_t t = 0; t < iters && !rc; ++t) {
        int started = 0;
        for (int k = 0; k < threads; ++k) {
            jobs[k] = (st_job){cur, nxt, nx, ny, chunk_lo(ny, k, threads), chunk_lo(ny, k + 1, threads), 0.0};
            if (pthread_create(&tid[k], NULL, st_run, &jobs[k]) != 0) { rc = 1; break; }
            ++started;
        }
        for (int k = 0; k < started; ++k) pthread_join(tid[k], NULL);
        if (rc) break;
        double r = 0.0;
        for (int k = 0; k < threads; ++k) r = jobs[k].resid > r ? jobs[k].resid : r;
        resid[t] = r;
        double *tmp = cur; cur = nxt; nxt = tmp;
    }
    if (!rc) memcpy(u_out, cur, npts * sizeof(double));
    free(cur);
    free(nxt);
    return rc;
}
