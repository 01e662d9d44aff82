// hx_srad.cu -- the SRAD-style fused nest: speckle reducing anisotropic
// diffusion, iterated.  Each iteration is a global reduce (the speckle scale
// q0^2 of a region of interest) feeding two stencil fork-joins (the
// diffusion coefficient c, then the flux update of the image).  The paper's
// SRAD schedule fuses the two large loops to remove global-memory traffic
// (Sec. 5.1) and turns the large sum into a GPU-only reduction tree
// (Sec. 5.2).  Here:
//
//   fused (one kernel per iteration): a CTA loads its 32 x 128 output tile
//   of J plus a halo into shared memory, computes c for the tile and one
//   extra row and column (the south / east neighbours' coefficients) into
//   shared memory, writes J', and accumulates the region-of-interest sums of
//   J' (float-float) for the NEXT iteration's q0^2 -- the reduce is fused
//   into the loop that produces its input.  Tile partials are combined by
//   the last region tile to arrive, in tile order; it writes q0^2[t+1].
//   HBM traffic: J read once (halo rows come from L2) and J' written once.
//
//   unfused (three kernels per iteration, the loop nest as written):
//   region reduce -> q0^2[t], coefficient kernel (J -> C), update kernel
//   (J, C -> J').
//
// Both evaluate every expression in single precision in one fixed order (no
// contraction), so the two paths give bit-identical images; q0^2 is formed
// in double from the float-float sums and rounded once.  Iterations chain
// with programmatic dependent launch.
#include "hx_internal.cuh"

namespace hx {
namespace {

constexpr int kTX = 128;          // tile columns
constexpr int kTY = 32;           // tile rows
constexpr int kThreads = 256;
constexpr int kJsW = kTX + 8;     // J tile: rows i0-1 .. i0+TY+1, cols j0-1 .. j0+TX+1 at x = 3 .. 133
constexpr int kJsH = kTY + 3;
constexpr int kCsW = kTX + 8;     // c tile: rows i0 .. i0+TY, cols j0 .. j0+TX at x = 4 .. 132
constexpr int kCsH = kTY + 1;

struct SradArgs {
    int nx, ny;
    int r0, r1, c0, c1;           // region of interest, half-open
    int tx0, ty0, ntx;            // first region tile and region tiles per row
    int roi_tiles;
    float k;                      // 0.25 * lambda
};

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

// Diffusion coefficient of a pixel from its value and its four neighbour
// differences.  The SRAD expression c = 1/(1 + (q^2 - q0sq)/(q0sq(1+q0sq)))
// with q^2 = num/den^2, num = G2/2 - L^2/16, den = 1 + L/4, G2 = S2/Jc^2 and
// L = S1/Jc (S1, S2: the sum of the differences and of their squares) is
// multiplied through by Jc^2 den^2, in which Jc^2 cancels:
//     E = Jc + S1/4 (= Jc den, the mean of the four neighbours),
//     c = E^2 / (E^2 + (S2/2 - S1^2/16 - q0sq E^2) iq)
// with iq = 1/(q0sq(1+q0sq)) once per launch.  Algebraically the SRAD
// expression (for Jc != 0), one division per pixel instead of five, and no
// reciprocal of Jc.  fp32, fixed order; each a*b + c is one fused
// multiply-add (a single rounding).
__device__ __forceinline__ float srad_coeff(float Jc, float dN, float dS, float dW, float dE, float q0sq, float iq) {
    const float S1 = (dN + dS) + (dW + dE);
    const float S2 = fmaf(dN, dN, dS * dS) + fmaf(dW, dW, dE * dE);
    const float E = fmaf(0.25f, S1, Jc);
    const float E2 = E * E;
    const float nm = fmaf(-0.0625f, S1 * S1, 0.5f * S2);
    float c = E2 / fmaf(fmaf(-q0sq, E2, nm), iq, E2);
    if (c < 0.0f) c = 0.0f;
    else if (c > 1.0f) c = 1.0f;
    return c;
}

// J' = Jc + k * D with the flux sum D = (cN dN + cS dS) + (cW dW + cE dE),
// fused multiply-adds as above.
__device__ __forceinline__ float srad_update(float Jc, float dN, float dS, float dW, float dE, float cN, float cS,
                                             float cW, float cE, float k) {
    const float D = fmaf(cN, dN, cS * dS) + fmaf(cW, dW, cE * dE);
    return fmaf(k, D, Jc);
}

// Region sums of one thread: s1 += v, s2 += v*v (the square kept exact as a
// float-float product).
struct RoiAcc {
    ff s1, s2;
};
__device__ __forceinline__ void roi_add(RoiAcc &a, float v) {
    a.s1 = ff_add_f(a.s1, v);
    const float p = v * v;
    a.s2 = ff_add(a.s2, ff{p, fmaf(v, v, -p)});
}

// CTA-wide combine of the threads' region sums (warp butterflies, then the
// warps in order), published as the tile's partial; the last region tile to
// arrive folds all partials in tile order and writes q0^2.  Fixed order
// throughout, so q0^2 depends only on the image and the region.
__device__ void roi_publish(RoiAcc a, const SradArgs &p, int roi_tile, NestWs *ws, float *q0sq_out) {
    __shared__ float4 red[kThreads / 32];
    __shared__ unsigned last;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    a.s1 = warp_sum(a.s1);
    a.s2 = warp_sum(a.s2);
    if (lane == 0) red[warp] = make_float4(a.s1.hi, a.s1.lo, a.s2.hi, a.s2.lo);
    __syncthreads();
    if (threadIdx.x == 0) {
        ff s1 = {0.0f, 0.0f}, s2 = {0.0f, 0.0f};
        for (int w = 0; w < kThreads / 32; ++w) {
            s1 = ff_add(s1, ff{red[w].x, red[w].y});
            s2 = ff_add(s2, ff{red[w].z, red[w].w});
        }
        ws->part[roi_tile] = make_float4(s1.hi, s1.lo, s2.hi, s2.lo);
        __threadfence();
        last = atomicAdd(&ws->tick[0], 1u) == (unsigned)(p.roi_tiles - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    RoiAcc t = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    for (int q = threadIdx.x; q < p.roi_tiles; q += kThreads) {
        const float4 v = __ldcg(&ws->part[q]);
        t.s1 = ff_add(t.s1, ff{v.x, v.y});
        t.s2 = ff_add(t.s2, ff{v.z, v.w});
    }
    t.s1 = warp_sum(t.s1);
    t.s2 = warp_sum(t.s2);
    __syncthreads();
    if (lane == 0) red[warp] = make_float4(t.s1.hi, t.s1.lo, t.s2.hi, t.s2.lo);
    __syncthreads();
    if (threadIdx.x == 0) {
        ff s1 = {0.0f, 0.0f}, s2 = {0.0f, 0.0f};
        for (int w = 0; w < kThreads / 32; ++w) {
            s1 = ff_add(s1, ff{red[w].x, red[w].y});
            s2 = ff_add(s2, ff{red[w].z, red[w].w});
        }
        const double npix = (double)(p.r1 - p.r0) * (double)(p.c1 - p.c0);
        const double mean = ff_to_double(s1) / npix;
        const double var = ff_to_double(s2) / npix - mean * mean;
        *q0sq_out = (float)(var / (mean * mean));
        ws->tick[0] = 0u;
    }
}

// Region sums of J itself (iteration 0, and every iteration of the unfused
// path).  One CTA per region tile, same tile geometry and order as the
// fused kernel.
__global__ void __launch_bounds__(kThreads) srad_stats_kernel(const float *__restrict__ J, SradArgs p, NestWs *ws,
                                                              float *q0sq_out) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const int roi_tile = blockIdx.x;
    const int i0 = (p.ty0 + roi_tile / p.ntx) * kTY, j0 = (p.tx0 + roi_tile % p.ntx) * kTX;
    RoiAcc a = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    for (int idx = threadIdx.x; idx < kTY * kTX; idx += kThreads) {
        const int i = i0 + idx / kTX, j = j0 + idx % kTX;
        if (i >= p.r0 && i < p.r1 && j >= p.c0 && j < p.c1) roi_add(a, J[(size_t)i * p.nx + j]);
    }
    roi_publish(a, p, roi_tile, ws, q0sq_out);
}

// Fast path of one interior tile: no clamping, 16-byte rows, outside the
// region of interest.  Warp w updates rows ra = i0 + 4w .. ra + 3; lane l
// holds columns j0 + 4l .. j0 + 4l + 3 of a row as one float4, and the west
// and east neighbours come by shuffle (lanes 0 and 31 take the halo columns
// j0 - 1 and j0 + 128).  A warp computes the coefficients of its own four
// rows in registers; the first of them also goes to shared memory (one row
// per warp, in Cs), because the warp above needs it as the south neighbour of
// its last row, and the last warp computes row i0 + 32 itself.  Lanes 0..3
// compute the coefficients of column j0 + 128 (the east neighbour of lane
// 31's last pixel) for the warp's four rows.  The per-pixel expressions and
// their operands are those of the element path, so the two agree bit for
// bit; only the data movement differs (J rows in registers, one barrier).
__device__ __forceinline__ void srad_fast_tile(const float *__restrict__ J, float *__restrict__ Jn, int nx, int i0,
                                               int j0, float q0sq, float iq, float k, float (*Cs)[kCsW]) {
    constexpr unsigned kAll = 0xffffffffu;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ra = i0 + 4 * warp;
    const bool last = warp == kThreads / 32 - 1;
    // rows ra - 1 .. ra + 4, and ra + 5 for the last warp (its row ra + 4
    // coefficient); halo columns of each
    float4 Jr[7];
    float hw[7], he[7];
#pragma unroll
    for (int t = 0; t < 7; ++t) {
        if (t < 6 || last) {
            const float *row = J + (size_t)(ra - 1 + t) * nx + j0;
            Jr[t] = __ldg(reinterpret_cast<const float4 *>(row) + lane);
            hw[t] = __ldg(row - 1);
            he[t] = __ldg(row + 128);
        } else {
            Jr[t] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            hw[t] = he[t] = 0.0f;
        }
    }
    // coefficient of row ra - 1 + t for this lane's four columns
    auto coeff_row = [&](int t) {
        const float4 up = Jr[t - 1], cur = Jr[t], dn = Jr[t + 1];
        float left = __shfl_up_sync(kAll, cur.w, 1), right = __shfl_down_sync(kAll, cur.x, 1);
        if (lane == 0) left = hw[t];
        if (lane == 31) right = he[t];
        float4 c;
        c.x = srad_coeff(cur.x, up.x - cur.x, dn.x - cur.x, left - cur.x, cur.y - cur.x, q0sq, iq);
        c.y = srad_coeff(cur.y, up.y - cur.y, dn.y - cur.y, cur.x - cur.y, cur.z - cur.y, q0sq, iq);
        c.z = srad_coeff(cur.z, up.z - cur.z, dn.z - cur.z, cur.y - cur.z, cur.w - cur.z, q0sq, iq);
        c.w = srad_coeff(cur.w, up.w - cur.w, dn.w - cur.w, cur.z - cur.w, right - cur.w, q0sq, iq);
        return c;
    };
    float4 c[4];
#pragma unroll
    for (int t = 1; t <= 4; ++t) c[t - 1] = coeff_row(t);
    float ce = 0.0f;   // lane q < 4: column j0 + 128 of row ra + q
    if (lane < 4) {
        const float *col = J + (size_t)(ra + lane) * nx + j0 + 128;
        const float Jc = __ldg(col);
        ce = srad_coeff(Jc, __ldg(col - nx) - Jc, __ldg(col + nx) - Jc, __ldg(col - 1) - Jc, __ldg(col + 1) - Jc,
                        q0sq, iq);
    }
    *reinterpret_cast<float4 *>(&Cs[warp][4 * lane]) = c[0];
    __syncthreads();
    float4 c_south;   // coefficients of row ra + 4
    if (last) c_south = coeff_row(5);
    else c_south = *reinterpret_cast<const float4 *>(&Cs[warp + 1][4 * lane]);
#pragma unroll
    for (int t = 1; t <= 4; ++t) {
        const float4 up = Jr[t - 1], cur = Jr[t], dn = Jr[t + 1];
        float left = __shfl_up_sync(kAll, cur.w, 1), right = __shfl_down_sync(kAll, cur.x, 1);
        if (lane == 0) left = hw[t];
        if (lane == 31) right = he[t];
        const float4 kc = c[t - 1];
        const float4 ks = t < 4 ? c[t] : c_south;
        float ke = __shfl_down_sync(kAll, kc.x, 1);
        const float ke31 = __shfl_sync(kAll, ce, t - 1);
        if (lane == 31) ke = ke31;
        float4 o;
        o.x = srad_update(cur.x, up.x - cur.x, dn.x - cur.x, left - cur.x, cur.y - cur.x, kc.x, ks.x, kc.x, kc.y, k);
        o.y = srad_update(cur.y, up.y - cur.y, dn.y - cur.y, cur.x - cur.y, cur.z - cur.y, kc.y, ks.y, kc.y, kc.z, k);
        o.z = srad_update(cur.z, up.z - cur.z, dn.z - cur.z, cur.y - cur.z, cur.w - cur.z, kc.z, ks.z, kc.z, kc.w, k);
        o.w = srad_update(cur.w, up.w - cur.w, dn.w - cur.w, cur.z - cur.w, right - cur.w, kc.w, ks.w, kc.w, ke, k);
        *reinterpret_cast<float4 *>(Jn + (size_t)(ra + t - 1) * nx + j0 + 4 * lane) = o;
    }
}

// One fused iteration: coefficient in shared memory, update, and the next
// iteration's region sums.  q0sq_next == nullptr on the last iteration.
//
// Shared tiles keep image column j0 + x - 4 at index x, so the tile's 128
// columns start on a 16-byte boundary (x = 4): J at x = 3 .. 133, c at
// x = 4 .. 132.  A tile whose halo lies inside the image, outside the
// region of interest, takes the vector path when rows are 16-byte aligned
// (vec): float4 loads and stores, four pixels per thread step.  Every other
// tile takes the element path with clamped loads.  Both evaluate the same
// per-pixel expressions on the same operands, so they agree bit for bit.
// Four CTAs per SM (a 64-register cap, a few words of spill): the fast path
// holds a warp's J rows and coefficients in registers and is latency-bound,
// so occupancy decides.  Measured on B300, 8192^2: 0.160 ms per iteration,
// against 0.201 ms uncapped (98 registers, 2 CTAs per SM) and 0.215 ms at
// five CTAs per SM (48 registers, heavy spill).
__global__ void __launch_bounds__(kThreads, 4) srad_fused_kernel(const float *__restrict__ J, float *__restrict__ Jn,
                                                              SradArgs p, const float *q0sq_t, NestWs *ws,
                                                              float *q0sq_next, int vec) {
    __shared__ __align__(16) float Js[kJsH][kJsW];
    __shared__ __align__(16) float Cs[kCsH][kCsW];
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const int i0 = blockIdx.y * kTY, j0 = blockIdx.x * kTX;
    const int nx = p.nx, ny = p.ny;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float q0sq = *q0sq_t;
    const float iq = 1.0f / (q0sq * (1.0f + q0sq));
    const bool in_roi_rows = i0 < p.r1 && i0 + kTY > p.r0;
    const bool roi_tile = in_roi_rows && j0 < p.c1 && j0 + kTX > p.c0;
    const bool in_roi = q0sq_next && roi_tile;
    const bool fast = vec && !roi_tile && i0 >= 1 && i0 + kTY + 1 < ny && j0 >= 1 && j0 + kTX + 1 < nx;
    if (fast) {
        srad_fast_tile(J, Jn, nx, i0, j0, q0sq, iq, p.k, Cs);
        return;
    }
    // Element path.  J tile with a halo of 1 above / left and 2 below /
    // right, clamped to the image (the clamp-to-edge neighbours): warp w
    // loads rows w, w+8, ...
    for (int r = warp; r < kJsH; r += kThreads / 32) {
        const float *row = J + (size_t)clampi(i0 - 1 + r, 0, ny - 1) * nx;
#pragma unroll
        for (int c = lane; c < kTX + 3; c += 32) Js[r][3 + c] = __ldg(row + clampi(j0 - 1 + c, 0, nx - 1));
    }
    __syncthreads();
    // coefficient of rows i0 .. i0+TY and cols j0 .. j0+TX (inside the image)
    for (int idx = threadIdx.x; idx < kCsH * (kTX + 1); idx += kThreads) {
        const int r = idx / (kTX + 1), c = idx - r * (kTX + 1);
        if (i0 + r < ny && j0 + c < nx) {
            const float Jc = Js[r + 1][c + 4];
            Cs[r][c + 4] = srad_coeff(Jc, Js[r][c + 4] - Jc, Js[r + 2][c + 4] - Jc, Js[r + 1][c + 3] - Jc,
                                      Js[r + 1][c + 5] - Jc, q0sq, iq);
        }
    }
    __syncthreads();
    RoiAcc a = {{0.0f, 0.0f}, {0.0f, 0.0f}};
    const int c = threadIdx.x & (kTX - 1);
    for (int r = threadIdx.x / kTX; r < kTY; r += kThreads / kTX) {
        const int i = i0 + r, j = j0 + c;
        if (i < ny && j < nx) {
            const float Jc = Js[r + 1][c + 4];
            const int rs = i + 1 < ny ? r + 1 : r, ce = j + 1 < nx ? c + 1 : c;
            const float v = srad_update(Jc, Js[r][c + 4] - Jc, Js[r + 2][c + 4] - Jc, Js[r + 1][c + 3] - Jc,
                                        Js[r + 1][c + 5] - Jc, Cs[r][c + 4], Cs[rs][c + 4], Cs[r][c + 4],
                                        Cs[r][ce + 4], p.k);
            Jn[(size_t)i * nx + j] = v;
            if (in_roi && i >= p.r0 && i < p.r1 && j >= p.c0 && j < p.c1) roi_add(a, v);
        }
    }
    if (in_roi) {
        const int roi_tile = (blockIdx.y - p.ty0) * p.ntx + (blockIdx.x - p.tx0);
        if (!HX_CHECK(roi_tile >= 0 && roi_tile < p.roi_tiles, kChkSradTile, roi_tile, p.roi_tiles)) return;
        roi_publish(a, p, roi_tile, ws, q0sq_next);
    }
}

// Unfused: the coefficient of every pixel into C.
__global__ void __launch_bounds__(kThreads) srad_coeff_kernel(const float *__restrict__ J, float *__restrict__ C,
                                                              SradArgs p, const float *q0sq_t) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const int j = blockIdx.x * kTX + (threadIdx.x & (kTX - 1));
    const int i = blockIdx.y * (kThreads / kTX) + (threadIdx.x / kTX);
    if (i >= p.ny || j >= p.nx) return;
    const int nx = p.nx;
    const float Jc = J[(size_t)i * nx + j];
    const float dN = J[(size_t)clampi(i - 1, 0, p.ny - 1) * nx + j] - Jc;
    const float dS = J[(size_t)clampi(i + 1, 0, p.ny - 1) * nx + j] - Jc;
    const float dW = J[(size_t)i * nx + clampi(j - 1, 0, nx - 1)] - Jc;
    const float dE = J[(size_t)i * nx + clampi(j + 1, 0, nx - 1)] - Jc;
    const float q0sq = *q0sq_t;
    C[(size_t)i * nx + j] = srad_coeff(Jc, dN, dS, dW, dE, q0sq, 1.0f / (q0sq * (1.0f + q0sq)));
}

// Unfused: the flux update from J and C.
__global__ void __launch_bounds__(kThreads) srad_update_kernel(const float *__restrict__ J,
                                                               const float *__restrict__ C, float *__restrict__ Jn,
                                                               SradArgs p) {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;");
    const int j = blockIdx.x * kTX + (threadIdx.x & (kTX - 1));
    const int i = blockIdx.y * (kThreads / kTX) + (threadIdx.x / kTX);
    if (i >= p.ny || j >= p.nx) return;
    const int nx = p.nx;
    const size_t is = (size_t)clampi(i + 1, 0, p.ny - 1), je = (size_t)clampi(j + 1, 0, nx - 1);
    const float Jc = J[(size_t)i * nx + j];
    const float dN = J[(size_t)clampi(i - 1, 0, p.ny - 1) * nx + j] - Jc;
    const float dS = J[is * nx + j] - Jc;
    const float dW = J[(size_t)i * nx + clampi(j - 1, 0, nx - 1)] - Jc;
    const float dE = J[(size_t)i * nx + je] - Jc;
    const float c = C[(size_t)i * nx + j];
    Jn[(size_t)i * nx + j] = srad_update(Jc, dN, dS, dW, dE, c, C[is * nx + j], c, C[(size_t)i * nx + je], p.k);
}

}  // namespace

HX_CHECKS_READER(checks_srad)

}  // namespace hx

extern "C" hx_status hx_srad(hx_ctx *ctx, float *J0, float *J1, float *C, int32_t nx, int32_t ny, int32_t iters,
                             float lambda, int32_t r0, int32_t r1, int32_t c0, int32_t c1, float *d_q0sq,
                             int32_t fused, int32_t *result_in_J1, hx_stream_t stream) {
    using namespace hx;
    if (!ctx) return fail(HX_ERR_INVALID, "hx_srad: ctx is NULL");
    if (nx < 1 || ny < 1 || nx > 65536 || ny > 65536 || (int64_t)nx * ny > ((int64_t)1 << 31))
        return fail(HX_ERR_INVALID, "hx_srad: image size out of range");
    if (iters < 0 || iters > (1 << 20)) return fail(HX_ERR_INVALID, "hx_srad: iters out of range");
    if (r0 < 0 || r1 > ny || r0 >= r1 || c0 < 0 || c1 > nx || c0 >= c1)
        return fail(HX_ERR_INVALID, "hx_srad: region of interest empty or outside the image");
    if (!J0 || !J1) return fail(HX_ERR_INVALID, "hx_srad: image pointer is NULL");
    if (iters > 0 && !d_q0sq) return fail(HX_ERR_INVALID, "hx_srad: d_q0sq is NULL");
    if (!fused && iters > 0 && !C) return fail(HX_ERR_INVALID, "hx_srad: the unfused path needs C");
    if ((((uintptr_t)J0 | (uintptr_t)J1 | (uintptr_t)C | (uintptr_t)d_q0sq) & 3u) != 0)
        return fail(HX_ERR_INVALID, "hx_srad: pointers must be 4-byte aligned");
    const size_t bytes = (size_t)nx * ny * sizeof(float);
    auto overlap = [bytes](const float *a, const float *b) {
        return a && b && (uintptr_t)a < (uintptr_t)b + bytes && (uintptr_t)b < (uintptr_t)a + bytes;
    };
    if (overlap(J0, J1) || (!fused && (overlap(J0, C) || overlap(J1, C))))
        return fail(HX_ERR_INVALID, "hx_srad: image buffers overlap");
    SradArgs p;
    p.nx = nx;
    p.ny = ny;
    p.r0 = r0;
    p.r1 = r1;
    p.c0 = c0;
    p.c1 = c1;
    p.tx0 = c0 / kTX;
    p.ty0 = r0 / kTY;
    p.ntx = (c1 - 1) / kTX - p.tx0 + 1;
    const int nty = (r1 - 1) / kTY - p.ty0 + 1;
    p.roi_tiles = p.ntx * nty;
    p.k = 0.25f * lambda;
    if (p.roi_tiles > kNestCap) return fail(HX_ERR_NOMEM, "hx_srad: region of interest spans too many tiles");
    if (result_in_J1) *result_in_J1 = iters & 1;
    if (iters == 0) return HX_OK;
    DeviceGuard g(ctx->device);
    WsSlot *slot = nullptr;
    hx_status st = slot_for(ctx, stream, &slot);
    if (st != HX_OK) return st;
    if (take_injected_failure(ctx)) return fail(HX_ERR_CUDA, "hx_srad: injected launch failure (test hook)");
    NestWs *ws = ctx->nest_ws + (slot - ctx->ws);

    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3(kThreads);
    cfg.stream = (cudaStream_t)stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const dim3 tiles((nx + kTX - 1) / kTX, (ny + kTY - 1) / kTY);
    // float4 rows: 16-byte aligned images whose rows are whole float4s
    const int vec = nx % 4 == 0 && (((uintptr_t)J0 | (uintptr_t)J1) & 15u) == 0;
    const dim3 rows_grid((nx + kTX - 1) / kTX, (ny + kThreads / kTX - 1) / (kThreads / kTX));
    cudaError_t e;
    for (int t = 0; t < iters; ++t) {
        const float *src = (t & 1) ? J1 : J0;
        float *dst = (t & 1) ? J0 : J1;
        if (t == 0 || !fused) {
            cfg.gridDim = dim3(p.roi_tiles);
            e = cudaLaunchKernelEx(&cfg, srad_stats_kernel, src, p, ws, d_q0sq + t);
            if (e != cudaSuccess) return cuda_fail(e, "hx_srad: stats launch");
        }
        if (fused) {
            cfg.gridDim = tiles;
            float *next = t + 1 < iters ? d_q0sq + t + 1 : nullptr;
            e = cudaLaunchKernelEx(&cfg, srad_fused_kernel, src, dst, p, (const float *)(d_q0sq + t), ws, next, vec);
        } else {
            cfg.gridDim = rows_grid;
            e = cudaLaunchKernelEx(&cfg, srad_coeff_kernel, src, C, p, (const float *)(d_q0sq + t));
            if (e == cudaSuccess) e = cudaLaunchKernelEx(&cfg, srad_update_kernel, src, (const float *)C, dst, p);
        }
        if (e != cudaSuccess) return cuda_fail(e, "hx_srad: launch");
    }
    return HX_OK;
}
