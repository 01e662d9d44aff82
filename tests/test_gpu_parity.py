"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Tolerances (stated once, used everywhere):
  * map output: bit-exact against the fp64 oracle rounded to fp32.  On the
    input lattice (multiples of 2^-23, a = 1.5) a*x+y is exact in fp64, so
    the correctly rounded fmaf result equals that rounding.
  * sum: |s_gpu - s_fp64| <= 1e-5 * |s_fp64| wherever |s_fp64| >= 1e-3 *
    sum|out_i| (the float-float accumulator carries about 48 bits, so the
    relative bound holds unless the sum nearly cancels); for a nearly
    cancelling sum, <= 1e-5 * sum|out_i| (the sum's condition number bounds
    what any fp32-output method can reach).
  * stencil: bit-exact against the fp32 evaluation of the same expression
    ((N+S)+(W+E))*0.25 and the same residual, and within 1e-5 normwise
    (max|diff| / max|u_fp64|) of the fp64 oracle.
  * histogram and scan: bit-exact.
"""

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
SUM_TOL = 1e-5
STENCIL_TOL = 1e-5


@pytest.fixture(scope="module")
def ctx(gpu):
    c = gpu.hx_create(0)
    yield c
    c.close()


def _mr(gpu, ctx, x, y, a, want_out=True, offset=0):
    n = x.size
    xd = torch.zeros(n + offset, dtype=torch.float32, device=DEV)
    yd = torch.zeros(n + offset, dtype=torch.float32, device=DEV)
    xd[offset:] = torch.from_numpy(x)
    yd[offset:] = torch.from_numpy(y)
    xv, yv = xd[offset:], yd[offset:]
    out = torch.empty(n + offset, dtype=torch.float32, device=DEV)[offset:] if want_out else None
    s32 = torch.empty(1, dtype=torch.float32, device=DEV)
    s64 = torch.empty(1, dtype=torch.float64, device=DEV)
    gpu.hx_map_reduce(ctx, xv, yv, a, out=out, sum_out=s32, sum64_out=s64)
    torch.cuda.synchronize()
    return (out.cpu().numpy() if want_out else None), float(s32.item()), float(s64.item())


def _check_mr(out_g, s32, s64, x, y, a):
    out_o, s_o = oracle.map_reduce(x, y, a)
    if out_g is not None:
        assert np.array_equal(out_g.view(np.uint32), out_o.astype(np.float32).view(np.uint32))
    cond = np.abs(out_o).sum()
    scale = abs(s_o) if abs(s_o) >= 1e-3 * cond else cond
    assert abs(s64 - s_o) <= SUM_TOL * scale + 1e-300
    assert np.float32(s64) == np.float32(s32)


@pytest.mark.parametrize("n", [0, 1, 2, 3, 4, 5, 31, 32, 33, 1023, 1024, 1025, 4095, 4096, 4097,
                               (1 << 20) - 1, (1 << 20) + 1, 3_000_001])
def test_map_reduce_sizes(gpu, ctx, n):
    x, y = workloads.map_reduce_inputs(n, seed=n + 17)
    out, s32, s64 = _mr(gpu, ctx, x, y, 1.5)
    _check_mr(out, s32, s64, x, y, 1.5)


def test_map_reduce_standard_workload_relative(gpu, ctx):
    x, y = workloads.map_reduce_inputs(1 << 20, seed=0)
    out, s32, s64 = _mr(gpu, ctx, x, y, 1.5)
    _check_mr(out, s32, s64, x, y, 1.5)
    _, s_o = oracle.map_reduce(x, y, 1.5, want_out=False)
    assert abs(s64 - s_o) <= SUM_TOL * abs(s_o)
    assert abs(s32 - s_o) <= SUM_TOL * abs(s_o)


def test_map_reduce_large_tiles(gpu, ctx):
    # above 2^23 elements a thread owns more than one unrolled group per tile
    n = (1 << 24) + 5
    x, y = workloads.map_reduce_inputs(n, seed=3)
    out, s32, s64 = _mr(gpu, ctx, x, y, 1.5)
    _check_mr(out, s32, s64, x, y, 1.5)


@pytest.mark.parametrize("offset", [1, 2, 3])
def test_map_reduce_misaligned_matches_aligned_bits(gpu, ctx, offset):
    n = 70_001
    x, y = workloads.map_reduce_inputs(n, seed=9)
    out_a, s32_a, s64_a = _mr(gpu, ctx, x, y, -0.75)
    out_m, s32_m, s64_m = _mr(gpu, ctx, x, y, -0.75, offset=offset)
    assert np.array_equal(out_a.view(np.uint32), out_m.view(np.uint32))
    assert s64_a == s64_m and s32_a == s32_m
    _check_mr(out_m, s32_m, s64_m, x, y, -0.75)


def test_map_reduce_without_out_and_deterministic(gpu, ctx):
    x, y = workloads.map_reduce_inputs(999_999, seed=4)
    _, s32a, s64a = _mr(gpu, ctx, x, y, 1.5, want_out=False)
    _, s32b, s64b = _mr(gpu, ctx, x, y, 1.5, want_out=True)
    assert s64a == s64b and s32a == s32b
    _check_mr(None, s32a, s64a, x, y, 1.5)


def test_map_reduce_closed_form(gpu, ctx):
    n = 1 << 20
    i = np.arange(n, dtype=np.float64)
    x = (i * 2.0**-20).astype(np.float32)
    y = (1.0 - i * 2.0**-21).astype(np.float32)
    out, s32, s64 = _mr(gpu, ctx, x, y, 1.5)
    assert np.array_equal(out.astype(np.float64), 1.0 + i * 2.0**-20)
    exact = n + (n * (n - 1) / 2) * 2.0**-20
    assert abs(s64 - exact) <= SUM_TOL * exact


def test_map_reduce_rejects_bad_args(gpu, ctx):
    x = torch.zeros(8, device=DEV)
    with pytest.raises(gpu.HxError):
        gpu.hx_map_reduce(ctx, x, x.clone(), 1.0, out=x)   # out overlaps x
    with pytest.raises(gpu.HxError):
        gpu.hx_stencil2d(ctx, x.view(2, 4), x.view(2, 4), 1)           # u0 and u1 overlap
    with pytest.raises(ValueError):
        gpu.hx_map_reduce(ctx, x, torch.zeros(7, device=DEV), 1.0)


# ------------------------------------------------------------------ stencil
def _st(gpu, ctx, u0_np, iters, offset=0):
    ny, nx = u0_np.shape
    n = ny * nx
    b0 = torch.zeros(n + offset, dtype=torch.float32, device=DEV)
    b1 = torch.zeros(n + offset, dtype=torch.float32, device=DEV)
    b0[offset:] = torch.from_numpy(u0_np.ravel())
    u0 = b0[offset:].view(ny, nx)
    u1 = b1[offset:].view(ny, nx)
    res = torch.full((max(iters, 1),), -1.0, dtype=torch.float32, device=DEV)
    fin, res = gpu.hx_stencil2d(ctx, u0, u1, iters, resid=res)
    torch.cuda.synchronize()
    return fin.cpu().numpy(), res.cpu().numpy()[:iters]


def _check_st(u_g, r_g, u0, iters):
    u32, r32 = oracle.jacobi(u0.astype(np.float32), iters, "f32")
    assert np.array_equal(u_g.view(np.uint32), u32.view(np.uint32))
    assert np.array_equal(r_g.view(np.uint32), r32.view(np.uint32))
    if iters:
        u64, r64 = oracle.jacobi(u0.astype(np.float64), iters, "f64")
        scale = max(np.abs(u64).max(), 1e-30)
        assert np.abs(u_g - u64).max() <= STENCIL_TOL * scale
        assert np.abs(r_g - r64).max() <= STENCIL_TOL * scale


@pytest.mark.parametrize("shape", [(1, 1), (1, 5), (7, 1), (3, 3), (4, 4), (5, 8), (17, 33), (64, 128),
                                   (65, 129), (100, 132), (70, 516), (257, 300)])
@pytest.mark.parametrize("iters", [1, 2, 5])
def test_stencil_shapes(gpu, ctx, shape, iters):
    u0 = workloads.stencil_grid(*shape, seed=shape[0] * 1000 + shape[1])
    u, r = _st(gpu, ctx, u0, iters)
    _check_st(u, r, u0, iters)


def test_stencil_zero_iterations(gpu, ctx):
    u0 = workloads.stencil_grid(8, 12, seed=5)
    u, r = _st(gpu, ctx, u0, 0)
    assert np.array_equal(u, u0) and r.size == 0


@pytest.mark.parametrize("offset", [1, 3])
def test_stencil_misaligned_scalar_path_same_bits(gpu, ctx, offset):
    u0 = workloads.stencil_grid(40, 256, seed=8)
    ua, ra = _st(gpu, ctx, u0, 3)
    um, rm = _st(gpu, ctx, u0, 3, offset=offset)
    assert np.array_equal(ua.view(np.uint32), um.view(np.uint32))
    assert np.array_equal(ra.view(np.uint32), rm.view(np.uint32))


def test_stencil_constant_field_fixed_point(gpu, ctx):
    u0 = np.full((33, 64), 0.625, np.float32)
    u, r = _st(gpu, ctx, u0, 4)
    assert np.all(u == 0.625) and np.all(r == 0)


@pytest.mark.slow
def test_stencil_standard_workload_full_size(gpu, ctx):
    u0 = workloads.stencil_grid(2048, 2048, seed=workloads.SEED_STENCIL)
    u, r = _st(gpu, ctx, u0, 20)
    _check_st(u, r, u0, 20)


# ------------------------------------------------------------------ histogram
def _hi(gpu, ctx, v, offset=0):
    n = v.size
    buf = torch.zeros(n + offset, dtype=torch.uint8, device=DEV)
    buf[offset:] = torch.from_numpy(v)
    bins, scan = gpu.hx_histogram(ctx, buf[offset:])
    torch.cuda.synchronize()
    return bins.cpu().numpy().view(np.uint32), scan.cpu().numpy().view(np.uint32)


def _check_hi(bins, scan, v):
    b_o, s_o = oracle.histogram(v)
    assert np.array_equal(bins, b_o)
    assert np.array_equal(scan, s_o)


@pytest.mark.parametrize("n", [0, 1, 15, 16, 17, 255, 256, 4097, 65536, (1 << 20) + 3])
@pytest.mark.parametrize("offset", [0, 1, 7, 15])
def test_histogram_sizes_and_alignment(gpu, ctx, n, offset):
    v = workloads.histogram_mixture_u8(n, seed=n + offset)
    bins, scan = _hi(gpu, ctx, v, offset)
    _check_hi(bins, scan, v)


def test_histogram_adversarial_inputs(gpu, ctx):
    n = 1 << 24
    v = np.full(n, 200, np.uint8)
    _check_hi(*_hi(gpu, ctx, v), v)
    v = (np.arange(n) % 256).astype(np.uint8)
    _check_hi(*_hi(gpu, ctx, v), v)


@pytest.mark.slow
def test_histogram_standard_workload_full_size(gpu, ctx):
    v = workloads.histogram_mixture_u8(1 << 26, seed=workloads.SEED_HISTOGRAM)
    bins, scan = _hi(gpu, ctx, v)
    _check_hi(bins, scan, v)
    assert int(scan[255]) + int(bins[255]) == 1 << 26


def test_histogram_repeat_is_clean(gpu, ctx):
    # the workspace resets itself: a second call does not see the first's counts
    v = workloads.histogram_mixture_u8(100_000, seed=1)
    a = _hi(gpu, ctx, v)
    b = _hi(gpu, ctx, v)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
