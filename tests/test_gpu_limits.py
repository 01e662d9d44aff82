"""Parity at the size limits of the C ABI (GPU).

Inputs as large as the ABI accepts, or past a 32-bit index:
  * a histogram of 2^32 - 1 bytes, the most whose u32 counts cannot
    overflow (one bin reaches 2^32 - 1);
  * a map->reduce over 2^31 + 5 elements (indices past 2^31);
  * one stencil sweep of a 32768 x 65536 grid: 2^31 points, rows of the
    widest accepted length;
  * generic nests over 2^31 + 7 elements: a sum on float4 slots, the same
    values through a transposed view (64-bit index division), and an argmax
    whose maximum lies past 2^31.
Outputs are checked against closed forms, or at sampled points against the
oracle evaluated on those points' own inputs; whole-output properties (every
value of a periodic output, the maximum of |u' - u|) with plain torch
reductions.  One past each limit is rejected before any device work.
"""

import ctypes

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

DEV = "cuda:0"


@pytest.fixture(scope="module")
def ctx(gpu):
    c = gpu.hx_create(0)
    yield c
    c.close()
    torch.cuda.empty_cache()


def _u32(t):
    return t.cpu().numpy().view(np.uint32)


def test_histogram_largest_input(gpu, ctx):
    n = (1 << 32) - 1
    buf = torch.empty(1 << 32, dtype=torch.uint8, device=DEV)
    v = buf[:n]
    # every byte one value: that bin holds 2^32 - 1
    v.fill_(7)
    bins, scan = gpu.hx_histogram(ctx, v)
    torch.cuda.synchronize()
    b, s = _u32(bins), _u32(scan)
    want = np.zeros(256, np.uint32)
    want[7] = 0xFFFFFFFF
    assert np.array_equal(b, want)
    assert np.array_equal(s, np.where(np.arange(256) > 7, 0xFFFFFFFF, 0).astype(np.uint32))
    # the ramp 0, 1, ..., 255, 0, ...: the last byte (255) is missing
    ramp = torch.arange(256, dtype=torch.int32, device=DEV).to(torch.uint8)
    v[: n - 255].view(-1, 256).copy_(ramp.expand((n - 255) // 256, 256))
    v[n - 255:].copy_(ramp[:255])
    bins, scan = gpu.hx_histogram(ctx, v)
    torch.cuda.synchronize()
    want = np.full(256, 1 << 24, np.uint32)
    want[255] -= 1
    assert np.array_equal(_u32(bins), want)
    assert np.array_equal(_u32(scan), (np.arange(256, dtype=np.uint64) << 24).astype(np.uint32))
    # one byte more is rejected
    with pytest.raises(gpu.HxError) as e:
        gpu.hx_histogram(ctx, buf)
    assert e.value.status == gpu.HX_ERR_INVALID
    del buf, v


def test_map_reduce_past_2p31(gpu, ctx):
    n = (1 << 31) + 5
    period = 1024
    k = torch.arange(period, dtype=torch.float64, device=DEV)
    reps = n // period + 1
    # x = k / 1024 and y = 1 - k / 2048 on the fp32 lattice: out = 1 + k / 1024 exactly
    x = (k * 2.0**-10).float().repeat(reps)[:n]
    y = (1.0 - k * 2.0**-11).float().repeat(reps)[:n]
    out = torch.empty(n, dtype=torch.float32, device=DEV)
    s32 = torch.empty(1, dtype=torch.float32, device=DEV)
    s64 = torch.empty(1, dtype=torch.float64, device=DEV)
    gpu.hx_map_reduce(ctx, x, y, 1.5, out=out, sum_out=s32, sum64_out=s64)
    torch.cuda.synchronize()
    full = n // period
    pattern = (1.0 + k * 2.0**-10).float()
    assert bool((out[: full * period].view(full, period) == pattern).all())
    assert torch.equal(out[full * period:], pattern[: n - full * period])
    # sampled points against the oracle on their own inputs
    rng = np.random.default_rng(31)
    idx = np.unique(np.concatenate([rng.integers(0, n, 4000), [0, (1 << 31) - 1, 1 << 31, n - 1]]))
    it = torch.from_numpy(idx).to(DEV)
    xs, ys, gs = x[it].cpu().numpy(), y[it].cpu().numpy(), out[it].cpu().numpy()
    out_o, _ = oracle.map_reduce(xs, ys, 1.5)
    assert np.array_equal(gs.view(np.uint32), out_o.astype(np.float32).view(np.uint32))
    # the sum in closed form: 2^21 whole periods plus k = 0..4
    exact = full * (period + (period - 1) / 2.0) + sum(1.0 + j * 2.0**-10 for j in range(n - full * period))
    assert abs(float(s64.item()) - exact) <= 1e-9 * exact
    assert np.float32(s64.item()) == np.float32(s32.item())
    del x, y, out


def test_stencil_widest_rows_2p31_points(gpu, ctx):
    ny, nx = 32768, 65536
    u0 = workloads.uniform01_f32_torch(41, ny * nx, DEV).view(ny, nx)
    u1 = torch.empty_like(u0)
    res = torch.full((1,), -1.0, dtype=torch.float32, device=DEV)
    fin, res = gpu.hx_stencil2d(ctx, u0, u1, 1, resid=res)
    torch.cuda.synchronize()
    assert fin.data_ptr() == u1.data_ptr()
    # sampled points: corners, edges and random interior points, each
    # against the oracle on its clamped 3 x 3 neighbourhood
    rng = np.random.default_rng(65536)
    pts = [(0, 0), (0, nx - 1), (ny - 1, 0), (ny - 1, nx - 1), (0, 12345), (ny - 1, 777), (4321, 0), (99, nx - 1)]
    pts += [(int(i), int(j)) for i, j in zip(rng.integers(0, ny, 300), rng.integers(0, nx, 300))]
    for i, j in pts:
        rows = [min(max(i + d, 0), ny - 1) for d in (-1, 0, 1)]
        cols = [min(max(j + d, 0), nx - 1) for d in (-1, 0, 1)]
        win = u0[rows][:, cols].cpu().numpy()
        u32, _ = oracle.jacobi(win, 1, "f32")
        assert np.float32(u1[i, j].item()).view(np.uint32) == u32[1, 1].view(np.uint32), (i, j)
    # the residual is the maximum of |u' - u| over all 2^31 points
    m = torch.zeros((), dtype=torch.float32, device=DEV)
    for r0 in range(0, ny, 2048):
        m = torch.maximum(m, (u1[r0:r0 + 2048] - u0[r0:r0 + 2048]).abs().max())
    assert np.float32(res[0].item()).view(np.uint32) == np.float32(m.item()).view(np.uint32)
    del u0, u1, fin


def test_one_past_the_size_limits_is_rejected(gpu, ctx):
    # host-side validation comes before any device work, so small real
    # buffers stand in for the (never touched) inputs
    lib = gpu._lib
    buf = torch.zeros(64, dtype=torch.float32, device=DEV)
    p = ctypes.c_void_p(buf.data_ptr())
    s = ctypes.c_void_p(buf[32:].data_ptr())
    rc = lib.hx_map_reduce(ctx.handle, p, p, None, 1.0, gpu.HX_MAP_REDUCE_MAX_N + 1, s, None, None)
    assert rc == gpu.HX_ERR_INVALID
    in_u1 = ctypes.c_int32(0)
    u0 = ctypes.c_void_p(buf.data_ptr())
    u1 = ctypes.c_void_p(buf[16:].data_ptr())
    for nx, ny in ((65537, 1), (1, 65537), (65536, 32769)):
        rc = lib.hx_stencil2d(ctx.handle, u0, u1, nx, ny, 1, s, ctypes.byref(in_u1), None)
        assert rc == gpu.HX_ERR_INVALID, (nx, ny)


def _ramp_sum(count, period=1024):
    """Exact sum of 1 + (i mod period) / period over i < count."""
    full, rem = divmod(count, period)
    return full * (period + (period - 1) / 2.0) + sum(1.0 + j / period for j in range(rem))


def test_nest_reductions_past_2p31(gpu, ctx):
    n = (1 << 31) + 7
    period = 1024
    k = torch.arange(period, dtype=torch.float64, device=DEV)
    x = (1.0 + k / period).float().repeat(n // period + 1)[:n]
    # sum over a linear input (float4 slots, about 2.7 chunks per resident warp)
    _, r, _, r64 = gpu.fork_reduce(ctx, [("in", 0)], [x], (n,), 1, "sum", want_result64=True)
    torch.cuda.synchronize()
    exact = _ramp_sum(n)
    assert abs(float(r64.item()) - exact) <= 1e-9 * exact
    assert np.float32(r64.item()) == np.float32(r.item())
    # the first 2m values through a transposed view: a 2 x m fork whose 2m
    # inner threads pass 2^31 (64-bit index division, element loads)
    m = n // 2
    xt = x[: 2 * m].view(m, 2).t()
    _, r, _, r64 = gpu.fork_reduce(ctx, [("in", 0)], [xt], (2, m), 2, "sum", want_result64=True)
    torch.cuda.synchronize()
    exact = _ramp_sum(2 * m)
    assert abs(float(r64.item()) - exact) <= 1e-9 * exact
    # argmax with its maximum past 2^31: ties go to the smaller index
    x.zero_()
    x[(1 << 31) + 3] = 2.0
    x[(1 << 31) + 5] = 2.0
    x[n - 1] = 1.5
    _, r, idx, _ = gpu.fork_reduce(ctx, [("in", 0)], [x], (n,), 1, "argmax")
    torch.cuda.synchronize()
    assert float(r.item()) == 2.0 and int(idx.item()) == (1 << 31) + 3
    del x, xt
