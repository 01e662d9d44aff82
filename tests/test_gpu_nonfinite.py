"""Sums and products that meet infinities, NaN or fp32 overflow, on the GPU
against the oracle.

A reduce is a left fold from its identity (Sec. 3.3), so a sum that meets
+inf is +inf, one that meets both infinities or a NaN is NaN, and a product
that meets +inf stays infinite.  The GPU accumulates sums and products in
float-float pairs, which have fp32's exponent range; it must keep such
values instead of turning them into NaN through the pair's error term.

The rule checked for every result r (fp32) and r64 (the double output)
against the oracle's fp64 fold `ref`:
  * ref is NaN                      -> r and r64 are NaN;
  * |ref| > FLT_MAX (incl. +-inf)   -> r == r64 == +-inf with ref's sign
                                       (fp32 rounding of ref; the double
                                       output shares fp32's range);
  * otherwise the usual tolerances.
Map outputs are compared bit for bit, with any NaN matching any NaN.
The cases run through hx_map_reduce (vector and element paths, several
tiles), a batch instance (alone == batched), and hx_fork_reduce's sum and
product under all three reduction trees.
"""

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
FLT_MAX = float(np.finfo(np.float32).max)
INF, NAN = float("inf"), float("nan")


def _check_special(r, r64, ref):
    if np.isnan(ref):
        assert np.isnan(r) and np.isnan(r64), (r, r64, ref)
    elif abs(ref) > FLT_MAX:
        want = np.copysign(INF, ref)
        assert r == want and r64 == want, (r, r64, ref)
    else:
        raise AssertionError(f"case expected to be non-finite in fp32, oracle gives {ref}")


def _same_values(a, b):
    """Bit-equal arrays, except that any NaN matches any NaN."""
    na, nb = np.isnan(a), np.isnan(b)
    assert np.array_equal(na, nb)
    assert np.array_equal(a[~na].view(np.uint32), b[~nb].view(np.uint32))


def _inputs(n, seed, specials):
    """Map inputs on the usual lattice with special values planted in x:
    specials = [(index, value), ...]."""
    x, y = workloads.map_reduce_inputs(n, seed=seed)
    for i, v in specials:
        x[i] = np.float32(v)
    return x, y


def _overflow_inputs(n):
    # every out[i] = 1.5 * 2^126 + 0: the sum leaves fp32's range after two terms
    x = np.full(n, np.float32(2.0 ** 126), dtype=np.float32)
    return x, np.zeros(n, dtype=np.float32)


def _special_cases():
    n = 70_001        # several tiles, a ragged last tile
    return {
        "inf_small": lambda: _inputs(3, 1, [(1, INF)]),                         # [a, inf, b]
        "neg_inf_first": lambda: _inputs(2, 2, [(0, -INF)]),                    # [-inf, b]
        "inf_mid_tile": lambda: _inputs(n, 3, [(20_000, INF)]),
        "inf_ragged_tail": lambda: _inputs(n, 4, [(n - 1, -INF)]),
        "both_infinities": lambda: _inputs(n, 5, [(10, INF), (60_000, -INF)]),
        "nan": lambda: _inputs(n, 6, [(33_333, NAN)]),
        "nan_and_inf": lambda: _inputs(n, 7, [(5, NAN), (6, INF)]),
        "overflow_small": lambda: _overflow_inputs(5),
        "overflow_tiles": lambda: _overflow_inputs(n),
    }


@pytest.fixture(scope="module")
def ctx(gpu):
    c = gpu.hx_create(0)
    yield c
    c.close()


def _mr(gpu, ctx, x, y, offset):
    n = x.size
    xd = torch.zeros(n + offset, device=DEV)
    yd = torch.zeros(n + offset, device=DEV)
    xd[offset:] = torch.from_numpy(x)
    yd[offset:] = torch.from_numpy(y)
    out = torch.empty(n + offset, device=DEV)[offset:]
    s32 = torch.empty(1, device=DEV)
    s64 = torch.empty(1, dtype=torch.float64, device=DEV)
    gpu.hx_map_reduce(ctx, xd[offset:], yd[offset:], 1.5, out=out, sum_out=s32, sum64_out=s64)
    torch.cuda.synchronize()
    return out.cpu().numpy(), float(s32.item()), float(s64.item())


@pytest.mark.parametrize("offset", [0, 1])
@pytest.mark.parametrize("case", sorted(_special_cases()))
def test_map_reduce_non_finite(gpu, ctx, case, offset):
    x, y = _special_cases()[case]()
    out, s32, s64 = _mr(gpu, ctx, x, y, offset)
    out_o, s_o = oracle.map_reduce(x, y, 1.5)
    _same_values(out, out_o.astype(np.float32))
    _check_special(s32, s64, s_o)


def test_map_reduce_finite_after_special_calls(gpu, ctx):
    # a context's workspace holds no leftover non-finite state
    x, y = _special_cases()["both_infinities"]()
    _mr(gpu, ctx, x, y, 0)
    x, y = workloads.map_reduce_inputs(70_001, seed=8)
    _, s32, s64 = _mr(gpu, ctx, x, y, 0)
    _, s_o = oracle.map_reduce(x, y, 1.5)
    assert abs(s64 - s_o) <= 1e-5 * abs(s_o)


def test_batch_non_finite_alone_equals_batched(gpu, ctx):
    cases = _special_cases()
    names = sorted(cases)
    data = [cases[k]() for k in names]
    bufs, tasks = [], []
    for x, y in data:
        xd, yd = torch.from_numpy(x).to(DEV), torch.from_numpy(y).to(DEV)
        out = torch.empty_like(xd)
        s32 = torch.empty(1, device=DEV)
        s64 = torch.empty(1, dtype=torch.float64, device=DEV)
        bufs.append((xd, yd, out, s32, s64))
        tasks.append(gpu.map_reduce_task(xd, yd, 1.5, s32, out=out, sum64_out=s64))
    # a finite instance in the same batch stays finite and correct
    xf, yf = workloads.map_reduce_inputs(100_003, seed=9)
    xfd, yfd = torch.from_numpy(xf).to(DEV), torch.from_numpy(yf).to(DEV)
    sf32 = torch.empty(1, device=DEV)
    sf64 = torch.empty(1, dtype=torch.float64, device=DEV)
    tasks.append(gpu.map_reduce_task(xfd, yfd, 1.5, sf32, sum64_out=sf64))
    b = gpu.hx_batch_plan(ctx, tasks)
    b.launch()
    torch.cuda.synchronize()
    for (x, y), (xd, yd, out, s32, s64) in zip(data, bufs):
        got = out.cpu().numpy()
        alone = _mr(gpu, ctx, x, y, 0)
        _same_values(got, alone[0])
        b32, b64 = float(s32.item()), float(s64.item())
        assert (b32 == alone[1] or (np.isnan(b32) and np.isnan(alone[1])))
        assert (b64 == alone[2] or (np.isnan(b64) and np.isnan(alone[2])))
        out_o, s_o = oracle.map_reduce(x, y, 1.5)
        _check_special(b32, b64, s_o)
    _, s_o = oracle.map_reduce(xf, yf, 1.5)
    assert abs(sf64.item() - s_o) <= 1e-5 * abs(s_o)
    b.close()


def _nest_cases():
    n = 100_003
    base = workloads.uniform_pm1_f32(11, n)
    near1 = (np.float32(1.0) + base * np.float32(1e-3)).astype(np.float32)

    def plant(a, specials):
        a = a.copy()
        for i, v in specials:
            a[i] = np.float32(v)
        return a

    return {
        ("sum", "inf"): plant(base, [(77, INF)]),
        ("sum", "neg_inf_last"): plant(base, [(n - 1, -INF)]),
        ("sum", "both_infinities"): plant(base, [(3, -INF), (90_000, INF)]),
        ("sum", "nan"): plant(base, [(50_000, NAN)]),
        ("sum", "overflow"): np.full(4097, np.float32(2.0 ** 127), dtype=np.float32),
        ("prod", "inf"): plant(near1, [(1234, INF)]),
        ("prod", "nan"): plant(near1, [(99_999, NAN)]),
        ("prod", "inf_times_zero"): plant(near1, [(10, INF), (20, 0.0)]),
        # 2^8 ... per factor: the product passes FLT_MAX after 16 factors
        ("prod", "overflow"): np.full(40, np.float32(256.0), dtype=np.float32),
        ("prod", "overflow_negative"): plant(np.full(41, np.float32(-256.0), dtype=np.float32), []),
    }


@pytest.mark.parametrize("tree", ["warp", "chunk", "seq"])
@pytest.mark.parametrize("key", sorted(_nest_cases()))
def test_nest_non_finite(gpu, ctx, tree, key):
    monoid, _ = key
    x = _nest_cases()[key]
    n = x.size
    xd = torch.from_numpy(x).to(DEV)
    _, res, _, res64 = gpu.fork_reduce(ctx, [("in", 0)], [xd], (n,), 1, monoid, want_result64=True, tree=tree)
    torch.cuda.synchronize()
    _, ref, _ = oracle.fork_reduce([("in", 0)], [x], (n,), 1, monoid, want_out=False)
    _check_special(float(res.item()), float(res64.item()), float(np.ravel(ref)[0]))


@pytest.mark.parametrize("tree", ["warp", "chunk", "seq"])
def test_nest_row_sums_mixed_rows(gpu, ctx, tree):
    # rows of one nest: a finite row beside rows with +inf, -inf, NaN and overflow
    rows, cols = 5, 20_011
    x = workloads.uniform_pm1_f32(12, rows * cols).reshape(rows, cols)
    x[1, 7] = INF
    x[2, cols - 1] = -INF
    x[3, 9000] = NAN
    x[4, :] = np.float32(2.0 ** 127)
    xd = torch.from_numpy(x).to(DEV)
    _, res, _, res64 = gpu.fork_reduce(ctx, [("in", 0)], [xd], (rows, cols), 1, "sum", want_result64=True,
                                       tree=tree)
    torch.cuda.synchronize()
    _, ref, _ = oracle.fork_reduce([("in", 0)], [x], (rows, cols), 1, "sum", want_out=False)
    r, r64 = res.cpu().numpy(), res64.cpu().numpy()
    assert abs(r64[0] - ref[0]) <= 1e-9 * np.abs(x[0].astype(np.float64)).sum()
    for k in range(1, rows):
        _check_special(float(r[k]), float(r64[k]), float(ref[k]))
