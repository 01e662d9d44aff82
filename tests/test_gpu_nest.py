"""Generic fork-join nests on the GPU against the oracle's sequential nest.

Map values (``out``) are compared bit for bit: both sides round every op once
to fp32.  Max / min / argmax / argmin are exact.  Sums and products are
float-float on the GPU and a double left fold in the oracle; the bound is
1e-5 of the condition (sum of |v|, resp. |prod|) for the fp32 result and
1e-9 for the double one.  The nests span several chunks and ragged tails,
all three reduction trees, strided / broadcast / reversed inputs, index ops
and empty segments.
"""

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu

TREES = ["warp", "chunk", "seq"]
MONOIDS = ["sum", "max", "min", "prod", "argmax", "argmin"]


def _np(shape, seed, lo=-1.0, scale=1.0):
    n = int(np.prod(shape))
    x = workloads.uniform_pm1_f32(seed, n) if n else np.zeros(0, np.float32)
    return (x.reshape(shape) * np.float32(scale) + np.float32(lo + 1.0)).astype(np.float32)


def _check(hx, ctx, program, arrays, view, dims, rd, monoid, consts=(), tree="warp", chunk=0, want_out=True):
    """Run one nest on the GPU (inputs = view(device copies)) and the oracle
    (inputs = view(numpy arrays)); compare."""
    np_in = view([a for a in arrays])
    dev = [torch.from_numpy(a).cuda() for a in arrays]
    t_in = view(dev)
    out, res, idx, res64 = hx.fork_reduce(ctx, program, t_in, dims, rd, monoid, consts, want_out=want_out,
                                          want_result64=rd > 0, tree=tree, chunk=chunk)
    torch.cuda.synchronize()
    ref_out, ref, ref_idx = oracle.fork_reduce(program, np_in, dims, rd, monoid, consts, want_out=True)
    if out is not None:
        np.testing.assert_array_equal(out.cpu().numpy().view(np.uint32), ref_out.view(np.uint32))
    if rd == 0:
        return out
    got = res.cpu().numpy().astype(np.float64)
    got64 = res64.cpu().numpy()
    if monoid in ("sum", "prod"):
        vals = ref_out.reshape(ref.shape + (-1,)).astype(np.float64)
        cond = np.abs(vals).sum(axis=-1) if monoid == "sum" else np.abs(ref)
        cond = np.maximum(cond, np.finfo(np.float32).tiny)
        assert np.all(np.abs(got - ref) <= 1e-5 * cond), (np.max(np.abs(got - ref) / cond))
        assert np.all(np.abs(got64 - ref) <= 1e-9 * cond), (np.max(np.abs(got64 - ref) / cond))
    else:
        np.testing.assert_array_equal(got, ref)
        np.testing.assert_array_equal(np.signbit(got), np.signbit(ref))
        np.testing.assert_array_equal(got64, ref)
    if monoid.startswith("arg"):
        np.testing.assert_array_equal(idx.cpu().numpy(), ref_idx)
    return res


ident = lambda xs: xs   # noqa: E731


@pytest.mark.parametrize("tree", TREES)
@pytest.mark.parametrize("monoid", MONOIDS)
@pytest.mark.parametrize("n", [0, 1, 31, 33, 1000, 4097, 100_003])
def test_full_reduce_1d(gpu, tree, monoid, n):
    hx = gpu
    x = _np((n,), 101, lo=-1.0)
    if monoid == "prod":
        x = (np.float32(1.0) + x * np.float32(1e-3)).astype(np.float32)
    with hx.hx_create(0) as ctx:
        _check(hx, ctx, [("in", 0)], [x], ident, (n,), 1, monoid, tree=tree)


@pytest.mark.parametrize("tree", TREES)
@pytest.mark.parametrize("monoid", MONOIDS)
@pytest.mark.parametrize("rows,cols", [(129, 5), (64, 31), (33, 1000), (3, 70_001)])
def test_row_reduce_fused_map(gpu, tree, monoid, rows, cols):
    # |x - y| * c + y over rows (the max-gradient shape of EDGE, Sec. 5.2)
    hx = gpu
    x = _np((rows, cols), 102)
    y = _np((rows, cols), 103)
    prog = [("in", 0), ("in", 1), "sub", "abs", ("const", 0), ("in", 1), "fma"]
    consts = [0.75]
    if monoid == "prod":
        prog = [("in", 0), ("const", 1), "mul", ("const", 2), "add"]   # 1 + x/1024: well conditioned
        consts = [0.75, 1.0 / 1024, 1.0]
    with hx.hx_create(0) as ctx:
        _check(hx, ctx, prog, [x, y], ident, (rows, cols), 1, monoid, consts, tree=tree)


@pytest.mark.parametrize("monoid", MONOIDS)
@pytest.mark.parametrize("rd", [1, 2, 3])
def test_3d_permuted_and_broadcast(gpu, monoid, rd):
    hx = gpu
    a = _np((7, 9, 33), 104)                      # viewed as (33, 7, 9): a permutation
    b = _np((9,), 105)                            # broadcast along dims 0 and 1
    view = lambda xs: [xs[0].transpose(2, 0, 1) if isinstance(xs[0], np.ndarray) else xs[0].permute(2, 0, 1),  # noqa: E731
                       (np.broadcast_to(xs[1], (33, 7, 9)) if isinstance(xs[1], np.ndarray)
                        else xs[1].expand(33, 7, 9))]
    prog = [("in", 0), ("in", 1), "mul", ("index", 2), ("const", 0), "mul", "add"]
    if monoid == "prod":
        prog = [("in", 0), ("const", 1), "mul", ("const", 2), "add"]
    with hx.hx_create(0) as ctx:
        _check(hx, ctx, prog, [a, b], view, (33, 7, 9), rd, monoid, [0.125, 1.0 / 256, 1.0])


@pytest.mark.parametrize("tree", TREES)
def test_index_only_program_and_map_only(gpu, tree):
    hx = gpu
    with hx.hx_create(0) as ctx:
        dims = (37, 61)
        out, _, _, _ = hx.fork_reduce(ctx, [("index", 0), ("const", 0), ("index", 1), "fma"], [], dims, 0,
                                      consts=[61.0], tree=tree, device="cuda:0")
        np.testing.assert_array_equal(out.cpu().numpy().ravel(), np.arange(37 * 61, dtype=np.float32))
        # argmax of -|j - i| is the diagonal
        _, res, idx, _ = hx.fork_reduce(ctx, [("index", 1), ("index", 0), "sub", "abs", "neg"], [], (50, 50), 1,
                                        "argmax", tree=tree, device="cuda:0")
        assert torch.equal(idx.cpu(), torch.arange(50))
        x = _np((300, 301), 106)
        _check(hx, ctx, [("in", 0), "abs", "sqrt", ("in", 0), "div"], [x], ident, (300, 301), 0, "sum", tree=tree)


def test_reversed_strides_through_the_abi(gpu):
    hx = gpu
    n = 10_001
    x = _np((n,), 107)
    with hx.hx_create(0) as ctx:
        t = torch.from_numpy(x).cuda()
        res = torch.empty((), dtype=torch.float32, device="cuda:0")
        idx = torch.empty((), dtype=torch.int64, device="cuda:0")
        out = torch.empty(n, dtype=torch.float32, device="cuda:0")
        nest = hx.make_nest([("in", 0)], [t], (n,), 1, "argmax", out=out, result=res, result_index=idx)
        nest.inputs[0] = t.data_ptr() + 4 * (n - 1)     # walk x backwards: stride -1
        nest.strides[0][0] = -1
        hx.hx_fork_reduce(ctx, nest)
        torch.cuda.synchronize()
        _, ref, ref_idx = oracle.fork_reduce([("in", 0)], [x[::-1]], (n,), 1, "argmax")
        np.testing.assert_array_equal(out.cpu().numpy(), x[::-1])
        assert float(res) == float(ref) and int(idx) == int(ref_idx)


def test_ties_nans_signed_zeros(gpu):
    hx = gpu
    nan = np.float32("nan")
    x = _np((6, 1000), 108)
    x[0, 10] = x[0, 900] = np.float32(7.0)
    x[1, :] = nan
    x[2, ::3] = nan
    x[3, :] = np.float32(-0.0)
    x[3, 500] = np.float32(0.0)
    x[4, :] = np.float32(0.0)
    x[4, 777] = np.float32(-0.0)
    x[5, 5] = x[5, 995] = np.float32(-9.0)
    with hx.hx_create(0) as ctx:
        for tree in TREES:
            for monoid in ("max", "min", "argmax", "argmin"):
                _check(hx, ctx, [("in", 0)], [x], ident, x.shape, 1, monoid, tree=tree)


def test_ties_nans_signed_zeros_short_and_long_segments(gpu):
    # The same special values in segments of 8 (groups narrower than a warp)
    # and in one segment of 2^20 + 5 that spans many chunks and the tree
    # above them (whole-warp groups, whose max / min fold is fmaxf / fminf).
    hx = gpu
    nan = np.float32("nan")
    s = _np((64, 8), 109)
    s[0, :] = nan
    s[1, ::2] = nan
    s[2, :] = np.float32(-0.0)
    s[2, 5] = np.float32(0.0)
    s[3, :] = np.float32(0.0)
    s[3, 2] = np.float32(-0.0)
    s[4, 1] = s[4, 6] = np.float32(1e30)
    n = (1 << 20) + 5
    g = np.abs(_np((n,), 110)) * np.float32(-1.0) - np.float32(1.0)   # all below -1
    g[::7] = nan
    g[123456] = np.float32(-0.0)
    g[987654] = np.float32(0.0)
    g[555] = np.float32(0.0)
    g[n - 1] = np.float32(-0.0)
    with hx.hx_create(0) as ctx:
        for tree in TREES:
            for monoid in ("max", "min", "argmax", "argmin"):
                _check(hx, ctx, [("in", 0)], [s], ident, s.shape, 1, monoid, tree=tree)
                _check(hx, ctx, [("in", 0)], [g], ident, g.shape, 1, monoid, tree=tree)


def test_map_ops_on_special_values(gpu):
    # MIN / MAX with NaN operands, and NEG / ABS / SQRT of signed zeros,
    # infinities, NaN, subnormals and negatives, against the oracle.  A NaN
    # result's payload and sign are unspecified on the GPU, so NaN results
    # are compared by NaN-ness and every other result bit for bit.
    hx = gpu
    sp = np.array([-0.0, 0.0, -1.5, 2.25, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 3.0], np.float32)
    x = np.tile(sp, 40)
    y = np.roll(x, 3)
    progs = [([("in", 0), ("in", 1), "min"], 2), ([("in", 0), ("in", 1), "max"], 2), ([("in", 0), "neg"], 1),
             ([("in", 0), "abs"], 1), ([("in", 0), "sqrt"], 1), ([("in", 0), ("in", 1), "min", "abs"], 2)]
    with hx.hx_create(0) as ctx:
        for prog, n_in in progs:
            ins = [x, y][:n_in]
            out, _, _, _ = hx.fork_reduce(ctx, prog, [torch.from_numpy(a).cuda() for a in ins], x.shape, 0, "sum")
            torch.cuda.synchronize()
            ref, _, _ = oracle.fork_reduce(prog, ins, x.shape, 0)
            got = out.cpu().numpy()
            nan = np.isnan(ref)
            np.testing.assert_array_equal(np.isnan(got), nan)
            np.testing.assert_array_equal(got[~nan].view(np.uint32), ref[~nan].view(np.uint32))


@pytest.mark.parametrize("chunk", [256, 1000, 4096])
def test_explicit_chunks_and_determinism(gpu, chunk):
    hx = gpu
    x = _np((4, 200_000), 109)
    with hx.hx_create(0) as ctx:
        r1 = _check(hx, ctx, [("in", 0), ("in", 0), "mul"], [x], ident, x.shape, 1, "sum", chunk=chunk)
        r2 = _check(hx, ctx, [("in", 0), ("in", 0), "mul"], [x], ident, x.shape, 1, "sum", chunk=chunk)
        assert torch.equal(r1, r2)


def test_large_full_reduce_caps_partials(gpu):
    # 2^26 elements: more chunks than the workspace holds, so the chunk grows
    hx = gpu
    n = (1 << 26) + 7
    x = workloads.uniform_pm1_f32(110, n)
    with hx.hx_create(0) as ctx:
        for monoid in ("sum", "argmax"):
            _check(hx, ctx, [("in", 0), "abs"], [x], ident, (n,), 1, monoid, want_out=False)


@pytest.mark.parametrize("dims", [(700, 150_001), (110_000_003,)])
def test_large_sums_spread_chunks(gpu, dims):
    # sums past 2.7 chunks per resident warp get longer chunks, about 2.7 per
    # warp (ragged last chunks; the odd row length takes the element path)
    hx = gpu
    x = _np(dims, 121)
    with hx.hx_create(0) as ctx:
        _check(hx, ctx, [("in", 0), ("in", 0), "mul"], [x], ident, dims, 1, "sum", want_out=False)


def test_large_dot_spreads_chunks(gpu):
    # a two-input sum (2 CTAs per SM, so fewer resident warps) past the
    # spreading threshold, with an odd length (element path, ragged last chunk)
    hx = gpu
    n = 100_000_001
    x, y = _np((n,), 122), _np((n,), 123)
    with hx.hx_create(0) as ctx:
        _check(hx, ctx, [("in", 0), ("in", 1), "mul"], [x, y], ident, (n,), 1, "sum", want_out=False)


def test_empty_segments_give_identities(gpu):
    hx = gpu
    with hx.hx_create(0) as ctx:
        x = torch.zeros((5, 0), device="cuda:0")
        for monoid, ident_v in (("sum", 0.0), ("prod", 1.0), ("max", -np.inf), ("min", np.inf)):
            _, res, _, _ = hx.fork_reduce(ctx, [("in", 0)], [x], (5, 0), 1, monoid)
            assert torch.equal(res.cpu(), torch.full((5,), ident_v))
        _, res, idx, _ = hx.fork_reduce(ctx, [("in", 0)], [x], (5, 0), 1, "argmin")
        assert torch.equal(idx.cpu(), torch.full((5,), -1))
        # outer extent 0: nothing to do, nothing written
        hx.fork_reduce(ctx, [("in", 0)], [torch.zeros((0, 4), device="cuda:0")], (0, 4), 1, "sum")


def test_streams_use_separate_workspace(gpu):
    hx = gpu
    x = _np((1 << 20,), 111)
    y = _np((1 << 20,), 112)
    with hx.hx_create(0) as ctx:
        tx, ty = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
        s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
        torch.cuda.synchronize()
        outs = []
        for _ in range(4):
            for s, t in ((s1, tx), (s2, ty)):
                with torch.cuda.stream(s):
                    outs.append(hx.fork_reduce(ctx, [("in", 0)], [t], t.shape, 1, "sum", stream=s)[1])
        torch.cuda.synchronize()
        for k, r in enumerate(outs):
            assert torch.equal(r, outs[k % 2])
        ref_x = oracle.fork_reduce([("in", 0)], [x], x.shape, 1, "sum")[1]
        assert abs(float(outs[0]) - float(ref_x)) <= 1e-5 * np.abs(x).astype(np.float64).sum()


def test_alignment_does_not_change_bits(gpu):
    # the same rows, once 16-byte aligned (float4 path) and once shifted by
    # one element (scalar path): identical lane assignment, identical bits
    hx = gpu
    x = torch.from_numpy(_np((4, 4096), 113)).cuda()
    buf = torch.zeros(4 * 4096 + 4, device="cuda:0")
    with hx.hx_create(0) as ctx:
        res = []
        for off in (0, 1):
            v = buf[off:off + 4 * 4096].view(4, 4096)
            v.copy_(x)
            for monoid in ("sum", "prod", "argmax"):
                src = hx.hx_nest_source(hx.make_nest([("in", 0)], [v], (4, 4096), 1, monoid,
                                                     result=torch.empty(4, device="cuda:0"),
                                                     result_index=torch.empty(4, dtype=torch.int64, device="cuda:0")))
                assert ("#define VEC 1" in src) == (off == 0)
                _, r, i, r64 = hx.fork_reduce(ctx, [("in", 0), ("const", 0), "mul", ("const", 1), "add"], [v],
                                              (4, 4096), 1, monoid, consts=[1.0 / 64, 1.0], want_result64=True)
                res.append((r.clone(), r64.clone(), None if i is None else i.clone()))
        torch.cuda.synchronize()
        for a, b in zip(res[:3], res[3:]):
            assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
            if a[2] is not None:
                assert torch.equal(a[2], b[2])


@pytest.mark.parametrize("monoid", ["sum", "argmin"])
def test_strided_float4_slots(gpu, monoid):
    # (5, 6, 12) viewed as (6, 5, 12): the inner dims (5, 12) are strided
    # (72, 1) but every slot of 4 threads is 4 aligned contiguous floats
    hx = gpu
    a = _np((5, 6, 12), 114)
    view = lambda xs: [xs[0].transpose(1, 0, 2) if isinstance(xs[0], np.ndarray) else xs[0].permute(1, 0, 2)]  # noqa: E731
    with hx.hx_create(0) as ctx:
        t = torch.from_numpy(a).cuda().permute(1, 0, 2)
        src = hx.hx_nest_source(hx.make_nest([("in", 0)], [t], (6, 5, 12), 2, monoid,
                                             result=torch.empty(6, device="cuda:0"),
                                             result_index=torch.empty(6, dtype=torch.int64, device="cuda:0")))
        assert "#define VEC 1" in src and "p.lin[0]" not in src
        _check(hx, ctx, [("in", 0), ("index", 2), ("const", 0), "mul", "add"], [a], view, (6, 5, 12), 2, monoid,
               [0.5])
        big = _np((64, 96, 128), 115)
        view2 = lambda xs: [xs[0].transpose(1, 0, 2) if isinstance(xs[0], np.ndarray) else xs[0].permute(1, 0, 2)]  # noqa: E731
        _check(hx, ctx, [("in", 0), "abs"], [big], view2, (96, 64, 128), 2, monoid)


@pytest.mark.slow
def test_bench_workloads_full_size(gpu):
    # the six nests bench.py times, at their sizes, against the oracle (whole
    # arrays where the oracle takes seconds, sampled rows / segments otherwise)
    hx = gpu
    dev = torch.device("cuda:0")
    big = workloads.uniform_pm1_f32_torch(120, 1 << 28, dev)
    x27, y27 = big[: 1 << 27], big[1 << 27:]
    rng = np.random.default_rng(0)
    with hx.hx_create(0) as ctx:
        # sum of 2^28 and argmax |x - y| over 2^27: whole arrays
        _, s, _, s64 = hx.fork_reduce(ctx, [("in", 0)], [big], (1 << 28,), 1, "sum", want_result64=True)
        _, m, mi, _ = hx.fork_reduce(ctx, [("in", 0), ("in", 1), "sub", "abs"], [x27, y27], (1 << 27,), 1, "argmax")
        torch.cuda.synchronize()
        host = big.cpu().numpy()
        _, ref, _ = oracle.fork_reduce([("in", 0)], [host], host.shape, 1, "sum", want_out=False)
        cond = float(np.abs(host).astype(np.float64).sum())
        assert abs(float(s) - float(ref)) <= 1e-5 * cond and abs(float(s64) - float(ref)) <= 1e-9 * cond
        hx27, hy27 = host[: 1 << 27], host[1 << 27:]
        _, rm, ri = oracle.fork_reduce([("in", 0), ("in", 1), "sub", "abs"], [hx27, hy27], hx27.shape, 1, "argmax",
                                       want_out=False)
        assert float(m) == float(rm) and int(mi) == int(ri)
        # row sums of 16384 x 16384: 64 sampled rows
        mat = big.view(16384, 16384)
        _, rs, _, _ = hx.fork_reduce(ctx, [("in", 0)], [mat], mat.shape, 1, "sum")
        rows = rng.choice(16384, 64, replace=False)
        sub = host.reshape(16384, 16384)[rows]
        _, rref, _ = oracle.fork_reduce([("in", 0)], [sub], sub.shape, 1, "sum", want_out=False)
        got = rs.cpu().numpy()[rows].astype(np.float64)
        assert np.all(np.abs(got - rref) <= 1e-5 * np.abs(sub).astype(np.float64).sum(axis=1))
        # max over 2^24 rows of 8: 100000 sampled rows, exact
        r8 = big[: 1 << 27].view(1 << 24, 8)
        _, mx, _, _ = hx.fork_reduce(ctx, [("in", 0)], [r8], r8.shape, 1, "max")
        rows = rng.choice(1 << 24, 100_000, replace=False)
        sub = host[: 1 << 27].reshape(1 << 24, 8)[rows]
        _, mref, _ = oracle.fork_reduce([("in", 0)], [sub], sub.shape, 1, "max", want_out=False)
        np.testing.assert_array_equal(mx.cpu().numpy()[rows].astype(np.float64), mref)
        # fused map over 2^27: sampled elements, bit for bit
        out, _, _, _ = hx.fork_reduce(ctx, [("in", 0), ("const", 0), ("in", 1), "fma"], [x27, y27], (1 << 27,), 0,
                                      consts=[1.5])
        idx = rng.choice(1 << 27, 1 << 20, replace=False)
        oref, _, _ = oracle.fork_reduce([("in", 0), ("const", 0), ("in", 1), "fma"],
                                        [np.ascontiguousarray(hx27[idx]), np.ascontiguousarray(hy27[idx])],
                                        (idx.size,), 0, consts=[1.5])
        np.testing.assert_array_equal(out.cpu().numpy()[idx].view(np.uint32), oref.view(np.uint32))
        # 3-D sum over dims 1, 2 of the permuted 1024 x 512 x 512 view: 8 sampled segments
        v3 = big.view(512, 1024, 512).permute(1, 0, 2)
        _, r3, _, _ = hx.fork_reduce(ctx, [("in", 0)], [v3], v3.shape, 2, "sum")
        segs = rng.choice(1024, 8, replace=False)
        h3 = host.reshape(512, 1024, 512)
        for sgm in segs:
            blk = np.ascontiguousarray(h3[:, sgm, :])
            _, bref, _ = oracle.fork_reduce([("in", 0)], [blk], blk.shape, 2, "sum", want_out=False)
            assert abs(float(r3[sgm]) - float(bref)) <= 1e-5 * float(np.abs(blk).astype(np.float64).sum())
