"""Pins of the oracle's generic fork-join nest (map program + monoid reduce).

Each pin checks ``oracle.fork_reduce`` against something fixed outside the
oracle: numpy's IEEE single-precision elementwise arithmetic (correctly
rounded like C's float operators), numpy reductions and index grids, exact
lattice arithmetic in double for the single-rounding FMA, and a Python left
fold for the Sec. 3.3 reduction order (thread IDs increasing, dimension 0
outermost).
"""

import functools
import math

import numpy as np
import pytest

import oracle
import workloads


def _x(n, seed, stride=1, phase=0):
    return workloads.uniform_pm1_f32(seed, n, stride, phase)


def _grid(shape, seed):
    return _x(int(np.prod(shape)), seed).reshape(shape)


BINARY = {"add": np.add, "sub": np.subtract, "mul": np.multiply, "div": np.divide,
          "min": np.minimum, "max": np.maximum}
UNARY = {"neg": np.negative, "abs": np.abs, "sqrt": np.sqrt}


@pytest.mark.parametrize("op", sorted(BINARY))
def test_nest_binary_ops_match_numpy_single(op):
    x = _grid((37, 53), 11)
    y = _grid((37, 53), 12) + np.float32(0.5 if op == "div" else 0.0)   # keep y away from 0 for div
    y = y.astype(np.float32)
    out, _, _ = oracle.fork_reduce([("in", 0), ("in", 1), op], [x, y], x.shape, 0)
    np.testing.assert_array_equal(out.view(np.uint32), BINARY[op](x, y).view(np.uint32))


@pytest.mark.parametrize("op", sorted(UNARY))
def test_nest_unary_ops_match_numpy_single(op):
    x = _grid((64, 33), 13)
    if op == "sqrt":
        x = np.abs(x)
    out, _, _ = oracle.fork_reduce([("in", 0), op], [x], x.shape, 0)
    np.testing.assert_array_equal(out.view(np.uint32), UNARY[op](x).view(np.uint32))


def test_nest_min_max_ops_skip_nan():
    # MIN / MAX return the other operand when one is NaN (IEEE minNum /
    # maxNum, numpy's fmin / fmax); NaNs sit in x and y at disjoint places
    x = _grid((31, 29), 21)
    y = _grid((31, 29), 22)
    x.reshape(-1)[::7] = np.nan
    y.reshape(-1)[3::11] = np.nan
    for op, ref in (("min", np.fmin), ("max", np.fmax)):
        out, _, _ = oracle.fork_reduce([("in", 0), ("in", 1), op], [x, y], x.shape, 0)
        np.testing.assert_array_equal(out.view(np.uint32), ref(x, y).view(np.uint32))


def test_nest_unary_ops_special_values():
    # signed zeros, infinities, NaN and a subnormal through NEG / ABS bit for
    # bit against numpy; SQRT keeps -0, and is NaN for every negative input
    sp = np.array([-0.0, 0.0, -1.5, 2.25, np.inf, -np.inf, np.nan, 1e-45, -1e-45], np.float32)
    for op in ("neg", "abs"):
        out, _, _ = oracle.fork_reduce([("in", 0), op], [sp], sp.shape, 0)
        np.testing.assert_array_equal(out.view(np.uint32), UNARY[op](sp).view(np.uint32))
    out, _, _ = oracle.fork_reduce([("in", 0), "sqrt"], [sp], sp.shape, 0)
    ok = ~(np.signbit(sp) & (sp != 0)) & ~np.isnan(sp)
    with np.errstate(invalid="ignore"):
        ref = np.sqrt(sp)
    np.testing.assert_array_equal(out[ok].view(np.uint32), ref[ok].view(np.uint32))
    assert np.all(np.isnan(out[~ok]))


def test_nest_const_and_operand_order():
    x = _grid((5, 7), 14)
    out, _, _ = oracle.fork_reduce([("const", 2), ("in", 0), "sub", ("const", 1), "div"], [x], x.shape, 0,
                                   consts=[0.0, 3.0, 1.25])
    ref = (np.float32(1.25) - x) / np.float32(3.0)
    np.testing.assert_array_equal(out.view(np.uint32), ref.astype(np.float32).view(np.uint32))


def test_nest_fma_is_one_rounding():
    # x on the 2^-23 lattice, a = 1.5: a*x needs 25 bits, a*x + y is exact in
    # double, so rounding the double once gives fmaf's single rounding.
    x = _grid((128, 64), 15)
    y = _grid((128, 64), 16)
    out, _, _ = oracle.fork_reduce([("in", 0), ("const", 0), ("in", 1), "fma"], [x, y], x.shape, 0,
                                   consts=[1.5])
    ref = (x.astype(np.float64) * 1.5 + y.astype(np.float64)).astype(np.float32)
    np.testing.assert_array_equal(out.view(np.uint32), ref.view(np.uint32))
    two_roundings = (x * np.float32(1.5)) + y
    assert np.count_nonzero(two_roundings != ref) > 0     # the pin separates fma from mul+add


def _rows():
    x = _grid((23, 301), 17)
    return np.concatenate([x, x[:3] - np.float32(2.0)], axis=0)   # last rows all negative


def test_nest_row_sums_match_numpy():
    x = _rows()
    _, res, _ = oracle.fork_reduce([("in", 0)], [x], x.shape, 1, "sum")
    ref = x.astype(np.float64).sum(axis=1)
    bound = 1e-13 * np.abs(x.astype(np.float64)).sum(axis=1)
    assert np.all(np.abs(res - ref) <= bound)


def test_nest_row_prods_match_numpy():
    x = (np.float32(1.0) + _grid((9, 200), 18) * np.float32(0.01)).astype(np.float32)
    _, res, _ = oracle.fork_reduce([("in", 0)], [x], x.shape, 1, "prod")
    ref = np.prod(x.astype(np.float64), axis=1)
    np.testing.assert_allclose(res, ref, rtol=1e-13)
    _, res0, _ = oracle.fork_reduce([("in", 0)], [x[:, :0]], (9, 0), 1, "prod")
    np.testing.assert_array_equal(res0, np.ones(9))


@pytest.mark.parametrize("monoid,fn", [("max", np.max), ("min", np.min)])
def test_nest_row_extrema_match_numpy(monoid, fn):
    x = _rows()
    _, res, _ = oracle.fork_reduce([("in", 0)], [x], x.shape, 1, monoid)
    np.testing.assert_array_equal(res, fn(x, axis=1).astype(np.float64))


@pytest.mark.parametrize("monoid,fn", [("argmax", np.argmax), ("argmin", np.argmin)])
def test_nest_row_arg_extrema_match_numpy(monoid, fn):
    x = _rows()
    x[4, 10] = x[4, 200] = np.float32(5.0)        # tie: the first one wins
    x[5, 7] = x[5, 8] = np.float32(-5.0)
    _, res, idx = oracle.fork_reduce([("in", 0)], [x], x.shape, 1, monoid)
    ref_i = fn(x, axis=1)
    np.testing.assert_array_equal(idx, ref_i)
    np.testing.assert_array_equal(res, x[np.arange(x.shape[0]), ref_i].astype(np.float64))
    assert idx[4 if monoid == "argmax" else 5] == (10 if monoid == "argmax" else 7)


def test_nest_3d_partial_reductions_match_numpy():
    x = _grid((4, 5, 6), 19)
    x64 = x.astype(np.float64)
    for rd, axes in ((1, (2,)), (2, (1, 2)), (3, (0, 1, 2))):
        out, res, _ = oracle.fork_reduce([("in", 0)], [x], x.shape, rd, "sum")
        np.testing.assert_array_equal(out, x)
        np.testing.assert_allclose(res, x64.sum(axis=axes), rtol=0, atol=1e-12)
    _, res, idx = oracle.fork_reduce([("in", 0)], [x], x.shape, 2, "argmax")
    flat = x.reshape(4, 30)
    np.testing.assert_array_equal(idx, flat.argmax(axis=1))


def test_nest_strided_and_broadcast_inputs():
    a = _grid((40, 70), 20)          # the fork walks a.T: dims (70, 40)
    b = _x(40, 21)
    bb = np.broadcast_to(b, (70, 40))
    out, res, _ = oracle.fork_reduce([("in", 0), ("in", 1), "add"], [a.T, bb], (70, 40), 1, "sum")
    np.testing.assert_array_equal(out.view(np.uint32), (a.T + bb).view(np.uint32))
    ref = (a.T + bb).astype(np.float64).sum(axis=1)
    assert np.all(np.abs(res - ref) <= 1e-13 * np.abs(a.T + bb).astype(np.float64).sum(axis=1))
    # a reversed (negative-stride) view
    out, _, _ = oracle.fork_reduce([("in", 0)], [a[::-1, ::-1]], a.shape, 0)
    np.testing.assert_array_equal(out, a[::-1, ::-1])


def test_nest_index_op_matches_index_grid():
    dims = (3, 4, 5)
    ii = np.indices(dims).astype(np.float32)
    for d in range(3):
        out, _, _ = oracle.fork_reduce([("index", d)], [], dims, 0)
        np.testing.assert_array_equal(out, ii[d])
    out, _, _ = oracle.fork_reduce([("index", 0), ("const", 0), "mul", ("index", 1), "add"], [], (7, 9), 0,
                                   consts=[9.0])
    np.testing.assert_array_equal(out.ravel(), np.arange(63, dtype=np.float32))
    _, res, idx = oracle.fork_reduce([("index", 1), ("index", 0), "sub", "abs", "neg"], [], (6, 6), 1, "argmax")
    np.testing.assert_array_equal(idx, np.arange(6))      # the diagonal is the only 0


def test_nest_fold_order_is_thread_id_order():
    # 2^54 + 1 rounds back to 2^54 in double: a left fold in thread-ID order
    # gives 0 for (2^54, 1, -2^54) and 1 for (2^54, -2^54, 1).
    for vals in ([2.0 ** 54, 1.0, -2.0 ** 54], [2.0 ** 54, -2.0 ** 54, 1.0], [1.0, 2.0 ** 54, -2.0 ** 54]):
        x = np.asarray(vals, dtype=np.float32)
        _, res, _ = oracle.fork_reduce([("in", 0)], [x], (3,), 1, "sum")
        assert float(res) == functools.reduce(lambda s, v: s + float(v), x, 0.0)
    assert math.fsum([2.0 ** 54, 1.0, -2.0 ** 54]) == 1.0     # the exact sum differs: order matters


def test_nest_nan_and_empty_rules():
    nan = np.float32("nan")
    x = np.asarray([[nan, 1.0, 3.0, nan, 3.0], [nan] * 5, [2.0, nan, -1.0, -1.0, nan]], dtype=np.float32)
    _, mx, _ = oracle.fork_reduce([("in", 0)], [x], x.shape, 1, "max")
    np.testing.assert_array_equal(mx, [3.0, -np.inf, 2.0])
    _, mn, _ = oracle.fork_reduce([("in", 0)], [x], x.shape, 1, "min")
    np.testing.assert_array_equal(mn, [1.0, np.inf, -1.0])
    _, v, i = oracle.fork_reduce([("in", 0)], [x], x.shape, 1, "argmax")
    np.testing.assert_array_equal(i, [2, -1, 0])
    np.testing.assert_array_equal(v, [3.0, -np.inf, 2.0])
    _, v, i = oracle.fork_reduce([("in", 0)], [x], x.shape, 1, "argmin")
    np.testing.assert_array_equal(i, [1, -1, 2])
    e = np.zeros((4, 0), dtype=np.float32)
    for monoid, ident in (("sum", 0.0), ("prod", 1.0), ("max", -np.inf), ("min", np.inf),
                          ("argmax", -np.inf), ("argmin", np.inf)):
        _, r, i = oracle.fork_reduce([("in", 0)], [e], e.shape, 1, monoid)
        np.testing.assert_array_equal(r, np.full(4, ident))
        if i is not None:
            np.testing.assert_array_equal(i, np.full(4, -1))
    # min / max ops inside the program ignore a NaN operand (maxNum / minNum)
    out, _, _ = oracle.fork_reduce([("in", 0), ("const", 0), "max"], [x], x.shape, 0, consts=[0.5])
    np.testing.assert_array_equal(out, np.fmax(x, np.float32(0.5)))


def test_nest_signed_zero_rules():
    for row in ([-0.0, 0.0], [0.0, -0.0]):
        x = np.asarray([row], dtype=np.float32)
        _, mx, _ = oracle.fork_reduce([("in", 0)], [x], x.shape, 1, "max")
        _, mn, _ = oracle.fork_reduce([("in", 0)], [x], x.shape, 1, "min")
        assert mx[0] == 0.0 and not math.copysign(1.0, mx[0]) < 0
        assert mn[0] == 0.0 and math.copysign(1.0, mn[0]) < 0


@pytest.mark.parametrize("program", [
    ["add"],                                  # underflow
    [("in", 0), ("in", 0)],                   # two values left
    [("in", 1)],                              # no such input
    [("index", 2)],                           # no such dimension for a 2-D fork
    [("const", 8)],                           # no such constant
    [("in", 0)] * 9 + ["add"] * 8,            # deeper than 8
    [("in", 0), (99, 0)],                    # no such op
])
def test_nest_rejects_malformed(program):
    x = np.zeros((2, 3), dtype=np.float32)
    for dims, arr in (((2, 3), x), ((0, 3), x[:0])):
        with pytest.raises(ValueError):
            oracle.fork_reduce(program, [arr], dims, 1, "sum")
