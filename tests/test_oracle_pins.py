"""Pins of the CPU oracle against facts that do not come from the oracle itself.

Each nest is checked against closed forms, invariants, library routines on
cases that reduce to them, hand-worked golden values, and exactness
arguments.  The inputs are chosen so that the plausible mistakes (a dropped
term, a transposed operand, a wrong sign, an off-by-one index or bound, a
wrong boundary rule) each change a checked value.
"""

import json
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.ndimage

import oracle
import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


# ------------------------------------------------------------ map -> reduce
def test_map_reduce_golden_tiny():
    g = _golden("map_reduce_tiny.json")
    out, s = oracle.map_reduce(np.array(g["x"]), np.array(g["y"]), g["a"])
    assert out.tolist() == g["out"]
    assert s == g["sum"]


def test_map_reduce_arithmetic_series():
    # x_i = i 2^-20, y_i = 1 - i 2^-21, a = 1.5  =>  out_i = 1 + i 2^-20,
    # s = n + 2^-20 n(n-1)/2.  Every partial sum is exact in fp64.
    n = 1 << 20
    i = np.arange(n, dtype=np.float64)
    x = (i * 2.0**-20).astype(np.float32)
    y = (1.0 - i * 2.0**-21).astype(np.float32)
    out, s = oracle.map_reduce(x, y, 1.5)
    assert np.array_equal(out, 1.0 + i * 2.0**-20)
    assert Fraction(s) == n + Fraction(n * (n - 1), 2) * Fraction(1, 1 << 20)


def test_map_reduce_negative_scale_series():
    # a = -0.75, x_i = 1 - i 2^-20, y_i = 0.75  =>  out_i = 0.75 i 2^-20.
    n = 3 * 1000 + 7
    i = np.arange(n, dtype=np.float64)
    x = (1.0 - i * 2.0**-20).astype(np.float32)
    y = np.full(n, 0.75, dtype=np.float32)
    out, s = oracle.map_reduce(x, y, -0.75)
    assert np.array_equal(out, 0.75 * i * 2.0**-20)
    assert Fraction(s) == Fraction(3, 4) * Fraction(n * (n - 1), 2) * Fraction(1, 1 << 20)


def test_map_reduce_zero_scale_is_library_sum():
    x, y = workloads.map_reduce_inputs(10_000, seed=11)
    out, s = oracle.map_reduce(x, y, 0.0)
    assert np.array_equal(out, y.astype(np.float64))
    assert s == math.fsum(y.astype(np.float64))


def test_map_reduce_unit_inputs_count():
    # x = 1, y = 0: s = a n exactly (n terms of a).
    n = 12345
    _, s = oracle.map_reduce(np.ones(n, np.float32), np.zeros(n, np.float32), 1.5)
    assert s == 1.5 * n


def test_map_reduce_exact_on_lattice():
    # On the 2^-23 lattice with a = 1.5 every out_i and every partial sum is
    # exact in fp64, so the oracle's fold equals the exact rational sum.
    x, y = workloads.map_reduce_inputs(4097, seed=0)
    out, s = oracle.map_reduce(x, y, 1.5)
    exact = [Fraction(3, 2) * Fraction(float(a)) + Fraction(float(b)) for a, b in zip(x, y)]
    assert [Fraction(v) for v in out] == exact
    assert Fraction(s) == sum(exact)


def test_map_reduce_empty_and_single():
    _, s = oracle.map_reduce(np.zeros(0, np.float32), np.zeros(0, np.float32), 1.5)
    assert s == 0.0
    out, s = oracle.map_reduce(np.array([0.5], np.float32), np.array([-2.0], np.float32), 3.0)
    assert out.tolist() == [-0.5] and s == -0.5


def test_monoid_reduce_against_library():
    x, y = workloads.map_reduce_inputs(5000, seed=5)
    v = 1.5 * x.astype(np.float64) + y.astype(np.float64)
    assert oracle.monoid_reduce("max", x, 1.5, y) == v.max()
    assert oracle.monoid_reduce("min", x, 1.5, y) == v.min()
    assert oracle.monoid_reduce("sum", x, 1.5, y) == math.fsum(v)  # exact on the lattice
    small = np.array([1.5, -2.0, 0.25, 4.0], np.float32)
    assert oracle.monoid_reduce("prod", small) == math.prod([1.5, -2.0, 0.25, 4.0])
    assert oracle.monoid_reduce("max", np.zeros(0, np.float32)) == -math.inf
    assert oracle.monoid_reduce("prod", np.zeros(0, np.float32)) == 1.0


# ----------------------------------------------------------------- stencil
def test_jacobi_golden_corner_spike():
    g = _golden("jacobi_corner_spike.json")
    u0 = np.array(g["u0"])
    u1, r1 = oracle.jacobi(u0, 1)
    u2, r2 = oracle.jacobi(u0, 2)
    assert u1.tolist() == g["after_1"]
    assert u2.tolist() == g["after_2"]
    assert r2.tolist() == g["resid"] and r1.tolist() == g["resid"][:1]
    u1f, r1f = oracle.jacobi(u0, 2, precision="f32")
    assert u1f.tolist() == g["after_2"] and r1f.tolist() == g["resid"]


@pytest.mark.parametrize("shape", [(1, 1), (1, 7), (9, 1), (2, 2), (31, 45)])
def test_jacobi_constant_field_is_fixed_point(shape):
    c = 0.3125
    u0 = np.full(shape, c)
    for prec in ("f64", "f32"):
        u, r = oracle.jacobi(u0, 20, precision=prec)
        assert np.all(u == c) and np.all(r == 0)


def test_jacobi_interior_spike():
    u0 = np.zeros((7, 9))
    u0[3, 4] = 1.0
    u, r = oracle.jacobi(u0, 1)
    expect = np.zeros((7, 9))
    for (i, j) in ((2, 4), (4, 4), (3, 3), (3, 5)):
        expect[i, j] = 0.25
    assert np.array_equal(u, expect)
    assert r.tolist() == [1.0]


def test_jacobi_linear_field_closed_form():
    # u = i + 2 j is harmonic: interior points are unchanged.  On the edges the
    # clamped neighbour replaces the missing one: e.g. column 0 (j = 0, interior
    # row) gets 0.25((i-1 + i+1) + (i + i+2)) = i + 0.5; row 0 gets
    # 0.25((2j + 1+2j) + (2j-2 + 2j+2)) = 2j + 0.25.
    ny, nx = 6, 8
    i, j = np.meshgrid(np.arange(ny, dtype=np.float64), np.arange(nx, dtype=np.float64), indexing="ij")
    u0 = i + 2 * j
    u, r = oracle.jacobi(u0, 1)
    assert np.array_equal(u[1:-1, 1:-1], u0[1:-1, 1:-1])
    assert np.array_equal(u[1:-1, 0], u0[1:-1, 0] + 0.5)
    assert np.array_equal(u[1:-1, -1], u0[1:-1, -1] - 0.5)
    assert np.array_equal(u[0, 1:-1], u0[0, 1:-1] + 0.25)
    assert np.array_equal(u[-1, 1:-1], u0[-1, 1:-1] - 0.25)
    assert u[0, 0] == 0.75 and r[0] == 0.75


def test_jacobi_checkerboard_interior_flips_sign():
    ny, nx = 8, 10
    i, j = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    u0 = np.where((i + j) % 2 == 0, 1.0, -1.0)
    u, _ = oracle.jacobi(u0, 1)
    assert np.array_equal(u[1:-1, 1:-1], -u0[1:-1, 1:-1])


def test_jacobi_matches_scipy_nearest_correlation():
    # scipy.ndimage.correlate with mode='nearest' is exactly clamp-to-edge.
    w = np.array([[0.0, 0.25, 0.0], [0.25, 0.0, 0.25], [0.0, 0.25, 0.0]])
    rng_u = workloads.uniform01_f32(99, 37 * 53).reshape(37, 53).astype(np.float64)
    ref = rng_u.copy()
    ref_res = []
    for _ in range(20):
        nxt = scipy.ndimage.correlate(ref, w, mode="nearest")
        ref_res.append(np.abs(nxt - ref).max())
        ref = nxt
    u, r = oracle.jacobi(rng_u, 20)
    assert np.max(np.abs(u - ref)) <= 1e-14
    assert np.max(np.abs(r - np.array(ref_res))) <= 1e-14


def test_jacobi_conserves_total_mass():
    # With clamp-to-edge every point is referenced exactly four times with
    # weight 1/4, so the sweep is doubly stochastic and preserves the sum.
    # Dyadic inputs with few bits keep every operation exact in fp64.
    u0 = np.floor(workloads.uniform01_f32(7, 17 * 23).astype(np.float64) * 16) / 16
    u0 = u0.reshape(17, 23)
    for t in (1, 3, 6):
        u, _ = oracle.jacobi(u0, t)
        assert u.sum() == u0.sum()


def test_jacobi_f32_equals_f64_on_coarse_dyadics():
    # Values k/16 in [0,1): each sweep adds at most two fraction bits, so for
    # 10 sweeps every fp32 operation is exact and the two precisions agree.
    u0 = (np.floor(workloads.uniform01_f32(8, 40 * 33) * 16) / 16).reshape(40, 33)
    u64, r64 = oracle.jacobi(u0.astype(np.float64), 10, "f64")
    u32, r32 = oracle.jacobi(u0.astype(np.float32), 10, "f32")
    assert np.array_equal(u32.astype(np.float64), u64)
    assert np.array_equal(r32.astype(np.float64), r64)


def test_jacobi_f32_within_rounding_bound_of_f64():
    # Each sweep adds at most 3 roundings of relative size 2^-24 to values in
    # [0, 1), and averaging does not amplify earlier error, so after t sweeps
    # |u32 - u64| <= 3 t 2^-24.
    u0 = workloads.stencil_grid(64, 48, seed=3)
    t = 20
    u64, r64 = oracle.jacobi(u0.astype(np.float64), t, "f64")
    u32, r32 = oracle.jacobi(u0, t, "f32")
    bound = 3 * t * 2.0**-24
    assert np.max(np.abs(u32 - u64)) <= bound
    assert np.max(np.abs(r32 - r64)) <= 2 * bound + 2.0**-24


def test_jacobi_residual_is_max_step_change():
    u0 = workloads.stencil_grid(19, 21, seed=4).astype(np.float64)
    prev = u0
    _, r = oracle.jacobi(u0, 5)
    for t in range(5):
        cur, _ = oracle.jacobi(u0, t + 1)
        assert r[t] == np.abs(cur - prev).max()
        prev = cur


def test_jacobi_zero_iterations_returns_input():
    u0 = workloads.stencil_grid(5, 6, seed=1).astype(np.float64)
    u, r = oracle.jacobi(u0, 0)
    assert np.array_equal(u, u0) and r.size == 0


# --------------------------------------------------------------- histogram
def test_histogram_golden_tiny():
    g = _golden("histogram_tiny.json")
    bins, scan = oracle.histogram(np.array(g["v"], dtype=np.uint8))
    expect = np.zeros(256, np.uint32)
    for k, c in g["nonzero_bins"].items():
        expect[int(k)] = c
    assert np.array_equal(bins, expect)
    for k, c in g["scan_points"].items():
        assert scan[int(k)] == c


def test_histogram_matches_bincount_and_cumsum():
    v = workloads.histogram_mixture_u8(1 << 18, seed=2)
    bins, scan = oracle.histogram(v)
    ref = np.bincount(v, minlength=256).astype(np.uint32)
    assert np.array_equal(bins, ref)
    assert np.array_equal(scan, np.concatenate([[0], np.cumsum(ref)[:-1]]).astype(np.uint32))
    assert int(scan[255]) + int(bins[255]) == v.size


def test_histogram_closed_forms():
    n = 256 * 1000
    bins, scan = oracle.histogram(np.full(n, 77, np.uint8))
    assert bins[77] == n and bins.sum() == n
    assert np.all(scan[:78] == 0) and np.all(scan[78:] == n)
    ramp = (np.arange(n) % 256).astype(np.uint8)
    bins, scan = oracle.histogram(ramp)
    assert np.all(bins == 1000)
    assert np.array_equal(scan, (np.arange(256) * 1000).astype(np.uint32))
    bins, scan = oracle.histogram(np.zeros(0, np.uint8))
    assert not bins.any() and not scan.any()
