"""Pins of the oracle's SRAD-style nest (``oracle.srad``).

What fixes it from outside the oracle:
  * flux conservation: with clamp-to-edge (zero-flux) borders the update is
    a sum of pairwise fluxes c*(J_nb - J) that cancel, so sum(J') = sum(J);
  * transpose symmetry of the scheme;
  * the maximum principle for lambda <= 1 (0 <= c <= 1 makes J' a convex
    combination of the pixel and its neighbours);
  * where every pixel's coefficient clamps to 1 the step is the weighted
    5-point Jacobi relaxation, checked against scipy.ndimage.correlate;
  * the speckle scale q0^2 = var/mean^2 of the region of interest against
    numpy's mean and (population) variance;
  * a closed form on a checkerboard: every interior pixel's four neighbours
    are equal, so its instantaneous coefficient of variation is
    q^2 = (a - b)^2 / a^2 (b = the pixel, a = its neighbours);
  * homogeneous regions: q0^2 = 0 gives NaN, a flat neighbourhood is left
    unchanged;
  * the diffusion coefficient c(q^2): values worked by hand with exact
    fractions from the published formula (tests/golden/srad_coefficient.json),
    including a clamped coefficient and the case q^2 = q0^2.
"""

import json
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import ndimage

import oracle
import workloads


def _img(ny, nx, seed):
    u = workloads.uniform01_f32(seed, ny * nx).reshape(ny, nx).astype(np.float64)
    return np.exp(u)


@pytest.mark.parametrize("lam", [0.25, 0.5, 1.0])
@pytest.mark.parametrize("shape", [(17, 23), (1, 9), (8, 1), (40, 40)])
def test_srad_conserves_mass(lam, shape):
    J = _img(*shape, 31)
    roi = (0, shape[0], 0, shape[1])
    out, _ = oracle.srad(J, 3, lam, roi)
    assert abs(out.sum() - J.sum()) <= 1e-13 * J.sum()


def test_srad_transpose_symmetry():
    J = _img(19, 27, 32)
    a, qa = oracle.srad(J, 2, 0.5, (2, 9, 3, 20))
    b, qb = oracle.srad(J.T.copy(), 2, 0.5, (3, 20, 2, 9))
    np.testing.assert_allclose(b, a.T, rtol=1e-12, atol=0)
    np.testing.assert_allclose(qb, qa, rtol=1e-12)


@pytest.mark.parametrize("lam", [0.5, 1.0])
def test_srad_maximum_principle(lam):
    J = _img(33, 31, 33)
    out, _ = oracle.srad(J, 1, lam, (0, 16, 0, 16))
    pad = np.pad(J, 1, mode="edge")
    nb = np.stack([pad[1:-1, 1:-1], pad[:-2, 1:-1], pad[2:, 1:-1], pad[1:-1, :-2], pad[1:-1, 2:]])
    assert np.all(out >= nb.min(axis=0) - 1e-12) and np.all(out <= nb.max(axis=0) + 1e-12)


@pytest.mark.parametrize("lam", [0.5, 1.0])
def test_srad_is_jacobi_relaxation_where_c_clamps_to_one(lam):
    # a steep smooth ramp with tiny noise: the whole-image speckle scale is
    # far above every pixel's local one, so every c clamps to 1
    ny, nx = 48, 64
    ramp = 1.0 + 0.9 * np.arange(nx)[None, :] / nx + 0.5 * np.arange(ny)[:, None] / ny
    J = ramp + 1e-3 * workloads.uniform01_f32(34, ny * nx).reshape(ny, nx)
    out, q0 = oracle.srad(J, 1, lam, (0, ny, 0, nx))
    cross = np.array([[0.0, 0.25, 0.0], [0.25, 0.0, 0.25], [0.0, 0.25, 0.0]])
    jac = ndimage.correlate(J, cross, mode="nearest")
    np.testing.assert_allclose(out, (1.0 - lam) * J + lam * jac, rtol=1e-12, atol=0)


def test_srad_speckle_scale_matches_numpy():
    J = _img(30, 40, 35)
    J[20:, :] *= 7.0                     # outside the region: must not count
    roi = (3, 17, 5, 33)
    _, q0 = oracle.srad(J, 1, 0.5, roi)
    reg = J[3:17, 5:33]
    assert abs(q0[0] - reg.var() / reg.mean() ** 2) <= 1e-12 * q0[0]


@pytest.mark.parametrize("a,b", [(2.0, 1.0), (1.0, 3.0), (1.5, 1.25)])
def test_srad_checkerboard_closed_form(a, b):
    ny, nx = 12, 16
    ii, jj = np.indices((ny, nx))
    J = np.where((ii + jj) % 2 == 0, b, a).astype(np.float64)
    lam = 0.5
    out, q0 = oracle.srad(J, 1, lam, (0, ny, 0, nx))
    # even counts of a and b: mean (a+b)/2, population variance ((a-b)/2)^2
    q0sq = (a - b) ** 2 / (a + b) ** 2
    assert abs(q0[0] - q0sq) <= 1e-14
    # a pixel of value p whose four neighbours are all o has q^2 = (o-p)^2/o^2
    def c_of(p, o):
        qsq = (o - p) ** 2 / o ** 2
        return min(1.0, max(0.0, 1.0 / (1.0 + (qsq - q0sq) / (q0sq * (1.0 + q0sq)))))
    c_b, c_a = c_of(b, a), c_of(a, b)
    # interior pixel whose S and E neighbours are interior too:
    # D = (a-b)*(c_self + c_other + c_self + c_other)
    inner = (slice(1, ny - 2), slice(1, nx - 2))
    want = np.where((ii + jj) % 2 == 0, b + 0.25 * lam * (a - b) * 2 * (c_b + c_a),
                    a + 0.25 * lam * (b - a) * 2 * (c_a + c_b))
    np.testing.assert_allclose(out[inner], want[inner], rtol=1e-13, atol=0)


def test_srad_homogeneous_cases():
    J = np.full((6, 5), 2.5)
    out, q0 = oracle.srad(J, 1, 0.5, (0, 6, 0, 5))
    assert q0[0] == 0.0 and np.all(np.isnan(out))          # 0/0 in the coefficient
    J = np.full((10, 10), 2.0)
    J[:2, :] = _img(2, 10, 36)                             # only the ROI rows vary
    out, _ = oracle.srad(J, 1, 0.5, (0, 2, 0, 10))
    np.testing.assert_array_equal(out[4:], J[4:])          # flat neighbourhoods do not move


def test_srad_f32_follows_f64():
    J = _img(37, 45, 37).astype(np.float32)
    a, qa = oracle.srad(J, 4, 0.5, (0, 20, 0, 20), "f64")
    b, qb = oracle.srad(J, 4, 0.5, (0, 20, 0, 20), "f32")
    np.testing.assert_allclose(b, a, rtol=2e-6, atol=0)
    np.testing.assert_allclose(qb, qa, rtol=1e-6)


def test_srad_rejects_bad_roi():
    J = _img(5, 5, 38)
    for roi in ((0, 0, 0, 5), (0, 6, 0, 5), (-1, 3, 0, 5), (0, 5, 4, 2)):
        with pytest.raises(ValueError):
            oracle.srad(J, 1, 0.5, roi)


def _checkerboard_case(g, case):
    ny, nx = g["shape"]
    a, b = float(Fraction(case["a"])), float(Fraction(case["b"]))
    ii, jj = np.indices((ny, nx))
    J = np.where((ii + jj) % 2 == 0, b, a).astype(np.float64)
    if case["roi_values"] is not None:
        vals = [float(Fraction(v)) for v in case["roi_values"]]
        J[0, :len(vals)] = vals
    even = ((ii + jj) % 2 == 0)[2:ny - 2, 1:nx - 2]
    want = np.where(even, float(Fraction(case["J_b"])), float(Fraction(case["J_a"])))
    return J, want


@pytest.mark.parametrize("k", [0, 1, 2])
def test_srad_coefficient_golden(k):
    with open(os.path.join(os.path.dirname(__file__), "golden", "srad_coefficient.json")) as f:
        g = json.load(f)
    case = g["cases"][k]
    J, want = _checkerboard_case(g, case)
    lam = float(Fraction(case["lambda"]))
    q0_want = float(Fraction(case["q0sq"]))
    out, q0 = oracle.srad(J, 1, lam, case["roi"])
    ny, nx = g["shape"]
    assert abs(q0[0] - q0_want) <= 1e-14 * q0_want
    np.testing.assert_allclose(out[2:ny - 2, 1:nx - 2], want, rtol=1e-14, atol=0)
    out32, q032 = oracle.srad(J.astype(np.float32), 1, lam, case["roi"], "f32")
    assert abs(float(q032[0]) - q0_want) <= 2 ** -24 * q0_want
    np.testing.assert_allclose(out32[2:ny - 2, 1:nx - 2], want, rtol=1e-6, atol=0)
