"""Plant plausible mistakes in a temporary copy of the oracle; the pins must catch each.

Each mutant is compiled on the CPU from an edited copy of the oracle source,
swapped in for the real library, and run through the pin tests of the nest it
touches.  At least one pin has to fail, or the pins would not protect the
oracle against that mistake.
"""

import ctypes
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "hx_oracle.c")

MAP_PINS = [pins.test_map_reduce_golden_tiny, pins.test_map_reduce_arithmetic_series,
            pins.test_map_reduce_negative_scale_series, pins.test_map_reduce_unit_inputs_count,
            pins.test_map_reduce_exact_on_lattice]
STENCIL_PINS = [pins.test_jacobi_golden_corner_spike, pins.test_jacobi_interior_spike,
                pins.test_jacobi_linear_field_closed_form, pins.test_jacobi_matches_scipy_nearest_correlation,
                pins.test_jacobi_residual_is_max_step_change]
HIST_PINS = [pins.test_histogram_golden_tiny, pins.test_histogram_matches_bincount_and_cumsum,
             pins.test_histogram_closed_forms]

MUTANTS = {
    "map_transposed": ("double v = a * (double)x[i] + (double)y[i];",
                       "double v = a * (double)y[i] + (double)x[i];", MAP_PINS),
    "map_dropped_y": ("double v = a * (double)x[i] + (double)y[i];",
                      "double v = a * (double)x[i];", MAP_PINS),
    "map_sign": ("double v = a * (double)x[i] + (double)y[i];",
                 "double v = a * (double)x[i] - (double)y[i];", MAP_PINS),
    "map_off_by_one": ("double v = a * (double)x[i] + (double)y[i];",
                       "double v = a * (double)x[i] + (double)y[i > 0 ? i - 1 : 0];", MAP_PINS),
    "map_short_bound": ("for (int64_t i = 0; i < n; ++i) {\n        double v = a * (double)x[i] + (double)y[i];",
                        "for (int64_t i = 0; i + 1 < n; ++i) {\n        double v = a * (double)x[i] + (double)y[i];",
                        MAP_PINS),
    "stencil_periodic": ("double west  = cur[i * nx + clampi(j - 1, 0, nx - 1)];",
                         "double west  = cur[i * nx + (j - 1 + nx) % nx];", STENCIL_PINS),
    "stencil_weight": ("double v = 0.25 * ((north + south) + (west + east));",
                       "double v = 0.2 * ((north + south) + (west + east) + cur[i * nx + j]);",
                       STENCIL_PINS),
    "stencil_north_is_south": ("double north = cur[clampi(i - 1, 0, ny - 1) * nx + j];",
                               "double north = cur[clampi(i + 1, 0, ny - 1) * nx + j];", STENCIL_PINS),
    "stencil_resid_signed": ("double d = fabs(v - cur[i * nx + j]);",
                             "double d = v - cur[i * nx + j];", STENCIL_PINS),
    "hist_inclusive_scan": ("excl_scan[k] = run;\n            run = run + bins[k];",
                            "run = run + bins[k];\n            excl_scan[k] = run;", HIST_PINS),
    "hist_drop_first": ("for (int64_t i = 0; i < n; ++i) bins[v[i]]",
                        "for (int64_t i = 1; i < n; ++i) bins[v[i]]", HIST_PINS),
}


def _load_mutant(tmp_path, name, old, new):
    with open(SRC) as f:
        text = f.read()
    assert text.count(old) == 1, f"mutation anchor for {name} not unique"
    src = tmp_path / f"{name}.c"
    src.write_text(text.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                           "-o", str(so), str(src), "-lm"])
    return ctypes.CDLL(str(so))


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, monkeypatch, name):
    old, new, tests = MUTANTS[name]
    real = oracle._get()
    mutant = _load_mutant(tmp_path, name, old, new)
    for fn in ("hxo_map_reduce_f64", "hxo_monoid_reduce_f64", "hxo_jacobi_f64",
               "hxo_jacobi_f32", "hxo_histogram_u8"):
        getattr(mutant, fn).argtypes = getattr(real, fn).argtypes
        getattr(mutant, fn).restype = getattr(real, fn).restype
    monkeypatch.setattr(oracle, "_lib", mutant)
    failures = 0
    for t in tests:
        try:
            t()
        except AssertionError:
            failures += 1
    assert failures > 0, f"no pin caught mutant {name}"
