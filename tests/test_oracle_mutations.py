"""Plant plausible mistakes in a temporary copy of the oracle; the pins must catch each.

Each mutant is compiled on the CPU from an edited copy of the oracle source,
swapped in for the real library, and run through the pin tests of the nest it
touches.  At least one pin has to fail, or the pins would not protect the
oracle against that mistake.

The pins run against a mutant in a forked child process.  Some planted
mistakes make the oracle read outside its buffers (reversed strides walk past
the end of a strided input): such a read can crash the process, and whether it
does depends on where the allocator placed the buffers.  In the child a crash
counts as caught, since the mutant did not pass the pins, and it cannot end the
test run.
"""

import ctypes
import os
import signal
import subprocess
import time

import pytest

import oracle
from tests import test_oracle_nest_pins as npins
from tests import test_oracle_pins as pins
from tests import test_oracle_srad_pins as spins

SRC = os.path.join(os.path.dirname(oracle.__file__), "hx_oracle.c")

MAP_PINS = [pins.test_map_reduce_golden_tiny, pins.test_map_reduce_arithmetic_series,
            pins.test_map_reduce_negative_scale_series, pins.test_map_reduce_unit_inputs_count,
            pins.test_map_reduce_exact_on_lattice]
STENCIL_PINS = [pins.test_jacobi_golden_corner_spike, pins.test_jacobi_interior_spike,
                pins.test_jacobi_linear_field_closed_form, pins.test_jacobi_matches_scipy_nearest_correlation,
                pins.test_jacobi_residual_is_max_step_change]
F32_STENCIL_PINS = [pins.test_jacobi_f32_equals_f64_on_coarse_dyadics, pins.test_jacobi_f32_within_rounding_bound_of_f64]
MONOID_PINS = [pins.test_monoid_reduce_against_library]
SRAD32_PINS = [lambda: spins.test_srad_f32_follows_f64(),
               *(lambda k=k: spins.test_srad_coefficient_golden(k) for k in range(3))]
HIST_PINS = [pins.test_histogram_golden_tiny, pins.test_histogram_matches_bincount_and_cumsum,
             pins.test_histogram_closed_forms]

NEST_PINS = [*(lambda op=op: npins.test_nest_binary_ops_match_numpy_single(op) for op in npins.BINARY),
             *(lambda op=op: npins.test_nest_unary_ops_match_numpy_single(op) for op in npins.UNARY),
             npins.test_nest_const_and_operand_order, npins.test_nest_fma_is_one_rounding,
             npins.test_nest_row_sums_match_numpy, npins.test_nest_row_prods_match_numpy,
             lambda: npins.test_nest_row_extrema_match_numpy("max", npins.np.max),
             lambda: npins.test_nest_row_extrema_match_numpy("min", npins.np.min),
             lambda: npins.test_nest_row_arg_extrema_match_numpy("argmax", npins.np.argmax),
             lambda: npins.test_nest_row_arg_extrema_match_numpy("argmin", npins.np.argmin),
             npins.test_nest_3d_partial_reductions_match_numpy, npins.test_nest_strided_and_broadcast_inputs,
             npins.test_nest_index_op_matches_index_grid, npins.test_nest_fold_order_is_thread_id_order,
             npins.test_nest_nan_and_empty_rules, npins.test_nest_signed_zero_rules,
             npins.test_nest_min_max_ops_skip_nan, npins.test_nest_unary_ops_special_values]

SRAD_PINS = [lambda: spins.test_srad_conserves_mass(0.5, (17, 23)), spins.test_srad_transpose_symmetry,
             lambda: spins.test_srad_maximum_principle(1.0),
             lambda: spins.test_srad_is_jacobi_relaxation_where_c_clamps_to_one(0.5),
             spins.test_srad_speckle_scale_matches_numpy,
             *(lambda a=a, b=b: spins.test_srad_checkerboard_closed_form(a, b)
               for a, b in ((2.0, 1.0), (1.0, 3.0), (1.5, 1.25))),
             spins.test_srad_homogeneous_cases,
             *(lambda k=k: spins.test_srad_coefficient_golden(k) for k in range(3))]
# The coefficient mapping alone, against values worked by hand from the
# published formula (no pin that restates the formula).
SRAD_C_PINS = [lambda k=k: spins.test_srad_coefficient_golden(k) for k in range(3)]

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
    "nest_sub_swapped": ("else if (code == 5) st[sp++] = a - b;", "else if (code == 5) st[sp++] = b - a;",
                         NEST_PINS),
    "nest_fma_two_roundings": ("st[sp++] = fmaf(a, b, c);", "st[sp++] = a * b + c;", NEST_PINS),
    "nest_argmax_last_tie": ("if (!isnan(v) && (best_i < 0 || v > best)) { best = v; best_i = r; }",
                             "if (!isnan(v) && (best_i < 0 || v >= best)) { best = v; best_i = r; }", NEST_PINS),
    "nest_dims_reversed": ("for (int d = ndim - 1; d >= 0; --d) {\n                idx[d] = rem % dims[d];",
                           "for (int d = 0; d < ndim; ++d) {\n                idx[d] = rem % dims[d];", NEST_PINS),
    "nest_strides_reversed": ("off += idx[d] * strides[arg * 3 + d];",
                              "off += idx[d] * strides[arg * 3 + (ndim - 1 - d)];", NEST_PINS),
    "nest_max_init_zero": ("case 1: case 4: best = -INFINITY; break;", "case 1: case 4: best = 0.0f; break;",
                           NEST_PINS),
    "nest_sum_in_float": ("case 0: acc = acc + (double)v; break;", "case 0: acc = (float)(acc + (double)v); break;",
                          NEST_PINS),
    "nest_prod_init_zero": ("case 3: acc = 1.0; break;\n        }\n        for (int64_t r",
                            "case 3: acc = 0.0; break;\n        }\n        for (int64_t r", NEST_PINS),
    "nest_index_off_by_one": ("st[sp++] = (float)idx[arg];", "st[sp++] = (float)(idx[arg] + 1);", NEST_PINS),
    "srad_cS_self": ("T cN = cc[i * nx + j], cS = cc[is * nx + j];", "T cN = cc[i * nx + j], cS = cc[i * nx + j];",
                     SRAD_PINS),
    "srad_cE_self": ("T cW = cc[i * nx + j], cE = cc[i * nx + je];", "T cW = cc[i * nx + j], cE = cc[i * nx + j];",
                     SRAD_PINS),
    "srad_step_half": ("const T k = QUARTER * lambda;", "const T k = HALF * lambda;", SRAD_PINS),
    "srad_var_n_minus_1": ("double var = s2 / npix - mean * mean;", "double var = s2 / (npix - 1.0) - mean * mean;",
                           SRAD_PINS),
    "srad_num_sign": ("T num = HALF * G2 - SIXTEENTH * (L * L);", "T num = HALF * G2 + SIXTEENTH * (L * L);",
                      SRAD_PINS),
    "srad_den_sign": ("T den = ONE + QUARTER * L;", "T den = ONE - QUARTER * L;", SRAD_PINS),
    "srad_no_upper_clamp": ("else if (c > ONE) c = ONE;", "else if (c > ONE) c = c;", SRAD_PINS),
    "srad_G2_over_J": ("(dW * dW + dE * dE)) / (Jc * Jc);", "(dW * dW + dE * dE)) / Jc;", SRAD_PINS),
    "srad_roi_rows_from_zero": ("for (int64_t i = r0; i < r1; i++)", "for (int64_t i = 0; i < r1; i++)", SRAD_PINS),
    "srad_dS_from_north": ("T dS = cur[is * nx + j] - Jc;", "T dS = cur[clampi(i - 1, 0, ny - 1) * nx + j] - Jc;",
                           SRAD_PINS),
    "stencil_f32_north_is_south": ("float north = cur[clampi(i - 1, 0, ny - 1) * nx + j];",
                                   "float north = cur[clampi(i + 1, 0, ny - 1) * nx + j];", F32_STENCIL_PINS),
    "stencil_f32_weight": ("float v = 0.25f * (ns + we);", "float v = 0.2f * (ns + we);", F32_STENCIL_PINS),
    "stencil_f32_resid_signed": ("float d = fabsf(v - cur[i * nx + j]);", "float d = v - cur[i * nx + j];",
                                 F32_STENCIL_PINS),
    "stencil_f32_periodic": ("float west  = cur[i * nx + clampi(j - 1, 0, nx - 1)];",
                             "float west  = cur[i * nx + (j - 1 + nx) % nx];", F32_STENCIL_PINS),
    "monoid_max_init_zero": ("case 1: acc = -INFINITY; break;", "case 1: acc = 0.0; break;", MONOID_PINS),
    "monoid_min_is_max": ("case 2: acc = (v < acc) ? v : acc; break;", "case 2: acc = (v > acc) ? v : acc; break;",
                          MONOID_PINS),
    "monoid_dropped_y": ("double v = a * (double)x[i] + (y ? (double)y[i] : 0.0);", "double v = a * (double)x[i];",
                         MONOID_PINS),
    "monoid_prod_init_zero": ("case 3: acc = 1.0; break;\n    default: return 1;",
                              "case 3: acc = 0.0; break;\n    default: return 1;", MONOID_PINS),
    "nest_argmin_last_tie": ("if (!isnan(v) && (best_i < 0 || v < best)) { best = v; best_i = r; }",
                             "if (!isnan(v) && (best_i < 0 || v <= best)) { best = v; best_i = r; }", NEST_PINS),
    "nest_argmax_takes_nan": ("if (!isnan(v) && (best_i < 0 || v > best)) { best = v; best_i = r; }",
                              "if ((best_i < 0 || v > best)) { best = v; best_i = r; }", NEST_PINS),
    "nest_div_swapped": ("else if (code == 7) st[sp++] = a / b;", "else if (code == 7) st[sp++] = b / a;", NEST_PINS),
    "nest_min_op_propagates_nan": ("else if (code == 11) st[sp++] = isnan(a) ? b : (isnan(b) ? a : (b < a ? b : a));",
                                   "else if (code == 11) st[sp++] = (b < a ? b : a);", NEST_PINS),
    "nest_abs_keeps_neg_zero": ("st[sp++] = code == 9 ? -a : (code == 10 ? fabsf(a) : sqrtf(a));",
                                "st[sp++] = code == 9 ? -a : (code == 10 ? (a < 0 ? -a : a) : sqrtf(a));", NEST_PINS),
    "nest_sqrt_of_abs": ("st[sp++] = code == 9 ? -a : (code == 10 ? fabsf(a) : sqrtf(a));",
                         "st[sp++] = code == 9 ? -a : (code == 10 ? fabsf(a) : sqrtf(fabsf(a)));", NEST_PINS),
    "srad32_quarter_is_half": ("HXO_SRAD_BODY(float, 0.5f, 0.0625f, 0.25f, 1.0f, 0.0f)",
                               "HXO_SRAD_BODY(float, 0.5f, 0.0625f, 0.5f, 1.0f, 0.0f)", SRAD32_PINS),
    "srad32_sixteenth_is_eighth": ("HXO_SRAD_BODY(float, 0.5f, 0.0625f, 0.25f, 1.0f, 0.0f)",
                                   "HXO_SRAD_BODY(float, 0.5f, 0.125f, 0.25f, 1.0f, 0.0f)", SRAD32_PINS),
    "srad_c_drops_one_plus_q0sq": ("T c = ONE / (ONE + (qsq - q0sq) / (q0sq * (ONE + q0sq)));",
                                   "T c = ONE / (ONE + (qsq - q0sq) / q0sq);", SRAD_C_PINS),
    "srad_c_one_minus_q0sq": ("T c = ONE / (ONE + (qsq - q0sq) / (q0sq * (ONE + q0sq)));",
                              "T c = ONE / (ONE + (qsq - q0sq) / (q0sq * (ONE - q0sq)));", SRAD_C_PINS),
    "srad_c_half_constant": ("T c = ONE / (ONE + (qsq - q0sq) / (q0sq * (ONE + q0sq)));",
                             "T c = ONE / (ONE + HALF * (qsq - q0sq) / (q0sq * (ONE + q0sq)));", SRAD_C_PINS),
    "srad_c_sign": ("T c = ONE / (ONE + (qsq - q0sq) / (q0sq * (ONE + q0sq)));",
                    "T c = ONE / (ONE + (q0sq - qsq) / (q0sq * (ONE + q0sq)));", SRAD_C_PINS),
    "srad_c_uses_q0": ("T c = ONE / (ONE + (qsq - q0sq) / (q0sq * (ONE + q0sq)));",
                       "T c = ONE / (ONE + (qsq - q0sq) / (q0sq * q0sq * (ONE + q0sq)));", SRAD_C_PINS),
    "srad_qsq_drops_den": ("T qsq = num / (den * den);", "T qsq = num / den;", SRAD_C_PINS),
    "hist_bin_shifted": ("for (int64_t i = 0; i < n; ++i) bins[v[i]] = bins[v[i]] + 1u;",
                         "for (int64_t i = 0; i < n; ++i) bins[(uint8_t)(v[i] + 1)] = bins[(uint8_t)(v[i] + 1)] + 1u;",
                         HIST_PINS),
    "stencil_east_is_self": ("double east  = cur[i * nx + clampi(j + 1, 0, nx - 1)];",
                             "double east  = cur[i * nx + clampi(j, 0, nx - 1)];", STENCIL_PINS),
    "nest_prod_in_float": ("case 3: acc = acc * (double)v; break;", "case 3: acc = (float)(acc * (double)v); break;",
                           NEST_PINS),
    "nest_const_shifted": ("st[sp++] = consts[arg];", "st[sp++] = consts[(arg + 1) & 7];", NEST_PINS),
    "nest_min_keeps_pos_zero": ("if (v < best || (v == 0.0f && best == 0.0f && !signbit(best) && signbit(v))) best = v;",
                                "if (v < best) best = v;", NEST_PINS),
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


_ORACLE_FUNCTIONS = ("hxo_map_reduce_f64", "hxo_monoid_reduce_f64", "hxo_jacobi_f64", "hxo_jacobi_f32",
                     "hxo_histogram_u8", "hxo_fork_reduce", "hxo_srad_f64", "hxo_srad_f32")
# child exit codes
_CAUGHT, _NOT_CAUGHT, _ERROR = 0, 1, 2


def _run_pins(mutant, tests):
    """In the child: the pins against the mutant library; returns an exit code."""
    real = oracle._get()
    for fn in _ORACLE_FUNCTIONS:
        getattr(mutant, fn).argtypes = getattr(real, fn).argtypes
        getattr(mutant, fn).restype = getattr(real, fn).restype
    oracle._lib = mutant
    failures = 0
    for t in tests:
        try:
            t()
        except (AssertionError, ValueError):
            failures += 1
    return _CAUGHT if failures else _NOT_CAUGHT


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(tmp_path, name):
    old, new, tests = MUTANTS[name]
    mutant = _load_mutant(tmp_path, name, old, new)
    oracle._get()   # the real library is loaded before the fork
    pid = os.fork()
    if pid == 0:
        code = _ERROR
        try:
            code = _run_pins(mutant, tests)
        except BaseException:
            code = _ERROR
        finally:
            os._exit(code)
    deadline = time.monotonic() + 300.0
    while True:
        done, status = os.waitpid(pid, os.WNOHANG)
        if done:
            break
        if time.monotonic() > deadline:
            os.kill(pid, signal.SIGKILL)
            os.waitpid(pid, 0)
            pytest.fail(f"the pins did not finish against mutant {name}")
        time.sleep(0.005)
    if os.WIFSIGNALED(status):
        return   # the mutant crashed under the pins: caught
    code = os.WEXITSTATUS(status)
    assert code != _ERROR, f"unexpected error running the pins against mutant {name}"
    assert code == _CAUGHT, f"no pin caught mutant {name}"
