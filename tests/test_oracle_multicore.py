"""The host (multicore) schedule against the sequential oracle.

Integer and max reductions and every map value must match exactly for any
thread count, including more threads than elements or rows; the fp64 sum may
differ from the sequential fold by rounding only.
"""

import numpy as np
import pytest

import oracle
import workloads
from oracle import multicore


@pytest.mark.parametrize("threads", [1, 3, 8, 64])
@pytest.mark.parametrize("n", [0, 1, 5, 1000, 100_003])
def test_map_reduce(threads, n):
    x, y = workloads.map_reduce_inputs(max(n, 1))
    x, y = x[:n], y[:n]
    out_s, s_s = oracle.map_reduce(x, y, 1.5)
    out_m, s_m = multicore.map_reduce(x, y, 1.5, threads)
    np.testing.assert_array_equal(out_m, out_s)
    assert abs(s_m - s_s) <= 1e-13 * max(1.0, float(np.abs(out_s).sum()))


@pytest.mark.parametrize("threads", [1, 2, 7, 300 // 3])
def test_histogram(threads):
    for v in (workloads.histogram_mixture_u8(200_001), np.zeros(0, np.uint8), np.full(17, 9, np.uint8)):
        b_s, sc_s = oracle.histogram(v)
        b_m, sc_m = multicore.histogram(v, threads)
        np.testing.assert_array_equal(b_m, b_s)
        np.testing.assert_array_equal(sc_m, sc_s)


@pytest.mark.parametrize("threads", [1, 4, 9])
@pytest.mark.parametrize("shape", [(1, 1), (3, 5), (37, 64), (130, 33)])
def test_jacobi(threads, shape):
    u0 = workloads.stencil_grid(*shape).astype(np.float64)
    for iters in (0, 1, 4):
        u_s, r_s = oracle.jacobi(u0, iters)
        u_m, r_m = multicore.jacobi(u0, iters, threads)
        np.testing.assert_array_equal(u_m, u_s)
        np.testing.assert_array_equal(r_m, r_s)


def test_bad_thread_counts():
    x = np.zeros(4, np.float32)
    for t in (0, -1, 257):
        with pytest.raises(RuntimeError):
            multicore.map_reduce(x, x, 1.0, t)
        with pytest.raises(RuntimeError):
            multicore.histogram(np.zeros(4, np.uint8), t)
        with pytest.raises(RuntimeError):
            multicore.jacobi(np.zeros((2, 2)), 1, t)
    assert multicore.host_cores() >= 1
