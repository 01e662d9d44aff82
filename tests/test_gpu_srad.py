"""SRAD-style fused nest on the GPU against the oracle.

The GPU evaluates the scheme in fp32 with the coefficient multiplied through
by Jc^2 den^2, in which Jc^2 cancels: E = Jc + S1/4 (the mean of the four
neighbours) and c = E^2 / (E^2 + (S2/2 - S1^2/16 - q0^2 E^2) iq) with
iq = 1/(q0^2 (1 + q0^2)) once per iteration, each a*b + c one fused
multiply-add.  That is one division per pixel instead of the five of the
literal expression, algebraically equal and rounded differently.  It is
therefore compared with the oracle's literal evaluations within a rounding
bound derived from the scheme (first order, u = 2^-24, k = lambda/4 <= 1/4,
a positive image with values in [m, M], D = M/m; diffusion keeps every
iterate in [m, M]):

  * per iteration, the literal fp32 evaluation's local error is at most
    (1 + k (132 + 24 D)) u M: the neighbour differences (4k u M), the flux
    sum (12k u M), the update (u M + 4k u M) and the coefficients (4k M
    times their relative error, at most (28 + 6 D) u); the kernel's form has
    fewer roundings, (1 + k (94 + 16 D)) u M;
  * the update is a convex combination of a pixel and its neighbours for
    lambda <= 1, so to first order the errors of T iterations add up:
    bound(T) = T (1 + k (132 + 24 D)) u, capped at the 1e-5 of the fp32
    tolerance.

The test asserts max|GPU - f64| <= bound(T) * max|f64| and
max|GPU - f32| <= 2 bound(T) * max|f64| (both fp32 evaluations lie within
bound(T) of the f64 one).  q0^2 of the first iteration depends only on the
input and is compared bit for bit (both sides round a double to fp32 once);
later ones within 1e-5 relative of the f64 oracle.  The fused path (one
kernel per iteration) and the unfused one (three kernels) must agree bit for
bit; so must the fused kernel's vector path (interior tiles, 16-byte rows)
and its element path (edge and region tiles, and images whose rows are not
whole float4s).
"""

import numpy as np
import pytest
import torch

import oracle
import workloads

pytestmark = pytest.mark.gpu


def _run(hx, ctx, J, iters, lam, roi, fused):
    J0 = torch.from_numpy(J).cuda()
    J1 = torch.empty_like(J0)
    out, q0 = hx.hx_srad(ctx, J0, J1, iters, lam, roi, fused=fused)
    torch.cuda.synchronize()
    return out.cpu().numpy(), q0[:iters].cpu().numpy()


CASES = [((17, 23), (0, 17, 0, 23)), ((16, 128), (3, 9, 5, 100)), ((33, 257), (0, 33, 0, 257)),
         ((130, 300), (17, 129, 130, 299)), ((1, 200), (0, 1, 10, 190)), ((200, 1), (5, 150, 0, 1)),
         ((512, 512), (0, 128, 0, 128)),
         # interior tiles on the vector path around region tiles on the element path
         ((100, 404), (40, 60, 150, 250)),
         # a vector-path tile (rows 32..63, columns 128..255) whose last warp
         # reads the image's last row (i0 + 33 = ny - 1)
         ((66, 260), (0, 10, 0, 10))]


U = 2.0 ** -24


def bound(iters, lam, J):
    k = 0.25 * lam
    d = float(np.max(J)) / float(np.min(J))
    return min(1e-5, iters * (1.0 + k * (132.0 + 24.0 * d)) * U)


def _check_against_oracle(got, q0, J, iters, lam, roi):
    ref32, q32 = oracle.srad(J, iters, lam, roi, "f32")
    ref64, q64 = oracle.srad(J, iters, lam, roi, "f64")
    scale = np.max(np.abs(ref64))
    b = bound(iters, lam, J)
    assert np.max(np.abs(got.astype(np.float64) - ref64)) <= b * scale
    assert np.max(np.abs(got.astype(np.float64) - ref32)) <= 2 * b * scale
    if iters:
        assert q0[0] == q32[0]
        np.testing.assert_allclose(q0.astype(np.float64), q64, rtol=1e-5, atol=0)


@pytest.mark.parametrize("shape,roi", CASES)
@pytest.mark.parametrize("iters", [1, 3, 10])
def test_srad_matches_oracle(gpu, shape, roi, iters):
    hx = gpu
    J = workloads.srad_image(*shape)
    lam = 0.5
    with hx.hx_create(0) as ctx:
        fused, qf = _run(hx, ctx, J, iters, lam, roi, True)
        unfused, qu = _run(hx, ctx, J, iters, lam, roi, False)
    _check_against_oracle(fused, qf, J, iters, lam, roi)
    np.testing.assert_array_equal(unfused.view(np.uint32), fused.view(np.uint32))
    np.testing.assert_array_equal(qu.view(np.uint32), qf.view(np.uint32))


@pytest.mark.parametrize("lam", [0.25, 1.0])
def test_srad_other_step_sizes(gpu, lam):
    hx = gpu
    J = workloads.srad_image(130, 300)
    roi = (17, 129, 130, 299)
    with hx.hx_create(0) as ctx:
        fused, qf = _run(hx, ctx, J, 5, lam, roi, True)
    _check_against_oracle(fused, qf, J, 5, lam, roi)


def test_srad_zero_iterations_and_homogeneous_region(gpu):
    hx = gpu
    with hx.hx_create(0) as ctx:
        J = workloads.srad_image(20, 30)
        out, _ = _run(hx, ctx, J, 0, 0.5, (0, 20, 0, 30), True)
        np.testing.assert_array_equal(out, J)
        flat = np.full((20, 30), 1.75, dtype=np.float32)
        for fused in (True, False):
            out, q0 = _run(hx, ctx, flat, 2, 0.5, (0, 20, 0, 30), fused)
            assert q0[0] == 0.0 and np.all(np.isnan(out))


def test_srad_rejects_bad_arguments(gpu):
    hx = gpu
    with hx.hx_create(0) as ctx:
        J0 = torch.ones(16, 16, device="cuda:0")
        J1 = torch.empty_like(J0)
        for roi in ((0, 0, 0, 16), (0, 17, 0, 16), (4, 2, 0, 16), (0, 16, -1, 3)):
            with pytest.raises(hx.HxError):
                hx.hx_srad(ctx, J0, J1, 1, 0.5, roi)
        with pytest.raises(hx.HxError):
            hx.hx_srad(ctx, J0, J0, 1, 0.5, (0, 16, 0, 16))          # in place
        with pytest.raises(hx.HxError):
            hx.hx_srad(ctx, J0, J1, 1, 0.5, (0, 16, 0, 16), fused=False, C=J1)


def test_srad_full_size_one_iteration(gpu):
    # the bench's image size: 8192 x 8192, Rodinia-style 128 x 128 region
    hx = gpu
    ny = nx = 8192
    roi = (0, 128, 0, 128)
    J = workloads.srad_image(ny, nx)
    with hx.hx_create(0) as ctx:
        J0 = torch.from_numpy(J).cuda()
        J1 = torch.empty_like(J0)
        out, q0 = hx.hx_srad(ctx, J0, J1, 1, 0.5, roi)
        torch.cuda.synchronize()
        got = out.cpu().numpy()
        _check_against_oracle(got, q0[:1].cpu().numpy(), J, 1, 0.5, roi)
        # flux conservation at any size (fp32 rounding per pixel only)
        tot_in = float(np.sum(J, dtype=np.float64))
        tot_out = float(out.double().sum().item())
        assert abs(tot_out - tot_in) <= 1e-6 * tot_in


@pytest.mark.parametrize("ny,nx,roi", [(96, 520, (0, 16, 0, 128)), (66, 260, (0, 10, 0, 10))])
def test_srad_vector_and_element_paths_agree(gpu, ny, nx, roi):
    # the same image with 16-byte aligned rows (vector path on interior tiles)
    # and at a 4-byte offset (element path everywhere)
    hx = gpu
    J = workloads.srad_image(ny, nx)
    with hx.hx_create(0) as ctx:
        outs = []
        for off in (0, 1):
            buf = torch.empty(2 * ny * nx + 8, device="cuda:0")
            J0 = buf[off: off + ny * nx].view(ny, nx)
            J1 = buf[ny * nx + 4 + off: ny * nx + 4 + off + ny * nx].view(ny, nx)
            J0.copy_(torch.from_numpy(J))
            out, _ = hx.hx_srad(ctx, J0, J1, 3, 0.5, roi)
            torch.cuda.synchronize()
            outs.append(out.cpu().numpy())
    np.testing.assert_array_equal(outs[1].view(np.uint32), outs[0].view(np.uint32))
    ref64, _ = oracle.srad(J, 3, 0.5, roi, "f64")
    assert np.max(np.abs(outs[0] - ref64)) <= bound(3, 0.5, J) * np.max(np.abs(ref64))
