"""The Cartesian second-order scheme (kind = "cartesian"; Sec. 3.1.1 with the
closed forms of App. A) through the library: the folded kernels against the
oracle's, F^x, F^y against the oracle's zero-padded convolution (FP64 within
1e-12 relative L2, FP32 within 1e-5), the adjoint, the convergence orders
on an off-centre sigma_{D_5} disk, and the option checks.  The plan's
columns are 2 N_y: sigma is zero in the last N_y, whose outputs are not
compared."""
import math

import numpy as np
import pytest
from tests.errbounds import assert_close, assert_close_1

from oracle import analytic as A
from oracle import cartesian as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01450_gb300 import build

    build.build()
    return torch


def _plan(nx, ny, h, dtype):
    from paper_1509_01450_gb300 import Plan

    return Plan(nx, 2 * ny, 0.0, h, 1.0, dtype).build(kind="cartesian")


def _padded(a, ny):
    out = np.zeros((a.shape[0], 2 * ny))
    out[:, :ny] = a
    return out


def _sigma(nx, ny, seed):
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx - 0.5
    y = (np.arange(ny) + 0.5) / ny - 0.5
    return np.exp(-8 * (x[:, None] ** 2 + (y[None, :] - 0.1) ** 2)) + 0.05 * rng.random((nx, ny))


@pytest.mark.parametrize("nx,ny", [(4, 2), (8, 8), (16, 32), (64, 16)])
def test_folded_kernels(torch_cuda, nx, ny):
    h = 1.0 / max(nx, ny)
    plan = _plan(nx, ny, h, "float64")
    assert plan.build_report() == (0, 0, 0, 0)
    Kx, Ky = C.fold(C.cells(nx, ny, h), h)
    gKx, gKy = plan.kernels()
    # offset q lands at q mod 2 N_y; column N_y stays zero
    cols = np.arange(-(ny - 1), ny) % (2 * ny)
    for g, ref in ((gKx, Kx), (gKy, Ky)):
        assert np.abs(g[:, cols] - ref).max() < 1e-12 * np.abs(ref).max()
        assert not np.any(g[:, ny])
    assert not np.any(plan.cells())


@pytest.mark.parametrize("nx,ny", [(4, 2), (8, 16), (32, 64), (256, 64), (64, 512)])
@pytest.mark.parametrize("dtype,tol", [("float64", 1e-12), ("float32", 1e-5)])
def test_forces_against_the_oracle(torch_cuda, nx, ny, dtype, tol):
    torch = torch_cuda
    h = 1.0 / max(nx, ny)
    plan = _plan(nx, ny, h, dtype)
    sigma = _sigma(nx, ny, 3)
    Fx_r, Fy_r = C.forces(sigma, *C.fold(C.cells(nx, ny, h), h))
    s = torch.tensor(_padded(sigma, ny), dtype=plan.dtype, device="cuda")
    Fx, Fy = plan.forces(s)
    torch.cuda.synchronize()
    plan.check()
    Fx = Fx.double().cpu().numpy()[:, :ny]
    Fy = Fy.double().cpu().numpy()[:, :ny]
    num = np.sum((Fx - Fx_r) ** 2) + np.sum((Fy - Fy_r) ** 2)
    den = np.sum(Fx_r ** 2) + np.sum(Fy_r ** 2)
    assert math.sqrt(num / den) < tol


@pytest.mark.parametrize("dtype,tol", [("float64", 1e-12), ("float32", 1e-5)])
def test_adjoint_against_the_oracle(torch_cuda, dtype, tol):
    """With the upstream gradients zero in the padding, the adjoint's first
    N_y columns are the transposed Cartesian map: correlations with the
    folded kernels."""
    torch = torch_cuda
    nx, ny = 32, 64
    h = 1.0 / 64
    plan = _plan(nx, ny, h, dtype)
    Kx, Ky = C.fold(C.cells(nx, ny, h), h)
    rng = np.random.default_rng(11)
    gx, gy = rng.standard_normal((nx, ny)), rng.standard_normal((nx, ny))
    flip = lambda K: K[::-1, ::-1]
    ref = C.forces(gx, flip(Kx), flip(Ky))[0] + C.forces(gy, flip(Kx), flip(Ky))[1]
    gs = plan.backward(torch.tensor(_padded(gx, ny), dtype=plan.dtype, device="cuda"),
                       torch.tensor(_padded(gy, ny), dtype=plan.dtype, device="cuda"))
    plan.check()
    got = gs.double().cpu().numpy()[:, :ny]
    assert_close_1(got, ref, tol)


def test_dn5_second_order_through_the_library(torch_cuda):
    """sigma_{D_5} (alpha = 0.25) centred at (0.1, -0.05) in [-0.5, 0.5]^2:
    FP64 forces of the library, maximum error at second order."""
    torch = torch_cuda
    alpha, xc, yc, M = 0.25, 0.1, -0.05, 0.5
    errs = []
    for n in (64, 128, 256):
        h = 2 * M / n
        x = -M + (np.arange(n) + 0.5) * h
        X, Y = x[:, None] - xc, x[None, :] - yc
        d = np.hypot(X, Y)
        f = A.dn_force(5, (d / alpha).ravel()).reshape(d.shape)
        plan = _plan(n, n, h, "float64")
        Fx, Fy = plan.forces(torch.tensor(_padded(A.dn_sigma(5, d / alpha), n), device="cuda"))
        Fx, Fy = Fx.cpu().numpy()[:, :n], Fy.cpu().numpy()[:, :n]
        errs.append(max(np.abs(Fx - f * X / d).max(), np.abs(Fy - f * Y / d).max()) / np.abs(f).max())
    order = math.log2(errs[-2] / errs[-1])
    assert order > 1.8 and errs[-1] < 3e-4, (errs, order)


def test_options(torch_cuda):
    from paper_1509_01450_gb300 import Plan, SgError, sg

    plan = Plan(16, 32, 0.0, 0.05, 1.0, "float32")
    for kw in ({"weight_p": 1}, {"radial_edges": 1}, {"n_tpz": 3}):
        with pytest.raises(SgError) as ei:
            plan.build(kind="cartesian", **kw)
        assert ei.value.status == sg.SG_ERR_ARG
