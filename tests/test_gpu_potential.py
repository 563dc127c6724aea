"""The potential (kind = "potential"; the method carried over to Phi, which
the paper's Sec. 6 says applies): the CUDA builder's cells and folded kernel
against the oracle's table, Phi against the oracle (FP64 within 1e-12
relative L2, FP32 within 1e-5), the adjoint, one-sided radial edges, the
Kuzmin disk's second order through the library, and the option checks."""
import math

import numpy as np
import pytest

import workloads
from tests.errbounds import assert_close, assert_close_1
from oracle import analytic as A

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01450_gb300 import build

    build.build()
    return torch


def _setup(oracle_mod, nu, nphi, r_in, r_out, dtype, **kw):
    from paper_1509_01450_gb300 import Plan

    u_min, du = workloads.grid_params(nu, r_in, r_out)
    plan = Plan(nu, nphi, u_min, du, 1.0, dtype).build(kind="potential", **kw)
    return plan, oracle_mod.Grid(nu, nphi, u_min, du), du


def _sigma(grid, seed):
    return workloads.spiral_clump(grid.r, grid.phi) + 0.05 * np.abs(workloads.random_field(grid.nu, grid.nphi, seed))


@pytest.mark.parametrize("nu,nphi", [(4, 8), (16, 64), (64, 32), (128, 128)])
def test_cells_and_folded_kernel(torch_cuda, oracle_mod, nu, nphi):
    plan, grid, du = _setup(oracle_mod, nu, nphi, 0.05, 20.0, "float64")
    assert plan.build_report() == (0, 0, 0, 0)
    ref = oracle_mod.potential_cells(nu, nphi, du)
    got = plan.cells()
    scale = np.abs(ref[0]) + 1e-3 * np.abs(ref[0]).max()
    for c in range(6):
        assert np.all(np.abs(got[c] - ref[c]) <= 2e-12 * scale), (c, np.abs(got[c] - ref[c]).max())
    K, Kz = oracle_mod.fold(ref, grid.beta, grid.dphi)
    assert not np.any(Kz)
    gK, gKz = plan.kernels()
    assert np.abs(gK - K).max() < 1e-12 * np.abs(K).max()
    assert not np.any(gKz)


@pytest.mark.parametrize("nu,nphi", [(8, 16), (32, 128), (256, 64), (128, 256)])
@pytest.mark.parametrize("dtype,tol,p", [("float64", 1e-12, 0), ("float64", 1e-12, 1), ("float64", 1e-12, 2),
                                         ("float32", 1e-5, 1)])
def test_potential_against_the_oracle(torch_cuda, oracle_mod, nu, nphi, dtype, tol, p):
    """FP32 at p = 1: the output carries r_i and the kernel grows like r'/r
    toward outer sources, so at p = 0 the transform's values span r_out /
    r_in and FP32 rounding at the outer rows reaches about 1e-5 of the norm;
    p = 1 evens both sides (about 1e-7)."""
    torch = torch_cuda
    plan, grid, du = _setup(oracle_mod, nu, nphi, 0.1, 10.0, dtype, weight_p=p)
    sigma = _sigma(grid, 4)
    ref = oracle_mod.potential(sigma, oracle_mod.potential_cells(nu, nphi, du), grid)
    Phi, Fz = plan.forces(torch.tensor(sigma, dtype=plan.dtype, device="cuda"))
    torch.cuda.synchronize()
    plan.check()
    Phi = Phi.double().cpu().numpy()
    assert_close_1(Phi, ref, tol, w=grid.r ** (p - 1.0))
    # the second output carries nothing but the rounding of the paired inverse FFT
    assert np.abs(Fz.double().cpu().numpy()).max() <= tol * np.abs(ref).max()


@pytest.mark.parametrize("dtype,tol", [("float64", 1e-12), ("float32", 1e-5)])
def test_adjoint_against_the_oracle(torch_cuda, oracle_mod, dtype, tol):
    """The transpose of Phi = diag(r) K sigma is K^T diag(r) g."""
    torch = torch_cuda
    nu, nphi = 64, 128
    plan, grid, du = _setup(oracle_mod, nu, nphi, 0.1, 10.0, dtype, weight_p=1)
    K, _ = oracle_mod.fold(oracle_mod.potential_cells(nu, nphi, du), grid.beta, grid.dphi)
    g = workloads.random_field(nu, nphi, 21)
    ref = oracle_mod.direct_sum_T(grid.r[:, None] * g, np.zeros_like(g), K, np.zeros_like(K))
    gt = torch.tensor(g, dtype=plan.dtype, device="cuda")
    gs = plan.backward(gt, torch.zeros_like(gt))
    plan.check()
    assert_close_1(gs.double().cpu().numpy(), ref, tol, w=grid.r ** -1.0)


def test_adjoint_dot_identity(torch_cuda, oracle_mod):
    torch = torch_cuda
    nu, nphi = 256, 64
    plan, grid, du = _setup(oracle_mod, nu, nphi, 0.01, 100.0, "float64")
    s = torch.tensor(workloads.random_field(nu, nphi, 1), device="cuda")
    g = torch.tensor(workloads.random_field(nu, nphi, 2), device="cuda")
    Phi, _ = plan.forces(s)
    gs = plan.backward(g, torch.zeros_like(g))
    lhs, rhs = float((g * Phi).sum()), float((gs * s).sum())
    assert abs(lhs - rhs) < 1e-12 * float((g.abs() * Phi.abs()).sum())


@pytest.mark.parametrize("dtype,tol", [("float64", 1e-12), ("float32", 1e-5)])
def test_onesided_radial_edges(torch_cuda, oracle_mod, dtype, tol):
    """radial_edges = 1: r_i times the one-sided sums over the potential's
    cells, forward and adjoint (dense matrix of the oracle's map, 8 x 16)."""
    torch = torch_cuda
    for nu, nphi in ((32, 64), (128, 32)):
        plan, grid, du = _setup(oracle_mod, nu, nphi, 0.1, 10.0, dtype, radial_edges=1, weight_p=1)
        cells = oracle_mod.potential_cells(nu, nphi, du)
        sigma = _sigma(grid, 7)
        ref = grid.r[:, None] * oracle_mod.onesided_forces(sigma, cells, grid)[0]
        Phi, _ = plan.forces(torch.tensor(sigma, dtype=plan.dtype, device="cuda"))
        plan.check()
        assert_close_1(Phi.double().cpu().numpy(), ref, tol)
    nu, nphi = 8, 16
    plan, grid, du = _setup(oracle_mod, nu, nphi, 0.1, 10.0, dtype, radial_edges=1, weight_p=1)
    cells = oracle_mod.potential_cells(nu, nphi, du)
    n = nu * nphi
    M = np.zeros((n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        M[:, c] = (grid.r[:, None] * oracle_mod.onesided_forces(e.reshape(nu, nphi), cells, grid)[0]).ravel()
    g = workloads.random_field(nu, nphi, 13)
    ref = (M.T @ g.ravel()).reshape(nu, nphi)
    gt = torch.tensor(g, dtype=plan.dtype, device="cuda")
    gs = plan.backward(gt, torch.zeros_like(gt))
    plan.check()
    assert_close_1(gs.double().cpu().numpy(), ref, tol, w=grid.r ** -1.0)


def test_kuzmin_second_order_through_the_library(torch_cuda):
    """FP64 Phi of a Kuzmin disk against the closed form less the mass off
    the grid, on interior rows (0.2 <= r <= 5): second order, as the
    oracle's own pin."""
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    errs = []
    for n in (32, 64, 128):
        u_min, du = workloads.grid_params(n, 0.05, 20.0)
        r, phi = workloads.centres(n, n, u_min, du)
        plan = Plan(n, n, u_min, du, 1.0, "float64").build(kind="potential")
        Phi, _ = plan.forces(torch.tensor(workloads.kuzmin(r, phi), device="cuda"))
        m = (r >= 0.2) & (r <= 5.0)
        truth = A.kuzmin_truncated_phi(r[m], 0.05, 20.0)
        errs.append(np.abs(Phi[:, 0].cpu().numpy()[m] - truth).max() / np.abs(truth).max())
    orders = [math.log2(a / b) for a, b in zip(errs[:-1], errs[1:])]
    assert orders[-1] > 1.7 and errs[-1] < 4e-4, (errs, orders)


def test_options_and_plan_file(torch_cuda, oracle_mod, tmp_path):
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan, SgError, sg

    plan, grid, du = _setup(oracle_mod, 32, 64, 0.1, 10.0, "float32")
    with pytest.raises(SgError) as ei:
        plan.build(kind="potential", n_tpz=19)
    assert ei.value.status == sg.SG_ERR_ARG
    plan.build(kind="potential")
    s = torch.tensor(_sigma(grid, 5), dtype=torch.float32, device="cuda")
    Phi, _ = plan.forces(s)
    path = str(tmp_path / "potential_plan.bin")
    plan.save(path)
    Phi2, _ = Plan.load(path).forces(s)
    torch.cuda.synchronize()
    assert torch.equal(Phi, Phi2)
