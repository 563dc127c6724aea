"""One-sided radial slopes at the grid's first and last rows (radial_edges =
1): the library's forward and adjoint against the oracle's one-sided sums
(FP64 within 1e-12 relative L2, FP32 within 1e-5), the full-grid second
order it restores on a Kuzmin disk, and the entry points that share the
forward passes."""
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


def _setup(oracle_mod, nu, nphi, r_in, r_out, dtype, p=0, **kw):
    from paper_1509_01450_gb300 import Plan

    u_min, du = workloads.grid_params(nu, r_in, r_out)
    plan = Plan(nu, nphi, u_min, du, 1.0, dtype).build(weight_p=p, radial_edges=1, **kw)
    grid = oracle_mod.Grid(nu, nphi, u_min, du)
    return plan, grid, u_min, du


@pytest.mark.parametrize("nu,nphi", [(4, 8), (8, 16), (16, 8), (32, 64), (64, 32), (256, 64), (128, 256)])
@pytest.mark.parametrize("dtype,tol,p", [("float64", 1e-12, 0), ("float64", 1e-12, 2), ("float32", 1e-5, 0)])
def test_forward_against_the_oracle(torch_cuda, oracle_mod, nu, nphi, dtype, tol, p):
    torch = torch_cuda
    plan, grid, u_min, du = _setup(oracle_mod, nu, nphi, 0.1, 10.0, dtype, p)
    cells = oracle_mod.kernel_cells(nu, nphi, du)
    r, phi = grid.r, grid.phi
    sigma = workloads.spiral_clump(r, phi) + 0.05 * np.abs(workloads.random_field(nu, nphi, 4))
    Fr_ref, Fp_ref = oracle_mod.onesided_forces(sigma, cells, grid)
    Fr, Fp = plan.forces(torch.tensor(sigma, dtype=plan.dtype, device="cuda"))
    torch.cuda.synchronize()
    plan.check()
    assert_close(Fr.double().cpu().numpy(), Fp.double().cpu().numpy(), Fr_ref, Fp_ref, tol, w=grid.r ** p)


@pytest.mark.parametrize("dtype,tol", [("float64", 1e-12), ("float32", 1e-5)])
def test_adjoint_is_the_transpose_of_the_oracle_map(torch_cuda, oracle_mod, dtype, tol):
    """The dense matrix of the oracle's one-sided map on an 8 x 16 grid,
    transposed, against the library's adjoint."""
    torch = torch_cuda
    nu, nphi = 8, 16
    plan, grid, u_min, du = _setup(oracle_mod, nu, nphi, 0.1, 10.0, dtype, 1)
    cells = oracle_mod.kernel_cells(nu, nphi, du)
    n = nu * nphi
    M = np.zeros((2 * n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        fr, fp = oracle_mod.onesided_forces(e.reshape(nu, nphi), cells, grid)
        M[:n, c], M[n:, c] = fr.ravel(), fp.ravel()
    gr, gp = workloads.random_field(nu, nphi, 11), workloads.random_field(nu, nphi, 12)
    ref = (M.T @ np.concatenate([gr.ravel(), gp.ravel()])).reshape(nu, nphi)
    gs = plan.backward(torch.tensor(gr, dtype=plan.dtype, device="cuda"),
                       torch.tensor(gp, dtype=plan.dtype, device="cuda"))
    plan.check()
    assert_close_1(gs.double().cpu().numpy(), ref, tol, w=grid.r ** -1.0)


@pytest.mark.parametrize("nu,nphi,r_in,r_out,p", [(64, 128, 0.01, 100.0, 0), (256, 64, 0.01, 100.0, 0),
                                                  (128, 64, 0.1, 10.0, 1)])
def test_adjoint_dot_identity(torch_cuda, oracle_mod, nu, nphi, r_in, r_out, p):
    """(p > 0 amplifies FP64 rounding by the spread of beta^{pk}, as for the
    convolution itself, so the wide grid is checked at p = 0.)"""
    torch = torch_cuda
    plan, grid, u_min, du = _setup(oracle_mod, nu, nphi, r_in, r_out, "float64", p)
    s = torch.tensor(workloads.random_field(nu, nphi, 1), device="cuda")
    gr = torch.tensor(workloads.random_field(nu, nphi, 2), device="cuda")
    gp = torch.tensor(workloads.random_field(nu, nphi, 3), device="cuda")
    Fr, Fp = plan.forces(s)
    gs = plan.backward(gr, gp)
    lhs = float((gr * Fr).sum() + (gp * Fp).sum())
    rhs = float((gs * s).sum())
    assert abs(lhs - rhs) < 1e-12 * float((gr.abs() * Fr.abs()).sum() + (gp.abs() * Fp.abs()).sum())


def test_kuzmin_full_grid_second_order(torch_cuda, oracle_mod):
    """The ghost rows' fictitious dipole at r_in keeps the full-grid error of
    the convolution at O(1); one-sided edge slopes converge at second order
    everywhere (FP64 forces of the library)."""
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    errs = {0: [], 1: []}
    for n in (32, 64, 128):
        u_min, du = workloads.grid_params(n, 0.05, 20.0)
        r, phi = workloads.centres(n, n, u_min, du)
        truth = A.kuzmin_truncated_Fr(r, 0.05, 20.0)
        s = torch.tensor(workloads.kuzmin(r, phi), device="cuda")
        for edges in (0, 1):
            plan = Plan(n, n, u_min, du, 1.0, "float64").build(radial_edges=edges)
            Fr, _ = plan.forces(s)
            errs[edges].append(np.abs(Fr[:, 0].cpu().numpy() - truth).max())
    assert math.log2(errs[1][-2] / errs[1][-1]) > 1.7 and errs[1][-1] < 1e-4, errs
    assert errs[0][-1] > 0.1, errs


def test_other_entry_points_and_kinds(torch_cuda, oracle_mod):
    torch = torch_cuda
    from paper_1509_01450_gb300 import SgError, forces_batched, sg

    nu, nphi = 32, 64
    plan, grid, u_min, du = _setup(oracle_mod, nu, nphi, 0.1, 10.0, "float32")
    sigma = workloads.spiral_clump(grid.r, grid.phi)
    s = torch.tensor(sigma, dtype=torch.float32, device="cuda")
    Fr, Fp = plan.forces(s)
    # batched and allocation-free forms run the same passes
    fr2, fp2 = torch.empty_like(s), torch.empty_like(s)
    forces_batched([(plan, s, fr2, fp2)])
    torch.cuda.synchronize()
    assert torch.equal(Fr, fr2) and torch.equal(Fp, fp2)
    fr3, fp3 = torch.empty_like(s), torch.empty_like(s)
    plan.forces_noalloc(s, fr3, fp3)
    torch.cuda.synchronize()
    assert torch.equal(Fr, fr3) and torch.equal(Fp, fp3)
    # the file format holds no edge tables
    with pytest.raises(SgError) as ei:
        plan.save("/tmp/sg_edges_plan.bin")
    assert ei.value.status == sg.SG_ERR_UNSUPPORTED
    with pytest.raises(SgError) as ei:
        plan.build(radial_edges=2)
    assert ei.value.status == sg.SG_ERR_ARG
    # the modified particle method with one-sided slopes: the same correction
    # over that kind's own slope kernels
    plan2, grid, u_min, du = _setup(oracle_mod, nu, nphi, 0.1, 10.0, "float64", 0, kind="particle+")
    cells = oracle_mod.particle_cells(nu, nphi, du, "particle+")
    Fr_ref, Fp_ref = oracle_mod.onesided_forces(sigma, cells, grid)
    Fr, Fp = plan2.forces(torch.tensor(sigma, device="cuda"))
    assert_close(Fr.cpu().numpy(), Fp.cpu().numpy(), Fr_ref, Fp_ref, 1e-12)
    # and rebuilt without, the plain convolution again
    plan2.build(kind="particle+")
    Kr, Kp = oracle_mod.fold(cells, grid.beta, grid.dphi)
    Fr_ref, Fp_ref = oracle_mod.direct_sum(sigma, Kr, Kp)
    Fr, Fp = plan2.forces(torch.tensor(sigma, device="cuda"))
    assert_close(Fr.cpu().numpy(), Fp.cpu().numpy(), Fr_ref, Fp_ref, 1e-12)


@pytest.mark.parametrize("nu,nphi", [(256, 64), (512, 128), (2048, 32)])
def test_fp32_adjoint_with_the_update_in_the_column_pass(torch_cuda, oracle_mod, nu, nphi):
    """FP32 columns of 512 points or more apply the transposed edge update
    inside the adjoint's column pass; the FP64 adjoint (the separate kernel,
    pinned to the oracle's transposed map above) is the reference."""
    torch = torch_cuda
    p32, grid, u_min, du = _setup(oracle_mod, nu, nphi, 0.1, 10.0, "float32", 1)
    p64, _, _, _ = _setup(oracle_mod, nu, nphi, 0.1, 10.0, "float64", 1)
    gr, gp = workloads.random_field(nu, nphi, 31), workloads.random_field(nu, nphi, 32)
    g32 = p32.backward(torch.tensor(gr, dtype=torch.float32, device="cuda"),
                       torch.tensor(gp, dtype=torch.float32, device="cuda"))
    g64 = p64.backward(torch.tensor(gr, device="cuda"), torch.tensor(gp, device="cuda"))
    p32.check()
    ref = g64.cpu().numpy()
    assert_close_1(g32.double().cpu().numpy(), ref, 1e-5, w=grid.r ** -1.0)
    # and the FP32 forward and adjoint are each other's transpose
    s = torch.tensor(workloads.random_field(nu, nphi, 33), dtype=torch.float32, device="cuda")
    Fr, Fp = p32.forces(s)
    lhs = float((torch.tensor(gr, device="cuda") * Fr.double()).sum() + (torch.tensor(gp, device="cuda") * Fp.double()).sum())
    rhs = float((g32.double() * s.double()).sum())
    scale = float((torch.tensor(gr, device="cuda").abs() * Fr.double().abs()).sum())
    assert abs(lhs - rhs) < 1e-5 * scale
