"""The fused FP32 configurations at large sizes, against the FP64 oracle.

- the origin wedge (Sec. 3.2.1, third terms of Eq. 27-29) with its update
  inside the column pass, at 1024 x 2048 and 2048 x 4096, on sampled target
  cells (the oracle's one-sided direct sums plus its wedge sums, one target
  at a time), and its adjoint by the dot identity at the same sizes;
- the one-sided radial edge update inside the column passes at N_u = 4096
  (8192-point columns), forward and adjoint against the oracle's whole
  field, with and without the wedge;
- the largest FP32 plan, 4096 x 8192, forward and adjoint on sampled target
  and source cells (direct sums over the oracle's kernel table).

Every comparison carries the global relative L2 bound and the local bounds
of tests/errbounds.py."""
import math

import numpy as np
import pytest

import workloads
from tests.errbounds import assert_close, assert_close_1

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01450_gb300 import build

    build.build()
    return torch


def _targets(nu, nphi, n, seed):
    """n random flat cells plus the corners and cells of the first two and
    the last two rows, where the edge and wedge terms act."""
    rng = np.random.default_rng(seed)
    t = rng.choice(nu * nphi, n, replace=False)
    j = rng.integers(0, nphi, 4)
    edge = [0, nphi - 1, (nu - 1) * nphi, nu * nphi - 1, j[0], nphi + j[1], (nu - 2) * nphi + j[2],
            (nu - 1) * nphi + j[3]]
    return np.unique(np.concatenate([t, edge]))


def _wedge_inputs(grid, seed):
    sigma = workloads.spiral_clump(grid.r, grid.phi) + 0.05 * np.abs(workloads.random_field(grid.nu, grid.nphi, seed))
    sigma_w = 0.5 + np.random.default_rng(seed).random(grid.nphi)
    return sigma, sigma_w


def _dot_identity(torch, plan, sigma, sigma_w, seed):
    """<g, A x> = <A^T g, x> over (sigma, sigma_w), in FP64 sums of the FP32
    fields, relative to |g| |A x|."""
    g = torch.Generator(device="cuda").manual_seed(seed)
    s = torch.tensor(sigma, dtype=torch.float32, device="cuda")
    sw = torch.tensor(sigma_w, dtype=torch.float32, device="cuda")
    Fr, Fp = plan.forces_wedge(s, sw)
    gr = torch.randn(Fr.shape, device="cuda", generator=g)
    gp = torch.randn(Fr.shape, device="cuda", generator=g)
    gs, gsw = plan.backward_wedge(gr, gp)
    plan.check()
    d = lambda a: a.double()
    lhs = float((d(gr) * d(Fr)).sum() + (d(gp) * d(Fp)).sum())
    rhs = float((d(gs) * d(s)).sum() + (d(gsw) * d(sw)).sum())
    scale = math.sqrt(float((d(gr) ** 2).sum() + (d(gp) ** 2).sum())) * math.sqrt(
        float((d(Fr) ** 2).sum() + (d(Fp) ** 2).sum()))
    assert abs(lhs - rhs) <= TOL * scale


@pytest.mark.parametrize("nu,nphi", [(1024, 2048), (2048, 4096)])
def test_fp32_wedge_sampled_targets(torch_cuda, oracle_mod, nu, nphi):
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    u_min, du = workloads.grid_params(nu, 0.1, 10.0)
    plan = Plan(nu, nphi, u_min, du, 1.0, "float32").build(radial_edges=1, wedge=1)
    assert plan.build_report() == (0, 0, 0, 0)
    grid = oracle_mod.Grid(nu, nphi, u_min, du)
    sigma, sigma_w = _wedge_inputs(grid, 5)
    t = _targets(nu, nphi, 192, nu)
    cells = oracle_mod.kernel_cells(nu, nphi, du)
    wcells = oracle_mod.wedge_cells(nu, nphi, du)
    Fr_ref, Fp_ref = oracle_mod.wedge_forces_at(sigma, sigma_w, cells, wcells, grid, t)
    del cells, wcells
    Fr, Fp = plan.forces_wedge(torch.tensor(sigma, dtype=torch.float32, device="cuda"),
                               torch.tensor(sigma_w, dtype=torch.float32, device="cuda"))
    plan.check()
    assert_close(Fr.double().cpu().numpy().ravel()[t], Fp.double().cpu().numpy().ravel()[t], Fr_ref, Fp_ref, TOL)
    _dot_identity(torch, plan, sigma, sigma_w, 7)


@pytest.mark.parametrize("wedge", [0, 1])
def test_edge_fused_columns_at_4096_rows(torch_cuda, oracle_mod, wedge):
    """4096 x 256 on r in [0.01, 100]: the radial edge update (and the wedge
    update) run inside the 8192-point column passes; the forward against the
    oracle's whole field, the adjoint (edges only) against its transpose, the
    wedge adjoint by the dot identity."""
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    nu, nphi = 4096, 256
    u_min, du = workloads.grid_params(nu, 0.01, 100.0)
    plan = Plan(nu, nphi, u_min, du, 1.0, "float32").build(radial_edges=1, wedge=wedge)
    assert plan.build_report() == (0, 0, 0, 0)
    grid = oracle_mod.Grid(nu, nphi, u_min, du)
    cells = oracle_mod.kernel_cells(nu, nphi, du)
    sigma, sigma_w = _wedge_inputs(grid, 9)
    s = torch.tensor(sigma, dtype=torch.float32, device="cuda")
    if wedge:
        Fr_ref, Fp_ref = oracle_mod.wedge_forces(sigma, sigma_w, cells, oracle_mod.wedge_cells(nu, nphi, du), grid)
        Fr, Fp = plan.forces_wedge(s, torch.tensor(sigma_w, dtype=torch.float32, device="cuda"))
    else:
        Fr_ref, Fp_ref = oracle_mod.onesided_forces(sigma, cells, grid)
        Fr, Fp = plan.forces(s)
    plan.check()
    assert_close(Fr.double().cpu().numpy(), Fp.double().cpu().numpy(), Fr_ref, Fp_ref, TOL)
    if wedge:
        _dot_identity(torch, plan, sigma, sigma_w, 11)
        return
    gr, gp = workloads.random_field(nu, nphi, 12), workloads.random_field(nu, nphi, 13)
    ref = oracle_mod.onesided_forces_T(gr, gp, cells, grid)
    gs = plan.backward(torch.tensor(gr, dtype=torch.float32, device="cuda"),
                       torch.tensor(gp, dtype=torch.float32, device="cuda"))
    plan.check()
    assert_close_1(gs.double().cpu().numpy(), ref, TOL)


def test_max_fp32_sampled_targets_and_sources(torch_cuda, oracle_mod):
    """4096 x 8192 on r in [0.01, 100] (512-thread row and column blocks,
    8192-point transforms both ways): sampled forward targets and adjoint
    sources against the direct sums over the oracle's kernel table."""
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    cfg = workloads.Config("max-fp32", 4096, 8192, 0.01, 100.0)
    nu, nphi = cfg.nu, cfg.nphi
    plan = Plan(nu, nphi, cfg.u_min, cfg.du, 1.0, "float32").build()
    assert plan.build_report() == (0, 0, 0, 0)
    r, phi = cfg.centres()
    sigma = workloads.lognormal_disk(r, phi, 4096)
    cells = oracle_mod.kernel_cells(nu, nphi, cfg.du)
    Kr, Kp = oracle_mod.fold(cells, math.exp(cfg.du), 2 * math.pi / nphi)
    del cells
    t = _targets(nu, nphi, 160, 1)
    Fr_ref, Fp_ref = oracle_mod.direct_sum(sigma, Kr, Kp, targets=t)
    Fr, Fp = plan.forces(torch.tensor(sigma, dtype=torch.float32, device="cuda"))
    plan.check()
    assert_close(Fr.double().cpu().numpy().ravel()[t], Fp.double().cpu().numpy().ravel()[t], Fr_ref, Fp_ref, TOL)
    del Fr, Fp
    gr, gp = workloads.random_field(nu, nphi, 21), workloads.random_field(nu, nphi, 22)
    src = _targets(nu, nphi, 160, 2)
    ref = oracle_mod.direct_sum_T(gr, gp, Kr, Kp, sources=src)
    gs = plan.backward(torch.tensor(gr, dtype=torch.float32, device="cuda"),
                       torch.tensor(gp, dtype=torch.float32, device="cuda"))
    plan.check()
    assert_close_1(gs.double().cpu().numpy().ravel()[src], ref, TOL)
