"""The origin wedge below the grid (wedge = 1; Sec. 3.2.1 and the third
terms of Eq. 27-29) through the library: the forward against the oracle's
one-sided sums plus its wedge sums (FP64 within 1e-12 relative L2, FP32
within 1e-5), the adjoint against the oracle's dense transposed map (both
gradients), the dot identity, the potential with a wedge, a Kuzmin disk held
by grid and wedge (second order), and the option checks."""
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


def _setup(oracle_mod, nu, nphi, r_in, r_out, dtype, p=0, kind="sim"):
    from paper_1509_01450_gb300 import Plan

    u_min, du = workloads.grid_params(nu, r_in, r_out)
    plan = Plan(nu, nphi, u_min, du, 1.0, dtype).build(weight_p=p, radial_edges=1, wedge=1, kind=kind)
    return plan, oracle_mod.Grid(nu, nphi, u_min, du), du


def _inputs(grid, seed):
    sigma = workloads.spiral_clump(grid.r, grid.phi) + 0.05 * np.abs(workloads.random_field(grid.nu, grid.nphi, seed))
    rng = np.random.default_rng(seed)
    sigma_w = 0.5 + rng.random(grid.nphi)
    return sigma, sigma_w


@pytest.mark.parametrize("nu,nphi", [(4, 8), (16, 64), (64, 32), (128, 256), (256, 64)])
@pytest.mark.parametrize("dtype,tol,p", [("float64", 1e-12, 0), ("float64", 1e-12, 1), ("float32", 1e-5, 0)])
def test_forward_against_the_oracle(torch_cuda, oracle_mod, nu, nphi, dtype, tol, p):
    torch = torch_cuda
    plan, grid, du = _setup(oracle_mod, nu, nphi, 0.1, 10.0, dtype, p)
    assert plan.build_report() == (0, 0, 0, 0)
    sigma, sigma_w = _inputs(grid, 4)
    Fr_ref, Fp_ref = oracle_mod.wedge_forces(sigma, sigma_w, oracle_mod.kernel_cells(nu, nphi, du),
                                             oracle_mod.wedge_cells(nu, nphi, du), grid)
    Fr, Fp = plan.forces_wedge(torch.tensor(sigma, dtype=plan.dtype, device="cuda"),
                               torch.tensor(sigma_w, dtype=plan.dtype, device="cuda"))
    torch.cuda.synchronize()
    plan.check()
    assert_close(Fr.double().cpu().numpy(), Fp.double().cpu().numpy(), Fr_ref, Fp_ref, tol, w=grid.r ** p)


@pytest.mark.parametrize("dtype,tol", [("float64", 1e-12), ("float32", 1e-5)])
def test_adjoint_is_the_transpose_of_the_oracle_map(torch_cuda, oracle_mod, dtype, tol):
    """The dense matrix of the oracle's map (sigma, sigma_w) -> (F_r, F_phi)
    on an 8 x 16 grid, transposed, against both gradients of the library."""
    torch = torch_cuda
    nu, nphi = 8, 16
    plan, grid, du = _setup(oracle_mod, nu, nphi, 0.1, 10.0, dtype, 1)
    cells, wcells = oracle_mod.kernel_cells(nu, nphi, du), oracle_mod.wedge_cells(nu, nphi, du)
    n = nu * nphi
    M = np.zeros((2 * n, n + nphi))
    for c in range(n + nphi):
        e = np.zeros(n + nphi)
        e[c] = 1.0
        fr, fp = oracle_mod.wedge_forces(e[:n].reshape(nu, nphi), e[n:], cells, wcells, grid)
        M[:n, c], M[n:, c] = fr.ravel(), fp.ravel()
    gr, gp = workloads.random_field(nu, nphi, 11), workloads.random_field(nu, nphi, 12)
    ref = M.T @ np.concatenate([gr.ravel(), gp.ravel()])
    gs, gsw = plan.backward_wedge(torch.tensor(gr, dtype=plan.dtype, device="cuda"),
                                  torch.tensor(gp, dtype=plan.dtype, device="cuda"))
    plan.check()
    got = np.concatenate([gs.double().cpu().numpy().ravel(), gsw.double().cpu().numpy()])
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < tol
    assert np.linalg.norm(got[n:] - ref[n:]) / np.linalg.norm(ref[n:]) < 10 * tol


def test_adjoint_dot_identity(torch_cuda, oracle_mod):
    torch = torch_cuda
    nu, nphi = 256, 64
    plan, grid, du = _setup(oracle_mod, nu, nphi, 0.01, 100.0, "float64")
    s = torch.tensor(workloads.random_field(nu, nphi, 1), device="cuda")
    sw = torch.tensor(np.random.default_rng(3).standard_normal(nphi), device="cuda")
    gr = torch.tensor(workloads.random_field(nu, nphi, 2), device="cuda")
    gp = torch.tensor(workloads.random_field(nu, nphi, 3), device="cuda")
    Fr, Fp = plan.forces_wedge(s, sw)
    gs, gsw = plan.backward_wedge(gr, gp)
    lhs = float((gr * Fr).sum() + (gp * Fp).sum())
    rhs = float((gs * s).sum() + (gsw * sw).sum())
    assert abs(lhs - rhs) < 1e-12 * float((gr.abs() * Fr.abs()).sum() + (gp.abs() * Fp.abs()).sum())


@pytest.mark.parametrize("nu,nphi", [(256, 128), (512, 64)])
def test_fp32_against_fp64_where_the_column_passes_fuse(torch_cuda, oracle_mod, nu, nphi):
    """FP32 columns of 512 points or more: the forward applies the wedge
    update inside the column pass, the adjoint beside the fused edge update.
    The FP64 plan (separate kernels, pinned to the oracle above) is the
    reference for both gradients."""
    torch = torch_cuda
    p32, grid, du = _setup(oracle_mod, nu, nphi, 0.1, 10.0, "float32", 1)
    p64, _, _ = _setup(oracle_mod, nu, nphi, 0.1, 10.0, "float64", 1)
    sigma, sigma_w = _inputs(grid, 21)
    F32 = p32.forces_wedge(torch.tensor(sigma, dtype=torch.float32, device="cuda"),
                           torch.tensor(sigma_w, dtype=torch.float32, device="cuda"))
    F64 = p64.forces_wedge(torch.tensor(sigma, device="cuda"), torch.tensor(sigma_w, device="cuda"))
    p32.check()
    num = sum(float(((a.double() - b) ** 2).sum()) for a, b in zip(F32, F64))
    den = sum(float((b ** 2).sum()) for b in F64)
    assert math.sqrt(num / den) < 1e-5
    gr, gp = workloads.random_field(nu, nphi, 22), workloads.random_field(nu, nphi, 23)
    g32, gw32 = p32.backward_wedge(torch.tensor(gr, dtype=torch.float32, device="cuda"),
                                   torch.tensor(gp, dtype=torch.float32, device="cuda"))
    g64, gw64 = p64.backward_wedge(torch.tensor(gr, device="cuda"), torch.tensor(gp, device="cuda"))
    p32.check()
    for a, b in ((g32, g64), (gw32, gw64)):
        ref = b.cpu().numpy()
        assert np.linalg.norm(a.double().cpu().numpy() - ref) / np.linalg.norm(ref) < 1e-5


def test_potential_with_the_wedge(torch_cuda, oracle_mod):
    torch = torch_cuda
    nu, nphi = 64, 128
    plan, grid, du = _setup(oracle_mod, nu, nphi, 0.1, 10.0, "float64", kind="potential")
    sigma, sigma_w = _inputs(grid, 9)
    ref = grid.r[:, None] * oracle_mod.wedge_forces(sigma, sigma_w, oracle_mod.potential_cells(nu, nphi, du),
                                                    oracle_mod.wedge_cells(nu, nphi, du, pot=True), grid)[0]
    Phi, _ = plan.forces_wedge(torch.tensor(sigma, device="cuda"), torch.tensor(sigma_w, device="cuda"))
    plan.check()
    assert_close_1(Phi.cpu().numpy(), ref, 1e-12, w=grid.r ** -1.0)


def test_kuzmin_held_by_grid_and_wedge(torch_cuda):
    """FP64 forces of the library with r_in halved per doubling (as the
    oracle's pin): full-grid second order against the closed form less the
    tail beyond r_out."""
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    errs = []
    for n, r_in in ((32, 0.2), (64, 0.1), (128, 0.05)):
        u_min, du = workloads.grid_params(n, r_in, 20.0)
        r, phi = workloads.centres(n, n, u_min, du)
        plan = Plan(n, n, u_min, du, 1.0, "float64").build(radial_edges=1, wedge=1)
        s = torch.tensor(workloads.kuzmin(r, phi), device="cuda")
        sw = torch.full((n,), float(A.kuzmin_sigma(0.5 * math.exp(u_min))), dtype=torch.float64, device="cuda")
        Fr, _ = plan.forces_wedge(s, sw)
        truth = A.kuzmin_truncated_Fr(r, 0.0, 20.0)
        errs.append(np.abs(Fr[:, 0].cpu().numpy() - truth).max() / np.abs(truth).max())
    order = math.log2(errs[-2] / errs[-1])
    assert order > 1.7 and errs[-1] < 4e-4, (errs, order)


def test_options(torch_cuda, oracle_mod, tmp_path):
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan, SgError, sg, forces_batched

    u_min, du = workloads.grid_params(32, 0.1, 10.0)
    plan = Plan(32, 64, u_min, du, 1.0, "float32")
    for kw in ({"wedge": 1}, {"wedge": 1, "radial_edges": 1, "kind": "particle"}, {"wedge": 2, "radial_edges": 1}):
        with pytest.raises(SgError) as ei:
            plan.build(**kw)
        assert ei.value.status == sg.SG_ERR_ARG
    plan.build(radial_edges=1, wedge=1)
    s = torch.rand(32, 64, device="cuda")
    with pytest.raises(SgError) as ei:
        plan.forces(s)
    assert ei.value.status == sg.SG_ERR_UNSUPPORTED
    with pytest.raises(SgError) as ei:
        forces_batched([(plan, s, torch.empty_like(s), torch.empty_like(s))])
    assert ei.value.status == sg.SG_ERR_UNSUPPORTED
    with pytest.raises(SgError) as ei:
        plan.forces_noalloc(s, torch.empty_like(s), torch.empty_like(s))
    assert ei.value.status == sg.SG_ERR_UNSUPPORTED
    with pytest.raises(SgError) as ei:
        plan.save(str(tmp_path / "wedge_plan.bin"))
    assert ei.value.status == sg.SG_ERR_UNSUPPORTED
    # a plan without the wedge refuses the wedge entry point
    plain = Plan(32, 64, u_min, du, 1.0, "float32").build()
    with pytest.raises(SgError) as ei:
        plain.forces_wedge(s, torch.zeros(64, device="cuda"))
    assert ei.value.status == sg.SG_ERR_ARG
    # rebuilt without the wedge, the plan computes through sg_forces again
    plan.build(radial_edges=1)
    plan.forces(s)
    torch.cuda.synchronize()
