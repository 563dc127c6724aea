"""The compensated FP32 plans (SG_F32X2): FP64 fields, double-float passes
on the FP32 pipes.  Against the FP64 oracle at the FP64 bar (1e-12 relative
L2 with the local bounds): the forward and adjoint on the default kernels,
the one-sided edges with the origin wedge, the potential, and the
checkpoint round trip; and the same numbers through the host entry point."""
import math

import numpy as np
import pytest

import workloads
from tests.errbounds import assert_close, assert_close_1

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01450_gb300 import build

    build.build()
    return torch


@pytest.mark.parametrize("nu,nphi", [(4, 8), (16, 64), (64, 32), (128, 256), (256, 512)])
def test_forward_and_adjoint_against_the_oracle(torch_cuda, oracle_mod, nu, nphi):
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    u_min, du = workloads.grid_params(nu, 0.01, 100.0)
    plan = Plan(nu, nphi, u_min, du, 1.0, "float32x2").build()
    assert plan.dtype == torch.float64
    Kr, Kp = oracle_mod.kernels(nu, nphi, du)
    sigma = np.abs(workloads.random_field(nu, nphi, nu + 7 * nphi)) + 0.1
    Fr_ref, Fp_ref = oracle_mod.fft_conv(sigma, Kr, Kp)
    Fr, Fp = plan.forces(torch.tensor(sigma, device="cuda"))
    plan.check()
    assert_close(Fr.cpu().numpy(), Fp.cpu().numpy(), Fr_ref, Fp_ref, TOL)
    gr, gp = workloads.random_field(nu, nphi, 5), workloads.random_field(nu, nphi, 6)
    ref = oracle_mod.fft_conv_T(gr, gp, Kr, Kp)
    gs = plan.backward(torch.tensor(gr, device="cuda"), torch.tensor(gp, device="cuda"))
    plan.check()
    assert_close_1(gs.cpu().numpy(), ref, TOL)


def test_edges_and_wedge_against_the_oracle(torch_cuda, oracle_mod):
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    nu, nphi = 64, 128
    u_min, du = workloads.grid_params(nu, 0.1, 10.0)
    grid = oracle_mod.Grid(nu, nphi, u_min, du)
    cells = oracle_mod.kernel_cells(nu, nphi, du)
    sigma = workloads.spiral_clump(grid.r, grid.phi) + 0.05 * np.abs(workloads.random_field(nu, nphi, 4))
    sigma_w = 0.5 + np.random.default_rng(4).random(nphi)
    plan = Plan(nu, nphi, u_min, du, 1.0, "float32x2").build(radial_edges=1)
    Fr_ref, Fp_ref = oracle_mod.onesided_forces(sigma, cells, grid)
    Fr, Fp = plan.forces(torch.tensor(sigma, device="cuda"))
    plan.check()
    assert_close(Fr.cpu().numpy(), Fp.cpu().numpy(), Fr_ref, Fp_ref, TOL)
    gr, gp = workloads.random_field(nu, nphi, 7), workloads.random_field(nu, nphi, 8)
    ref = oracle_mod.onesided_forces_T(gr, gp, cells, grid)
    gs = plan.backward(torch.tensor(gr, device="cuda"), torch.tensor(gp, device="cuda"))
    assert_close_1(gs.cpu().numpy(), ref, TOL)
    plan.build(radial_edges=1, wedge=1)
    Fr_ref, Fp_ref = oracle_mod.wedge_forces(sigma, sigma_w, cells, oracle_mod.wedge_cells(nu, nphi, du), grid)
    Fr, Fp = plan.forces_wedge(torch.tensor(sigma, device="cuda"), torch.tensor(sigma_w, device="cuda"))
    plan.check()
    assert_close(Fr.cpu().numpy(), Fp.cpu().numpy(), Fr_ref, Fp_ref, TOL)
    # the wedge adjoint by the dot identity over (sigma, sigma_w)
    g1, g2 = torch.tensor(gr, device="cuda"), torch.tensor(gp, device="cuda")
    gs, gsw = plan.backward_wedge(g1, g2)
    plan.check()
    lhs = float((g1 * Fr).sum() + (g2 * Fp).sum())
    rhs = float((gs.cpu() * torch.tensor(sigma)).sum() + (gsw.cpu() * torch.tensor(sigma_w)).sum())
    assert abs(lhs - rhs) <= 1e-12 * float((g1.abs() * Fr.abs()).sum() + (g2.abs() * Fp.abs()).sum())


def test_potential_against_the_oracle(torch_cuda, oracle_mod):
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    nu, nphi = 128, 256
    u_min, du = workloads.grid_params(nu, 0.1, 10.0)
    grid = oracle_mod.Grid(nu, nphi, u_min, du)
    plan = Plan(nu, nphi, u_min, du, 1.0, "float32x2").build(kind="potential", weight_p=1)
    sigma = np.abs(workloads.random_field(nu, nphi, 3)) + 0.1
    ref = oracle_mod.potential(sigma, oracle_mod.potential_cells(nu, nphi, du), grid)
    Phi, _ = plan.forces(torch.tensor(sigma, device="cuda"))
    plan.check()
    assert_close_1(Phi.cpu().numpy(), ref, TOL)


def test_save_load_and_host_entry(torch_cuda, tmp_path):
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan, sg

    nu, nphi = 256, 512
    u_min, du = workloads.grid_params(nu, 0.01, 100.0)
    plan = Plan(nu, nphi, u_min, du, 1.0, "float32x2").build()
    s = torch.tensor(np.abs(workloads.random_field(nu, nphi, 9)) + 0.1, device="cuda")
    Fr, Fp = plan.forces(s)
    path = str(tmp_path / "c.sg")
    plan.save(path)
    loaded = Plan.load(path)
    assert loaded.code == sg.SG_F32X2
    a, b = loaded.forces(s)
    assert torch.equal(a, Fr) and torch.equal(b, Fp)
    sh = s.cpu()
    fr, fp = torch.empty_like(sh), torch.empty_like(sh)
    plan.forces_host(sh, fr, fp)
    assert torch.equal(fr, Fr.cpu()) and torch.equal(fp, Fp.cpu())
    with pytest.raises(sg.SgError) as ei:
        plan.forces_noalloc(s, torch.empty_like(s), torch.empty_like(s))
    assert ei.value.status == sg.SG_ERR_UNSUPPORTED


def test_compensated_reaches_the_fp64_bar_where_fp32_does_not(torch_cuda, oracle_mod):
    """At 512 x 1024 the compensated plan's forward is within the FP64 bar of
    the oracle's FFT convolution, the FP32 plan's is not (about 1e-7)."""
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    nu, nphi = 512, 1024
    u_min, du = workloads.grid_params(nu, 0.01, 100.0)
    Kr, Kp = oracle_mod.kernels(nu, nphi, du)
    sigma = workloads.spiral_clump(*workloads.centres(nu, nphi, u_min, du))
    Fr_ref, Fp_ref = oracle_mod.fft_conv(sigma, Kr, Kp)
    errs = {}
    for dt in ("float32", "float32x2"):
        plan = Plan(nu, nphi, u_min, du, 1.0, dt).build()
        Fr, Fp = plan.forces(torch.tensor(sigma, dtype=plan.dtype, device="cuda"))
        plan.check()
        errs[dt] = oracle_mod.rel_l2(Fr.double().cpu().numpy(), Fp.double().cpu().numpy(), Fr_ref, Fp_ref)
    print(f"512 x 1024 rel-L2: FP32 {errs['float32']:.2e}, compensated {errs['float32x2']:.2e}")
    assert errs["float32x2"] < TOL < errs["float32"]
