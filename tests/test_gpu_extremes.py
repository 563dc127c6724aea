"""The largest and the most lopsided plans.

FP32 4096 x 8192 (the largest FP32 plan; its column and row passes run at
512 threads per block) is too large for the oracle's kernel table, so it is
checked by properties that hold at any size: the adjoint identity, and the
truncated Kuzmin disk's closed-form force (an independent truth; the
method's own error there is about 4e-7 of the peak force at this size,
extrapolated from the oracle's 6.2e-5 at 256 and 1.7e-5 at 512 rows).
The extreme shapes (N_u or N_phi at its limit, the other at 4) are compared
with the oracle's direct sum."""
import math

import numpy as np
import pytest

import workloads
from tests.errbounds import assert_close, assert_close_1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01450_gb300 import build

    build.build()
    return torch


@pytest.fixture(scope="module")
def max_plan(torch_cuda):
    from paper_1509_01450_gb300 import Plan

    cfg = workloads.Config("max-fp32", 4096, 8192, 0.01, 100.0)
    plan = Plan(cfg.nu, cfg.nphi, cfg.u_min, cfg.du, 1.0, "float32").build()
    assert plan.build_report() == (0, 0, 0, 0)
    return cfg, plan


def test_max_fp32_kuzmin_closed_form(torch_cuda, max_plan):
    torch = torch_cuda
    from oracle import analytic

    cfg, plan = max_plan
    r, phi = cfg.centres()
    Fr, Fp = plan.forces(torch.tensor(workloads.kuzmin(r, phi), dtype=torch.float32, device="cuda"))
    plan.check()
    Fr = Fr.double().cpu().numpy()
    Fp = Fp.double().cpu().numpy()
    rr = r[:, 0] if r.ndim == 2 else r
    rows = np.where((rr >= 0.04) & (rr <= 25.0))[0][::64]  # interior rows (the radial edges carry the R4 ghost dipole)
    truth = analytic.kuzmin_truncated_Fr(rr[rows], cfg.r_in, cfg.r_out)
    peak = np.abs(truth).max()
    assert np.abs(Fr[rows] - truth[:, None]).max() <= 1e-5 * peak  # every phi column of each row
    assert np.abs(Fp).max() <= 1e-5 * peak  # axisymmetric: no azimuthal force


def test_max_fp32_adjoint_identity(torch_cuda, max_plan):
    torch = torch_cuda
    cfg, plan = max_plan
    g = torch.Generator(device="cuda").manual_seed(3)
    sig = torch.rand(cfg.nu, cfg.nphi, device="cuda", generator=g)
    gr = torch.randn(cfg.nu, cfg.nphi, device="cuda", generator=g)
    gp = torch.randn(cfg.nu, cfg.nphi, device="cuda", generator=g)
    Fr, Fp = plan.forces(sig)
    gs = plan.backward(gr, gp)
    plan.check()
    lhs = float((gr.double() * Fr.double()).sum() + (gp.double() * Fp.double()).sum())
    rhs = float((gs.double() * sig.double()).sum())
    scale = math.sqrt(float((gr.double() ** 2).sum() + (gp.double() ** 2).sum())) * math.sqrt(
        float((Fr.double() ** 2).sum() + (Fp.double() ** 2).sum()))
    assert abs(lhs - rhs) <= 1e-5 * scale


# (4096, 4) on r in [1e-4, 1e4]: at r in [0.05, 20] its self cell is 1075 times
# longer in phi than in r, beyond what the oracle's self-cell quadrature
# resolves (it does up to about 500); the wider range keeps it near 350
@pytest.mark.parametrize("nu,nphi,r_in,r_out,dtype,tol", [(4096, 4, 1e-4, 1e4, "float32", 1e-5),
                                                         (4, 8192, 0.05, 20.0, "float32", 1e-5),
                                                         (2048, 4, 0.05, 20.0, "float64", 1e-12),
                                                         (4, 4096, 0.05, 20.0, "float64", 1e-12)])
def test_extreme_shapes_match_oracle(torch_cuda, oracle_mod, nu, nphi, r_in, r_out, dtype, tol):
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    u_min, du = workloads.grid_params(nu, r_in, r_out)
    plan = Plan(nu, nphi, u_min, du, 1.0, dtype).build()
    sigma = np.abs(workloads.random_field(nu, nphi, nu + 3 * nphi)) + 0.1
    cells = oracle_mod.kernel_cells(nu, nphi, du)
    Kr, Kp = oracle_mod.fold(cells, math.exp(du), 2 * math.pi / nphi)
    Fr_ref, Fp_ref = oracle_mod.direct_sum(sigma, Kr, Kp)
    Fr, Fp = plan.forces(torch.tensor(sigma, dtype=plan.dtype, device="cuda"))
    plan.check()
    got_r, got_p = Fr.double().cpu().numpy(), Fp.double().cpu().numpy()
    assert_close(got_r, got_p, Fr_ref, Fp_ref, tol)
    # the adjoint on the same plan, on independent upstream gradients
    gr, gp = workloads.random_field(nu, nphi, 5), workloads.random_field(nu, nphi, 6)
    ref = oracle_mod.direct_sum_T(gr, gp, Kr, Kp)
    gs = plan.backward(torch.tensor(gr, dtype=plan.dtype, device="cuda"),
                       torch.tensor(gp, dtype=plan.dtype, device="cuda"))
    plan.check()
    assert_close_1(gs.double().cpu().numpy(), ref, tol)
