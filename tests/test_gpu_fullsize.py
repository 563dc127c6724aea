"""Parity at the full 2048 x 4096 size, in the launch configuration the
benchmark times (FP32 forward and adjoint, FP64, and the compensated FP32
plans at the FP64 bar), on sampled target and
source cells that the FP64 oracle computes one by one (direct sums over its
own kernel table)."""
import math

import numpy as np
import pytest

import workloads
from tests.errbounds import assert_close, assert_close_1

pytestmark = pytest.mark.gpu

NU, NPHI = 2048, 4096


@pytest.fixture(scope="module")
def full(oracle_mod):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cfg = workloads.GRF_2048
    r, phi = cfg.centres()
    sigma = workloads.lognormal_disk(r, phi, 1509)
    Kr, Kp = oracle_mod.kernels(NU, NPHI, cfg.du)
    tg = np.random.default_rng(7).choice(NU * NPHI, 256, replace=False)
    tg = np.concatenate([tg, [0, NPHI - 1, NU * NPHI - 1, (NU // 2) * NPHI]])  # edges included
    Fr, Fp = oracle_mod.direct_sum(sigma, Kr, Kp, targets=tg)
    return torch, cfg, sigma, tg, Fr, Fp, Kr, Kp


@pytest.mark.parametrize("dtype,tol", [("float32", 1e-5), ("float64", 1e-12), ("float32x2", 1e-12)])
def test_full_size_sampled_targets(oracle_mod, full, dtype, tol):
    torch, cfg, sigma, tg, Fr_ref, Fp_ref, _, _ = full
    from paper_1509_01450_gb300 import Plan

    plan = Plan(NU, NPHI, cfg.u_min, cfg.du, 1.0, dtype).build()
    assert plan.build_report() == (0, 0, 0, 0)
    s = torch.tensor(sigma, dtype=plan.dtype, device="cuda")
    Fr, Fp = plan.forces(s)
    torch.cuda.synchronize()
    fr = Fr.double().cpu().numpy().ravel()[tg]
    fp = Fp.double().cpu().numpy().ravel()[tg]
    assert_close(fr, fp, Fr_ref, Fp_ref, tol)
    # the timed-entry variant gives the same numbers
    Fr2, Fp2 = torch.empty_like(Fr), torch.empty_like(Fp)
    ms = plan.forces_timed(s, Fr2, Fp2)
    assert torch.equal(Fr, Fr2) and torch.equal(Fp, Fp2) and all(m > 0 for m in ms)


@pytest.mark.parametrize("dtype,tol", [("float32", 1e-5), ("float64", 1e-12), ("float32x2", 1e-12)])
def test_full_size_adjoint_sampled_sources(oracle_mod, full, dtype, tol):
    torch, cfg, sigma, tg, _, _, Kr, Kp = full
    from paper_1509_01450_gb300 import Plan

    plan = Plan(NU, NPHI, cfg.u_min, cfg.du, 1.0, dtype).build()
    gr, gp = workloads.random_field(NU, NPHI, 31), workloads.random_field(NU, NPHI, 32)
    ref = oracle_mod.direct_sum_T(gr, gp, Kr, Kp, sources=tg)
    gs = plan.backward(torch.tensor(gr, dtype=plan.dtype, device="cuda"),
                       torch.tensor(gp, dtype=plan.dtype, device="cuda"))
    plan.check()
    assert_close_1(gs.double().cpu().numpy().ravel()[tg], ref, tol)
    # the timed-entry variant gives the same numbers
    g2 = torch.empty_like(gs)
    ms = plan.backward_timed(torch.tensor(gr, dtype=plan.dtype, device="cuda"),
                             torch.tensor(gp, dtype=plan.dtype, device="cuda"), g2)
    assert torch.equal(gs, g2) and all(m > 0 for m in ms)
