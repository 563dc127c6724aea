"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Bars (from the required agreement of the method's two precisions):
FP64 forward / adjoint within 1e-12 relative L2 of the oracle, FP32 within
1e-5; the GPU kernel builder's FP64 cell integrals within 1e-12 of each
cell's own scale.  rel-L2 = sqrt(sum dF_r^2 + dF_phi^2) / sqrt(sum F_r^2 +
F_phi^2) over the compared cells.
"""
import math

import numpy as np
import pytest

import workloads
from tests.errbounds import assert_close, assert_close_1

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
FP32_TOL = 1e-5

_tables = {}


def oracle_kernels(oracle_mod, nu, nphi, du):
    key = (nu, nphi, round(du, 15))
    if key not in _tables:
        cells = oracle_mod.kernel_cells(nu, nphi, du)
        Kr, Kp = oracle_mod.fold(cells, math.exp(du), 2 * math.pi / nphi)
        _tables[key] = (cells, Kr, Kp)
    return _tables[key]


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01450_gb300 import build

    build.build()
    return torch


def make_plan(nu, nphi, r_in, r_out, dtype, p=0):
    from paper_1509_01450_gb300 import Plan

    u_min, du = workloads.grid_params(nu, r_in, r_out)
    return Plan(nu, nphi, u_min, du, 1.0, dtype).build(weight_p=p), u_min, du


def cell_scale(cells, c):
    """Scale of component c of each cell: its own magnitude plus
    |K^{r,0}| + |K^{phi,0}| of the cell and 1e-3 of the row's largest."""
    base = np.abs(cells[0]) + np.abs(cells[3])
    row = base.max(axis=1, keepdims=True)
    return np.abs(cells[c]) + base + 1e-3 * row


@pytest.mark.parametrize("nu,nphi,r_in,r_out", [(4, 4, 0.5, 2.0), (8, 16, 0.1, 10.0), (16, 8, 0.1, 10.0),
                                                 (64, 64, 0.05, 20.0), (32, 128, 0.01, 100.0),
                                                 (128, 32, 0.01, 100.0)])
def test_kernel_builder_matches_oracle(torch_cuda, oracle_mod, nu, nphi, r_in, r_out):
    plan, u_min, du = make_plan(nu, nphi, r_in, r_out, "float64")
    got = plan.cells()
    ref, Kr, Kp = oracle_kernels(oracle_mod, nu, nphi, du)
    for c in range(6):
        err = np.abs(got[c] - ref[c]) / cell_scale(ref, c)
        assert err.max() < 2e-12, (c, err.max(), np.unravel_index(err.argmax(), err.shape))
    gKr, gKp = plan.kernels()
    sk = np.abs(Kr).max() + np.abs(Kp).max()
    assert np.abs(gKr - Kr).max() < 1e-12 * sk
    assert np.abs(gKp - Kp).max() < 1e-12 * sk


def _forward(torch, plan, sigma):
    s = torch.tensor(sigma, dtype=plan.dtype, device="cuda")
    Fr, Fp = plan.forces(s)
    torch.cuda.synchronize()
    return Fr.double().cpu().numpy(), Fp.double().cpu().numpy()


@pytest.mark.parametrize("dtype,tol", [("float64", FP64_TOL), ("float32", FP32_TOL)])
def test_forward_kuzmin_64(torch_cuda, oracle_mod, dtype, tol):
    cfg = workloads.KUZMIN_64
    plan, u_min, du = make_plan(cfg.nu, cfg.nphi, cfg.r_in, cfg.r_out, dtype)
    r, phi = cfg.centres()
    sigma = workloads.kuzmin(r, phi)
    _, Kr, Kp = oracle_kernels(oracle_mod, cfg.nu, cfg.nphi, du)
    Fr_ref, Fp_ref = oracle_mod.direct_sum(sigma, Kr, Kp)
    Fr, Fp = _forward(torch_cuda, plan, sigma)
    assert_close(Fr, Fp, Fr_ref, Fp_ref, tol)


@pytest.mark.parametrize("nu,nphi", [(4, 4), (4, 8), (8, 4), (8, 16), (16, 8), (32, 64), (64, 32), (16, 256),
                                     (256, 16), (8, 512)])
@pytest.mark.parametrize("dtype,tol", [("float64", FP64_TOL), ("float32", FP32_TOL)])
def test_forward_sizes_random_density(torch_cuda, oracle_mod, nu, nphi, dtype, tol):
    plan, u_min, du = make_plan(nu, nphi, 0.1, 10.0, dtype)
    sigma = np.abs(workloads.random_field(nu, nphi, nu * 131 + nphi)) + 0.1
    _, Kr, Kp = oracle_kernels(oracle_mod, nu, nphi, du)
    Fr_ref, Fp_ref = oracle_mod.direct_sum(sigma, Kr, Kp)
    Fr, Fp = _forward(torch_cuda, plan, sigma)
    plan.check()  # no pass timed out waiting for its input copies
    assert_close(Fr, Fp, Fr_ref, Fp_ref, tol)


@pytest.mark.parametrize("dtype,tol", [("float64", FP64_TOL), ("float32", FP32_TOL)])
@pytest.mark.parametrize("nu,nphi", [(64, 64), (16, 128), (128, 16)])
def test_backward_matches_transposed_sum(torch_cuda, oracle_mod, nu, nphi, dtype, tol):
    torch = torch_cuda
    plan, u_min, du = make_plan(nu, nphi, 0.05, 20.0, dtype)
    gr = workloads.random_field(nu, nphi, 21)
    gp = workloads.random_field(nu, nphi, 22)
    _, Kr, Kp = oracle_kernels(oracle_mod, nu, nphi, du)
    ref = oracle_mod.direct_sum_T(gr, gp, Kr, Kp)
    gs = plan.backward(torch.tensor(gr, dtype=plan.dtype, device="cuda"),
                       torch.tensor(gp, dtype=plan.dtype, device="cuda"))
    plan.check()
    got = gs.double().cpu().numpy()
    assert_close_1(got, ref, tol)


def test_adjoint_dot_identity_fp64(torch_cuda):
    torch = torch_cuda
    plan, _, _ = make_plan(32, 64, 0.05, 20.0, "float64")
    s = torch.tensor(workloads.random_field(32, 64, 1), device="cuda")
    gr = torch.tensor(workloads.random_field(32, 64, 2), device="cuda")
    gp = torch.tensor(workloads.random_field(32, 64, 3), device="cuda")
    Fr, Fp = plan.forces(s)
    gs = plan.backward(gr, gp)
    lhs = float((gr * Fr).sum() + (gp * Fp).sum())
    rhs = float((gs * s).sum())
    assert abs(lhs - rhs) < 1e-13 * (float(gs.abs().sum() * s.abs().max()))


@pytest.mark.parametrize("p,tol", [(0, FP64_TOL), (1, FP64_TOL), (2, 1e-10)])
def test_weighting_is_neutral(torch_cuda, oracle_mod, p, tol):
    """sigma e^{pu} with kernels beta^{pk} and result e^{-pu} is algebraically
    the same map; rounding is amplified by up to beta^{p N_u} (1.6e5 for
    p = 2 on r in [0.05, 20]), which is why p = 0 is the default."""
    cfg = workloads.KUZMIN_64
    plan, u_min, du = make_plan(cfg.nu, cfg.nphi, cfg.r_in, cfg.r_out, "float64", p=p)
    r, phi = cfg.centres()
    sigma = workloads.spiral_clump(r, phi)
    _, Kr, Kp = oracle_kernels(oracle_mod, cfg.nu, cfg.nphi, du)
    Fr_ref, Fp_ref = oracle_mod.direct_sum(sigma, Kr, Kp)
    Fr, Fp = _forward(torch_cuda, plan, sigma)
    assert_close(Fr, Fp, Fr_ref, Fp_ref, tol, w=workloads.centres(cfg.nu, 1, u_min, du)[0] ** p)


def test_batched_equals_single(torch_cuda):
    torch = torch_cuda
    from paper_1509_01450_gb300 import forces_batched

    shapes = [(16, 32), (32, 16), (16, 32), (64, 64)]
    plans, items, singles = [], [], []
    for n, (nu, nphi) in enumerate(shapes):
        plan, _, _ = make_plan(nu, nphi, 0.05, 20.0, "float32")
        s = torch.tensor(workloads.random_field(nu, nphi, 40 + n), dtype=torch.float32, device="cuda")
        fr, fp = torch.empty_like(s), torch.empty_like(s)
        plans.append(plan)
        items.append((plan, s, fr, fp))
        singles.append(plan.forces(s))
    forces_batched(items)
    torch.cuda.synchronize()
    for (plan, s, fr, fp), (rr, pp) in zip(items, singles):
        assert torch.equal(fr, rr) and torch.equal(fp, pp)


def test_not_built_and_bad_pointers(torch_cuda):
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan, SgError, sg

    plan = Plan(16, 16, 0.0, 0.1, 1.0, "float32")
    s = torch.zeros((16, 16), device="cuda")
    with pytest.raises(SgError) as ei:
        plan.forces(s)
    assert ei.value.status == sg.SG_ERR_NOT_BUILT
    plan.build()
    big = torch.zeros(16 * 16 + 1, device="cuda")
    mis = big[1:].view(16, 16)  # 4-byte offset: not 16-byte aligned
    with pytest.raises(SgError) as ei:
        plan.forces(mis)
    assert ei.value.status == sg.SG_ERR_ARG


@pytest.mark.parametrize("dtype,tol", [("float64", FP64_TOL), ("float32", FP32_TOL)])
def test_spiral_clump_512x1024(torch_cuda, oracle_mod, dtype, tol):
    cfg = workloads.SPIRAL_512
    plan, u_min, du = make_plan(cfg.nu, cfg.nphi, cfg.r_in, cfg.r_out, dtype)
    r, phi = cfg.centres()
    sigma = workloads.spiral_clump(r, phi)
    _, Kr, Kp = oracle_kernels(oracle_mod, cfg.nu, cfg.nphi, du)
    Fr_ref, Fp_ref = oracle_mod.fft_conv(sigma, Kr, Kp)
    Fr, Fp = _forward(torch_cuda, plan, sigma)
    assert_close(Fr, Fp, Fr_ref, Fp_ref, tol)
    # sampled targets against the direct sum as well
    t = np.random.default_rng(0).choice(cfg.nu * cfg.nphi, 64, replace=False)
    dr, dp = oracle_mod.direct_sum(sigma, Kr, Kp, targets=t)
    assert_close(Fr.ravel()[t], Fp.ravel()[t], dr, dp, tol)


@pytest.mark.parametrize("nu,nphi,r_in,r_out", [(4, 4096, 0.5, 2.0), (8, 4096, 0.5, 2.0), (2048, 16, 0.01, 100.0),
                                                 (2048, 64, 0.01, 100.0)])
def test_fixed_length_passes(torch_cuda, oracle_mod, nu, nphi, r_in, r_out):
    """FP32 transforms of 4096 points run passes whose length is fixed at
    compile time: 4096-point rows with few (and, at N_u = 4, fewer than one
    per block) row blocks, and 4096-point columns with few modes, against
    the oracle, forward and adjoint."""
    torch = torch_cuda
    plan, u_min, du = make_plan(nu, nphi, r_in, r_out, "float32")
    Kr, Kp = oracle_mod.kernels(nu, nphi, du)
    sigma = np.abs(workloads.random_field(nu, nphi, nu + nphi)) + 0.1
    Fr_ref, Fp_ref = oracle_mod.fft_conv(sigma, Kr, Kp)
    Fr, Fp = _forward(torch, plan, sigma)
    plan.check()
    assert_close(Fr, Fp, Fr_ref, Fp_ref, FP32_TOL)
    gr, gp = workloads.random_field(nu, nphi, 5), workloads.random_field(nu, nphi, 6)
    ref = oracle_mod.fft_conv_T(gr, gp, Kr, Kp)
    gs = plan.backward(torch.tensor(gr, dtype=torch.float32, device="cuda"),
                       torch.tensor(gp, dtype=torch.float32, device="cuda"))
    assert_close_1(gs.double().cpu().numpy(), ref, FP32_TOL)
