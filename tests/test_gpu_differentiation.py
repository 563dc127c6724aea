"""Differentiation workload: d(loss)/d(sigma) through the adjoint passes.

Loss L(sigma) = sum over cells of w ((F_r - F_r*)^2 + (F_phi - F_phi*)^2),
w the cell area, F* the forces of a target disk (Kuzmin x (1 + 0.15 cos(2 phi
- ln r / tan 20 deg))), sigma starting at the plain Kuzmin disk, 1024 x 2048
on r in [0.01, 100].  Its gradient is A^T (2 w (F - F*)), which the library
computes with sg_forces_backward.  L is quadratic in sigma, so the FP64
central difference (L(sigma + h e_c) - L(sigma - h e_c)) / 2h equals dL/dsigma_c
up to rounding, for any h: it pins the FP64 gradient on 64 random cells.  On
a 64 x 64 copy of the problem the gradient is also compared with the oracle's
transposed direct sum.

In FP32 the forward pass's rounding error is nearly uniform over the grid
(about 6e-7 of the largest force), while w grows like r^2 and the residual
F - F* is small where r is large: the loss weights exactly the cells where
that error is largest relative to the residual.  The FP32 adjoint is
therefore checked on its own (on the FP64 residual) at the FP32 bar, and the
end-to-end FP32 gradient is checked to differ from the FP64 one by the
adjoint of the forward pass's rounding and nothing more.
"""
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
def problem(torch_cuda):
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    cfg = workloads.DIFF_1024
    start, target, w = workloads.diff_problem(cfg)
    p64 = Plan(cfg.nu, cfg.nphi, cfg.u_min, cfg.du, 1.0, "float64").build()
    p32 = Plan(cfg.nu, cfg.nphi, cfg.u_min, cfg.du, 1.0, "float32").build()
    dev = lambda a, dt: torch.tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")  # noqa: E731
    W = np.broadcast_to(np.asarray(w, dtype=np.float64).reshape(cfg.nu, -1), (cfg.nu, cfg.nphi))
    Ts = p64.forces(dev(target, torch.float64))
    return dict(cfg=cfg, start=start, W=W, p64=p64, p32=p32, Ts=Ts, dev=dev)


def _loss64(torch, pr, sigma64):
    Fr, Fp = pr["p64"].forces(sigma64)
    W = pr["W64"]
    return float((W * ((Fr - pr["Ts"][0]) ** 2 + (Fp - pr["Ts"][1]) ** 2)).sum())


def _grad(torch, plan, pr, sigma, dtype):
    Fr, Fp = plan.forces(sigma)
    W = torch.tensor(np.ascontiguousarray(pr["W"]), dtype=dtype, device="cuda")
    gr = (2 * W * (Fr - pr["Ts"][0].to(dtype))).contiguous()
    gp = (2 * W * (Fp - pr["Ts"][1].to(dtype))).contiguous()
    return plan.backward(gr, gp)


def test_gradient_matches_fp64_central_differences(torch_cuda, problem):
    torch = torch_cuda
    pr = problem
    cfg = pr["cfg"]
    pr["W64"] = torch.tensor(np.ascontiguousarray(pr["W"]), dtype=torch.float64, device="cuda")
    s64 = pr["dev"](pr["start"], torch.float64)
    g64 = _grad(torch, pr["p64"], pr, s64, torch.float64).cpu().numpy()
    rng = np.random.default_rng(7)
    cells = rng.choice(cfg.nu * cfg.nphi, 64, replace=False)
    fd = np.empty(64)
    for n, c in enumerate(cells):
        i, j = divmod(int(c), cfg.nphi)
        h = 0.5 * max(abs(pr["start"][i, j]), 1e-3)
        sp = s64.clone()
        sp[i, j] += h
        sm = s64.clone()
        sm[i, j] -= h
        fd[n] = (_loss64(torch, pr, sp) - _loss64(torch, pr, sm)) / (2 * h)
    scale = np.abs(fd).max()
    assert scale > 0
    # the FP64 adjoint against the differences: rounding only
    assert np.abs(g64.reshape(-1)[cells] - fd).max() <= 1e-9 * scale
    pr["g64"], pr["fd"], pr["fd_cells"] = g64, fd, cells


def test_fp32_gradient(torch_cuda, problem):
    """The FP32 adjoint meets the FP32 bar on its own (applied to the FP64
    residual); end to end, what it misses beyond that is the adjoint of the
    FP32 forward pass's own rounding, A^T (2 w dF), and nothing else."""
    torch = torch_cuda
    pr = problem
    if "g64" not in pr:
        pytest.skip("needs the FP64 gradient of the previous test")
    g64 = pr["g64"]
    W64 = pr["W64"]
    s64 = pr["dev"](pr["start"], torch.float64)
    s32 = pr["dev"](pr["start"], torch.float32)
    F64 = pr["p64"].forces(s64)
    v64 = [(2 * W64 * (F64[k] - pr["Ts"][k])).contiguous() for k in range(2)]
    # (1) the FP32 adjoint on the exact residual
    ga = pr["p32"].backward(v64[0].float(), v64[1].float()).double().cpu().numpy()
    nrm = np.linalg.norm(g64)
    assert np.linalg.norm(ga - g64) / nrm < 1e-5
    cells = pr["fd_cells"]
    assert np.abs(ga.reshape(-1)[cells] - pr["fd"]).max() <= 1e-5 * np.abs(g64).max()
    # (2) end to end: FP32 forward, FP32 residual, FP32 adjoint
    ge = _grad(torch, pr["p32"], pr, s32, torch.float32).double().cpu().numpy()
    F32 = pr["p32"].forces(s32)
    dF = [(F32[k].double() - F64[k]).contiguous() for k in range(2)]
    pred = pr["p64"].backward((2 * W64 * dF[0]).contiguous(), (2 * W64 * dF[1]).contiguous()).cpu().numpy()
    rel_e2e = np.linalg.norm(ge - g64) / nrm
    rel_fwd = math.sqrt(sum(float((d ** 2).sum()) for d in dF) / sum(float((f ** 2).sum()) for f in F64))
    print(f"FP32 gradient: adjoint alone rel-L2 {np.linalg.norm(ga - g64) / nrm:.2e}, end to end {rel_e2e:.2e}"
          f" (FP32 forward rel-L2 {rel_fwd:.2e})")
    assert rel_fwd < 1e-5
    assert np.linalg.norm((ge - g64) - pred) / nrm < 2e-5


def test_autograd_function_matches_adjoint(torch_cuda, problem):
    torch = torch_cuda
    from paper_1509_01450_gb300 import self_gravity

    pr = problem
    s32 = pr["dev"](pr["start"], torch.float32).requires_grad_(True)
    W = torch.tensor(np.ascontiguousarray(pr["W"]), dtype=torch.float32, device="cuda")
    Fr, Fp = self_gravity(s32, pr["p32"])
    L = (W * ((Fr - pr["Ts"][0].float()) ** 2 + (Fp - pr["Ts"][1].float()) ** 2)).sum()
    L.backward()
    ref = _grad(torch, pr["p32"], pr, s32.detach(), torch.float32)
    assert torch.allclose(s32.grad, ref, rtol=1e-5, atol=1e-6 * float(ref.abs().max()))


@pytest.mark.parametrize("dtype,tol", [("float64", 1e-12), ("float32", 1e-5), ("float32x2", 1e-12)])
def test_gradient_matches_oracle_transposed_sum_64x64(torch_cuda, oracle_mod, dtype, tol):
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    cfg = workloads.Config("diff-64x64", 64, 64, 0.01, 100.0)
    start, target, w = workloads.diff_problem(cfg)
    W = np.broadcast_to(np.asarray(w, dtype=np.float64).reshape(cfg.nu, -1), (cfg.nu, cfg.nphi))
    cells = oracle_mod.kernel_cells(cfg.nu, cfg.nphi, cfg.du)
    Kr, Kp = oracle_mod.fold(cells, math.exp(cfg.du), 2 * math.pi / cfg.nphi)
    Fr, Fp = oracle_mod.direct_sum(start, Kr, Kp)
    Tr, Tp = oracle_mod.direct_sum(target, Kr, Kp)
    ref = oracle_mod.direct_sum_T(2 * W * (Fr - Tr), 2 * W * (Fp - Tp), Kr, Kp)
    plan = Plan(cfg.nu, cfg.nphi, cfg.u_min, cfg.du, 1.0, dtype).build()
    dt = plan.dtype  # FP64 fields for the compensated plans too
    gr = torch.tensor(2 * W * (Fr - Tr), dtype=dt, device="cuda")
    gp = torch.tensor(2 * W * (Fp - Tp), dtype=dt, device="cuda")
    got = plan.backward(gr, gp).double().cpu().numpy()
    assert_close_1(got, ref, tol)


def test_compensated_fp32_gradient_end_to_end(torch_cuda, problem):
    """The compensated FP32 plans (double-float passes on the FP32 pipes):
    forward, residual and adjoint end to end meet the FP32 bar against the
    FP64 gradient where the plain FP32 chain cannot (its forward rounding,
    weighted by w, dominates the residual), and in fact the FP64 one."""
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    pr = problem
    if "g64" not in pr:
        pytest.skip("needs the FP64 gradient of the first test")
    cfg = pr["cfg"]
    pc = Plan(cfg.nu, cfg.nphi, cfg.u_min, cfg.du, 1.0, "float32x2").build()
    s = pr["dev"](pr["start"], torch.float64)
    g = _grad(torch, pc, pr, s, torch.float64)
    pc.check()
    g = g.cpu().numpy()
    g64 = pr["g64"]
    rel = np.linalg.norm(g - g64) / np.linalg.norm(g64)
    print(f"compensated FP32 gradient: rel-L2 {rel:.2e} against FP64")
    assert_close_1(g, g64, 1e-5)
    assert rel < 1e-8  # the FP64 gradient itself carries the residual's cancellation (about 1e-10)
    # plain FP32 end to end, with the kernels stored at weighting p = 0, 1, 2
    for p in (0, 1, 2):
        p32 = Plan(cfg.nu, cfg.nphi, cfg.u_min, cfg.du, 1.0, "float32").build(weight_p=p)
        g32 = _grad(torch, p32, pr, pr["dev"](pr["start"], torch.float32), torch.float32).double().cpu().numpy()
        r32 = np.linalg.norm(g32 - g64) / np.linalg.norm(g64)
        print(f"plain FP32 gradient at p = {p}: rel-L2 {r32:.2e} against FP64")
        assert rel < r32
    assert np.abs(g.reshape(-1)[pr["fd_cells"]] - pr["fd"]).max() <= 1e-9 * np.abs(pr["fd"]).max()
