"""The tensor-core DFT form of the short azimuthal transforms (build option
short_dft: split-TF32 DFT-matrix products on tcgen05, FP32 accumulate)
against the FP64 oracle at the FP32 bar, beside the FFT path, across the
shapes it takes (N_phi 32 .. 256, partial 128-row tiles, one K chunk):
forward and adjoint (the oracle's transposed sum, the dot identity, an
autograd gradient), with the column-pass options, the allocation-free and
batched entry points, the refused configurations and a wait that gives up."""
import numpy as np
import pytest

import workloads
from tests.errbounds import assert_close, assert_close_1, rel_l2

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
_tables = {}


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01450_gb300 import build

    build.build()
    return torch


def kernels(oracle_mod, nu, nphi, du):
    key = (nu, nphi, round(du, 15))
    if key not in _tables:
        _tables[key] = oracle_mod.kernels(nu, nphi, du)
    return _tables[key]


def plans(nu, nphi, r_in=0.01, r_out=100.0, **opts):
    from paper_1509_01450_gb300 import Plan

    u_min, du = workloads.grid_params(nu, r_in, r_out)
    tc = Plan(nu, nphi, u_min, du, 1.0, "float32").build(short_dft=1, **opts)
    fft = Plan(nu, nphi, u_min, du, 1.0, "float32").build(**opts)
    return tc, fft, u_min, du


def density(nu, nphi, u_min, du, seed):
    r, phi = workloads.centres(nu, nphi, u_min, du)
    return workloads.lognormal_disk(r, phi, seed)


def run(torch, plan, sigma):
    s = torch.tensor(sigma, dtype=torch.float32, device="cuda")
    Fr, Fp = plan.forces(s)
    plan.check()
    return Fr.double().cpu().numpy(), Fp.double().cpu().numpy()


@pytest.mark.parametrize("nu,nphi", [(4, 32), (16, 64), (64, 128), (128, 32), (32, 256), (128, 256),
                                     (256, 64)])
def test_matches_oracle_direct_sum(torch_cuda, oracle_mod, nu, nphi):
    tc, fft, u_min, du = plans(nu, nphi)
    sigma = density(nu, nphi, u_min, du, 7 + nu)
    Kr, Kp = kernels(oracle_mod, nu, nphi, du)
    Fr_ref, Fp_ref = oracle_mod.direct_sum(sigma, Kr, Kp)
    Fr, Fp = run(torch_cuda, tc, sigma)
    assert_close(Fr, Fp, Fr_ref, Fp_ref, FP32_TOL, what=f"short_dft {nu}x{nphi}")
    # beside the FFT path: both meet the FP32 bar, and agree within it
    Gr, Gp = run(torch_cuda, fft, sigma)
    e_tc, e_fft = rel_l2(Fr, Fp, Fr_ref, Fp_ref), rel_l2(Gr, Gp, Fr_ref, Fp_ref)
    print(f"short_dft {nu}x{nphi}: rel-L2 vs oracle {e_tc:.2e} (FFT rows {e_fft:.2e})")
    assert rel_l2(Fr, Fp, Gr, Gp) < FP32_TOL


@pytest.mark.parametrize("nu,nphi", [(1024, 256), (4096, 256), (2048, 32)])
def test_large_plans_on_sampled_targets(torch_cuda, oracle_mod, nu, nphi):
    """Many 128-row tiles and every column tile, checked on sampled targets
    (the oracle's direct sums one by one), edges and the last row included."""
    tc, _, u_min, du = plans(nu, nphi)
    sigma = density(nu, nphi, u_min, du, 3)
    Kr, Kp = kernels(oracle_mod, nu, nphi, du)
    n = nu * nphi
    tg = np.random.default_rng(nu + nphi).choice(n, 200, replace=False)
    tg = np.concatenate([tg, [0, nphi - 1, n - nphi, n - 1, (nu // 2) * nphi + nphi // 2]])
    Fr_ref, Fp_ref = oracle_mod.direct_sum(sigma, Kr, Kp, targets=tg)
    Fr, Fp = run(torch_cuda, tc, sigma)
    print(f"short_dft {nu}x{nphi}: sampled rel-L2 vs oracle {rel_l2(Fr.ravel()[tg], Fp.ravel()[tg], Fr_ref, Fp_ref):.2e}")
    assert_close(Fr.ravel()[tg], Fp.ravel()[tg], Fr_ref, Fp_ref, FP32_TOL, what=f"short_dft {nu}x{nphi}")


def test_kuzmin_closed_form(torch_cuda):
    """The Kuzmin disk at 256 x 256 keeps the FFT path's closed-form error."""
    nu = nphi = 256
    tc, fft, u_min, du = plans(nu, nphi, 0.05, 20.0)
    r, phi = workloads.centres(nu, nphi, u_min, du)
    sigma = workloads.kuzmin(r, phi)
    Fr, Fp = run(torch_cuda, tc, sigma)
    Gr, Gp = run(torch_cuda, fft, sigma)
    exact = -r / (r * r + 1.0) ** 1.5
    e_tc = np.sqrt(np.mean((Fr - exact) ** 2) / np.mean(exact ** 2))
    e_fft = np.sqrt(np.mean((Gr - exact) ** 2) / np.mean(exact ** 2))
    assert abs(e_tc - e_fft) < 1e-5 * (1 + e_fft), (e_tc, e_fft)
    assert np.abs(Fp).max() < 1e-5 * np.abs(exact).max()


@pytest.mark.parametrize("wedge", [0, 1])
def test_with_edge_and_wedge_options(torch_cuda, wedge):
    """The row transforms are independent of the column-pass options: with
    one-sided edges (and the origin wedge) the forces match the FFT plan."""
    torch = torch_cuda
    nu, nphi = 256, 128
    tc, fft, u_min, du = plans(nu, nphi, radial_edges=1, wedge=wedge)
    sigma = density(nu, nphi, u_min, du, 11)
    s = torch.tensor(sigma, dtype=torch.float32, device="cuda")
    if wedge:
        sw = torch.tensor(np.random.default_rng(5).uniform(0.5, 1.5, nphi), dtype=torch.float32, device="cuda")
        a, b = tc.forces_wedge(s, sw), fft.forces_wedge(s, sw)
    else:
        a, b = tc.forces(s), fft.forces(s)
    tc.check()
    fft.check()
    got = [t.double().cpu().numpy() for t in a]
    ref = [t.double().cpu().numpy() for t in b]
    assert rel_l2(got[0], got[1], ref[0], ref[1]) < FP32_TOL


def test_allocation_free_and_batched_entry_points(torch_cuda):
    """sg_forces_noalloc and sg_forces_batched on short_dft plans give
    sg_forces' numbers bit for bit (the batch runs such plans' items through
    per-plan launches)."""
    torch = torch_cuda
    from paper_1509_01450_gb300 import forces_batched

    shapes = [(128, 256), (64, 128), (256, 32)]
    items, refs = [], []
    for k, (nu, nphi) in enumerate(shapes):
        tc, _, u_min, du = plans(nu, nphi)
        s = torch.tensor(density(nu, nphi, u_min, du, 20 + k), dtype=torch.float32, device="cuda")
        Fr, Fp = tc.forces(s)
        Nr, Np = torch.empty_like(Fr), torch.empty_like(Fp)
        tc.forces_noalloc(s, Nr, Np)
        torch.cuda.synchronize()
        assert torch.equal(Fr, Nr) and torch.equal(Fp, Np)
        items.append((tc, s, torch.empty_like(Fr), torch.empty_like(Fp)))
        refs.append((Fr, Fp))
    forces_batched(items)
    torch.cuda.synchronize()
    for (plan, _, Br, Bp), (Fr, Fp) in zip(items, refs):
        plan.check()
        assert torch.equal(Br, Fr) and torch.equal(Bp, Fp)


@pytest.mark.parametrize("dtype,nphi", [("float64", 64), ("float32x2", 64), ("float32", 16), ("float32", 512)])
def test_unsupported_configurations_are_refused(torch_cuda, dtype, nphi):
    from paper_1509_01450_gb300 import Plan, sg

    u_min, du = workloads.grid_params(16, 0.1, 10.0)
    plan = Plan(16, nphi, u_min, du, 1.0, dtype)
    with pytest.raises(sg.SgError) as e:
        plan.build(short_dft=1)
    assert e.value.status == sg.SG_ERR_UNSUPPORTED


def test_wait_that_gives_up_reports_a_timeout(torch_cuda):
    """With a zero wait budget every bounded wait of the kernels gives up at
    once: the flag reads SG_ERR_TIMEOUT, the context stays usable, and with
    the budget restored the same plan computes correct forces again."""
    torch = torch_cuda
    from paper_1509_01450_gb300 import sg

    nu, nphi = 256, 256
    tc, fft, u_min, du = plans(nu, nphi)
    sigma = density(nu, nphi, u_min, du, 9)
    s = torch.tensor(sigma, dtype=torch.float32, device="cuda")
    tc.set_wait_limit(0.0)
    tc.forces(s)
    with pytest.raises(sg.SgError) as e:
        tc.check()
    assert e.value.status == sg.SG_ERR_TIMEOUT
    tc.set_wait_limit(1.0)
    Fr, Fp = run(torch, tc, sigma)
    Gr, Gp = run(torch, fft, sigma)
    assert rel_l2(Fr, Fp, Gr, Gp) < FP32_TOL


@pytest.mark.parametrize("nu,nphi", [(4, 32), (64, 128), (128, 64), (32, 256), (256, 256), (512, 32)])
def test_adjoint_matches_oracle_transposed_sum(torch_cuda, oracle_mod, nu, nphi):
    """P1b and P3b on the tensor cores: gsigma against the oracle's transposed
    direct sum on random gradients, beside the FFT adjoint."""
    torch = torch_cuda
    tc, fft, u_min, du = plans(nu, nphi)
    Kr, Kp = kernels(oracle_mod, nu, nphi, du)
    gr, gp = workloads.random_field(nu, nphi, 41), workloads.random_field(nu, nphi, 42)
    ref = oracle_mod.direct_sum_T(gr, gp, Kr, Kp)
    tgr = torch.tensor(gr, dtype=torch.float32, device="cuda")
    tgp = torch.tensor(gp, dtype=torch.float32, device="cuda")
    g = tc.backward(tgr, tgp)
    tc.check()
    h = fft.backward(tgr, tgp)
    got, other = g.double().cpu().numpy(), h.double().cpu().numpy()
    e_tc = rel_l2(got, 0 * got, ref, 0 * ref)
    e_fft = rel_l2(other, 0 * other, ref, 0 * ref)
    print(f"short_dft adjoint {nu}x{nphi}: rel-L2 vs oracle {e_tc:.2e} (FFT rows {e_fft:.2e})")
    assert_close_1(got, ref, FP32_TOL, what=f"short_dft adjoint {nu}x{nphi}")
    assert rel_l2(got, 0 * got, other, 0 * other) < FP32_TOL


def test_adjoint_dot_identity_and_gradient(torch_cuda):
    """<F(sigma), g> = <sigma, F^T(g)> through the tensor-core passes, and
    the autograd function's gradient of a weighted force loss against the FFT
    plan's."""
    torch = torch_cuda
    from paper_1509_01450_gb300 import self_gravity

    nu, nphi = 512, 256
    tc, fft, u_min, du = plans(nu, nphi)
    sigma = density(nu, nphi, u_min, du, 13)
    gr, gp = workloads.random_field(nu, nphi, 51), workloads.random_field(nu, nphi, 52)
    s = torch.tensor(sigma, dtype=torch.float32, device="cuda")
    Fr, Fp = tc.forces(s)
    gs = tc.backward(torch.tensor(gr, dtype=torch.float32, device="cuda"),
                     torch.tensor(gp, dtype=torch.float32, device="cuda"))
    tc.check()
    lhs = float(np.sum(Fr.double().cpu().numpy() * gr) + np.sum(Fp.double().cpu().numpy() * gp))
    rhs = float(np.sum(sigma * gs.double().cpu().numpy()))
    assert abs(lhs - rhs) <= 1e-5 * (abs(lhs) + abs(rhs))

    def grad(plan):
        x = s.clone().requires_grad_(True)
        Fr, Fp = self_gravity(x, plan)
        w = torch.linspace(0.5, 1.5, nu, device="cuda")[:, None]
        loss = (w * (Fr - 1.0) ** 2).sum() + (w * Fp ** 2).sum()
        loss.backward()
        return x.grad.double().cpu().numpy()

    a, b = grad(tc), grad(fft)
    assert rel_l2(a, 0 * a, b, 0 * b) < FP32_TOL
