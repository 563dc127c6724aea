"""Repeatability: every pass is deterministic (no atomics in the force
path, fixed reduction orders), so repeated calls must give identical bits
however the work is scheduled: back to back, interleaved with other plans,
from forked streams (sg_forces_batched) and from a replayed CUDA graph.  A
race in a persistent pass, a ring or stage buffer, or between passes that
launch early would show up here as a changed bit."""
import numpy as np
import pytest

import workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01450_gb300 import build

    build.build()
    return torch


def _plan(nu, nphi, dtype="float32"):
    from paper_1509_01450_gb300 import Plan

    u_min, du = workloads.grid_params(nu, 0.01, 100.0)
    return Plan(nu, nphi, u_min, du, 1.0, dtype).build()


@pytest.mark.parametrize("nu,nphi,dtype", [(2048, 4096, "float32"), (512, 8192, "float32"), (1024, 1024, "float64")])
def test_repeated_calls_are_bit_identical(torch_cuda, nu, nphi, dtype):
    torch = torch_cuda
    from paper_1509_01450_gb300 import forces_batched

    plan = _plan(nu, nphi, dtype)
    other = _plan(256, 512, dtype)
    dt = plan.dtype
    sig = torch.tensor(np.abs(workloads.random_field(nu, nphi, 13)) + 0.1, dtype=dt, device="cuda")
    sig_o = torch.tensor(np.abs(workloads.random_field(256, 512, 14)) + 0.1, dtype=dt, device="cuda")
    Fr0, Fp0 = plan.forces(sig)
    g0 = plan.backward(Fr0, Fp0)
    Fr, Fp, g = torch.empty_like(Fr0), torch.empty_like(Fp0), torch.empty_like(g0)
    for rep in range(12):
        if rep % 3 == 1:
            other.forces(sig_o)
        if rep % 4 == 2:
            a, b = torch.empty_like(sig_o), torch.empty_like(sig_o)
            forces_batched([(plan, sig, Fr, Fp), (other, sig_o, a, b)])
        else:
            plan.forces(sig, Fr, Fp)
        plan.backward(Fr, Fp, g)
        torch.cuda.synchronize()
        assert torch.equal(Fr, Fr0) and torch.equal(Fp, Fp0) and torch.equal(g, g0), rep
    # the same passes captured once and replayed
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):
        plan.forces(sig, Fr, Fp, stream=side)
        plan.backward(Fr, Fp, g, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        plan.forces(sig, Fr, Fp)
        plan.backward(Fr, Fp, g)
    for _ in range(3):
        Fr.zero_()
        g.zero_()
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(Fr, Fr0) and torch.equal(Fp, Fp0) and torch.equal(g, g0)
    plan.check()
    other.check()
