"""sg_forces_host: the same forces from host buffers as sg_forces from device
buffers, bit for bit, on both of its paths: pinned (mapped) buffers, which
the kernels read and write over the host link, and pageable buffers, which
go through the plan's device staging copies."""
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


@pytest.mark.parametrize("nu,nphi", [(16, 32), (512, 1024), (2048, 4096)])
@pytest.mark.parametrize("dtype", ["float32", "float64"])
@pytest.mark.parametrize("pinned", [True, False])
def test_host_buffers_equal_device_call(torch_cuda, nu, nphi, dtype, pinned):
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    if dtype == "float64" and nphi > 4096:
        pytest.skip("FP64 plans stop at N_phi = 4096")
    u_min, du = workloads.grid_params(nu, 0.01, 100.0)
    plan = Plan(nu, nphi, u_min, du, 1.0, dtype).build()
    tdt = torch.float32 if dtype == "float32" else torch.float64
    sig = torch.tensor(np.abs(workloads.random_field(nu, nphi, 77)) + 0.1, dtype=tdt)
    Fr_d, Fp_d = plan.forces(sig.cuda())
    if pinned:
        sig = sig.pin_memory()
        fr = torch.empty_like(sig).pin_memory()
        fp = torch.empty_like(sig).pin_memory()
    else:
        fr = torch.empty_like(sig)
        fp = torch.empty_like(sig)
    for _ in range(2):  # twice: the staging buffers are made on the first call
        fr.fill_(float("nan"))
        fp.fill_(float("nan"))
        plan.forces_host(sig, fr, fp)
        assert torch.equal(fr, Fr_d.cpu()) and torch.equal(fp, Fp_d.cpu())
