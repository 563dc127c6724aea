"""sg_forces_noalloc through the C ABI: the forward pass for callers that may
not allocate device memory when they compute forces (their memory is owned
by another framework's allocator, or their loop must not allocate).  Its
scratch is a fixed array the library reserves on the device, so it must give
the results of sg_forces (same tolerance as the parity tests), on two calls
in a row with different inputs, and reject plans too large for that array.

This file sorts last so that a run stopping at its first failure has run
every other test already."""
import ctypes

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


def rel_l2(a_r, a_p, b_r, b_p):
    num = float(((a_r - b_r) ** 2).sum() + ((a_p - b_p) ** 2).sum())
    den = float((b_r ** 2).sum() + (b_p ** 2).sum())
    return (num / den) ** 0.5


# (N_u, N_phi, dtype, tolerance, build options): the default kernels, the
# one-sided radial edge slopes (their update runs inside the column pass),
# the potential and the Cartesian scheme (other tables on the same passes)
CASES = [(256, 512, "float32", 1e-5, {}), (1024, 2048, "float32", 1e-5, {}),
         (128, 256, "float64", 1e-12, {}), (1024, 1024, "float64", 1e-12, {}),
         (256, 512, "float32", 1e-5, {"radial_edges": 1}), (64, 128, "float64", 1e-12, {"radial_edges": 1}),
         (256, 512, "float32", 1e-5, {"kind": "potential", "weight_p": 1}),
         (128, 256, "float32", 1e-5, {"kind": "cartesian"})]


@pytest.mark.parametrize("nu,nphi,dtype,tol,kw", CASES)
def test_noalloc_matches_forces_twice(torch_cuda, nu, nphi, dtype, tol, kw):
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan, sg

    L = sg.lib()
    u_min, du = workloads.grid_params(nu, 0.01, 100.0)
    if kw.get("kind") == "cartesian":
        du = 2.0 / nu  # square cells over [-1, 1]
    plan = Plan(nu, nphi, u_min, du, 1.0, dtype).build(**kw)
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call, seed in enumerate((1, 2)):
        s = torch.tensor(np.abs(workloads.random_field(nu, nphi, seed)) + 0.1, dtype=plan.dtype, device="cuda")
        if kw.get("kind") == "cartesian":
            s[:, nphi // 2:] = 0  # the Cartesian plan's y-padding
        ref_r, ref_p = plan.forces(s)
        fr = torch.full_like(s, float("nan"))
        fp = torch.full_like(s, float("nan"))
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        st = L.sg_forces_noalloc(plan.handle, ctypes.c_void_p(s.data_ptr()), ctypes.c_void_p(fr.data_ptr()),
                                 ctypes.c_void_p(fp.data_ptr()), stream)
        assert st == sg.SG_OK, sg.status_string(st)
        torch.cuda.synchronize()
        # the call took no device memory (the scratch and the modules were
        # set up when the plan was built)
        assert torch.cuda.mem_get_info()[0] == free_before, call
        assert torch.isfinite(fr).all() and torch.isfinite(fp).all()
        assert rel_l2(fr.double(), fp.double(), ref_r.double(), ref_p.double()) <= tol, call


def test_noalloc_rejects_plans_beyond_its_scratch(torch_cuda):
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan, SgError, sg

    u_min, du = workloads.grid_params(2048, 0.01, 100.0)
    plan = Plan(2048, 4096, u_min, du, 1.0, "float32").build()
    s = torch.zeros((2048, 4096), device="cuda")
    with pytest.raises(SgError) as ei:
        plan.forces_noalloc(s, torch.empty_like(s), torch.empty_like(s))
    assert ei.value.status == sg.SG_ERR_UNSUPPORTED
