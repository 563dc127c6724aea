"""Plan checkpoints and the device-side timeout path.

A plan saved and loaded again computes the same forces bit for bit without
a rebuild; damaged or foreign files are refused with SG_ERR_IO.  With the
wait budget set to zero every pass gives up on its input copies at once:
the host then sees SG_ERR_TIMEOUT (sg_plan_check, sg_forces_host), and with
the budget restored the plan computes as before.  Nothing here can fault a
GPU: a pass that gives up still waits (with the full budget) for the copies
it has started before it leaves.
"""
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


def _plan(nu, nphi, dtype, p=0):
    from paper_1509_01450_gb300 import Plan

    u_min, du = workloads.grid_params(nu, 0.01, 100.0)
    return Plan(nu, nphi, u_min, du, 1.0, dtype).build(weight_p=p)


@pytest.mark.parametrize("nu,nphi,dtype,p", [(64, 128, "float32", 0), (128, 64, "float64", 0), (32, 256, "float32", 2)])
def test_saved_plan_gives_the_same_forces(torch_cuda, tmp_path, nu, nphi, dtype, p):
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    plan = _plan(nu, nphi, dtype, p)
    sig = torch.tensor(np.abs(workloads.random_field(nu, nphi, 5)) + 0.1, dtype=plan.dtype, device="cuda")
    fr, fp = plan.forces(sig)
    path = str(tmp_path / "plan.sg")
    plan.save(path)
    again = Plan.load(path)
    assert again.info() == plan.info()
    fr2, fp2 = again.forces(sig)
    assert torch.equal(fr, fr2) and torch.equal(fp, fp2)
    g = again.backward(fr, fp)
    assert torch.equal(g, plan.backward(fr, fp))


def test_bad_plan_files_are_refused(torch_cuda, tmp_path):
    from paper_1509_01450_gb300 import Plan, SgError
    from paper_1509_01450_gb300.sg import SG_ERR_IO

    plan = _plan(16, 32, "float32")
    good = tmp_path / "good.sg"
    plan.save(str(good))
    data = good.read_bytes()
    cases = {"missing": None, "truncated": data[:-8], "longer": data + b"\0", "foreign": b"NOTAPLAN" + data[8:]}
    for name, content in cases.items():
        path = tmp_path / f"{name}.sg"
        if content is not None:
            path.write_bytes(content)
        with pytest.raises(SgError) as e:
            Plan.load(str(path))
        assert e.value.status == SG_ERR_IO, name


def test_zero_wait_budget_reports_a_timeout(torch_cuda):
    torch = torch_cuda
    from paper_1509_01450_gb300 import SgError, forces_batched
    from paper_1509_01450_gb300.sg import SG_ERR_TIMEOUT

    plan = _plan(256, 512, "float32")
    sig = torch.tensor(np.abs(workloads.random_field(256, 512, 9)) + 0.1, dtype=torch.float32, device="cuda")
    ref_r, ref_p = plan.forces(sig)
    plan.check()
    plan.set_wait_limit(0.0)
    try:
        plan.forces(sig)
        with pytest.raises(SgError) as e:
            plan.check()
        assert e.value.status == SG_ERR_TIMEOUT
        plan.backward(ref_r, ref_p)
        with pytest.raises(SgError) as e:
            plan.check()
        assert e.value.status == SG_ERR_TIMEOUT
        h = sig.cpu().pin_memory()
        with pytest.raises(SgError) as e:
            plan.forces_host(h, torch.empty_like(h).pin_memory(), torch.empty_like(h).pin_memory())
        assert e.value.status == SG_ERR_TIMEOUT
        fr, fp = torch.empty_like(sig), torch.empty_like(sig)
        forces_batched([(plan, sig, fr, fp)])
        with pytest.raises(SgError):
            plan.check()
    finally:
        plan.set_wait_limit(1.0)
    plan.check()  # the flag was cleared by the reads above
    fr, fp = plan.forces(sig)
    plan.check()
    assert torch.equal(fr, ref_r) and torch.equal(fp, ref_p)
