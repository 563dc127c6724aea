"""Batching workload: 256 exponential disks of uneven sizes (N_u in
{128..1024}, N_phi in {256..2048}, m = 1..4 spirals) through
sg_forces_batched, one stream.

Each disk's forces must equal its own sg_forces call bit for bit (same
passes, same plan); the smallest disks are compared with the FP64 oracle's
direct sum on sampled targets; and the whole batch, captured once in a CUDA
graph and replayed on new densities, must give the eager results.
"""
import math

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


@pytest.fixture(scope="module")
def batch(torch_cuda):
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan

    disks = workloads.batch_disks(256, 1450)
    plans = {}
    for d in disks:
        if (d.nu, d.nphi) not in plans:
            plans[(d.nu, d.nphi)] = Plan(d.nu, d.nphi, d.u_min, d.du, 1.0, "float32").build()
    sig = [torch.tensor(d.sigma(), dtype=torch.float32, device="cuda") for d in disks]
    return disks, plans, sig


def _outputs(torch, sig):
    return [torch.empty_like(s) for s in sig], [torch.empty_like(s) for s in sig]


def test_batch_equals_single_calls(torch_cuda, batch):
    torch = torch_cuda
    from paper_1509_01450_gb300 import forces_batched

    disks, plans, sig = batch
    assert len(plans) <= 16
    Fr, Fp = _outputs(torch, sig)
    forces_batched([(plans[(d.nu, d.nphi)], s, a, b) for d, s, a, b in zip(disks, sig, Fr, Fp)])
    for p in plans.values():
        p.check()
    bad = []
    for n, (d, s, a, b) in enumerate(zip(disks, sig, Fr, Fp)):
        er, ep = plans[(d.nu, d.nphi)].forces(s)
        if not (torch.equal(a, er) and torch.equal(b, ep)):
            scale = float(torch.maximum(er.abs().max(), ep.abs().max()))
            bad.append((n, d.nu, d.nphi, float((a - er).abs().max()) / scale, float((b - ep).abs().max()) / scale))
    assert not bad, f"{len(bad)} disks differ (index, N_u, N_phi, max |dF_r|, |dF_phi| / max |F|): {bad[:8]}"


def test_smallest_disks_match_oracle(torch_cuda, batch, oracle_mod):
    torch = torch_cuda
    from paper_1509_01450_gb300 import forces_batched

    disks, plans, sig = batch
    small = [n for n, d in enumerate(disks) if (d.nu, d.nphi) == (128, 256)][:3]
    assert small
    d0 = disks[small[0]]
    cells = oracle_mod.kernel_cells(d0.nu, d0.nphi, d0.du)
    Kr, Kp = oracle_mod.fold(cells, math.exp(d0.du), 2 * math.pi / d0.nphi)
    Fr, Fp = _outputs(torch, [sig[n] for n in small])
    forces_batched([(plans[(128, 256)], sig[n], a, b) for n, a, b in zip(small, Fr, Fp)])
    rng = np.random.default_rng(11)
    targets = rng.choice(d0.nu * d0.nphi, 2048, replace=False)
    for n, a, b in zip(small, Fr, Fp):
        rr, rp = oracle_mod.direct_sum(disks[n].sigma(), Kr, Kp, targets=targets)
        gr = a.double().cpu().numpy().reshape(-1)[targets]
        gp = b.double().cpu().numpy().reshape(-1)[targets]
        num = np.sum((gr - rr) ** 2 + (gp - rp) ** 2)
        den = np.sum(rr ** 2 + rp ** 2)
        assert math.sqrt(num / den) < 1e-5


def test_batch_replays_from_a_cuda_graph(torch_cuda, batch):
    torch = torch_cuda
    from paper_1509_01450_gb300 import forces_batched

    disks, plans, sig = batch
    n = 32  # a slice of the batch keeps the graph small
    src = [s.clone() for s in sig[:n]]
    Fr, Fp = _outputs(torch, src)
    items = [(plans[(d.nu, d.nphi)], s, a, b) for d, s, a, b in zip(disks[:n], src, Fr, Fp)]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(side):  # warm-up outside capture: attributes, occupancy queries
        forces_batched(items, stream=side)
    torch.cuda.current_stream().wait_stream(side)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        forces_batched(items, stream=torch.cuda.current_stream())
    rng = np.random.default_rng(5)
    for rep in range(2):
        for s in src:
            s.mul_(float(rng.uniform(0.5, 1.5)))
        g.replay()
        torch.cuda.synchronize()
        for d, s, a, b in zip(disks[:n], src, Fr, Fp):
            er, ep = plans[(d.nu, d.nphi)].forces(s)
            assert torch.equal(a, er) and torch.equal(b, ep)


def test_persistent_path_is_taken_and_others_fall_back(torch_cuda, batch):
    """The 256-disk batch qualifies for the one persistent launch
    (sg_batch_prepare accepts it); a batch with a plan built with the edge
    update does not, and still runs on the per-plan path."""
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan, SgError, batch_prepare, forces_batched, sg

    disks, plans, sig = batch
    Fr, Fp = _outputs(torch, sig)
    batch_prepare([(plans[(d.nu, d.nphi)], s, a, b) for d, s, a, b in zip(disks, sig, Fr, Fp)])
    d = disks[0]
    pe = Plan(d.nu, d.nphi, d.u_min, d.du, 1.0, "float32").build(radial_edges=1)
    items = [(pe, sig[0], Fr[0], Fp[0])]
    with pytest.raises(SgError) as ei:
        batch_prepare(items)
    assert ei.value.status == sg.SG_ERR_UNSUPPORTED
    forces_batched(items)
    er, ep = pe.forces(sig[0])
    assert torch.equal(Fr[0], er) and torch.equal(Fp[0], ep)


def test_bounded_waits_report_a_timeout(torch_cuda, batch):
    """With every plan's wait budget at 0 each wait of the persistent kernel
    gives up at once: every plan reports SG_ERR_TIMEOUT, and with the budget
    back the same plans give the single-call forces again."""
    torch = torch_cuda
    from paper_1509_01450_gb300 import SgError, forces_batched, sg

    disks, plans, sig = batch
    n = 24
    Fr, Fp = _outputs(torch, sig[:n])
    items = [(plans[(d.nu, d.nphi)], s, a, b) for d, s, a, b in zip(disks[:n], sig[:n], Fr, Fp)]
    used = {id(p): p for p, _, _, _ in items}.values()
    try:
        for p in used:
            p.set_wait_limit(0.0)
        forces_batched(items)
        torch.cuda.synchronize()
        for p in used:
            with pytest.raises(SgError) as ei:
                p.check()
            assert ei.value.status == sg.SG_ERR_TIMEOUT
    finally:
        for p in used:
            p.set_wait_limit(1.0)
    forces_batched(items)
    for p in used:
        p.check()
    for d, s, a, b in zip(disks[:n], sig[:n], Fr, Fp):
        er, ep = plans[(d.nu, d.nphi)].forces(s)
        assert torch.equal(a, er) and torch.equal(b, ep)


def test_tuned_schedule_is_cached_and_bit_equal(torch_cuda, batch, tmp_path):
    """sg_batch_tune picks a schedule (no slower than the default), appends
    it to the cache file, and takes it from there the second time; the
    tuned batch still equals the single calls."""
    torch = torch_cuda
    from paper_1509_01450_gb300 import batch_tune, forces_batched

    disks, plans, sig = batch
    n = 64
    Fr, Fp = _outputs(torch, sig[:n])
    items = [(plans[(d.nu, d.nphi)], s, a, b) for d, s, a, b in zip(disks[:n], sig[:n], Fr, Fp)]
    cache = str(tmp_path / "schedules.txt")
    t0, t1 = batch_tune(items, cache)
    assert 0 < t1 <= t0 * 1.02
    lines = open(cache).read().splitlines()
    assert len(lines) == 1 and lines[0].startswith("sg-batch-schedule v2 sms=")
    batch_tune(items, cache)  # found in the file: nothing appended
    assert open(cache).read().splitlines() == lines
    forces_batched(items)
    for d, s, a, b in zip(disks[:n], sig[:n], Fr, Fp):
        er, ep = plans[(d.nu, d.nphi)].forces(s)
        assert torch.equal(a, er) and torch.equal(b, ep)


def test_tensor_core_rows_keep_the_persistent_path(torch_cuda, batch):
    """The batch with its N_phi = 256 disks on plans built with short_dft
    (rows as tensor-core DFT products) still qualifies for the persistent
    path: those disks' row passes run as two batched tensor-core launches
    around the persistent column kernel.  Every disk equals its single call
    bit for bit, eagerly and replayed from a CUDA graph; the tensor-core
    disks also match the FFT plans within the FP32 bar."""
    torch = torch_cuda
    from paper_1509_01450_gb300 import Plan, batch_prepare, forces_batched

    disks, plans, sig = batch
    tcp = {}
    for d in disks:
        if d.nphi == 256 and (d.nu, d.nphi) not in tcp:
            tcp[(d.nu, d.nphi)] = Plan(d.nu, d.nphi, d.u_min, d.du, 1.0, "float32").build(short_dft=1)
    assert tcp, "the batch has disks with rows of 256"
    use = [tcp.get((d.nu, d.nphi), plans[(d.nu, d.nphi)]) for d in disks]
    Fr, Fp = _outputs(torch, sig)
    items = [(p, s, a, b) for p, s, a, b in zip(use, sig, Fr, Fp)]
    batch_prepare(items)  # raises unless the persistent path takes these items
    forces_batched(items)
    torch.cuda.synchronize()
    for p in set(use):
        p.check()
    for k, (p, s) in enumerate(zip(use, sig)):
        er, ep = p.forces(s)
        assert torch.equal(Fr[k], er) and torch.equal(Fp[k], ep), k
        if p in tcp.values():
            d = disks[k]
            gr, gp = plans[(d.nu, d.nphi)].forces(s)
            num = float(((er.double() - gr.double()) ** 2).sum() + ((ep.double() - gp.double()) ** 2).sum())
            den = float((gr.double() ** 2).sum() + (gp.double() ** 2).sum())
            assert (num / den) ** 0.5 < 1e-5, k
    Gr, Gp = _outputs(torch, sig)
    gitems = [(p, s, a, b) for p, s, a, b in zip(use, sig, Gr, Gp)]
    batch_prepare(gitems)  # the list is built outside the capture, which then records the persistent launches
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        forces_batched(gitems, stream=torch.cuda.current_stream())
    g.replay()
    torch.cuda.synchronize()
    assert all(torch.equal(a, b) for a, b in zip(Gr + Gp, Fr + Fp))
