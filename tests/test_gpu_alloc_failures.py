"""The SG_ERR_ALLOC paths, by host-side injection (sg_test_fail_alloc): for
every device allocation that plan creation, the kernel build (with the edge
and wedge tables and the allocation-free set-up), the host-buffer entry
point and plan loading make, the call is repeated with that allocation
failing.  Each must return SG_ERR_ALLOC, release what it took (the
library's count of live allocations returns to where it was), and leave the
plan usable: a rebuilt
or reloaded plan gives the same forces as one that never failed."""
import gc

import pytest

import workloads

pytestmark = pytest.mark.gpu

NU, NPHI = 256, 512


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1509_01450_gb300 import build, sg

    build.build()
    L = sg.lib()
    yield torch, sg, L
    L.sg_test_fail_alloc(-1)


def _count(L, fn):
    """Number of allocations fn makes (the hook's budget it used)."""
    L.sg_test_fail_alloc(1 << 30)
    try:
        fn()
    finally:
        left = L.sg_test_fail_alloc(-1)
    return (1 << 30) - left


def _fails_at_each(torch, sg, L, fn, n, make=None, after=None):
    """fn(obj) with its k-th allocation failing, k = 0 .. n-1, obj = make()
    made afresh each time (before the hook is set): SG_ERR_ALLOC each time,
    and every allocation released once the objects are gone (the library's
    own count of live allocations; the device's free memory also moves with
    the CUDA driver's and torch's own caches)."""
    # plans that earlier tests left in reference cycles (a traceback keeps
    # its frames) are released now, not by a collection inside the loop
    gc.collect()
    torch.cuda.synchronize()
    live0 = L.sg_test_live_allocations()
    for k in range(n):
        obj = make() if make else None
        L.sg_test_fail_alloc(k)
        try:
            with pytest.raises(sg.SgError) as ei:
                fn(obj)
        finally:
            L.sg_test_fail_alloc(-1)
        assert ei.value.status == sg.SG_ERR_ALLOC, (k, str(ei.value))
        if after:
            after(obj)
        if obj is not None:
            obj.close()
    gc.collect()
    torch.cuda.synchronize()
    assert L.sg_test_live_allocations() == live0


def _grid():
    return workloads.grid_params(NU, 0.1, 10.0)


def _sigma(torch):
    return torch.tensor(workloads.random_field(NU, NPHI, 3) ** 2 + 0.1, dtype=torch.float32, device="cuda")


def test_plan_create(env):
    torch, sg, L = env
    from paper_1509_01450_gb300 import Plan

    u_min, du = _grid()
    n = _count(L, lambda: Plan(NU, NPHI, u_min, du, 1.0, "float32").close())
    assert n >= 10  # the plan's buffers, one allocation each
    _fails_at_each(torch, sg, L, lambda _: Plan(NU, NPHI, u_min, du, 1.0, "float32"), n)


@pytest.mark.parametrize("opts", [{}, {"radial_edges": 1, "wedge": 1}])
def test_kernel_build_leaves_the_plan_unbuilt(env, opts):
    torch, sg, L = env
    from paper_1509_01450_gb300 import Plan

    u_min, du = _grid()
    ref = Plan(NU, NPHI, u_min, du, 1.0, "float32").build(**opts)
    plan = Plan(NU, NPHI, u_min, du, 1.0, "float32")
    n = _count(L, lambda: plan.build(**opts))
    assert n >= 5  # the build's scratch, the allocation-free set-up's fields (and the edge and wedge tables)
    plan.close()
    s = _sigma(torch)
    sw = torch.full((NPHI,), 0.7, device="cuda")

    def unbuilt(p):
        with pytest.raises(sg.SgError) as ei:
            p.forces(s)
        assert ei.value.status == sg.SG_ERR_NOT_BUILT

    _fails_at_each(torch, sg, L, lambda p: p.build(**opts), n,
                   make=lambda: Plan(NU, NPHI, u_min, du, 1.0, "float32"), after=unbuilt)
    plan = Plan(NU, NPHI, u_min, du, 1.0, "float32")
    L.sg_test_fail_alloc(n - 1)
    try:
        with pytest.raises(sg.SgError):
            plan.build(**opts)  # a failed build, then a good one on the same plan
    finally:
        L.sg_test_fail_alloc(-1)
    plan.build(**opts)
    if opts.get("wedge"):
        a, b = plan.forces_wedge(s, sw), ref.forces_wedge(s, sw)
    else:
        a, b = plan.forces(s), ref.forces(s)
    plan.check()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_host_entry_point(env):
    torch, sg, L = env
    from paper_1509_01450_gb300 import Plan

    u_min, du = _grid()
    plan = Plan(NU, NPHI, u_min, du, 1.0, "float32").build()
    s = _sigma(torch)
    # pageable host memory takes the staged path, which allocates its three
    # device buffers on the first call
    sh = s.cpu()
    fr, fp = torch.empty_like(sh), torch.empty_like(sh)
    _fails_at_each(torch, sg, L, lambda p: p.forces_host(sh, fr, fp), 3,
                   make=lambda: Plan(NU, NPHI, u_min, du, 1.0, "float32").build())
    L.sg_test_fail_alloc(1)
    try:
        with pytest.raises(sg.SgError):
            plan.forces_host(sh, fr, fp)  # one buffer taken, then the call goes through
    finally:
        L.sg_test_fail_alloc(-1)
    plan.forces_host(sh, fr, fp)
    Fr, Fp = plan.forces(s)
    assert torch.equal(fr, Fr.cpu()) and torch.equal(fp, Fp.cpu())


def test_plan_load(env, tmp_path):
    torch, sg, L = env
    from paper_1509_01450_gb300 import Plan

    u_min, du = _grid()
    plan = Plan(NU, NPHI, u_min, du, 1.0, "float32").build()
    path = str(tmp_path / "plan.sg")
    plan.save(path)
    n = _count(L, lambda: Plan.load(path).close())
    assert n >= 10
    _fails_at_each(torch, sg, L, lambda _: Plan.load(path), n)
    s = _sigma(torch)
    a, b = Plan.load(path).forces(s), plan.forces(s)
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])
