"""Cases for the checked-build test (tests/test_gpu_checked.py): every pass
kernel family of the library (the tensor-core row kernels included), small
and full size.  run_all() computes them
with whichever library sg.lib() loads; run as a script (with
SG_LIBRARY_VARIANT=checked) it builds and loads the index-checked library,
runs them, checks every plan's flags, and saves the results to the .npz
file named by its argument."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads  # noqa: E402

# (name, N_u, N_phi, dtype, build options, what to run)
CASES = [
    ("fixed-256x512", 256, 512, "float32", {}, "fb"),
    ("fixed-2048x4096", 2048, 4096, "float32", {}, "fb"),
    ("fixed-16x4096", 16, 4096, "float32", {}, "fb"),
    ("fixed-edges-4096x256", 4096, 256, "float32", {"radial_edges": 1}, "fb"),
    ("fixed-wedge-1024x2048", 1024, 2048, "float32", {"radial_edges": 1, "wedge": 1}, "w"),
    ("runtime-16x64", 16, 64, "float32", {}, "fb"),
    ("runtime-2048x16", 2048, 16, "float32", {}, "fb"),
    ("runtime-edges-64x128", 64, 128, "float32", {"radial_edges": 1}, "fb"),
    ("fp64-256x512", 256, 512, "float64", {}, "fb"),
    ("fp64-wedge-128x256", 128, 256, "float64", {"radial_edges": 1, "wedge": 1}, "w"),
    ("noalloc-256x512", 256, 512, "float32", {}, "n"),
    ("host-256x512", 256, 512, "float32", {}, "h"),
    ("tensor-core-rows-4096x256", 4096, 256, "float32", {"short_dft": 1}, "fb"),
    ("tensor-core-rows-128x128", 128, 128, "float32", {"short_dft": 1}, "fb"),
    ("tensor-core-rows-64x32", 64, 32, "float32", {"short_dft": 1}, "fb"),
]


def run_all():
    import torch

    from paper_1509_01450_gb300 import Plan, forces_batched

    out = {}
    for name, nu, nphi, dtype, opts, what in CASES:
        u_min, du = workloads.grid_params(nu, 0.1, 10.0)
        plan = Plan(nu, nphi, u_min, du, 1.0, dtype).build(**opts)
        dt = plan.dtype
        s = torch.tensor(np.abs(workloads.random_field(nu, nphi, nu + nphi)) + 0.1, dtype=dt, device="cuda")
        gr = torch.tensor(workloads.random_field(nu, nphi, 1), dtype=dt, device="cuda")
        gp = torch.tensor(workloads.random_field(nu, nphi, 2), dtype=dt, device="cuda")
        res = []
        if what == "fb":
            res += list(plan.forces(s)) + [plan.backward(gr, gp)]
        elif what == "w":
            sw = torch.tensor(0.5 + np.random.default_rng(nu).random(nphi), dtype=dt, device="cuda")
            res += list(plan.forces_wedge(s, sw)) + list(plan.backward_wedge(gr, gp))
        elif what == "n":
            fr, fp = torch.empty_like(s), torch.empty_like(s)
            res += list(plan.forces_noalloc(s, fr, fp))
        elif what == "h":
            sh = s.cpu()
            fr, fp = torch.empty_like(sh), torch.empty_like(sh)
            res += list(plan.forces_host(sh, fr, fp))
        plan.check()  # raises SgError (SG_ERR_BOUNDS) if an index check failed
        for k, a in enumerate(res):
            out[f"{name}/{k}"] = a.double().cpu().numpy()
        plan.close()
    # the batched entry point over plans of several sizes
    plans, items = [], []
    for n, (nu, nphi) in enumerate([(64, 128), (256, 512), (64, 128)]):
        u_min, du = workloads.grid_params(nu, 0.1, 10.0)
        p = Plan(nu, nphi, u_min, du, 1.0, "float32").build()
        s = torch.tensor(workloads.random_field(nu, nphi, 50 + n), dtype=torch.float32, device="cuda")
        plans.append(p)
        items.append((p, s, torch.empty_like(s), torch.empty_like(s)))
    forces_batched(items)
    for n, (p, s, fr, fp) in enumerate(items):
        p.check()
        out[f"batch/{n}/0"] = fr.double().cpu().numpy()
        out[f"batch/{n}/1"] = fp.double().cpu().numpy()
    # a persistent batch whose rows of 256 run on the tensor cores
    items = []
    for n, (nu, nphi, tc) in enumerate([(256, 256, 1), (256, 512, 0), (128, 256, 1)]):
        u_min, du = workloads.grid_params(nu, 0.1, 10.0)
        p = Plan(nu, nphi, u_min, du, 1.0, "float32").build(short_dft=tc)
        s = torch.tensor(workloads.random_field(nu, nphi, 60 + n), dtype=torch.float32, device="cuda")
        plans.append(p)
        items.append((p, s, torch.empty_like(s), torch.empty_like(s)))
    forces_batched(items)
    for n, (p, s, fr, fp) in enumerate(items):
        p.check()
        out[f"batch-tc/{n}/0"] = fr.double().cpu().numpy()
        out[f"batch-tc/{n}/1"] = fp.double().cpu().numpy()
    return out


if __name__ == "__main__":
    assert os.environ.get("SG_LIBRARY_VARIANT") == "checked"
    from paper_1509_01450_gb300 import build, sg

    build.build(checked=True)
    assert sg.lib().sg_checked_build() == 1
    res = run_all()
    np.savez(sys.argv[1], **res)
    print("checked run: %d arrays, last bounds site %d" % (len(res), sg.lib().sg_last_bounds_site()))
