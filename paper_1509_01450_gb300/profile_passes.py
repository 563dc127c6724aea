"""Run the forward and adjoint passes a few times on one plan, for an
external profiler (ncu) to capture: ``python -m
paper_1509_01450_gb300.profile_passes N_u N_phi [float32|float64]``.

The plan spans r in [0.01, 100] with the exact SIM kernels; the density is
uniform random.  One forward pass, then three forward + adjoint pairs (so a
capture that skips the first forward's launches sees warm code and the
steady-state launch order); the plan's device-side error flag is checked at
the end."""
import math
import sys


def main(argv=None):
    import torch

    from .sg import Plan

    argv = sys.argv[1:] if argv is None else argv
    nu, nphi = int(argv[0]), int(argv[1])
    dtype = argv[2] if len(argv) > 2 else "float32"
    plan = Plan(nu, nphi, math.log(0.01), math.log(1e4) / nu, 1.0, dtype).build()
    s = torch.rand(nu, nphi, dtype=plan.dtype, device="cuda")
    Fr, Fp = plan.forces(s)
    for _ in range(3):
        plan.forces(s, Fr, Fp)
        plan.backward(Fr, Fp)
    torch.cuda.synchronize()
    plan.check()
    print("ok")


if __name__ == "__main__":
    main()
