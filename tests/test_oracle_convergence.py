"""End-to-end pins of the oracle against analytic disks (Sec. 5).

* Kuzmin disk (the closed form F_r = -r/(r^2+1)^{3/2}, with the mass the
  finite grid does not hold removed by ring integrals): second-order
  convergence on interior targets.
* sigma_{D_2} and sigma_{D_5} disks of Sec. 5.3 (alpha = 0.25 centred at
  (0.5, 0.1) on the destination grid [0.01, 1] x [0, 2 pi)): fitted orders in
  the L1, L2, Linf norms of Eq. 47-49 compared with the SIM column of Table 1
  (tests/golden/table1_sim_orders.txt).
* Momentum: sum sigma A (F_x, F_y) -> 0 under refinement.

The oracle's direct sum equals its FFT evaluation to ~1e-14
(test_oracle_sums), so the larger grids here use the FFT form.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import analytic as A
from tests.conftest import load_golden


def _solve(oracle_mod, n, r_in, r_out, sigma_fn):
    u_min, du = workloads.grid_params(n, r_in, r_out)
    Kr, Kp = oracle_mod.kernels(n, n, du)
    r, phi = workloads.centres(n, n, u_min, du)
    sig = sigma_fn(r, phi)
    Fr, Fp = oracle_mod.fft_conv(sig, Kr, Kp)
    return r, phi, sig, Fr, Fp, du


def test_kuzmin_second_order_interior(oracle_mod):
    errs = []
    for n in (32, 64, 128):
        r, phi, sig, Fr, Fp, _ = _solve(oracle_mod, n, 0.05, 20.0, workloads.kuzmin)
        truth = A.kuzmin_truncated_Fr(r, 0.05, 20.0)
        m = (r >= 0.2) & (r <= 5.0)  # 4 r_in .. r_out / 4
        errs.append(np.abs(Fr[:, 0] - truth)[m].max())
        assert np.abs(Fp).max() < 1e-14 * np.abs(Fr).max()
    orders = [math.log2(a / b) for a, b in zip(errs[:-1], errs[1:])]
    assert orders[-1] > 1.75 and orders[-1] > orders[0], orders
    assert errs[-1] < 5e-5


@pytest.fixture(scope="module")
def dn_orders(oracle_mod):
    out = {}
    for n, sizes in ((2, (64, 128, 256)), (5, (128, 256, 512))):
        errs = []
        for N in sizes:
            r, phi, sig, Fr, Fp, _ = _solve(oracle_mod, N, 0.01, 1.0,
                                            lambda r, p: workloads.sigma_dn(n, 0.25, 0.5, 0.1, r, p))
            Ar, Ap = A.dn_offcentre_forces(n, 0.25, 0.5, 0.1, r, phi)
            errs.append((oracle_mod.norms(Fr, Ar), oracle_mod.norms(Fp, Ap)))
        fit = {}
        for comp, ci in (("r", 0), ("phi", 1)):
            for norm, ni in (("L1", 0), ("L2", 1), ("Linf", 2)):
                e = [x[ci][ni] for x in errs]
                fit[(norm, comp)] = math.log2(e[-2] / e[-1])
        out[f"D{n}"] = fit
    return out


def test_dn_orders_against_table1(dn_orders):
    paper = {(d, norm, comp): float(v) for d, norm, comp, v in load_golden("table1_sim_orders.txt")}
    for (disk, norm, comp), want in paper.items():
        got = dn_orders[disk][(norm, comp)]
        if disk == "D5" or norm != "Linf":
            # smooth density (or global norms): second order as in Table 1
            assert got > 1.7 and abs(got - want) < 0.3, (disk, norm, comp, got, want)
        else:
            # sigma_{D_2} has a singular second derivative at its edge: the
            # max-norm order stays below 2 (Table 1: 1.4 - 1.5)
            assert 1.0 < got < 1.9, (disk, norm, comp, got, want)


def test_momentum_vanishes_under_refinement(oracle_mod):
    rel = []
    for n in (64, 128):
        r, phi, sig, Fr, Fp, du = _solve(oracle_mod, n, 0.01, 1.0,
                                         lambda r, p: workloads.sigma_dn(5, 0.25, 0.5, 0.1, r, p))
        area = workloads.cell_areas(n, n, math.log(0.01), du)[:, None]
        c, s = np.cos(phi)[None, :], np.sin(phi)[None, :]
        Fx, Fy = Fr * c - Fp * s, Fr * s + Fp * c
        w = sig * area
        P = math.hypot(np.sum(w * Fx), np.sum(w * Fy))
        rel.append(P / np.sum(w * np.hypot(Fx, Fy)))
    assert rel[1] < rel[0] and rel[1] < 1e-3, rel
