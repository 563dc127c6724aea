"""Pins for the oracle's trapezoidal kernels (Eq. 41-43, the paper's SIM with
N_tpz trapezoids per cell in phi), against things other than the oracle's
own quadrature:

* Eq. 41-43 written out with the paper's closed-form eta-antiderivatives
  (App. A, 40-digit mpmath) at the trapezoid nodes, for N_tpz = 1 (Eq.
  38-40) and 3;
* the trapezoidal rule's second order: the gap to the exact cell integrals
  falls like N_tpz^-2;
* K^{phi,0}, K^{phi,r} and the own cell stay exact;
* the SIM orders of Table 1 with N_tpz = 19, the value of Sec. 5.3.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import analytic as A
from tests.conftest import load_golden

mpmath = pytest.importorskip("mpmath")
from tests.test_oracle_kernels import DU64, NPHI64, H_p1, H_p3, H_r1, H_r2  # noqa: E402

NU64 = 64


def closed_form_tpz(du, nphi, k, q, ntpz):
    """K^{r,0}, K^{r,r}, K^{r,phi}, K^{phi,phi} of Eq. 41-43 (and the same
    rule for K^{phi,phi}): the App. A antiderivative differences across the
    radial faces, summed by the trapezoidal rule over the azimuths
    phi'_m = phi_{j'-1/2} + (m - 1) dtheta."""
    mpmath.mp.dps = 40
    beta = mpmath.e ** mpmath.mpf(du)
    dphi = 2 * mpmath.pi / nphi
    qs = q % nphi
    if 2 * qs > nphi:
        qs -= nphi
    ec = beta ** (-k)
    el, eu = ec * 2 / (beta + 1), ec * 2 * beta / (beta + 1)
    xl = (-qs - mpmath.mpf(1) / 2) * dphi
    dth = dphi / ntpz
    nodes = [xl + m * dth for m in range(ntpz + 1)]

    def T(f):
        v = [f(x) for x in nodes]
        return dth * (sum(v) - (v[0] + v[-1]) / 2)

    r1 = lambda x: H_r1(eu, x) - H_r1(el, x)
    Kr0 = -T(r1)
    Krr = -T(lambda x: H_r2(eu, x) - H_r2(el, x)) - ec * Kr0  # Eq. 42: ... - (r_i'/r_i) K^{r,0}
    Krp = -T(lambda x: (x + qs * dphi) * r1(x))  # Eq. 43: phibar - phi_j' = xi - xi_c
    # K^{phi,phi}: the eta-integral of xi sin-kernel is H^phi_3's difference, and
    # that of the plain sin-kernel the xi-derivative of H^phi_1's corner form
    gp0 = lambda x: mpmath.diff(lambda y: H_p1(eu, y) - H_p1(el, y), x)
    Kpp = T(lambda x: (H_p3(eu, x) - H_p3(el, x)) + qs * dphi * gp0(x))
    return np.array([float(v) for v in (Kr0, Krr, Krp, Kpp)])


TPZ_CELLS = [(0, 1), (1, 0), (-1, 0), (1, 1), (-1, 63), (0, 2), (3, 60), (-4, 5), (7, 20), (-30, 3), (64, 0)]


@pytest.fixture(scope="module")
def tpz_tables(oracle_mod):
    return {n: oracle_mod.kernel_cells_tpz(NU64, NPHI64, DU64, n) for n in (1, 3)}


@pytest.mark.parametrize("ntpz", [1, 3])
@pytest.mark.parametrize("k,q", TPZ_CELLS)
def test_tpz_matches_eq41_43(tpz_tables, ntpz, k, q):
    got = tpz_tables[ntpz][[0, 1, 2, 5], k + NU64, q]
    ref = closed_form_tpz(DU64, NPHI64, k, q, ntpz)
    scale = abs(ref[0]) + 1e-300  # the cell's K^{r,0}
    for c in range(4):
        s = max(scale, abs(ref[c]))
        assert abs(got[c] - ref[c]) <= 2e-12 * s, (ntpz, k, q, c, got[c], ref[c])


def test_tpz_is_second_order_in_ntpz(oracle_mod):
    nu = nphi = 32
    du = math.log(100.0) / nu
    exact = oracle_mod.kernel_cells(nu, nphi, du)
    gaps = []
    for n in (9, 27, 81):
        t = oracle_mod.kernel_cells_tpz(nu, nphi, du, n)
        gaps.append([np.abs(t[c] - exact[c]).max() / np.abs(exact[c]).max() for c in (0, 1, 2, 5)])
        # exact where the paper is exact: K^{phi,0}, K^{phi,r}, and the own cell
        assert np.array_equal(t[3], exact[3]) and np.array_equal(t[4], exact[4])
        assert np.array_equal(t[:, nu, 0], exact[:, nu, 0])
    for g0, g1 in zip(gaps[:-1], gaps[1:]):
        for a, b in zip(g0, g1):
            assert 7.0 < a / b < 11.0, gaps  # 3x the trapezoids: 9x smaller


def test_sim_tpz19_orders_against_table1(oracle_mod):
    paper = {(d, norm, comp): float(v) for d, norm, comp, v in load_golden("table1_sim_orders.txt")}
    for n, sizes in ((2, (64, 128, 256)), (5, (128, 256, 512))):
        errs = []
        for N in sizes:
            u_min, du = workloads.grid_params(N, 0.01, 1.0)
            Kr, Kp = oracle_mod.kernels_tpz(N, N, du, 19)
            r, phi = workloads.centres(N, N, u_min, du)
            sig = workloads.sigma_dn(n, 0.25, 0.5, 0.1, r, phi)
            Fr, Fp = oracle_mod.fft_conv(sig, Kr, Kp)
            Ar, Ap = A.dn_offcentre_forces(n, 0.25, 0.5, 0.1, r, phi)
            errs.append((oracle_mod.norms(Fr, Ar), oracle_mod.norms(Fp, Ap)))
        for comp, ci in (("r", 0), ("phi", 1)):
            for norm, ni in (("L1", 0), ("L2", 1), ("Linf", 2)):
                got = math.log2(errs[-2][ci][ni] / errs[-1][ci][ni])
                want = paper[(f"D{n}", norm, comp)]
                if n == 5 or norm != "Linf":
                    assert got > 1.7 and abs(got - want) < 0.3, (n, norm, comp, got, want)
                else:
                    assert 1.0 < got < 1.9, (n, norm, comp, got, want)
