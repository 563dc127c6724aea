"""Pins for the analytic truth used by the oracle tests (oracle/analytic.py).

* Ring force (elliptic integrals) against direct quadrature over the ring.
* Kuzmin and Maclaurin (sigma_{D_1}) closed forms against ring integration of
  their densities.
* sigma_{D_n} forces: the recursion Eq. 52 evaluated by numerical quadrature,
  the mass rule F -> -M_n / r^2, continuity at the disk edge, and the
  Chebyshev coefficients of Eq. 53 for n = 1 and n = 2 (the n = 2 values from
  one step of the printed recursion Eq. 54-55; tests/golden).
"""
import math
from fractions import Fraction

import numpy as np
import pytest
from scipy.integrate import quad

from oracle import analytic as A
from tests.conftest import load_golden


@pytest.mark.parametrize("r,rp", [(1.0, 0.3), (1.0, 3.0), (2.0, 1.9), (0.5, 0.51), (0.05, 20.0)])
def test_ring_force_matches_quadrature(r, rp):
    f = lambda p: -(r - rp * math.cos(p)) / (r * r + rp * rp - 2 * r * rp * math.cos(p)) ** 1.5
    ref = quad(f, 0, 2 * math.pi, points=[math.pi], limit=400, epsabs=0, epsrel=1e-13)[0]
    # E/(r - r') and K/(r + r') cancel to O(m) for a distant ring: ~1e-11
    assert abs(float(A.ring_Q(r, rp)) - ref) < 1e-10 * abs(ref)
    assert abs(float(A.ring_Q_offset(r, rp - r)) - ref) < 1e-10 * abs(ref)


def _axisym_pv(sigma_fn, r, r1, r2):
    """Force at r of sigma over [r1, r2] with r inside: the ring through the
    target makes a principal value, taken by folding about r' = r."""
    f = lambda rp: sigma_fn(rp) * rp * float(A.ring_Q(r, rp))
    fo = lambda d: sigma_fn(r + d) * (r + d) * float(A.ring_Q_offset(r, d))
    h = min(r - r1, r2 - r)
    v = quad(lambda t: fo(t) + fo(-t), 0.0, h, limit=400, epsabs=0, epsrel=1e-12)[0]
    if r - h > r1:
        v += quad(f, r1, r - h, limit=400, epsabs=0, epsrel=1e-12)[0]
    if r + h < r2:
        v += quad(f, r + h, r2, limit=400, epsabs=0, epsrel=1e-12)[0]
    return v


@pytest.mark.parametrize("r", [0.3, 1.0, 2.5])
def test_kuzmin_closed_form_by_ring_integration(r):
    sig = lambda rp: float(A.kuzmin_sigma(rp))
    ref = _axisym_pv(sig, r, 0.0, 2 * r) + A.axisym_Fr(sig, r, 2 * r, np.inf)
    assert abs(float(A.kuzmin_Fr(r)) - ref) < 1e-9 * abs(ref)


@pytest.mark.parametrize("x", [0.25, 0.7, 1.3, 3.0])
def test_maclaurin_closed_form_by_ring_integration(x):
    sig = lambda rp: math.sqrt(max(1.0 - rp * rp, 0.0))
    if x < 1.0:
        ref = _axisym_pv(sig, x, 0.0, 1.0)
    else:
        ref = A.axisym_Fr(sig, x, 0.0, 1.0)
    assert abs(A.dn_force(1, x) - ref) < 1e-8 * abs(ref)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_dn_recursion_eq52(n):
    for x in (0.3, 0.9, 1.5, 4.0):
        f = lambda s: s ** (2 * (n - 1)) * A.dn_force(n - 1, x / s)
        v = quad(f, 0, 1, points=[x] if x < 1 else None, limit=200, epsabs=0, epsrel=1e-13)[0]
        # float64 evaluation of the outside branch is good to ~1e-11 (dn_force)
        assert abs((2 * n - 1) * v - A.dn_force(n, x)) < 1e-11 * abs(A.dn_force(n, x))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_dn_mass_and_edge(n):
    x = 1e3
    assert abs(A.dn_force(n, x) * x * x + A.dn_mass(n)) < 1e-5 * A.dn_mass(n)
    if n >= 2:  # continuous at the edge (n = 1 has a sqrt cusp)
        assert abs(A.dn_force(n, 1 - 1e-9) - A.dn_force(n, 1 + 1e-9)) < 1e-7


def _cheb_T(k):
    """Coefficients of T_k as {power: int}."""
    a, b = {0: 1}, {1: 1}
    if k == 0:
        return a
    for _ in range(k - 1):
        c = {}
        for p, v in b.items():
            c[p + 1] = c.get(p + 1, 0) + 2 * v
        for p, v in a.items():
            c[p] = c.get(p, 0) - v
        a, b = b, c
    return b


def test_eq53_chebyshev_coefficients_match_paper():
    """The exact outside polynomials P_n (asin part) and Q_n (sqrt part) equal
    sum b^n_{2k} T_{2k}(z) and sum a^n_{2k+1} T_{2k+1}(z) with the paper's
    coefficients (Eq. 53; n = 2 from Eq. 54-55)."""
    rows = load_golden("dn_chebyshev_coefficients.txt")
    coef = {}
    for n, kind, idx, num, den in rows:
        coef.setdefault(int(n), {})[(kind, int(idx))] = Fraction(int(num), int(den))
    for n, cs in coef.items():
        _, (e, P, Q, R) = A.dn_coefficients(n)
        assert e == 2 * n - 1 and not R
        wantP, wantQ = {}, {}
        for (kind, idx), v in cs.items():
            tgt = wantP if kind == "b" else wantQ
            for p, c in _cheb_T(idx).items():
                tgt[p] = tgt.get(p, Fraction(0)) + v * c
        clean = lambda d: {p: v for p, v in d.items() if v != 0}
        assert clean(wantP) == clean(P), (n, wantP, P)
        assert clean(wantQ) == clean(Q), (n, wantQ, Q)
        # inside branch: (pi^2/2) x^{2n-1} sum b T_{2k}(1/x), a polynomial in x
        ins, _ = A.dn_coefficients(n)
        for x in (0.2, 0.6, 0.95):
            z = 1.0 / x
            val = 0.5 * math.pi ** 2 * x ** (2 * n - 1) * sum(
                float(v) * sum(c * z ** p for p, c in _cheb_T(idx).items())
                for (kind, idx), v in cs.items() if kind == "b")
            assert abs(val - A.dn_force(n, x)) < 1e-12 * abs(val)
