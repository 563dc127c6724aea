"""Closed-form thin-disk forces used as truth for the oracle (test infrastructure).

Sec. 5.1 of Wang, Yen & Taam selects disks whose in-plane force is known in
closed form.  This module provides, with G = 1 unless given:

* Kuzmin disk: sigma = M a / (2 pi (r^2 + a^2)^{3/2}),
  F_r = -G M r / (r^2 + a^2)^{3/2}.
* The radial force of an axisymmetric annulus (complete elliptic integrals),
  used to remove the mass that a finite log-polar grid does not hold.
* The finite disks sigma_{D_n} = (1 - r^2/alpha^2)^{n - 1/2} (Eq. 50) and their
  radial forces.  The n = 1 member (Maclaurin disk) is Eq. 53 with
  b^1_0 = -1, a^1_1 = 1.  Higher members follow from the recursion Eq. 52,
  F_{n+1}(r; alpha) = (2n+1)/alpha^{2n+1} int_0^alpha ahat^{2n} F_n(r; ahat),
  evaluated here exactly: with x = r/alpha and z = 1/x the outside force is
  pi z^{-(2n-1)} [P(z) asin z + Q(z) sqrt(1-z^2) + R(z)] with rational
  polynomials P, Q, R, and the inside force is an odd polynomial in x whose
  coefficients are rational combinations of pi^2 and pi.  The coefficient
  recursion printed as Eq. 54-55 is garbled in the source and is not used.
"""
from __future__ import annotations

import math
from fractions import Fraction
from functools import lru_cache

import numpy as np

try:  # mpmath ships with sympy; needed only to evaluate the large-x tails
    import mpmath as _mp
except ImportError:  # pragma: no cover
    _mp = None


# --------------------------------------------------------------------------
# Kuzmin disk
# --------------------------------------------------------------------------
def kuzmin_sigma(r, M=1.0, a=1.0):
    r = np.asarray(r, dtype=np.float64)
    return M * a / (2.0 * math.pi * (r * r + a * a) ** 1.5)


def kuzmin_Fr(r, M=1.0, a=1.0, G=1.0):
    r = np.asarray(r, dtype=np.float64)
    return -G * M * r / (r * r + a * a) ** 1.5


# --------------------------------------------------------------------------
# Axisymmetric rings
# --------------------------------------------------------------------------
def ring_Q(r, rp):
    """Radial in-plane force at radius r per unit (sigma r' dr') of a thin ring
    of radius r' (G = 1):
        Q = -int_0^{2pi} (r - r' cos psi) / (r^2 + r'^2 - 2 r r' cos psi)^{3/2} dpsi.
    With A = r^2 + r'^2, B = 2 r r', m = 2B/(A+B) = 4 r r' / (r + r')^2:
        int dpsi (A - B cos)^{-3/2}     = 4 E(m) / ((A-B) sqrt(A+B))
        int dpsi (A - B cos)^{-1/2}     = 4 K(m) / sqrt(A+B)
        int dpsi cos (A - B cos)^{-3/2} = (A/B) I3 - (1/B) I1,
    which combine, without cancellation, to
        Q = -(2/r) [E(m) / (r - r') + K(m) / (r + r')].
    """
    from scipy.special import ellipe, ellipkm1

    r = np.asarray(r, dtype=np.float64)
    rp = np.asarray(rp, dtype=np.float64)
    p = ((r - rp) / (r + rp)) ** 2  # 1 - m, exact even where m rounds to 1
    return -(2.0 / r) * (ellipe(1.0 - p) / (r - rp) + ellipkm1(p) / (r + rp))


def ring_Q_offset(r, d):
    """ring_Q(r, r + d) with the offset d = r' - r given exactly (no
    rounding of r + d near the target's own ring)."""
    from scipy.special import ellipe, ellipkm1

    r = np.asarray(r, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    s = 2.0 * r + d  # r + r'
    p = (d / s) ** 2
    return -(2.0 / r) * (ellipe(1.0 - p) / (-d) + ellipkm1(p) / s)


def axisym_Fr(sigma_fn, r, r1, r2):
    """Radial force at r (scalar, r outside [r1, r2] or on its edge) of the
    axisymmetric density sigma_fn over r1 <= r' <= r2 (r2 may be inf)."""
    from scipy.integrate import quad

    f = lambda rp: sigma_fn(rp) * rp * ring_Q(r, rp)
    if math.isinf(r2):
        val, _ = quad(f, r1, np.inf, limit=400, epsabs=0.0, epsrel=1e-13)
    else:
        val, _ = quad(f, r1, r2, limit=400, epsabs=0.0, epsrel=1e-13)
    return val


def kuzmin_truncated_Fr(r, r_in, r_out, M=1.0, a=1.0):
    """Force of the part of a Kuzmin disk that lies in r_in <= r' <= r_out:
    the closed form minus the inner disk r' < r_in and the outer tail
    r' > r_out (each an axisymmetric ring integral)."""
    sig = lambda rp: float(kuzmin_sigma(rp, M, a))
    out = []
    for rr in np.atleast_1d(np.asarray(r, dtype=np.float64)):
        F = float(kuzmin_Fr(rr, M, a))
        F -= axisym_Fr(sig, rr, 0.0, r_in)
        F -= axisym_Fr(sig, rr, r_out, np.inf)
        out.append(F)
    return np.array(out)


def kuzmin_phi(r, M=1.0, a=1.0, G=1.0):
    """Potential of the Kuzmin disk in its plane, -G M / sqrt(r^2 + a^2)."""
    r = np.asarray(r, dtype=np.float64)
    return -G * M / np.sqrt(r * r + a * a)


def ring_phi(r, rp):
    """In-plane potential at radius r per unit (sigma r' dr') of a thin ring of
    radius r' (G = 1): -int_0^{2pi} dpsi / sqrt(r^2 + r'^2 - 2 r r' cos psi)
    = -4 K(m) / (r + r'), m = 4 r r' / (r + r')^2."""
    from scipy.special import ellipkm1

    r = np.asarray(r, dtype=np.float64)
    rp = np.asarray(rp, dtype=np.float64)
    p = ((r - rp) / (r + rp)) ** 2  # 1 - m
    return -4.0 * ellipkm1(p) / (r + rp)


def kuzmin_truncated_phi(r, r_in, r_out, M=1.0, a=1.0):
    """Potential of the part of a Kuzmin disk in r_in <= r' <= r_out: the
    closed form minus the rings r' < r_in and r' > r_out (targets r must lie
    inside (r_in, r_out), where neither integral meets the logarithmic
    singularity of its ring)."""
    from scipy.integrate import quad

    out = []
    for rr in np.atleast_1d(np.asarray(r, dtype=np.float64)):
        f = lambda rp: float(kuzmin_sigma(rp, M, a)) * rp * float(ring_phi(rr, rp))
        inner = quad(f, 0.0, r_in, limit=200, epsabs=0.0, epsrel=1e-12)[0]
        outer = quad(f, r_out, np.inf, limit=200, epsabs=0.0, epsrel=1e-12)[0]
        out.append(float(kuzmin_phi(rr, M, a)) - inner - outer)
    return np.array(out)


# --------------------------------------------------------------------------
# sigma_{D_n} family (Eq. 50-53), exact recursion
# --------------------------------------------------------------------------
# A polynomial is a dict {power: Fraction}.  An "outside" expression is the
# triple (P, Q, R) meaning P(w) asin w + Q(w) sqrt(1 - w^2) + R(w).


def _padd(a, b, s=1):
    out = dict(a)
    for k, v in b.items():
        out[k] = out.get(k, Fraction(0)) + s * v
    return {k: v for k, v in out.items() if v != 0}


def _pscale(a, s):
    return {k: v * s for k, v in a.items() if v * s != 0}


@lru_cache(maxsize=None)
def _I(p):
    """int w^p / sqrt(1 - w^2) dw as (P, Q, R):
    I_0 = asin w, I_1 = -sqrt(1-w^2),
    I_p = (-w^{p-1} sqrt(1-w^2) + (p-1) I_{p-2}) / p."""
    if p == 0:
        return ({0: Fraction(1)}, {}, {})
    if p == 1:
        return ({}, {0: Fraction(-1)}, {})
    P2, Q2, R2 = _I(p - 2)
    f = Fraction(p - 1, p)
    return (_pscale(P2, f), _padd(_pscale(Q2, f), {p - 1: Fraction(-1, p)}), _pscale(R2, f))


def _tadd(x, y, s=1):
    return tuple(_padd(a, b, s) for a, b in zip(x, y))


def _tscale(x, s):
    return tuple(_pscale(a, s) for a in x)


def _antideriv(P, Q, R):
    """Antiderivative of w * [P asin w + Q sqrt(1-w^2) + R] as (P', Q', R')."""
    acc = ({}, {}, {})
    for m0, c in P.items():  # int w^m asin w = w^{m+1} asin/(m+1) - I_{m+1}/(m+1)
        m = m0 + 1
        term = ({m + 1: Fraction(1, m + 1)}, {}, {})
        term = _tadd(term, _tscale(_I(m + 1), Fraction(-1, m + 1)))
        acc = _tadd(acc, _tscale(term, c))
    for m0, c in Q.items():  # int w^m sqrt(1-w^2) = I_m - I_{m+2}
        m = m0 + 1
        term = _tadd(_I(m), _I(m + 2), -1)
        acc = _tadd(acc, _tscale(term, c))
    for m0, c in R.items():
        m = m0 + 1
        acc = _tadd(acc, ({}, {}, {m + 1: c / (m + 1)}))
    return acc


def _peval(P, w):
    return sum(float(c) * w ** k for k, c in P.items()) if P else 0.0


@lru_cache(maxsize=None)
def dn_coefficients(n: int):
    """Exact representation of F_{D_n} (sigma_0 = G = 1) as a function of
    x = r / alpha.  Returns (inside, outside):
      inside  : {power: (a, b)} meaning sum (a pi^2 + b pi) x^power
      outside : (e, P, Q, R) meaning pi z^{-e} [P asin z + Q sqrt(1-z^2) + R],
                z = 1/x.
    """
    if n < 1:
        raise ValueError("n >= 1")
    inside = {1: (Fraction(-1, 2), Fraction(0))}  # Maclaurin: -pi^2 x / 2
    outside = (1, {0: Fraction(-1)}, {1: Fraction(1)}, {})  # pi z^{-1}[-asin z + z sqrt(1-z^2)]
    for k in range(1, n):
        e, P, Q, R = outside
        assert e == 2 * k - 1
        A = _antideriv(P, Q, R)
        A0 = A[1].get(0, Fraction(0)) + A[2].get(0, Fraction(0))  # value at w = 0
        Rn = _padd(A[2], {0: A0}, -1)
        f = Fraction(2 * k + 1)
        new_out = (2 * k + 1, _pscale(A[0], f), _pscale(A[1], f), _pscale(Rn, f))
        # C_k = int_1^inf f_k(y) y^{-2k-2} dy = pi [P_A(1) pi/2 + R_A(1) - A0]
        PA1 = sum(A[0].values(), Fraction(0))
        RA1 = sum(A[2].values(), Fraction(0))
        C = (PA1 / 2, RA1 - A0)  # (pi^2 coeff, pi coeff)
        new_in = {}
        # f_{k+1}^in(x) = (2k+1)[sum_j c_j (x^{2k+1} - x^{2j+1}) / (2j - 2k) + C x^{2k+1}]
        top = 2 * k + 1
        for pw, (a, b) in inside.items():
            jj = (pw - 1) // 2
            d = Fraction(1, 2 * jj - 2 * k)
            for p2, s in ((top, 1), (pw, -1)):
                a0, b0 = new_in.get(p2, (Fraction(0), Fraction(0)))
                new_in[p2] = (a0 + s * f * d * a, b0 + s * f * d * b)
        a0, b0 = new_in.get(top, (Fraction(0), Fraction(0)))
        new_in[top] = (a0 + f * C[0], b0 + f * C[1])
        inside = {p: v for p, v in new_in.items() if v[0] != 0 or v[1] != 0}
        outside = new_out
    return inside, outside


def dn_force(n: int, x):
    """Radial force f_n(x) of sigma_{D_n} with sigma_0 = G = 1 at x = r/alpha
    (negative = toward the disk centre).

    The outside branch is a difference of O(1) terms that leaves
    O(z^{2n+1}); it is evaluated in float64 where that cancellation costs at
    most 5 digits (z^{-(2n+1)} <= 1e5) and in 60-digit mpmath beyond."""
    inside, (e, P, Q, R) = dn_coefficients(n)
    xs = np.atleast_1d(np.asarray(x, dtype=np.float64))
    out = np.empty_like(xs)
    pi = math.pi
    ins = xs <= 1.0
    xi = xs[ins]
    out[ins] = sum((float(a) * pi * pi + float(b) * pi) * xi ** p for p, (a, b) in inside.items())
    xcut = 1e5 ** (1.0 / (2 * n + 1))
    near = (~ins) & (xs <= xcut)
    z = 1.0 / xs[near]
    pe = lambda poly: sum(float(c) * z ** k for k, c in poly.items()) if poly else 0.0
    out[near] = pi * z ** (-e) * (pe(P) * np.arcsin(z) + pe(Q) * np.sqrt(1.0 - z * z) + pe(R))
    far = np.nonzero(xs > xcut)[0]
    if far.size:
        if _mp is None:
            raise RuntimeError("mpmath needed far outside the disk")
        with _mp.workdps(60):
            for idx in far:
                zz = _mp.mpf(1) / _mp.mpf(xs[idx])
                pm = lambda poly: sum((_mp.mpf(c.numerator) / c.denominator) * zz ** k for k, c in poly.items())
                val = pm(P) * _mp.asin(zz) + pm(Q) * _mp.sqrt(1 - zz * zz) + pm(R)
                out[idx] = float(_mp.pi * zz ** (-e) * val)
    return out if np.ndim(x) else float(out[0])


def dn_sigma(n: int, x):
    """sigma_{D_n} / sigma_0 at x = r/alpha (Eq. 50)."""
    x = np.asarray(x, dtype=np.float64)
    return np.where(x < 1.0, np.clip(1.0 - x * x, 0.0, None) ** (n - 0.5), 0.0)


def dn_mass(n: int, alpha: float = 1.0) -> float:
    """Mass of sigma_{D_n} with sigma_0 = 1: 2 pi alpha^2 / (2n + 1)."""
    return 2.0 * math.pi * alpha * alpha / (2 * n + 1)


def dn_offcentre_forces(n: int, alpha: float, xc: float, yc: float, r, phi):
    """(F_r, F_phi) on the polar grid points (r[:, None], phi[None, :]) of a
    sigma_{D_n} disk centred at (xc, yc): the force is radial about the disk
    centre with magnitude f_n(d / alpha), projected on r-hat and phi-hat."""
    r = np.asarray(r, dtype=np.float64)[:, None]
    phi = np.asarray(phi, dtype=np.float64)[None, :]
    X = r * np.cos(phi) - xc
    Y = r * np.sin(phi) - yc
    d = np.sqrt(X * X + Y * Y)
    f = dn_force(n, (d / alpha).ravel()).reshape(d.shape)
    with np.errstate(invalid="ignore", divide="ignore"):
        ux = np.where(d > 0, X / d, 0.0)
        uy = np.where(d > 0, Y / d, 0.0)
    Fx, Fy = f * ux, f * uy
    Fr = Fx * np.cos(phi) + Fy * np.sin(phi)
    Fp = -Fx * np.sin(phi) + Fy * np.cos(phi)
    return Fr, Fp
