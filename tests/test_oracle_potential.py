"""Pins for the oracle's potential cells and potential (the paper's method
carried over to the potential, which its Sec. 6 says applies), against
things other than the oracle's quadrature:

* the closed-form eta-antiderivatives of eta / F and eta^2 / F, with the
  remaining xi integral in 40-digit mpmath, at 9 offsets including the own
  cell;
* the Kuzmin disk, Phi = -G M / sqrt(r^2 + a^2), minus the potential of the
  mass that the finite grid does not hold (ring potentials, -2 G dm K(m) /
  (pi (r + r'))): second-order convergence on interior targets;
* the forces: the central difference of Phi along r converges to the
  oracle's F_r at second order.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import analytic as A

mpmath = pytest.importorskip("mpmath")

DU64 = math.log(400.0) / 64
NPHI64 = 64


def _uFL(e, x):
    """u = eta - c, F, and ln(u + F) without cancellation (for u < 0,
    u + F = s^2 / (F - u))."""
    c, s = mpmath.cos(x), mpmath.sin(x)
    u = e - c
    F = mpmath.sqrt(u * u + s * s)
    L = mpmath.log(u + F) if u >= 0 else mpmath.log(s * s) - mpmath.log(F - u)
    return c, s, u, F, L


def _P(e, x):
    """d/deta P = eta / F (F^2 = (eta - c)^2 + s^2, c, s = cos, sin x)."""
    c, s, u, F, L = _uFL(e, x)
    return F + c * L


def _Q(e, x):
    """d/deta Q = eta^2 / F."""
    c, s, u, F, L = _uFL(e, x)
    return (u * F - s * s * L) / 2 + 2 * c * F + c * c * L


def closed_form_potential_cell(du, nphi, k, q):
    mpmath.mp.dps = 40
    beta = mpmath.e ** mpmath.mpf(du)
    dphi = 2 * mpmath.pi / nphi
    qs = q % nphi
    if 2 * qs > nphi:
        qs -= nphi
    ec = beta ** (-k)
    el, eu = ec * 2 / (beta + 1), ec * 2 * beta / (beta + 1)
    xl, xu = (-qs - mpmath.mpf(1) / 2) * dphi, (-qs + mpmath.mpf(1) / 2) * dphi
    pts = [xl, 0, xu] if (xl < 0 < xu) else [xl, xu]
    quadx = lambda f: mpmath.quad(f, pts)
    p = lambda x: _P(eu, x) - _P(el, x)
    K0 = -quadx(p)
    Kr = -quadx(lambda x: (_Q(eu, x) - _Q(el, x)) - ec * p(x))
    Kf = -quadx(lambda x: (x + qs * dphi) * p(x))
    return np.array([float(K0), float(Kr), float(Kf)])


@pytest.mark.parametrize("k,q", [(0, 0), (0, 1), (1, 0), (-1, 0), (1, 1), (3, 60), (-4, 5), (20, 32), (-30, 3)])
def test_potential_cells_match_closed_forms(oracle_mod, k, q):
    got = oracle_mod.potential_cell(DU64, NPHI64, k, q)
    ref = closed_form_potential_cell(DU64, NPHI64, k, q)
    scale = abs(ref[0])
    for c in range(3):
        assert abs(got[c] - ref[c]) <= 2e-12 * scale, (k, q, c, got[c], ref[c])
    assert not np.any(got[3:])


def test_kuzmin_potential_second_order_interior(oracle_mod):
    errs = []
    for n in (32, 64, 128):
        u_min, du = workloads.grid_params(n, 0.05, 20.0)
        grid = oracle_mod.Grid(n, n, u_min, du)
        cells = oracle_mod.potential_cells(n, n, du)
        sig = workloads.kuzmin(grid.r, grid.phi)
        Phi = oracle_mod.potential(sig, cells, grid)
        m = (grid.r >= 0.2) & (grid.r <= 5.0)
        truth = A.kuzmin_truncated_phi(grid.r[m], 0.05, 20.0)
        errs.append(np.abs(Phi[m, 0] - truth).max() / np.abs(truth).max())
        assert np.ptp(Phi, axis=1).max() < 1e-13 * np.abs(Phi).max()  # axisymmetric
    orders = [math.log2(a / b) for a, b in zip(errs[:-1], errs[1:])]
    assert orders[-1] > 1.7 and errs[-1] < 4e-4, (errs, orders)


def test_potential_gradient_is_the_radial_force(oracle_mod):
    """-(Phi_{i+1} - Phi_{i-1}) / (r_{i+1} - r_{i-1}) against F_r on the
    interior rows of a spiral disk (0.3 <= r <= 1.5): the gap falls at
    second order."""
    gaps = []
    for n in (32, 64, 128):
        u_min, du = workloads.grid_params(n, 0.05, 20.0)
        grid = oracle_mod.Grid(n, n, u_min, du)
        sig = workloads.spiral_clump(grid.r, grid.phi)
        Phi = oracle_mod.potential(sig, oracle_mod.potential_cells(n, n, du), grid)
        Kr, Kp = oracle_mod.kernels(n, n, du)
        Fr, _ = oracle_mod.fft_conv(sig, Kr, Kp)
        dPhi = -(Phi[2:] - Phi[:-2]) / (grid.r[2:] - grid.r[:-2])[:, None]
        m = (grid.r[1:-1] >= 0.3) & (grid.r[1:-1] <= 1.5)  # inside the clump at r = 3 (scale 0.2)
        gaps.append(np.abs(dPhi[m] - Fr[1:-1][m]).max() / np.abs(Fr[1:-1][m]).max())
    orders = [math.log2(a / b) for a, b in zip(gaps[:-1], gaps[1:])]
    assert orders[-1] > 1.8 and gaps[-1] < 2e-3, (gaps, orders)


@pytest.mark.parametrize("r,rp", [(1.0, 0.3), (0.5, 2.0), (3.0, 2.9), (0.2, 20.0)])
def test_ring_potential_closed_form(r, rp):
    """The ring potential's elliptic form against the angle integral itself."""
    from scipy.integrate import quad

    ref = -quad(lambda p: 1.0 / math.sqrt(r * r + rp * rp - 2 * r * rp * math.cos(p)), 0.0, 2 * math.pi,
                epsabs=0, epsrel=1e-13, limit=400)[0]
    assert abs(A.ring_phi(r, rp) - ref) < 1e-12 * abs(ref)
