"""Pins for the oracle's Cartesian second-order scheme (Sec. 3.1.1, App. A),
against things other than its own closed forms:

* the six cell integrals (Eq. 13-15 and their y forms) by adaptive 2-D
  quadrature of the raw integrands, at offsets off the own cell, for square
  and oblong cells;
* the own cell: K^{x,0}, K^{y,0}, K^{x,y} vanish by symmetry, and
  K^{x,x} over a square of half-side h is 4 h ln(1 + sqrt 2) (the polar
  integral of cos^2 theta rho_max(theta)), over an oblong cell the same
  integral by quadrature;
* the fold equals the literal sums, the FFT convolution equals both;
* the y kernels are the x kernels with the axes swapped on square cells;
* off-centre sigma_{D_5} and sigma_{D_2} disks inside the square: the
  convergence orders of the force error to the closed form (Sec. 5.1).
"""
import math

import numpy as np
import pytest
from scipy.integrate import dblquad, quad

from oracle import analytic as A
from oracle import cartesian as C


def _raw(k, q, dx, dy):
    xl, xu = (-k - 0.5) * dx, (-k + 0.5) * dx
    yl, yu = (-q - 0.5) * dy, (-q + 0.5) * dy
    R3 = lambda X, Y: (X * X + Y * Y) ** 1.5
    fs = [lambda Y, X: X / R3(X, Y),
          lambda Y, X: X * (X + k * dx) / R3(X, Y),
          lambda Y, X: X * (Y + q * dy) / R3(X, Y),
          lambda Y, X: Y / R3(X, Y),
          lambda Y, X: (X + k * dx) * Y / R3(X, Y),
          lambda Y, X: Y * (Y + q * dy) / R3(X, Y)]
    return np.array([dblquad(f, xl, xu, yl, yu, epsabs=0, epsrel=1e-12)[0] for f in fs])


@pytest.mark.parametrize("dx,dy", [(0.1, 0.1), (0.1, 0.07)])
@pytest.mark.parametrize("k,q", [(1, 0), (0, 1), (1, 1), (2, -3), (-4, 1), (7, 5), (0, -9)])
def test_cells_against_quadrature(k, q, dx, dy):
    K = C.cells(10, 10, dx, dy)
    got = K[:, k + 10, q + 10]
    ref = _raw(k, q, dx, dy)
    scale = np.abs(ref).max()
    assert np.all(np.abs(got - ref) <= 1e-10 * scale), (got, ref)


def _own_xx(hx, hy):
    """int int X^2 / R^3 over [-hx, hx] x [-hy, hy] in polar form."""
    t = math.atan2(hy, hx)
    f1 = lambda th: math.cos(th) ** 2 * hx / math.cos(th)
    f2 = lambda th: math.cos(th) ** 2 * hy / math.sin(th)
    return 4.0 * (quad(f1, 0.0, t, epsabs=0, epsrel=1e-13)[0] + quad(f2, t, math.pi / 2, epsabs=0, epsrel=1e-13)[0])


@pytest.mark.parametrize("dx,dy", [(0.1, 0.1), (0.1, 0.07), (0.03, 0.2)])
def test_own_cell(dx, dy):
    K = C.cells(3, 3, dx, dy)[:, 3, 3]
    s = abs(K[1])
    assert abs(K[0]) < 1e-15 * s and abs(K[3]) < 1e-15 * s and abs(K[2]) < 1e-15 * s and abs(K[4]) < 1e-15 * s
    assert abs(K[1] - _own_xx(dx / 2, dy / 2)) < 1e-13 * s
    assert abs(K[5] - _own_xx(dy / 2, dx / 2)) < 1e-13 * s
    if dx == dy:
        assert abs(K[1] - 4 * (dx / 2) * math.log(1 + math.sqrt(2))) < 1e-14 * s


def test_axis_swap_and_parity():
    K = C.cells(6, 6, 0.05)
    for a, b in ((0, 3), (1, 5), (2, 4)):
        assert np.abs(K[a] - K[b].T).max() < 1e-14 * np.abs(K[a]).max()
    assert np.abs(K[0] + K[0][::-1, :]).max() < 1e-14 * np.abs(K[0]).max()  # odd in k
    assert np.abs(K[0] - K[0][:, ::-1]).max() < 1e-14 * np.abs(K[0]).max()  # even in q


@pytest.mark.parametrize("nx,ny,dy", [(5, 6, 0.2), (4, 4, 0.25), (6, 3, 0.13)])
def test_fold_and_fft_equal_the_literal_sums(nx, ny, dy):
    rng = np.random.default_rng(7)
    sigma = rng.random((nx, ny))
    dx = 0.2
    K = C.cells(nx, ny, dx, dy)
    Fx, Fy = C.three_sum(sigma, K, dx, dy)
    Kx, Ky = C.fold(K, dx, dy)
    Gx, Gy = C.forces(sigma, Kx, Ky)
    s = np.abs(Fx).max() + np.abs(Fy).max()
    assert np.abs(Gx - Fx).max() < 1e-13 * s and np.abs(Gy - Fy).max() < 1e-13 * s
    # the slopes of the edge cells reach the ghost cells: leaving them out changes the sums
    Kn = K.copy()
    Kn[[1, 2, 4, 5]] = 0.0
    Hx, _ = C.three_sum(sigma, Kn, dx, dy)
    assert np.abs(Hx - Fx).max() > 1e-3 * s


@pytest.mark.parametrize("nd", [5, 2])
def test_dn_second_order(nd):
    """sigma_{D_n} (alpha = 0.25) centred at (0.1, -0.05) in [-0.5, 0.5]^2,
    N = 64, 128, 256.  D_5: the maximum error converges at second order;
    D_2, whose second derivative is singular at the rim: the mean error at
    second order, the maximum at about 1.5 (as the paper finds on the polar
    grid, Sec. 5.3)."""
    alpha, xc, yc, M = 0.25, 0.1, -0.05, 0.5
    emax, emean = [], []
    for n in (64, 128, 256):
        dx = 2 * M / n
        x = -M + (np.arange(n) + 0.5) * dx
        X, Y = x[:, None] - xc, x[None, :] - yc
        d = np.hypot(X, Y)
        sigma = A.dn_sigma(nd, d / alpha)
        f = A.dn_force(nd, (d / alpha).ravel()).reshape(d.shape)
        Fx_t, Fy_t = f * X / d, f * Y / d
        Kx, Ky = C.fold(C.cells(n, n, dx), dx)
        Fx, Fy = C.forces(sigma, Kx, Ky)
        emax.append(max(np.abs(Fx - Fx_t).max(), np.abs(Fy - Fy_t).max()) / np.abs(f).max())
        emean.append((np.abs(Fx - Fx_t).mean() + np.abs(Fy - Fy_t).mean()) / np.abs(f).mean())
    omax = math.log2(emax[-2] / emax[-1])
    omean = math.log2(emean[-2] / emean[-1])
    assert omean > 1.85, (emean, omean)
    if nd == 5:
        assert omax > 1.8 and emax[-1] < 3e-4, (emax, omax)
    else:
        assert 1.3 < omax < 1.8, (emax, omax)
