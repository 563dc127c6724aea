"""Pins for the oracle's sums: the three-term form of Eq. 26-29 / A8-A10, the
folded single-kernel convolution, its transpose and its FFT evaluation.

Independent references: a brute-force quadrature (scipy, physical
coordinates) of the piecewise-linear density of Eq. 25 against the exact
point kernel of Eq. 23-24; impulse responses; exact invariants (rotation
equivariance, F_phi = 0 for axisymmetric sigma); the dot-product identity of
the adjoint.
"""
import math

import numpy as np
import pytest

import workloads


def _tables(oracle_mod, nu, nphi, du):
    cells = oracle_mod.kernel_cells(nu, nphi, du)
    Kr, Kp = oracle_mod.fold(cells, math.exp(du), 2 * math.pi / nphi)
    return cells, Kr, Kp


@pytest.fixture(scope="module")
def small(oracle_mod):
    nu, nphi = 8, 12
    u_min, du = workloads.grid_params(nu, 0.5, 4.0)
    grid = oracle_mod.Grid(nu, nphi, u_min, du)
    cells, Kr, Kp = _tables(oracle_mod, nu, nphi, du)
    return grid, cells, Kr, Kp


def test_fold_equals_three_sum(oracle_mod, small):
    """The folded kernels reproduce the literal three-term sums, including the
    slope terms of the ghost rows the central stencil reaches."""
    grid, cells, Kr, Kp = small
    rng = np.random.default_rng(3)
    sigma = rng.uniform(0.5, 1.5, (grid.nu, grid.nphi))  # nonzero at both radial edges
    Fr3, Fp3 = oracle_mod.three_sum(sigma, cells, grid, G=1.3)
    Fr, Fp = oracle_mod.direct_sum(sigma, Kr, Kp, G=1.3)
    scale = np.abs(Fr3).max() + np.abs(Fp3).max()
    assert np.abs(Fr - Fr3).max() < 1e-13 * scale
    assert np.abs(Fp - Fp3).max() < 1e-13 * scale


def test_impulse_response(oracle_mod, small):
    """sigma = e_{m,l} gives F[i,j] = G K[i-m, (j-l) mod Nphi]."""
    grid, cells, Kr, Kp = small
    nu, nphi = grid.nu, grid.nphi
    for m, l in ((0, 0), (3, 5), (7, 11)):
        sigma = np.zeros((nu, nphi))
        sigma[m, l] = 1.0
        Fr, Fp = oracle_mod.direct_sum(sigma, Kr, Kp, G=2.0)
        for i in range(nu):
            for j in range(nphi):
                assert Fr[i, j] == 2.0 * Kr[i - m + nu - 1, (j - l) % nphi]
                assert Fp[i, j] == 2.0 * Kp[i - m + nu - 1, (j - l) % nphi]


def test_direct_equals_fft(oracle_mod):
    nu, nphi = 24, 32
    u_min, du = workloads.grid_params(nu, 0.1, 10.0)
    _, Kr, Kp = _tables(oracle_mod, nu, nphi, du)
    sigma = workloads.random_field(nu, nphi, 5)
    Fr, Fp = oracle_mod.direct_sum(sigma, Kr, Kp)
    Gr, Gp = oracle_mod.fft_conv(sigma, Kr, Kp)
    assert oracle_mod.rel_l2(Gr, Gp, Fr, Fp) < 1e-13
    # sampled targets give the same numbers as the full sum
    t = np.array([0, 5, nphi * 7 + 3, nu * nphi - 1])
    tr, tp = oracle_mod.direct_sum(sigma, Kr, Kp, targets=t)
    assert np.array_equal(tr, Fr.ravel()[t]) and np.array_equal(tp, Fp.ravel()[t])


def test_transpose_identity(oracle_mod):
    """<g, A sigma> = <A^T g, sigma> for both the direct and the FFT forms."""
    nu, nphi = 16, 20
    u_min, du = workloads.grid_params(nu, 0.1, 10.0)
    _, Kr, Kp = _tables(oracle_mod, nu, nphi, du)
    sigma = workloads.random_field(nu, nphi, 1)
    gr = workloads.random_field(nu, nphi, 2)
    gp = workloads.random_field(nu, nphi, 3)
    Fr, Fp = oracle_mod.direct_sum(sigma, Kr, Kp, G=0.7)
    gs = oracle_mod.direct_sum_T(gr, gp, Kr, Kp, G=0.7)
    lhs = np.sum(gr * Fr) + np.sum(gp * Fp)
    rhs = np.sum(gs * sigma)
    assert abs(lhs - rhs) < 1e-13 * (abs(lhs) + np.abs(gs).sum())
    gs2 = oracle_mod.fft_conv_T(gr, gp, Kr, Kp, G=0.7)
    assert np.abs(gs2 - gs).max() < 1e-13 * np.abs(gs).max()
    # sampled sources
    s = np.array([0, 33, nu * nphi - 1])
    assert np.allclose(oracle_mod.direct_sum_T(gr, gp, Kr, Kp, G=0.7, sources=s), gs.ravel()[s], rtol=0, atol=0)


def test_axisymmetric_has_no_azimuthal_force(oracle_mod):
    nu, nphi = 16, 16
    u_min, du = workloads.grid_params(nu, 0.05, 20.0)
    _, Kr, Kp = _tables(oracle_mod, nu, nphi, du)
    r, phi = workloads.centres(nu, nphi, u_min, du)
    sigma = workloads.kuzmin(r, phi)
    Fr, Fp = oracle_mod.direct_sum(sigma, Kr, Kp)
    assert np.abs(Fp).max() < 1e-14 * np.abs(Fr).max()
    assert np.all(Fr[nu // 2:] < 0)  # attractive away from the inner edge of the annulus
    # every column the same
    assert np.abs(Fr - Fr[:, :1]).max() < 1e-14 * np.abs(Fr).max()


def test_rotation_equivariance(oracle_mod, small):
    grid, cells, Kr, Kp = small
    sigma = workloads.random_field(grid.nu, grid.nphi, 9)
    Fr, Fp = oracle_mod.direct_sum(sigma, Kr, Kp)
    for s in (1, 5):
        Rr, Rp = oracle_mod.direct_sum(np.roll(sigma, s, axis=1), Kr, Kp)
        assert np.abs(Rr - np.roll(Fr, s, axis=1)).max() < 1e-14 * np.abs(Fr).max()
        assert np.abs(Rp - np.roll(Fp, s, axis=1)).max() < 1e-14 * np.abs(Fr).max()


# ---------------------------------------------------------------------------
# Brute force: piecewise-linear sigma (Eq. 25, central slopes, zero outside
# the grid) integrated against the point kernel of Eq. 23-24 by scipy.
# ---------------------------------------------------------------------------
def _brute_force(sigma, u_min, du, nphi, ti, tj, edges="ghost"):
    """edges = "ghost": central radial slopes wherever the stencil touches the
    grid (ghost rows -1 and Nu included); "onesided": the grid's rows only,
    one-sided radial slopes at the first and last rows."""
    from scipy.integrate import quad

    nu = sigma.shape[0]
    beta = math.exp(du)
    dphi = 2 * math.pi / nphi
    face = lambda i: math.exp(u_min + du * i)
    cen = lambda i: 0.5 * (face(i) + face(i + 1))
    sig = lambda i, j: sigma[i, j % nphi] if 0 <= i < nu else 0.0
    ri, pj = cen(ti), (tj + 0.5) * dphi
    Fr = Fp = 0.0
    rows = range(-1, nu + 1) if edges == "ghost" else range(nu)
    for ip in rows:
        lo, hi, rc = face(ip), face(ip + 1), cen(ip)
        for jp in range(nphi):
            s0 = sig(ip, jp)
            if edges == "ghost":
                sr = (sig(ip + 1, jp) - sig(ip - 1, jp)) / (cen(ip + 1) - cen(ip - 1))
            else:
                a, b = max(ip - 1, 0), min(ip + 1, nu - 1)
                sr = (sig(b, jp) - sig(a, jp)) / (cen(b) - cen(a))
            sp = (sig(ip, jp + 1) - sig(ip, jp - 1)) / (2 * dphi) if 0 <= ip < nu else 0.0
            if s0 == 0.0 and sr == 0.0 and sp == 0.0:
                continue
            pc = (jp + 0.5) * dphi
            # xi = phibar - phi_j, taken near 0 for the nearest image
            off = ((pc - pj + math.pi) % (2 * math.pi)) - math.pi

            def integrand(rb, xi, comp):
                srec = s0 + sr * (rb - rc) + sp * (xi - off)
                c, s = math.cos(xi), math.sin(xi)
                D3 = ((rb - ri * c) ** 2 + (ri * s) ** 2) ** 1.5
                if comp == 0:
                    return -srec * rb * (ri - rb * c) / D3
                return srec * rb * rb * s / D3

            def g(xi, comp):
                pts = [ri * math.cos(xi)] if lo < ri * math.cos(xi) < hi else None
                return quad(integrand, lo, hi, args=(xi, comp), points=pts, limit=200, epsabs=1e-14,
                            epsrel=1e-12)[0]

            self_cell = ip == ti and jp == tj
            for comp in (0, 1):
                if self_cell:  # principal value in xi about the target: pair xi, -xi
                    v = quad(lambda x: g(x, comp) + g(-x, comp), 0.0, dphi / 2, limit=200, epsabs=1e-13,
                             epsrel=1e-11)[0]
                else:
                    v = quad(lambda x: g(x, comp), off - dphi / 2, off + dphi / 2, limit=200, epsabs=1e-14,
                             epsrel=1e-12)[0]
                if comp == 0:
                    Fr += v
                else:
                    Fp += v
    return Fr, Fp


@pytest.mark.slow
def test_brute_force_tiny_grid(oracle_mod):
    nu, nphi = 4, 6
    u_min, du = workloads.grid_params(nu, 0.5, 2.0)
    _, Kr, Kp = _tables(oracle_mod, nu, nphi, du)
    r, phi = workloads.centres(nu, nphi, u_min, du)
    sigma = 1.0 + 0.3 * np.cos(phi)[None, :] + 0.2 * r[:, None]  # nonzero at the radial edges
    Fr, Fp = oracle_mod.direct_sum(sigma, Kr, Kp)
    for ti, tj in ((0, 0), (2, 3), (3, 5)):
        br, bp = _brute_force(sigma, u_min, du, nphi, ti, tj)
        scale = abs(br) + abs(bp)
        assert abs(Fr[ti, tj] - br) < 1e-8 * scale, (ti, tj, Fr[ti, tj], br)
        assert abs(Fp[ti, tj] - bp) < 1e-8 * scale, (ti, tj, Fp[ti, tj], bp)


@pytest.mark.slow
def test_brute_force_tiny_grid_onesided_edges(oracle_mod):
    """The one-sided edge slopes (no ghost rows) of onesided_forces against the
    same brute force with those slopes, at edge and interior targets."""
    nu, nphi = 4, 6
    u_min, du = workloads.grid_params(nu, 0.5, 2.0)
    grid = oracle_mod.Grid(nu, nphi, u_min, du)
    cells, _, _ = _tables(oracle_mod, nu, nphi, du)
    r, phi = workloads.centres(nu, nphi, u_min, du)
    sigma = 1.0 + 0.3 * np.cos(phi)[None, :] + 0.2 * r[:, None]
    Fr, Fp = oracle_mod.onesided_forces(sigma, cells, grid)
    for ti, tj in ((0, 0), (1, 2), (3, 5)):
        br, bp = _brute_force(sigma, u_min, du, nphi, ti, tj, edges="onesided")
        scale = abs(br) + abs(bp)
        assert abs(Fr[ti, tj] - br) < 1e-8 * scale, (ti, tj, Fr[ti, tj], br)
        assert abs(Fp[ti, tj] - bp) < 1e-8 * scale, (ti, tj, Fp[ti, tj], bp)
