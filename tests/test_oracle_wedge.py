"""Pins for the oracle's origin wedge (the cells R^_j = [0, r_in] x one
azimuthal cell below the grid's first row, Sec. 3.2.1, and the third terms
of Eq. 27-29 with the kernels K-bar), against things other than the
oracle's own integrator:

* the wedge kernels, the forces' and the potential's, by 2-D quadrature of
  the raw integrands in physical coordinates (r', phi');
* the wedge's single sums against a brute-force quadrature of the
  piecewise-linear wedge density (the value at the wedge centre r_in / 2,
  the one-sided radial slope toward the first row, the central azimuthal
  slope) times the point kernel;
* a Kuzmin disk held by the grid and the wedge together, with r_in halved
  as N doubles (as the paper shrinks M^s_in): the full-grid force error
  converges at second order, and without the wedge it stays O(1).
"""
import math

import numpy as np
import pytest
from scipy.integrate import dblquad

import workloads
from oracle import analytic as A

NU, NPHI = 8, 16
DU = math.log(400.0) / 64


def _raw_wedge(i, q, du, nphi):
    """The six K-bar integrals for a wedge of outer radius 1 seen from the
    centre of row i (r_i = beta^i (1 + beta) / 2), in physical coordinates."""
    beta = math.exp(du)
    ri = 0.5 * beta ** i * (1.0 + beta)
    dphi = 2 * math.pi / nphi
    rw = 0.5
    lo, hi = (-q - 0.5) * dphi, (-q + 0.5) * dphi  # psi = phi' - phi_j over the source wedge

    def d3(r, p):
        return (r * r + ri * ri - 2 * r * ri * math.cos(p)) ** 1.5

    f0 = lambda r, p: -r * (ri - r * math.cos(p)) / d3(r, p)
    g0 = lambda r, p: r * r * math.sin(p) / d3(r, p)
    fs = [f0, lambda r, p: f0(r, p) * (r - rw) / ri, lambda r, p: f0(r, p) * (p + q * dphi),
          g0, lambda r, p: g0(r, p) * (r - rw) / ri, lambda r, p: g0(r, p) * (p + q * dphi)]
    return np.array([dblquad(f, lo, hi, 0.0, 1.0, epsabs=0, epsrel=1e-12)[0] for f in fs])


@pytest.mark.parametrize("i,q", [(0, 0), (0, 1), (1, 3), (5, 0), (3, -2), (7, 8)])
def test_wedge_cells_against_quadrature(oracle_mod, i, q):
    W = oracle_mod.wedge_cells(NU, NPHI, DU)
    got = W[:, i, q % NPHI]
    ref = _raw_wedge(i, q, DU, NPHI)
    scale = abs(ref[0]) + abs(ref[3])
    assert np.all(np.abs(got - ref) <= 1e-10 * scale), (got, ref)


def test_wedge_sums_against_brute_force(oracle_mod):
    nu, nphi = 3, 6
    u_min, du = 0.0, math.log(400.0) / 64 * 8
    grid = oracle_mod.Grid(nu, nphi, u_min, du)
    rng = np.random.default_rng(5)
    sigma, sigma_w = rng.random((nu, nphi)), rng.random(nphi)
    W = oracle_mod.wedge_cells(nu, nphi, du)
    Fr, Fp = oracle_mod.wedge_sums(sigma, sigma_w, W, grid)
    r_in, dphi = grid.faces[0], grid.dphi
    r_w = 0.5 * r_in
    dr = (sigma[0] - sigma_w) / (grid.r[0] - r_w)
    dp = (np.roll(sigma_w, -1) - np.roll(sigma_w, 1)) / (2 * dphi)
    for i in range(nu):
        for j in range(nphi):
            ri, pj = grid.r[i], grid.phi[j]
            br = bp = 0.0
            for jp in range(nphi):
                pc = grid.phi[jp]
                dens = lambda r, p: sigma_w[jp] + dr[jp] * (r - r_w) + dp[jp] * (p - pc)
                d3 = lambda r, p: (r * r + ri * ri - 2 * r * ri * math.cos(p - pj)) ** 1.5
                br += dblquad(lambda r, p: -dens(r, p) * r * (ri - r * math.cos(p - pj)) / d3(r, p),
                              pc - dphi / 2, pc + dphi / 2, 0.0, r_in, epsabs=0, epsrel=1e-11)[0]
                bp += dblquad(lambda r, p: dens(r, p) * r * r * math.sin(p - pj) / d3(r, p),
                              pc - dphi / 2, pc + dphi / 2, 0.0, r_in, epsabs=0, epsrel=1e-11)[0]
            s = np.abs(Fr).max()
            assert abs(Fr[i, j] - br) < 1e-9 * s and abs(Fp[i, j] - bp) < 1e-9 * s, (i, j)


def test_kuzmin_with_the_wedge_second_order(oracle_mod):
    errs, errs0 = [], []
    for n, r_in in ((32, 0.2), (64, 0.1), (128, 0.05)):
        u_min, du = workloads.grid_params(n, r_in, 20.0)
        grid = oracle_mod.Grid(n, n, u_min, du)
        sigma = workloads.kuzmin(grid.r, grid.phi)
        sigma_w = np.full(n, float(A.kuzmin_sigma(0.5 * grid.faces[0])))
        cells = oracle_mod.kernel_cells(n, n, du)
        Fr, Fp = oracle_mod.wedge_forces(sigma, sigma_w, cells, oracle_mod.wedge_cells(n, n, du), grid)
        Fr0, _ = oracle_mod.onesided_forces(sigma, cells, grid)
        truth = A.kuzmin_truncated_Fr(grid.r, 0.0, 20.0)  # only the tail beyond r_out is missing
        errs.append(np.abs(Fr[:, 0] - truth).max() / np.abs(truth).max())
        errs0.append(np.abs(Fr0[:, 0] - truth).max() / np.abs(truth).max())
        assert np.abs(Fp).max() < 1e-12 * np.abs(Fr).max()
    order = math.log2(errs[-2] / errs[-1])
    assert order > 1.7 and errs[-1] < 4e-4, (errs, order)
    assert min(errs0) > 0.5, errs0


@pytest.mark.parametrize("i,q", [(0, 0), (0, 2), (3, -1), (6, 8)])
def test_potential_wedge_cells_against_quadrature(oracle_mod, i, q):
    """The potential's wedge kernels: -int r' / (r_i d) and its two slope
    moments over the wedge of outer radius 1, in physical coordinates."""
    W = oracle_mod.wedge_cells(NU, NPHI, DU, pot=True)
    beta = math.exp(DU)
    ri = 0.5 * beta ** i * (1.0 + beta)
    dphi = 2 * math.pi / NPHI
    lo, hi = (-q - 0.5) * dphi, (-q + 0.5) * dphi
    f0 = lambda r, p: -r / (ri * math.sqrt(r * r + ri * ri - 2 * r * ri * math.cos(p)))
    fs = [f0, lambda r, p: f0(r, p) * (r - 0.5) / ri, lambda r, p: f0(r, p) * (p + q * dphi)]
    ref = np.array([dblquad(f, lo, hi, 0.0, 1.0, epsabs=0, epsrel=1e-12)[0] for f in fs])
    got = W[:3, i, q % NPHI]
    assert np.all(np.abs(got - ref) <= 1e-10 * abs(ref[0])), (got, ref)
    assert not np.any(W[3:])


def test_sampled_form_equals_the_whole_field(oracle_mod):
    """wedge_forces_at (at chosen cells, for grids too large for the whole
    field) gives the whole-field values."""
    nu, nphi = 16, 32
    u_min, du = workloads.grid_params(nu, 0.1, 10.0)
    grid = oracle_mod.Grid(nu, nphi, u_min, du)
    cells = oracle_mod.kernel_cells(nu, nphi, du)
    wcells = oracle_mod.wedge_cells(nu, nphi, du)
    sigma = np.abs(workloads.random_field(nu, nphi, 4)) + 0.1
    sigma_w = 0.5 + np.random.default_rng(4).random(nphi)
    Fr, Fp = oracle_mod.wedge_forces(sigma, sigma_w, cells, wcells, grid)
    t = np.random.default_rng(2).permutation(nu * nphi)[: nu * nphi // 2]
    ar, ap = oracle_mod.wedge_forces_at(sigma, sigma_w, cells, wcells, grid, t)
    scale = np.abs(Fr).max() + np.abs(Fp).max()
    assert np.abs(ar - Fr.ravel()[t]).max() < 1e-14 * scale and np.abs(ap - Fp.ravel()[t]).max() < 1e-14 * scale
