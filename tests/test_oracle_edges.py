"""Pins for the oracle's one-sided radial edge slopes (no ghost rows; the
alternative to the zero-extended central slopes, where the paper is silent on
the grid's radial edges):

* the fast form (convolution plus the slope-term difference on the four
  affected rows) equals the literal three-term sums of Eq. 26-29 / A8-A10
  with those slopes;
* the brute force of tests/test_oracle_sums (piecewise-linear density
  against the point kernel) with the same slopes;
* on a Kuzmin disk, which does not vanish at the inner edge, the full-grid
  error converges at second order with one-sided slopes and does not with
  ghost rows.
"""
import math

import numpy as np
import pytest

import workloads
from oracle import analytic as A


@pytest.mark.parametrize("nu,nphi", [(4, 8), (8, 16), (16, 8)])
def test_fast_form_equals_three_sums(oracle_mod, nu, nphi):
    u_min, du = workloads.grid_params(nu, 0.1, 10.0)
    grid = oracle_mod.Grid(nu, nphi, u_min, du)
    cells = oracle_mod.kernel_cells(nu, nphi, du)
    sigma = workloads.random_field(nu, nphi, nu + nphi)
    a = oracle_mod.three_sum(sigma, cells, grid, 1.3, edges="onesided")
    b = oracle_mod.onesided_forces(sigma, cells, grid, 1.3)
    scale = np.abs(a[0]).max() + np.abs(a[1]).max()
    assert np.abs(a[0] - b[0]).max() < 1e-13 * scale and np.abs(a[1] - b[1]).max() < 1e-13 * scale
    # and the change is confined to what the edge rows' slopes reach
    g = oracle_mod.three_sum(sigma, cells, grid, 1.3, edges="ghost")
    assert np.abs(a[0] - g[0]).max() > 1e-6 * scale


def test_interior_slopes_unchanged(oracle_mod):
    nu, nphi = 8, 8
    grid = oracle_mod.Grid(nu, nphi, math.log(0.1), math.log(100.0) / nu)
    sigma = workloads.random_field(nu, nphi, 2)
    dg, dpg, rows = oracle_mod.slopes(sigma, grid, "ghost")
    do, dpo, rows_o = oracle_mod.slopes(sigma, grid, "onesided")
    assert list(rows_o) == list(range(nu))
    assert np.allclose(do[1:nu - 1], dg[2:nu], rtol=1e-14, atol=0) and np.array_equal(dpo, dpg)
    assert np.allclose(do[0], (sigma[1] - sigma[0]) / (grid.r[1] - grid.r[0]), rtol=1e-15)


def test_kuzmin_full_grid_second_order(oracle_mod):
    errs = {"ghost": [], "onesided": []}
    for n in (32, 64, 128):
        u_min, du = workloads.grid_params(n, 0.05, 20.0)
        grid = oracle_mod.Grid(n, n, u_min, du)
        cells = oracle_mod.kernel_cells(n, n, du)
        r, phi = workloads.centres(n, n, u_min, du)
        sig = workloads.kuzmin(r, phi)
        truth = A.kuzmin_truncated_Fr(r, 0.05, 20.0)
        Kr, Kp = oracle_mod.fold(cells, grid.beta, grid.dphi)
        Fg, _ = oracle_mod.fft_conv(sig, Kr, Kp)
        Fo, Fpo = oracle_mod.onesided_forces(sig, cells, grid)
        errs["ghost"].append(np.abs(Fg[:, 0] - truth).max())
        errs["onesided"].append(np.abs(Fo[:, 0] - truth).max())
        assert np.abs(Fpo).max() < 1e-14 * np.abs(Fo).max()  # still axisymmetric
    order = {k: math.log2(v[-2] / v[-1]) for k, v in errs.items()}
    assert order["onesided"] > 1.7 and errs["onesided"][-1] < 1e-4, errs
    assert order["ghost"] < 0.5 and errs["ghost"][-1] > 0.1, errs  # the ghost rows' dipole at r_in


@pytest.mark.parametrize("nu,nphi", [(8, 16), (16, 32)])
def test_sampled_form_equals_the_whole_field(oracle_mod, nu, nphi):
    """onesided_forces_at (the sums at chosen cells, for grids too large for
    the whole field) gives the whole-field values at every cell."""
    u_min, du = workloads.grid_params(nu, 0.1, 10.0)
    grid = oracle_mod.Grid(nu, nphi, u_min, du)
    cells = oracle_mod.kernel_cells(nu, nphi, du)
    sigma = workloads.random_field(nu, nphi, 3)
    Fr, Fp = oracle_mod.onesided_forces(sigma, cells, grid, 1.3)
    t = np.random.default_rng(1).permutation(nu * nphi)
    ar, ap = oracle_mod.onesided_forces_at(sigma, cells, grid, t, 1.3)
    scale = np.abs(Fr).max() + np.abs(Fp).max()
    assert np.abs(ar - Fr.ravel()[t]).max() < 1e-14 * scale and np.abs(ap - Fp.ravel()[t]).max() < 1e-14 * scale


@pytest.mark.parametrize("nu,nphi", [(6, 8), (8, 16)])
def test_transpose_is_the_transposed_dense_map(oracle_mod, nu, nphi):
    """onesided_forces_T against the dense matrix of onesided_forces (built
    column by column from unit densities), transposed."""
    u_min, du = workloads.grid_params(nu, 0.1, 10.0)
    grid = oracle_mod.Grid(nu, nphi, u_min, du)
    cells = oracle_mod.kernel_cells(nu, nphi, du)
    n = nu * nphi
    M = np.zeros((2 * n, n))
    for c in range(n):
        e = np.zeros(n)
        e[c] = 1.0
        fr, fp = oracle_mod.onesided_forces(e.reshape(nu, nphi), cells, grid, 0.7)
        M[:n, c], M[n:, c] = fr.ravel(), fp.ravel()
    gr, gp = workloads.random_field(nu, nphi, 11), workloads.random_field(nu, nphi, 12)
    ref = (M.T @ np.concatenate([gr.ravel(), gp.ravel()])).reshape(nu, nphi)
    got = oracle_mod.onesided_forces_T(gr, gp, cells, grid, 0.7)
    assert np.abs(got - ref).max() < 1e-13 * np.abs(ref).max()


def test_transpose_dot_identity(oracle_mod):
    nu, nphi = 32, 64
    u_min, du = workloads.grid_params(nu, 0.01, 100.0)
    grid = oracle_mod.Grid(nu, nphi, u_min, du)
    cells = oracle_mod.kernel_cells(nu, nphi, du)
    sigma = workloads.random_field(nu, nphi, 21)
    gr, gp = workloads.random_field(nu, nphi, 22), workloads.random_field(nu, nphi, 23)
    Fr, Fp = oracle_mod.onesided_forces(sigma, cells, grid)
    gs = oracle_mod.onesided_forces_T(gr, gp, cells, grid)
    lhs = float((gr * Fr).sum() + (gp * Fp).sum())
    rhs = float((gs * sigma).sum())
    assert abs(lhs - rhs) < 1e-13 * float(np.abs(gr * Fr).sum() + np.abs(gp * Fp).sum())
