"""Error bounds for the parity tests: the global relative L2 error of both
force components together, and beside it local bounds, so that an error
confined to a few rows or cells (an edge row, a ragged tail, one tile) cannot
hide inside a small global norm.

The FFT convolution's rounding error is spread over the whole output in the
domain the transform works in: sigma e^{p u} in, e^{p u_i} F out (weight_p =
p).  So the local bounds are taken there, with the row weight w_i = r_i^p
(1 for p = 0), against the RMS of the weighted reference:

    every row i:   RMS_j |w_i dF_ij|  <= ROW * tol * RMS(w F)
    every cell:    |w_i dF_ij|        <= CELL * tol * RMS(w F)

For a uniform error of global relative size e <= tol the row RMS is about
e RMS(w F) and the largest of n Gaussian-like cell errors about
sqrt(2 ln n) e RMS(w F) (under 6 e for n below 10^8), so ROW = 10 and CELL =
50 fail only an error concentrated well beyond its share of the budget."""
import math

import numpy as np

ROW = 10.0
CELL = 50.0


def _d(a):
    return np.asarray(a, dtype=np.float64)


def rel_l2(Fr, Fp, Fr_ref, Fp_ref) -> float:
    num = np.sum((_d(Fr) - _d(Fr_ref)) ** 2) + np.sum((_d(Fp) - _d(Fp_ref)) ** 2)
    den = np.sum(_d(Fr_ref) ** 2) + np.sum(_d(Fp_ref) ** 2)
    return float(math.sqrt(num / den))


def assert_close(Fr, Fp, Fr_ref, Fp_ref, tol, w=None, what=""):
    """Global rel-L2 < tol, then the row and cell bounds above.  2-D fields
    (rows i, columns j) get both local bounds; flat arrays (sampled targets)
    get the cell bound.  w: the row weight r_i^p, one value per row of a 2-D
    field or per sampled target; None for p = 0."""
    Fr, Fp, Fr_ref, Fp_ref = _d(Fr), _d(Fp), _d(Fr_ref), _d(Fp_ref)
    e = rel_l2(Fr, Fp, Fr_ref, Fp_ref)
    assert e < tol, f"{what} global rel-L2 {e:.3e} >= {tol:.1e}"
    if w is None:
        w = np.ones(Fr_ref.shape[0])
    w = _d(w).reshape((-1,) + (1,) * (Fr_ref.ndim - 1))
    rms = math.sqrt(0.5 * (np.mean((w * Fr_ref) ** 2) + np.mean((w * Fp_ref) ** 2)))
    if rms == 0.0:
        assert np.all(Fr == 0) and np.all(Fp == 0), what
        return
    dr = np.abs(w * (Fr - Fr_ref))
    dp = np.abs(w * (Fp - Fp_ref))
    worst = max(dr.max(), dp.max()) / rms
    assert worst <= CELL * tol, f"{what} largest cell error {worst:.3e} x RMS > {CELL * tol:.1e}"
    if Fr_ref.ndim == 2:
        row = np.sqrt(0.5 * (np.mean(dr ** 2, axis=1) + np.mean(dp ** 2, axis=1))) / rms
        i = int(np.argmax(row))
        assert row[i] <= ROW * tol, f"{what} row {i} RMS error {row[i]:.3e} x RMS > {ROW * tol:.1e}"


def assert_close_1(g, ref, tol, w=None, what=""):
    """The same bounds for one field (an adjoint gradient)."""
    z = np.zeros_like(_d(ref))
    assert_close(g, z, ref, z, tol, w, what)
