"""FP64 CPU oracle for the log-polar thin-disk self-gravity path.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / reference leg of ``bench.py`` may import this package.  The
product library never imports, loads or calls it, and it shares no code with
the CUDA path (the seeded input generators live in ``workloads/``).

What it computes follows Wang, Yen & Taam, "Self-gravitational force
calculation of second order accuracy for infinitesimally thin gaseous disks in
polar coordinates":

* ``grid``               -- Sec. 3.2.1: log-spaced faces, arithmetic centres.
* ``kernel_cells``       -- Eq. 30-32, A11-A13: the six exact cell integrals
                            (C, adaptive Gauss-Legendre; see sg_oracle.c).
* ``slopes``             -- Eq. 25 with central differences (Sec. 5.3).
* ``three_sum``          -- Eq. 26-29 and A8-A10 on the single grid, the
                            literal three-term form.
* ``kernel_cells_tpz``   -- Eq. 41-43: the same kernels with the trapezoidal
                            rule in phi (the paper's SIM with N_tpz).
* ``potential_cells``    -- the same construction for the potential, which
                            the paper says carries over (Sec. 6); and
                            ``potential``, the potential at the centres.
* ``particle_cells``     -- Eq. 35-37 and Sec. 5.3: the particle method, the
                            modified particle method and the softened
                            particle kernel of the comparison (BM08), as
                            cell tables of the same shape.
* ``fold``               -- the same sums collapsed to one kernel per force
                            component (the exact algebra in ``fold``'s doc).
* ``direct_sum``         -- the O(N^2) convolution with the folded kernels.
* ``direct_sum_T``       -- its transpose (adjoint), for the sigma-gradient.
* ``fft_conv``           -- the same convolution with numpy's FFT as a
                            library step (zero-padded in u, periodic in phi).
* ``onesided_forces``    -- the sums with one-sided radial slopes at the
                            first and last rows (no ghost rows).
* ``wedge_cells``,        -- the origin wedge below the grid (Sec. 3.2.1,
  ``wedge_sums``,            the third terms of Eq. 27-29): its kernels seen
  ``wedge_forces``           from every row, its single sums, and the grid's
                            one-sided sums plus them.
* ``cartesian``          -- Sec. 3.1.1 and App. A: the Cartesian scheme's
                            closed-form kernels, literal sums, fold and
                            zero-padded convolution (its own module).
* ``analytic``           -- closed-form disks used as truth (Sec. 5.1).
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sg_oracle.c")
_LIB = os.path.join(_HERE, "libsg_oracle.so")
_lib = None

NC = 6
COMPONENTS = ("r0", "rr", "rphi", "phi0", "phir", "phiphi")


def build(force: bool = False) -> str:
    """Compile the C part of the oracle (plain gcc, OpenMP) in place."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-o", _LIB + ".tmp", _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(_LIB + ".tmp", _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        lp = ctypes.POINTER(ctypes.c_long)
        lib.sgo_cell.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
        lib.sgo_cell.restype = ctypes.c_int
        lib.sgo_cells_table.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp, ctypes.c_int]
        lib.sgo_cells_table.restype = ctypes.c_int
        lib.sgo_cells_table_tpz.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                            ctypes.c_double, dp, ctypes.c_int]
        lib.sgo_cell_pot.argtypes = [ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_double, dp]
        lib.sgo_cell_pot.restype = ctypes.c_int
        lib.sgo_cells_table_pot.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, dp,
                                            ctypes.c_int]
        lib.sgo_cells_table_pot.restype = ctypes.c_int
        lib.sgo_cells_table_tpz.restype = ctypes.c_int
        lib.sgo_wedge_table.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                        dp, ctypes.c_int]
        lib.sgo_wedge_table.restype = ctypes.c_int
        lib.sgo_direct_sum.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp, dp, lp, ctypes.c_long,
                                       dp, dp, ctypes.c_int]
        lib.sgo_direct_sum.restype = None
        lib.sgo_direct_sum_T.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_double, dp, dp, dp, dp, lp,
                                         ctypes.c_long, dp, ctypes.c_int]
        lib.sgo_direct_sum_T.restype = None
        lib.sgo_max_threads.argtypes = []
        lib.sgo_max_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def max_threads() -> int:
    return int(_load().sgo_max_threads())


# --------------------------------------------------------------------------
# Sec. 3.2.1 grid
# --------------------------------------------------------------------------
class Grid:
    """Log-polar grid of Sec. 3.2.1 (0-based indices).

    faces  r_{i-1/2} = e^{u_min} beta^i, i = 0..Nu      (beta = e^{du})
    centre r_i = (r_{i-1/2} + r_{i+1/2}) / 2, i = 0..Nu-1  (arithmetic mean)
    phi_j = (j + 1/2) dphi, dphi = 2 pi / Nphi
    """

    def __init__(self, nu: int, nphi: int, u_min: float, du: float):
        self.nu, self.nphi, self.u_min, self.du = int(nu), int(nphi), float(u_min), float(du)
        self.beta = math.exp(du)
        self.dphi = 2.0 * math.pi / nphi
        i = np.arange(nu + 1, dtype=np.float64)
        self.faces = np.exp(u_min + du * i)
        self.r = 0.5 * (self.faces[:-1] + self.faces[1:])
        self.dr = self.faces[1:] - self.faces[:-1]
        self.phi = (np.arange(nphi, dtype=np.float64) + 0.5) * self.dphi
        self.area = self.r * self.dr * self.dphi  # exact cell area (arithmetic centre)

    def centre(self, i):
        """Centre radius of row i for any integer i (ghost rows included)."""
        return 0.5 * math.exp(self.u_min + self.du * i) * (1.0 + self.beta)


# --------------------------------------------------------------------------
# Eq. 30-32, A11-A13: cell integrals
# --------------------------------------------------------------------------
def kernel_cell(du: float, nphi: int, k: int, q: int, rtol: float = 2e-14) -> np.ndarray:
    """The six kernels K^{r,0}, K^{r,r}, K^{r,phi}, K^{phi,0}, K^{phi,r},
    K^{phi,phi} for the offset (k, q) = (i - i', j - j')."""
    out = np.zeros(NC)
    bad = _load().sgo_cell(float(du), int(nphi), int(k), int(q), float(rtol), _dp(out))
    if bad:
        raise RuntimeError(f"oracle quadrature did not converge for k={k} q={q}")
    return out


def kernel_cells(nu: int, nphi: int, du: float, rtol: float = 2e-14, nthreads: int = 0) -> np.ndarray:
    """Kernel table [6, 2Nu+1, Nphi] for k in [-Nu, Nu] (row k + Nu), q in [0, Nphi)."""
    out = np.zeros((NC, 2 * nu + 1, nphi))
    bad = _load().sgo_cells_table(int(nu), int(nphi), float(du), float(rtol), _dp(out), int(nthreads))
    if bad:
        raise RuntimeError(f"oracle quadrature did not converge for {bad} integrals")
    return out


PARTICLE_KINDS = ("particle", "particle+", "softened")


def particle_cells(nu: int, nphi: int, du: float, kind: str, soften: float = 0.0, rtol: float = 2e-14) -> np.ndarray:
    """Cell table [6, 2Nu+1, Nphi] of the particle methods (Sec. 3.2.2 for
    the Cartesian form, Eq. 35-37 in polar coordinates).

    Each source cell is a point of mass M = sigma A' at its centre.  With the
    target radius r_i as the unit, the source centre is r' = beta^{-k} (the
    ratio of two arithmetic centres), its faces r' 2/(1+beta) and
    r' 2 beta/(1+beta), A' = r' (r'_+ - r'_-) dphi its area, and the angle to
    it Delta = phi_{j'} - phi_j = -q dphi.  Eq. 35 and its azimuthal
    counterpart (the point form of Eq. A11) per unit sigma:
        K^{r,0}   <- -A' (1 - r' cos Delta) / d^3,
        K^{phi,0} <-  A' r' sin Delta / d^3,
    with d^2 = 1 + r'^2 - 2 r' cos Delta (law of cosines, written as
    (1 - r')^2 + 4 r' sin^2(Delta/2), and 1 - r' cos Delta as
    (1 - r') + 2 r' sin^2(Delta/2), so that neighbouring cells keep their
    digits).  The slope kernels are zero.

    kind "particle":  nothing from the target's own cell (Eq. 35, the (0, 0)
                      entry is 0).
    kind "particle+": the modified method of Eq. 36-37: the own cell's exact
                      K^{.,0}_{0,0}, K^{.,r}_{0,0}, K^{.,phi}_{0,0} (from
                      ``kernel_cell``) at (0, 0); ``fold`` turns the slope
                      ones into the sigma differences of delta^r, delta^phi.
    kind "softened":  eps^2 = (soften r_i)^2 added to d^2, own cell included
                      (the comparison method of Sec. 5.3).
    """
    if kind not in PARTICLE_KINDS:
        raise ValueError(kind)
    beta = math.exp(du)
    dphi = 2.0 * math.pi / nphi
    out = np.zeros((NC, 2 * nu + 1, nphi))
    delta = -np.arange(nphi, dtype=np.float64) * dphi
    s2 = np.sin(0.5 * delta) ** 2
    for kk in range(2 * nu + 1):
        k = kk - nu
        rp = beta ** (-k)
        area = rp * (rp * 2.0 * beta / (1.0 + beta) - rp * 2.0 / (1.0 + beta)) * dphi
        d2 = (1.0 - rp) ** 2 + 4.0 * rp * s2
        if kind == "softened":
            d2 = d2 + soften * soften
        with np.errstate(divide="ignore", invalid="ignore"):
            d3 = d2 * np.sqrt(d2)
            out[0, kk] = -area * ((1.0 - rp) + 2.0 * rp * s2) / d3
            out[3, kk] = area * rp * np.sin(delta) / d3
    if kind != "softened":
        out[0, nu, 0] = out[3, nu, 0] = 0.0  # the own cell holds no point mass
    if kind == "particle+":
        out[:, nu, 0] = kernel_cell(du, nphi, 0, 0, rtol)
    return out


def particle_kernels(nu: int, nphi: int, du: float, kind: str, soften: float = 0.0):
    """Folded kernels (Kr, Kphi) of a particle method."""
    return fold(particle_cells(nu, nphi, du, kind, soften), math.exp(du), 2.0 * math.pi / nphi)


def potential_cell(du: float, nphi: int, k: int, q: int, rtol: float = 2e-14) -> np.ndarray:
    """The potential's cells for the offset (k, q) (the paper's method
    carried over to the potential, Sec. 6): [-int eta / F, -int eta (eta -
    beta^-k) / F, -int eta (xi + q dphi) / F, 0, 0, 0] over the source cell
    in d eta d xi."""
    out = np.zeros(NC)
    bad = _load().sgo_cell_pot(float(du), int(nphi), int(k), int(q), float(rtol), _dp(out))
    if bad:
        raise RuntimeError(f"oracle quadrature did not converge for k={k} q={q}")
    return out


def potential_cells(nu: int, nphi: int, du: float, rtol: float = 2e-14, nthreads: int = 0) -> np.ndarray:
    """Table [6, 2Nu+1, Nphi] of ``potential_cell`` (slots 3-5 zero)."""
    out = np.zeros((NC, 2 * nu + 1, nphi))
    bad = _load().sgo_cells_table_pot(int(nu), int(nphi), float(du), float(rtol), _dp(out), int(nthreads))
    if bad:
        raise RuntimeError(f"oracle quadrature did not converge for {bad} integrals")
    return out


def potential(sigma: np.ndarray, cells: np.ndarray, grid: Grid, G: float = 1.0):
    """Phi at the cell centres: r_i times the convolution of sigma with the
    folded potential kernel (the slope terms fold as for the forces)."""
    Kp, _ = fold(cells, grid.beta, grid.dphi)
    Phi, _ = fft_conv(sigma, Kp, np.zeros_like(Kp), G)
    return grid.r[:, None] * Phi


# --------------------------------------------------------------------------
# The origin wedge (Sec. 3.2.1, third terms of Eq. 27-29)
# --------------------------------------------------------------------------
def wedge_cells(nu: int, nphi: int, du: float, pot: bool = False, rtol: float = 2e-14,
                nthreads: int = 0) -> np.ndarray:
    """Table [6, Nu, Nphi] of the wedge kernels K-bar seen from grid row i
    (slots as the cell table: K^{r,0}, K^{r,r}, K^{r,phi}, K^{phi,0},
    K^{phi,r}, K^{phi,phi}; the potential's three and zeros with pot).  The
    wedge is [0, r_in] x one azimuthal cell, with r_in the grid's inner face
    and its centre at r_in / 2 (sg_oracle.c)."""
    out = np.zeros((NC, nu, nphi))
    bad = _load().sgo_wedge_table(int(nu), int(nphi), float(du), float(rtol), int(bool(pot)), _dp(out),
                                  int(nthreads))
    if bad:
        raise RuntimeError(f"oracle quadrature did not converge for {bad} integrals")
    return out


def wedge_sums(sigma: np.ndarray, sigma_w: np.ndarray, wcells: np.ndarray, grid: Grid, G: float = 1.0):
    """The third terms of Eq. 27-29 (and A8-A10) as literal single sums over
    the wedge cells j':
        F_i,j += G sum_j' [sigma_w[j'] Kb^{.,0}[i, j - j'] + r_i dr_w[j'] Kb^{.,r}[i, j - j']
                            + dphi_w[j'] Kb^{.,phi}[i, j - j']],
    with the wedge's radial slope one-sided toward the first grid row,
    dr_w = (sigma[0] - sigma_w) / (r_0 - r_in / 2), and its azimuthal slope
    central and periodic."""
    nu, nphi = sigma.shape
    sigma_w = np.asarray(sigma_w, dtype=np.float64)
    r_w = 0.5 * grid.faces[0]
    dr = (np.asarray(sigma[0], dtype=np.float64) - sigma_w) / (grid.r[0] - r_w)
    dp = (np.roll(sigma_w, -1) - np.roll(sigma_w, 1)) / (2.0 * grid.dphi)
    Fr = np.zeros((nu, nphi))
    Fp = np.zeros((nu, nphi))
    j = np.arange(nphi)
    ri = grid.r[:, None]
    for jp in range(nphi):
        col = (j - jp) % nphi
        Fr += sigma_w[jp] * wcells[0][:, col] + ri * dr[jp] * wcells[1][:, col] + dp[jp] * wcells[2][:, col]
        Fp += sigma_w[jp] * wcells[3][:, col] + ri * dr[jp] * wcells[4][:, col] + dp[jp] * wcells[5][:, col]
    return G * Fr, G * Fp


def wedge_forces(sigma: np.ndarray, sigma_w: np.ndarray, cells: np.ndarray, wcells: np.ndarray, grid: Grid,
                 G: float = 1.0):
    """Forces on the grid with the origin wedge below its first row: the grid's
    own sums with one-sided radial slopes at its first and last rows (no ghost
    rows: the region below the first row is the wedge's) plus the wedge's
    single sums."""
    Fr, Fp = onesided_forces(sigma, cells, grid, G)
    Wr, Wp = wedge_sums(sigma, sigma_w, wcells, grid, G)
    return Fr + Wr, Fp + Wp


def kernel_cells_tpz(nu: int, nphi: int, du: float, n_tpz: int, rtol: float = 2e-14, nthreads: int = 0) -> np.ndarray:
    """Kernel table [6, 2Nu+1, Nphi] of the trapezoidal form (Eq. 41-43;
    the paper's SIM with N_tpz trapezoids per cell in phi): K^{r,0},
    K^{r,r}, K^{r,phi}, K^{phi,phi} by the trapezoidal rule over N_tpz + 1
    azimuths of exact eta-integrals, K^{phi,0}, K^{phi,r} and the own cell
    exact (sg_oracle.c)."""
    out = np.zeros((NC, 2 * nu + 1, nphi))
    bad = _load().sgo_cells_table_tpz(int(nu), int(nphi), float(du), int(n_tpz), float(rtol), _dp(out),
                                      int(nthreads))
    if bad:
        raise RuntimeError(f"oracle quadrature did not converge for {bad} integrals")
    return out


def kernels_tpz(nu: int, nphi: int, du: float, n_tpz: int, rtol: float = 2e-14, nthreads: int = 0):
    """Folded kernels (Kr, Kphi) of the trapezoidal form."""
    cells = kernel_cells_tpz(nu, nphi, du, n_tpz, rtol=rtol, nthreads=nthreads)
    return fold(cells, math.exp(du), 2.0 * math.pi / nphi)


# --------------------------------------------------------------------------
# Eq. 25 slopes and the three-term sums of Eq. 26-29 / A8-A10
# --------------------------------------------------------------------------
def slopes(sigma: np.ndarray, grid: Grid, edges: str = "ghost"):
    """Slopes of the piecewise-linear density (Eq. 25; Sec. 5.3 uses central
    differences).

    edges = "ghost" (the default): sigma is zero outside the grid and the
    central stencil is applied wherever it touches the grid, so the returned
    rows are i' = -1 .. Nu (the two ghost rows included):
        dr[i'] = (sigma_{i'+1} - sigma_{i'-1}) / (r_{i'+1} - r_{i'-1}).
    edges = "onesided": only the grid's rows i' = 0 .. Nu-1 carry slopes,
    central inside and one-sided at the first and last rows:
        dr[0] = (sigma_1 - sigma_0) / (r_1 - r_0),
        dr[Nu-1] = (sigma_{Nu-1} - sigma_{Nu-2}) / (r_{Nu-1} - r_{Nu-2}).
    Returns (dr, dphi_slope, rows) with dr[n] the slope of row rows[n] and
    dphi_slope[i', j'] = (sigma_{j'+1} - sigma_{j'-1}) / (2 dphi), periodic.
    """
    nu, nphi = sigma.shape
    dphi_slope = (np.roll(sigma, -1, axis=1) - np.roll(sigma, 1, axis=1)) / (2.0 * grid.dphi)
    if edges == "onesided":
        rows = np.arange(nu)
        dr = np.empty((nu, nphi))
        for i in range(nu):
            lo, hi = max(i - 1, 0), min(i + 1, nu - 1)
            dr[i] = (sigma[hi] - sigma[lo]) / (grid.r[hi] - grid.r[lo])
        return dr, dphi_slope, rows
    if edges != "ghost":
        raise ValueError(edges)
    ext = np.zeros((nu + 4, nphi))  # rows -2 .. Nu+1
    ext[2:nu + 2] = sigma
    rows = np.arange(-1, nu + 1)
    rc = np.array([grid.centre(i) for i in range(-2, nu + 2)])
    dr = np.empty((nu + 2, nphi))
    for n, ip in enumerate(rows):
        e = ip + 2
        dr[n] = (ext[e + 1] - ext[e - 1]) / (rc[e + 1] - rc[e - 1])
    return dr, dphi_slope, rows


def three_sum(sigma: np.ndarray, cells: np.ndarray, grid: Grid, G: float = 1.0, edges: str = "ghost"):
    """Eq. 26-29 (radial) and A8-A10 (azimuthal) on the single grid, term by
    term: F^r = F^{r,0} + r_i sum delta^r K^{r,r} + sum delta^phi K^{r,phi},
    and the same for F^phi, with the slopes of ``slopes(..., edges)``.
    O(N^4); for small grids."""
    nu, nphi = sigma.shape
    dr, dph, rows = slopes(sigma, grid, edges)
    Fr = np.zeros((nu, nphi))
    Fp = np.zeros((nu, nphi))
    Frr = np.zeros((nu, nphi))
    Fpr = np.zeros((nu, nphi))
    i = np.arange(nu)[:, None]
    j = np.arange(nphi)[None, :]
    for ip in range(nu):
        for jp in range(nphi):
            k = i - ip + nu
            q = (j - jp) % nphi
            s, sp = sigma[ip, jp], dph[ip, jp]
            Fr += s * cells[0][k, q] + sp * cells[2][k, q]
            Fp += s * cells[3][k, q] + sp * cells[5][k, q]
    for n, ip in enumerate(rows):
        for jp in range(nphi):
            d = dr[n, jp]
            if d == 0.0:
                continue
            k = i - ip + nu
            q = (j - jp) % nphi
            Frr += d * cells[1][k, q]
            Fpr += d * cells[4][k, q]
    Fr += grid.r[:, None] * Frr
    Fp += grid.r[:, None] * Fpr
    return G * Fr, G * Fp


def onesided_forces(sigma: np.ndarray, cells: np.ndarray, grid: Grid, G: float = 1.0):
    """The sums of ``three_sum(..., edges="onesided")`` for any grid size: the
    convolution with the folded kernels (the ghost-row slopes) plus the
    radial slope terms of Eq. 28 / A9 for the difference of the two slope
    sets, which is non-zero on the rows -1, 0, Nu-1 and Nu only:
        r_i sum_{i', j'} (dr_onesided - dr_ghost)[i', j'] K^{.,r}[i - i', j - j']."""
    nu, nphi = sigma.shape
    Kr, Kp = fold(cells, grid.beta, grid.dphi)
    Fr, Fp = fft_conv(sigma, Kr, Kp, G)
    # the two slope sets differ on those four rows only (elsewhere both are
    # the same central difference, up to the rounding of its two forms)
    diff, rows_d = _edge_slope_difference(sigma, grid)
    i = np.arange(nu)[:, None]
    j = np.arange(nphi)[None, :]
    Frr = np.zeros((nu, nphi))
    Fpr = np.zeros((nu, nphi))
    for n, ip in enumerate(rows_d):
        for jp in range(nphi):
            k = i - ip + nu
            q = (j - jp) % nphi
            Frr += diff[n, jp] * cells[1][k, q]
            Fpr += diff[n, jp] * cells[4][k, q]
    return Fr + G * grid.r[:, None] * Frr, Fp + G * grid.r[:, None] * Fpr


def _edge_slope_difference(sigma: np.ndarray, grid: Grid):
    """The one-sided minus the ghost-row radial slopes on the four rows where
    they differ: rows (-1, 0, Nu-1, Nu) and their difference rows (for the
    ghost rows -1 and Nu the one-sided set has no slope: minus the ghost one)."""
    nu = sigma.shape[0]
    dg, _, rows_g = slopes(sigma, grid, "ghost")
    do, _, _ = slopes(sigma, grid, "onesided")
    diff = -dg
    diff[1:nu + 1] += do  # rows_g[n] = n - 1
    keep = [0, 1, nu, nu + 1]
    return diff[keep], rows_g[keep]


def onesided_forces_at(sigma: np.ndarray, cells: np.ndarray, grid: Grid, targets, G: float = 1.0):
    """onesided_forces at the flat target cells i*Nphi + j only, for grids too
    large for the whole field: the convolution by the direct sum at the
    targets plus, per target, the radial slope terms of Eq. 28 / A9 for the
    slope difference on the four rows where it is not zero,
        G r_i sum_{ip, j'} diff[ip, j'] K^{.,r}[i - ip, j - j']."""
    nu, nphi = sigma.shape
    t = np.asarray(targets, dtype=np.int64)
    Kr, Kp = fold(cells, grid.beta, grid.dphi)
    Fr, Fp = direct_sum(sigma, Kr, Kp, G, targets=t)
    diff, rows = _edge_slope_difference(sigma, grid)
    ti, tj = t // nphi, t % nphi
    q = (tj[:, None] - np.arange(nphi)[None, :]) % nphi
    for d, ip in zip(diff, rows):
        k = (ti - ip + nu)[:, None]
        Fr = Fr + G * grid.r[ti] * (cells[1][k, q] * d[None, :]).sum(axis=1)
        Fp = Fp + G * grid.r[ti] * (cells[4][k, q] * d[None, :]).sum(axis=1)
    return Fr, Fp


def onesided_forces_T(gFr: np.ndarray, gFp: np.ndarray, cells: np.ndarray, grid: Grid, G: float = 1.0):
    """Transpose of onesided_forces: the correlation with the folded kernels
    (fft_conv_T) plus the transpose of the slope-difference terms.  The slope
    difference of each column is linear in that column's rows (0, 1, Nu-2,
    Nu-1): diff[ip] = sum_b D[ip, b] sigma[b] (D from _edge_slope_difference
    on unit rows), so with, for each of the four slope rows ip,
        t[ip, j'] = G sum_{i, j} r_i (gFr[i, j] K^{r,r}[i - ip, j - j'] + gFphi[i, j] K^{phi,r}[i - ip, j - j'])
    (a circular correlation along phi per row, taken by numpy's FFT),
        gsigma[b] += sum_ip D[ip, b] t[ip]."""
    nu, nphi = gFr.shape
    Kr, Kp = fold(cells, grid.beta, grid.dphi)
    gs = fft_conv_T(gFr, gFp, Kr, Kp, G)
    brows = [0, 1, nu - 2, nu - 1]
    D = np.zeros((4, 4))
    col = Grid(nu, 1, grid.u_min, grid.du)  # the radial slopes do not depend on N_phi
    for b, rb in enumerate(brows):
        e = np.zeros((nu, 1))
        e[rb, 0] = 1.0
        d, rows = _edge_slope_difference(e, col)
        D[:, b] = d[:, 0]
    ar = np.fft.rfft(gFr * grid.r[:, None], axis=1)
    ap = np.fft.rfft(gFp * grid.r[:, None], axis=1)
    t = np.zeros((4, nphi))
    for a, ip in enumerate(rows):
        k = np.arange(nu) - ip + nu
        c = (ar * np.conj(np.fft.rfft(cells[1][k], axis=1))).sum(axis=0) + \
            (ap * np.conj(np.fft.rfft(cells[4][k], axis=1))).sum(axis=0)
        t[a] = G * np.fft.irfft(c, n=nphi)
    for b, rb in enumerate(brows):
        gs[rb] += D[:, b] @ t
    return gs


def wedge_sums_at(sigma: np.ndarray, sigma_w: np.ndarray, wcells: np.ndarray, grid: Grid, targets,
                  G: float = 1.0):
    """wedge_sums at the flat target cells i*Nphi + j only: the same single
    sums over the wedge cells j', per target."""
    nu, nphi = sigma.shape
    t = np.asarray(targets, dtype=np.int64)
    sigma_w = np.asarray(sigma_w, dtype=np.float64)
    r_w = 0.5 * grid.faces[0]
    dr = (np.asarray(sigma[0], dtype=np.float64) - sigma_w) / (grid.r[0] - r_w)
    dp = (np.roll(sigma_w, -1) - np.roll(sigma_w, 1)) / (2.0 * grid.dphi)
    ti, tj = t // nphi, t % nphi
    q = (tj[:, None] - np.arange(nphi)[None, :]) % nphi
    ri = grid.r[ti][:, None]
    out = []
    for c0, cr, cp in ((0, 1, 2), (3, 4, 5)):
        terms = sigma_w[None, :] * wcells[c0][ti[:, None], q] + ri * dr[None, :] * wcells[cr][ti[:, None], q] + \
            dp[None, :] * wcells[cp][ti[:, None], q]
        out.append(G * terms.sum(axis=1))
    return out[0], out[1]


def wedge_forces_at(sigma: np.ndarray, sigma_w: np.ndarray, cells: np.ndarray, wcells: np.ndarray, grid: Grid,
                    targets, G: float = 1.0):
    """wedge_forces at the flat target cells only."""
    Fr, Fp = onesided_forces_at(sigma, cells, grid, targets, G)
    Wr, Wp = wedge_sums_at(sigma, sigma_w, wcells, grid, targets, G)
    return Fr + Wr, Fp + Wp


def fold(cells: np.ndarray, beta: float, dphi: float):
    """Collapse the three sums into one kernel per component.

    With delta^r_{i'} = (sigma_{i'+1} - sigma_{i'-1}) / (r_{i'} (beta - 1/beta))
    (r_{i'+-1} = beta^{+-1} r_{i'}) and r_i / r_{i'} = beta^{i-i'}, and the
    periodic delta^phi, every term is linear in sigma and depends on (i-i',
    j-j') only, so for k in [-(Nu-1), Nu-1]:
      K^eff[k,q] = K^{.,0}[k,q]
                   + (beta^{k+1} K^{.,r}[k+1,q] - beta^{k-1} K^{.,r}[k-1,q]) / (beta - 1/beta)
                   + (K^{.,phi}[k,q+1] - K^{.,phi}[k,q-1]) / (2 dphi).
    Input cells [6, 2Nu+1, Nphi] (k in [-Nu, Nu]); output Kr, Kphi
    [2Nu-1, Nphi] (row k + Nu - 1).
    """
    nk = cells.shape[1]
    nu = (nk - 1) // 2
    k = np.arange(-(nu - 1), nu)[:, None].astype(np.float64)
    mid = slice(1, nk - 1)
    up = slice(2, nk)
    dn = slice(0, nk - 2)
    bb = beta - 1.0 / beta
    out = []
    for c0, cr, cp in ((0, 1, 2), (3, 4, 5)):
        K = cells[c0][mid].copy()
        K += (beta ** (k + 1) * cells[cr][up] - beta ** (k - 1) * cells[cr][dn]) / bb
        K += (np.roll(cells[cp][mid], -1, axis=1) - np.roll(cells[cp][mid], 1, axis=1)) / (2.0 * dphi)
        out.append(K)
    return out[0], out[1]


def direct_sum(sigma: np.ndarray, Kr: np.ndarray, Kp: np.ndarray, G: float = 1.0, targets=None, nthreads: int = 0):
    """F_r, F_phi = G sum_{m,l} sigma[m,l] K[i-m, (j-l) mod Nphi] (direct O(N^2)).

    targets: optional flat indices i*Nphi + j; returns flat arrays then."""
    sigma = np.ascontiguousarray(sigma, dtype=np.float64)
    nu, nphi = sigma.shape
    Kr = np.ascontiguousarray(Kr, dtype=np.float64)
    Kp = np.ascontiguousarray(Kp, dtype=np.float64)
    assert Kr.shape == (2 * nu - 1, nphi) and Kp.shape == Kr.shape
    lib = _load()
    if targets is None:
        Fr = np.zeros((nu, nphi))
        Fp = np.zeros((nu, nphi))
        lib.sgo_direct_sum(nu, nphi, float(G), _dp(Kr), _dp(Kp), _dp(sigma), None, 0, _dp(Fr), _dp(Fp), int(nthreads))
        return Fr, Fp
    t = np.ascontiguousarray(targets, dtype=np.int64)
    Fr = np.zeros(t.size)
    Fp = np.zeros(t.size)
    lib.sgo_direct_sum(nu, nphi, float(G), _dp(Kr), _dp(Kp), _dp(sigma),
                       t.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), t.size, _dp(Fr), _dp(Fp), int(nthreads))
    return Fr, Fp


def direct_sum_T(gFr: np.ndarray, gFp: np.ndarray, Kr: np.ndarray, Kp: np.ndarray, G: float = 1.0,
                 sources=None, nthreads: int = 0):
    """Transpose of direct_sum: gsigma[m,l] = G sum_{i,j} (gFr[i,j] Kr[i-m,(j-l)] + gFphi[i,j] Kphi[i-m,(j-l)])."""
    gFr = np.ascontiguousarray(gFr, dtype=np.float64)
    gFp = np.ascontiguousarray(gFp, dtype=np.float64)
    nu, nphi = gFr.shape
    Kr = np.ascontiguousarray(Kr, dtype=np.float64)
    Kp = np.ascontiguousarray(Kp, dtype=np.float64)
    lib = _load()
    if sources is None:
        gs = np.zeros((nu, nphi))
        lib.sgo_direct_sum_T(nu, nphi, float(G), _dp(Kr), _dp(Kp), _dp(gFr), _dp(gFp), None, 0, _dp(gs), int(nthreads))
        return gs
    s = np.ascontiguousarray(sources, dtype=np.int64)
    gs = np.zeros(s.size)
    lib.sgo_direct_sum_T(nu, nphi, float(G), _dp(Kr), _dp(Kp), _dp(gFr), _dp(gFp),
                         s.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), s.size, _dp(gs), int(nthreads))
    return gs


def fft_conv(sigma: np.ndarray, Kr: np.ndarray, Kp: np.ndarray, G: float = 1.0):
    """The direct_sum convolution evaluated with numpy's FFT (a library step):
    sigma zero-padded to 2Nu rows, the kernel placed cyclically at row k mod 2Nu
    (row Nu left zero), periodic in phi; rows 0..Nu-1 of the cyclic result."""
    nu, nphi = sigma.shape
    L = 2 * nu
    sp = np.zeros((L, nphi))
    sp[:nu] = sigma
    S = np.fft.rfft2(sp)
    out = []
    for K in (Kr, Kp):
        Kc = np.zeros((L, nphi))
        k = np.arange(-(nu - 1), nu)
        Kc[k % L] = K
        out.append(G * np.fft.irfft2(S * np.fft.rfft2(Kc), s=(L, nphi))[:nu])
    return out[0], out[1]


def fft_conv_T(gFr: np.ndarray, gFp: np.ndarray, Kr: np.ndarray, Kp: np.ndarray, G: float = 1.0):
    """Transpose of fft_conv (correlation with the kernels), by numpy's FFT."""
    nu, nphi = gFr.shape
    L = 2 * nu
    acc = np.zeros((L, nphi), dtype=np.complex128)
    for g, K in ((gFr, Kr), (gFp, Kp)):
        gp = np.zeros((L, nphi))
        gp[:nu] = g
        Kc = np.zeros((L, nphi))
        k = np.arange(-(nu - 1), nu)
        Kc[k % L] = K
        acc += np.fft.fft2(gp) * np.conj(np.fft.fft2(Kc))
    return G * np.real(np.fft.ifft2(acc))[:nu]


def kernels(nu: int, nphi: int, du: float, rtol: float = 2e-14, nthreads: int = 0):
    """Folded kernels (Kr, Kphi) for a grid; the one-time preparation step."""
    cells = kernel_cells(nu, nphi, du, rtol=rtol, nthreads=nthreads)
    return fold(cells, math.exp(du), 2.0 * math.pi / nphi)


# --------------------------------------------------------------------------
# Eq. 47-49 error norms and the relative L2 used for parity
# --------------------------------------------------------------------------
def norms(F_num: np.ndarray, F_ana: np.ndarray, mask=None):
    """L1, L2, Linf of Eq. 47-49 (unweighted over the chosen cells)."""
    d = np.abs(np.asarray(F_num) - np.asarray(F_ana))
    if mask is not None:
        d = d[mask]
    return float(d.mean()), float(np.sqrt((d * d).mean())), float(d.max())


def rel_l2(Fr, Fp, Fr_ref, Fp_ref) -> float:
    """sqrt(sum dFr^2 + dFphi^2) / sqrt(sum Fr_ref^2 + Fphi_ref^2), both
    components together, unweighted over cells."""
    num = np.sum((np.asarray(Fr, np.float64) - Fr_ref) ** 2) + np.sum((np.asarray(Fp, np.float64) - Fp_ref) ** 2)
    den = np.sum(np.asarray(Fr_ref) ** 2) + np.sum(np.asarray(Fp_ref) ** 2)
    return float(math.sqrt(num / den))
