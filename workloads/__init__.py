"""Seeded synthetic inputs for the thin-disk force path.

This module holds only input generation: surface densities evaluated at cell
centres, seeded random fields and the batch recipe.  It contains none of the
method's arithmetic (no kernels, slopes, sums or transforms) and is the one
module that both the tests' oracle side and the CUDA side may use.

The paper's workloads are analytic disks, not a dataset; every input here is
a formula evaluated on the grid, or a seeded numpy (PCG64) draw.

Grid: u = ln r is uniform with step du starting at the inner face radius
r_in; cell centres are the arithmetic means of the two faces (Sec. 3.2.1 of
the paper), azimuths phi_j = (j + 1/2) 2 pi / N_phi.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np


def grid_params(nu: int, r_in: float, r_out: float):
    """(u_min, du) for Nu log-spaced rows between the faces r_in and r_out."""
    return math.log(r_in), math.log(r_out / r_in) / nu


def centres(nu: int, nphi: int, u_min: float, du: float):
    """Cell-centre radii r[Nu] and azimuths phi[Nphi]."""
    i = np.arange(nu, dtype=np.float64)
    lo = np.exp(u_min + du * i)
    r = 0.5 * (lo + lo * math.exp(du))
    phi = (np.arange(nphi, dtype=np.float64) + 0.5) * (2.0 * math.pi / nphi)
    return r, phi


def cell_areas(nu: int, nphi: int, u_min: float, du: float):
    """r_i (r_{i+1/2} - r_{i-1/2}) dphi per row (loss weights)."""
    i = np.arange(nu, dtype=np.float64)
    lo = np.exp(u_min + du * i)
    hi = lo * math.exp(du)
    return 0.5 * (lo + hi) * (hi - lo) * (2.0 * math.pi / nphi)


# --------------------------------------------------------------------------
# Named configurations (sizes and radial extents)
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class Config:
    name: str
    nu: int
    nphi: int
    r_in: float
    r_out: float

    @property
    def u_min(self):
        return grid_params(self.nu, self.r_in, self.r_out)[0]

    @property
    def du(self):
        return grid_params(self.nu, self.r_in, self.r_out)[1]

    def centres(self):
        return centres(self.nu, self.nphi, self.u_min, self.du)


KUZMIN_64 = Config("kuzmin-64x64", 64, 64, 0.05, 20.0)
SPIRAL_512 = Config("spiral-clump-512x1024", 512, 1024, 0.01, 100.0)
GRF_2048 = Config("lognormal-grf-2048x4096", 2048, 4096, 0.01, 100.0)
DIFF_1024 = Config("diff-kuzmin-spiral-1024x2048", 1024, 2048, 0.01, 100.0)


# --------------------------------------------------------------------------
# Densities
# --------------------------------------------------------------------------
def kuzmin(r, phi, M=1.0, a=1.0):
    """Kuzmin disk sigma = M a / (2 pi (r^2 + a^2)^{3/2}) on the (r, phi) grid."""
    r = np.asarray(r, dtype=np.float64)[:, None]
    s = M * a / (2.0 * math.pi * (r * r + a * a) ** 1.5)
    return np.broadcast_to(s, (r.shape[0], np.asarray(phi).size)).copy()


def log_spiral(r, phi, m=2, amp=0.1, pitch_deg=20.0, phase=0.0):
    """1 + amp cos(m phi - ln r / tan(pitch) + phase)."""
    r = np.asarray(r, dtype=np.float64)[:, None]
    phi = np.asarray(phi, dtype=np.float64)[None, :]
    return 1.0 + amp * np.cos(m * phi - np.log(r) / math.tan(math.radians(pitch_deg)) + phase)


def offcentre_kuzmin(r, phi, M, a, rc, phic):
    """Kuzmin profile in the distance d from the point (rc, phic)."""
    r = np.asarray(r, dtype=np.float64)[:, None]
    phi = np.asarray(phi, dtype=np.float64)[None, :]
    X = r * np.cos(phi) - rc * math.cos(phic)
    Y = r * np.sin(phi) - rc * math.sin(phic)
    d2 = X * X + Y * Y
    return M * a / (2.0 * math.pi * (d2 + a * a) ** 1.5)


def spiral_clump(r, phi):
    """Kuzmin(a=1) x (1 + 0.1 cos(2 phi - ln r / tan 20 deg)) plus a Kuzmin
    clump (M = 0.05, a = 0.2) centred at r = 3, phi = 1.0 rad."""
    return kuzmin(r, phi) * log_spiral(r, phi, 2, 0.1, 20.0) + offcentre_kuzmin(r, phi, 0.05, 0.2, 3.0, 1.0)


def gaussian_random_field(nu: int, nphi: int, seed: int = 1509, slope: float = 3.0):
    """Gaussian random field on the Nu x Nphi index torus with power spectrum
    P(k) ~ |k|^-slope (k != 0), the k = 0 mode removed, scaled to unit
    variance.  White noise from numpy's PCG64 filtered in Fourier space."""
    rng = np.random.default_rng(seed)
    w = rng.standard_normal((nu, nphi))
    ku = np.fft.fftfreq(nu) * nu
    kp = np.fft.fftfreq(nphi) * nphi
    k = np.sqrt(ku[:, None] ** 2 + kp[None, :] ** 2)
    amp = np.zeros_like(k)
    amp[k > 0] = k[k > 0] ** (-slope / 2.0)
    g = np.real(np.fft.ifft2(np.fft.fft2(w) * amp))
    g -= g.mean()
    g /= g.std()
    return g


def lognormal_disk(r, phi, seed: int = 1509):
    """sigma = exp(0.5 g) e^{-r/3} with g the unit-variance k^-3 field."""
    nu, nphi = np.asarray(r).size, np.asarray(phi).size
    g = gaussian_random_field(nu, nphi, seed)
    return np.exp(0.5 * g) * np.exp(-np.asarray(r, dtype=np.float64)[:, None] / 3.0)


def sigma_dn(n: int, alpha: float, xc: float, yc: float, r, phi):
    """sigma_{D_n} = (1 - d^2/alpha^2)^{n-1/2} for d < alpha (Eq. 50 of the
    paper, sigma_0 = 1) with d the distance from (xc, yc)."""
    r = np.asarray(r, dtype=np.float64)[:, None]
    phi = np.asarray(phi, dtype=np.float64)[None, :]
    X = r * np.cos(phi) - xc
    Y = r * np.sin(phi) - yc
    x2 = (X * X + Y * Y) / (alpha * alpha)
    return np.where(x2 < 1.0, np.clip(1.0 - x2, 0.0, None) ** (n - 0.5), 0.0)


def random_field(nu: int, nphi: int, seed: int):
    """Plain N(0, 1) field (edge cases, adjoint dot tests)."""
    return np.random.default_rng(seed).standard_normal((nu, nphi))


# --------------------------------------------------------------------------
# Batch recipe: 256 exponential disks with m = 1..4 log spirals
# --------------------------------------------------------------------------
@dataclass(frozen=True)
class BatchDisk:
    nu: int
    nphi: int
    m: int
    amp: float
    pitch_deg: float
    r_in: float = 0.01
    r_out: float = 100.0

    @property
    def u_min(self):
        return grid_params(self.nu, self.r_in, self.r_out)[0]

    @property
    def du(self):
        return grid_params(self.nu, self.r_in, self.r_out)[1]

    def sigma(self):
        r, phi = centres(self.nu, self.nphi, self.u_min, self.du)
        return np.exp(-r / 3.0)[:, None] * log_spiral(r, phi, self.m, self.amp, self.pitch_deg)


def batch_disks(n: int = 256, seed: int = 1450, nus=(128, 256, 512, 1024), nphis=(256, 512, 1024, 2048)):
    """The seeded list of n disks: N_u and N_phi drawn independently and
    uniformly from the given sets, m ~ U{1..4}, amplitude ~ U(0, 0.2),
    pitch ~ U(10, 30) degrees."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nu = int(rng.choice(nus))
        nphi = int(rng.choice(nphis))
        m = int(rng.integers(1, 5))
        amp = float(rng.uniform(0.0, 0.2))
        pitch = float(rng.uniform(10.0, 30.0))
        out.append(BatchDisk(nu, nphi, m, amp, pitch))
    return out


# --------------------------------------------------------------------------
# Differentiation recipe
# --------------------------------------------------------------------------
def diff_problem(cfg: Config = DIFF_1024):
    """(sigma_start, sigma_target, w): start = plain Kuzmin, target = Kuzmin x
    (1 + 0.15 cos(2 phi - ln r / tan 20 deg)), w = cell area per row."""
    r, phi = cfg.centres()
    start = kuzmin(r, phi)
    target = kuzmin(r, phi) * log_spiral(r, phi, 2, 0.15, 20.0)
    w = cell_areas(cfg.nu, cfg.nphi, cfg.u_min, cfg.du)
    return start, target, w
