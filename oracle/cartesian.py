"""Oracle for the Cartesian second-order scheme (Sec. 3.1.1, Eq. 6-15, with
the closed-form kernels of App. A) -- test infrastructure only.

Grid: square cells of side dx = dy on N_x x N_y cells, sigma zero outside.
For a target cell (i, j) and a source cell (i', j') with offsets
k = i - i', q = j - j', the source cell relative to the target centre is
X in [(-k - 1/2) dx, (-k + 1/2) dx], Y in [(-q - 1/2) dy, (-q + 1/2) dy].
The six cell integrals are (App. A; the y ones by symmetry)

    K^{x,0} = dbl[-ln(Y + R)],          K^{y,0} = dbl[-ln(X + R)],
    K^{x,x} = k dx K^{x,0} + dbl[Y ln(X + R)],
    K^{y,y} = q dy K^{y,0} + dbl[X ln(Y + R)],
    K^{x,y} = q dy K^{x,0} + dbl[-R],   K^{y,x} = k dx K^{y,0} + dbl[-R],

R = sqrt(X^2 + Y^2), dbl[f] = f(x_u, y_u) - f(x_l, y_u) - f(x_u, y_l) + f(x_l, y_l)
(the App. A double difference).  For Y < 0, ln(Y + R) is evaluated as
2 ln|X| - ln(R - Y), which has no cancellation; no corner has X = 0 or
Y = 0, because corners sit at half-integer multiples of the cell side.

The forces are F^x = G (sum sigma K^{x,0} + sum delta^x K^{x,x} + sum delta^y K^{x,y})
(Eq. 9-12) and likewise F^y, with central slopes delta^x = (sigma_{i+1} -
sigma_{i-1}) / (2 dx) taken wherever the stencil touches the grid (the
ghost cells one beyond each edge included), as for the polar grid.
"""
from __future__ import annotations

import numpy as np

__all__ = ["cells", "three_sum", "fold", "forces", "slopes"]


def _log_sum(a, b):
    """ln(a + sqrt(a^2 + b^2)) for b != 0, without cancellation for a < 0."""
    R = np.hypot(a, b)
    with np.errstate(divide="ignore"):
        return np.where(a >= 0, np.log(a + R), 2.0 * np.log(np.abs(b)) - np.log(R - a))


def _dbl(f, xl, xu, yl, yu):
    return f(xu, yu) - f(xl, yu) - f(xu, yl) + f(xl, yl)


def cells(nx: int, ny: int, dx: float, dy: float | None = None) -> np.ndarray:
    """Kernel table [6, 2 nx + 1, 2 ny + 1] over k in [-nx, nx], q in [-ny, ny]:
    K^{x,0}, K^{x,x}, K^{x,y}, K^{y,0}, K^{y,x}, K^{y,y} (App. A)."""
    dy = dx if dy is None else dy
    k = np.arange(-nx, nx + 1, dtype=np.float64)[:, None]
    q = np.arange(-ny, ny + 1, dtype=np.float64)[None, :]
    xl, xu = (-k - 0.5) * dx, (-k + 0.5) * dx
    yl, yu = (-q - 0.5) * dy, (-q + 0.5) * dy
    Kx0 = _dbl(lambda X, Y: -_log_sum(Y, X), xl, xu, yl, yu)
    Ky0 = _dbl(lambda X, Y: -_log_sum(X, Y), xl, xu, yl, yu)
    Kxx = k * dx * Kx0 + _dbl(lambda X, Y: Y * _log_sum(X, Y), xl, xu, yl, yu)
    Kyy = q * dy * Ky0 + _dbl(lambda X, Y: X * _log_sum(Y, X), xl, xu, yl, yu)
    mR = _dbl(lambda X, Y: -np.hypot(X, Y), xl, xu, yl, yu)
    Kxy = q * dy * Kx0 + mR
    Kyx = k * dx * Ky0 + mR
    return np.stack([Kx0, Kxx, Kxy, Ky0, Kyx, Kyy])


def slopes(sigma: np.ndarray, dx: float, dy: float | None = None):
    """Central slopes on the grid padded by one ghost cell on every side
    (sigma zero there): arrays [N_x + 2, N_y + 2]; index 0 is the ghost cell
    before the first row or column."""
    dy = dx if dy is None else dy
    s = np.pad(np.asarray(sigma, dtype=np.float64), 2)
    ddx = (s[2:, 1:-1] - s[:-2, 1:-1]) / (2.0 * dx)
    ddy = (s[1:-1, 2:] - s[1:-1, :-2]) / (2.0 * dy)
    return ddx, ddy


def three_sum(sigma: np.ndarray, K: np.ndarray, dx: float, dy: float | None = None, G: float = 1.0):
    """F^x, F^y by the literal sums of Eq. 10-12 (and their y forms): every
    source cell, ghost cells included, with its sigma and its two slopes
    against the kernel at its offset.  O(N^4); small grids only."""
    nx, ny = sigma.shape
    ddx, ddy = slopes(sigma, dx, dy)
    sp = np.pad(np.asarray(sigma, dtype=np.float64), 1)
    Fx = np.zeros((nx, ny))
    Fy = np.zeros((nx, ny))
    for i in range(nx):
        for j in range(ny):
            for a in range(nx + 2):  # source index a - 1
                for b in range(ny + 2):
                    k, q = i - (a - 1), j - (b - 1)
                    kk, qq = k + K.shape[1] // 2, q + K.shape[2] // 2
                    s0, sx, sy = sp[a, b], ddx[a, b], ddy[a, b]
                    Fx[i, j] += s0 * K[0, kk, qq] + sx * K[1, kk, qq] + sy * K[2, kk, qq]
                    Fy[i, j] += s0 * K[3, kk, qq] + sx * K[4, kk, qq] + sy * K[5, kk, qq]
    return G * Fx, G * Fy


def fold(K: np.ndarray, dx: float, dy: float | None = None):
    """The slope terms folded into one kernel per component over
    k in [-(nx-1), nx-1], q in [-(ny-1), ny-1]:
    K^eff = K^{.,0} + (K^{.,x}[k+1] - K^{.,x}[k-1]) / (2 dx)
                    + (K^{.,y}[q+1] - K^{.,y}[q-1]) / (2 dy)."""
    dy = dx if dy is None else dy
    c = slice(1, -1)
    out = []
    for z, zx, zy in ((0, 1, 2), (3, 4, 5)):
        out.append(K[z][c, c] + (K[zx][2:, c] - K[zx][:-2, c]) / (2.0 * dx)
                   + (K[zy][c, 2:] - K[zy][c, :-2]) / (2.0 * dy))
    return out[0], out[1]


def forces(sigma: np.ndarray, Kx: np.ndarray, Ky: np.ndarray, G: float = 1.0):
    """F = G sum sigma[m, l] K^eff[i - m, j - l]: the linear 2-D convolution
    of sigma with the folded kernels, by numpy's FFT on the (2 N_x) x (2 N_y)
    zero-padded grid (a library step)."""
    sigma = np.asarray(sigma, dtype=np.float64)
    nx, ny = sigma.shape
    Lx, Ly = 2 * nx, 2 * ny
    S = np.fft.rfft2(sigma, s=(Lx, Ly))
    out = []
    for K in (Kx, Ky):
        P = np.zeros((Lx, Ly))
        kk = np.arange(-(nx - 1), nx) % Lx
        qq = np.arange(-(ny - 1), ny) % Ly
        P[np.ix_(kk, qq)] = K
        out.append(G * np.fft.irfft2(S * np.fft.rfft2(P), s=(Lx, Ly))[:nx, :ny])
    return out[0], out[1]
