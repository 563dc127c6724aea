"""Pins for the oracle's cell-integrated kernels (Eq. 30-32, A11-A13).

The oracle integrates the raw integrands numerically (nested adaptive
Gauss-Legendre).  These tests pin it to things other than itself:

* the paper's closed-form eta-antiderivatives H^r_1, H^r_2, H^phi_1, H^phi_2,
  H^phi_3 (App. A), evaluated in 40-digit mpmath with the remaining xi
  integral by tanh-sinh quadrature: an independent formula and method;
* ring sum rules: the sum over q of a row of kernels is the force of a
  uniform annulus, a one-dimensional elliptic-integral quadrature;
* exact symmetries in q and the zero self-cell values of the odd kernels;
* the far-field point-mass limit (Eq. 62);
* the paper's own Cartesian "fan" method for the self cell (Sec. 4, Fig. 1).
"""
import math

import numpy as np
import pytest

mpmath = pytest.importorskip("mpmath")

DU64 = math.log(400.0) / 64
NPHI64 = 64


# ---------------------------------------------------------------------------
# App. A closed forms (eta = rbar / r_i, xi = phibar - phi_j)
# ---------------------------------------------------------------------------
def _L(e, x):
    c, s = mpmath.cos(x), mpmath.sin(x)
    F = mpmath.sqrt((e - c) ** 2 + s * s)
    arg = e - c + F
    if e < c:  # e - c + F = sin^2 / (F - e + c) without cancellation
        arg = s * s / (F - e + c)
    return F, mpmath.log(arg)


def H_r1(e, x):
    c = mpmath.cos(x)
    F, L = _L(e, x)
    return -c * L + (2 * c * e - 1) / F


def H_r2(e, x):
    c = mpmath.cos(x)
    F, L = _L(e, x)
    return -((3 * c * c - 1) * L + (-6 * e * c * c + 3 * c + e * e * c + e) / F)


def H_p1(e, x):
    c = mpmath.cos(x)
    F, L = _L(e, x)
    return -(F + c * L)


def H_p2(e, x):
    # the printed cos(phi) in the log coefficient is cos(xi) (checked by differentiation)
    c = mpmath.cos(x)
    F, L = _L(e, x)
    return -((e / 2 + mpmath.mpf(3) / 2 * c) * F + (mpmath.mpf(3) / 2 * c * c - mpmath.mpf(1) / 2) * L)


def H_p3(e, x):
    c, s = mpmath.cos(x), mpmath.sin(x)
    F, L = _L(e, x)
    cot2 = (c / s) ** 2
    return x * s * ((-e - c + e * cot2 - c * cot2) / F + L)


def closed_form_cell(du, nphi, k, q):
    """All six kernels of offset (k, q) from the App. A formulas."""
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
    quad = lambda f: mpmath.quad(f, pts)
    Kr0 = -quad(lambda x: H_r1(eu, x) - H_r1(el, x))
    Krr = -quad(lambda x: H_r2(eu, x) - H_r2(el, x)) - ec * Kr0
    Krp = -quad(lambda x: x * (H_r1(eu, x) - H_r1(el, x))) + qs * dphi * Kr0
    corner = lambda H: (H(eu, xu) - H(el, xu)) - (H(eu, xl) - H(el, xl))
    Kp0 = corner(H_p1)
    Kpr = corner(H_p2) - ec * Kp0
    Kpp = quad(lambda x: H_p3(eu, x) - H_p3(el, x)) + qs * dphi * Kp0
    return np.array([float(v) for v in (Kr0, Krr, Krp, Kp0, Kpr, Kpp)])


CELLS = [(0, 1), (1, 0), (-1, 0), (1, 1), (-1, 63), (0, 2), (2, 1), (3, 60), (-4, 5), (7, 20), (-9, 31),
         (20, 32), (-30, 3), (64, 0), (-64, 17), (40, 50)]


@pytest.mark.parametrize("k,q", CELLS)
def test_cells_match_appendix_A_closed_forms(oracle_mod, k, q):
    got = oracle_mod.kernel_cell(DU64, NPHI64, k, q)
    ref = closed_form_cell(DU64, NPHI64, k, q)
    # natural scale of the cell: |K^{r,0}| + |K^{phi,0}| plus the slope
    # kernels' own magnitude
    scale = abs(ref[0]) + abs(ref[3]) + 1e-300
    for c in range(6):
        s = scale * (1.0 if c in (0, 3) else max(abs(ref[c]) / scale, DU64 * 0.05))
        assert abs(got[c] - ref[c]) <= 2e-12 * s, (c, got[c], ref[c])


def test_self_cell_matches_closed_forms(oracle_mod):
    got = oracle_mod.kernel_cell(DU64, NPHI64, 0, 0)
    ref = closed_form_cell(DU64, NPHI64, 0, 0)
    for c in (0, 1, 5):
        assert abs(got[c] - ref[c]) <= 1e-12 * abs(ref[c]), (c, got[c], ref[c])
    # the kernels odd in xi vanish on the self cell (Sec. 3.2.2, App. A)
    for c in (2, 3, 4):
        assert got[c] == 0.0
        assert abs(ref[c]) < 1e-25


def test_self_cell_invariant_of_position(oracle_mod):
    """Eq. 33: the self-cell values depend only on (beta, dphi).  Integrate the
    physical integrand of Eq. 30 (rbar, phibar, not the dimensionless form)
    over the self cells of two rows at very different radii and compare with
    the oracle's single dimensionless value."""
    mpmath.mp.dps = 30
    beta = mpmath.e ** mpmath.mpf(DU64)
    dphi = 2 * mpmath.pi / NPHI64
    ref = oracle_mod.kernel_cell(DU64, NPHI64, 0, 0)[0]
    for ri in (mpmath.mpf("0.3"), mpmath.mpf(7)):
        lo, hi = ri * 2 / (beta + 1), ri * 2 * beta / (beta + 1)

        def inner(x):
            c, s = mpmath.cos(x), mpmath.sin(x)
            # rbar^2 + r_i^2 - 2 rbar r_i cos = (rbar - r_i cos)^2 + (r_i sin)^2
            f = lambda rb: -rb * (ri - rb * c) / ((rb - ri * c) ** 2 + (ri * s) ** 2) ** 1.5
            return mpmath.quad(f, [lo, ri * c, hi])

        # the integrand is even in xi: 2 x the half cell
        v = 2 * mpmath.quad(inner, [0, dphi / 2])
        assert abs(float(v) - ref) < 1e-12 * abs(ref), (float(v), ref)


@pytest.fixture(scope="module")
def table64(oracle_mod):
    return oracle_mod.kernel_cells(64, 64, DU64)


def test_q_symmetries(table64):
    """K^{r,0}, K^{r,r}, K^{phi,phi} even in q; K^{r,phi}, K^{phi,0}, K^{phi,r}
    odd (mirror xi -> -xi of the source cell)."""
    T = table64
    qneg = (-np.arange(64)) % 64
    for c, sgn in ((0, 1), (1, 1), (5, 1), (2, -1), (3, -1), (4, -1)):
        A = T[c]
        B = sgn * A[:, qneg]
        scale = np.abs(T[0]).max(axis=1, keepdims=True) + np.abs(T[3]).max(axis=1, keepdims=True)
        assert np.max(np.abs(A - B) / scale) < 1e-13, c


def _ring_row_sum(du, k, power):
    """int over the source annulus of eta^{1+power} ... : sum_q of the K^{r,*}
    row equals int_a^b eta * Q(1, eta) * (eta - eta_c)^power d eta, with Q the
    ring force (elliptic integrals) at unit target radius."""
    from scipy.integrate import quad

    from oracle.analytic import ring_Q

    beta = math.exp(du)
    ec = beta ** (-k)
    a, b = ec * 2 / (beta + 1), ec * 2 * beta / (beta + 1)
    f = lambda e: float(e * ring_Q(1.0, e)) * (e - ec) ** power
    if a < 1.0 < b:
        # the ring force ~ 1/(eta - 1) near the target's own ring: principal
        # value; the row k = 0 is symmetric about eta = 1, so fold it there
        from oracle.analytic import ring_Q_offset

        h = b - 1.0
        fo = lambda d: float((1.0 + d) * ring_Q_offset(1.0, d)) * (d + 1.0 - ec) ** power
        g = lambda t: fo(t) + fo(-t)
        return quad(g, 0.0, h, limit=400, epsabs=0, epsrel=1e-12)[0]
    return quad(f, a, b, limit=400, epsabs=0, epsrel=1e-13)[0]


@pytest.mark.parametrize("k", [-20, -3, -1, 0, 1, 2, 9, 40])
def test_ring_sum_rule(table64, k):
    """sum_q K^{r,0}[k,q] and sum_q K^{r,r}[k,q] equal the radial force of the
    uniform annulus (self cell included when k = 0); the odd kernels sum to 0."""
    T = table64
    row = k + 64
    for c, power in ((0, 0), (1, 1)):
        s = T[c][row].sum()
        ref = _ring_row_sum(DU64, k, power)
        scale = np.abs(T[c][row]).sum()
        assert abs(s - ref) <= 1e-11 * scale, (c, s, ref)
    for c in (2, 3, 4):
        assert abs(T[c][row].sum()) <= 1e-13 * np.abs(T[c][row]).sum() + 1e-300


def test_far_field_point_mass(table64):
    """Eq. 62: far from the target a cell acts as a point mass at its centre
    (area r_i^2 eta_c (b - a) dphi in the dimensionless variables); the force
    vector's relative error is O(h^2 / d^2)."""
    beta = math.exp(DU64)
    dphi = 2 * math.pi / 64
    errs = []
    for k in (-40, -20, 20, 40):
        ec = beta ** (-k)
        a, b = ec * 2 / (beta + 1), ec * 2 * beta / (beta + 1)
        area = ec * (b - a) * dphi
        for q in (8, 16, 32):
            xi = -q * dphi
            F3 = (ec * ec - 2 * ec * math.cos(xi) + 1) ** 1.5
            pr = -(1 - ec * math.cos(xi)) / F3 * area
            pp = ec * math.sin(xi) / F3 * area
            d = math.sqrt(ec * ec - 2 * ec * math.cos(xi) + 1) / max(ec, 1.0)
            h = max(b - a, ec * dphi) / max(ec, 1.0)
            dr = table64[0][k + 64, q] - pr
            dp = table64[3][k + 64, q] - pp
            errs.append(math.hypot(dr, dp) / math.hypot(pr, pp) / (h / d) ** 2)
    assert max(errs) < 5.0, errs


def _fan_self_cell(du, nphi, n):
    """Sec. 4 (Fig. 1): cover the self cell (unit target radius) with n x n
    Cartesian cells, apply the Cartesian second-order formula (Eq. 9-15 with
    the closed-form kernels of App. A) to sigma = 1, rbar - r_m and
    phibar - phi_m, and return (K^{r,0}_00, r_m K^{r,r}_00, K^{phi,phi}_00)."""
    beta = math.exp(du)
    dphi = 2 * math.pi / nphi
    r_lo, r_hi = 2 / (beta + 1), 2 * beta / (beta + 1)
    rm = 1.0
    x0, x1 = r_lo * math.cos(dphi / 2), r_hi
    y1 = r_hi * math.sin(dphi / 2)
    # put the target at the centre of a Cartesian cell in both directions
    nx = n
    hx = (x1 - x0) / nx
    ix = math.floor((rm - x0) / hx)
    x0 = rm - (ix + 0.5) * hx
    nx = int(math.ceil((x1 - x0) / hx))
    ny = n if n % 2 else n + 1
    hy = 2 * y1 / ny
    xe = x0 + hx * np.arange(nx + 1)
    ye = -y1 + hy * np.arange(ny + 1)
    xc = 0.5 * (xe[:-1] + xe[1:])[:, None]
    yc = 0.5 * (ye[:-1] + ye[1:])[None, :]
    rc = np.sqrt(xc ** 2 + yc ** 2)
    pc = np.arctan2(yc, xc)
    inside = (rc >= r_lo) & (rc <= r_hi) & (np.abs(pc) <= dphi / 2)
    X = [xe[:-1][:, None] - rm, xe[1:][:, None] - rm]
    Y = [ye[:-1][None, :], ye[1:][None, :]]
    rho = lambda a, b: np.sqrt(a * a + b * b)

    def corners(h):
        return h(X[1], Y[1]) - h(X[0], Y[1]) - h(X[1], Y[0]) + h(X[0], Y[0])

    Kx0 = corners(lambda a, b: -np.log(b + rho(a, b)))
    Ky0 = corners(lambda a, b: -np.log(a + rho(a, b)))
    xi_m_xs = rm - xc  # x_i - x_{i'}
    yj_m_ys = 0.0 - yc  # y_j - y_{j'}
    Kxx = xi_m_xs * Kx0 + corners(lambda a, b: b * np.log(a + rho(a, b)))
    Kxy = yj_m_ys * Kx0 + corners(lambda a, b: -rho(a, b))
    Kyy = yj_m_ys * Ky0 + corners(lambda a, b: a * np.log(b + rho(a, b)))
    Kyx = xi_m_xs * Ky0 + corners(lambda a, b: -rho(a, b))
    m = inside.astype(float)
    # (a) sigma = 1
    Fa = np.sum(m * Kx0)
    # (b) sigma = rbar - r_m: value r - r_m, gradient (x/r, y/r)
    Fb = np.sum(m * ((rc - rm) * Kx0 + (xc / rc) * Kxx + (yc / rc) * Kxy))
    # (c) sigma = phibar - phi_m: value phi, gradient (-y/r^2, x/r^2); F^y
    Fc = np.sum(m * (pc * Ky0 + (xc / rc ** 2) * Kyy + (-yc / rc ** 2) * Kyx))
    return Fa, Fb, Fc


def test_fan_method_converges_to_self_cell(oracle_mod):
    """The paper's SIM self-cell construction converges, as the Cartesian
    covering is refined, to the exact self-cell integrals of the oracle.
    (Cartesian cells are in or out by their centre, so the covering's
    boundary error makes the convergence irregular at coarse resolution.)"""
    got = oracle_mod.kernel_cell(DU64, NPHI64, 0, 0)
    ref = np.array([got[0], got[1], got[5]])
    e320 = np.abs(np.array(_fan_self_cell(DU64, NPHI64, 320)) - ref) / np.abs(ref)
    e640 = np.abs(np.array(_fan_self_cell(DU64, NPHI64, 640)) - ref) / np.abs(ref)
    assert np.all(e640 < e320), (e320, e640)
    assert e640[0] < 0.03 and e640[1] < 5e-4 and e640[2] < 5e-4, e640


def test_tolerance_sensitivity(oracle_mod):
    """Tightening the quadrature tolerance moves no kernel by more than the
    looser tolerance times the cell's scale."""
    for k, q in ((0, 0), (0, 1), (1, 0), (5, 7), (-12, 30)):
        a = oracle_mod.kernel_cell(DU64, NPHI64, k, q, rtol=1e-11)
        b = oracle_mod.kernel_cell(DU64, NPHI64, k, q, rtol=1e-14)
        scale = abs(b[0]) + abs(b[3])
        assert np.max(np.abs(a - b)) <= 1e-10 * scale
