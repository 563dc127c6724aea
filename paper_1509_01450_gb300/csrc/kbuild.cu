// kbuild.cu -- FP64 construction of the cell-integrated force kernels
// (run once per grid: by Sec. 2 the kernels depend only on the grid, so
// they are built once and kept).
//
// In the dimensionless variables of Eq. 33, eta = rbar / r_i and
// xi = phibar - phi_j, with F^2 = (eta - cos xi)^2 + sin^2 xi, the six
// kernels of Eq. 30-32 and A11-A13 for the offset (k, q) = (i - i', j - j')
// are integrals over the source cell
//     eta in beta^-k [2/(beta+1), 2 beta/(beta+1)],
//     xi  in [(-q - 1/2) dphi, (-q + 1/2) dphi]
// of
//     -eta (1 - eta cos xi) / F^3          times 1, (eta - beta^-k), (xi + q dphi)
//      eta^2 sin xi / F^3                  times 1, (eta - beta^-k), (xi + q dphi).
//
// k_cells: one warp per offset, q in [0, N_phi/2] (the other half follows
// from the mirror xi -> -xi: K^{r,0}, K^{r,r}, K^{phi,phi} even in q,
// K^{r,phi}, K^{phi,0}, K^{phi,r} odd).  Each rectangle is integrated by the
// 8- and 12-point tensor Gauss-Legendre rules; if they differ by more than
// rtol times the integral of |f_r| + |f_phi| of the same kind (the force
// vector's size) the rectangle is split (a depth-first stack
// in shared memory): in two across its physically longer side when one side
// is more than twice the other, else in four.  Otherwise the 12-point value
// is kept.
//
// k_self_cell: the self cell (k, q) = (0, 0) contains the point eta = 1,
// xi = 0 where the integrand of K^{r,0} behaves like x / rho^3 (x = eta - 1):
// integrable only as a principal value.  The cell is symmetric under
// (x, xi) -> (-x, -xi), so it is integrated in polar coordinates about the
// singular point with the pair sum f(p) + f(-p) written so that the odd
// 1/rho^2 part cancels algebraically: over the square of side 2 min(h, d)
// about the point (one triangle of each opposite pair, composite
// Gauss-Legendre in angle and radius, where rho f is smooth) and over the
// two strips beyond it (geometric panels along the long side).  A coarse
// and a fine rule must agree.  K^{r,phi}, K^{phi,0}, K^{phi,r} vanish on
// the self cell by symmetry (Sec. 3.2.2 and App. A).
//
// The potential (SG_KERNEL_POTENTIAL): k_cells and k_self_cell with the
// integrand -eta / F in place of the radial force's (the slope factors
// (eta - beta^-k) and (xi + q dphi) as for the forces; the azimuthal slots
// zero).  In the own cell's polar rule it behaves like 1 / rho, which the
// rule's rho weight absorbs.
//
// k_point_cells: the particle kinds of sg_kernel_kind (Eq. 35-37 and the
// softened comparison method of Sec. 5.3).  The source centre of offset
// (k, q) sits at eta_c = beta^-k, xi_c = -q' dphi (q' = q taken into
// (-N_phi/2, N_phi/2]); its mass in units of sigma r_i^2 is
// a = eta_c^2 2 tanh(du/2) dphi (A' / r_i^2 of the cell with arithmetic
// centre r_i'), and
//     K^{r,0}   <- -a (1 - eta_c cos xi_c) / D^3,
//     K^{phi,0} <-  a eta_c sin xi_c / D^3,
//     D^2 = (1 - eta_c)^2 + 4 eta_c sin^2(xi_c / 2)  (+ s^2 softened),
// with 1 - eta_c = -expm1(-k du) and 1 - cos xi = 2 sin^2(xi / 2), so the
// neighbouring cells lose no digits.  The four slope cells are zero; the own
// cell (0, 0) is zero for the particle kinds (k_self_cell then writes the
// exact own-cell values for the modified method) and has D = s, with both
// numerators zero, when softened.
//
// k_cells_tpz: the trapezoidal form of the cell integrals (Eq. 41-43 for
// K^{r,0}, K^{r,r}, K^{r,phi}; the same rule for K^{phi,phi}, App. A), which
// the paper's SIM uses with N_tpz = 19: at the N_tpz + 1 equally spaced
// azimuths xi - xi_c = -dphi/2 + m dphi / N_tpz of the source cell the
// eta-integrals are taken exactly (adaptively: 8- and 12-point
// Gauss-Legendre per panel, bisected until they agree, with a breakpoint at
// eta = cos xi where the integrand peaks) and combined by the trapezoidal
// rule.  K^{phi,0}, K^{phi,r} (exact in the paper too) and the own cell
// (Sec. 4) keep the values of k_cells and k_self_cell.
//
// k_fold: the slope terms of Eq. 28-29 / A9-A10 with central differences
// fold into one kernel per component:
//   K^eff[k,q] = K^{.,0}[k,q] + (beta^{k+1} K^{.,r}[k+1,q]
//                - beta^{k-1} K^{.,r}[k-1,q]) / (beta - 1/beta)
//                + (K^{.,phi}[k,q+1] - K^{.,phi}[k,q-1]) / (2 dphi),
// then the weighted, normalised kernel G beta^{p k} K^eff / (L N_phi) is
// placed cyclically at row k mod L (L = 2 N_u, row N_u left zero).
//
// k_cart_fold: the Cartesian scheme of Sec. 3.1.1 (SG_KERNEL_CARTESIAN) on
// square cells of side h = du.  The six cell integrals of Eq. 13-15 and
// their y forms have the closed forms of App. A: double differences over
// the source cell's corners (X, Y relative to the target centre) of
// -ln(Y + R), -ln(X + R), Y ln(X + R), X ln(Y + R) and -R, R = |(X, Y)|,
// plus k h or q h times the zeroth kernel.  They fold with central slopes
// (beta = 1):
//   K^eff[k,q] = K^{.,0} + (K^{.,x}[k+1] - K^{.,x}[k-1]) / 2h
//                        + (K^{.,y}[q+1] - K^{.,y}[q-1]) / 2h,
// evaluated directly at every true offset, so the table needs no ring in
// q.  Row k lands at k mod 2 N_x as for the polar grid; offset q at
// q mod N_phi for |q| < N_phi / 2, with column N_phi / 2 left zero: sigma
// zero in its last N_phi / 2 columns then makes the periodic transform in
// the second direction a linear convolution over the first N_phi / 2.
#include <math.h>
#include <stdio.h>

#include "sg_internal.cuh"

namespace sg {

__constant__ double c_x8[8], c_w8[8], c_x12[12], c_w12[12], c_x16[16], c_w16[16];

// Gauss-Legendre nodes and weights on [-1, 1]: Newton iteration on the
// three-term recurrence of P_n from the asymptotic first guess.
void gauss_legendre(int n, double* x, double* w)
{
    for (int k = 1; k <= n; k++) {
        double z = (1.0 - 1.0 / (8.0 * n * n) + 1.0 / (8.0 * n * n * n)) * cos(M_PI * (4.0 * k - 1.0) / (4.0 * n + 2.0));
        double dp = 0.0;
        for (int it = 0; it < 50; it++) {
            double p0 = 1.0, p1 = z;
            for (int j = 2; j <= n; j++) {
                double p2 = ((2 * j - 1) * z * p1 - (j - 1) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (p0 - z * p1) / (1.0 - z * z);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) <= 1e-16 * fabs(z) + 1e-300) break;
        }
        double p0 = 1.0, p1 = z;
        for (int j = 2; j <= n; j++) {
            double p2 = ((2 * j - 1) * z * p1 - (j - 1) * p0) / j;
            p0 = p1;
            p1 = p2;
        }
        dp = n * (p0 - z * p1) / (1.0 - z * z);
        x[k - 1] = z;
        w[k - 1] = 2.0 / ((1.0 - z * z) * dp * dp);
    }
}

static cudaError_t upload_rules()
{
    static int done_dev = -1;
    int dev;
    cudaGetDevice(&dev);
    if (done_dev == dev) return cudaSuccess;
    double x[32], w[32];
    cudaError_t e;
    gauss_legendre(8, x, w);
    if ((e = cudaMemcpyToSymbol(c_x8, x, 8 * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_w8, w, 8 * sizeof(double))) != cudaSuccess) return e;
    gauss_legendre(12, x, w);
    if ((e = cudaMemcpyToSymbol(c_x12, x, 12 * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_w12, w, 12 * sizeof(double))) != cudaSuccess) return e;
    gauss_legendre(16, x, w);
    if ((e = cudaMemcpyToSymbol(c_x16, x, 16 * sizeof(double))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(c_w16, w, 16 * sizeof(double))) != cudaSuccess) return e;
    done_dev = dev;
    return cudaSuccess;
}

// the six integrands at eta = eta_c + del and xi = xi_c + dp (dp is the
// azimuth measured from the source-cell centre, the factor of K^{.,phi}),
// accumulated with weight w; c, s = cos xi, sin xi.  em1 = eta_c - 1 (exact
// for k = 0).  eta - 1, eta - cos xi and
// 1 - eta cos xi are formed from 1 - cos xi = sin^2 xi / (1 + cos xi)
// (or 1 - cos xi directly when cos xi <= 0) and eta - 1 = em1 + del, so they
// keep full relative precision near the singular point eta = 1, xi = 0.
__device__ __forceinline__ void acc6(double del, double eta_c, double em1, double dp, double c, double s, double w,
                                     double* I, double* A, int pot = 0)
{
    const double vc = c > 0.0 ? s * s / (1.0 + c) : 1.0 - c;  // 1 - cos xi
    const double e1 = em1 + del;                               // eta - 1
    const double eta = eta_c + del;
    const double d = e1 + vc;                                  // eta - cos xi
    const double om = vc - e1 * c;                             // 1 - eta cos xi
    const double F2 = d * d + s * s;
    const double iF = 1.0 / sqrt(F2);
    const double iF3 = iF * iF * iF;
    // pot: the potential's integrand -eta / F in the first three slots
    const double ir0 = pot ? -eta * iF : -eta * om * iF3;
    const double ip0 = pot ? 0.0 : eta * eta * s * iF3;
    const double v[6] = {ir0, ir0 * del, ir0 * dp, ip0, ip0 * del, ip0 * dp};
#pragma unroll
    for (int c6 = 0; c6 < 6; c6++) {
        I[c6] += w * v[c6];
        if (A) A[c6] += w * fabs(v[c6]);
    }
}

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

#define SG_STACK 64
#define SG_MAXRECT 20000

// The six integrals over one source cell, (eta - eta_c, xi - xi_c) in
// [-hw, hw] x [-dphi/2, dphi/2] (sc, cc = sin, cos xi_c; em1 = eta_c - 1),
// by one warp: 8- and 12-point Gauss-Legendre products per rectangle,
// bisected until they agree.  Returns 1 if the rectangle budget ran out.
__device__ int cell_quad(double eta_c, double em1, double hw, double sc, double cc, double dphi, double rtol, int pot,
                         double4_16a* stack, int lane, double res[6])
{
    int sp = 0, nrect = 0, bad = 0;
#pragma unroll
    for (int c6 = 0; c6 < 6; c6++) res[c6] = 0.0;
    // rectangles in (eta - eta_c, xi - xi_c)
    stack[0] = make_double4_16a(-hw, hw, -0.5 * dphi, 0.5 * dphi);
    sp = 1;
    while (sp > 0) {
        __syncwarp();
        const double4_16a R = stack[--sp];
        __syncwarp();
        nrect++;
        const double he = 0.5 * (R.y - R.x), me = 0.5 * (R.y + R.x);
        const double hx = 0.5 * (R.w - R.z), mx = 0.5 * (R.w + R.z);
        double I8[6] = {0, 0, 0, 0, 0, 0}, I12[6] = {0, 0, 0, 0, 0, 0}, A12[6] = {0, 0, 0, 0, 0, 0};
        for (int p = lane; p < 64; p += 32) {
            const int a = p >> 3, b = p & 7;
            const double del = me + he * c_x8[a], t = mx + hx * c_x8[b];
            double st, ct;
            sincos(t, &st, &ct);
            acc6(del, eta_c, em1, t, ct * cc - st * sc, st * cc + ct * sc, he * hx * c_w8[a] * c_w8[b], I8,
                 nullptr, pot);
        }
        for (int p = lane; p < 144; p += 32) {
            const int a = p / 12, b = p % 12;
            const double del = me + he * c_x12[a], t = mx + hx * c_x12[b];
            double st, ct;
            sincos(t, &st, &ct);
            acc6(del, eta_c, em1, t, ct * cc - st * sc, st * cc + ct * sc, he * hx * c_w12[a] * c_w12[b], I12,
                 A12, pot);
        }
        bool ok = true;
#pragma unroll
        for (int c6 = 0; c6 < 6; c6++) {
            I8[c6] = warp_sum(I8[c6]);
            I12[c6] = warp_sum(I12[c6]);
            A12[c6] = warp_sum(A12[c6]);
        }
#pragma unroll
        for (int c6 = 0; c6 < 6; c6++) {
            // the radial and azimuthal kernels of each kind form one force
            // vector: measure both against its size (so a component that
            // nearly vanishes, on the curve eta cos xi = 1, needs no more
            // than the vector's precision), plus the rounding level of a
            // 144-term sum
            const double scale = A12[c6] + A12[(c6 + 3) % 6];
            if (fabs(I12[c6] - I8[c6]) > (rtol + 64.0 * 2.220446049250313e-16) * scale) ok = false;
        }
        if (!ok && (sp + 4 > SG_STACK || nrect >= SG_MAXRECT)) {
            ok = true;
            bad = 1;
        }
        if (ok) {
#pragma unroll
            for (int c6 = 0; c6 < 6; c6++) res[c6] += I12[c6];
        } else {
            // split the side that is longer in physical length (the
            // azimuthal side measures (xi extent) x eta); both when the
            // rectangle is roughly square
            const double le = R.y - R.x, lx = (R.w - R.z) * (eta_c + me);
            __syncwarp();
            if (le > 2.0 * lx) {
                if (lane == 0) {
                    stack[sp + 0] = make_double4_16a(R.x, me, R.z, R.w);
                    stack[sp + 1] = make_double4_16a(me, R.y, R.z, R.w);
                }
                sp += 2;
            } else if (lx > 2.0 * le) {
                if (lane == 0) {
                    stack[sp + 0] = make_double4_16a(R.x, R.y, R.z, mx);
                    stack[sp + 1] = make_double4_16a(R.x, R.y, mx, R.w);
                }
                sp += 2;
            } else {
                if (lane == 0) {
                    stack[sp + 0] = make_double4_16a(R.x, me, R.z, mx);
                    stack[sp + 1] = make_double4_16a(me, R.y, R.z, mx);
                    stack[sp + 2] = make_double4_16a(R.x, me, mx, R.w);
                    stack[sp + 3] = make_double4_16a(me, R.y, mx, R.w);
                }
                sp += 4;
            }
        }
    }
    return bad;
}

__global__ void __launch_bounds__(128) k_cells(int nu, int nphi, double du, double rtol, double* __restrict__ cells,
                                               int* __restrict__ flag, int pot)
{
    __shared__ double4_16a stack_all[4][SG_STACK];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double4_16a* stack = stack_all[wib];
    const double beta = exp(du), dphi = 2.0 * M_PI / nphi;
    const int nq = nphi / 2 + 1;
    const long noff = (long)(2 * nu + 1) * nq;
    const long per = (long)(2 * nu + 1) * nphi;
    const long wstride = (long)gridDim.x * 4;
    for (long off = (long)blockIdx.x * 4 + wib; off < noff; off += wstride) {
        const int k = (int)(off / nq) - nu;
        const int q = (int)(off % nq);
        if (k == 0 && q == 0) continue;  // self cell: k_self_cell
        const double eta_c = exp(-du * k), em1 = expm1(-du * k);
        const double hw = eta_c * tanh(0.5 * du);  // half width in eta, (beta - 1)/(beta + 1) exactly
        // centre azimuth xi_c = -q dphi = -2 pi q / N_phi, its sine and cosine
        // exact at the quarter points
        double sc, cc;
        sincospi(-2.0 * q / nphi, &sc, &cc);
        double res[6];
        const int bad = cell_quad(eta_c, em1, hw, sc, cc, dphi, rtol, pot, stack, lane, res);
        if (lane == 0) {
            const long row = (long)(k + nu) * nphi;
            const int qm = (nphi - q) & (nphi - 1);
#pragma unroll
            for (int c6 = 0; c6 < 6; c6++) {
                cells[c6 * per + row + q] = res[c6];
                const bool odd = (c6 == 2 || c6 == 3 || c6 == 4);
                if (qm != q) cells[c6 * per + row + qm] = odd ? -res[c6] : res[c6];
            }
            if (bad) {
                atomicOr(flag, 1);
                atomicAdd(flag + 1, 1);
                atomicExch(flag + 2, k);
                atomicExch(flag + 3, q);
            }
        }
    }
}

// eta-integrals of the six integrands over the source cell (del = eta -
// eta_c in [-hw, hw]) at one azimuth xi = xi_c + t (c, s = cos xi, sin xi);
// returns 1 if a panel could not meet the tolerance.
#define SG_TSTACK 48
#define SG_TMAXPAN 4000
__device__ int eta_integral(double eta_c, double em1, double hw, double t, double c, double s, double rtol, double* I)
{
    double2 stk[SG_TSTACK];
    int sp = 0, npan = 0, bad = 0;
#pragma unroll
    for (int c6 = 0; c6 < 6; c6++) I[c6] = 0.0;
    const double vc = c > 0.0 ? s * s / (1.0 + c) : 1.0 - c;
    const double peak = -vc - em1;  // del of eta = cos xi
    if (peak > -hw && peak < hw) {
        stk[sp++] = make_double2(peak, hw);
        stk[sp++] = make_double2(-hw, peak);
    } else {
        stk[sp++] = make_double2(-hw, hw);
    }
    while (sp > 0) {
        const double2 P = stk[--sp];
        const double h = 0.5 * (P.y - P.x), mid = 0.5 * (P.x + P.y);
        double I8[6] = {0, 0, 0, 0, 0, 0}, I12[6] = {0, 0, 0, 0, 0, 0}, A12[6] = {0, 0, 0, 0, 0, 0};
        for (int a = 0; a < 8; a++) acc6(mid + h * c_x8[a], eta_c, em1, t, c, s, h * c_w8[a], I8, nullptr);
        for (int a = 0; a < 12; a++) acc6(mid + h * c_x12[a], eta_c, em1, t, c, s, h * c_w12[a], I12, A12);
        bool ok = true;
#pragma unroll
        for (int c6 = 0; c6 < 6; c6++) {
            const double scale = A12[c6] + A12[(c6 + 3) % 6];  // the force vector's size, as in k_cells
            if (fabs(I12[c6] - I8[c6]) > (rtol + 64.0 * 2.220446049250313e-16) * scale) ok = false;
        }
        if (!ok && (sp + 2 > SG_TSTACK || ++npan > SG_TMAXPAN)) {
            ok = true;
            bad = 1;
        }
        if (ok) {
#pragma unroll
            for (int c6 = 0; c6 < 6; c6++) I[c6] += I12[c6];
        } else {
            stk[sp++] = make_double2(mid, P.y);
            stk[sp++] = make_double2(P.x, mid);
        }
    }
    return bad;
}

// One warp per offset (q in [0, N_phi/2], the rest by the mirror xi -> -xi),
// one lane per azimuth node.
__global__ void __launch_bounds__(128) k_cells_tpz(int nu, int nphi, double du, int ntpz, double rtol,
                                                   double* __restrict__ cells, int* __restrict__ flag)
{
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    const double dphi = 2.0 * M_PI / nphi, dth = dphi / ntpz;
    const int nq = nphi / 2 + 1;
    const long noff = (long)(2 * nu + 1) * nq;
    const long per = (long)(2 * nu + 1) * nphi;
    const long wstride = (long)gridDim.x * 4;
    for (long off = (long)blockIdx.x * 4 + wib; off < noff; off += wstride) {
        const int k = (int)(off / nq) - nu;
        const int q = (int)(off % nq);
        if (k == 0 && q == 0) continue;  // own cell: exact (k_self_cell)
        const double eta_c = exp(-du * k), em1 = expm1(-du * k);
        const double hw = eta_c * tanh(0.5 * du);
        double sc, cc;
        sincospi(-2.0 * q / nphi, &sc, &cc);
        double acc[4] = {0, 0, 0, 0};
        int bad = 0;
        for (int m = lane; m <= ntpz; m += 32) {
            const double t = m == ntpz ? 0.5 * dphi : -0.5 * dphi + m * dth;
            double st, ct;
            sincos(t, &st, &ct);
            double I[6];
            bad |= eta_integral(eta_c, em1, hw, t, ct * cc - st * sc, st * cc + ct * sc, rtol, I);
            const double w = (m == 0 || m == ntpz) ? 0.5 * dth : dth;
            acc[0] += w * I[0];  // K^{r,0}
            acc[1] += w * I[1];  // K^{r,r}
            acc[2] += w * I[2];  // K^{r,phi}
            acc[3] += w * I[5];  // K^{phi,phi}
        }
#pragma unroll
        for (int c4 = 0; c4 < 4; c4++) acc[c4] = warp_sum(acc[c4]);
        bad = __any_sync(0xffffffffu, bad);
        if (lane == 0) {
            const long row = (long)(k + nu) * nphi;
            const int qm = (nphi - q) & (nphi - 1);
            const int comp[4] = {0, 1, 2, 5};
#pragma unroll
            for (int c4 = 0; c4 < 4; c4++) {
                cells[comp[c4] * per + row + q] = acc[c4];
                if (qm != q) cells[comp[c4] * per + row + qm] = comp[c4] == 2 ? -acc[c4] : acc[c4];
            }
            if (bad) {
                atomicOr(flag, 1);
                atomicAdd(flag + 1, 1);
                atomicExch(flag + 2, k);
                atomicExch(flag + 3, q);
            }
        }
    }
}

// The self-cell integrands of K^{r,0}, K^{r,r}, K^{phi,phi} summed over the
// point pair p = (x, y) and -p (x = eta - 1, y = xi), written so that the
// odd 1/rho^2 parts cancel algebraically rather than in rounding.  With
// vc = 1 - cos y, F_+-^2 = (x +- vc)^2 + sin^2 y, A = (F_+^2 + F_-^2)/2,
// B = 2 x vc, N_+- = (1 +- x)(vc -+ x cos y):
//   f(p) + f(-p) = -2 (Ns Gs + Nd Gd),  f(p) - f(-p) = -2 (Ns Gd + Nd Gs),
// Ns = vc - x^2 cos y, Nd = -x (1 - 2 vc), Gs = (F_+^-3 + F_-^-3) / 2 and
// Gd = (F_+^-3 - F_-^-3) / 2 = -B (3 A^2 + B^2) / ((F_+^3 + F_-^3) F_+^3 F_-^3).
__device__ __forceinline__ void self_pair(double x, double y, double* v, int pot)
{
    const double s = sin(y), sh = sin(0.5 * y);
    const double vc = 2.0 * sh * sh;
    const double c = 1.0 - vc;
    const double P = (x + vc) * (x + vc) + s * s;
    const double M = (x - vc) * (x - vc) + s * s;
    if (pot) {  // the potential: -eta / F at p and -p (both ~ 1/rho: the polar rule absorbs it)
        const double a = (1.0 + x) / sqrt(P), b = (1.0 - x) / sqrt(M);
        v[0] = -(a + b);      // K^{P,0}
        v[1] = -x * (a - b);  // K^{P,r}: (eta - 1) = x at p, -x at -p
        v[2] = 0.0;           // K^{P,phi}: odd in y, zero over the cell
        return;
    }
    const double Fp3 = P * sqrt(P), Fm3 = M * sqrt(M);
    const double A = 0.5 * (P + M), B = 2.0 * x * vc;
    const double Gs = 0.5 * (1.0 / Fp3 + 1.0 / Fm3);
    const double Gd = -B * (3.0 * A * A + B * B) / ((Fp3 + Fm3) * Fp3 * Fm3);
    const double Ns = vc - x * x * c, Nd = -x * (1.0 - 2.0 * vc);
    v[0] = -2.0 * (Ns * Gs + Nd * Gd);                                   // K^{r,0}
    v[1] = x * (-2.0 * (Ns * Gd + Nd * Gs));                             // K^{r,r}: x (f(p) - f(-p))
    v[2] = s * y * ((1.0 + x) * (1.0 + x) / Fp3 + (1.0 - x) * (1.0 - x) / Fm3);  // K^{phi,phi}
}

// block-wide sum of three doubles; the result is valid in every thread
__device__ void block_sum3(double* acc, double* out)
{
    __shared__ double red[3][32];
#pragma unroll
    for (int c3 = 0; c3 < 3; c3++) {
        double v = warp_sum(acc[c3]);
        if ((threadIdx.x & 31) == 0) red[c3][threadIdx.x >> 5] = v;
    }
    __syncthreads();
    for (int c3 = 0; c3 < 3; c3++) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) t += red[c3][w];
        out[c3] = t;
    }
    __syncthreads();
}

// Square [-m, m]^2 about the singular point, in polar coordinates: one
// triangle of each opposite pair (rays to x = m for |theta| < pi/4, to
// y = m for pi/4 < theta < 3 pi/4), np x np composite 16-point panels in
// (angle, radius), integrand self_pair.
__device__ void self_square(double m, int np, double* out, int pot)
{
    const double thc = 0.25 * M_PI;
    double acc[3] = {0, 0, 0};
    const int per_reg = np * np * 256;
    for (int p = threadIdx.x; p < 2 * per_reg; p += blockDim.x) {
        const int reg = p / per_reg, rem = p % per_reg;
        const int pan = rem >> 8, node = rem & 255;
        const int pt = pan / np, pr = pan % np, a = node >> 4, b = node & 15;
        const double t0 = (reg == 0 ? -thc : thc) + 2.0 * thc * pt / np;
        const double t1 = (reg == 0 ? -thc : thc) + 2.0 * thc * (pt + 1) / np;
        const double th = 0.5 * (t0 + t1) + 0.5 * (t1 - t0) * c_x16[a];
        const double thw = 0.5 * (t1 - t0) * c_w16[a];
        double ct, st;
        sincos(th, &st, &ct);
        const double rmax = reg == 0 ? m / ct : m / st;
        const double u0 = (double)pr / np, u1 = (double)(pr + 1) / np;
        const double tau = 0.5 * (u0 + u1) + 0.5 * (u1 - u0) * c_x16[b];
        const double rho = rmax * tau;
        const double w = thw * 0.5 * (u1 - u0) * c_w16[b] * rmax * rmax * tau;
        double v[3];
        self_pair(rho * ct, rho * st, v, pot);
#pragma unroll
        for (int c3 = 0; c3 < 3; c3++) acc[c3] += w * v[c3];
    }
    block_sum3(acc, out);
}

// Strip at distance >= m from the singular point: the long coordinate runs
// over [m, L] in geometric panels (ratio), the short one over [-w, w] in
// nshort panels; radial = 1 means the long coordinate is x = eta - 1.
// (Its point reflection is the opposite strip, which self_pair includes.)
__device__ void self_strip(double m, double L, double w, double ratio, int nshort, int radial, double* out, int pot)
{
    double acc[3] = {0, 0, 0};
    double a = m;
    while (a < L) {  // uniform across the block: same arithmetic in every thread
        double b = fmin(a * ratio, L);
        if (L - b < 0.25 * (b - a)) b = L;
        for (int p = threadIdx.x; p < nshort * 256; p += blockDim.x) {
            const int j = p >> 8, node = p & 255, ia = node >> 4, ib = node & 15;
            const double s0 = -w + 2.0 * w * j / nshort, s1 = -w + 2.0 * w * (j + 1) / nshort;
            const double l = 0.5 * (a + b) + 0.5 * (b - a) * c_x16[ia];
            const double sh = 0.5 * (s0 + s1) + 0.5 * (s1 - s0) * c_x16[ib];
            const double wt = 0.5 * (b - a) * c_w16[ia] * 0.5 * (s1 - s0) * c_w16[ib];
            double v[3];
            if (radial)
                self_pair(l, sh, v, pot);
            else
                self_pair(sh, l, v, pot);
#pragma unroll
            for (int c3 = 0; c3 < 3; c3++) acc[c3] += wt * v[c3];
        }
        a = b;
    }
    block_sum3(acc, out);
}

// The self cell [-h, h] x [-d, d] (x = eta - 1, y = xi) as the square of
// side 2 min(h, d) about the singular point plus the two strips beyond it,
// at a coarse and a fine resolution; the fine value is kept and the two
// must agree.
__device__ void self_cell_rule(double h, double d, int fine, double* out, int pot)
{
    const double m = fmin(h, d);
    double sq[3], st[3] = {0, 0, 0};
    self_square(m, fine ? 8 : 4, sq, pot);
    const double ratio = fine ? 1.4142135623730951 : 2.0;
    const int ns = fine ? 8 : 4;
    if (h > m) self_strip(m, h, d, ratio, ns, 1, st, pot);
    if (d > m) self_strip(m, d, h, ratio, ns, 0, st, pot);
    for (int c3 = 0; c3 < 3; c3++) out[c3] = sq[c3] + st[c3];
}

__global__ void __launch_bounds__(256) k_self_cell(int nu, int nphi, double du, double rtol,
                                                   double* __restrict__ cells, int* __restrict__ flag, int pot)
{
    const double dphi = 2.0 * M_PI / nphi;
    const double h = tanh(0.5 * du), d = 0.5 * dphi;  // (beta - 1)/(beta + 1) without cancellation
    double coarse[3], fine[3];
    self_cell_rule(h, d, 0, coarse, pot);
    self_cell_rule(h, d, 1, fine, pot);
    if (threadIdx.x == 0) {
        const long per = (long)(2 * nu + 1) * nphi;
        const long at = (long)nu * nphi;  // k = 0, q = 0
        cells[0 * per + at] = fine[0];
        cells[1 * per + at] = fine[1];
        cells[2 * per + at] = 0.0;
        cells[3 * per + at] = 0.0;
        cells[4 * per + at] = 0.0;
        cells[5 * per + at] = fine[2];
        bool conv = true;
        for (int c3 = 0; c3 < 3; c3++)
            if (fabs(fine[c3] - coarse[c3]) > fmax(rtol, 1e-14) * fabs(fine[c3])) conv = false;
        if (!conv) atomicOr(flag, 2);
    }
}

__global__ void k_point_cells(int nu, int nphi, double du, int kind, double s, double* __restrict__ cells)
{
    const long per = (long)(2 * nu + 1) * nphi;
    const double a0 = 2.0 * tanh(0.5 * du) * (2.0 * M_PI / nphi);
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < per; idx += (long)gridDim.x * blockDim.x) {
        const int k = (int)(idx / nphi) - nu, q = (int)(idx % nphi);
        const int qr = q <= nphi / 2 ? q : q - nphi;
        double sx, cx, sh, ch;
        sincospi(-2.0 * qr / nphi, &sx, &cx);  // xi_c
        sincospi(-1.0 * qr / nphi, &sh, &ch);  // xi_c / 2
        const double eta = exp(-k * du), om = -expm1(-k * du);
        double D2 = om * om + 4.0 * eta * sh * sh;
        if (kind == SG_KERNEL_SOFTENED) D2 += s * s;
        double kr = 0.0, kp = 0.0;
        if (kind == SG_KERNEL_SOFTENED || k != 0 || q != 0) {
            const double a = eta * eta * a0, inv = 1.0 / (D2 * sqrt(D2));
            kr = -a * (om + 2.0 * eta * sh * sh) * inv;
            kp = a * eta * sx * inv;
        }
        cells[idx] = kr;
        cells[per + idx] = 0.0;
        cells[2 * per + idx] = 0.0;
        cells[3 * per + idx] = kp;
        cells[4 * per + idx] = 0.0;
        cells[5 * per + idx] = 0.0;
    }
}

__global__ void k_fold(int nu, int nphi, double du, double G, int p, const double* __restrict__ cells,
                       double* __restrict__ keff, double* __restrict__ nsr, double* __restrict__ nsp)
{
    const int L = 2 * nu;
    const long total = (long)L * nphi;
    const long per = (long)(2 * nu + 1) * nphi;
    const long perk = (long)(2 * nu - 1) * nphi;
    const double bb = 2.0 * sinh(du), dphi = 2.0 * M_PI / nphi;  // beta - 1/beta without cancellation
    const double norm = G / ((double)L * nphi);
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int kk = (int)(idx / nphi), q = (int)(idx % nphi);
        if (kk == nu) {
            nsr[idx] = 0.0;
            nsp[idx] = 0.0;
            continue;
        }
        const int k = kk < nu ? kk : kk - L;
        const int qp = (q + 1) & (nphi - 1), qm = (q - 1) & (nphi - 1);
        const double* C0 = cells + 0 * per;
        const double* C1 = cells + 1 * per;
        const double* C2 = cells + 2 * per;
        const double* C3 = cells + 3 * per;
        const double* C4 = cells + 4 * per;
        const double* C5 = cells + 5 * per;
        const long rk = (long)(k + nu) * nphi, ru = rk + nphi, rd = rk - nphi;
        const double bu = exp((k + 1) * du), bd = exp((k - 1) * du);
        const double Kr = C0[rk + q] + (bu * C1[ru + q] - bd * C1[rd + q]) / bb + (C2[rk + qp] - C2[rk + qm]) / (2.0 * dphi);
        const double Kp = C3[rk + q] + (bu * C4[ru + q] - bd * C4[rd + q]) / bb + (C5[rk + qp] - C5[rk + qm]) / (2.0 * dphi);
        keff[(long)(k + nu - 1) * nphi + q] = Kr;
        keff[perk + (long)(k + nu - 1) * nphi + q] = Kp;
        const double sc = norm * exp(p * k * du);
        nsr[idx] = Kr * sc;
        nsp[idx] = Kp * sc;
    }
}

cudaError_t launch_cells(int nu, int nphi, double du, double rtol, double* cells, int* flag, cudaStream_t st, int pot)
{
    cudaError_t e = upload_rules();
    if (e != cudaSuccess) return e;
    int dev, nsm;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long noff = (long)(2 * nu + 1) * (nphi / 2 + 1);
    long blocks = (noff + 3) / 4;
    const long cap = (long)nsm * 32;
    if (blocks > cap) blocks = cap;
    k_cells<<<(int)blocks, 128, 0, st>>>(nu, nphi, du, rtol, cells, flag, pot);
    k_self_cell<<<1, 256, 0, st>>>(nu, nphi, du, rtol, cells, flag, pot);
    return cudaGetLastError();
}

// k_edge_spec: the phi-spectra of the radial slope kernels for the
// one-sided edge slopes.  For k in [-N_u, N_u] and mode m in [0, N_phi/2]
// (rows of sg_edge_stride elements):
//   gr[m][k + N_u] = G beta^k / N_phi  sum_q K^{r,r}[k, q]   cos(2 pi m q / N_phi),
//   gp[m][k + N_u] = G beta^k / N_phi  sum_q K^{phi,r}[k, q] sin(2 pi m q / N_phi),
// the forward phi-DFTs of the two kernels being gr and -i gp (K^{r,r} is even
// in q, K^{phi,r} odd).  FP64 sums over q in [0, N_phi/2] with the mirror
// folded in; cosines and sines from the FP64 twiddle table.  One block per
// k, one thread per mode.
template <typename T>
__global__ void k_edge_spec(int nu, int nphi, double du, double G, const double* __restrict__ cells,
                            const double2* __restrict__ tw64, T* __restrict__ gr, T* __restrict__ gp)
{
    const int kk = blockIdx.x, k = kk - nu, half = nphi / 2;
    const long per = (long)(2 * nu + 1) * nphi;
    const double* K1 = cells + 1 * per + (long)kk * nphi;  // K^{r,r}[k, .]
    const double* K4 = cells + 4 * per + (long)kk * nphi;  // K^{phi,r}[k, .]
    const int stride = SG_NMAX / nphi;
    const double sc = G * exp(k * du) / nphi;
    const int ks = sg_edge_stride(nu, sizeof(T));
    for (int m = threadIdx.x; m <= half; m += blockDim.x) {
        double c = K1[0] + ((m & 1) ? -K1[half] : K1[half]), s = 0.0;
        for (int q = 1; q < half; q++) {
            const double2 w = tw64[(long)((m * q) & (nphi - 1)) * stride];  // e^{-2 pi i m q / N_phi}
            c += 2.0 * K1[q] * w.x;
            s -= 2.0 * K4[q] * w.y;
        }
        gr[(long)m * ks + kk] = (T)(sc * c);
        gp[(long)m * ks + kk] = (T)(sc * s);
    }
}

template <typename T>
cudaError_t launch_edge_spectra(int nu, int nphi, double du, double G, const double* cells, const void* tw64, T* gr,
                                T* gp, cudaStream_t st)
{
    k_edge_spec<T><<<2 * nu + 1, 256, 0, st>>>(nu, nphi, du, G, cells, (const double2*)tw64, gr, gp);
    return cudaGetLastError();
}
template cudaError_t launch_edge_spectra<float>(int, int, double, double, const double*, const void*, float*, float*,
                                                cudaStream_t);
template cudaError_t launch_edge_spectra<double>(int, int, double, double, const double*, const void*, double*,
                                                 double*, cudaStream_t);
template cudaError_t launch_edge_spectra<dfloat>(int, int, double, double, const double*, const void*, dfloat*,
                                                  dfloat*, cudaStream_t);

cudaError_t launch_cells_tpz(int nu, int nphi, double du, int ntpz, double rtol, double* cells, int* flag,
                             cudaStream_t st)
{
    int dev, nsm;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long noff = (long)(2 * nu + 1) * (nphi / 2 + 1);
    long blocks = (noff + 3) / 4;
    const long cap = (long)nsm * 32;
    if (blocks > cap) blocks = cap;
    k_cells_tpz<<<(int)blocks, 128, 0, st>>>(nu, nphi, du, ntpz, rtol, cells, flag);
    return cudaGetLastError();
}

cudaError_t launch_point_cells(int nu, int nphi, double du, int kind, double soften, double rtol, double* cells,
                               int* flag, cudaStream_t st)
{
    const long per = (long)(2 * nu + 1) * nphi;
    long blocks = (per + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    k_point_cells<<<(int)blocks, 256, 0, st>>>(nu, nphi, du, kind, soften, cells);
    if (kind == SG_KERNEL_PARTICLE_PLUS) {
        cudaError_t e = upload_rules();  // the own cell's Gauss-Legendre rules
        if (e != cudaSuccess) return e;
        k_self_cell<<<1, 256, 0, st>>>(nu, nphi, du, rtol, cells, flag, 0);
    }
    return cudaGetLastError();
}

// k_wedge_cells: the origin wedge [0, r_in] x [phi_{j'-1/2}, phi_{j'+1/2}]
// below the grid (Sec. 3.2.1; the kernels K-bar of the third terms of
// Eq. 27-29) seen from the centre of grid row i: the six integrals of k_cells
// over eta in [0, eta_w], eta_w = r_in / r_i = 2 / (beta^i (1 + beta)), the
// slope factors measured from the wedge centre eta_w / 2 (the mean of its
// faces 0 and r_in).  The wedge lies inside every target radius, so no
// integrand is singular.  Table [6][N_u][N_phi], mirrored in q as k_cells.
__global__ void __launch_bounds__(128) k_wedge_cells(int nu, int nphi, double du, double rtol, int pot,
                                                     double* __restrict__ wcells, int* __restrict__ flag)
{
    __shared__ double4_16a stack_all[4][SG_STACK];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    double4_16a* stack = stack_all[wib];
    const double beta = exp(du), dphi = 2.0 * M_PI / nphi;
    const int nq = nphi / 2 + 1;
    const long noff = (long)nu * nq, per = (long)nu * nphi;
    for (long off = (long)blockIdx.x * 4 + wib; off < noff; off += (long)gridDim.x * 4) {
        const int i = (int)(off / nq), q = (int)(off % nq);
        const double eta_w = 2.0 / (exp(du * i) * (1.0 + beta)), eta_c = 0.5 * eta_w;
        double sc, cc;
        sincospi(-2.0 * q / nphi, &sc, &cc);
        double res[6];
        const int bad = cell_quad(eta_c, eta_c - 1.0, eta_c, sc, cc, dphi, rtol, pot, stack, lane, res);
        if (lane == 0) {
            const long row = (long)i * nphi;
            const int qm = (nphi - q) & (nphi - 1);
#pragma unroll
            for (int c6 = 0; c6 < 6; c6++) {
                wcells[c6 * per + row + q] = res[c6];
                const bool odd = (c6 == 2 || c6 == 3 || c6 == 4);
                if (qm != q) wcells[c6 * per + row + qm] = odd ? -res[c6] : res[c6];
            }
            if (bad) {
                atomicOr(flag, 4);
                atomicAdd(flag + 1, 1);
                atomicExch(flag + 2, i);
                atomicExch(flag + 3, q);
            }
        }
    }
}

// k_wedge_spec: the wedge's single sums as two phi-convolutions per target
// row, one with sigma_w and one with the first grid row sigma_0 (through the
// wedge's one-sided radial slope (sigma_0 - sigma_w) / (r_0 - r_in / 2),
// times r_i: rho_i = r_i / (r_0 - r_in / 2) = beta^{i-1} (1 + beta)), the
// azimuthal slope folded in:
//   W[i, q] = Kb^{.,0} + (Kb^{.,phi}[q+1] - Kb^{.,phi}[q-1]) / 2 dphi - rho_i Kb^{.,r},
//   V[i, q] = rho_i Kb^{.,r}.
// Their phi-DFTs, G / N_phi times, are real for the radial component (even in
// q) and -i times real for the azimuthal one (odd): tables
// tab[t][m][i], t = Wr, Wphi, Vr, Vphi, m in [0, N_phi/2].  One block per
// row, one thread per mode; FP64 sums over q in [0, N_phi/2] with the mirror.
template <typename T>
__global__ void k_wedge_spec(int nu, int nphi, double du, double G, const double* __restrict__ wcells,
                             const double2* __restrict__ tw64, T* __restrict__ tab)
{
    const int i = blockIdx.x, half = nphi / 2;
    const long per = (long)nu * nphi;
    const double* K[6];
#pragma unroll
    for (int c6 = 0; c6 < 6; c6++) K[c6] = wcells + c6 * per + (long)i * nphi;
    const double beta = exp(du), rho = exp(du * (i - 1)) * (1.0 + beta), i2d = nphi / (4.0 * M_PI);
    const int stride = SG_NMAX / nphi;
    const double sc = G / nphi;
    const long tsz = (long)(half + 1) * nu;
    auto Wr = [&](int q) {
        const int qp = (q + 1) & (nphi - 1), qm = (q - 1) & (nphi - 1);
        return K[0][q] + (K[2][qp] - K[2][qm]) * i2d - rho * K[1][q];
    };
    auto Wp = [&](int q) {
        const int qp = (q + 1) & (nphi - 1), qm = (q - 1) & (nphi - 1);
        return K[3][q] + (K[5][qp] - K[5][qm]) * i2d - rho * K[4][q];
    };
    for (int m = threadIdx.x; m <= half; m += blockDim.x) {
        const double sg = (m & 1) ? -1.0 : 1.0;
        double wr = Wr(0) + sg * Wr(half), vr = rho * (K[1][0] + sg * K[1][half]), wp = 0.0, vp = 0.0;
        for (int q = 1; q < half; q++) {
            const double2 w = tw64[(long)((m * q) & (nphi - 1)) * stride];  // e^{-2 pi i m q / N_phi}
            wr += 2.0 * Wr(q) * w.x;
            vr += 2.0 * rho * K[1][q] * w.x;
            wp -= 2.0 * Wp(q) * w.y;
            vp -= 2.0 * rho * K[4][q] * w.y;
        }
        const long at = (long)m * nu + i;
        tab[0 * tsz + at] = (T)(sc * wr);
        tab[1 * tsz + at] = (T)(sc * wp);
        tab[2 * tsz + at] = (T)(sc * vr);
        tab[3 * tsz + at] = (T)(sc * vp);
    }
}

template <typename T>
cudaError_t launch_wedge_tables(int nu, int nphi, double du, double G, double rtol, int pot, double* wcells,
                                const void* tw64, T* tab, int* flag, cudaStream_t st)
{
    cudaError_t e = upload_rules();
    if (e != cudaSuccess) return e;
    int dev, nsm;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    const long noff = (long)nu * (nphi / 2 + 1);
    long blocks = (noff + 3) / 4;
    if (blocks > (long)nsm * 32) blocks = (long)nsm * 32;
    k_wedge_cells<<<(int)blocks, 128, 0, st>>>(nu, nphi, du, rtol, pot, wcells, flag);
    k_wedge_spec<T><<<nu, 256, 0, st>>>(nu, nphi, du, G, wcells, (const double2*)tw64, tab);
    return cudaGetLastError();
}
template cudaError_t launch_wedge_tables<float>(int, int, double, double, double, int, double*, const void*, float*,
                                                int*, cudaStream_t);
template cudaError_t launch_wedge_tables<double>(int, int, double, double, double, int, double*, const void*,
                                                 double*, int*, cudaStream_t);
template cudaError_t launch_wedge_tables<dfloat>(int, int, double, double, double, int, double*, const void*,
                                                 dfloat*, int*, cudaStream_t);

// ln(a + sqrt(a^2 + b^2)) for b != 0; for a < 0 as ln(b^2) - ln(R - a),
// which does not cancel
__device__ __forceinline__ double cart_lsum(double a, double b)
{
    const double R = hypot(a, b);
    return a >= 0.0 ? log(a + R) : 2.0 * log(fabs(b)) - log(R - a);
}

// The six cell integrals at offset (k, q) on square cells of side h, in
// the order K^{x,0}, K^{x,x}, K^{x,y}, K^{y,0}, K^{y,x}, K^{y,y}.  Corners
// sit at half-integer multiples of h, so no corner has X = 0 or Y = 0.
__device__ void cart_cell(int k, int q, double h, double K[6])
{
    const double xs[2] = {(-k - 0.5) * h, (-k + 0.5) * h}, ys[2] = {(-q - 0.5) * h, (-q + 0.5) * h};
    double a0 = 0, b0 = 0, ax = 0, by = 0, mr = 0;
#pragma unroll
    for (int u = 0; u < 2; u++)
#pragma unroll
        for (int w = 0; w < 2; w++) {
            const double X = xs[u], Y = ys[w], sg = (u == w) ? 1.0 : -1.0;
            const double ly = cart_lsum(Y, X), lx = cart_lsum(X, Y);
            a0 -= sg * ly;     // -ln(Y + R)
            b0 -= sg * lx;     // -ln(X + R)
            ax += sg * Y * lx; //  Y ln(X + R)
            by += sg * X * ly; //  X ln(Y + R)
            mr -= sg * hypot(X, Y);
        }
    K[0] = a0;
    K[1] = k * h * a0 + ax;
    K[2] = q * h * a0 + mr;
    K[3] = b0;
    K[4] = k * h * b0 + mr;
    K[5] = q * h * b0 + by;
}

__global__ void k_cart_fold(int nu, int nphi, double h, double G, double* __restrict__ keff,
                            double* __restrict__ nsr, double* __restrict__ nsp)
{
    const int L = 2 * nu;
    const long total = (long)L * nphi;
    const long perk = (long)(2 * nu - 1) * nphi;
    const double norm = G / ((double)L * nphi), i2h = 0.5 / h;
    for (long idx = (long)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += (long)gridDim.x * blockDim.x) {
        const int kk = (int)(idx / nphi), qs = (int)(idx % nphi);
        double Kx = 0.0, Ky = 0.0;
        if (kk != nu && qs != nphi / 2) {
            const int k = kk < nu ? kk : kk - L, q = qs < nphi / 2 ? qs : qs - nphi;
            double c[6], xu[6], xd[6], yu[6], yd[6];
            cart_cell(k, q, h, c);
            cart_cell(k + 1, q, h, xu);
            cart_cell(k - 1, q, h, xd);
            cart_cell(k, q + 1, h, yu);
            cart_cell(k, q - 1, h, yd);
            Kx = c[0] + (xu[1] - xd[1]) * i2h + (yu[2] - yd[2]) * i2h;
            Ky = c[3] + (xu[4] - xd[4]) * i2h + (yu[5] - yd[5]) * i2h;
        }
        if (kk != nu) {
            const int k = kk < nu ? kk : kk - L;
            keff[(long)(k + nu - 1) * nphi + qs] = Kx;
            keff[perk + (long)(k + nu - 1) * nphi + qs] = Ky;
        }
        nsr[idx] = Kx * norm;
        nsp[idx] = Ky * norm;
    }
}

cudaError_t launch_cart_fold(int nu, int nphi, double h, double G, double* cells, double* keff, double* nsr,
                             double* nsp, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(cells, 0, (size_t)6 * (2 * nu + 1) * nphi * sizeof(double), st);
    if (e != cudaSuccess) return e;
    const long total = (long)2 * nu * nphi;
    long blocks = (total + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    k_cart_fold<<<(int)blocks, 256, 0, st>>>(nu, nphi, h, G, keff, nsr, nsp);
    return cudaGetLastError();
}

cudaError_t launch_fold(int nu, int nphi, double du, double G, int p, const double* cells, double* keff, double* nsr,
                        double* nsp, cudaStream_t st)
{
    const long total = (long)2 * nu * nphi;
    long blocks = (total + 255) / 256;
    if (blocks > 65535) blocks = 65535;
    k_fold<<<(int)blocks, 256, 0, st>>>(nu, nphi, du, G, p, cells, keff, nsr, nsp);
    return cudaGetLastError();
}

}  // namespace sg
