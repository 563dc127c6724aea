/*
 * sg_oracle.c -- FP64 CPU oracle for the log-polar thin-disk force path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or table with the CUDA path.
 *
 * What it computes (Wang, Yen & Taam 2015, "Self-gravitational force
 * calculation of second order accuracy for infinitesimally thin gaseous disks
 * in polar coordinates"):
 *
 *  1. The six cell-integrated force kernels of Eq. 30-32 (radial) and
 *     Eq. A11-A13 (azimuthal), written in the dimensionless variables
 *     eta = rbar / r_i and xi = phibar - phi_j that Eq. 33 introduces:
 *
 *        K^{r,0}      = - int int eta (1 - eta cos xi) / F^3
 *        K^{r,r}      = - int int eta (1 - eta cos xi) (eta - beta^-k) / F^3
 *        K^{r,phi}    = - int int eta (1 - eta cos xi) (xi + q dphi) / F^3
 *        K^{phi,0}    =   int int eta^2 sin xi / F^3
 *        K^{phi,r}    =   int int eta^2 sin xi (eta - beta^-k) / F^3
 *        K^{phi,phi}  =   int int eta^2 sin xi (xi + q dphi) / F^3
 *
 *     with F^2 = eta^2 - 2 eta cos xi + 1 = (eta - cos xi)^2 + sin^2 xi.
 *     For the offset (k, q) = (i - i', j - j') the source cell is
 *        eta in beta^-k [2/(beta+1), 2 beta/(beta+1)],
 *        xi  in [(-q - 1/2) dphi, (-q + 1/2) dphi],
 *     (Sec. 3.2.1 grid: arithmetic cell centres, log-spaced faces), and
 *     xi + q dphi is the source point's azimuth measured from the source
 *     cell centre (phibar - phi_{j'} in Eq. 32 and A13).
 *
 *     The integrals are the exact cell integrals (the limit the paper's
 *     N_tpz-trapezoid rule of Eq. 41-43 tends to).  They are computed as
 *     iterated integrals, eta inside and xi outside, each by globally
 *     adaptive Gauss-Legendre quadrature (12 nodes per panel, error taken as
 *     the change when a panel is halved).  For the self cell (k, q) = (0, 0)
 *     the point eta = 1, xi = 0 is singular (Sec. 4): the xi range is split
 *     at 0 and the inner eta integral uses the substitution
 *     eta = cos xi + |sin xi| sinh t, which turns the near-singular peak of
 *     width |sin xi| into a smooth function of t.  The iterated integral over
 *     the eta-symmetric self cell is the principal value that the force of a
 *     uniform sheet takes at an interior point.
 *
 *  2. The direct O(N^2) convolution sums F = G sum sigma K^eff over the
 *     single grid, and the transposed sum used to check the adjoint.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NC 6 /* K^{r,0}, K^{r,r}, K^{r,phi}, K^{phi,0}, K^{phi,r}, K^{phi,phi} */
#define NV (2 * NC) /* value components followed by their scale components */
#define GLN 12
#define MAXPAN 4096
/* The inner (eta) integrals are resolved this much tighter than the outer
   (xi) one, so that their remaining error does not look like noise to the
   outer error estimate. */
#define INNER_FRAC 0.1
/* rounding level of a 12-node panel sum, in units of the panel's integral of
   |f| (50 unit roundoffs) */
#define NOISE (50.0 * 2.220446049250313e-16)

static double gl_x[GLN], gl_w[GLN];
static int gl_ready = 0;

/* Gauss-Legendre nodes and weights on [-1, 1] by Newton iteration on P_n. */
static void gl_init(void)
{
    if (gl_ready) return;
    for (int i = 0; i < GLN; i++) {
        double x = cos(M_PI * (i + 0.75) / (GLN + 0.5));
        double p0 = 1.0, p1 = x, dp = 1.0;
        for (int it = 0; it < 100; it++) {
            p0 = 1.0;
            p1 = x;
            for (int n = 2; n <= GLN; n++) {
                double p2 = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
                p0 = p1;
                p1 = p2;
            }
            dp = GLN * (x * p1 - p0) / (x * x - 1.0);
            double dx = p1 / dp;
            x -= dx;
            if (fabs(dx) < 1e-17) break;
        }
        p0 = 1.0;
        p1 = x;
        for (int n = 2; n <= GLN; n++) {
            double p2 = ((2.0 * n - 1.0) * x * p1 - (n - 1.0) * p0) / n;
            p0 = p1;
            p1 = p2;
        }
        dp = GLN * (x * p1 - p0) / (x * x - 1.0);
        gl_x[i] = x;
        gl_w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
    }
    gl_ready = 1;
}

typedef void (*vfun)(double x, const void* ctx, double out[NV]);

/* One Gauss-Legendre panel: value and integral of |f| per component. */
static void gl_panel(vfun f, const void* ctx, double a, double b, double val[NV], double av[NV])
{
    double h = 0.5 * (b - a), m = 0.5 * (a + b), v[NV];
    for (int c = 0; c < NV; c++) val[c] = av[c] = v[c] = 0.0;
    for (int i = 0; i < GLN; i++) {
        f(m + h * gl_x[i], ctx, v);
        for (int c = 0; c < NV; c++) {
            val[c] += gl_w[i] * v[c];
            av[c] += gl_w[i] * fabs(v[c]);
        }
    }
    for (int c = 0; c < NV; c++) {
        val[c] *= h;
        av[c] *= h;
    }
}

typedef struct {
    double a, b;
    double whole[NV]; /* one panel over [a, b] */
    double val[NV];   /* sum of the two half panels */
    double av[NV];
    double err[NV];
} panel_t;

static void panel_eval(vfun f, const void* ctx, panel_t* p)
{
    double m = 0.5 * (p->a + p->b), v1[NV], a1[NV], v2[NV], a2[NV];
    gl_panel(f, ctx, p->a, m, v1, a1);
    gl_panel(f, ctx, m, p->b, v2, a2);
    for (int c = 0; c < NV; c++) {
        p->val[c] = v1[c] + v2[c];
        p->av[c] = a1[c] + a2[c];
        p->err[c] = fabs(p->val[c] - p->whole[c]);
    }
    /* a change below the rounding level of the panel sums is noise: once
       the one-panel rule agrees with the two half panels that closely, the
       half panels are exact to rounding.  The level is that of the force
       vector (radial and azimuthal kernel of the same kind together). */
    for (int c = 0; c < NC; c++) {
        double e = p->err[c] - NOISE * (p->av[c] + p->av[(c + 3) % NC]);
        p->err[c] = e > 0.0 ? e : 0.0;
    }
}

/*
 * Globally adaptive quadrature of the vector f over the partition
 * bp[0] < bp[1] < ... < bp[nbp-1].  Panels are bisected, worst first, until
 * for each value component c < NC the summed error estimate is at most
 * rtol * (S_c + S_c') + atol, where c' = (c + 3) mod 6 is the other
 * component of the same force vector (radial / azimuthal) and S_c is the
 * integral of |f_c| (aux == 0) or of the scale component f_{NC+c} (aux ==
 * 1; the caller supplies there the integral of |integrand| over the inner
 * variable).  res gets the
 * NV integrals, resabs the integrals of |f|.  Returns the number of panels,
 * or a negative number if the panel budget ran out (the result is then the
 * best estimate).
 */
static int adapt(vfun f, const void* ctx, const double* bp, int nbp, double rtol, double atol, int aux,
                 double res[NV], double resabs[NV])
{
    int cap = nbp + 32, np = 0, status = 0;
    panel_t* P = (panel_t*)malloc(sizeof(panel_t) * cap);
    for (int s = 0; s + 1 < nbp; s++) {
        if (!(bp[s + 1] > bp[s])) continue;
        panel_t* p = &P[np++];
        p->a = bp[s];
        p->b = bp[s + 1];
        double av[NV];
        gl_panel(f, ctx, p->a, p->b, p->whole, av);
        panel_eval(f, ctx, p);
    }
    for (;;) {
        double E[NV], A[NV], V[NV];
        for (int c = 0; c < NV; c++) E[c] = A[c] = V[c] = 0.0;
        for (int i = 0; i < np; i++)
            for (int c = 0; c < NV; c++) {
                E[c] += P[i].err[c];
                A[c] += P[i].av[c];
                V[c] += P[i].val[c];
            }
        double tol[NC];
        int done = 1;
        for (int c = 0; c < NC; c++) {
            /* scale of the force vector: radial and azimuthal kernels of the
               same kind (components c and c +- 3) together */
            const int cp = (c + 3) % NC;
            tol[c] = rtol * (aux ? fabs(V[NC + c]) + fabs(V[NC + cp]) : A[c] + A[cp]) + atol;
            if (E[c] > tol[c]) done = 0;
        }
        if (done) {
            for (int c = 0; c < NV; c++) {
                res[c] = V[c];
                resabs[c] = A[c];
            }
            status = np;
            break;
        }
        if (np + 1 >= MAXPAN) {
            for (int c = 0; c < NV; c++) {
                res[c] = V[c];
                resabs[c] = A[c];
            }
            status = -np;
            break;
        }
        /* bisect the panel with the largest normalised error */
        int worst = 0;
        double wv = -1.0;
        for (int i = 0; i < np; i++) {
            double e = 0.0;
            for (int c = 0; c < NC; c++) {
                double r = P[i].err[c] / (tol[c] > 0 ? tol[c] : 1e-300);
                if (r > e) e = r;
            }
            if (e > wv) {
                wv = e;
                worst = i;
            }
        }
        panel_t old = P[worst];
        double m = 0.5 * (old.a + old.b);
        if (!(m > old.a && m < old.b)) { /* cannot split further */
            for (int c = 0; c < NV; c++) P[worst].err[c] = 0.0;
            continue;
        }
        if (np + 1 > cap) {
            cap *= 2;
            P = (panel_t*)realloc(P, sizeof(panel_t) * cap);
        }
        panel_t* L = &P[worst];
        panel_t* R = &P[np++];
        L->a = old.a;
        L->b = m;
        R->a = m;
        R->b = old.b;
        double av[NV];
        gl_panel(f, ctx, L->a, L->b, L->whole, av);
        gl_panel(f, ctx, R->a, R->b, R->whole, av);
        panel_eval(f, ctx, L);
        panel_eval(f, ctx, R);
    }
    free(P);
    return status;
}

/* ---------------------------------------------------------------------- */
/* Integrands                                                              */
/* ---------------------------------------------------------------------- */

typedef struct {
    double eta_lo, eta_hi; /* source cell in eta */
    double xi_lo, xi_hi;   /* source cell in xi */
    double eta_c;          /* beta^-k: the source centre r_{i'} / r_i */
    double qd;             /* q * dphi, q taken in (-N/2, N/2] */
    int self;              /* k == 0 and q == 0 */
    double rtol;
    int* bad; /* count of integrals that ran out of panels */
} cell_t;

typedef struct {
    const cell_t* cell;
    double xi, c, s; /* outer node and cos, sin of it */
    double vc;       /* 1 - cos xi = 2 sin^2(xi/2), without cancellation */
} inner_t;

/* The six integrands at (eta, xi); om = 1 - eta cos xi, F3 = F^3. */
static inline void six(double eta, double xi, double s, double om, double F3, double eta_c, double qd,
                       double out[NC])
{
    double ir0 = -eta * om / F3;
    double ip0 = eta * eta * s / F3;
    double dr = eta - eta_c, dp = xi + qd;
    out[0] = ir0;
    out[1] = ir0 * dr;
    out[2] = ir0 * dp;
    out[3] = ip0;
    out[4] = ip0 * dr;
    out[5] = ip0 * dp;
}

/* inner integrand in eta (ordinary cells) */
static void f_eta(double eta, const void* vctx, double out[NV])
{
    const inner_t* ic = (const inner_t*)vctx;
    /* eta - cos xi and 1 - eta cos xi from eta - 1 (exact near eta = 1) and
       1 - cos xi, so that both keep their relative precision where they are
       small */
    double e1 = eta - 1.0;
    double d = e1 + ic->vc;
    double F2 = d * d + ic->s * ic->s;
    double F3 = F2 * sqrt(F2);
    double om = ic->vc - e1 * ic->c;
    six(eta, ic->xi, ic->s, om, F3, ic->cell->eta_c, ic->cell->qd, out);
}

/* inner integrand in t for the self cell: eta = c + |s| sinh t,
   F = |s| cosh t, d eta = |s| cosh t dt, 1 - eta c = s^2 - c |s| sinh t. */
static void f_t(double t, const void* vctx, double out[NV])
{
    const inner_t* ic = (const inner_t*)vctx;
    double as = fabs(ic->s), sh = sinh(t), ch = cosh(t);
    double eta = ic->c + as * sh;
    double F = as * ch;
    double F3 = F * F * F;
    double om = ic->s * ic->s - ic->c * as * sh;
    double v[NC];
    /* eta - 1 for the self cell, written without cancellation */
    double sh2 = sin(0.5 * ic->xi);
    six(eta, ic->xi, ic->s, om, F3, 1.0, ic->cell->qd, v);
    /* replace the (eta - eta_c) factor by the accurate form */
    double dr = -2.0 * sh2 * sh2 + as * sh;
    double ir0 = -eta * om / F3, ip0 = eta * eta * ic->s / F3;
    v[1] = ir0 * dr;
    v[4] = ip0 * dr;
    for (int c = 0; c < NC; c++) out[c] = v[c] * F; /* Jacobian |s| cosh t */
    /* K^{r,0}: with eta = c + |s| sinh t,
         f d eta = [-eta / cosh^2 t + c tanh^2 t] dt + (c^2/|s|) sinh t / cosh^2 t dt.
       The last term is an odd pair of lobes of height 1/|s| whose sum is
       small; its integral, c^2 (1/F(eta_lo) - 1/F(eta_hi)), is added by the
       caller, and only the bounded remainder is integrated here. */
    double th = sh / ch;
    out[0] = -eta / (ch * ch) + ic->c * th * th;
}

/* outer integrand in xi: the inner eta integrals (out[0..5]) and the inner
   integrals of their absolute integrands (out[6..11], the error scale) */
static void f_xi(double xi, const void* vctx, double out[NV])
{
    const cell_t* cell = (const cell_t*)vctx;
    inner_t ic;
    ic.cell = cell;
    ic.xi = xi;
    ic.c = cos(xi);
    ic.s = sin(xi);
    ic.vc = 2.0 * sin(0.5 * xi) * sin(0.5 * xi);
    double abs_[NV];
    int st;
    if (cell->self && ic.s != 0.0) {
        double as = fabs(ic.s);
        double ta = asinh((cell->eta_lo - ic.c) / as);
        double tb = asinh((cell->eta_hi - ic.c) / as);
        /* initial partition into panels of width <= 1 in t */
        int npan = (int)ceil(tb - ta);
        if (npan < 1) npan = 1;
        if (npan > 200) npan = 200;
        double bp[202];
        for (int i = 0; i <= npan; i++) bp[i] = ta + (tb - ta) * i / npan;
        bp[npan] = tb;
        st = adapt(f_t, &ic, bp, npan + 1, INNER_FRAC * cell->rtol, 0.0, 0, out, abs_);
        /* the lobe term of K^{r,0} removed from the integrand in f_t */
        double Fa = sqrt((cell->eta_lo - ic.c) * (cell->eta_lo - ic.c) + ic.s * ic.s);
        double Fb = sqrt((cell->eta_hi - ic.c) * (cell->eta_hi - ic.c) + ic.s * ic.s);
        out[0] += ic.c * ic.c * (1.0 / Fa - 1.0 / Fb);
    } else {
        double bp[3];
        int nb = 0;
        bp[nb++] = cell->eta_lo;
        if (ic.c > cell->eta_lo && ic.c < cell->eta_hi) bp[nb++] = ic.c; /* nearest point to the pole */
        bp[nb++] = cell->eta_hi;
        st = adapt(f_eta, &ic, bp, nb, INNER_FRAC * cell->rtol, 0.0, 0, out, abs_);
    }
    for (int c = 0; c < NC; c++) out[NC + c] = abs_[c];
    if (st < 0) {
#ifdef _OPENMP
#pragma omp atomic
#endif
        (*cell->bad)++;
    }
}

/* Self cell: the cell is symmetric in xi, and the inner integrals of the
   components odd in xi (K^{r,phi}, K^{phi,0}, K^{phi,r}) behave like 1/xi,
   so the xi integral exists as a principal value.  Integrate g(xi) + g(-xi)
   over [0, dphi/2]: the odd parts cancel pointwise, the even parts double. */
static void f_xi_pair(double xi, const void* vctx, double out[NV])
{
    double a[NV], b[NV];
    for (int c = 0; c < NV; c++) out[c] = 0.0;
    if (!(fabs(sin(xi)) > 1e-200)) return; /* measure-zero neighbourhood of the pole */
    f_xi(xi, vctx, a);
    f_xi(-xi, vctx, b);
    /* the inner |integrand| integrals grow like 1/|xi| here, so the scale
       comes from |g| itself (aux == 0 in the outer call) */
    for (int c = 0; c < NC; c++) out[c] = a[c] + b[c];
}

/*
 * The six kernel values for offset (k, q) on a grid with beta = e^du and
 * dphi = 2 pi / N_phi.  q is any integer; it is reduced to (-N/2, N/2] by the
 * caller through qd.  Returns 0, or the number of sub-integrals that ran out
 * of panels.
 */
int sgo_cell(double du, int nphi, int k, int q, double rtol, double out6[NC])
{
    gl_init();
    double beta = exp(du), dphi = 2.0 * M_PI / nphi;
    int qs = ((q % nphi) + nphi) % nphi;
    if (2 * qs > nphi) qs -= nphi;
    int bad = 0;
    cell_t cell;
    cell.eta_c = exp(-du * k);
    cell.eta_lo = cell.eta_c * 2.0 / (beta + 1.0);
    cell.eta_hi = cell.eta_c * 2.0 * beta / (beta + 1.0);
    cell.xi_lo = (-qs - 0.5) * dphi;
    cell.xi_hi = (-qs + 0.5) * dphi;
    cell.qd = qs * dphi;
    cell.self = (k == 0 && qs == 0);
    cell.rtol = rtol;
    cell.bad = &bad;
    double bp[3], abs_[NV], out[NV];
    int nb = 0, st;
    if (cell.self) {
        /* rounding in the near-singular inner integrals, relative to a cell
           value that shrinks with the cell, sets a floor on what this cell
           can resolve: try 1e-14, then 1e-13, then 1e-12 */
        bp[nb++] = 0.0;
        bp[nb++] = cell.xi_hi;
        double floors[3] = {1e-14, 1e-13, 1e-12};
        for (int attempt = 0; attempt < 3; attempt++) {
            cell.rtol = rtol > floors[attempt] ? rtol : floors[attempt];
            bad = 0;
            st = adapt(f_xi_pair, &cell, bp, nb, cell.rtol, 0.0, 0, out, abs_);
            if (st > 0 && bad == 0) break;
        }
    } else {
        bp[nb++] = cell.xi_lo;
        if (cell.xi_lo < 0.0 && cell.xi_hi > 0.0) bp[nb++] = 0.0;
        bp[nb++] = cell.xi_hi;
        st = adapt(f_xi, &cell, bp, nb, rtol, 0.0, 1, out, abs_);
    }
    if (st < 0) bad++;
    for (int c = 0; c < NC; c++) out6[c] = out[c];
    return bad;
}

/*
 * Kernel table for k in [-Nu, Nu], q in [0, Nphi):
 * out[c][(k + Nu) * Nphi + q], c = 0..5.  Returns the number of integrals
 * that ran out of panels (0 when all converged).
 */
int sgo_cells_table(int nu, int nphi, double du, double rtol, double* out, int nthreads)
{
    gl_init();
    long nk = 2L * nu + 1, per = nk * nphi;
    int bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : bad)
#endif
    for (long idx = 0; idx < per; idx++) {
        int k = (int)(idx / nphi) - nu;
        int q = (int)(idx % nphi);
        double v[NC];
        bad += sgo_cell(du, nphi, k, q, rtol, v);
        for (int c = 0; c < NC; c++) out[c * per + idx] = v[c];
    }
    return bad;
}

/*
 * Direct O(N^2) sum (the convolution form of Eq. 27-29 and A8-A10 after the
 * slope terms are folded into one kernel per component):
 *   F_r[i,j]   = G sum_{m,l} sigma[m,l] Kr  [i-m, (j-l) mod Nphi]
 *   F_phi[i,j] = G sum_{m,l} sigma[m,l] Kphi[i-m, (j-l) mod Nphi]
 * Kr, Kphi: [(2Nu-1) * Nphi], row index k + Nu - 1.
 * targets: flat target indices i*Nphi + j (or NULL for all cells).
 */
void sgo_direct_sum(int nu, int nphi, double G, const double* Kr, const double* Kp, const double* sigma,
                    const long* targets, long ntargets, double* Fr, double* Fp, int nthreads)
{
    long ncell = (long)nu * nphi;
    long nt = targets ? ntargets : ncell;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (long t = 0; t < nt; t++) {
        long cellidx = targets ? targets[t] : t;
        int i = (int)(cellidx / nphi), j = (int)(cellidx % nphi);
        double sr = 0.0, sp = 0.0;
        for (int m = 0; m < nu; m++) {
            const double* kr = Kr + (long)(i - m + nu - 1) * nphi;
            const double* kp = Kp + (long)(i - m + nu - 1) * nphi;
            const double* sg = sigma + (long)m * nphi;
            for (int l = 0; l < nphi; l++) {
                int q = j - l;
                if (q < 0) q += nphi;
                sr += sg[l] * kr[q];
                sp += sg[l] * kp[q];
            }
        }
        Fr[t] = G * sr;
        Fp[t] = G * sp;
    }
}

/*
 * Transposed sum: gsigma[m,l] = G sum_{i,j} (gFr[i,j] Kr[i-m, (j-l)] +
 * gFphi[i,j] Kphi[i-m, (j-l)]), i.e. A^T g for the map A of sgo_direct_sum.
 */
void sgo_direct_sum_T(int nu, int nphi, double G, const double* Kr, const double* Kp, const double* gFr,
                      const double* gFp, const long* sources, long nsources, double* gs, int nthreads)
{
    long ncell = (long)nu * nphi;
    long ns = sources ? nsources : ncell;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 4)
#endif
    for (long t = 0; t < ns; t++) {
        long cellidx = sources ? sources[t] : t;
        int m = (int)(cellidx / nphi), l = (int)(cellidx % nphi);
        double acc = 0.0;
        for (int i = 0; i < nu; i++) {
            const double* kr = Kr + (long)(i - m + nu - 1) * nphi;
            const double* kp = Kp + (long)(i - m + nu - 1) * nphi;
            const double* gr = gFr + (long)i * nphi;
            const double* gp = gFp + (long)i * nphi;
            for (int j = 0; j < nphi; j++) {
                int q = j - l;
                if (q < 0) q += nphi;
                acc += gr[j] * kr[q] + gp[j] * kp[q];
            }
        }
        gs[t] = G * acc;
    }
}

int sgo_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* The inner eta integral at one xi (for the tests of the quadrature). */
int sgo_inner(double du, int nphi, int k, int q, double xi, double rtol, double out[NV])
{
    gl_init();
    double beta = exp(du), dphi = 2.0 * M_PI / nphi;
    int qs = ((q % nphi) + nphi) % nphi;
    if (2 * qs > nphi) qs -= nphi;
    int bad = 0;
    cell_t cell;
    cell.eta_c = exp(-du * k);
    cell.eta_lo = cell.eta_c * 2.0 / (beta + 1.0);
    cell.eta_hi = cell.eta_c * 2.0 * beta / (beta + 1.0);
    cell.xi_lo = (-qs - 0.5) * dphi;
    cell.xi_hi = (-qs + 0.5) * dphi;
    cell.qd = qs * dphi;
    cell.self = (k == 0 && qs == 0);
    cell.rtol = rtol;
    cell.bad = &bad;
    f_xi(xi, &cell, out);
    return bad;
}
