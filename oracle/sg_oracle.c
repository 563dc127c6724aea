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
 *     iterated integrals, eta inside and xi outside (as offsets from the
 *     cell centre, eta - beta^-k and xi + q dphi), each by globally adaptive
 *     Gauss-Legendre quadrature (12 nodes per panel, error taken as the
 *     change when a panel is halved).  For the self cell (k, q) = (0, 0)
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
static int adapt_n(vfun f, const void* ctx, const double* bp, int nbp, double rtol, double atol, int aux,
                   int maxpan, double res[NV], double resabs[NV])
{
    panel_t local[48];
    int cap = 48, np = 0, status = 0;
    panel_t* P = local;
    if (nbp + 32 > cap) {
        cap = nbp + 32;
        P = (panel_t*)malloc(sizeof(panel_t) * cap);
    }
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
        if (np + 1 >= maxpan) {
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
            if (P == local) {
                P = (panel_t*)malloc(sizeof(panel_t) * cap);
                memcpy(P, local, sizeof(local));
            } else {
                P = (panel_t*)realloc(P, sizeof(panel_t) * cap);
            }
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
    if (P != local) free(P);
    return status;
}

static int adapt(vfun f, const void* ctx, const double* bp, int nbp, double rtol, double atol, int aux,
                 double res[NV], double resabs[NV])
{
    return adapt_n(f, ctx, bp, nbp, rtol, atol, aux, MAXPAN, res, resabs);
}

/* ---------------------------------------------------------------------- */
/* Integrands                                                              */
/* ---------------------------------------------------------------------- */

typedef struct {
    double eta_lo, eta_hi; /* source cell in eta */
    double eta_c;          /* beta^-k: the source centre r_{i'} / r_i */
    double em1;            /* eta_c - 1, exact for k = 0 */
    double hw;             /* half width in eta: eta_c (beta - 1)/(beta + 1) */
    double sc, cc;         /* sine and cosine of the centre azimuth -q dphi */
    double half_dphi;
    double qd;             /* q * dphi, q taken in (-N/2, N/2] */
    int self;              /* k == 0 and q == 0 */
    int pot;               /* the potential's cells instead of the forces' */
    double rtol;
    int* bad; /* count of integrals that ran out of panels */
} cell_t;

/* The inner variable is del = eta - eta_c (so eta - eta_c is exact) and the
   outer one t = xi - xi_c with xi_c = -q dphi the centre azimuth (so the
   local azimuth of K^{.,phi} is t itself and sin xi, cos xi follow from t
   and the exact centre values by angle addition). */
typedef struct {
    const cell_t* cell;
    double t, c, s; /* outer node t and cos, sin of xi = xi_c + t */
    double vc;      /* 1 - cos xi without cancellation */
} inner_t;

/* inner integrand in del = eta - eta_c (ordinary cells) */
static void f_eta(double del, const void* vctx, double out[NV])
{
    const inner_t* ic = (const inner_t*)vctx;
    const cell_t* cl = ic->cell;
    /* eta - cos xi and 1 - eta cos xi from eta - 1 = (eta_c - 1) + del and
       1 - cos xi, so that both keep their relative precision where they are
       small */
    double eta = cl->eta_c + del;
    double e1 = cl->em1 + del;
    double d = e1 + ic->vc;
    double F2 = d * d + ic->s * ic->s;
    double F3 = F2 * sqrt(F2);
    double om = ic->vc - e1 * ic->c;
    double ir0 = -eta * om / F3;
    double ip0 = eta * eta * ic->s / F3;
    if (cl->pot) { /* the potential: -eta / F and its slope factors */
        ir0 = -eta / sqrt(F2);
        ip0 = 0.0;
    }
    out[0] = ir0;
    out[1] = ir0 * del;
    out[2] = ir0 * ic->t;
    out[3] = ip0;
    out[4] = ip0 * del;
    out[5] = ip0 * ic->t;
}

/* inner integrand in tau for the self cell (xi_c = 0, eta_c = 1, so xi = t):
   eta = c + |s| sinh tau, F = |s| cosh tau, d eta = |s| cosh tau d tau,
   1 - eta c = s^2 - c |s| sinh tau, eta - 1 = |s| sinh tau - (1 - c). */
static void f_tau(double tau, const void* vctx, double out[NV])
{
    const inner_t* ic = (const inner_t*)vctx;
    double as = fabs(ic->s), sh = sinh(tau), ch = cosh(tau);
    double eta = ic->c + as * sh;
    double F = as * ch;
    double F3 = F * F * F;
    double om = ic->s * ic->s - ic->c * as * sh;
    double dr = as * sh - ic->vc;
    double ir0 = -eta * om / F3, ip0 = eta * eta * ic->s / F3;
    if (ic->cell->pot) { /* (-eta / F) d eta = -eta d tau: smooth */
        out[0] = -eta;
        out[1] = -eta * dr;
        out[2] = -eta * ic->t;
        out[3] = out[4] = out[5] = 0.0;
        return;
    }
    out[0] = ir0 * F;
    out[1] = ir0 * dr * F;
    out[2] = ir0 * ic->t * F;
    out[3] = ip0 * F;
    out[4] = ip0 * dr * F;
    out[5] = ip0 * ic->t * F;
    /* K^{r,0}: f d eta = [-eta / cosh^2 tau + c tanh^2 tau] d tau
                          + (c^2/|s|) sinh tau / cosh^2 tau d tau.
       The last term is an odd pair of lobes of height 1/|s| whose sum is
       small; its integral, c^2 (1/F(eta_lo) - 1/F(eta_hi)), is added by the
       caller, and only the bounded remainder is integrated here. */
    double th = sh / ch;
    out[0] = -eta / (ch * ch) + ic->c * th * th;
}

/* outer integrand in t = xi - xi_c: the inner integrals (out[0..5]) and the
   inner integrals of their absolute integrands (out[6..11], the error scale) */
static void f_xi(double t, const void* vctx, double out[NV])
{
    const cell_t* cell = (const cell_t*)vctx;
    inner_t ic;
    ic.cell = cell;
    ic.t = t;
    double st = sin(t), ct = cos(t);
    ic.c = cell->cc * ct - cell->sc * st;
    ic.s = cell->sc * ct + cell->cc * st;
    ic.vc = ic.c > 0.0 ? ic.s * ic.s / (1.0 + ic.c) : 1.0 - ic.c;
    double abs_[NV];
    int st_;
    if (cell->self && ic.s != 0.0) {
        double as = fabs(ic.s);
        double ta = asinh((cell->eta_lo - ic.c) / as);
        double tb = asinh((cell->eta_hi - ic.c) / as);
        /* initial partition into panels of width <= 1 in tau */
        int npan = (int)ceil(tb - ta);
        if (npan < 1) npan = 1;
        if (npan > 200) npan = 200;
        double bp[202];
        for (int i = 0; i <= npan; i++) bp[i] = ta + (tb - ta) * i / npan;
        bp[npan] = tb;
        st_ = adapt(f_tau, &ic, bp, npan + 1, INNER_FRAC * cell->rtol, 0.0, 0, out, abs_);
        /* the lobe term of K^{r,0} removed from the integrand in f_tau */
        if (!cell->pot) {
            double Fa = sqrt((cell->eta_lo - ic.c) * (cell->eta_lo - ic.c) + ic.s * ic.s);
            double Fb = sqrt((cell->eta_hi - ic.c) * (cell->eta_hi - ic.c) + ic.s * ic.s);
            out[0] += ic.c * ic.c * (1.0 / Fa - 1.0 / Fb);
        }
    } else {
        double bp[3];
        int nb = 0;
        bp[nb++] = -cell->hw;
        double peak = -ic.vc - cell->em1; /* eta = cos xi: the point nearest the pole */
        if (peak > -cell->hw && peak < cell->hw) bp[nb++] = peak;
        bp[nb++] = cell->hw;
        st_ = adapt(f_eta, &ic, bp, nb, INNER_FRAC * cell->rtol, 0.0, 0, out, abs_);
    }
    for (int c = 0; c < NC; c++) out[NC + c] = abs_[c];
    if (st_ < 0) {
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
static void f_xi_pair(double t, const void* vctx, double out[NV])
{
    double a[NV], b[NV];
    for (int c = 0; c < NV; c++) out[c] = 0.0;
    if (!(fabs(sin(t)) > 1e-200)) return; /* measure-zero neighbourhood of the pole */
    f_xi(t, vctx, a);
    f_xi(-t, vctx, b);
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
/* sin and cos of 2 pi num / den (den a power of two, |num| <= den) with the
   argument reduced exactly to the first octant */
static void sincos_2pi_frac(long num, long den, double* s, double* c)
{
    long n = ((num % den) + den) % den; /* [0, den) */
    long e8 = den / 8 > 0 ? den / 8 : 0;
    if (e8 == 0) { /* den < 8: direct */
        *s = sin(2.0 * M_PI * (double)n / den);
        *c = cos(2.0 * M_PI * (double)n / den);
        return;
    }
    int o = (int)(n / e8);
    long r = n - o * e8;
    double a, sa, ca;
    if ((o & 1) == 0) {
        a = 2.0 * M_PI * r / den;
        sa = sin(a);
        ca = cos(a);
        switch (o) {
            case 0: *c = ca; *s = sa; break;
            case 2: *c = -sa; *s = ca; break;
            case 4: *c = -ca; *s = -sa; break;
            default: *c = sa; *s = -ca; break;
        }
    } else {
        a = 2.0 * M_PI * (e8 - r) / den;
        sa = sin(a);
        ca = cos(a);
        switch (o) {
            case 1: *c = sa; *s = ca; break;
            case 3: *c = -ca; *s = sa; break;
            case 5: *c = -sa; *s = -ca; break;
            default: *c = ca; *s = -sa; break;
        }
    }
}

static void cell_setup(cell_t* cell, double du, int nphi, int k, int qs, double rtol, int* bad)
{
    double beta = exp(du), dphi = 2.0 * M_PI / nphi;
    cell->eta_c = exp(-du * k);
    cell->em1 = expm1(-du * k);
    cell->hw = cell->eta_c * tanh(0.5 * du);
    cell->eta_lo = cell->eta_c * 2.0 / (beta + 1.0);
    cell->eta_hi = cell->eta_c * 2.0 * beta / (beta + 1.0);
    sincos_2pi_frac(-(long)qs, nphi, &cell->sc, &cell->cc);
    cell->half_dphi = 0.5 * dphi;
    cell->qd = qs * dphi;
    cell->self = (k == 0 && qs == 0);
    cell->pot = 0;
    cell->rtol = rtol;
    cell->bad = bad;
}

/*
 * The six kernel values for offset (k, q) on a grid with beta = e^du and
 * dphi = 2 pi / N_phi.  q is any integer (reduced to (-N/2, N/2]).  Returns
 * 0, or the number of sub-integrals that ran out of panels.
 */
static int cell_of(double du, int nphi, int k, int q, double rtol, int pot, double out6[NC])
{
    gl_init();
    int qs = ((q % nphi) + nphi) % nphi;
    if (2 * qs > nphi) qs -= nphi;
    int bad = 0;
    cell_t cell;
    cell_setup(&cell, du, nphi, k, qs, rtol, &bad);
    cell.pot = pot;
    double bp[3], abs_[NV], out[NV];
    int nb = 0, st;
    if (cell.self) {
        /* rounding in the near-singular inner integrals, relative to a cell
           value that shrinks with the cell, sets a floor on what this cell
           can resolve: try 1e-14, then 1e-13, ... up to 1e-10 (cells of
           about 0.003 radians on a side, N_phi = 2048 and beyond, need
           1e-11 or 1e-10) */
        bp[nb++] = 0.0;
        bp[nb++] = cell.half_dphi;
        double floors[5] = {1e-14, 1e-13, 1e-12, 1e-11, 1e-10};
        for (int attempt = 0; attempt < 5; attempt++) {
            cell.rtol = rtol > floors[attempt] ? rtol : floors[attempt];
            bad = 0;
            /* a log-singular endpoint needs about 60 bisections; more
               panels than that only chase rounding */
            st = adapt_n(f_xi_pair, &cell, bp, nb, cell.rtol, 0.0, 0, attempt < 2 ? 400 : MAXPAN, out, abs_);
            if (st > 0 && bad == 0) break;
        }
    } else {
        bp[nb++] = -cell.half_dphi;
        bp[nb++] = cell.half_dphi;
        st = adapt(f_xi, &cell, bp, nb, rtol, 0.0, 1, out, abs_);
    }
    if (st < 0) bad++;
    for (int c = 0; c < NC; c++) out6[c] = out[c];
    return bad;
}

int sgo_cell(double du, int nphi, int k, int q, double rtol, double out6[NC])
{
    return cell_of(du, nphi, k, q, rtol, 0, out6);
}

/*
 * The potential's cells for the offset (k, q): out6[0..2] = -int eta / F,
 * -int eta (eta - beta^-k) / F, -int eta (xi + q dphi) / F over the source
 * cell (d eta d xi), out6[3..5] = 0.  With them the potential at the centre
 * of target row i is Phi = G r_i sum sigma (K^{P,0} + slope terms), the
 * slopes entering as for the forces.
 */
int sgo_cell_pot(double du, int nphi, int k, int q, double rtol, double out6[NC])
{
    return cell_of(du, nphi, k, q, rtol, 1, out6);
}

/*
 * Kernel table for k in [-Nu, Nu], q in [0, Nphi):
 * out[c][(k + Nu) * Nphi + q], c = 0..5.  The cells with q in (Nphi/2, Nphi)
 * are the mirror images xi -> -xi of those with Nphi - q (K^{r,0}, K^{r,r},
 * K^{phi,phi} even, K^{r,phi}, K^{phi,0}, K^{phi,r} odd).  Returns the number
 * of integrals that ran out of panels (0 when all converged).
 */
static int cells_table_of(int nu, int nphi, double du, double rtol, int pot, double* out, int nthreads);

int sgo_cells_table(int nu, int nphi, double du, double rtol, double* out, int nthreads)
{
    return cells_table_of(nu, nphi, du, rtol, 0, out, nthreads);
}

int sgo_cells_table_pot(int nu, int nphi, double du, double rtol, double* out, int nthreads)
{
    return cells_table_of(nu, nphi, du, rtol, 1, out, nthreads);
}

static int cells_table_of(int nu, int nphi, double du, double rtol, int pot, double* out, int nthreads)
{
    gl_init();
    long nk = 2L * nu + 1, per = nk * nphi, nq = nphi / 2 + 1;
    int bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : bad)
#endif
    for (long idx = 0; idx < nk * nq; idx++) {
        int k = (int)(idx / nq) - nu;
        int q = (int)(idx % nq);
        double v[NC];
        bad += cell_of(du, nphi, k, q, rtol, pot, v);
        long row = (long)(k + nu) * nphi;
        int qm = (nphi - q) % nphi;
        for (int c = 0; c < NC; c++) {
            out[c * per + row + q] = v[c];
            if (qm != q) out[c * per + row + qm] = (c == 2 || c == 3 || c == 4) ? -v[c] : v[c];
        }
    }
    return bad;
}

/*
 * The origin wedge R^_j' = [0, r_in] x [phi_{j'-1/2}, phi_{j'+1/2}] (Sec. 3.2.1
 * and the third terms of Eq. 27-29, kernels K-bar) seen from the centre of
 * grid row i: the same six integrals over eta in [0, eta_w], eta_w = r_in / r_i
 * = 2 / (beta^i (1 + beta)), with the slope factors measured from the wedge's
 * centre eta_w / 2 (the arithmetic mean of its faces 0 and r_in).  The wedge
 * lies inside every target radius, so no integrand is singular.  Table
 * out[c][i * Nphi + q], i in [0, Nu), q in [0, Nphi), mirrored as
 * sgo_cells_table; returns the number of integrals that ran out of panels.
 */
static int wedge_cell_of(double du, int nphi, int i, int q, double rtol, int pot, double out6[NC])
{
    int qs = ((q % nphi) + nphi) % nphi;
    if (2 * qs > nphi) qs -= nphi;
    int bad = 0;
    cell_t cell;
    cell_setup(&cell, du, nphi, 1, qs, rtol, &bad); /* azimuth and tolerances; eta limits below */
    const double beta = exp(du), eta_w = 2.0 / (exp(du * i) * (1.0 + beta));
    cell.eta_lo = 0.0;
    cell.eta_hi = eta_w;
    cell.eta_c = 0.5 * eta_w;
    cell.em1 = 0.5 * eta_w - 1.0;
    cell.hw = 0.5 * eta_w;
    cell.self = 0;
    cell.pot = pot;
    double bp[2] = {-cell.half_dphi, cell.half_dphi}, abs_[NV], out[NV];
    int st = adapt(f_xi, &cell, bp, 2, rtol, 0.0, 1, out, abs_);
    if (st < 0) bad++;
    for (int c = 0; c < NC; c++) out6[c] = out[c];
    return bad;
}

int sgo_wedge_table(int nu, int nphi, double du, double rtol, int pot, double* out, int nthreads)
{
    gl_init();
    long per = (long)nu * nphi, nq = nphi / 2 + 1;
    int bad = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : bad)
#endif
    for (long idx = 0; idx < nu * nq; idx++) {
        int i = (int)(idx / nq), q = (int)(idx % nq);
        double v[NC];
        bad += wedge_cell_of(du, nphi, i, q, rtol, pot, v);
        long row = (long)i * nphi;
        int qm = (nphi - q) % nphi;
        for (int c = 0; c < NC; c++) {
            out[c * per + row + q] = v[c];
            if (qm != q) out[c * per + row + qm] = (c == 2 || c == 3 || c == 4) ? -v[c] : v[c];
        }
    }
    return bad;
}

/*
 * The trapezoidal form of the kernels (Eq. 41-43 for K^{r,0}, K^{r,r},
 * K^{r,phi}, the same rule for K^{phi,phi} of App. A): for every cell but
 * the own one, the eta-integrals at the N_tpz + 1 azimuths
 * phi'_m = phi_{j'-1/2} + m dtheta, dtheta = dphi / N_tpz, of the source cell
 * (f_xi: adaptive, exact to rtol) combined by the trapezoidal rule.
 * K^{phi,0}, K^{phi,r} are exact in the paper too, and the own cell is the
 * singular integral of Sec. 4: those entries keep the exact table of
 * sgo_cells_table, which this fills first.  Same layout and return value.
 */
int sgo_cells_table_tpz(int nu, int nphi, double du, int ntpz, double rtol, double* out, int nthreads)
{
    int bad = sgo_cells_table(nu, nphi, du, rtol, out, nthreads);
    long nk = 2L * nu + 1, per = nk * nphi, nq = nphi / 2 + 1;
    const int comp[4] = {0, 1, 2, 5};
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : bad)
#endif
    for (long idx = 0; idx < nk * nq; idx++) {
        int k = (int)(idx / nq) - nu;
        int q = (int)(idx % nq);
        if (k == 0 && q == 0) continue;
        int cbad = 0;
        cell_t cell;
        cell_setup(&cell, du, nphi, k, q, rtol, &cbad);
        double dth = 2.0 * cell.half_dphi / ntpz, sum[NC] = {0, 0, 0, 0, 0, 0};
        for (int m = 0; m <= ntpz; m++) {
            double t = (m == ntpz) ? cell.half_dphi : -cell.half_dphi + m * dth;
            double g[NV];
            f_xi(t, &cell, g);
            double w = (m == 0 || m == ntpz) ? 0.5 : 1.0;
            for (int c = 0; c < NC; c++) sum[c] += w * g[c];
        }
        bad += cbad;
        long row = (long)(k + nu) * nphi;
        int qm = (nphi - q) % nphi;
        for (int i = 0; i < 4; i++) {
            int c = comp[i];
            out[c * per + row + q] = sum[c] * dth;
            if (qm != q) out[c * per + row + qm] = (c == 2) ? -sum[c] * dth : sum[c] * dth;
        }
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

/* The inner integral at one outer node t = xi - xi_c (for the tests of the
   quadrature). */
int sgo_inner(double du, int nphi, int k, int q, double t, double rtol, double out[NV])
{
    gl_init();
    int qs = ((q % nphi) + nphi) % nphi;
    if (2 * qs > nphi) qs -= nphi;
    int bad = 0;
    cell_t cell;
    cell_setup(&cell, du, nphi, k, qs, rtol, &bad);
    f_xi(t, &cell, out);
    return bad;
}
