/*
 * lmfmm_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU restatement of the method of Cho & Huang,
 * "Adapting free-space fast multipole method for layered media Green's
 * function: algorithm and analysis" (arXiv:1902.08250), for a three-layer
 * medium (interfaces y = 0 and y = -d, wave numbers k1 | k2 | k3) with sources
 * and targets in the middle layer.  It exists to check the GPU library and is
 * loaded only by the test-suite, the smoke check and the benchmark's CPU
 * baseline leg; the library never links, loads or calls it, and the two share
 * no code.
 *
 * Contents, in the paper's order:
 *   - the branch of sqrt(lambda^2 - k^2)                     (Sec. 3, Eq. (Green))
 *   - image densities: the paper's top-layer-source system and closed forms
 *     (Sec. 3, Example 4) and the middle-layer-source densities obtained from
 *     the same interface conditions (reading R1)
 *   - Sommerfeld integrals on a deformed contour with a north (original) or
 *     east (alternative direction) tail                      (Sec. 2.1, Sec. 4.2, Sec. 5 first contour)
 *   - direct summation (the exact result the FMM approximates) (Eq. (direct_sum))
 *   - a uniform strip-forest quadtree and its interaction lists (Algorithm 1, step 1)
 *   - S2M, M2M, M2L (free space and layered), L2L, L2T, S2T and the FMM driver
 *     (Sec. 2.1 lemmas, Algorithm 1)
 *   - derivatives of the direct sum for gradient checks: the target gradient
 *     (free part through H1, reflected part by i lambda and -s2 dh/dy in the
 *     Sommerfeld integrand) and d/dd (chain rule on sigma_m e^{-s2 h_m})
 *
 * Quadrature: adaptive Gauss-Kronrod (7/15) with a global error estimate.
 * Bessel functions: the C library's jn / yn (a library primitive used as a step).
 */
#define _DEFAULT_SOURCE
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cx;

typedef struct {
    double k1, k2, k3, d;
} orc_medium;

/* ------------------------------------------------------------------------- */
/* Branch of s_j(lambda) = sqrt(lambda^2 - k_j^2) (Sec. 3, Eq. (Green)).      */
/* The paper never states it; the outgoing/decaying choice is                 */
/* s = -i r, r = sqrt(k^2 - lambda^2) with Im r >= 0 (Re r >= 0 if Im r = 0), */
/* i.e. Re s >= 0, s = -i sqrt(k^2 - lambda^2) on the propagating interval.   */
/* ------------------------------------------------------------------------- */
static cx sroot(cx lam, double k)
{
    cx r = csqrt(k * k - lam * lam);
    if (cimag(r) < 0.0 || (cimag(r) == 0.0 && creal(r) < 0.0)) r = -r;
    return -I * r;
}

void orc_sroot(const double *lam, double k, double *out)
{
    cx s = sroot(lam[0] + I * lam[1], k);
    out[0] = creal(s);
    out[1] = cimag(s);
}

/* ------------------------------------------------------------------------- */
/* Paper's three-layer densities for a source in the TOP layer (Example 4):   */
/* the 4x4 system as printed, solved by Gaussian elimination, and the printed */
/* closed forms (sigma_1, sigma_2^t, sigma_2^b, sigma_3).                     */
/* ------------------------------------------------------------------------- */
static int csolve(int n, cx *A, cx *b)
{
    /* Gaussian elimination with partial pivoting; A is n x n row-major. */
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (cabs(A[r * n + c]) > cabs(A[piv * n + c])) piv = r;
        if (cabs(A[piv * n + c]) == 0.0) return -1;
        if (piv != c) {
            for (int j = 0; j < n; ++j) {
                cx t = A[c * n + j];
                A[c * n + j] = A[piv * n + j];
                A[piv * n + j] = t;
            }
            cx t = b[c];
            b[c] = b[piv];
            b[piv] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            cx f = A[r * n + c] / A[c * n + c];
            for (int j = c; j < n; ++j) A[r * n + j] -= f * A[c * n + j];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        cx acc = b[r];
        for (int j = r + 1; j < n; ++j) acc -= A[r * n + j] * b[j];
        b[r] = acc / A[r * n + r];
    }
    return 0;
}

void orc_sigma_paper_solve(const double *lam, double k1, double k2, double k3, double d,
                           double *out)
{
    cx l = lam[0] + I * lam[1];
    cx s1 = sroot(l, k1), s2 = sroot(l, k2), s3 = sroot(l, k3);
    cx e = cexp(-d * s2);
    cx A[16] = {-1.0, s1 / s2, e * s1 / s2, 0.0,
                0.0, e, 1.0, -s2 / s3,
                1.0, 1.0, -e, 0.0,
                0.0, e, -1.0, -1.0};
    cx b[4] = {1.0, 0.0, 1.0, 0.0};
    csolve(4, A, b);
    for (int i = 0; i < 4; ++i) {
        out[2 * i] = creal(b[i]);
        out[2 * i + 1] = cimag(b[i]);
    }
}

/* The printed closed forms, literally (overflow for large |lambda| d). */
void orc_sigma_paper_closed(const double *lam, double k1, double k2, double k3, double d,
                            double *out)
{
    cx l = lam[0] + I * lam[1];
    cx s1 = sroot(l, k1), s2 = sroot(l, k2), s3 = sroot(l, k3);
    cx l2 = l * l, K2 = k2 * k2;
    cx sh = csinh(d * s2), ch = ccosh(d * s2);
    cx den = sh * (l2 + s1 * s3 - K2) + s2 * (s1 + s3) * ch;
    cx sig[4];
    sig[0] = (sh * (-l2 + s1 * s3 + K2) + s2 * (s1 - s3) * ch) / den;
    sig[1] = cexp(d * s2) * (l2 + s2 * s3 - K2) / den;
    sig[2] = -cexp(d * s2) * (-l2 + s2 * s3 + K2) / den;
    sig[3] = 2.0 * s2 * s3 * cexp(d * s3) / den;
    for (int i = 0; i < 4; ++i) {
        out[2 * i] = creal(sig[i]);
        out[2 * i + 1] = cimag(sig[i]);
    }
}

/* sigma_2^t of Example 4 with numerator and denominator divided by e^{d s2}
 * (same function, no overflow). */
static cx sigma2t_safe(cx l, double k1, double k2, double k3, double d)
{
    cx s1 = sroot(l, k1), s2 = sroot(l, k2), s3 = sroot(l, k3);
    cx E = cexp(-2.0 * d * s2);
    cx l2 = l * l, K2 = k2 * k2;
    cx num = l2 + s2 * s3 - K2;
    cx den = 0.5 * (1.0 - E) * (l2 + s1 * s3 - K2) + 0.5 * s2 * (s1 + s3) * (1.0 + E);
    return num / den;
}

void orc_sigma2t_safe(const double *lam, double k1, double k2, double k3, double d, double *out)
{
    cx v = sigma2t_safe(lam[0] + I * lam[1], k1, k2, k3, d);
    out[0] = creal(v);
    out[1] = cimag(v);
}

/* ------------------------------------------------------------------------- */
/* Middle-layer source (reading R1): the reflected spectral field.           */
/* With R_t = (s2-s1)/(s2+s1), R_b = (s2-s3)/(s2+s3), S = 1/(1-R_t R_b e^{-2d s2}):
 *   sigma_tt = R_t S,  sigma_bb = R_b S,  sigma_tb = R_t R_b S, and
 *   g_r^(lambda; y, y0) = [ sigma_tt e^{s2(y+y0)} + sigma_bb e^{-s2(y+y0+2d)}
 *                          + sigma_tb (e^{-s2(2d-(y-y0))} + e^{-s2(2d+(y-y0))}) ] / s2.
 * Each of the four terms has the form of Eq. (Green): exp(-s2 h_m) with
 *   h_tt = -(y+y0), h_bb = y+y0+2d, h_tb = -y+y0+2d, h_bt = y-y0+2d.
 * R_t and R_b are written as (k1^2-k2^2)/(s2+s1)^2 and (k3^2-k2^2)/(s2+s3)^2
 * (the same numbers, without cancellation at large lambda).                 */
/* ------------------------------------------------------------------------- */
/* Other media (Sec. 3, Examples 2 and 3): either interface of the middle
 * layer may instead be a wall with a one-sided condition.  Its reflection
 * coefficient replaces R_t or R_b in the formulas above:
 *   Dirichlet (u = 0): -1;  Neumann (du/dn = 0): +1;
 *   impedance: the image term of Eq. (halfspace), (s2 + i k2 alpha)/(s2 - i k2 alpha)
 *   (reading: the printed image term defines the condition, du/dn - i k2 alpha u = 0
 *   with n the layer's outward normal; it tends to the Dirichlet value as alpha
 *   grows and equals the Neumann value at alpha = 0).
 * The kinds are process-wide settings of the oracle (orc_set_boundaries). */
enum { ORC_BC_TRANSMISSION = 0, ORC_BC_DIRICHLET = 1, ORC_BC_NEUMANN = 2, ORC_BC_IMPEDANCE = 3 };
static int g_bc_kind[2] = {ORC_BC_TRANSMISSION, ORC_BC_TRANSMISSION}; /* top (y = 0), bottom (y = -d) */
static double g_bc_alpha[2] = {0.0, 0.0};
void orc_set_boundaries(int top, double top_alpha, int bottom, double bottom_alpha)
{
    g_bc_kind[0] = top;
    g_bc_alpha[0] = top_alpha;
    g_bc_kind[1] = bottom;
    g_bc_alpha[1] = bottom_alpha;
}
/* reflection coefficient of boundary b (0 top, 1 bottom); kj, sj: the outer layer's */
static cx refl_coef(int b, cx s2, double k2, cx sj, double kj)
{
    switch (g_bc_kind[b]) {
    case ORC_BC_DIRICHLET: return -1.0;
    case ORC_BC_NEUMANN: return 1.0;
    case ORC_BC_IMPEDANCE: {
        cx beta = I * k2 * g_bc_alpha[b];
        return (s2 + beta) / (s2 - beta);
    }
    default: return (kj * kj - k2 * k2) / ((s2 + sj) * (s2 + sj));
    }
}

static void sig_layer2(cx l, const orc_medium *m, cx *s2o, cx sig[3])
{
    cx s1 = sroot(l, m->k1), s2 = sroot(l, m->k2), s3 = sroot(l, m->k3);
    cx Rt = refl_coef(0, s2, m->k2, s1, m->k1);
    cx Rb = refl_coef(1, s2, m->k2, s3, m->k3);
    cx S = 1.0 / (1.0 - Rt * Rb * cexp(-2.0 * m->d * s2));
    sig[0] = Rt * S;
    sig[1] = Rb * S;
    sig[2] = Rt * Rb * S;
    *s2o = s2;
}

void orc_sigma_layer2(const double *lam, double k1, double k2, double k3, double d, double *out)
{
    orc_medium m = {k1, k2, k3, d};
    cx s2, sig[3];
    sig_layer2(lam[0] + I * lam[1], &m, &s2, sig);
    for (int i = 0; i < 3; ++i) {
        out[2 * i] = creal(sig[i]);
        out[2 * i + 1] = cimag(sig[i]);
    }
}

/* term heights h_m(y, y0) and density index; term order tt, bb, tb, bt */
static void term_h(const orc_medium *m, double y, double y0, double h[4])
{
    h[0] = -(y + y0);
    h[1] = y + y0 + 2.0 * m->d;
    h[2] = -y + y0 + 2.0 * m->d;
    h[3] = y - y0 + 2.0 * m->d;
}
static const int term_sig[4] = {0, 1, 2, 2};

void orc_spectral_refl(const double *lam, double k1, double k2, double k3, double d,
                       double y, double y0, double *out)
{
    orc_medium m = {k1, k2, k3, d};
    cx l = lam[0] + I * lam[1], s2, sig[3];
    sig_layer2(l, &m, &s2, sig);
    double h[4];
    term_h(&m, y, y0, h);
    cx acc = 0.0;
    for (int t = 0; t < 4; ++t) acc += sig[term_sig[t]] * cexp(-s2 * h[t]);
    acc /= s2;
    out[0] = creal(acc);
    out[1] = cimag(acc);
}

/* The same spectral field from the interface conditions directly: in layer 2
 * the total field is e^{-s2|y-y0|}/s2 + A e^{s2 y} + B e^{-s2 y}; layer 1 carries
 * C e^{-s1 y}, layer 3 D e^{s3 (y+d)}; the field and its y-derivative are
 * continuous at y = 0 and y = -d (the transmission conditions behind the
 * paper's 4x4 system).  Returns A e^{s2 y} + B e^{-s2 y}. */
void orc_spectral_refl_solve(const double *lam, double k1, double k2, double k3, double d,
                             double y, double y0, double *out)
{
    cx l = lam[0] + I * lam[1];
    cx s1 = sroot(l, k1), s2 = sroot(l, k2), s3 = sroot(l, k3);
    cx up = cexp(s2 * y0);            /* free field at y = 0 is e^{s2 y0}/s2      */
    cx dn = cexp(-s2 * (d + y0));     /* free field at y = -d is e^{-s2(d+y0)}/s2 */
    cx em = cexp(-s2 * d), ep = cexp(s2 * d);
    /* unknowns (A, B, C, D) */
    cx M[16] = {1.0, 1.0, -1.0, 0.0,
                s2, -s2, s1, 0.0,
                em, ep, 0.0, -1.0,
                s2 * em, -s2 * ep, 0.0, -s3};
    cx b[4] = {-up / s2, up, -dn / s2, -dn};
    csolve(4, M, b);
    cx v = b[0] * cexp(s2 * y) + b[1] * cexp(-s2 * y);
    out[0] = creal(v);
    out[1] = cimag(v);
}

/* ------------------------------------------------------------------------- */
/* Adaptive Gauss-Kronrod 7/15 on [a, b] for complex integrands.              */
/* ------------------------------------------------------------------------- */
typedef cx (*cfun)(double t, void *ctx);

static const double gk_x[8] = {
    0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
    0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
    0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
    0.207784955007898467600689403773245, 0.000000000000000000000000000000000};
static const double gk_wk[8] = {
    0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
    0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
    0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
    0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double gk_wg[4] = {
    0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
    0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

static void gk15(cfun f, void *ctx, double a, double b, cx *res, double *err)
{
    double c = 0.5 * (a + b), h = 0.5 * (b - a);
    cx fc = f(c, ctx);
    cx rk = fc * gk_wk[7], rg = fc * gk_wg[3];
    for (int j = 0; j < 7; ++j) {
        double dx = h * gk_x[j];
        cx f1 = f(c - dx, ctx), f2 = f(c + dx, ctx);
        rk += gk_wk[j] * (f1 + f2);
        if (j & 1) rg += gk_wg[j / 2] * (f1 + f2);
    }
    *res = rk * h;
    *err = cabs((rk - rg) * h);
}

#define GK_MAXSEG 4000
/* Returns 0 on convergence, 1 if the segment budget ran out (result is the
 * best estimate).  Error target: max(atol, rtol * |I|), or, when g_l1 is set,
 * max(atol, rtol * sum_i |I_i|) -- relative to the L1 size of the integrand
 * (used where the integral itself cancels to far below its integrand). */
static _Thread_local int g_l1 = 0;
static int gk_adapt(cfun f, void *ctx, double a, double b, int ninit, double atol,
                    double rtol, cx *out)
{
    double *sa = malloc(sizeof(double) * GK_MAXSEG), *sb = malloc(sizeof(double) * GK_MAXSEG);
    double *se = malloc(sizeof(double) * GK_MAXSEG);
    cx *sr = malloc(sizeof(cx) * GK_MAXSEG);
    int n = 0;
    cx tot = 0.0;
    double terr = 0.0;
    for (int i = 0; i < ninit; ++i) {
        sa[n] = a + (b - a) * i / ninit;
        sb[n] = a + (b - a) * (i + 1) / ninit;
        gk15(f, ctx, sa[n], sb[n], &sr[n], &se[n]);
        tot += sr[n];
        terr += se[n];
        ++n;
    }
    int status = 0;
    for (;;) {
        double scale = cabs(tot);
        if (g_l1) {
            scale = 0.0;
            for (int i = 0; i < n; ++i) scale += cabs(sr[i]);
        }
        if (terr <= fmax(atol, rtol * scale)) break;
        if (n + 1 >= GK_MAXSEG) {
            status = 1;
            break;
        }
        int w = 0;
        for (int i = 1; i < n; ++i)
            if (se[i] > se[w]) w = i;
        double m = 0.5 * (sa[w] + sb[w]);
        cx r1, r2;
        double e1, e2;
        gk15(f, ctx, sa[w], m, &r1, &e1);
        gk15(f, ctx, m, sb[w], &r2, &e2);
        sa[n] = m;
        sb[n] = sb[w];
        sr[n] = r2;
        se[n] = e2;
        sb[w] = m;
        sr[w] = r1;
        se[w] = e1;
        ++n;
        tot = 0.0;
        terr = 0.0;
        for (int i = 0; i < n; ++i) {
            tot += sr[i];
            terr += se[i];
        }
    }
    free(sa);
    free(sb);
    free(se);
    free(sr);
    *out = tot;
    return status;
}

static double g_atol = 1e-15, g_rtol = 1e-13;
void orc_set_tolerance(double atol, double rtol)
{
    g_atol = atol;
    g_rtol = rtol;
}

/* test hook for the Kronrod constants: integral of t^n on [a, b] with one GK15 panel */
typedef struct {
    int n;
} powctx;
static cx f_pow(double t, void *c) { return pow(t, ((powctx *)c)->n); }
void orc_gk15_pow(int n, double a, double b, double *out)
{
    powctx c = {n};
    cx r;
    double e;
    gk15(f_pow, &c, a, b, &r, &e);
    out[0] = creal(r);
    out[1] = e;
}

/* ------------------------------------------------------------------------- */
/* Sommerfeld integrals of the form of Eq. (Green) for points at horizontal   */
/* distance X >= 0:                                                           */
/*     (1/4pi) Int_R e^{i lambda X} F(lambda) d lambda,  F even in lambda,    */
/* on the first contour of Sec. 5:                                            */
/*   segment: lambda(t) = t - i a sin(pi t / c), t in [0, c] (the negative   */
/*            half folded onto it, giving 2 cos(lambda X)),                   */
/*   tail:    north: the real axis [c, inf);                                  */
/*            east:  i Int_0^inf [e^{i(c+i tau)X} F(c+i tau)                  */
/*                               - e^{-i(c-i tau)X} F(c-i tau)] d tau         */
/*            (the alternative-direction form, Sec. 4.2 contour argument).   */
/* c = 1.5 max(k) + 1, a = min(0.5, 1/X).                                     */
/* ------------------------------------------------------------------------- */
typedef cx (*specfun)(cx lam, void *ctx); /* F(lambda) */

/* dX = 1 takes d/dX of the integral instead: e^{i lambda X} -> i lambda e^{i lambda X},
 * so 2 cos(lambda X) -> -2 lambda sin(lambda X). */
typedef struct {
    specfun F;
    void *fctx;
    double X, c, a, L;
    int dX;
} contour_ctx;

static cx fold_cos(cx lam, const contour_ctx *c)
{
    return c->dX ? -2.0 * lam * csin(lam * c->X) : 2.0 * ccos(lam * c->X);
}
static cx f_segment(double t, void *vc)
{
    contour_ctx *c = vc;
    double ph = M_PI * t / c->c;
    cx lam = t - I * c->a * sin(ph);
    cx dl = 1.0 - I * c->a * (M_PI / c->c) * cos(ph);
    return fold_cos(lam, c) * c->F(lam, c->fctx) * dl;
}
static cx f_north(double u, void *vc)
{
    contour_ctx *c = vc;
    double t = c->L * u / (1.0 - u), dt = c->L / ((1.0 - u) * (1.0 - u));
    cx lam = c->c + t;
    return fold_cos(lam, c) * c->F(lam, c->fctx) * dt;
}
static cx f_east(double u, void *vc)
{
    contour_ctx *c = vc;
    double tau = c->L * u / (1.0 - u), dt = c->L / ((1.0 - u) * (1.0 - u));
    cx lp = c->c + I * tau, lm = c->c - I * tau;
    cx ep = cexp(I * lp * c->X), em = cexp(-I * lm * c->X);
    if (c->dX) {
        ep *= I * lp;
        em *= -I * lm;
    }
    cx v = I * (ep * c->F(lp, c->fctx) - em * c->F(lm, c->fctx));
    return v * dt;
}

/* tail: 0 = north, 1 = east. rate = decay rate used to scale the tail map. */
static int sommerfeld_x(specfun F, void *fctx, double kmax, double X, int tail, double rate,
                        int do_segment, int do_tail, int dX, cx *out)
{
    contour_ctx c;
    c.F = F;
    c.fctx = fctx;
    c.X = X;
    c.dX = dX;
    c.c = 1.5 * kmax + 1.0;
    c.a = fmin(0.5, 1.0 / fmax(X, 1e-3));
    c.L = 1.0 / (rate + 1.0 / c.c);
    cx seg = 0.0, tl = 0.0;
    int st = 0;
    int nosc = 8 + (int)(c.c * X / M_PI);
    if (nosc > 400) nosc = 400;
    if (do_segment) st |= gk_adapt(f_segment, &c, 0.0, c.c, nosc, g_atol, g_rtol, &seg);
    if (do_tail) {
        if (tail == 0)
            st |= gk_adapt(f_north, &c, 0.0, 1.0, 16, g_atol, g_rtol, &tl);
        else
            st |= gk_adapt(f_east, &c, 0.0, 1.0, 16, g_atol, g_rtol, &tl);
    }
    *out = (seg + tl) / (4.0 * M_PI);
    return st;
}
static int sommerfeld(specfun F, void *fctx, double kmax, double X, int tail, double rate,
                      int do_segment, int do_tail, cx *out)
{
    return sommerfeld_x(F, fctx, kmax, X, tail, rate, do_segment, do_tail, 0, out);
}

/* --- free space: F = e^{-s|Y|}/s; equals (i/4) H0^(1)(k r) (Example 1) --- */
typedef struct {
    double k, Y;
} free_ctx;
static cx F_free(cx l, void *v)
{
    free_ctx *f = v;
    cx s = sroot(l, f->k);
    return cexp(-s * fabs(f->Y)) / s;
}
int orc_sommerfeld_free(double k, double X, double Y, int tail, double *out)
{
    free_ctx f = {k, Y};
    cx r;
    int st = sommerfeld(F_free, &f, k, fabs(X), tail, tail == 0 ? fabs(Y) : fabs(X), 1, 1, &r);
    out[0] = creal(r);
    out[1] = cimag(r);
    return st;
}

/* --- Dirichlet half space (Example 2): sigma = -1, image at (x0, -y0) --- */
typedef struct {
    double k, h;
} dir_ctx;
static cx F_dirichlet(cx l, void *v)
{
    dir_ctx *f = v;
    cx s = sroot(l, f->k);
    return -cexp(-s * f->h) / s;
}
int orc_dirichlet(double k, double x, double y, double x0, double y0, int tail, double *out)
{
    dir_ctx f = {k, y + y0};
    double X = fabs(x - x0);
    cx r;
    int st = sommerfeld(F_dirichlet, &f, k, X, tail, tail == 0 ? f.h : X, 1, 1, &r);
    out[0] = creal(r);
    out[1] = cimag(r);
    return st;
}

/* --- paper's literal g_2^t (Example 4): top-layer source y0 > 0, target in layer 2 --- */
typedef struct {
    orc_medium m;
    double y, y0;
} g2t_ctx;
static cx F_g2t(cx l, void *v)
{
    g2t_ctx *g = v;
    cx s1 = sroot(l, g->m.k1), s2 = sroot(l, g->m.k2);
    return cexp(s2 * g->y - s1 * g->y0) * sigma2t_safe(l, g->m.k1, g->m.k2, g->m.k3, g->m.d) / s2;
}
int orc_g2t_paper(double k1, double k2, double k3, double d, double x, double y, double x0,
                  double y0, int tail, double *out)
{
    g2t_ctx g = {{k1, k2, k3, d}, y, y0};
    double X = fabs(x - x0), h = y0 - y;
    double km = fmax(k1, fmax(k2, k3));
    cx r;
    int st = sommerfeld(F_g2t, &g, km, X, tail, tail == 0 ? h : X, 1, 1, &r);
    out[0] = creal(r);
    out[1] = cimag(r);
    return st;
}

/* --- Example 4 as printed, layer-1 source (y0 > 0): the cross-layer fields --- */
/* Closed forms of sigma_1, sigma_2^t, sigma_2^b with numerator and denominator
 * divided by e^{d s2} / 2 (the same functions, no overflow):
 *   D' = (1 - E)(lambda^2 + s1 s3 - k2^2) + s2 (s1 + s3)(1 + E),  E = e^{-2 d s2}
 *   sigma_1   = [(1 - E)(-lambda^2 + s1 s3 + k2^2) + s2 (s1 - s3)(1 + E)] / D'
 *   sigma_2^t = 2 (lambda^2 + s2 s3 - k2^2) / D'
 *   sigma_2^b = -2 (-lambda^2 + s2 s3 + k2^2) / D'                            */
static void sigma_cross_safe(cx l, const orc_medium *m, cx *s1o, cx *s2o, cx sig[3])
{
    cx s1 = sroot(l, m->k1), s2 = sroot(l, m->k2), s3 = sroot(l, m->k3);
    cx E = cexp(-2.0 * m->d * s2);
    cx l2 = l * l, K2 = m->k2 * m->k2;
    cx den = (1.0 - E) * (l2 + s1 * s3 - K2) + s2 * (s1 + s3) * (1.0 + E);
    sig[0] = ((1.0 - E) * (-l2 + s1 * s3 + K2) + s2 * (s1 - s3) * (1.0 + E)) / den;
    sig[1] = 2.0 * (l2 + s2 * s3 - K2) / den;
    sig[2] = -2.0 * (-l2 + s2 * s3 + K2) / den;
    *s1o = s1;
    *s2o = s2;
}

/* which = bit 0: g_2^t, bit 1: g_2^b (target in layer 2), bit 2: g_1^s (target in
 * layer 1); dy = 1 takes d/dy (target) inside the integrand */
typedef struct {
    orc_medium m;
    double y, y0;
    int which, dy;
} cross_ctx;
static cx F_cross(cx l, void *v)
{
    cross_ctx *c = v;
    cx s1, s2, sig[3];
    sigma_cross_safe(l, &c->m, &s1, &s2, sig);
    cx acc = 0.0, src = cexp(-s1 * c->y0);
    if (c->which & 1) acc += (c->dy ? s2 : 1.0) * cexp(s2 * c->y) * sig[1] / s2;
    if (c->which & 2) acc += (c->dy ? -s2 : 1.0) * cexp(-s2 * (c->y + 2.0 * c->m.d)) * sig[2] / s2;
    if (c->which & 4) acc += (c->dy ? -s1 : 1.0) * cexp(-s1 * c->y) * sig[0] / s1;
    return acc * src;
}
/* the printed fields of Example 4 by the Sommerfeld quadrature of this file;
 * the tail decays like e^{-lambda h}, h = y0 - y (layer 2) or y0 + y (layer 1) */
static int cross_field(const orc_medium *m, double x, double y, double x0, double y0, int which, int dy,
                       cx *out)
{
    cross_ctx c = {*m, y, y0, which, dy};
    double X = fabs(x - x0), h = (which & 4) ? y0 + y : y0 - y;
    double km = fmax(m->k1, fmax(m->k2, m->k3));
    g_l1 = 1;
    int st = sommerfeld(F_cross, &c, km, X, h >= X ? 0 : 1, h >= X ? h : X, 1, 1, out);
    g_l1 = 0;
    return st;
}
int orc_cross_field(double k1, double k2, double k3, double d, double x, double y, double x0, double y0,
                    int which, int dy, double *out)
{
    orc_medium m = {k1, k2, k3, d};
    cx r;
    int st = cross_field(&m, x, y, x0, y0, which, dy, &r);
    out[0] = creal(r);
    out[1] = cimag(r);
    return st;
}

/* Direct sum of the cross-layer operator: sources (xs, ys) in layer 1
 * (0 < ys), targets (xt, yt) in layer 2:  u_i = sum_j q_j (g_2^t + g_2^b)(x_i, x_j).
 * q: [nvec][ns]; u: [nvec][ntgt] at targets tgt[] (NULL = all nt). */
int orc_cross_direct(double k1, double k2, double k3, double d, int64_t ns, const double *xs,
                     const double *ys, int64_t nt, const double *xt, const double *yt, int nvec,
                     const double *q, int64_t ntgt, const int64_t *tgt, int nthreads, double *u)
{
    orc_medium m = {k1, k2, k3, d};
    const cx *Q = (const cx *)q;
    cx *U = (cx *)u;
    int64_t n = tgt ? ntgt : nt;
    int fail = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 1) reduction(| : fail)
    for (int64_t ii = 0; ii < n; ++ii) {
        int64_t i = tgt ? tgt[ii] : ii;
        cx *acc = calloc(nvec, sizeof(cx));
        for (int64_t j = 0; j < ns; ++j) {
            cx g;
            fail |= cross_field(&m, xt[i], yt[i], xs[j], ys[j], 3, 0, &g);
            for (int v = 0; v < nvec; ++v) acc[v] += g * Q[(int64_t)v * ns + j];
        }
        for (int v = 0; v < nvec; ++v) U[(int64_t)v * n + ii] = acc[v];
        free(acc);
    }
    return fail;
}

/* --- middle-layer reflected field, any subset of the four terms --- */
/* Derivatives of each term sigma_m(lambda; d) e^{-s2 h_m} / s2, by the chain rule:
 *   d/dy (target):  -s2 (dh_m/dy) sigma_m e^{-s2 h_m}/s2
 *   d/dd:           [d sigma_m/dd - s2 (dh_m/dd) sigma_m] e^{-s2 h_m}/s2
 * with dh/dy = (-1, +1, -1, +1) and dh/dd = (0, 2, 2, 2) for (tt, bb, tb, bt);
 * d/dx (target) is taken on the contour (dX) times sign(x - x0).           */
enum { ORC_VALUE = 0, ORC_DX = 1, ORC_DY = 2, ORC_DD = 3 };
static const double dh_dy[4] = {-1.0, 1.0, -1.0, 1.0};
static const double dh_dd[4] = {0.0, 2.0, 2.0, 2.0};

/* d sigma_m / dd at fixed lambda: only S = 1/D, D = 1 - R_t R_b e^{-2 d s2}, depends on d,
 * dS/dd = -(dD/dd) S^2 = -2 s2 R_t R_b e^{-2 d s2} S^2. */
static void sig_layer2_dd(cx l, const orc_medium *m, cx dsig[3])
{
    cx s1 = sroot(l, m->k1), s2 = sroot(l, m->k2), s3 = sroot(l, m->k3);
    cx Rt = refl_coef(0, s2, m->k2, s1, m->k1);
    cx Rb = refl_coef(1, s2, m->k2, s3, m->k3);
    cx E = Rt * Rb * cexp(-2.0 * m->d * s2);
    cx S = 1.0 / (1.0 - E);
    cx dS = -2.0 * s2 * E * S * S;
    dsig[0] = Rt * dS;
    dsig[1] = Rb * dS;
    dsig[2] = Rt * Rb * dS;
}

typedef struct {
    orc_medium m;
    double h[4];
    int mask, deriv;
} refl_ctx;
static cx F_refl(cx l, void *v)
{
    refl_ctx *r = v;
    cx s2, sig[3], dsig[3];
    sig_layer2(l, &r->m, &s2, sig);
    if (r->deriv == ORC_DD) sig_layer2_dd(l, &r->m, dsig);
    cx acc = 0.0;
    for (int t = 0; t < 4; ++t) {
        if (!(r->mask & (1 << t))) continue;
        cx e = cexp(-s2 * r->h[t]), sg = sig[term_sig[t]];
        if (r->deriv == ORC_DY)
            acc += -s2 * dh_dy[t] * sg * e;
        else if (r->deriv == ORC_DD)
            acc += (dsig[term_sig[t]] - s2 * dh_dd[t] * sg) * e;
        else
            acc += sg * e;
    }
    return acc / s2;
}

/* tailmode: -1 = per term (north if h_m >= X, else east), 0 = all north, 1 = all east */
static int green_refl_x(const orc_medium *m, double x, double y, double x0, double y0, int mask,
                        int tailmode, int deriv, cx *out)
{
    refl_ctx r;
    r.m = *m;
    term_h(m, y, y0, r.h);
    double X = fabs(x - x0);
    double km = fmax(m->k1, fmax(m->k2, m->k3));
    int st = 0;
    cx seg = 0.0;
    r.mask = mask;
    r.deriv = deriv;
    const int dX = deriv == ORC_DX;
    /* the four terms can cancel in the sum: measure the error against the
     * integrand's L1 size, not against the (possibly much smaller) integral */
    g_l1 = 1;
    st |= sommerfeld_x(F_refl, &r, km, X, 0, 0.0, 1, 0, dX, &seg);
    cx tails = 0.0;
    for (int dir = 0; dir < 2; ++dir) {
        int sub = 0;
        double hmin = 1e300;
        for (int t = 0; t < 4; ++t) {
            if (!(mask & (1 << t))) continue;
            int east = (tailmode == -1) ? (r.h[t] < X) : tailmode;
            if (east == dir) {
                sub |= 1 << t;
                hmin = fmin(hmin, r.h[t]);
            }
        }
        if (!sub) continue;
        r.mask = sub;
        cx tl;
        st |= sommerfeld_x(F_refl, &r, km, X, dir, dir == 0 ? hmin : X, 0, 1, dX, &tl);
        tails += tl;
    }
    g_l1 = 0;
    *out = seg + tails;
    if (dX) *out *= (x > x0) ? 1.0 : (x < x0 ? -1.0 : 0.0);
    return st;
}
static int green_refl(const orc_medium *m, double x, double y, double x0, double y0, int mask,
                      int tailmode, cx *out)
{
    return green_refl_x(m, x, y, x0, y0, mask, tailmode, ORC_VALUE, out);
}

/* d/dx, d/dy (target) or d/dd of G_r; deriv = 1, 2, 3 */
int orc_green_refl_deriv(double k1, double k2, double k3, double d, double x, double y, double x0,
                         double y0, int mask, int deriv, double *out)
{
    orc_medium m = {k1, k2, k3, d};
    cx r;
    int st = green_refl_x(&m, x, y, x0, y0, mask, -1, deriv, &r);
    out[0] = creal(r);
    out[1] = cimag(r);
    return st;
}

int orc_green_refl(double k1, double k2, double k3, double d, double x, double y, double x0,
                   double y0, int mask, int tailmode, double *out)
{
    orc_medium m = {k1, k2, k3, d};
    cx r;
    int st = green_refl(&m, x, y, x0, y0, mask, tailmode, &r);
    out[0] = creal(r);
    out[1] = cimag(r);
    return st;
}

/* free-space part (i/4) H0^(1)(k r) (Example 1) */
static cx green_free(double k, double r) { return 0.25 * I * (j0(k * r) + I * y0(k * r)); }
/* its target gradient: d/dr H0^(1)(k r) = -k H1^(1)(k r), times (dx, dy)/r */
static void green_free_grad(double k, double dx, double dy, cx *gx, cx *gy)
{
    double r = hypot(dx, dy);
    cx dr = 0.25 * I * (-k) * (j1(k * r) + I * y1(k * r));
    *gx = dr * (dx / r);
    *gy = dr * (dy / r);
}
void orc_green_free_grad(double k, double dx, double dy, double *out)
{
    cx gx, gy;
    green_free_grad(k, dx, dy, &gx, &gy);
    out[0] = creal(gx);
    out[1] = cimag(gx);
    out[2] = creal(gy);
    out[3] = cimag(gy);
}

/* ------------------------------------------------------------------------- */
/* Direct summation (Eq. (direct_sum)) for targets = sources = the points:    */
/*   u_i = sum_{j != i} q_j (i/4) H0(k2 |x_i - x_j|) + sum_j q_j G_r(x_i, x_j)*/
/* q, u: [nvec][n] complex (interleaved re/im). Only targets listed in tgt    */
/* (ntgt of them; NULL = all) are written, u laid out [nvec][ntgt].           */
/* ------------------------------------------------------------------------- */
int orc_direct_apply(double k1, double k2, double k3, double d, int64_t n, const double *x,
                     const double *y, int nvec, const double *q, int64_t ntgt,
                     const int64_t *tgt, int refl_mask, int nthreads, double *u)
{
    orc_medium m = {k1, k2, k3, d};
    const cx *Q = (const cx *)q;
    cx *U = (cx *)u;
    int64_t nt = tgt ? ntgt : n;
    int fail = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 1) reduction(| : fail)
    for (int64_t ii = 0; ii < nt; ++ii) {
        int64_t i = tgt ? tgt[ii] : ii;
        cx *acc = calloc(nvec, sizeof(cx));
        for (int64_t j = 0; j < n; ++j) {
            cx g = 0.0;
            if (j != i) {
                double r = hypot(x[i] - x[j], y[i] - y[j]);
                g += green_free(m.k2, r);
            }
            if (refl_mask) {
                cx gr;
                fail |= green_refl(&m, x[i], y[i], x[j], y[j], refl_mask, -1, &gr);
                g += gr;
            }
            for (int v = 0; v < nvec; ++v) acc[v] += g * Q[(int64_t)v * n + j];
        }
        for (int v = 0; v < nvec; ++v) U[(int64_t)v * nt + ii] = acc[v];
        free(acc);
    }
    return fail;
}

/* Derivatives of the direct sum (Eq. (direct_sum)) at the listed targets:
 *   deriv 1, 2: d/dx_i, d/dy_i of u_i with the sources held fixed
 *               (free part over j != i, reflected part over all j);
 *   deriv 3:    d/dd of u_i (reflected part only; the free part has no d).
 * Layouts as orc_direct_apply. */
int orc_direct_apply_deriv(double k1, double k2, double k3, double d, int64_t n, const double *x,
                           const double *y, int nvec, const double *q, int64_t ntgt,
                           const int64_t *tgt, int deriv, int nthreads, double *u)
{
    orc_medium m = {k1, k2, k3, d};
    const cx *Q = (const cx *)q;
    cx *U = (cx *)u;
    int64_t nt = tgt ? ntgt : n;
    int fail = 0;
    if (deriv < ORC_DX || deriv > ORC_DD) return 2;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#endif
#pragma omp parallel for schedule(dynamic, 1) reduction(| : fail)
    for (int64_t ii = 0; ii < nt; ++ii) {
        int64_t i = tgt ? tgt[ii] : ii;
        cx *acc = calloc(nvec, sizeof(cx));
        for (int64_t j = 0; j < n; ++j) {
            cx g = 0.0;
            if (j != i && deriv != ORC_DD) {
                cx gx, gy;
                green_free_grad(m.k2, x[i] - x[j], y[i] - y[j], &gx, &gy);
                g += deriv == ORC_DX ? gx : gy;
            }
            cx gr;
            fail |= green_refl_x(&m, x[i], y[i], x[j], y[j], 15, -1, deriv, &gr);
            g += gr;
            for (int v = 0; v < nvec; ++v) acc[v] += g * Q[(int64_t)v * n + j];
        }
        for (int v = 0; v < nvec; ++v) U[(int64_t)v * nt + ii] = acc[v];
        free(acc);
    }
    return fail;
}

/* ------------------------------------------------------------------------- */
/* Tree (Algorithm 1 step 1; readings G11): a forest of R roots, each a d x d */
/* square, tiling [x_origin, x_origin + R d) x (-d, 0), refined uniformly to  */
/* depth L.  Level l has ncol = R 2^l columns and nrow = 2^l rows of width   */
/* w = d 2^-l; row 0 touches y = 0.  Box id = row * ncol + col.              */
/* x_origin = floor(min x / d) d, R = floor(max x / d) - floor(min x / d) + 1.*/
/* A point's leaf: col = floor((x - x_origin)/w_L), row = floor(-y / w_L),    */
/* clamped to the grid.  Points are ordered by (leaf id, input index).       */
/* ------------------------------------------------------------------------- */
typedef struct {
    double d, x0;
    int R, L;
} orc_grid;

static void make_grid(int64_t n, const double *x, double d, int L, orc_grid *g)
{
    double mn = x[0], mx = x[0];
    for (int64_t i = 1; i < n; ++i) {
        mn = fmin(mn, x[i]);
        mx = fmax(mx, x[i]);
    }
    double f0 = floor(mn / d), f1 = floor(mx / d);
    g->d = d;
    g->x0 = f0 * d;
    g->R = (int)(f1 - f0) + 1;
    g->L = L;
}

static int64_t leaf_of(const orc_grid *g, double x, double y)
{
    double w = ldexp(g->d, -g->L);
    int64_t ncol = (int64_t)g->R << g->L, nrow = (int64_t)1 << g->L;
    int64_t c = (int64_t)floor((x - g->x0) / w), r = (int64_t)floor(-y / w);
    if (c < 0) c = 0;
    if (c > ncol - 1) c = ncol - 1;
    if (r < 0) r = 0;
    if (r > nrow - 1) r = nrow - 1;
    return r * ncol + c;
}

typedef struct {
    int64_t key, idx;
} kv;
static int kv_cmp(const void *a, const void *b)
{
    const kv *p = a, *q = b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    return p->idx < q->idx ? -1 : (p->idx > q->idx);
}

/* outputs: hdr = {x_origin, R}, perm[n] (tree position -> input index),
 * leaf_start[nleaf + 1] */
int orc_tree_build(int64_t n, const double *x, const double *y, double d, int L, double *hdr,
                   int64_t *perm, int64_t *leaf_start)
{
    orc_grid g;
    make_grid(n, x, d, L, &g);
    int64_t nleaf = ((int64_t)g.R << L) << L;
    kv *a = malloc(sizeof(kv) * n);
    for (int64_t i = 0; i < n; ++i) {
        a[i].key = leaf_of(&g, x[i], y[i]);
        a[i].idx = i;
    }
    qsort(a, n, sizeof(kv), kv_cmp);
    for (int64_t b = 0; b <= nleaf; ++b) leaf_start[b] = 0;
    for (int64_t i = 0; i < n; ++i) {
        perm[i] = a[i].idx;
        leaf_start[a[i].key + 1]++;
    }
    for (int64_t b = 0; b < nleaf; ++b) leaf_start[b + 1] += leaf_start[b];
    hdr[0] = g.x0;
    hdr[1] = g.R;
    free(a);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* Interaction lists.  Terms: 0 = free space, 1 = tt, 2 = bb, 3 = tb, 4 = bt.  */
/* The image of a source box (row r, level with nrow rows) is the box of the  */
/* same column in image row:  tt: -1-r (mirror in y = 0);  bb: 2 nrow-1-r     */
/* (mirror in y = -d);  tb: r - 2 nrow (shift by +2d);  bt: r + 2 nrow        */
/* (shift by -2d).  For the free term the "image" is the box itself.  The     */
/* standard FMM rules are applied between the target box and the image:     */
/*   V list (level l): image not adjacent to target, and (l = 0 or the        */
/*          parents are adjacent);                                            */
/*   U list (leaf level): image adjacent to target (free: includes itself).   */
/* Two boxes are adjacent when both column and row differ by at most one.    */
/* Entry order: by target box id, then term, then source box id.             */
/* ------------------------------------------------------------------------- */
static int64_t img_row(int term, int64_t r, int64_t nrow)
{
    switch (term) {
    case 0: return r;
    case 1: return -1 - r;
    case 2: return 2 * nrow - 1 - r;
    case 3: return r - 2 * nrow;
    default: return r + 2 * nrow;
    }
}
static int64_t fdiv2(int64_t a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }
static int adjacent(int64_t c1, int64_t r1, int64_t c2, int64_t r2)
{
    return llabs(c1 - c2) <= 1 && llabs(r1 - r2) <= 1;
}

/* V list at level l; writes up to cap entries of (target, term, source);
 * returns the count (or the count needed when cap is too small). */
int64_t orc_vlist(int R, int l, int64_t cap, int64_t *out)
{
    int64_t ncol = (int64_t)R << l, nrow = (int64_t)1 << l, cnt = 0;
    for (int64_t rt = 0; rt < nrow; ++rt)
        for (int64_t ct = 0; ct < ncol; ++ct)
            for (int term = 0; term < 5; ++term)
                for (int64_t rs = 0; rs < nrow; ++rs)
                    for (int64_t cs = 0; cs < ncol; ++cs) {
                        int64_t ri = img_row(term, rs, nrow);
                        if (adjacent(ct, rt, cs, ri)) continue;
                        if (l > 0 && !adjacent(ct / 2, fdiv2(rt), cs / 2, fdiv2(ri))) continue;
                        if (cnt < cap) {
                            out[3 * cnt] = rt * ncol + ct;
                            out[3 * cnt + 1] = term;
                            out[3 * cnt + 2] = rs * ncol + cs;
                        }
                        ++cnt;
                    }
    return cnt;
}

/* U list at the leaf level L */
int64_t orc_ulist(int R, int L, int64_t cap, int64_t *out)
{
    int64_t ncol = (int64_t)R << L, nrow = (int64_t)1 << L, cnt = 0;
    for (int64_t rt = 0; rt < nrow; ++rt)
        for (int64_t ct = 0; ct < ncol; ++ct)
            for (int term = 0; term < 5; ++term)
                for (int64_t rs = 0; rs < nrow; ++rs)
                    for (int64_t cs = 0; cs < ncol; ++cs) {
                        if (!adjacent(ct, rt, cs, img_row(term, rs, nrow))) continue;
                        if (cnt < cap) {
                            out[3 * cnt] = rt * ncol + ct;
                            out[3 * cnt + 1] = term;
                            out[3 * cnt + 2] = rs * ncol + cs;
                        }
                        ++cnt;
                    }
    return cnt;
}

/* ------------------------------------------------------------------------- */
/* Adaptive tree (Algorithm 1, step 1: "an adaptive hierarchical tree").     */
/* Reading: the strip forest of d x d roots as for the uniform tree; a box    */
/* (level l, column c, row r) holding more than s points with l < Lmax is     */
/* split into its four children (all four exist, empty or not).  A point's   */
/* cell at level l is (floor((x - x0)/w_l), floor(-y/w_l)), clamped, as       */
/* before.  Boxes are numbered level by level and, within a level, by         */
/* r * ncol_l + c.  Points are ordered by the number of their leaf, then by   */
/* input index; boxes that are not leaves own no points.                      */
/*                                                                            */
/* Lists by dual traversal, per term m (0 free, 1 tt, 2 bb, 3 tb, 4 bt), from */
/* every pair of roots.  A target box t and the image of a source box s (its  */
/* row mapped as for the uniform lists, at the source's level) are well       */
/* separated when the larger of |dx|, |dy| between their centres is at least  */
/* w_t + w_s: then (t, m, s) is a V entry (M2L).  Otherwise two leaves give a */
/* U entry (direct); otherwise the larger box is split -- never a leaf; both  */
/* when the levels are equal -- and the traversal goes on with the child      */
/* pairs.  On a uniform tree this is exactly the uniform V and U lists.       */
/* ------------------------------------------------------------------------- */
typedef struct {
    int level;
    int64_t col, row, npts;
    int leaf;
} orc_abox;

typedef struct {
    orc_grid g; /* d, x0, R */
    int Lmax;
    int64_t nbox, *lev_start; /* boxes of level l: [lev_start[l], lev_start[l + 1]) */
    orc_abox *box;
} orc_atree;

static int64_t a_key(const orc_atree *T, int l, int64_t c, int64_t r) { return r * ((int64_t)T->g.R << l) + c; }

/* id of box (l, c, r), or -1 */
static int64_t a_find(const orc_atree *T, int l, int64_t c, int64_t r)
{
    if (l > T->Lmax) return -1;
    int64_t a = T->lev_start[l], b = T->lev_start[l + 1] - 1, key = a_key(T, l, c, r);
    while (a <= b) {
        int64_t mid = (a + b) / 2, k = a_key(T, l, T->box[mid].col, T->box[mid].row);
        if (k == key) return mid;
        if (k < key) a = mid + 1;
        else b = mid - 1;
    }
    return -1;
}

static void a_cell(const orc_grid *g, int l, double x, double y, int64_t *c, int64_t *r)
{
    double w = ldexp(g->d, -l);
    int64_t ncol = (int64_t)g->R << l, nrow = (int64_t)1 << l;
    *c = (int64_t)floor((x - g->x0) / w);
    *r = (int64_t)floor(-y / w);
    if (*c < 0) *c = 0;
    if (*c > ncol - 1) *c = ncol - 1;
    if (*r < 0) *r = 0;
    if (*r > nrow - 1) *r = nrow - 1;
}

static void atree_build(int64_t n, const double *x, const double *y, double d, int s, int Lmax, orc_atree *T)
{
    make_grid(n, x, d, 0, &T->g);
    T->Lmax = Lmax;
    int64_t cap = 64 + 8 * (int64_t)T->g.R, nb = 0;
    T->box = malloc(sizeof(orc_abox) * cap);
    T->lev_start = calloc(Lmax + 2, sizeof(int64_t));
    for (int64_t c = 0; c < T->g.R; ++c) {
        orc_abox b = {0, c, 0, 0, 1};
        T->box[nb++] = b;
    }
    T->lev_start[1] = nb;
    for (int l = 0; l <= Lmax; ++l) {
        const int64_t lo = T->lev_start[l], hi = T->lev_start[l + 1];
        for (int64_t i = 0; i < n; ++i) { /* count each point in its box of this level, if present */
            int64_t c, r;
            a_cell(&T->g, l, x[i], y[i], &c, &r);
            int64_t b = a_find(T, l, c, r);
            if (b >= 0) T->box[b].npts++;
        }
        if (l == Lmax) break;
        int64_t first = nb;
        for (int64_t b = lo; b < hi; ++b) {
            if (T->box[b].npts <= s) continue;
            T->box[b].leaf = 0;
            for (int k = 0; k < 4; ++k) {
                if (nb == cap) {
                    cap *= 2;
                    T->box = realloc(T->box, sizeof(orc_abox) * cap);
                }
                orc_abox ch = {l + 1, 2 * T->box[b].col + (k & 1), 2 * T->box[b].row + (k >> 1), 0, 1};
                T->box[nb++] = ch;
            }
        }
        const int64_t m = nb - first, ncol1 = (int64_t)T->g.R << (l + 1);
        kv *ord = malloc(sizeof(kv) * (m ? m : 1));
        orc_abox *tmp = malloc(sizeof(orc_abox) * (m ? m : 1));
        for (int64_t i = 0; i < m; ++i) {
            ord[i].key = T->box[first + i].row * ncol1 + T->box[first + i].col;
            ord[i].idx = first + i;
        }
        qsort(ord, m, sizeof(kv), kv_cmp);
        for (int64_t i = 0; i < m; ++i) tmp[i] = T->box[ord[i].idx];
        memcpy(T->box + first, tmp, sizeof(orc_abox) * m);
        free(tmp);
        free(ord);
        T->lev_start[l + 2] = nb;
    }
    T->nbox = nb;
}

/* separation of target t and the image of source s under term m, in units of half
 * the finest width of the pair: centres (2c + 1) S, S = 2^(lmax - l), image rows */
static int a_separated(const orc_atree *T, int64_t t, int64_t s, int m)
{
    const orc_abox *A = &T->box[t], *B = &T->box[s];
    int lm = A->level > B->level ? A->level : B->level;
    int64_t SA = (int64_t)1 << (lm - A->level), SB = (int64_t)1 << (lm - B->level);
    int64_t ri = img_row(m, B->row, (int64_t)1 << B->level);
    int64_t X2 = llabs((2 * A->col + 1) * SA - (2 * B->col + 1) * SB);
    int64_t Y2 = llabs((2 * A->row + 1) * SA - (2 * ri + 1) * SB);
    int64_t M2 = X2 > Y2 ? X2 : Y2;
    return M2 >= 2 * (SA + SB);
}

typedef struct {
    int64_t *rows, cnt, cap;
} a_list;
static void a_push(a_list *L, int64_t t, int m, int64_t s)
{
    if (L->cnt == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 1024;
        L->rows = realloc(L->rows, sizeof(int64_t) * 3 * L->cap);
    }
    L->rows[3 * L->cnt] = t;
    L->rows[3 * L->cnt + 1] = m;
    L->rows[3 * L->cnt + 2] = s;
    L->cnt++;
}
static int64_t a_child(const orc_atree *T, int64_t b, int k)
{
    const orc_abox *B = &T->box[b];
    return a_find(T, B->level + 1, 2 * B->col + (k & 1), 2 * B->row + (k >> 1));
}
static void a_visit(const orc_atree *T, int64_t t, int64_t s, int m, a_list *V, a_list *U)
{
    if (a_separated(T, t, s, m)) {
        a_push(V, t, m, s);
        return;
    }
    const orc_abox *A = &T->box[t], *B = &T->box[s];
    if (A->leaf && B->leaf) {
        a_push(U, t, m, s);
        return;
    }
    if (A->leaf || (!B->leaf && B->level < A->level)) {
        for (int k = 0; k < 4; ++k) a_visit(T, t, a_child(T, s, k), m, V, U);
    } else if (B->leaf || A->level < B->level) {
        for (int k = 0; k < 4; ++k) a_visit(T, a_child(T, t, k), s, m, V, U);
    } else {
        for (int k = 0; k < 4; ++k)
            for (int j = 0; j < 4; ++j) a_visit(T, a_child(T, t, k), a_child(T, s, j), m, V, U);
    }
}
typedef struct {
    int64_t a, b, c;
} i3;
static int i3_cmp(const void *p, const void *q)
{
    const i3 *u = p, *v = q;
    if (u->a != v->a) return u->a < v->a ? -1 : 1;
    if (u->b != v->b) return u->b < v->b ? -1 : 1;
    return u->c < v->c ? -1 : (u->c > v->c);
}
static void a_sort(a_list *L)
{
    qsort(L->rows, L->cnt, sizeof(i3), i3_cmp);
}

/* Tree: returns the box count (or -1 if cap is too small); boxes[nbox][4] =
 * (level, col, row, leaf); hdr = {x_origin, R}; perm[n] (position -> input
 * index); pstart[nbox + 1] (points of box b: [pstart[b], pstart[b + 1])). */
int64_t orc_adaptive_tree(int64_t n, const double *x, const double *y, double d, int s, int Lmax, int64_t cap,
                          double *hdr, int64_t *boxes, int64_t *perm, int64_t *pstart)
{
    orc_atree T;
    atree_build(n, x, y, d, s, Lmax, &T);
    int64_t nb = T.nbox;
    if (nb <= cap) {
        for (int64_t b = 0; b < nb; ++b) {
            boxes[4 * b] = T.box[b].level;
            boxes[4 * b + 1] = T.box[b].col;
            boxes[4 * b + 2] = T.box[b].row;
            boxes[4 * b + 3] = T.box[b].leaf;
        }
        /* leaf of each point: descend from its root */
        kv *a = malloc(sizeof(kv) * (n ? n : 1));
        for (int64_t i = 0; i < n; ++i) {
            int64_t b = -1;
            for (int l = 0; l <= Lmax; ++l) {
                int64_t c, r;
                a_cell(&T.g, l, x[i], y[i], &c, &r);
                b = a_find(&T, l, c, r);
                if (T.box[b].leaf) break;
            }
            a[i].key = b;
            a[i].idx = i;
        }
        qsort(a, n, sizeof(kv), kv_cmp);
        for (int64_t b = 0; b <= nb; ++b) pstart[b] = 0;
        for (int64_t i = 0; i < n; ++i) {
            perm[i] = a[i].idx;
            pstart[a[i].key + 1]++;
        }
        for (int64_t b = 0; b < nb; ++b) pstart[b + 1] += pstart[b];
        free(a);
        hdr[0] = T.g.x0;
        hdr[1] = T.g.R;
    }
    free(T.box);
    free(T.lev_start);
    return nb <= cap ? nb : -1;
}

/* Lists: which = 0 (V) or 1 (U); rows (target, term, source) sorted; returns the
 * count (rows written only if count <= cap). */
int64_t orc_adaptive_lists(int64_t n, const double *x, const double *y, double d, int s, int Lmax, int which,
                           int64_t cap, int64_t *out)
{
    orc_atree T;
    atree_build(n, x, y, d, s, Lmax, &T);
    a_list V = {0, 0, 0}, U = {0, 0, 0};
    for (int64_t t = 0; t < T.g.R; ++t)
        for (int64_t sb = 0; sb < T.g.R; ++sb)
            for (int m = 0; m < 5; ++m) a_visit(&T, t, sb, m, &V, &U);
    a_list *L = which ? &U : &V;
    a_sort(L);
    int64_t cnt = L->cnt;
    if (cnt <= cap) memcpy(out, L->rows, sizeof(int64_t) * 3 * cnt);
    free(V.rows);
    free(U.rows);
    free(T.box);
    free(T.lev_start);
    return cnt;
}

/* ------------------------------------------------------------------------- */
/* Expansions (Sec. 2.1).  Orders -p..p, stored at index p + P0 (P0 = p).     */
/*   S2M:  M_q = sum_j q_j J_q(k r_j) e^{-i q theta_j}        (Eq. (multipole_coef))
 *   L2T:  u(x) = sum_p L_p J_p(k r) e^{i p theta}            (Eq. (local))
 *   M2M:  M'_p = sum_q M_{p-q} J_q(k r12) e^{-i q theta12},  (r12, theta12) = child centre
 *         relative to the parent centre   (Lemma M2M; reading G3 for the sign)
 *   L2L:  L'_p = sum_q L_{p-q} J_q(k r12) e^{-i q theta12},  (r12, theta12) = parent centre
 *         relative to the child centre    (Lemma L2L; reading G3 for the phase)
 *   free-space M2L (Rokhlin's translation, named in Sec. 2.2):
 *         L_p += (i/4) sum_q M_q H_{q-p}(k |c|) e^{i (q-p) arg c},  c = x_c^t - x_c^s
 *   layered M2L (Lemma M2L; reading G2 for the phase i^{p-q}):
 *         A_pq = (i^{p-q}/4pi) Int Z_t^p Z_s^q e^{i lambda dx} e^{-s2 h} sigma_m / s2 d lambda,
 *         Z_t = (lambda + tau s2)/k2, Z_s = (lambda + vs s2)/k2, h = tau y_c^t + vs y_c^s + c_m,
 *         (tau, vs, c_m) = tt (-1,-1,0), bb (+1,+1,2d), tb (-1,+1,2d), bt (+1,-1,2d).     */
/* ------------------------------------------------------------------------- */
static double besj(int n, double x)
{
    if (n < 0) return (n & 1) ? -jn(-n, x) : jn(-n, x);
    return jn(n, x);
}
static cx hank(int n, double x)
{
    int a = n < 0 ? -n : n;
    double s = (n < 0 && (a & 1)) ? -1.0 : 1.0;
    return s * (jn(a, x) + I * yn(a, x));
}
static cx ipow(int n)
{
    static const cx t[4] = {1.0, I, -1.0, -I};
    return t[((n % 4) + 4) % 4];
}

static const int term_tau[5] = {+1, -1, +1, -1, +1};
static const int term_vs[5] = {-1, -1, +1, +1, -1};

/* Z = (lambda + sgn s2)/k, evaluated in whichever of the two equal forms
 * (lambda + sgn s)/k or k/(lambda - sgn s) does not cancel. */
static cx zfac(cx lam, cx s, int sgn, double k)
{
    cx a = lam + sgn * s, b = lam - sgn * s;
    return (cabs(a) >= cabs(b)) ? a / k : k / b;
}

static cx cpowi(cx z, int n)
{
    cx r = 1.0, b = z;
    int e = n < 0 ? -n : n;
    while (e) {
        if (e & 1) r *= b;
        b *= b;
        e >>= 1;
    }
    return n < 0 ? 1.0 / r : r;
}

typedef struct {
    orc_medium m;
    int term, p, q;
    double dx, h, c, a, L;
    int tail;   /* 0 north, 1 east up/down */
    int side;   /* +1 right tail, -1 left tail */
} a_ctx;

static cx a_integrand(cx lam, a_ctx *A)
{
    cx s2, sig[3];
    sig_layer2(lam, &A->m, &s2, sig);
    cx zt = zfac(lam, s2, term_tau[A->term], A->m.k2);
    cx zs = zfac(lam, s2, term_vs[A->term], A->m.k2);
    cx ex = cexp(I * lam * A->dx - s2 * A->h);
    return cpowi(zt, A->p) * cpowi(zs, A->q) * ex * sig[term_sig[A->term - 1]] / s2;
}
static cx fa_segment(double t, void *v)
{
    a_ctx *A = v;
    double ph = M_PI * t / A->c;
    cx lam = t - I * A->a * sin(ph);
    cx dl = 1.0 - I * A->a * (M_PI / A->c) * cos(ph);
    return a_integrand(lam, A) * dl;
}
static cx fa_tail(double u, void *v)
{
    a_ctx *A = v;
    double t = A->L * u / (1.0 - u), dt = A->L / ((1.0 - u) * (1.0 - u));
    cx lam, dir;
    if (A->tail == 0) {
        dir = A->side;                 /* along the real axis outward */
    } else {
        /* rotate towards decay of e^{i lambda dx}: up if dx > 0, down if dx < 0 */
        dir = (A->dx > 0) ? I : -I;
    }
    lam = A->side * A->c + t * dir;
    /* orientation: the right tail runs from c outward (+), the left tail runs
     * from -inf to -c, i.e. the negative of the outward path. */
    return (double)A->side * a_integrand(lam, A) * dir * dt;
}

static int m2l_image_entry(const orc_medium *m, int term, int p, int q, double dx, double h,
                           cx *out)
{
    a_ctx A;
    A.m = *m;
    A.term = term;
    A.p = p;
    A.q = q;
    A.dx = dx;
    A.h = h;
    double km = fmax(m->k1, fmax(m->k2, m->k3));
    A.c = 1.5 * km + 1.0;
    A.a = fmin(0.5, 1.0 / fmax(fabs(dx), 1e-3));
    int st = 0;
    cx seg, tr, tl;
    int nosc = 16 + (int)(A.c * fabs(dx) / M_PI);
    g_l1 = 1;
    st |= gk_adapt(fa_segment, &A, -A.c, A.c, nosc, 0.0, g_rtol, &seg);
    A.tail = (h >= fabs(dx)) ? 0 : 1;
    double rate = A.tail == 0 ? h : fabs(dx);
    A.L = (1.0 + abs(p) + abs(q)) / (rate + 1.0 / A.c);
    A.side = +1;
    st |= gk_adapt(fa_tail, &A, 0.0, 1.0, 16, 0.0, g_rtol, &tr);
    A.side = -1;
    st |= gk_adapt(fa_tail, &A, 0.0, 1.0, 16, 0.0, g_rtol, &tl);
    g_l1 = 0;
    *out = ipow(p - q) * (seg + tr + tl) / (4.0 * M_PI);
    return st;
}

/* table of one layered M2L class: out[(p+P)(2P+1) + (q+P)] */
int orc_m2l_image_table(double k1, double k2, double k3, double d, int term, double dx,
                        double h, int P, double *out)
{
    orc_medium m = {k1, k2, k3, d};
    int np = 2 * P + 1, st = 0;
    cx *o = (cx *)out;
#pragma omp parallel for collapse(2) schedule(dynamic, 4) reduction(| : st)
    for (int p = -P; p <= P; ++p)
        for (int q = -P; q <= P; ++q) {
            cx v;
            st |= m2l_image_entry(&m, term, p, q, dx, h, &v);
            o[(p + P) * np + (q + P)] = v;
        }
    return st;
}

/* field of one image term for a single source, for checking expansions:
 * G_m(x, x0) = (1/4pi) Int e^{i lambda (x-x0)} e^{-s2 h_m} sigma_m/s2 d lambda */
int orc_green_term(double k1, double k2, double k3, double d, int term, double x, double y,
                   double x0, double y0, double *out)
{
    orc_medium m = {k1, k2, k3, d};
    cx r;
    int st = green_refl(&m, x, y, x0, y0, 1 << (term - 1), -1, &r);
    out[0] = creal(r);
    out[1] = cimag(r);
    return st;
}

/* ------------------------------------------------------------------------- */
/* FMM (Algorithm 1), plain: one density vector at a time.                    */
/* ------------------------------------------------------------------------- */
typedef struct tabent {
    int l, term;
    int64_t dc, dr;
    cx *tab;
    struct tabent *next;
} tabent;

typedef struct {
    orc_medium m;
    orc_grid g;
    int P;
    int status;
    tabent *head;
} fmm_ctx;

static cx *get_table(fmm_ctx *F, int l, int term, int64_t dc, int64_t dr)
{
    for (tabent *e = F->head; e; e = e->next)
        if (e->l == l && e->term == term && e->dc == dc && e->dr == dr) return e->tab;
    int np = 2 * F->P + 1;
    double w = ldexp(F->g.d, -l);
    cx *tab = malloc(sizeof(cx) * np * np);
    if (term == 0) {
        double cxv = dc * w, cyv = -(double)dr * w; /* centre offset (target - source); rows grow downward */
        double rr = hypot(cxv, cyv), th = atan2(cyv, cxv);
        for (int p = -F->P; p <= F->P; ++p)
            for (int q = -F->P; q <= F->P; ++q)
                tab[(p + F->P) * np + (q + F->P)] =
                    0.25 * I * hank(q - p, F->m.k2 * rr) * cexp(I * (q - p) * th);
    } else {
        /* image term: h = tau y_c^t + vs y_c^s + c_m, which equals the vertical
         * distance between target centre and image centre, |dr| w. */
        double h = fabs((double)dr) * w;
        F->status |= orc_m2l_image_table(F->m.k1, F->m.k2, F->m.k3, F->m.d, term, dc * w, h,
                                         F->P, (double *)tab);
    }
    tabent *e = malloc(sizeof(tabent));
    e->l = l;
    e->term = term;
    e->dc = dc;
    e->dr = dr;
    e->tab = tab;
    e->next = F->head;
    F->head = e;
    return tab;
}

static void box_centre(const orc_grid *g, int l, int64_t id, double *cxo, double *cyo)
{
    int64_t ncol = (int64_t)g->R << l;
    double w = ldexp(g->d, -l);
    int64_t r = id / ncol, c = id % ncol;
    *cxo = g->x0 + (c + 0.5) * w;
    *cyo = -(r + 0.5) * w;
}

/* Apply with expansion order P at depth L. q, u: [nvec][n] complex.
 * Direct-interaction reflected pairs use the per-term Sommerfeld integral. */
int orc_fmm_apply(double k1, double k2, double k3, double d, int64_t n, const double *x,
                  const double *y, int L, int P, int nvec, const double *q, double *u)
{
    fmm_ctx F;
    F.m = (orc_medium){k1, k2, k3, d};
    make_grid(n, x, d, L, &F.g);
    F.P = P;
    F.status = 0;
    F.head = NULL;
    const double k = k2;
    const int np = 2 * P + 1;
    int st = 0;
    int64_t *perm = malloc(sizeof(int64_t) * n);
    int64_t nleaf = ((int64_t)F.g.R << L) << L;
    int64_t *ls = malloc(sizeof(int64_t) * (nleaf + 1));
    double hdr[2];
    orc_tree_build(n, x, y, d, L, hdr, perm, ls);
    int64_t *nbox = malloc(sizeof(int64_t) * (L + 1));
    cx **M = malloc(sizeof(cx *) * (L + 1)), **Lc = malloc(sizeof(cx *) * (L + 1));
    for (int l = 0; l <= L; ++l) {
        nbox[l] = ((int64_t)F.g.R << l) << l;
        M[l] = malloc(sizeof(cx) * nbox[l] * np);
        Lc[l] = malloc(sizeof(cx) * nbox[l] * np);
    }
    /* lists */
    int64_t **V = malloc(sizeof(int64_t *) * (L + 1)), *nv = malloc(sizeof(int64_t) * (L + 1));
    for (int l = 0; l <= L; ++l) {
        nv[l] = orc_vlist(F.g.R, l, 0, NULL);
        V[l] = malloc(sizeof(int64_t) * 3 * (nv[l] + 1));
        orc_vlist(F.g.R, l, nv[l], V[l]);
    }
    int64_t nu = orc_ulist(F.g.R, L, 0, NULL);
    int64_t *U = malloc(sizeof(int64_t) * 3 * (nu + 1));
    orc_ulist(F.g.R, L, nu, U);
    /* pre-build all tables (serially, each table internally parallel) */
    for (int l = 0; l <= L; ++l) {
        int64_t ncol = (int64_t)F.g.R << l, nrow = (int64_t)1 << l;
        for (int64_t e = 0; e < nv[l]; ++e) {
            int64_t t = V[l][3 * e], term = V[l][3 * e + 1], s = V[l][3 * e + 2];
            int64_t dc = t % ncol - s % ncol, dr = t / ncol - img_row(term, s / ncol, nrow);
            get_table(&F, l, (int)term, dc, dr);
        }
    }
    const cx *Q = (const cx *)q;
    cx *Uo = (cx *)u;
    for (int v = 0; v < nvec; ++v) {
        const cx *qv = Q + (int64_t)v * n;
        cx *uv = Uo + (int64_t)v * n;
        /* Step 2: upward pass */
        for (int64_t b = 0; b < nleaf; ++b) {
            double cxv, cyv;
            box_centre(&F.g, L, b, &cxv, &cyv);
            for (int pp = -P; pp <= P; ++pp) {
                cx acc = 0.0;
                for (int64_t i = ls[b]; i < ls[b + 1]; ++i) {
                    int64_t j = perm[i];
                    double rx = x[j] - cxv, ry = y[j] - cyv;
                    acc += qv[j] * besj(pp, k * hypot(rx, ry)) * cexp(-I * pp * atan2(ry, rx));
                }
                M[L][b * np + pp + P] = acc;
            }
        }
        for (int l = L - 1; l >= 0; --l) {
            int64_t ncol = (int64_t)F.g.R << l, ncc = ncol * 2;
            memset(M[l], 0, sizeof(cx) * nbox[l] * np);
            for (int64_t b = 0; b < nbox[l]; ++b) {
                int64_t r = b / ncol, c = b % ncol;
                double pxv, pyv;
                box_centre(&F.g, l, b, &pxv, &pyv);
                for (int dy = 0; dy < 2; ++dy)
                    for (int dxx = 0; dxx < 2; ++dxx) {
                        int64_t ch = (2 * r + dy) * ncc + (2 * c + dxx);
                        double cxv, cyv;
                        box_centre(&F.g, l + 1, ch, &cxv, &cyv);
                        double r12 = hypot(cxv - pxv, cyv - pyv), t12 = atan2(cyv - pyv, cxv - pxv);
                        for (int pp = -P; pp <= P; ++pp)
                            for (int qq = -P; qq <= P; ++qq) {
                                int src = pp - qq;
                                if (src < -P || src > P) continue;
                                M[l][b * np + pp + P] += M[l + 1][ch * np + src + P] *
                                                         besj(qq, k * r12) * cexp(-I * qq * t12);
                            }
                    }
            }
        }
        /* Step 3: downward pass */
        for (int l = 0; l <= L; ++l) {
            int64_t ncol = (int64_t)F.g.R << l, nrow = (int64_t)1 << l;
            memset(Lc[l], 0, sizeof(cx) * nbox[l] * np);
            if (l > 0) {
                int64_t pcol = ncol / 2;
                for (int64_t b = 0; b < nbox[l]; ++b) {
                    int64_t r = b / ncol, c = b % ncol, par = (r / 2) * pcol + c / 2;
                    double cxv, cyv, pxv, pyv;
                    box_centre(&F.g, l, b, &cxv, &cyv);
                    box_centre(&F.g, l - 1, par, &pxv, &pyv);
                    double r12 = hypot(pxv - cxv, pyv - cyv), t12 = atan2(pyv - cyv, pxv - cxv);
                    for (int pp = -P; pp <= P; ++pp)
                        for (int qq = -P; qq <= P; ++qq) {
                            int src = pp - qq;
                            if (src < -P || src > P) continue;
                            Lc[l][b * np + pp + P] += Lc[l - 1][par * np + src + P] *
                                                      besj(qq, k * r12) * cexp(-I * qq * t12);
                        }
                }
            }
            for (int64_t e = 0; e < nv[l]; ++e) {
                int64_t t = V[l][3 * e], term = V[l][3 * e + 1], s = V[l][3 * e + 2];
                int64_t dc = t % ncol - s % ncol, dr = t / ncol - img_row(term, s / ncol, nrow);
                cx *A = get_table(&F, l, (int)term, dc, dr);
                for (int pp = 0; pp < np; ++pp) {
                    cx acc = 0.0;
                    for (int qq = 0; qq < np; ++qq) acc += A[pp * np + qq] * M[l][s * np + qq];
                    Lc[l][t * np + pp] += acc;
                }
            }
        }
        /* Step 4: evaluate */
        for (int64_t i = 0; i < n; ++i) uv[i] = 0.0;
        for (int64_t b = 0; b < nleaf; ++b) {
            double cxv, cyv;
            box_centre(&F.g, L, b, &cxv, &cyv);
            for (int64_t ii = ls[b]; ii < ls[b + 1]; ++ii) {
                int64_t i = perm[ii];
                double rx = x[i] - cxv, ry = y[i] - cyv;
                double rr = hypot(rx, ry), th = atan2(ry, rx);
                cx acc = 0.0;
                for (int pp = -P; pp <= P; ++pp)
                    acc += Lc[L][b * np + pp + P] * besj(pp, k * rr) * cexp(I * pp * th);
                uv[i] += acc;
            }
        }
        for (int64_t e = 0; e < nu; ++e) {
            int64_t t = U[3 * e], term = U[3 * e + 1], s = U[3 * e + 2];
            for (int64_t ii = ls[t]; ii < ls[t + 1]; ++ii) {
                int64_t i = perm[ii];
                cx acc = 0.0;
                for (int64_t jj = ls[s]; jj < ls[s + 1]; ++jj) {
                    int64_t j = perm[jj];
                    if (term == 0) {
                        if (j != i) acc += qv[j] * green_free(k, hypot(x[i] - x[j], y[i] - y[j]));
                    } else {
                        cx g;
                        st |= green_refl(&F.m, x[i], y[i], x[j], y[j], 1 << (term - 1), -1, &g);
                        acc += qv[j] * g;
                    }
                }
                uv[i] += acc;
            }
        }
    }
    for (int l = 0; l <= L; ++l) {
        free(M[l]);
        free(Lc[l]);
        free(V[l]);
    }
    free(M);
    free(Lc);
    free(V);
    free(nv);
    free(U);
    free(nbox);
    free(perm);
    free(ls);
    st |= F.status;
    while (F.head) {
        tabent *e = F.head;
        F.head = e->next;
        free(e->tab);
        free(e);
    }
    return st;
}

/* single-operator hooks for tests (one box, nvec = 1) */
void orc_s2m(int64_t n, const double *x, const double *y, const double *q, double cxv,
             double cyv, double k, int P, double *out)
{
    const cx *Q = (const cx *)q;
    cx *o = (cx *)out;
    for (int p = -P; p <= P; ++p) {
        cx acc = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            double rx = x[j] - cxv, ry = y[j] - cyv;
            acc += Q[j] * besj(p, k * hypot(rx, ry)) * cexp(-I * p * atan2(ry, rx));
        }
        o[p + P] = acc;
    }
}
void orc_l2t(int64_t n, const double *x, const double *y, const double *Lc, double cxv,
             double cyv, double k, int P, double *out)
{
    const cx *Lv = (const cx *)Lc;
    cx *o = (cx *)out;
    for (int64_t i = 0; i < n; ++i) {
        double rx = x[i] - cxv, ry = y[i] - cyv, rr = hypot(rx, ry), th = atan2(ry, rx);
        cx acc = 0.0;
        for (int p = -P; p <= P; ++p) acc += Lv[p + P] * besj(p, k * rr) * cexp(I * p * th);
        o[i] = acc;
    }
}
/* shift: mode 0 = M2M (child -> parent; (sx, sy) = child centre - parent centre),
 *        mode 1 = L2L (parent -> child; (sx, sy) = parent centre - child centre) */
void orc_shift(const double *in, double sx, double sy, double k, int P, double *out)
{
    const cx *I0 = (const cx *)in;
    cx *o = (cx *)out;
    double r12 = hypot(sx, sy), t12 = atan2(sy, sx);
    for (int p = -P; p <= P; ++p) {
        cx acc = 0.0;
        for (int qq = -P; qq <= P; ++qq) {
            int src = p - qq;
            if (src < -P || src > P) continue;
            acc += I0[src + P] * besj(qq, k * r12) * cexp(-I * qq * t12);
        }
        o[p + P] = acc;
    }
}
void orc_m2l_free_table(double k, double cxv, double cyv, int P, double *out)
{
    int np = 2 * P + 1;
    cx *o = (cx *)out;
    double rr = hypot(cxv, cyv), th = atan2(cyv, cxv);
    for (int p = -P; p <= P; ++p)
        for (int q = -P; q <= P; ++q)
            o[(p + P) * np + (q + P)] = 0.25 * I * hank(q - p, k * rr) * cexp(I * (q - p) * th);
}
double orc_besj(int n, double x) { return besj(n, x); }
void orc_green_free(double k, double r, double *out)
{
    cx g = green_free(k, r);
    out[0] = creal(g);
    out[1] = cimag(g);
}

/* ------------------------------------------------------------------------- */
/* Sec. 5, three-layer local-expansion experiment: the evanescent part of the */
/* local basis for g_2^t,                                                     */
/*   Psi_p = Int_{k2}^{inf} Z^p e^{-s2 Y} e^{i lambda X} sigma_2^t / (4 pi s2) d lambda,
 * Z = (lambda + s2)/k2 (the printed (lambda - i sqrt(k2^2 - lambda^2))/k2 on  */
/* this range), with (X, Y) the horizontal and modified vertical distances.  */
/* Theorem 1 predicts |J_{p+1}(k2 r) Psi_{p+1}| / |J_p(k2 r) Psi_p| -> r/rho. */
/* ------------------------------------------------------------------------- */
typedef struct {
    orc_medium m;
    int p;
    double X, Y, L;
} psi_ctx;
static cx f_psi(double u, void *v)
{
    psi_ctx *c = v;
    /* lambda = k2 + L w^2, w = u/(1-u): the square removes the 1/s2 endpoint singularity */
    double w = u / (1.0 - u);
    double t = c->L * w * w, dt = 2.0 * c->L * w / ((1.0 - u) * (1.0 - u));
    /* integrate along the ray lambda = k2 + t e^{i phi}, phi = atan2(X, Y), where
     * e^{-s2 Y + i lambda X} decays without oscillating (the closing arc lies in
     * the first quadrant, where the integrand decays) */
    cx dir = cexp(I * atan2(c->X, c->Y));
    cx lam = c->m.k2 + t * dir;
    cx s2 = sroot(lam, c->m.k2);
    cx z = (lam + s2) / c->m.k2;
    cx sg = sigma2t_safe(lam, c->m.k1, c->m.k2, c->m.k3, c->m.d);
    /* combine all exponents before a single exp */
    cx e = cexp(c->p * clog(z) - s2 * c->Y + I * lam * c->X);
    return e * sg / (4.0 * M_PI * s2) * dt * dir;
}
int orc_psi_e4(double k1, double k2, double k3, double d, int p, double X, double Y,
               double *out)
{
    psi_ctx c = {{k1, k2, k3, d}, p, X, Y, 0.0};
    c.L = sqrt((1.0 + p) / hypot(X, Y));
    cx r;
    int st = gk_adapt(f_psi, &c, 0.0, 1.0, 32, 0.0, 1e-12, &r);
    out[0] = creal(r);
    out[1] = cimag(r);
    return st;
}
