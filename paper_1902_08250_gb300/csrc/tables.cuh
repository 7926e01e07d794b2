// tables.cuh -- device code shared by the table builders of the middle-layer
// operator (lmfmm_setup.cu) and the cross-layer operator (lmfmm_cross.cu):
// Gauss-Legendre nodes, the image densities and the M2L table integral.
#pragma once
#include "internal.h"

// ---------------------------------------------------------------------------
// Gauss-Legendre nodes on [-1, 1] by Newton's method on P_n (three-term
// recurrence), initial guess cos(pi (i + 3/4) / (n + 1/2)).
// ---------------------------------------------------------------------------
__device__ inline void gl_node(int n, int i, double *x, double *w)
{
    double z = cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 1.0;
    for (int it = 0; it < 100; ++it) {
        double p1 = 1.0, p2 = 0.0;
        for (int j = 1; j <= n; ++j) {
            double p3 = p2;
            p2 = p1;
            p1 = ((2.0 * j - 1.0) * z * p2 - (j - 1.0) * p3) / j;
        }
        pp = n * (z * p1 - p2) / (z * z - 1.0);
        double dz = p1 / pp;
        z -= dz;
        if (fabs(dz) < 1e-16) break;
    }
    *x = -z; // ascending order
    *w = 2.0 / ((1.0 - z * z) * pp * pp);
}

// ---------------------------------------------------------------------------
// Image densities (reading R1 of the paper's Example 4 for a middle-layer
// source): R_t = (k1^2-k2^2)/(s2+s1)^2, R_b = (k3^2-k2^2)/(s2+s3)^2,
// Sigma = 1/(1 - R_t R_b e^{-2 d s2}); sigma_tt = R_t Sigma, sigma_bb =
// R_b Sigma, sigma_tb = R_t R_b Sigma.
// ---------------------------------------------------------------------------
// With deriv set (the kernel dG/dd): each density becomes
// d/dd[sigma_m e^{-s2 c_m}] e^{s2 c_m} = -2 s2 (E S + [m != tt]) sigma_m, E = R_t R_b e^{-2 d s2},
// since only S = 1/(1 - E) and c_m (0 for tt, 2d otherwise) depend on d.
struct MediumD {
    double k1, k2, k3, d;
    int deriv;
    int bc[2];       // lm_boundary of the top (y = 0) and bottom (y = -d) interfaces
    double alpha[2]; // impedance parameters
};
// reflection coefficient of interface b: a wall's (Dirichlet -1, Neumann +1,
// impedance (s2 + i k2 alpha)/(s2 - i k2 alpha)) or the transmission value
// (kj^2 - k2^2)/(s2 + sj)^2 to the outer layer of wave number kj
__device__ inline zd refl_coef(const MediumD &m, int b, zd s2, zd sj, double kj)
{
    switch (m.bc[b]) {
    case LM_BC_DIRICHLET: return zd{-1.0, 0.0};
    case LM_BC_NEUMANN: return zd{1.0, 0.0};
    case LM_BC_IMPEDANCE: {
        const zd beta = {0.0, m.k2 * m.alpha[b]};
        return cdiv(s2 + beta, s2 - beta);
    }
    default: {
        zd a = s2 + sj;
        return cdiv(zd{kj * kj - m.k2 * m.k2, 0.0}, a * a);
    }
    }
}
// Limit of the reflected density sigma_tt (b = 0) or sigma_bb (b = 1) as Re s2 -> inf
// (Sigma -> 1): a wall's constant reflection coefficient (Dirichlet -1, Neumann and
// impedance +1), 0 for a transmission (R ~ 1/lambda^2) and for the dG/dd kernel.  The
// near-field quadratures integrate sigma - R_inf; the pair adds R_inf (i/4) H0(k2 rho)
// of the image point in closed form (the Sommerfeld identity), since sigma -> R_inf
// leaves an integrand decaying only like e^{-lambda h}/lambda: the image's log
// singularity, which fixed rules cannot follow as the pair nears the wall.
__host__ __device__ inline double refl_inf(const MediumD &m, int b)
{
    if (m.deriv) return 0.0;
    switch (m.bc[b]) {
    case LM_BC_DIRICHLET: return -1.0;
    case LM_BC_NEUMANN:
    case LM_BC_IMPEDANCE: return 1.0;
    default: return 0.0;
    }
}
// k2 alpha of an impedance wall b (0 otherwise): R - 1 = 2 i beta / (s2 - i beta) ~ 2 i beta / s2.
// The target gradient's h-derivative integrates (R - 1) s2 ~ 2 i beta, which does not decay
// beyond e^{-lambda h}; it takes 2 i beta / s2 out of its integrand and adds the closed form
// -2 i beta (i/4) H0(k2 rho) instead.
__host__ __device__ inline double imp_beta(const MediumD &m, int b)
{
    return (!m.deriv && m.bc[b] == LM_BC_IMPEDANCE) ? m.k2 * m.alpha[b] : 0.0;
}
__device__ inline void densities(const MediumD &m, zd lam, zd *s2o, zd sig[3])
{
    zd s1 = sbranch(lam, m.k1), s2 = sbranch(lam, m.k2), s3 = sbranch(lam, m.k3);
    zd Rt = refl_coef(m, 0, s2, s1, m.k1);
    zd Rb = refl_coef(m, 1, s2, s3, m.k3);
    zd E = Rt * Rb * cexpd(-2.0 * m.d * s2);
    zd S = cdiv(zd{1.0, 0.0}, zd{1.0, 0.0} - E);
    sig[0] = Rt * S;
    sig[1] = Rb * S;
    sig[2] = Rt * Rb * S;
    if (m.deriv) {
        zd f = -2.0 * s2 * (E * S);
        zd g = f - 2.0 * s2;
        sig[0] = f * sig[0];
        sig[1] = g * sig[1];
        sig[2] = g * sig[2];
    }
    *s2o = s2;
}

#define TB_CHUNK 16
// One class's table.  The integrand is sig(lambda) e^{i lambda dx - s2 ht - ss hs} / s2
// with target Z_t = (lambda + tau s2)/k2 (scale sc = k2 w) and source
// Z_s = (lambda + vs ss)/ks (scale scs = ks w), ss = sqrt(lambda^2 - ks^2); the
// density functor sigf(lambda, &s2, &ss) returns sig.  ks = k2 (ss = s2) for
// the middle layer's image terms; ks = k1 for the layer-1 sources of the
// cross-layer operator.
template <class SigF>
__device__ inline void m2l_table_body(SigF sigf, double km, double kmin, double k2, double ks, int P, double sc,
                               double scs, int tau, int vs, double dx, double ht, double hs, zd *tabout,
                               int *flag)
{
    extern __shared__ unsigned char smem[];
    int np = 2 * P + 1;
    zd *ZT = (zd *)smem;                 // [TB_CHUNK][np]
    zd *ZS = ZT + TB_CHUNK * np;         // [TB_CHUNK][np]
    zd *BW = ZS + TB_CHUNK * np;         // [TB_CHUNK]
    const double h = ht + hs;
    double c = 1.5 * km + 1.0;
    double a = fmin(0.5, 1.0 / fmax(fabs(dx), 1e-3));
    double delta = fmin(0.25, 0.5 * kmin);
    double width = fmin(fmin(0.5, 2.0 * a), 1.5 / fmax(fabs(dx), 1e-3));
    int nflat = (int)ceil((c - 2.0 * delta) / width);
    const int ORD = 24;
    int nseg_half = (nflat + 2) * ORD;
    double rho = hypot(dx, h);
    double tmax = 1.5 * (2.0 * P + 60.0) / rho;
    // Panels of ORD nodes on [0, tmax], geometrically graded: the first is at
    // most 1 wide (low orders vary on the scale of c near the start of the ray),
    // later ones widen by the ratio g (high orders peak near t = 2P / rho).
    // Uniform panels lost accuracy for small boxes, where tmax ~ 1/rho is large.
    const int TPAN = P + 16 > 32 ? P + 16 : 32;
    const double h0 = fmin(1.0, tmax / TPAN);
    double g = 1.0;
    if (h0 * TPAN < tmax) { // solve h0 (g^TPAN - 1)/(g - 1) = tmax for g > 1 by bisection
        double lo = 1.0, hi = 2.0;
        while (h0 * (pow(hi, TPAN) - 1.0) / (hi - 1.0) < tmax) hi *= 2.0;
        for (int it = 0; it < 100; ++it) {
            const double mid = 0.5 * (lo + hi);
            if (h0 * (pow(mid, TPAN) - 1.0) / (mid - 1.0) < tmax) lo = mid;
            else hi = mid;
        }
        g = hi;
    }
    auto tpan = [&](int j) { return g == 1.0 ? h0 * j : h0 * (pow(g, j) - 1.0) / (g - 1.0); };
    int ntail = TPAN * ORD;
    int ntot = 2 * nseg_half + 2 * ntail;
    double phi = atan2(dx, h);
    zd er = {cos(phi), sin(phi)};       // right ray direction
    zd el = {-cos(phi), sin(phi)};      // left ray direction: -e^{-i phi}
    // accumulators: each thread owns entries idx = tid + k*blockDim
    const int MAXE = (2 * LM_MAXP + 1) * (2 * LM_MAXP + 1);
    (void)MAXE;
    int nent = np * np;
    int per = (nent + blockDim.x - 1) / blockDim.x;
    zd acc[48];
    for (int e = 0; e < per && e < 48; ++e) acc[e] = zd{0.0, 0.0};
    if (per > 48) {
        if (threadIdx.x == 0) atomicOr(flag, 8);
        return;
    }
    for (int base = 0; base < ntot; base += TB_CHUNK) {
        __syncthreads();
        // thread j < TB_CHUNK builds node base + j
        if (threadIdx.x < TB_CHUNK) {
            int i = base + threadIdx.x;
            zd lam = {0.0, 0.0}, dl = {0.0, 0.0};
            bool valid = i < ntot;
            if (valid) {
                if (i < 2 * nseg_half) {
                    int side = i < nseg_half ? 1 : -1;
                    int ii = i % nseg_half, pan = ii / ORD, j = ii % ORD;
                    double x, gw;
                    gl_node(ORD, j, &x, &gw);
                    zd z0, z1;
                    double flat = (c - 2.0 * delta) / nflat;
                    if (pan == 0) {
                        z0 = {0.0, 0.0};
                        z1 = {delta, -a};
                    } else if (pan == nflat + 1) {
                        z0 = {c - delta, -a};
                        z1 = {c, 0.0};
                    } else {
                        z0 = {delta + (pan - 1) * flat, -a};
                        z1 = {delta + pan * flat, -a};
                    }
                    zd dz = z1 - z0;
                    lam = z0 + (0.5 * (x + 1.0)) * dz;
                    dl = (0.5 * gw) * dz;
                    if (side < 0) {
                        // mirror through the origin; orientation -c -> 0 keeps dl
                        lam = -lam;
                    }
                } else {
                    int ii = i - 2 * nseg_half;
                    int side = ii < ntail ? 1 : -1;
                    ii %= ntail;
                    int pan = ii / ORD, j = ii % ORD;
                    double x, gw;
                    gl_node(ORD, j, &x, &gw);
                    double t0 = tpan(pan), t1 = tpan(pan + 1);
                    double t = t0 + 0.5 * (x + 1.0) * (t1 - t0), wt = 0.5 * gw * (t1 - t0);
                    if (side > 0) {
                        lam = zd{c, 0.0} + t * er;
                        dl = wt * er;
                    } else {
                        lam = zd{-c, 0.0} + t * el;
                        dl = -wt * el; // runs from -inf to -c
                    }
                }
                zd s2, ss;
                const zd sg = sigf(lam, &s2, &ss);
                zd ex = cexpd(zd{-lam.im * dx, lam.re * dx} - ht * s2 - hs * ss);
                BW[threadIdx.x] = cdiv(dl * ex * sg, s2) * (1.0 / (4.0 * M_PI));
                // Z = (lam + sgn s2)/k2, non-cancelling form; its inverse (lam - sgn s2)/k2
                zd zt_p, zt_m, zs_p, zs_m;
                {
                    zd ap = lam + (double)tau * s2, am = lam - (double)tau * s2;
                    if (abs2(ap) >= abs2(am)) {
                        zt_p = (1.0 / k2) * ap;
                        zt_m = cdiv(zd{k2, 0.0}, ap);
                    } else {
                        zt_p = cdiv(zd{k2, 0.0}, am);
                        zt_m = (1.0 / k2) * am;
                    }
                    zd bp = lam + (double)vs * ss, bm = lam - (double)vs * ss;
                    if (abs2(bp) >= abs2(bm)) {
                        zs_p = (1.0 / ks) * bp;
                        zs_m = cdiv(zd{ks, 0.0}, bp);
                    } else {
                        zs_p = cdiv(zd{ks, 0.0}, bm);
                        zs_m = (1.0 / ks) * bm;
                    }
                }
                zd *zt = ZT + threadIdx.x * np + P, *zs = ZS + threadIdx.x * np + P;
                zt[0] = zd{1.0, 0.0};
                zs[0] = zd{1.0, 0.0};
                zd up = zd{1.0, 0.0}, dn = zd{1.0, 0.0}, su = zd{1.0, 0.0}, sd = zd{1.0, 0.0};
                for (int n = 1; n <= P; ++n) {
                    const double f = 0.5 * sc / n, fs = 0.5 * scs / n;
                    up = up * (f * zt_p);
                    dn = dn * (f * zt_m);
                    su = su * (fs * zs_p);
                    sd = sd * (fs * zs_m);
                    zt[n] = up;
                    zt[-n] = dn;
                    zs[n] = su;
                    zs[-n] = sd;
                }
            } else {
                BW[threadIdx.x] = zd{0.0, 0.0};
                for (int n = 0; n < np; ++n) {
                    ZT[threadIdx.x * np + n] = zd{0.0, 0.0};
                    ZS[threadIdx.x * np + n] = zd{0.0, 0.0};
                }
            }
        }
        __syncthreads();
        for (int e = 0; e < per; ++e) {
            int idx = threadIdx.x + e * blockDim.x;
            if (idx >= nent) break;
            int pi = idx / np, qi = idx % np;
            zd s = acc[e];
            for (int j = 0; j < TB_CHUNK; ++j) cfma(s, BW[j] * ZT[j * np + pi], ZS[j * np + qi]);
            acc[e] = s;
        }
    }
    zd *T = tabout;
    for (int e = 0; e < per; ++e) {
        int idx = threadIdx.x + e * blockDim.x;
        if (idx >= nent) break;
        int p = idx / np - P, q = idx % np - P;
        int ph = ((p - q) % 4 + 4) % 4; // i^{p-q}
        zd v = acc[e];
        zd r = ph == 0 ? v : ph == 1 ? zd{-v.im, v.re} : ph == 2 ? -v : zd{v.im, -v.re};
        if (!isfinite(r.re) || !isfinite(r.im)) atomicOr(flag, 16);
        T[idx] = r;
    }
}

