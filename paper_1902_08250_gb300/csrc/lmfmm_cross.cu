// lmfmm_cross.cu -- the cross-layer operator of Sec. 3, Example 4 as printed:
// sources in layer 1 (0 < y0 < d), targets in the middle layer (-d < y < 0),
//     u_i = sum_j q_j [g_2^t + g_2^b](x_i, x_j),
// through the FMM with two wave numbers (Sec. 2.1: multipoles in k0 = k1 about
// the source boxes, local expansions in k = k2 about the target boxes), on a
// source tree and a target tree that share one lattice.
//
// The sources are mirrored through y = 0 (y' = -y0), onto the lattice of the
// middle layer.  Then g_2^t has the geometry of the middle layer's tt image
// term (source factor e^{-s1 y0} = e^{s1 y'}, target factor e^{s2 y}) and
// g_2^b that of its bt term (target factor e^{-s2 (y + 2d)}), with the source
// side in k1: multipoles M_q = sum q_j J_q(k1 r_j) e^{-i q theta_j} about the
// mirrored box centres, Z_s = (lambda - s1)/k1, and M2M in k1.  The lists are
// the middle layer's image lists for these two terms; since s1 != s2, an M2L
// table depends on the target and source rows separately, so a class is
// (term, dc, rt, rs).  g_2^b never reaches the near field (its image is d or
// more below every target).
// Precision: LM_FP64 runs every step in FP64.  LM_MIXED builds the tables and the
// near-field quadrature in FP64 and keeps FP32 copies of the tables; the
// expansions and every multiply-add are FP32, the near kernel values FP64 rounded
// to FP32.
#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include <cmath>

#include "internal.h"
#include "tables.cuh"

// kernels shared with the middle-layer operator
__global__ void k_minmax(const double *x, const double *y, int64_t n, double d, double *bmin, double *bmax,
                         int *flag);
__global__ void k_keys(const double *x, const double *y, int64_t n, double x0, double w, int64_t ncol,
                       int64_t nrow, int32_t *key, int32_t *cnt);
__global__ void k_scan(const int32_t *cnt, int64_t m, int64_t *start);
__global__ void k_scatter(const int32_t *key, int64_t n, const int64_t *start, int32_t *cursor, int64_t *tmp);
__global__ void k_leafsort(const int64_t *start, int64_t *idx, int *flag);
__global__ void k_gather_pts(const double *x, const double *y, const int64_t *perm, int64_t n, double *xs,
                             double *ys);
__global__ void k_shift_tables(double k, int P, double wc, const double *sc_child, const double *sc_par, zd *m2m,
                               zd *l2l);
__global__ void k_p2m64(LeafGeom g, int P, double k, const double *xs, const double *ys, const int64_t *ls,
                        const zd *qs, int64_t n, int nvec, zd *M);
__global__ void k_m2m64(int64_t ncol, int64_t nbox, int P, int nvec, const zd *tabs, const zd *Mc, zd *Mp);
__global__ void k_l2l64(int64_t ncol, int64_t nbox, int P, int nvec, const zd *tabs, const zd *Lp, zd *Lc);
__global__ void k_m2l64(int64_t nbox, int P, int nvec, const int64_t *vstart, const int32_t *vsrc,
                        const int32_t *vslot, const zd *tab, const zd *M, zd *Lc);
__global__ void k_permute_in(const zd *q, const int64_t *perm, int64_t n, int nvec, int conjugate, zd *qs);
__global__ void k_permute_out(const zd *us, const int64_t *perm, int64_t n, int nvec, int conjugate, zd *u);
#define CROSS_P2M_CHUNK 16 // points staged per round by k_p2m64

struct CrossLevel {
    int64_t ncol, nrow, nbox;
    double w;
    double *sc_t, *sc_s; // S(n) = (k w / 2)^n / n! for k2 (targets) and k1 (sources)
    zd *m2m, *l2l;       // [4][np][np]: k1 (child -> this level), k2 (parent -> this level)
    zd *M, *Lc;          // [nbox][np][LM_MAXV]
    int64_t nv;
    int64_t *vstart;
    int32_t *vsrc, *vslot;
    int ncls;
    zd *tab; // [ncls][np][np]
    // mixed form: FP32 copies of the tables, FP32 expansions
    zf *tab32, *m2m32, *l2l32, *M32, *L32;
};

struct lm_cross_s {
    lm_medium_s med;
    int p, L, R;
    double x0;
    int64_t ns, nt, nleaf;
    int64_t *perm_s, *ls_s, *perm_t, *ls_t;
    double *xs_s, *ys_s, *xs_t, *ys_t; // tree order; ys_s mirrored (y' = -y0)
    std::vector<CrossLevel> lev;
    int64_t nu;
    int64_t *ustart;
    int32_t *usrc;
    // near-field quadrature of g_2^t: segment nodes and tail rays (P, M weights)
    int nseg, nray, ntail;
    zd *seg_lam, *seg_s1, *seg_s2, *seg_w, *tail_lam, *tail_s1, *tail_s2, *tail_w;
    zd *qs, *us; // [LM_MAXV][ns], [LM_MAXV][nt]
    int *dflag;
    std::vector<void *> allocs;
};

template <typename T>
static lm_status calloc_dev(lm_cross_s *c, T **p, size_t count)
{
    *p = nullptr;
    if (cudaMalloc((void **)p, std::max<size_t>(1, count) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        lm_set_error("build_cross: device allocation of %zu bytes failed", count * sizeof(T));
        return LM_ENOMEM;
    }
    c->allocs.push_back(*p);
    return LM_OK;
}
#define CTRY(x)                         \
    do {                                \
        lm_status s_ = (x);             \
        if (s_ != LM_OK) return s_;     \
    } while (0)

// ---------------------------------------------------------------------------
// Densities of Example 4 (closed forms as printed), numerator and denominator
// divided by e^{d s2}/2 so that nothing overflows:
//   D' = (1 - E)(lambda^2 + s1 s3 - k2^2) + s2 (s1 + s3)(1 + E),  E = e^{-2 d s2},
//   sigma_2^t = 2 (lambda^2 + s2 s3 - k2^2) / D',
//   sigma_2^b = -2 (-lambda^2 + s2 s3 + k2^2) / D'.
// ---------------------------------------------------------------------------
__device__ inline void sigma_cross(double k1, double k2, double k3, double d, zd lam, zd *s1o, zd *s2o, zd *st,
                                   zd *sb)
{
    const zd s1 = sbranch(lam, k1), s2 = sbranch(lam, k2), s3 = sbranch(lam, k3);
    const zd E = cexpd(-2.0 * d * s2);
    const zd l2 = lam * lam, one = {1.0, 0.0};
    const zd K2 = {k2 * k2, 0.0};
    const zd den = (one - E) * (l2 + s1 * s3 - K2) + s2 * (s1 + s3) * (one + E);
    *st = cdiv(2.0 * (l2 + s2 * s3 - K2), den);
    *sb = cdiv(-2.0 * (s2 * s3 + K2 - l2), den);
    *s1o = s1;
    *s2o = s2;
}

// M2L tables of the cross classes: term 0 = g_2^t (target factor e^{s2 y}), 1 =
// g_2^b (e^{-s2 (y + 2d)}); the mirrored source side carries e^{s1 y'} in both
__global__ void __launch_bounds__(256) k_cross_m2l(double k1, double k2, double k3, double d, int P, double w,
                                                   double sc_t, double sc_s, const int *cterm, const int *cdc,
                                                   const int *crt, const int *crs, int ncls, zd *tab, int *flag)
{
    const int ci = blockIdx.x;
    if (ci >= ncls) return;
    const int term = cterm[ci];
    auto sigf = [&](zd lam, zd *s2, zd *ss) {
        zd st, sb;
        sigma_cross(k1, k2, k3, d, lam, ss, s2, &st, &sb);
        return term == 0 ? st : sb;
    };
    const double km = fmax(k1, fmax(k2, k3)), kmin = fmin(k1, fmin(k2, k3));
    const double yt = (crt[ci] + 0.5) * w;                 // depth of the target centre below y = 0
    const double ht = term == 0 ? yt : 2.0 * d - yt;       // target exponent: -s2 ht
    const double hs = (crs[ci] + 0.5) * w;                 // height of the source centre above y = 0
    m2l_table_body(sigf, km, kmin, k2, k1, P, sc_t, sc_s, term == 0 ? -1 : 1, -1, cdc[ci] * w, ht, hs,
                   tab + (int64_t)ci * (2 * P + 1) * (2 * P + 1), flag);
}

// Near-field nodes of g_2^t.  sigma_2^t -> 1 as lambda grows, so g_2^t carries
// the free-space near-singularity when source and target sit at the interface;
// it is split as (i/4) H0(k2 R), R = |x - x0| (closed form), plus the integral
// of [sigma_2^t e^{-s1 y0} - e^{-s2 y0}] e^{s2 y} / s2, which decays like
// e^{-lambda h}/lambda^2.  Two weight sets: a (sigma_2^t, source factor e^{-s1 y0})
// and b (1, source factor e^{-s2 y0}).  The segment is folded (weights with
// 2 cos); the tail rays keep their mirror images below the axis (P = W_u + W_l,
// M = W_u - W_l).
__global__ void k_cross_near_seg(double k1, double k2, double k3, double d, double c, double a, double delta,
                                 int nflat, int order, zd *lam_o, zd *s1_o, zd *s2_o, zd *w_o, int nseg)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nseg) return;
    int pan = i / order, j = i % order;
    double x, wq;
    gl_node(order, j, &x, &wq);
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
    zd lam = z0 + (0.5 * (x + 1.0)) * dz;
    zd s1, s2, st, sb;
    sigma_cross(k1, k2, k3, d, lam, &s1, &s2, &st, &sb);
    lam_o[i] = lam;
    s1_o[i] = s1;
    s2_o[i] = s2;
    const zd base = cdiv((0.5 * wq / (4.0 * M_PI)) * dz, s2);
    w_o[i] = base * st;
    w_o[nseg + i] = base;
}

__global__ void k_cross_near_tail(double k1, double k2, double k3, double d, double c, int nray, int order,
                                  zd *lam_o, zd *s1_o, zd *s2_o, zd *w_o)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int tot = nray * order;
    if (i >= tot) return;
    int k = i / order, j = i % order;
    double x, wq;
    gl_node(order, j, &x, &wq);
    double v = 0.5 * (x + 1.0), wv = 0.5 * wq;
    double t = c * v / (1.0 - v), dt = c / ((1.0 - v) * (1.0 - v));
    double phi = (nray > 1) ? k * (0.5 * M_PI) / (nray - 1) : 0.0;
    zd e = {cos(phi), sin(phi)};
    zd lam = zd{c, 0.0} + t * e, laml = conj(lam);
    zd s1, s2, st, sb, s1l, s2l, stl, sbl;
    sigma_cross(k1, k2, k3, d, lam, &s1, &s2, &st, &sb);
    sigma_cross(k1, k2, k3, d, laml, &s1l, &s2l, &stl, &sbl);
    const zd bu = cdiv((wv * dt / (4.0 * M_PI)) * e, s2), bl = cdiv((wv * dt / (4.0 * M_PI)) * conj(e), s2l);
    lam_o[i] = lam;
    s1_o[i] = s1;
    s2_o[i] = s2;
    w_o[i] = bu * st + bl * stl;           // P_a
    w_o[tot + i] = bu * st - bl * stl;     // M_a
    w_o[2 * tot + i] = bu + bl;            // P_b
    w_o[3 * tot + i] = bu - bl;            // M_b
}

// g_2^t of one near pair: X = |x - x0|, target depth-side exponent s2 y (y < 0),
// source factor e^{-s1 y0} (y0 > 0)
struct CrossNear {
    int nseg, nray, ntail;
    const zd *seg_lam, *seg_s1, *seg_s2, *seg_w, *tail_lam, *tail_s1, *tail_s2, *tail_w;
};
__device__ zd cross_near(const CrossNear &q, double k2, double X, double y, double y0)
{
    // closed-form part: (i/4) H0(k2 R)
    const double R = hypot(X, y0 - y);
    zd acc = {-0.25 * ::y0(k2 * R), 0.25 * j0(k2 * R)};
    for (int i = 0; i < q.nseg; ++i) {
        const zd lam = q.seg_lam[i], s1 = q.seg_s1[i], s2 = q.seg_s2[i];
        const zd ph = {-lam.im * X, lam.re * X};
        const zd va = y * s2 - y0 * s1, vb = (y - y0) * s2;
        cfma(acc, q.seg_w[i], cexpd(va + ph) + cexpd(va - ph));
        cfma(acc, -1.0 * q.seg_w[q.nseg + i], cexpd(vb + ph) + cexpd(vb - ph));
    }
    const int k = q.nray > 1 ? (int)rint(atan2(X, y0 - y) * (q.nray - 1) / (0.5 * M_PI)) : 0;
    const int64_t tot = (int64_t)q.nray * q.ntail, o = (int64_t)k * q.ntail;
    for (int i = 0; i < q.ntail; ++i) {
        const zd lam = q.tail_lam[o + i], s1 = q.tail_s1[o + i], s2 = q.tail_s2[o + i];
        const zd ph = {-lam.im * X, lam.re * X};
        const zd ea = cexpd(y * s2 - y0 * s1 + ph), eb = cexpd((y - y0) * s2 + ph);
        const zd Pa = q.tail_w[o + i], Ma = q.tail_w[tot + o + i];
        const zd Pb = q.tail_w[2 * tot + o + i], Mb = q.tail_w[3 * tot + o + i];
        acc = acc + ea.re * Pa + ea.im * zd{-Ma.im, Ma.re}; // P Re(E) + i M Im(E)
        acc = acc - (eb.re * Pb + eb.im * zd{-Mb.im, Mb.re});
    }
    return acc;
}

// L2T (k2) and the near g_2^t pairs of every target of a leaf
__global__ void k_cross_leaf(LeafGeom g, int P, double k2, const double *xt, const double *yt, const int64_t *lt,
                             const int64_t *ustart, const int32_t *usrc, const double *xs, const double *ysm,
                             const int64_t *lsrc, CrossNear nq, const zd *Lc, const zd *qs, int64_t ns,
                             int64_t nt, int nvec, zd *us)
{
    const int np = 2 * P + 1;
    const int64_t b = blockIdx.x;
    double cx, cy;
    leaf_centre(g, b, &cx, &cy);
    const double sc = k2 * g.w;
    const zd *Lb = Lc + b * np * LM_MAXV;
    for (int64_t i = lt[b] + threadIdx.x; i < lt[b + 1]; i += blockDim.x) {
        const double xi = xt[i], yi = yt[i];
        zd acc[LM_MAXV];
        for (int v = 0; v < nvec; ++v) acc[v] = zd{0.0, 0.0};
        {
            double rx = xi - cx, ry = yi - cy, r = hypot(rx, ry);
            double J[LM_MAXP + 1];
            bessel_j_scaled<double>(P, k2 * r, sc, J);
            zd z = r > 0.0 ? zd{rx / r, ry / r} : zd{1.0, 0.0};
            zd zp = {1.0, 0.0};
            for (int v = 0; v < nvec; ++v) cfma(acc[v], zd{J[0], 0.0}, Lb[P * LM_MAXV + v]);
            for (int m = 1; m <= P; ++m) {
                zp = zp * z;
                const zd bp = J[m] * zp, bn = ((m & 1) ? -J[m] : J[m]) * conj(zp);
                for (int v = 0; v < nvec; ++v) {
                    cfma(acc[v], bp, Lb[(P + m) * LM_MAXV + v]);
                    cfma(acc[v], bn, Lb[(P - m) * LM_MAXV + v]);
                }
            }
        }
        for (int64_t e = ustart[b]; e < ustart[b + 1]; ++e) {
            const int32_t s = usrc[e];
            for (int64_t j = lsrc[s]; j < lsrc[s + 1]; ++j) {
                const zd gij = cross_near(nq, k2, fabs(xi - xs[j]), yi, -ysm[j]);
                for (int v = 0; v < nvec; ++v) cfma(acc[v], gij, qs[(int64_t)v * ns + j]);
            }
        }
        for (int v = 0; v < nvec; ++v) us[(int64_t)v * nt + i] = acc[v];
    }
}

// ---------------------------------------------------------------------------
// Mixed-precision form: the same steps with the expansions, the translation
// tables (built in FP64, rounded once) and every multiply-add in FP32; the
// near-field kernel values g_2^t come from the FP64 contour quadrature above
// and are rounded per pair.
// ---------------------------------------------------------------------------
__global__ void k_cross_to32(const zd *a, int64_t n, zf *b)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = zf{(float)a[i].re, (float)a[i].im};
}

__device__ __forceinline__ void cfma32(zf &a, zf b, zf c)
{
    a.re = fmaf(b.re, c.re, fmaf(-b.im, c.im, a.re));
    a.im = fmaf(b.re, c.im, fmaf(b.im, c.re, a.im));
}

#define CROSS32_CHUNK 32
// S2M in k1 about the mirrored source leaves: one block per leaf, points staged
// CROSS32_CHUNK at a time (basis row and densities), one thread per (order, vector)
__global__ void __launch_bounds__(128) k_cross_p2m32(LeafGeom g, int P, double k, const double *xs,
                                                     const double *ys, const int64_t *ls, const zd *qs, int64_t n,
                                                     int nvec, zf *M)
{
    __shared__ zf B[CROSS32_CHUNK][2 * LM_MAXP + 1];
    __shared__ zf Q[CROSS32_CHUNK][LM_MAXV];
    const int np = 2 * P + 1;
    const int64_t b = blockIdx.x, lo = ls[b], hi = ls[b + 1];
    double cx, cy;
    leaf_centre(g, b, &cx, &cy);
    const float sc = (float)(k * g.w);
    const int nent = np * nvec;
    zf acc[8];
    for (int e = 0; e < 8; ++e) acc[e] = zf{0.f, 0.f};
    for (int64_t base = lo; base < hi; base += CROSS32_CHUNK) {
        __syncthreads();
        const int j = threadIdx.x;
        if (j < CROSS32_CHUNK) {
            const int64_t i = base + j;
            zf *row = B[j] + P;
            if (i < hi) {
                const float rx = (float)(xs[i] - cx), ry = (float)(ys[i] - cy), r = sqrtf(rx * rx + ry * ry);
                float J[LM_MAXP + 1];
                bessel_j_scaled<float>(P, (float)k * r, sc, J);
                const zf z = r > 0.f ? zf{rx / r, -ry / r} : zf{1.f, 0.f}; // e^{-i theta}
                zf zp = {1.f, 0.f};
                row[0] = zf{J[0], 0.f};
                for (int m = 1; m <= P; ++m) {
                    zp = zp * z;
                    row[m] = J[m] * zp;
                    row[-m] = ((m & 1) ? -J[m] : J[m]) * conj(zp);
                }
                for (int v = 0; v < nvec; ++v) {
                    const zd qd = qs[(int64_t)v * n + i];
                    Q[j][v] = zf{(float)qd.re, (float)qd.im};
                }
            } else {
                for (int m = -P; m <= P; ++m) row[m] = zf{0.f, 0.f};
                for (int v = 0; v < nvec; ++v) Q[j][v] = zf{0.f, 0.f};
            }
        }
        __syncthreads();
        for (int e = 0; e < 8; ++e) {
            const int idx = threadIdx.x + e * blockDim.x;
            if (idx >= nent) break;
            const int qi = idx / nvec, v = idx % nvec;
            zf s = zf{0.f, 0.f}; // each chunk summed on its own (blocked accumulation)
            for (int jj = 0; jj < CROSS32_CHUNK; ++jj) cfma32(s, B[jj][qi], Q[jj][v]);
            acc[e] = acc[e] + s;
        }
    }
    for (int e = 0; e < 8; ++e) {
        const int idx = threadIdx.x + e * blockDim.x;
        if (idx >= nent) break;
        const int qi = idx / nvec, v = idx % nvec;
        M[(b * np + qi) * LM_MAXV + v] = acc[e];
    }
}

// M2M in k1 (Lemma M2M): parent from its four children
__global__ void k_cross_m2m32(int64_t ncol, int64_t nbox, int P, int nvec, const zf *tabs, const zf *Mc, zf *Mp)
{
    const int np = 2 * P + 1;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nbox * np * nvec) return;
    const int v = idx % nvec, p = (idx / nvec) % np;
    const int64_t b = idx / (nvec * np), r = b / ncol, c = b % ncol, ncc = 2 * ncol;
    zf acc = {0.f, 0.f};
    for (int pos = 0; pos < 4; ++pos) {
        const int64_t ch = (2 * r + (pos >> 1)) * ncc + 2 * c + (pos & 1);
        const zf *T = tabs + ((int64_t)pos * np + p) * np;
        const zf *m = Mc + ch * np * LM_MAXV + v;
        for (int q = 0; q < np; ++q) cfma32(acc, T[q], m[q * LM_MAXV]);
    }
    Mp[(b * np + p) * LM_MAXV + v] = acc;
}

// L2L in k2 (Lemma L2L): child from its parent; sets L
__global__ void k_cross_l2l32(int64_t ncol, int64_t nbox, int P, int nvec, const zf *tabs, const zf *Lp, zf *Lc)
{
    const int np = 2 * P + 1;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nbox * np * nvec) return;
    const int v = idx % nvec, p = (idx / nvec) % np;
    const int64_t b = idx / (nvec * np), r = b / ncol, c = b % ncol;
    const int pos = (int)((r & 1) * 2 + (c & 1));
    const int64_t par = (r / 2) * (ncol / 2) + c / 2;
    const zf *T = tabs + ((int64_t)pos * np + p) * np;
    const zf *m = Lp + par * np * LM_MAXV + v;
    zf acc = {0.f, 0.f};
    for (int q = 0; q < np; ++q) cfma32(acc, T[q], m[q * LM_MAXV]);
    Lc[(b * np + p) * LM_MAXV + v] = acc;
}

// M2L over the cross V list (classes (term, dc, rt, rs)); adds to L, each entry summed on its own
__global__ void k_cross_m2l32(int64_t nbox, int P, int nvec, const int64_t *vstart, const int32_t *vsrc,
                              const int32_t *vslot, const zf *tab, const zf *M, zf *Lc)
{
    const int np = 2 * P + 1;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nbox * np * nvec) return;
    const int v = idx % nvec, p = (idx / nvec) % np;
    const int64_t b = idx / (nvec * np);
    zf acc = {0.f, 0.f};
    for (int64_t e = vstart[b]; e < vstart[b + 1]; ++e) {
        const zf *T = tab + ((int64_t)vslot[e] * np + p) * np;
        const zf *m = M + (int64_t)vsrc[e] * np * LM_MAXV + v;
        zf s = {0.f, 0.f};
        for (int q = 0; q < np; ++q) cfma32(s, T[q], m[q * LM_MAXV]);
        acc = acc + s;
    }
    Lc[(b * np + p) * LM_MAXV + v] = Lc[(b * np + p) * LM_MAXV + v] + acc;
}

// L2T in k2 (FP32) and the near g_2^t pairs (kernel values from the FP64 quadrature,
// multiply-adds in FP32), one thread per target of a leaf
__global__ void k_cross_leaf32(LeafGeom g, int P, double k2, const double *xt, const double *yt, const int64_t *lt,
                               const int64_t *ustart, const int32_t *usrc, const double *xs, const double *ysm,
                               const int64_t *lsrc, CrossNear nq, const zf *Lc, const zd *qs, int64_t ns,
                               int64_t nt, int nvec, zd *us)
{
    const int np = 2 * P + 1;
    const int64_t b = blockIdx.x;
    double cx, cy;
    leaf_centre(g, b, &cx, &cy);
    const float sc = (float)(k2 * g.w);
    const zf *Lb = Lc + b * np * LM_MAXV;
    for (int64_t i = lt[b] + threadIdx.x; i < lt[b + 1]; i += blockDim.x) {
        const double xi = xt[i], yi = yt[i];
        zf acc[LM_MAXV];
        for (int v = 0; v < nvec; ++v) acc[v] = zf{0.f, 0.f};
        {
            const float rx = (float)(xi - cx), ry = (float)(yi - cy), r = sqrtf(rx * rx + ry * ry);
            float J[LM_MAXP + 1];
            bessel_j_scaled<float>(P, (float)k2 * r, sc, J);
            const zf z = r > 0.f ? zf{rx / r, ry / r} : zf{1.f, 0.f};
            zf zp = {1.f, 0.f};
            for (int v = 0; v < nvec; ++v) cfma32(acc[v], zf{J[0], 0.f}, Lb[P * LM_MAXV + v]);
            for (int m = 1; m <= P; ++m) {
                zp = zp * z;
                const zf bp = J[m] * zp, bn = ((m & 1) ? -J[m] : J[m]) * conj(zp);
                for (int v = 0; v < nvec; ++v) {
                    cfma32(acc[v], bp, Lb[(P + m) * LM_MAXV + v]);
                    cfma32(acc[v], bn, Lb[(P - m) * LM_MAXV + v]);
                }
            }
        }
        for (int64_t e = ustart[b]; e < ustart[b + 1]; ++e) {
            const int32_t s = usrc[e];
            zf part[LM_MAXV]; // one source leaf summed on its own
            for (int v = 0; v < nvec; ++v) part[v] = zf{0.f, 0.f};
            for (int64_t j = lsrc[s]; j < lsrc[s + 1]; ++j) {
                const zd gd = cross_near(nq, k2, fabs(xi - xs[j]), yi, -ysm[j]);
                const zf gij = {(float)gd.re, (float)gd.im};
                for (int v = 0; v < nvec; ++v) {
                    const zd qd = qs[(int64_t)v * ns + j];
                    cfma32(part[v], gij, zf{(float)qd.re, (float)qd.im});
                }
            }
            for (int v = 0; v < nvec; ++v) acc[v] = acc[v] + part[v];
        }
        for (int v = 0; v < nvec; ++v) us[(int64_t)v * nt + i] = zd{acc[v].re, acc[v].im};
    }
}

__global__ void k_mirror(const double *y, int64_t n, double *out)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = -y[i];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
static int gridc(int64_t n, int b) { return (int)((n + b - 1) / b); }
static int64_t floordiv2(int64_t a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }
static bool adjacent(int64_t c1, int64_t r1, int64_t c2, int64_t r2)
{
    return std::abs(c1 - c2) <= 1 && std::abs(r1 - r2) <= 1;
}
// image row of mirrored source row rs: g_2^t (term 0) like tt, g_2^b (term 1) like bt
static int64_t cross_img_row(int term, int64_t rs, int64_t nrow) { return term == 0 ? -1 - rs : rs + 2 * nrow; }

// one point set onto the shared lattice (x0, R, L): perm, leaf starts, sorted points
static lm_status cross_tree(lm_cross_s *c, const double *x, const double *y, int64_t n, int64_t **perm,
                            int64_t **ls, double **xs, double **ys, cudaStream_t st)
{
    const int64_t ncol = (int64_t)c->R << c->L, nrow = (int64_t)1 << c->L;
    const double w = ldexp(c->med.d, -c->L);
    int32_t *key, *cnt, *cur;
    CTRY(calloc_dev(c, &key, n));
    CTRY(calloc_dev(c, &cnt, c->nleaf));
    CTRY(calloc_dev(c, &cur, c->nleaf));
    CTRY(calloc_dev(c, ls, c->nleaf + 1));
    CTRY(calloc_dev(c, perm, n));
    CTRY(calloc_dev(c, xs, n));
    CTRY(calloc_dev(c, ys, n));
    LM_CUDA(cudaMemsetAsync(cnt, 0, c->nleaf * sizeof(int32_t), st));
    LM_CUDA(cudaMemsetAsync(cur, 0, c->nleaf * sizeof(int32_t), st));
    k_keys<<<gridc(n, 256), 256, 0, st>>>(x, y, n, c->x0, w, ncol, nrow, key, cnt);
    k_scan<<<1, 1024, 0, st>>>(cnt, c->nleaf, *ls);
    k_scatter<<<gridc(n, 256), 256, 0, st>>>(key, n, *ls, cur, *perm);
    k_leafsort<<<(unsigned)c->nleaf, 256, 0, st>>>(*ls, *perm, c->dflag);
    k_gather_pts<<<gridc(n, 256), 256, 0, st>>>(x, y, *perm, n, *xs, *ys);
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

// x-extent and validity (-d < y < 0) of one point set
static lm_status cross_extent(lm_cross_s *c, const double *x, const double *y, int64_t n, double *mn, double *mx,
                              cudaStream_t st)
{
    const int nb = (int)std::min<int64_t>(1024, (n + 255) / 256);
    double *bmin, *bmax;
    CTRY(calloc_dev(c, &bmin, nb));
    CTRY(calloc_dev(c, &bmax, nb));
    LM_CUDA(cudaMemsetAsync(c->dflag, 0, 4 * sizeof(int), st));
    k_minmax<<<nb, 256, 0, st>>>(x, y, n, c->med.d, bmin, bmax, c->dflag);
    std::vector<double> hmin(nb), hmax(nb);
    int hflag = 0;
    LM_CUDA(cudaMemcpyAsync(hmin.data(), bmin, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaMemcpyAsync(hmax.data(), bmax, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaMemcpyAsync(&hflag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    if (hflag & 1) {
        lm_set_error("build_cross: a point is non-finite, or a source not inside 0 < y < d, or a target not "
                     "inside -d < y < 0");
        return LM_EINVAL;
    }
    for (int i = 0; i < nb; ++i) {
        *mn = fmin(*mn, hmin[i]);
        *mx = fmax(*mx, hmax[i]);
    }
    return LM_OK;
}

static lm_status cross_setup(lm_cross_s *c, const double *xs, const double *ys, const double *xt, const double *yt,
                             cudaStream_t st)
{
    const int P = c->p, np = 2 * P + 1;
    const double k1 = c->med.k1, k2 = c->med.k2, k3 = c->med.k3, d = c->med.d;
    CTRY(calloc_dev(c, &c->dflag, 4));
    double *ym;
    CTRY(calloc_dev(c, &ym, c->ns));
    k_mirror<<<gridc(c->ns, 256), 256, 0, st>>>(ys, c->ns, ym);
    double mn = 1e300, mx = -1e300;
    CTRY(cross_extent(c, xs, ym, c->ns, &mn, &mx, st));
    CTRY(cross_extent(c, xt, yt, c->nt, &mn, &mx, st));
    const double f0 = floor(mn / d), f1 = floor(mx / d);
    // root count checked in double before it becomes an int
    const double roots = f1 - f0 + 1.0;
    if (!std::isfinite(roots) || roots < 1.0 || roots > (double)(1 << 30)) {
        lm_set_error("build_cross: the x extent spans %g layer thicknesses; at most 2^30 roots are supported",
                     roots);
        return LM_EINVAL;
    }
    c->x0 = f0 * d;
    c->R = (int)roots;
    const int64_t nmax = std::max(c->ns, c->nt);
    if (c->med.opt.depth >= 0) {
        c->L = c->med.opt.depth;
    } else {
        int L = 0;
        while ((double)nmax > (double)c->med.opt.leaf_target * c->R * pow(4.0, L)) ++L;
        c->L = L;
    }
    const int L = c->L;
    c->nleaf = ((int64_t)c->R << L) << L;
    if (c->nleaf > (int64_t)1 << 28) {
        lm_set_error("build_cross: %lld leaves is beyond this build", (long long)c->nleaf);
        return LM_ENOTSUP;
    }
    LM_CUDA(cudaMemsetAsync(c->dflag, 0, 4 * sizeof(int), st));
    CTRY(cross_tree(c, xs, ym, c->ns, &c->perm_s, &c->ls_s, &c->xs_s, &c->ys_s, st));
    CTRY(cross_tree(c, xt, yt, c->nt, &c->perm_t, &c->ls_t, &c->xs_t, &c->ys_t, st));

    // levels: scales, expansions, shift tables (sources in k1, targets in k2)
    c->lev.resize(L + 1);
    for (int l = 0; l <= L; ++l) {
        CrossLevel &lv = c->lev[l];
        lv.ncol = (int64_t)c->R << l;
        lv.nrow = (int64_t)1 << l;
        lv.nbox = lv.ncol * lv.nrow;
        lv.w = ldexp(d, -l);
        std::vector<double> at(P + 1), as(P + 1);
        double vt = 1.0, vs = 1.0;
        for (int n = 0; n <= P; ++n) {
            at[n] = vt;
            as[n] = vs;
            vt *= 0.5 * k2 * lv.w / (n + 1);
            vs *= 0.5 * k1 * lv.w / (n + 1);
        }
        CTRY(calloc_dev(c, &lv.sc_t, P + 1));
        CTRY(calloc_dev(c, &lv.sc_s, P + 1));
        LM_CUDA(cudaMemcpyAsync(lv.sc_t, at.data(), (P + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
        LM_CUDA(cudaMemcpyAsync(lv.sc_s, as.data(), (P + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
        CTRY(calloc_dev(c, &lv.M, (size_t)lv.nbox * np * LM_MAXV));
        CTRY(calloc_dev(c, &lv.Lc, (size_t)lv.nbox * np * LM_MAXV));
        lv.m2m = lv.l2l = nullptr;
        if (l < L) CTRY(calloc_dev(c, &lv.m2m, 4 * np * np));
        if (l > 0) CTRY(calloc_dev(c, &lv.l2l, 4 * np * np));
    }
    for (int l = 0; l < L; ++l) {
        CrossLevel &par = c->lev[l], &ch = c->lev[l + 1];
        k_shift_tables<<<gridc(4 * np * np, 128), 128, 0, st>>>(k1, P, ch.w, ch.sc_s, par.sc_s, par.m2m, nullptr);
        k_shift_tables<<<gridc(4 * np * np, 128), 128, 0, st>>>(k2, P, ch.w, ch.sc_t, par.sc_t, nullptr, ch.l2l);
    }

    // V lists and classes (host): target-major, then term, then source box
    const size_t shm = (2 * 16 * np + 16) * sizeof(zd); // m2l_table_body's staging
    LM_CUDA(lm_raise_smem((const void *)k_cross_m2l, LM_SMEM_CROSS_M2L, (int)shm));
    for (int l = 0; l <= L; ++l) {
        CrossLevel &lv = c->lev[l];
        std::map<std::tuple<int, int, int, int>, int> cls;
        std::vector<int> ct_, cd_, crt_, crs_;
        std::vector<int64_t> vstart(lv.nbox + 1, 0);
        std::vector<int32_t> vsrc, vslot;
        for (int64_t b = 0; b < lv.nbox; ++b) {
            const int64_t rt = b / lv.ncol, ctc = b % lv.ncol;
            for (int term = 0; term < 2; ++term) {
                for (int64_t rs = 0; rs < lv.nrow; ++rs) {
                    const int64_t ri = cross_img_row(term, rs, lv.nrow);
                    if (l > 0 && (ri < rt - 3 || ri > rt + 3)) continue;
                    const int64_t clo = l > 0 ? std::max<int64_t>(0, ctc - 3) : 0;
                    const int64_t chi = l > 0 ? std::min<int64_t>(lv.ncol - 1, ctc + 3) : lv.ncol - 1;
                    for (int64_t cs = clo; cs <= chi; ++cs) {
                        if (adjacent(ctc, rt, cs, ri)) continue;
                        if (l > 0 && !adjacent(ctc / 2, rt / 2, cs / 2, floordiv2(ri))) continue;
                        const auto key = std::make_tuple(term, (int)(ctc - cs), (int)rt, (int)rs);
                        auto it = cls.find(key);
                        int slot;
                        if (it == cls.end()) {
                            slot = (int)ct_.size();
                            cls[key] = slot;
                            ct_.push_back(term);
                            cd_.push_back((int)(ctc - cs));
                            crt_.push_back((int)rt);
                            crs_.push_back((int)rs);
                        } else {
                            slot = it->second;
                        }
                        vsrc.push_back((int32_t)(rs * lv.ncol + cs));
                        vslot.push_back(slot);
                    }
                }
            }
            vstart[b + 1] = (int64_t)vsrc.size();
        }
        lv.nv = (int64_t)vsrc.size();
        lv.ncls = (int)ct_.size();
        CTRY(calloc_dev(c, &lv.vstart, lv.nbox + 1));
        CTRY(calloc_dev(c, &lv.vsrc, lv.nv));
        CTRY(calloc_dev(c, &lv.vslot, lv.nv));
        CTRY(calloc_dev(c, &lv.tab, (size_t)std::max(1, lv.ncls) * np * np));
        LM_CUDA(cudaMemcpyAsync(lv.vstart, vstart.data(), vstart.size() * sizeof(int64_t), cudaMemcpyHostToDevice,
                                st));
        if (lv.nv > 0) {
            LM_CUDA(cudaMemcpyAsync(lv.vsrc, vsrc.data(), vsrc.size() * 4, cudaMemcpyHostToDevice, st));
            LM_CUDA(cudaMemcpyAsync(lv.vslot, vslot.data(), vslot.size() * 4, cudaMemcpyHostToDevice, st));
        }
        if (lv.ncls > 0) {
            int *dbuf;
            CTRY(calloc_dev(c, &dbuf, 4 * lv.ncls));
            std::vector<int> hb;
            for (auto *v : {&ct_, &cd_, &crt_, &crs_}) hb.insert(hb.end(), v->begin(), v->end());
            LM_CUDA(cudaMemcpyAsync(dbuf, hb.data(), hb.size() * sizeof(int), cudaMemcpyHostToDevice, st));
            k_cross_m2l<<<lv.ncls, 256, shm, st>>>(k1, k2, k3, d, P, lv.w, k2 * lv.w, k1 * lv.w, dbuf,
                                                   dbuf + lv.ncls, dbuf + 2 * lv.ncls, dbuf + 3 * lv.ncls,
                                                   lv.ncls, lv.tab, c->dflag);
            LM_CUDA(cudaGetLastError());
        }
        LM_CUDA(cudaStreamSynchronize(st)); // host vectors go out of scope
    }
    // U list at the leaf level: adjacent g_2^t pairs (target row 0, mirrored source row 0)
    {
        const CrossLevel &lv = c->lev[L];
        std::vector<int64_t> us(lv.nbox + 1, 0);
        std::vector<int32_t> src;
        for (int64_t b = 0; b < lv.nbox; ++b) {
            const int64_t rt = b / lv.ncol, ctc = b % lv.ncol;
            for (int64_t rs = 0; rs < lv.nrow; ++rs) {
                const int64_t ri = cross_img_row(0, rs, lv.nrow);
                if (ri < rt - 1 || ri > rt + 1) continue;
                for (int64_t cs = std::max<int64_t>(0, ctc - 1); cs <= std::min<int64_t>(lv.ncol - 1, ctc + 1); ++cs)
                    src.push_back((int32_t)(rs * lv.ncol + cs));
            }
            us[b + 1] = (int64_t)src.size();
        }
        c->nu = (int64_t)src.size();
        CTRY(calloc_dev(c, &c->ustart, lv.nbox + 1));
        CTRY(calloc_dev(c, &c->usrc, c->nu));
        LM_CUDA(cudaMemcpyAsync(c->ustart, us.data(), us.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        if (c->nu > 0)
            LM_CUDA(cudaMemcpyAsync(c->usrc, src.data(), src.size() * 4, cudaMemcpyHostToDevice, st));
        LM_CUDA(cudaStreamSynchronize(st));
    }
    // near-field quadrature of g_2^t (same contour and orders as the middle layer's)
    {
        const double km = fmax(k1, fmax(k2, k3)), kmin = fmin(k1, fmin(k2, k3));
        const double cc = 1.5 * km + 1.0, a = 0.5, delta = fmin(0.25, 0.5 * kmin);
        const int nflat = (int)ceil((cc - 2.0 * delta) / 1.0), order = c->med.opt.seg_order;
        c->nseg = (nflat + 2) * order;
        c->nray = c->med.opt.tail_rays;
        c->ntail = c->med.opt.tail_order;
        const int nt = c->nray * c->ntail;
        CTRY(calloc_dev(c, &c->seg_lam, c->nseg));
        CTRY(calloc_dev(c, &c->seg_s1, c->nseg));
        CTRY(calloc_dev(c, &c->seg_s2, c->nseg));
        CTRY(calloc_dev(c, &c->seg_w, 2 * c->nseg));
        CTRY(calloc_dev(c, &c->tail_lam, nt));
        CTRY(calloc_dev(c, &c->tail_s1, nt));
        CTRY(calloc_dev(c, &c->tail_s2, nt));
        CTRY(calloc_dev(c, &c->tail_w, 4 * nt));
        k_cross_near_seg<<<gridc(c->nseg, 64), 64, 0, st>>>(k1, k2, k3, d, cc, a, delta, nflat, order, c->seg_lam,
                                                            c->seg_s1, c->seg_s2, c->seg_w, c->nseg);
        k_cross_near_tail<<<gridc(nt, 64), 64, 0, st>>>(k1, k2, k3, d, cc, c->nray, c->ntail, c->tail_lam,
                                                        c->tail_s1, c->tail_s2, c->tail_w);
    }
    CTRY(calloc_dev(c, &c->qs, (size_t)LM_MAXV * c->ns));
    CTRY(calloc_dev(c, &c->us, (size_t)LM_MAXV * c->nt));
    int hflag = 0;
    LM_CUDA(cudaGetLastError());
    LM_CUDA(cudaMemcpyAsync(&hflag, c->dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    if (hflag & 2) {
        lm_set_error("build_cross: a leaf holds more than %d points; use a deeper tree", LM_MAXLEAF);
        return LM_ENOTSUP;
    }
    if (hflag & (8 | 16)) {
        lm_set_error("build_cross: an M2L table could not be built at this order");
        return LM_ENOTSUP;
    }
    if (c->med.opt.precision == LM_MIXED) {
        for (int l = 0; l <= L; ++l) {
            CrossLevel &lv = c->lev[l];
            const int64_t nt2 = (int64_t)std::max(1, lv.ncls) * np * np, ns2 = 4 * np * np;
            CTRY(calloc_dev(c, &lv.tab32, nt2));
            CTRY(calloc_dev(c, &lv.M32, (size_t)lv.nbox * np * LM_MAXV));
            CTRY(calloc_dev(c, &lv.L32, (size_t)lv.nbox * np * LM_MAXV));
            k_cross_to32<<<gridc(nt2, 256), 256, 0, st>>>(lv.tab, nt2, lv.tab32);
            lv.m2m32 = lv.l2l32 = nullptr;
            if (lv.m2m) {
                CTRY(calloc_dev(c, &lv.m2m32, ns2));
                k_cross_to32<<<gridc(ns2, 256), 256, 0, st>>>(lv.m2m, ns2, lv.m2m32);
            }
            if (lv.l2l) {
                CTRY(calloc_dev(c, &lv.l2l32, ns2));
                k_cross_to32<<<gridc(ns2, 256), 256, 0, st>>>(lv.l2l, ns2, lv.l2l32);
            }
        }
        LM_CUDA(cudaGetLastError());
        LM_CUDA(cudaStreamSynchronize(st));
    }
    return LM_OK;
}

extern "C" void lm_destroy_cross(lm_cross c)
{
    if (!c) return;
    for (void *p : c->allocs) cudaFree(p);
    delete c;
}

extern "C" lm_status lm_build_cross(lm_medium m, const double *xs, const double *ys, int64_t ns, const double *xt,
                                    const double *yt, int64_t nt, void *stream, lm_cross *out)
{
    if (!out || !m || !xs || !ys || !xt || !yt || ns < 1 || nt < 1) {
        lm_set_error("build_cross: NULL argument or empty point set");
        return LM_EINVAL;
    }
    *out = nullptr;
    if (m->opt.kernel != LM_KERNEL_G || m->opt.top_bc != LM_BC_TRANSMISSION ||
        m->opt.bottom_bc != LM_BC_TRANSMISSION) {
        lm_set_error("build_cross: the cross-layer operator is kernel G, with transmission interfaces");
        return LM_ENOTSUP;
    }
    lm_cross_s *c = new (std::nothrow) lm_cross_s();
    if (!c) {
        lm_set_error("build_cross: host allocation failed");
        return LM_ENOMEM;
    }
    c->med = *m;
    c->p = m->opt.p;
    c->ns = ns;
    c->nt = nt;
    lm_status s = cross_setup(c, xs, ys, xt, yt, (cudaStream_t)stream);
    if (s != LM_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);
        lm_destroy_cross(c);
        return s;
    }
    *out = c;
    return LM_OK;
}

extern "C" lm_status lm_cross_info(lm_cross c, int64_t *ns, int64_t *nt, int *R, int *depth, double *x_origin)
{
    if (!c) {
        lm_set_error("cross_info: NULL handle");
        return LM_EINVAL;
    }
    if (ns) *ns = c->ns;
    if (nt) *nt = c->nt;
    if (R) *R = c->R;
    if (depth) *depth = c->L;
    if (x_origin) *x_origin = c->x0;
    return LM_OK;
}

extern "C" lm_status lm_cross_apply(lm_cross c, const void *q, int nvec, void *u, void *stream)
{
    if (!c || !q || !u || nvec < 1) {
        lm_set_error("cross_apply: NULL handle or buffer, or nvec < 1");
        return LM_EINVAL;
    }
    const char *a = (const char *)q, *b = (const char *)u;
    if (a < b + (size_t)nvec * c->nt * sizeof(zd) && b < a + (size_t)nvec * c->ns * sizeof(zd)) {
        lm_set_error("cross_apply: q and u overlap");
        return LM_EINVAL;
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int L = c->L, P = c->p, np = 2 * P + 1;
    CrossNear nq{c->nseg, c->nray, c->ntail, c->seg_lam, c->seg_s1, c->seg_s2, c->seg_w,
                 c->tail_lam, c->tail_s1, c->tail_s2, c->tail_w};
    const zd *qd = (const zd *)q;
    zd *ud = (zd *)u;
    for (int v0 = 0; v0 < nvec; v0 += LM_MAXV) {
        const int nv = std::min(LM_MAXV, nvec - v0);
        k_permute_in<<<gridc(c->ns, 256), 256, 0, st>>>(qd + (int64_t)v0 * c->ns, c->perm_s, c->ns, nv, 0, c->qs);
        if (c->med.opt.precision == LM_MIXED) {
            {
                const CrossLevel &lv = c->lev[L];
                k_cross_p2m32<<<(unsigned)lv.nbox, 128, 0, st>>>(LeafGeom{lv.ncol, c->x0, lv.w}, P, c->med.k1,
                                                                  c->xs_s, c->ys_s, c->ls_s, c->qs, c->ns, nv, lv.M32);
            }
            for (int l = L - 1; l >= 0; --l) {
                const CrossLevel &lv = c->lev[l];
                k_cross_m2m32<<<gridc(lv.nbox * np * nv, 128), 128, 0, st>>>(lv.ncol, lv.nbox, P, nv, lv.m2m32,
                                                                            c->lev[l + 1].M32, lv.M32);
            }
            for (int l = 0; l <= L; ++l) {
                const CrossLevel &lv = c->lev[l];
                const int64_t tot = lv.nbox * np * nv;
                if (l == 0)
                    LM_CUDA(cudaMemsetAsync(lv.L32, 0, lv.nbox * np * LM_MAXV * sizeof(zf), st));
                else
                    k_cross_l2l32<<<gridc(tot, 128), 128, 0, st>>>(lv.ncol, lv.nbox, P, nv, lv.l2l32,
                                                                   c->lev[l - 1].L32, lv.L32);
                if (lv.nv > 0)
                    k_cross_m2l32<<<gridc(tot, 128), 128, 0, st>>>(lv.nbox, P, nv, lv.vstart, lv.vsrc, lv.vslot,
                                                                   lv.tab32, lv.M32, lv.L32);
            }
            const CrossLevel &lv = c->lev[L];
            k_cross_leaf32<<<(unsigned)lv.nbox, 64, 0, st>>>(LeafGeom{lv.ncol, c->x0, lv.w}, P, c->med.k2, c->xs_t,
                                                             c->ys_t, c->ls_t, c->ustart, c->usrc, c->xs_s, c->ys_s,
                                                             c->ls_s, nq, lv.L32, c->qs, c->ns, c->nt, nv, c->us);
            k_permute_out<<<gridc(c->nt, 256), 256, 0, st>>>(c->us, c->perm_t, c->nt, nv, 0, ud + (int64_t)v0 * c->nt);
            LM_CUDA(cudaGetLastError());
            continue;
        }
        {
            const CrossLevel &lv = c->lev[L];
            const size_t shm = (CROSS_P2M_CHUNK * np + CROSS_P2M_CHUNK * LM_MAXV) * sizeof(zd);
            k_p2m64<<<(unsigned)lv.nbox, 256, shm, st>>>(LeafGeom{lv.ncol, c->x0, lv.w}, P, c->med.k1, c->xs_s,
                                                         c->ys_s, c->ls_s, c->qs, c->ns, nv, lv.M);
        }
        for (int l = L - 1; l >= 0; --l) {
            const CrossLevel &lv = c->lev[l];
            k_m2m64<<<gridc(lv.nbox * np * nv, 128), 128, 0, st>>>(lv.ncol, lv.nbox, P, nv, lv.m2m,
                                                                   c->lev[l + 1].M, lv.M);
        }
        for (int l = 0; l <= L; ++l) {
            const CrossLevel &lv = c->lev[l];
            const int64_t tot = lv.nbox * np * nv;
            if (l == 0)
                LM_CUDA(cudaMemsetAsync(lv.Lc, 0, lv.nbox * np * LM_MAXV * sizeof(zd), st));
            else
                k_l2l64<<<gridc(tot, 128), 128, 0, st>>>(lv.ncol, lv.nbox, P, nv, lv.l2l, c->lev[l - 1].Lc, lv.Lc);
            if (lv.nv > 0)
                k_m2l64<<<gridc(tot, 128), 128, 0, st>>>(lv.nbox, P, nv, lv.vstart, lv.vsrc, lv.vslot, lv.tab,
                                                         lv.M, lv.Lc);
        }
        {
            const CrossLevel &lv = c->lev[L];
            k_cross_leaf<<<(unsigned)lv.nbox, 64, 0, st>>>(LeafGeom{lv.ncol, c->x0, lv.w}, P, c->med.k2, c->xs_t,
                                                           c->ys_t, c->ls_t, c->ustart, c->usrc, c->xs_s, c->ys_s,
                                                           c->ls_s, nq, lv.Lc, c->qs, c->ns, c->nt, nv, c->us);
        }
        k_permute_out<<<gridc(c->nt, 256), 256, 0, st>>>(c->us, c->perm_t, c->nt, nv, 0, ud + (int64_t)v0 * c->nt);
        LM_CUDA(cudaGetLastError());
    }
    return LM_OK;
}
