// lmfmm_setup.cu -- Algorithm 1, step 1 on the device: the strip-forest
// quadtree, interaction lists, translation tables and near-field quadrature.
#include <math.h>
#include <cmath>
#include <stdio.h>
#include <algorithm>
#include <map>
#include <tuple>

#include "internal.h"
#include "tables.cuh"

// ---------------------------------------------------------------------------
// Tree
// ---------------------------------------------------------------------------
__global__ void k_minmax(const double *x, const double *y, int64_t n, double d, double *bmin,
                         double *bmax, int *flag)
{
    __shared__ double smin[256], smax[256];
    double mn = 1e308, mx = -1e308;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        double xi = x[i], yi = y[i];
        if (!isfinite(xi) || !isfinite(yi) || !(yi < 0.0) || !(yi > -d)) atomicOr(flag, 1);
        mn = fmin(mn, xi);
        mx = fmax(mx, xi);
    }
    smin[threadIdx.x] = mn;
    smax[threadIdx.x] = mx;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) {
            smin[threadIdx.x] = fmin(smin[threadIdx.x], smin[threadIdx.x + s]);
            smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + s]);
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        bmin[blockIdx.x] = smin[0];
        bmax[blockIdx.x] = smax[0];
    }
}

// leaf of each point: col = floor((x - x0)/w), row = floor(-y/w), clamped
__global__ void k_keys(const double *x, const double *y, int64_t n, double x0, double w,
                       int64_t ncol, int64_t nrow, int32_t *key, int32_t *cnt)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t c = (int64_t)floor((x[i] - x0) / w), r = (int64_t)floor(-y[i] / w);
    c = c < 0 ? 0 : (c > ncol - 1 ? ncol - 1 : c);
    r = r < 0 ? 0 : (r > nrow - 1 ? nrow - 1 : r);
    int32_t k = (int32_t)(r * ncol + c);
    key[i] = k;
    atomicAdd(&cnt[k], 1);
}

// exclusive scan of cnt[0..m) into start[0..m] by one block
__global__ void k_scan(const int32_t *cnt, int64_t m, int64_t *start)
{
    __shared__ int64_t part[1024];
    int64_t chunk = (m + blockDim.x - 1) / blockDim.x;
    int64_t lo = threadIdx.x * chunk, hi = min(m, lo + chunk);
    int64_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += cnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            int64_t v = part[i];
            part[i] = acc;
            acc += v;
        }
        start[m] = acc;
    }
    __syncthreads();
    int64_t acc = part[threadIdx.x];
    for (int64_t i = lo; i < hi; ++i) {
        start[i] = acc;
        acc += cnt[i];
    }
}

__global__ void k_scatter(const int32_t *key, int64_t n, const int64_t *start, int32_t *cursor,
                          int64_t *tmp)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int32_t k = key[i];
    int pos = atomicAdd(&cursor[k], 1);
    tmp[start[k] + pos] = i;
}

// sort each leaf's input indices ascending (bitonic sort in shared memory)
__global__ void k_leafsort(const int64_t *start, int64_t *idx, int *flag)
{
    __shared__ int32_t s[LM_MAXLEAF];
    int64_t b = blockIdx.x;
    int64_t lo = start[b], cnt = start[b + 1] - lo;
    if (cnt <= 1) return;
    if (cnt > LM_MAXLEAF) {
        if (threadIdx.x == 0) atomicOr(flag, 2);
        return;
    }
    int m = 1;
    while (m < cnt) m <<= 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) s[i] = i < cnt ? (int32_t)idx[lo + i] : INT32_MAX;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                int ixj = i ^ j;
                if (ixj > i) {
                    bool up = (i & k) == 0;
                    int32_t a = s[i], c = s[ixj];
                    if ((a > c) == up) {
                        s[i] = c;
                        s[ixj] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) idx[lo + i] = s[i];
}

__global__ void k_gather_pts(const double *x, const double *y, const int64_t *perm, int64_t n,
                             double *xs, double *ys)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    xs[i] = x[j];
    ys[i] = y[j];
}

// ---------------------------------------------------------------------------
// Interaction lists.  Image row of source row r for term m at a level with
// nrow rows: free r; tt -1-r (mirror in y = 0); bb 2nrow-1-r (mirror in
// y = -d); tb r-2nrow (shift +2d); bt r+2nrow (shift -2d).
// ---------------------------------------------------------------------------
// inverse: source row whose image row is ri
__host__ __device__ inline int64_t src_row(int term, int64_t ri, int64_t nrow)
{
    switch (term) {
    case 0: return ri;
    case 1: return -1 - ri;
    case 2: return 2 * nrow - 1 - ri;
    case 3: return ri + 2 * nrow;
    default: return ri - 2 * nrow;
    }
}
__host__ __device__ inline int64_t floordiv2(int64_t a) { return a >= 0 ? a / 2 : -((-a + 1) / 2); }
__host__ __device__ inline bool adj(int64_t c1, int64_t r1, int64_t c2, int64_t r2)
{
    return (c1 - c2 <= 1 && c2 - c1 <= 1) && (r1 - r2 <= 1 && r2 - r1 <= 1);
}
__host__ __device__ inline bool v_rule(int l, int64_t ct, int64_t rt, int64_t cs, int64_t ri)
{
    if (adj(ct, rt, cs, ri)) return false;
    if (l == 0) return true;
    return adj(ct / 2, floordiv2(rt), cs / 2, floordiv2(ri));
}

struct SlotMap {
    int DC;          // dc in [-DC, DC]
    int32_t *map;    // [5][2DC+1][7] slot or -1 (dr in [-3, 3])
};
__host__ __device__ inline int slot_index(int DC, int term, int dc, int dr)
{
    return (term * (2 * DC + 1) + (dc + DC)) * 7 + (dr + 3);
}

// pass 0: count; pass 1: fill. One thread per target box.
__global__ void k_vlist(int l, int64_t ncol, int64_t nrow, int DC, const int32_t *slotmap,
                        int64_t *vstart, int32_t *vsrc, int32_t *vslot, int32_t *vterm, int pass,
                        int *flag)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ncol * nrow) return;
    int64_t rt = t / ncol, ct = t % ncol;
    int64_t pos = pass ? vstart[t] : 0, cnt = 0;
    for (int term = 0; term < 5; ++term) {
        // source rows in ascending order
        int64_t rlo = 0, rhi = nrow - 1;
        if (l > 0) {
            int64_t a = src_row(term, rt - 3, nrow), b = src_row(term, rt + 3, nrow);
            rlo = max((int64_t)0, min(a, b));
            rhi = min(nrow - 1, max(a, b));
        }
        int64_t clo = l > 0 ? max((int64_t)0, ct - 3) : 0;
        int64_t chi = l > 0 ? min(ncol - 1, ct + 3) : ncol - 1;
        for (int64_t rs = rlo; rs <= rhi; ++rs) {
            int64_t ri = img_row(term, rs, nrow);
            for (int64_t cs = clo; cs <= chi; ++cs) {
                if (!v_rule(l, ct, rt, cs, ri)) continue;
                if (pass) {
                    int64_t dc = ct - cs, dr = rt - ri;
                    int slot = -1;
                    if (dc >= -DC && dc <= DC && dr >= -3 && dr <= 3)
                        slot = slotmap[slot_index(DC, term, (int)dc, (int)dr)];
                    if (slot < 0) atomicOr(flag, 4);
                    vsrc[pos] = (int32_t)(rs * ncol + cs);
                    vslot[pos] = slot < 0 ? 0 : slot;
                    vterm[pos] = term;
                    ++pos;
                }
                ++cnt;
            }
        }
    }
    if (!pass) vstart[t] = cnt; // counts, scanned on the host side afterwards
}

// U list at the leaf level: image adjacent to target (free term includes itself)
__global__ void k_ulist(int64_t ncol, int64_t nrow, int64_t *ustart, int32_t *usrc, int32_t *uterm,
                        int pass)
{
    int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ncol * nrow) return;
    int64_t rt = t / ncol, ct = t % ncol;
    int64_t pos = pass ? ustart[t] : 0, cnt = 0;
    for (int term = 0; term < 5; ++term) {
        int64_t a = src_row(term, rt - 1, nrow), b = src_row(term, rt + 1, nrow);
        int64_t rlo = max((int64_t)0, min(a, b)), rhi = min(nrow - 1, max(a, b));
        for (int64_t rs = rlo; rs <= rhi; ++rs) {
            int64_t ri = img_row(term, rs, nrow);
            for (int64_t cs = max((int64_t)0, ct - 1); cs <= min(ncol - 1, ct + 1); ++cs) {
                if (!adj(ct, rt, cs, ri)) continue;
                if (pass) {
                    usrc[pos] = (int32_t)(rs * ncol + cs);
                    uterm[pos] = term;
                    ++pos;
                }
                ++cnt;
            }
        }
    }
    if (!pass) ustart[t] = cnt;
}

// in-place exclusive scan of counts c[0..m) (stored as int64) -> start[0..m]
__global__ void k_scan64(int64_t *c, int64_t m)
{
    __shared__ int64_t part[1024];
    int64_t chunk = (m + blockDim.x - 1) / blockDim.x;
    int64_t lo = threadIdx.x * chunk, hi = min(m, lo + chunk);
    int64_t s = 0;
    for (int64_t i = lo; i < hi; ++i) s += c[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int64_t acc = 0;
        for (int i = 0; i < (int)blockDim.x; ++i) {
            int64_t v = part[i];
            part[i] = acc;
            acc += v;
        }
        c[m] = acc;
    }
    __syncthreads();
    int64_t acc = part[threadIdx.x];
    for (int64_t i = lo; i < hi; ++i) {
        int64_t v = c[i];
        c[i] = acc;
        acc += v;
    }
}

// ---------------------------------------------------------------------------
// Near-field quadrature tables.
//  Segment (first contour, Sec. 5): a trapezoid from 0 down to delta - i a,
//  along -i a to c - delta - i a, and up to c; the negative half is folded
//  onto it (integrand 2 cos(lambda X) ...).  Gauss-Legendre panels.
//  Tail: rays lambda = c + t e^{i phi_k}, phi_k = k (pi/2) / (nray - 1),
//  t = c v/(1-v), Gauss-Legendre in v.  The half-line integrals of
//  e^{+i lambda X} F and e^{-i lambda X} F go to the ray and its mirror image
//  below the axis, with weights W_u, W_l; with E = e^{i lambda X - s2 h} the
//  mirror's factor is conj(E), so the tail is sum P Re(Z) + i M Im(Z) with
//  P = W_u + W_l, M = W_u - W_l and Z = E (or its X- or h-derivative).  For
//  transmission and Dirichlet/Neumann walls sigma(conj lambda) = conj(sigma)
//  and the tail is real; an impedance wall makes it complex.
// ---------------------------------------------------------------------------
// c_o (optional, [2][nseg]): the weights of 2 i beta / s2 (imp_beta) for the gradient's h-derivative
__global__ void k_near_seg(MediumD m, double c, double a, double delta, int nflat, int order,
                           zd *lam_o, zd *s2_o, zd *w_o, int nseg, zd *c_o = nullptr)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nseg) return;
    int pan = i / order, j = i % order;
    double x, w;
    gl_node(order, j, &x, &w);
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
    zd s2, sig[3];
    densities(m, lam, &s2, sig);
    zd base = cdiv((0.5 * w / (4.0 * M_PI)) * dz, s2);
    lam_o[i] = lam;
    s2_o[i] = s2;
    w_o[i] = base * (sig[0] - zd{refl_inf(m, 0), 0.0});
    w_o[nseg + i] = base * (sig[1] - zd{refl_inf(m, 1), 0.0});
    if (c_o)
        for (int mm = 0; mm < 2; ++mm) c_o[mm * nseg + i] = base * cdiv(zd{0.0, 2.0 * imp_beta(m, mm)}, s2);
}

// With w2_o set (walls on both sides, FP64): w_o takes the single reflection R - R_inf
// and w2_o the multiple reflections sigma - R, summed on different rays (see NearQuad).
// c_o (optional, layout of w_o): P, M weights of 2 i beta / s2 for the gradient's h-derivative
__global__ void k_near_tail(MediumD m, double c, int nray, int order, zd *lam_o, zd *s2_o, zd *w_o,
                            zd *w2_o = nullptr, zd *c_o = nullptr)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int tot = nray * order;
    if (i >= tot) return;
    int k = i / order, j = i % order;
    double x, w;
    gl_node(order, j, &x, &w);
    double v = 0.5 * (x + 1.0), wv = 0.5 * w;
    double t = c * v / (1.0 - v), dt = c / ((1.0 - v) * (1.0 - v));
    double phi = (nray > 1) ? k * (0.5 * M_PI) / (nray - 1) : 0.0;
    // upper ray (for e^{+i lam X}) and its mirror below the axis (for e^{-i lam X})
    zd e = {cos(phi), sin(phi)};
    zd lam = zd{c, 0.0} + t * e, laml = conj(lam);
    zd s2, sig[3], s2l, sigl[3];
    densities(m, lam, &s2, sig);
    densities(m, laml, &s2l, sigl);
    zd bu = cdiv((wv * dt / (4.0 * M_PI)) * e, s2), bl = cdiv((wv * dt / (4.0 * M_PI)) * conj(e), s2l);
    lam_o[i] = lam;
    s2_o[i] = s2;
    for (int mm = 0; mm < 2; ++mm) {
        const zd ri = {refl_inf(m, mm), 0.0};
        if (c_o) {
            const zd tb = {0.0, 2.0 * imp_beta(m, mm)};
            const zd cu = bu * cdiv(tb, s2), cl = bl * cdiv(tb, s2l);
            c_o[((size_t)(2 * mm) * tot) + i] = cu + cl;
            c_o[((size_t)(2 * mm + 1) * tot) + i] = cu - cl;
        }
        if (w2_o) {
            const double kj = mm == 0 ? m.k1 : m.k3;
            const zd r = refl_coef(m, mm, s2, sbranch(lam, kj), kj), rl = refl_coef(m, mm, s2l, sbranch(laml, kj), kj);
            const zd au = bu * (r - ri), al = bl * (rl - ri), mu = bu * (sig[mm] - r), ml = bl * (sigl[mm] - rl);
            w_o[((size_t)(2 * mm) * tot) + i] = au + al;
            w_o[((size_t)(2 * mm + 1) * tot) + i] = au - al;
            w2_o[((size_t)(2 * mm) * tot) + i] = mu + ml;
            w2_o[((size_t)(2 * mm + 1) * tot) + i] = mu - ml;
            continue;
        }
        const zd wu = bu * (sig[mm] - ri), wl = bl * (sigl[mm] - ri);
        w_o[((size_t)(2 * mm) * tot) + i] = wu + wl;     // P
        w_o[((size_t)(2 * mm + 1) * tot) + i] = wu - wl; // M
    }
}

// ---------------------------------------------------------------------------
// Translation tables (scaled; S_l(n) = (k w_l / 2)^|n| / |n|!):
//  M2M (Lemma M2M, reading G3): M_p += sum_q M_q J_{p-q}(k r) e^{-i (p-q) theta},
//     (r, theta) = child centre - parent centre; scaled by S_child(q)/S_parent(p).
//  L2L (Lemma L2L, reading G3): L_p += sum_q L_q J_{p-q}(k r) e^{-i (p-q) theta},
//     (r, theta) = parent centre - child centre; scaled by S_child(p)/S_parent(q).
// ---------------------------------------------------------------------------
__device__ double besj_int(int n, double x)
{
    int a = n < 0 ? -n : n;
    double v = jn(a, x);
    return (n < 0 && (a & 1)) ? -v : v;
}

__global__ void k_shift_tables(double k, int P, double wc, const double *sc_child,
                               const double *sc_par, zd *m2m, zd *l2l)
{
    int np = 2 * P + 1;
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 4 * np * np) return;
    int pos = idx / (np * np), p = (idx / np) % np - P, q = idx % np - P;
    int dy = pos >> 1, dx = pos & 1;
    // child centre - parent centre
    double sx = (dx - 0.5) * wc, sy = -(dy - 0.5) * wc;
    double r = hypot(sx, sy), th = atan2(sy, sx);
    int n = p - q;
    if (m2m) {
        double j = besj_int(n, k * r);
        double s = sc_child[q < 0 ? -q : q] / sc_par[p < 0 ? -p : p];
        m2m[idx] = zd{j * cos(n * th) * s, -j * sin(n * th) * s};
    }
    if (l2l) {
        // parent centre - child centre = -(sx, sy)
        double th2 = atan2(-sy, -sx);
        double j = besj_int(n, k * r);
        double s = sc_child[p < 0 ? -p : p] / sc_par[q < 0 ? -q : q];
        l2l[idx] = zd{j * cos(n * th2) * s, -j * sin(n * th2) * s};
    }
}

// Free-space M2L (Rokhlin's translation): A_pq = (i/4) H_{q-p}(k rho) e^{i (q-p) theta},
// c = target centre - source centre = (dc w, -dr w); scaled by S(p) S(q).
__global__ void k_free_m2l(double k, int P, double w, const int *cdc, const int *cdr,
                           const int *cidx, int ncls, const double *sc, zd *tab)
{
    int np = 2 * P + 1;
    int ci = blockIdx.y;
    if (ci >= ncls) return;
    double cx = cdc[ci] * w, cy = -cdr[ci] * w;
    double rho = hypot(cx, cy), th = atan2(cy, cx);
    zd *T = tab + (int64_t)cidx[ci] * np * np;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < np * np;
         idx += gridDim.x * blockDim.x) {
        int p = idx / np - P, q = idx % np - P;
        int n = q - p, a = n < 0 ? -n : n;
        double jv = jn(a, k * rho), yv = yn(a, k * rho);
        if (n < 0 && (a & 1)) {
            jv = -jv;
            yv = -yv;
        }
        double s = sc[p < 0 ? -p : p] * sc[q < 0 ? -q : q];
        // (i/4)(J + iY) = (-Y/4) + i (J/4)
        zd h = {-0.25 * yv * s, 0.25 * jv * s};
        zd e = {cos(n * th), sin(n * th)};
        T[idx] = h * e;
    }
}

// Layered M2L (Lemma M2L, reading G2 for the phase i^{p-q}):
//   A_pq = (i^{p-q}/4pi) Int Z_t^p Z_s^q e^{i lambda dx - s2 h} sigma_m / s2 d lambda,
//   Z_t = (lambda + tau s2)/k2, Z_s = (lambda + vs s2)/k2,
// scaled by S(p) S(q): the powers are formed as (Z sc/2)^|p| / |p|!.
// Contour: trapezoid segment over [-c, c] (down on the right, up on the
// left) at depth a = min(0.5, 1/|dx|), then steepest-descent rays from +-c.
// One block per class; nodes staged in chunks through shared memory.

__global__ void __launch_bounds__(256) k_image_m2l(MediumD m, int P, double w, double sc, const int *cterm,
                                                   const int *cdc, const int *cdr, const int *cidx, int ncls,
                                                   zd *tab, int *flag)
{
    const int ci = blockIdx.x;
    if (ci >= ncls) return;
    const int term = cterm[ci];
    const int tau = (term == 2 || term == 4) ? 1 : -1;
    const int vs = (term == 2 || term == 3) ? 1 : -1;
    const int is = term == 1 ? 0 : (term == 2 ? 1 : 2);
    auto sigf = [&](zd lam, zd *s2, zd *ss) {
        zd sig[3];
        densities(m, lam, s2, sig);
        *ss = *s2;
        return sig[is];
    };
    const double km = fmax(m.k1, fmax(m.k2, m.k3)), kmin = fmin(m.k1, fmin(m.k2, m.k3));
    m2l_table_body(sigf, km, kmin, m.k2, m.k2, P, sc, sc, tau, vs, cdc[ci] * w, fabs((double)cdr[ci]) * w, 0.0,
                   tab + (int64_t)cidx[ci] * (2 * P + 1) * (2 * P + 1), flag);
}

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
template <typename T>
static lm_status dalloc(lm_tree_s *t, T **p, size_t count)
{
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
    if (e != cudaSuccess) {
        lm_set_error("cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
        return LM_ENOMEM;
    }
    t->bytes += count * sizeof(T);
    return LM_OK;
}
#define TRY(x)                       \
    do {                             \
        lm_status s_ = (x);          \
        if (s_ != LM_OK) return s_;  \
    } while (0)

static int grid_for(int64_t n, int b) { return (int)((n + b - 1) / b); }

lm_status lm_setup_tree(lm_tree_s *t, const double *x, const double *y, cudaStream_t st)
{
    const int64_t n = t->n;
    const double d = t->med.d;
    TRY(dalloc(t, &t->dflag, 4));
    LM_CUDA(cudaMemsetAsync(t->dflag, 0, 4 * sizeof(int), st));
    int nb = (int)std::min<int64_t>(1024, (n + 255) / 256);
    double *bmin, *bmax;
    TRY(dalloc(t, &bmin, nb));
    TRY(dalloc(t, &bmax, nb));
    k_minmax<<<nb, 256, 0, st>>>(x, y, n, d, bmin, bmax, t->dflag);
    std::vector<double> hmin(nb), hmax(nb);
    int hflag = 0;
    LM_CUDA(cudaMemcpyAsync(hmin.data(), bmin, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaMemcpyAsync(hmax.data(), bmax, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaMemcpyAsync(&hflag, t->dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    cudaFree(bmin);
    cudaFree(bmax);
    t->bytes -= 2 * nb * sizeof(double);
    if (hflag & 1) {
        lm_set_error("build_tree: a point is non-finite or not strictly inside -d < y < 0");
        return LM_EINVAL;
    }
    double mn = hmin[0], mx = hmax[0];
    for (int i = 1; i < nb; ++i) {
        mn = fmin(mn, hmin[i]);
        mx = fmax(mx, hmax[i]);
    }
    double f0 = floor(mn / d), f1 = floor(mx / d);
    // the number of d x d roots, checked in double before it becomes an int: an
    // x extent of more than 2^30 thicknesses (or one that overflows) is rejected
    const double roots = f1 - f0 + 1.0;
    if (!std::isfinite(roots) || roots < 1.0 || roots > (double)(1 << 30)) {
        lm_set_error("build_tree: the x extent spans %g layer thicknesses; at most 2^30 roots are supported",
                     roots);
        return LM_EINVAL;
    }
    t->x0 = f0 * d;
    t->R = (int)roots;
    if (t->med.opt.depth >= 0) {
        t->L = t->med.opt.depth;
    } else {
        // least L with n <= leaf_target R 4^L, then deeper while the points share
        // a leaf with more than 1.5 leaf_target points on average over the points
        // (sum n_leaf^2 / n: what the direct interactions cost), as long as the
        // leaves stay fewer than twice the points (clustered inputs)
        int L = 0;
        while ((double)n > (double)t->med.opt.leaf_target * t->R * pow(4.0, L)) ++L;
        int32_t *key = nullptr, *cnt = nullptr;
        TRY(dalloc(t, &key, n));
        for (;; ++L) {
            const int64_t ncol = (int64_t)t->R << L, nrow = (int64_t)1 << L, nl = ncol * nrow;
            if (L >= 14 || nl > std::max<int64_t>(2 * n, t->R)) {
                --L;
                break;
            }
            TRY(dalloc(t, &cnt, nl));
            LM_CUDA(cudaMemsetAsync(cnt, 0, nl * sizeof(int32_t), st));
            k_keys<<<grid_for(n, 256), 256, 0, st>>>(x, y, n, t->x0, ldexp(d, -L), ncol, nrow, key, cnt);
            std::vector<int32_t> hc(nl);
            LM_CUDA(cudaMemcpyAsync(hc.data(), cnt, nl * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            LM_CUDA(cudaStreamSynchronize(st));
            cudaFree(cnt);
            t->bytes -= nl * sizeof(int32_t);
            double s2 = 0.0;
            for (int32_t c : hc) s2 += (double)c * c;
            if (s2 / n <= 1.5 * t->med.opt.leaf_target) break;
        }
        cudaFree(key);
        t->bytes -= n * sizeof(int32_t);
        t->L = std::max(L, 0);
    }
    const int L = t->L;
    const int64_t ncol = (int64_t)t->R << L, nrow = (int64_t)1 << L;
    t->nleaf = ncol * nrow;
    if (t->nleaf > (int64_t)1 << 30) {
        lm_set_error("build_tree: %lld leaves is beyond this build", (long long)t->nleaf);
        return LM_ENOTSUP;
    }
    int32_t *key, *cnt, *cursor;
    int64_t *tmp;
    TRY(dalloc(t, &key, n));
    TRY(dalloc(t, &cnt, t->nleaf));
    TRY(dalloc(t, &cursor, t->nleaf));
    TRY(dalloc(t, &t->leaf_start, t->nleaf + 1));
    TRY(dalloc(t, &t->perm, n));
    LM_CUDA(cudaMemsetAsync(cnt, 0, t->nleaf * sizeof(int32_t), st));
    LM_CUDA(cudaMemsetAsync(cursor, 0, t->nleaf * sizeof(int32_t), st));
    double w = ldexp(d, -L);
    k_keys<<<grid_for(n, 256), 256, 0, st>>>(x, y, n, t->x0, w, ncol, nrow, key, cnt);
    k_scan<<<1, 1024, 0, st>>>(cnt, t->nleaf, t->leaf_start);
    tmp = t->perm;
    k_scatter<<<grid_for(n, 256), 256, 0, st>>>(key, n, t->leaf_start, cursor, tmp);
    k_leafsort<<<(unsigned)t->nleaf, 256, 0, st>>>(t->leaf_start, t->perm, t->dflag);
    TRY(dalloc(t, &t->xs, n));
    TRY(dalloc(t, &t->ys, n));
    k_gather_pts<<<grid_for(n, 256), 256, 0, st>>>(x, y, t->perm, n, t->xs, t->ys);
    LM_CUDA(cudaGetLastError());
    LM_CUDA(cudaMemcpyAsync(&hflag, t->dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    cudaFree(key);
    cudaFree(cnt);
    cudaFree(cursor);
    t->bytes -= (n + 2 * t->nleaf) * sizeof(int32_t);
    if (hflag & 2) {
        lm_set_error("build_tree: a leaf holds more than %d points; use a deeper tree", LM_MAXLEAF);
        return LM_ENOTSUP;
    }
    return LM_OK;
}

// classes (term, dc, dr) reachable under the list rules at level l
static void enumerate_classes(int l, int R, std::vector<std::tuple<int, int, int>> &out)
{
    const int64_t nrow = (int64_t)1 << l, ncol = (int64_t)R << l;
    std::map<std::tuple<int, int, int>, int> seen;
    for (int term = 0; term < 5; ++term)
        for (int64_t rt = 0; rt < nrow; ++rt) {
            int64_t rlo = 0, rhi = nrow - 1;
            if (l > 0) {
                int64_t a = src_row(term, rt - 3, nrow), b = src_row(term, rt + 3, nrow);
                rlo = std::max((int64_t)0, std::min(a, b));
                rhi = std::min(nrow - 1, std::max(a, b));
            }
            for (int64_t rs = rlo; rs <= rhi; ++rs) {
                int64_t ri = img_row(term, rs, nrow);
                if (l == 0) {
                    for (int64_t cs = 0; cs < ncol; ++cs) {
                        int64_t ct = 0; // all dc are reached by some pair at level 0
                        for (ct = 0; ct < ncol; ++ct)
                            if (v_rule(0, ct, rt, cs, ri)) seen[{term, (int)(ct - cs), (int)(rt - ri)}] = 1;
                    }
                } else {
                    for (int64_t ct = 8; ct <= 9; ++ct)
                        for (int64_t cs = ct - 3; cs <= ct + 3; ++cs)
                            if (v_rule(l, ct, rt, cs, ri)) seen[{term, (int)(ct - cs), (int)(rt - ri)}] = 1;
                }
            }
        }
    for (auto &kv : seen) out.push_back(kv.first);
}

// Levels 0..L of the strip forest: scale vectors, the M2M / L2L tables and,
// with boxes set, the per-level expansion arrays of the uniform tree.
lm_status lm_setup_levels(lm_tree_s *t, int L, bool boxes, cudaStream_t st)
{
    const int P = t->p, np = 2 * P + 1;
    const double k = t->med.k2, d = t->med.d;
    t->lev.resize(L + 1);
    for (int l = 0; l <= L; ++l) {
        Level &lv = t->lev[l];
        lv.l = l;
        lv.ncol = (int64_t)t->R << l;
        lv.nrow = (int64_t)1 << l;
        lv.nbox = lv.ncol * lv.nrow;
        lv.w = ldexp(d, -l);
        std::vector<double> sc(P + 1);
        double f = 0.5 * k * lv.w, v = 1.0;
        for (int n = 0; n <= P; ++n) {
            sc[n] = v;
            v *= f / (n + 1);
        }
        TRY(dalloc(t, &lv.scale, P + 1));
        LM_CUDA(cudaMemcpyAsync(lv.scale, sc.data(), (P + 1) * sizeof(double), cudaMemcpyHostToDevice, st));
        if (boxes) {
            TRY(dalloc(t, &lv.M, lv.nbox * np * LM_MAXV));
            TRY(dalloc(t, &lv.Lc, lv.nbox * np * LM_MAXV));
        }
    }
    // shift tables
    for (int l = 0; l <= L; ++l) {
        Level &lv = t->lev[l];
        lv.m2m = nullptr;
        lv.l2l = nullptr;
        if (l < L) TRY(dalloc(t, &lv.m2m, 4 * np * np));
        if (l > 0) TRY(dalloc(t, &lv.l2l, 4 * np * np));
    }
    for (int l = 0; l < L; ++l) {
        // child level l+1 -> parent level l
        Level &par = t->lev[l], &ch = t->lev[l + 1];
        k_shift_tables<<<grid_for(4 * np * np, 128), 128, 0, st>>>(k, P, ch.w, ch.scale, par.scale,
                                                                   par.m2m, ch.l2l);
    }
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

// Near-field quadrature tables of the reflected direct terms (shared by both tree kinds)
lm_status lm_setup_near(lm_tree_s *t, cudaStream_t st)
{
    MediumD md{t->med.k1,
               t->med.k2,
               t->med.k3,
               t->med.d,
               t->med.opt.kernel == LM_KERNEL_DG_DD,
               {t->med.opt.top_bc, t->med.opt.bottom_bc},
               {t->med.opt.top_alpha, t->med.opt.bottom_alpha}};
    NearQuad &q = t->nq;
    q.rinf[0] = refl_inf(md, 0);
    q.rinf[1] = refl_inf(md, 1);
    const bool walls = !md.deriv && md.bc[0] != LM_BC_TRANSMISSION && md.bc[1] != LM_BC_TRANSMISSION;
    const bool imp = md.bc[0] == LM_BC_IMPEDANCE || md.bc[1] == LM_BC_IMPEDANCE;
    q.hray = (walls && !imp) ? 2.0 * md.d : 0.0; // single table (mixed form): shift only for constant R
    q.split = walls && t->precision == LM_FP64;   // FP64: single and multiple reflections apart
    q.a_zero = !imp;                              // Dirichlet / Neumann: R - R_inf = 0
    double km = fmax(md.k1, fmax(md.k2, md.k3)), kmin = fmin(md.k1, fmin(md.k2, md.k3));
    q.c = 1.5 * km + 1.0;
    double a = 0.5, delta = fmin(0.25, 0.5 * kmin);
    int nflat = (int)ceil((q.c - 2.0 * delta) / 1.0);
    int order = t->med.opt.seg_order;
    q.nseg = (nflat + 2) * order;
    q.nray = t->med.opt.tail_rays;
    q.ntail = t->med.opt.tail_order;
    TRY(dalloc(t, &q.seg_lam, q.nseg));
    TRY(dalloc(t, &q.seg_s2, q.nseg));
    TRY(dalloc(t, &q.seg_w, 2 * q.nseg));
    int nt = q.nray * q.ntail;
    TRY(dalloc(t, &q.tail_lam, nt));
    TRY(dalloc(t, &q.tail_s2, nt));
    TRY(dalloc(t, &q.tail_w, 4 * nt));
    const bool impc = t->precision == LM_FP64 && (imp_beta(md, 0) != 0.0 || imp_beta(md, 1) != 0.0);
    q.beta[0] = imp_beta(md, 0);
    q.beta[1] = imp_beta(md, 1);
    if (impc) TRY(dalloc(t, &q.seg_c, 2 * q.nseg));
    k_near_seg<<<grid_for(q.nseg, 64), 64, 0, st>>>(md, q.c, a, delta, nflat, order, q.seg_lam, q.seg_s2,
                                                     q.seg_w, q.nseg, impc ? q.seg_c : nullptr);
    if (q.split) TRY(dalloc(t, &q.tail_w2, 4 * nt));
    k_near_tail<<<grid_for(nt, 64), 64, 0, st>>>(md, q.c, q.nray, q.ntail, q.tail_lam, q.tail_s2, q.tail_w,
                                                  q.split ? q.tail_w2 : nullptr);
    if (t->precision == LM_FP64) {
        q.ntail_g = std::max(64, q.ntail);
        const int ng = q.nray * q.ntail_g;
        TRY(dalloc(t, &q.tail_lam_g, ng));
        TRY(dalloc(t, &q.tail_s2_g, ng));
        TRY(dalloc(t, &q.tail_w_g, 4 * ng));
        if (q.split) TRY(dalloc(t, &q.tail_w2_g, 4 * ng));
        if (impc) TRY(dalloc(t, &q.tail_c_g, 4 * ng));
        k_near_tail<<<grid_for(ng, 64), 64, 0, st>>>(md, q.c, q.nray, q.ntail_g, q.tail_lam_g, q.tail_s2_g,
                                                      q.tail_w_g, q.split ? q.tail_w2_g : nullptr,
                                                      impc ? q.tail_c_g : nullptr);
    }
    LM_CUDA(cudaGetLastError());
    // FP64: factorise the segment per leaf when its coefficients fit in shared memory
    const size_t pw = lm_near_pw64_smem(q.nseg);
    t->near_pw64 = false;
    if (t->precision == LM_FP64 && pw <= 200 * 1024) {
        TRY(lm_near_pw64_attr(pw));
        t->near_pw64 = true;
        TRY(lm_setup_pwsrc(t, st));
    }
    return LM_OK;
}

lm_status lm_setup_tables(lm_tree_s *t, cudaStream_t st)
{
    const int L = t->L, P = t->p, np = 2 * P + 1;
    const double k = t->med.k2;
    MediumD md{t->med.k1,
               t->med.k2,
               t->med.k3,
               t->med.d,
               t->med.opt.kernel == LM_KERNEL_DG_DD,
               {t->med.opt.top_bc, t->med.opt.bottom_bc},
               {t->med.opt.top_alpha, t->med.opt.bottom_alpha}};
    TRY(lm_setup_levels(t, L, true, st));
    // lists and M2L classes
    for (int l = 0; l <= L; ++l) {
        Level &lv = t->lev[l];
        std::vector<std::tuple<int, int, int>> cls;
        enumerate_classes(l, t->R, cls);
        int DC = l == 0 ? (int)std::max<int64_t>(3, lv.ncol - 1) : 3;
        std::vector<int32_t> smap((size_t)5 * (2 * DC + 1) * 7, -1);
        for (size_t i = 0; i < cls.size(); ++i) {
            int term = std::get<0>(cls[i]), dc = std::get<1>(cls[i]), dr = std::get<2>(cls[i]);
            lv.cls_term.push_back(term);
            lv.cls_dc.push_back(dc);
            lv.cls_dr.push_back(dr);
            smap[slot_index(DC, term, dc, dr)] = (int32_t)i;
        }
        int32_t *dmap;
        TRY(dalloc(t, &dmap, smap.size()));
        LM_CUDA(cudaMemcpyAsync(dmap, smap.data(), smap.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        TRY(dalloc(t, &lv.vstart, lv.nbox + 1));
        k_vlist<<<grid_for(lv.nbox, 128), 128, 0, st>>>(l, lv.ncol, lv.nrow, DC, dmap, lv.vstart,
                                                        nullptr, nullptr, nullptr, 0, t->dflag);
        k_scan64<<<1, 1024, 0, st>>>(lv.vstart, lv.nbox);
        LM_CUDA(cudaMemcpyAsync(&lv.nv, lv.vstart + lv.nbox, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        LM_CUDA(cudaStreamSynchronize(st));
        TRY(dalloc(t, &lv.vsrc, lv.nv));
        TRY(dalloc(t, &lv.vslot, lv.nv));
        TRY(dalloc(t, &lv.vterm, lv.nv));
        k_vlist<<<grid_for(lv.nbox, 128), 128, 0, st>>>(l, lv.ncol, lv.nrow, DC, dmap, lv.vstart,
                                                        lv.vsrc, lv.vslot, lv.vterm, 1, t->dflag);
        // tables
        int ncls = (int)cls.size();
        TRY(dalloc(t, &lv.tab, (size_t)std::max(1, ncls) * np * np));
        std::vector<int> fdc, fdr, fidx, idc, idr, iterm, iidx;
        for (int i = 0; i < ncls; ++i) {
            if (lv.cls_term[i] == 0) {
                fdc.push_back(lv.cls_dc[i]);
                fdr.push_back(lv.cls_dr[i]);
                fidx.push_back(i);
            } else {
                iterm.push_back(lv.cls_term[i]);
                idc.push_back(lv.cls_dc[i]);
                idr.push_back(lv.cls_dr[i]);
                iidx.push_back(i);
            }
        }
        int *dbuf;
        int nf = (int)fdc.size(), ni = (int)idc.size();
        TRY(dalloc(t, &dbuf, 3 * nf + 4 * ni + 1));
        std::vector<int> hb;
        hb.insert(hb.end(), fdc.begin(), fdc.end());
        hb.insert(hb.end(), fdr.begin(), fdr.end());
        hb.insert(hb.end(), fidx.begin(), fidx.end());
        hb.insert(hb.end(), iterm.begin(), iterm.end());
        hb.insert(hb.end(), idc.begin(), idc.end());
        hb.insert(hb.end(), idr.begin(), idr.end());
        hb.insert(hb.end(), iidx.begin(), iidx.end());
        if (!hb.empty())
            LM_CUDA(cudaMemcpyAsync(dbuf, hb.data(), hb.size() * sizeof(int), cudaMemcpyHostToDevice, st));
        if (md.deriv) // the free part does not depend on d: its tables stay zero
            LM_CUDA(cudaMemsetAsync(lv.tab, 0, (size_t)std::max(1, ncls) * np * np * sizeof(zd), st));
        if (nf > 0 && !md.deriv) {
            dim3 g(grid_for(np * np, 256), nf);
            k_free_m2l<<<g, 256, 0, st>>>(k, P, lv.w, dbuf, dbuf + nf, dbuf + 2 * nf, nf, lv.scale, lv.tab);
        }
        if (ni > 0) {
            size_t shm = (2 * TB_CHUNK * np + TB_CHUNK) * sizeof(zd);
            LM_CUDA(lm_raise_smem((const void *)k_image_m2l, LM_SMEM_IMAGE_M2L, (int)shm));
            k_image_m2l<<<ni, 256, shm, st>>>(md, P, lv.w, k * lv.w, dbuf + 3 * nf, dbuf + 3 * nf + ni,
                                              dbuf + 3 * nf + 2 * ni, dbuf + 3 * nf + 3 * ni, ni, lv.tab,
                                              t->dflag);
        }
        LM_CUDA(cudaGetLastError());
        LM_CUDA(cudaStreamSynchronize(st));
        cudaFree(dbuf);
        cudaFree(dmap);
        t->bytes -= (3 * nf + 4 * ni + 1) * sizeof(int) + smap.size() * sizeof(int32_t);
    }
    // U list
    {
        const int64_t ncol = (int64_t)t->R << L, nrow = (int64_t)1 << L;
        TRY(dalloc(t, &t->ustart, t->nleaf + 1));
        k_ulist<<<grid_for(t->nleaf, 128), 128, 0, st>>>(ncol, nrow, t->ustart, nullptr, nullptr, 0);
        k_scan64<<<1, 1024, 0, st>>>(t->ustart, t->nleaf);
        LM_CUDA(cudaMemcpyAsync(&t->nu, t->ustart + t->nleaf, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        LM_CUDA(cudaStreamSynchronize(st));
        TRY(dalloc(t, &t->usrc, t->nu));
        TRY(dalloc(t, &t->uterm, t->nu));
        k_ulist<<<grid_for(t->nleaf, 128), 128, 0, st>>>(ncol, nrow, t->ustart, t->usrc, t->uterm, 1);
    }
    TRY(lm_setup_near(t, st));
    // tree-order scratch for densities and potentials
    TRY(dalloc(t, &t->qs, (size_t)LM_MAXV * t->n));
    TRY(dalloc(t, &t->us, (size_t)LM_MAXV * t->n));
    int hflag = 0;
    LM_CUDA(cudaGetLastError());
    LM_CUDA(cudaMemcpyAsync(&hflag, t->dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    if (hflag & 4) {
        lm_set_error("build_tree: internal error, an interaction has no translation class");
        return LM_ECUDA;
    }
    if (hflag & 8) {
        lm_set_error("build_tree: expansion order too large for the table builder");
        return LM_ENOTSUP;
    }
    if (hflag & 16) {
        lm_set_error("build_tree: a layered M2L table overflowed; lower p");
        return LM_ENOTSUP;
    }
    if (t->precision == LM_MIXED) return lm_setup_mixed(t, st);
    return lm_setup_df(t, st);
}

lm_status lm_list_to_host(lm_tree_s *t, int which, int level, std::vector<int64_t> &rows,
                          cudaStream_t st)
{
    int64_t nb, ne;
    const int64_t *start;
    const int32_t *src, *term;
    if (which == 0) {
        if (level < 0 || level > t->L) {
            lm_set_error("list_export: level %d out of range", level);
            return LM_EINVAL;
        }
        Level &lv = t->lev[level];
        nb = lv.nbox;
        ne = lv.nv;
        start = lv.vstart;
        src = lv.vsrc;
        term = lv.vterm;
    } else {
        nb = t->nleaf;
        ne = t->nu;
        start = t->ustart;
        src = t->usrc;
        term = t->uterm;
    }
    std::vector<int64_t> hs(nb + 1);
    std::vector<int32_t> hsrc(ne), hterm(ne);
    LM_CUDA(cudaMemcpyAsync(hs.data(), start, (nb + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    if (ne > 0) {
        LM_CUDA(cudaMemcpyAsync(hsrc.data(), src, ne * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        LM_CUDA(cudaMemcpyAsync(hterm.data(), term, ne * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    }
    LM_CUDA(cudaStreamSynchronize(st));
    rows.resize(3 * ne);
    for (int64_t b = 0; b < nb; ++b)
        for (int64_t e = hs[b]; e < hs[b + 1]; ++e) {
            rows[3 * e] = b;
            rows[3 * e + 1] = hterm[e];
            rows[3 * e + 2] = hsrc[e];
        }
    return LM_OK;
}

void lm_free_tree_device(lm_tree_s *t)
{
    lm_free_mixed(t);
    lm_free_adaptive(t);
    void *ptrs[] = {t->xs, t->ys, t->perm, t->leaf_start, t->ustart, t->usrc, t->uterm, t->qs, t->us,
                    t->dflag, t->qexp, t->pwidx, t->pwC, t->nq.seg_lam, t->nq.seg_s2, t->nq.seg_w, t->nq.tail_lam, t->nq.tail_s2,
                    t->nq.tail_w, t->nq.tail_lam_g, t->nq.tail_s2_g, t->nq.tail_w_g, t->nq.tail_w2,
                    t->nq.tail_w2_g, t->nq.seg_c, t->nq.tail_c_g};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (Level &lv : t->lev) {
        void *lp[] = {lv.vstart, lv.vsrc, lv.vslot, lv.vterm, lv.tab, lv.scale, lv.m2m, lv.l2l, lv.M, lv.Lc,
                      lv.tabdf, lv.tabdft, lv.Mdf, lv.m2mdf, lv.l2ldf};
        for (void *p : lp)
            if (p) cudaFree(p);
    }
    cudaGetLastError(); // teardown leaves no error behind for the caller's next call
}
