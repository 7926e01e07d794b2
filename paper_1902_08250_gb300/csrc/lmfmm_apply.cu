// lmfmm_apply.cu -- Algorithm 1, steps 2-4 (upward pass, downward pass,
// evaluation) as device kernels, FP64 form.
#include <algorithm>

#include "internal.h"

static int gridn(int64_t n, int b) { return (int)((n + b - 1) / b); }

// Box geometry of a launch: block i works on box id(i), whose centre and width
// come from centre().
struct GridLeaves { // uniform tree: leaf i of the leaf lattice
    LeafGeom g;
    __device__ int64_t id(int64_t i) const { return i; }
    __device__ void centre(int64_t b, double *cx, double *cy, double *w) const
    {
        leaf_centre(g, b, cx, cy);
        *w = g.w;
    }
};
struct EdgeRowLeaves { // uniform tree: the leaves of the top row, then (nrow > 1) of the bottom row
    LeafGeom g;
    int64_t nrow;
    __device__ int64_t id(int64_t i) const { return ((nrow == 1 || i < g.ncol) ? 0 : nrow - 1) * g.ncol + i % g.ncol; }
    __device__ void centre(int64_t b, double *cx, double *cy, double *w) const
    {
        leaf_centre(g, b, cx, cy);
        *w = g.w;
    }
};
struct ListBoxes { // adaptive tree: box ids[i], centres and widths from arrays
    const int32_t *ids;
    const double *bx, *by, *bw;
    __device__ int64_t id(int64_t i) const { return ids[i]; }
    __device__ void centre(int64_t b, double *cx, double *cy, double *w) const
    {
        *cx = bx[b];
        *cy = by[b];
        *w = bw[b];
    }
};

// q (input order, [nvec][n]) -> qs (tree order, [nvec][n]), optionally conjugated
__global__ void k_permute_in(const zd *q, const int64_t *perm, int64_t n, int nvec, int conjugate,
                             zd *qs)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    for (int v = 0; v < nvec; ++v) {
        zd a = q[(int64_t)v * n + j];
        qs[(int64_t)v * n + i] = conjugate ? conj(a) : a;
    }
}
__global__ void k_permute_out(const zd *us, const int64_t *perm, int64_t n, int nvec, int conjugate,
                              zd *u)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t j = perm[i];
    for (int v = 0; v < nvec; ++v) {
        zd a = us[(int64_t)v * n + i];
        u[(int64_t)v * n + j] = conjugate ? conj(a) : a;
    }
}


// ---------------------------------------------------------------------------
// S2M (Eq. (multipole_coef)), scaled: Mhat_q = sum_j q_j Jhat_q(k r_j) e^{-i q theta_j}
// One block per leaf; points staged 16 at a time.
// ---------------------------------------------------------------------------
#define P2M_CHUNK 16
template <class Geo>
__device__ __forceinline__ void p2m64_body(Geo geo, int P, double k, const double *xs, const double *ys,
                                           const int64_t *ls, const zd *qs, int64_t n, int nvec, zd *M)
{
    extern __shared__ unsigned char smem[];
    const int np = 2 * P + 1;
    zd *B = (zd *)smem;                      // [P2M_CHUNK][np]
    zd *Q = B + P2M_CHUNK * np;              // [P2M_CHUNK][LM_MAXV]
    const int64_t b = geo.id(blockIdx.x);
    const int64_t lo = ls[b], hi = ls[b + 1];
    double cx, cy, bw;
    geo.centre(b, &cx, &cy, &bw);
    const double sc = k * bw;
    const int nent = np * nvec;
    zd acc[12];
    for (int e = 0; e < 12; ++e) acc[e] = zd{0.0, 0.0};
    for (int64_t base = lo; base < hi; base += P2M_CHUNK) {
        __syncthreads();
        int j = threadIdx.x;
        if (j < P2M_CHUNK) {
            int64_t i = base + j;
            zd *row = B + j * np + P;
            if (i < hi) {
                double rx = xs[i] - cx, ry = ys[i] - cy, r = hypot(rx, ry);
                double J[LM_MAXP + 1];
                bessel_j_scaled<double>(P, k * r, sc, J);
                zd z = r > 0.0 ? zd{rx / r, -ry / r} : zd{1.0, 0.0}; // e^{-i theta}
                zd zp = {1.0, 0.0};
                row[0] = zd{J[0], 0.0};
                for (int m = 1; m <= P; ++m) {
                    zp = zp * z;
                    row[m] = J[m] * zp;
                    double s = (m & 1) ? -J[m] : J[m];
                    row[-m] = s * conj(zp);
                }
                for (int v = 0; v < nvec; ++v) Q[j * LM_MAXV + v] = qs[(int64_t)v * n + i];
            } else {
                for (int m = -P; m <= P; ++m) row[m] = zd{0.0, 0.0};
                for (int v = 0; v < nvec; ++v) Q[j * LM_MAXV + v] = zd{0.0, 0.0};
            }
        }
        __syncthreads();
        for (int e = 0; e < 12; ++e) {
            int idx = threadIdx.x + e * blockDim.x;
            if (idx >= nent) break;
            int qi = idx / nvec, v = idx % nvec;
            zd s = acc[e];
            for (int jj = 0; jj < P2M_CHUNK; ++jj) cfma(s, B[jj * np + qi], Q[jj * LM_MAXV + v]);
            acc[e] = s;
        }
    }
    for (int e = 0; e < 12; ++e) {
        int idx = threadIdx.x + e * blockDim.x;
        if (idx >= nent) break;
        int qi = idx / nvec, v = idx % nvec;
        M[(b * np + qi) * LM_MAXV + v] = acc[e];
    }
}
__global__ void k_p2m64(LeafGeom g, int P, double k, const double *xs, const double *ys,
                        const int64_t *ls, const zd *qs, int64_t n, int nvec, zd *M)
{
    p2m64_body(GridLeaves{g}, P, k, xs, ys, ls, qs, n, nvec, M);
}
__global__ void k_p2m64_list(ListBoxes geo, int P, double k, const double *xs, const double *ys,
                             const int64_t *ls, const zd *qs, int64_t n, int nvec, zd *M)
{
    p2m64_body(geo, P, k, xs, ys, ls, qs, n, nvec, M);
}

// M2M over the parents of one level of the adaptive tree: parent par[i] from its four children
__global__ void k_m2m64a(int64_t npar, const int32_t *par, const int32_t *child, int P, int nvec,
                         const zd *tabs, zd *M)
{
    const int np = 2 * P + 1;
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= npar * np * nvec) return;
    int v = idx % nvec;
    int p = (idx / nvec) % np;
    const int64_t b = par[idx / (nvec * np)];
    zd acc = {0.0, 0.0};
    for (int pos = 0; pos < 4; ++pos) {
        const int64_t ch = child[4 * b + pos];
        const zd *T = tabs + ((int64_t)pos * np + p) * np;
        const zd *m = M + ch * np * LM_MAXV + v;
        for (int q = 0; q < np; ++q) cfma(acc, T[q], m[q * LM_MAXV]);
    }
    M[(b * np + p) * LM_MAXV + v] = acc;
}

// L2L over the boxes b0 .. b0 + nb - 1 of one level (>= 1) of the adaptive tree; initialises L
__global__ void k_l2l64a(int64_t b0, int64_t nb, const int32_t *parent, const int32_t *bpos, int P, int nvec,
                         const zd *tabs, zd *Lc)
{
    const int np = 2 * P + 1;
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nb * np * nvec) return;
    int v = idx % nvec;
    int p = (idx / nvec) % np;
    const int64_t b = b0 + idx / (nvec * np);
    const zd *T = tabs + ((int64_t)bpos[b] * np + p) * np;
    const zd *m = Lc + (int64_t)parent[b] * np * LM_MAXV + v;
    zd acc = {0.0, 0.0};
    for (int q = 0; q < np; ++q) cfma(acc, T[q], m[q * LM_MAXV]);
    Lc[(b * np + p) * LM_MAXV + v] = acc;
}

// M2M (Lemma M2M): parent (level l) from its four children (level l+1)
__global__ void k_m2m64(int64_t ncol, int64_t nbox, int P, int nvec, const zd *tabs, const zd *Mc,
                        zd *Mp)
{
    const int np = 2 * P + 1;
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nbox * np * nvec) return;
    int v = idx % nvec;
    int p = (idx / nvec) % np;
    int64_t b = idx / (nvec * np);
    int64_t r = b / ncol, c = b % ncol, ncc = 2 * ncol;
    zd acc = {0.0, 0.0};
    for (int pos = 0; pos < 4; ++pos) {
        int dy = pos >> 1, dx = pos & 1;
        int64_t ch = (2 * r + dy) * ncc + 2 * c + dx;
        const zd *T = tabs + ((int64_t)pos * np + p) * np;
        const zd *m = Mc + ch * np * LM_MAXV + v;
        for (int q = 0; q < np; ++q) cfma(acc, T[q], m[q * LM_MAXV]);
    }
    Mp[(b * np + p) * LM_MAXV + v] = acc;
}

// L2L (Lemma L2L): child (level l) from its parent (level l-1); initialises L
__global__ void k_l2l64(int64_t ncol, int64_t nbox, int P, int nvec, const zd *tabs, const zd *Lp,
                        zd *Lc)
{
    const int np = 2 * P + 1;
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nbox * np * nvec) return;
    int v = idx % nvec;
    int p = (idx / nvec) % np;
    int64_t b = idx / (nvec * np);
    int64_t r = b / ncol, c = b % ncol;
    int pos = (int)((r & 1) * 2 + (c & 1));
    int64_t par = (r / 2) * (ncol / 2) + c / 2;
    const zd *T = tabs + ((int64_t)pos * np + p) * np;
    const zd *m = Lp + par * np * LM_MAXV + v;
    zd acc = {0.0, 0.0};
    for (int q = 0; q < np; ++q) cfma(acc, T[q], m[q * LM_MAXV]);
    Lc[(b * np + p) * LM_MAXV + v] = acc;
}

// M2L over the V list (free space and image terms)
__global__ void k_m2l64(int64_t nbox, int P, int nvec, const int64_t *vstart, const int32_t *vsrc,
                        const int32_t *vslot, const zd *tab, const zd *M, zd *Lc)
{
    const int np = 2 * P + 1;
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nbox * np * nvec) return;
    int v = idx % nvec;
    int p = (idx / nvec) % np;
    int64_t b = idx / (nvec * np);
    zd acc = {0.0, 0.0};
    for (int64_t e = vstart[b]; e < vstart[b + 1]; ++e) {
        const zd *T = tab + ((int64_t)vslot[e] * np + p) * np;
        const zd *m = M + (int64_t)vsrc[e] * np * LM_MAXV + v;
        for (int q = 0; q < np; ++q) cfma(acc, T[q], m[q * LM_MAXV]);
    }
    Lc[(b * np + p) * LM_MAXV + v] += acc;
}

// ---------------------------------------------------------------------------
// M2L in double-float on the FP32 pipes (Dekker's representation: a value is
// hi + lo, two FP32 numbers with |lo| <= ulp(hi)/2, 48 significand bits).  A
// product is exact as p + e with p = hi*hi rounded and e = fma(hi, hi, -p),
// plus the two cross terms; a sum is made exact by Knuth's TwoSum, whose
// error joins the running low word.  The FP64 form keeps every other step in
// IEEE FP64; GB300 issues FP32 at about 60 times its FP64 rate, so the
// 48 FP32 instructions of a complex multiply-add cost less than its 4 DFMAs.
// Multipoles are scaled by 2^-qexp (qexp: the binary exponent of the largest
// density component of the apply), so that they stay inside FP32's exponent
// range; tables are scaled (S_l) and of order one already.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float4 df_split(zd a)
{
    const float rh = __double2float_rn(a.re), ih = __double2float_rn(a.im);
    return make_float4(rh, __double2float_rn(a.re - (double)rh), ih, __double2float_rn(a.im - (double)ih));
}
// (sh, sl) += (ah + al)(bh + bl)
__device__ __forceinline__ void df_mac(float &sh, float &sl, float ah, float al, float bh, float bl)
{
    const float p = __fmul_rn(ah, bh);
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    const float s = __fadd_rn(sh, p);
    const float bb = __fsub_rn(s, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(err, e));
}
// complex: acc += t m, each part a double-float (x, y) = real, (z, w) = imaginary
__device__ __forceinline__ void dfc_mac(float4 &acc, const float4 t, const float4 m)
{
    df_mac(acc.x, acc.y, t.x, t.y, m.x, m.y);
    df_mac(acc.x, acc.y, -t.z, -t.w, m.z, m.w);
    df_mac(acc.z, acc.w, t.x, t.y, m.z, m.w);
    df_mac(acc.z, acc.w, t.z, t.w, m.x, m.y);
}

__global__ void k_tab_df(const zd *tab, int64_t count, float4 *out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < count) out[i] = df_split(tab[i]);
}
// the same, each np x np table transposed ([q][p])
__global__ void k_tab_df_t(const zd *tab, int64_t count, int np, float4 *out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    const int64_t slot = i / ((int64_t)np * np);
    const int r = (int)(i % ((int64_t)np * np)), p = r / np, q = r % np;
    out[slot * np * np + (int64_t)q * np + p] = df_split(tab[i]);
}

// largest |re|, |im| of the densities [nvec][n] -> its binary exponent, max-reduced into *qexp
__global__ void k_qexp(const zd *qs, int64_t n, int nvec, int *qexp)
{
    double mx = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n * nvec; i += (int64_t)gridDim.x * blockDim.x) {
        const zd a = qs[i];
        mx = fmax(mx, fmax(fabs(a.re), fabs(a.im)));
    }
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if ((threadIdx.x & 31) == 0 && mx > 0.0) {
        int e;
        frexp(mx, &e);
        atomicMax(qexp, e);
    }
}
__device__ __forceinline__ int qexp_of(const int *qexp)
{
    const int e = *qexp;
    return e < -1000 ? 0 : e; // all densities zero: no scaling
}

// multipoles of boxes b0 .. b0 + nb - 1 -> double-float, scaled by 2^-qexp
__global__ void k_m_df(int64_t b0, int64_t nb, int P, int nvec, const zd *M, const int *qexp, float4 *Mdf)
{
    const int np = 2 * P + 1;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nb * np * nvec) return;
    const int v = idx % nvec;
    const int64_t r = (b0 * np + idx / nvec) * LM_MAXV + v; // row (box, q), vector v
    const int e = -qexp_of(qexp);
    const zd a = M[r];
    Mdf[r] = df_split(zd{ldexp(a.re, e), ldexp(a.im, e)});
}

// M2L over the V list, double-float: one thread per (target box, order p, vector).
// TR: tables transposed ([q][p]).  With few vectors a warp spans 32 orders p of one
// box, and the transposed rows make its table reads contiguous; with many vectors
// a warp spans 2 orders, each thread reads its own row, and the row-major layout
// keeps a thread's reads on few cache lines.
template <bool TR>
__global__ void __launch_bounds__(128) k_m2l_df(int64_t nbox, int P, int nvec, const int64_t *vstart,
                                                const int32_t *vsrc, const int32_t *vslot, const float4 *tab,
                                                const float4 *Mdf, const int *qexp, zd *Lc)
{
    const int np = 2 * P + 1;
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= nbox * np * nvec) return;
    const int v = idx % nvec;
    const int p = (idx / nvec) % np;
    const int64_t b = idx / (nvec * np);
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t e = vstart[b]; e < vstart[b + 1]; ++e) {
        const float4 *T = tab + (int64_t)vslot[e] * np * np + (TR ? p : (int64_t)p * np);
        const int ts = TR ? np : 1;
        const float4 *m = Mdf + (int64_t)vsrc[e] * np * LM_MAXV + v;
        for (int q = 0; q < np; ++q) dfc_mac(acc, T[q * ts], m[q * LM_MAXV]);
    }
    const int ex = qexp_of(qexp);
    zd &o = Lc[(b * np + p) * LM_MAXV + v];
    o = o + zd{ldexp((double)acc.x + (double)acc.y, ex), ldexp((double)acc.z + (double)acc.w, ex)};
}

// M2M and L2L in double-float: one block per parent box.  The parent's children
// (M2M: their multipoles, one child position at a time) or the parent's local
// expansion (L2L) are converted once into shared memory, scaled by 2^-qexp;
// each thread accumulates up to DF_MAXO outputs (order, vector).
#define DF_THREADS 128
#define DF_TR_NV 2 // applies of up to this many vectors read the transposed M2L tables
#define DF_MAXO 13 // (2 * LM_MAXP + 1) * LM_MAXV / DF_THREADS, rounded up
// threads of a double-float M2M / L2L block: 64 while its outputs (M2M: one box, L2L: four children)
// fit, else DF_THREADS
static int df_threads(int nout) { return nout <= 64 ? 64 : DF_THREADS; }
// threads of an S2M block: the (order, vector) entries rounded up to warps, 64 to 256
static int p2m_threads(int nent) { return std::max(64, std::min(256, (nent + 31) / 32 * 32)); }
struct GridParents { // uniform tree: parent i of a level with ncol columns; children one level down
    int64_t ncol;
    __device__ int64_t parent(int64_t i) const { return i; }
    __device__ int64_t child(int64_t b, int pos) const
    {
        const int64_t r = b / ncol, c = b % ncol;
        return (2 * r + (pos >> 1)) * (2 * ncol) + 2 * c + (pos & 1);
    }
};
struct ListParents { // adaptive tree: parent ids[i], children from the box links
    const int32_t *ids, *kids;
    __device__ int64_t parent(int64_t i) const { return ids[i]; }
    __device__ int64_t child(int64_t b, int pos) const { return kids[4 * b + pos]; }
};

template <class Geo>
__global__ void __launch_bounds__(DF_THREADS) k_m2m_df(Geo geo, int P, int nvec, const float4 *tabs, const zd *Mc,
                                                       const int *qexp, zd *Mp)
{
    extern __shared__ float4 sm4[]; // [np][nvec]: one child's multipole
    const int np = 2 * P + 1, nout = np * nvec;
    const int64_t b = geo.parent(blockIdx.x);
    const int e = qexp_of(qexp);
    float4 acc[DF_MAXO];
#pragma unroll
    for (int k = 0; k < DF_MAXO; ++k) acc[k] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int pos = 0; pos < 4; ++pos) {
        const int64_t ch = geo.child(b, pos);
        __syncthreads();
        for (int i = threadIdx.x; i < nout; i += blockDim.x) {
            const zd a = Mc[(ch * np + i / nvec) * LM_MAXV + i % nvec];
            sm4[i] = df_split(zd{ldexp(a.re, -e), ldexp(a.im, -e)});
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < DF_MAXO; ++k) {
            const int o = threadIdx.x + k * blockDim.x;
            if (o < nout) {
                const int p = o / nvec, v = o % nvec;
                const float4 *T = tabs + ((int64_t)pos * np + p) * np;
                for (int q = 0; q < np; ++q) dfc_mac(acc[k], T[q], sm4[q * nvec + v]);
            }
        }
    }
#pragma unroll
    for (int k = 0; k < DF_MAXO; ++k) {
        const int o = threadIdx.x + k * blockDim.x;
        if (o < nout)
            Mp[(b * np + o / nvec) * LM_MAXV + o % nvec] =
                zd{ldexp((double)acc[k].x + (double)acc[k].y, e), ldexp((double)acc[k].z + (double)acc[k].w, e)};
    }
}

template <class Geo>
__global__ void __launch_bounds__(DF_THREADS) k_l2l_df(Geo geo, int P, int nvec, const float4 *tabs, const zd *Lp,
                                                       const int *qexp, zd *Lc)
{
    extern __shared__ float4 sm4[]; // [np][nvec]: the parent's local expansion
    const int np = 2 * P + 1, nout = np * nvec;
    const int64_t b = geo.parent(blockIdx.x);
    const int e = qexp_of(qexp);
    for (int i = threadIdx.x; i < nout; i += blockDim.x) {
        const zd a = Lp[(b * np + i / nvec) * LM_MAXV + i % nvec];
        sm4[i] = df_split(zd{ldexp(a.re, -e), ldexp(a.im, -e)});
    }
    __syncthreads();
    for (int o = threadIdx.x; o < 4 * nout; o += blockDim.x) {
        const int pos = o / nout, r = o % nout, p = r / nvec, v = r % nvec;
        const float4 *T = tabs + ((int64_t)pos * np + p) * np;
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int q = 0; q < np; ++q) dfc_mac(acc, T[q], sm4[q * nvec + v]);
        Lc[(geo.child(b, pos) * np + p) * LM_MAXV + v] =
            zd{ldexp((double)acc.x + (double)acc.y, e), ldexp((double)acc.z + (double)acc.w, e)};
    }
}

// ---------------------------------------------------------------------------
// Free-space kernel (i/4) H0^(1)(x) = (i/4)(J0(x) + i Y0(x)) of a near pair in
// FP64.  For x <= 2 the ascending series (Abramowitz & Stegun 9.1.12, 9.1.13),
// with z = x^2/4:
//   J0 = sum_m (-z)^m / (m!)^2,
//   Y0 = (2/pi) [(ln(x/2) + gamma) J0 - sum_{m>=1} H_m (-z)^m / (m!)^2],
// H_m the harmonic numbers, gamma Euler's constant; 14 terms leave the first
// omitted one below 2e-21 for z <= 1 (within 5e-16 of scipy's J0, Y0 on
// (0, 2]).  Horner form: 28 FMAs and one log in place of the library's j0 and
// y0 (1M FP64 strip: leaf kernel 72.0 -> 65.7 ms).  Larger x: j0, y0.
// ---------------------------------------------------------------------------
#define H0S_TERMS 14
struct H0Series {
    double cj[H0S_TERMS], cy[H0S_TERMS]; // (-1)^m / (m!)^2, -(-1)^m H_m / (m!)^2
    constexpr H0Series() : cj(), cy()
    {
        double f = 1.0, h = 0.0; // 1/(m!)^2, H_m
        for (int m = 0; m < H0S_TERMS; ++m) {
            if (m > 0) {
                f /= (double)m * (double)m;
                h += 1.0 / m;
            }
            cj[m] = (m & 1) ? -f : f;
            cy[m] = (m & 1) ? h * f : -h * f;
        }
    }
};
__constant__ H0Series c_h0s = H0Series();
// J1 and Y1 for the target gradient (A&S 9.1.10, 9.1.11 with n = 1):
//   J1 = (x/2) sum_m (-z)^m / (m! (m+1)!),
//   Y1 = -2/(pi x) + (2/pi) ln(x/2) J1 - (x/(2 pi)) sum_m (-z)^m (psi(m+1) + psi(m+2)) / (m! (m+1)!),
// psi(m+1) = H_m - gamma; within 5e-16 of scipy's J1, Y1 on (0, 2]
struct H1Series {
    double c[H0S_TERMS], e[H0S_TERMS]; // (-1)^m / (m! (m+1)!), (-1)^m (psi(m+1) + psi(m+2)) / (m! (m+1)!)
    constexpr H1Series() : c(), e()
    {
        double f = 1.0, h = 0.0; // 1/(m! (m+1)!), H_m
        for (int m = 0; m < H0S_TERMS; ++m) {
            if (m > 0) {
                f /= (double)m * (double)(m + 1);
                h += 1.0 / m;
            }
            const double psi = (h - 0.57721566490153286061) + (h + 1.0 / (m + 1) - 0.57721566490153286061);
            c[m] = (m & 1) ? -f : f;
            e[m] = (m & 1) ? -psi * f : psi * f;
        }
    }
};
__constant__ H1Series c_h1s = H1Series();
// (i/4) H0^(1)(x) and (i/4) H1^(1)(x) together (series for x <= 2, else the library's)
__device__ __forceinline__ void h01_free64(double x, zd *h0, zd *h1)
{
    if (x > 2.0) {
        *h0 = zd{-0.25 * y0(x), 0.25 * j0(x)};
        *h1 = zd{-0.25 * y1(x), 0.25 * j1(x)};
        return;
    }
    const double z = 0.25 * x * x;
    double j = c_h0s.cj[H0S_TERMS - 1], sy = c_h0s.cy[H0S_TERMS - 1];
    double a = c_h1s.c[H0S_TERMS - 1], b = c_h1s.e[H0S_TERMS - 1];
#pragma unroll
    for (int m = H0S_TERMS - 2; m >= 0; --m) {
        j = fma(j, z, c_h0s.cj[m]);
        sy = fma(sy, z, c_h0s.cy[m]);
        a = fma(a, z, c_h1s.c[m]);
        b = fma(b, z, c_h1s.e[m]);
    }
    const double tpi = 0.63661977236758134308, lg = log(0.5 * x);
    const double yv0 = tpi * ((lg + 0.57721566490153286061) * j + sy);
    const double jv1 = 0.5 * x * a;
    const double yv1 = -tpi / x + tpi * lg * jv1 - 0.5 * tpi * 0.5 * x * b;
    *h0 = zd{-0.25 * yv0, 0.25 * j};
    *h1 = zd{-0.25 * yv1, 0.25 * jv1};
}
__device__ __forceinline__ zd h0_free64(double x)
{
    if (x > 2.0) return zd{-0.25 * y0(x), 0.25 * j0(x)};
    const double z = 0.25 * x * x;
    double j = c_h0s.cj[H0S_TERMS - 1], sy = c_h0s.cy[H0S_TERMS - 1];
#pragma unroll
    for (int m = H0S_TERMS - 2; m >= 0; --m) {
        j = fma(j, z, c_h0s.cj[m]);
        sy = fma(sy, z, c_h0s.cy[m]);
    }
    const double y = 0.63661977236758134308 * ((log(0.5 * x) + 0.57721566490153286061) * j + sy);
    return zd{-0.25 * y, 0.25 * j};
}

// ---------------------------------------------------------------------------
// Direct interaction of one reflected term (tt: term 1, bb: term 2) for a
// pair at horizontal distance X and image height h, by the near-field
// quadrature tables (segment + nearest steepest-descent ray).
// ---------------------------------------------------------------------------
struct NearQuadD {
    int nseg, nray, ntail;
    const zd *seg_lam, *seg_s2, *seg_w, *tail_lam, *tail_s2, *tail_w;
    double rinf[2]; // wall limit of sigma_tt, sigma_bb: the tables hold sigma - rinf (refl_inf)
    double hray;    // added to h when the tail ray is chosen (see NearQuad)
    const zd *tail_w2; // multiple-reflection tail weights (walls on both sides), else null
    int a_zero;        // the single-reflection part tail_w is identically zero
    double d2;         // 2d: the multiple reflections' extra image height
    // the target gradient with an impedance wall: weights of 2 i beta / s2 on the segment and
    // on the tail rays of tail_w, taken out of the h-derivative (null otherwise), and beta per wall
    const zd *seg_c, *tail_c;
    double beta[2];
};
// tail ray nearest the steepest-descent direction of (X, h)
__device__ __forceinline__ int tail_ray(const NearQuadD &q, double X, double h)
{
    return q.nray > 1 ? (int)rint(atan2(X, h) * (q.nray - 1) / (0.5 * M_PI)) : 0;
}
// sum P Re(E) + i M Im(E) over ray k of the weight table W (layout of NearQuad::tail_w)
__device__ __forceinline__ zd tail_sum(const NearQuadD &q, const zd *W, int m, int k, double X, double h)
{
    const zd *tl = q.tail_lam + (int64_t)k * q.ntail, *ts = q.tail_s2 + (int64_t)k * q.ntail;
    const int64_t tot = (int64_t)q.nray * q.ntail;
    const zd *tP = W + (2 * m) * tot + (int64_t)k * q.ntail, *tM = tP + tot;
    zd acc = {0.0, 0.0};
    for (int i = 0; i < q.ntail; ++i) {
        const zd lam = tl[i], s2 = ts[i];
        const zd e = cexpd(zd{-lam.im * X - s2.re * h, lam.re * X - s2.im * h});
        acc = acc + e.re * tP[i] + e.im * zd{-tM[i].im, tM[i].re};
    }
    return acc;
}
__device__ zd near_refl64(const NearQuadD &q, int m, double X, double h, bool seg = true)
{
    zd acc = {0.0, 0.0};
    const zd *W = q.seg_w + (int64_t)m * q.nseg;
    for (int i = 0; i < (seg ? q.nseg : 0); ++i) {
        zd lam = q.seg_lam[i], s2 = q.seg_s2[i];
        // e^{+i lam X - s2 h} + e^{-i lam X - s2 h}
        double er = -s2.re * h, ei = -s2.im * h;
        zd e1 = cexpd(zd{er - lam.im * X, ei + lam.re * X});
        zd e2 = cexpd(zd{er + lam.im * X, ei - lam.re * X});
        cfma(acc, W[i], e1 + e2);
    }
    if (q.tail_w2) { // walls on both sides: single reflection on the ray of (X, h), multiples on (X, h + 2d)
        if (!q.a_zero) acc = acc + tail_sum(q, q.tail_w, m, tail_ray(q, X, h), X, h);
        return acc + tail_sum(q, q.tail_w2, m, tail_ray(q, X, h + q.d2), X, h);
    }
    return acc + tail_sum(q, q.tail_w, m, tail_ray(q, X, h + q.hray), X, h);
}

// ---------------------------------------------------------------------------
// Step 4: L2T (Eq. (local)) and S2T for every target of a leaf.  L2T takes one
// thread per target.  The direct interactions take one warp per target: the
// leaf's U entries are flattened (in chunks) into one list of near sources,
// the lanes split it, and a butterfly of shuffles sums the lanes in a fixed
// order.  A thread per target left most lanes idle on small leaves while the
// FP64 pipes stepped through the per-pair tails.
// ---------------------------------------------------------------------------
#define LEAF64_THREADS 128
#define LEAF64_UCHUNK 64
template <class Geo>
__global__ void __launch_bounds__(LEAF64_THREADS)
    k_leaf64(Geo geo, int P, double k, double d, const double *xs, const double *ys, const int64_t *ls,
             const int64_t *ustart, const int32_t *usrc, const int32_t *uterm, NearQuadD nq, const zd *Lc,
             const zd *qs, int64_t n, int nvec, int free_on, int pw, zd *us)
{
    __shared__ int64_t fj0[LEAF64_UCHUNK]; // first tree position of each entry's source leaf
    __shared__ int fpre[LEAF64_UCHUNK + 1]; // running count of near sources before each entry
    __shared__ int fterm[LEAF64_UCHUNK];
    const int np = 2 * P + 1;
    const int64_t b = geo.id(blockIdx.x);
    double cx, cy, bw;
    geo.centre(b, &cx, &cy, &bw);
    const double sc = k * bw;
    const zd *Lb = Lc + b * np * LM_MAXV;
    const int64_t lo = ls[b], hi = ls[b + 1];
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x) {
        const double xi = xs[i], yi = ys[i];
        zd acc[LM_MAXV];
        for (int v = 0; v < nvec; ++v) acc[v] = zd{0.0, 0.0};
        double rx = xi - cx, ry = yi - cy, r = hypot(rx, ry);
        double J[LM_MAXP + 1];
        bessel_j_scaled<double>(P, k * r, sc, J);
        zd z = r > 0.0 ? zd{rx / r, ry / r} : zd{1.0, 0.0}; // e^{i theta}
        zd zp = {1.0, 0.0};
        for (int v = 0; v < nvec; ++v) cfma(acc[v], zd{J[0], 0.0}, Lb[P * LM_MAXV + v]);
        for (int m = 1; m <= P; ++m) {
            zp = zp * z;
            zd bp = J[m] * zp;
            zd bn = ((m & 1) ? -J[m] : J[m]) * conj(zp);
            for (int v = 0; v < nvec; ++v) {
                cfma(acc[v], bp, Lb[(P + m) * LM_MAXV + v]);
                cfma(acc[v], bn, Lb[(P - m) * LM_MAXV + v]);
            }
        }
        for (int v = 0; v < nvec; ++v) us[(int64_t)v * n + i] = acc[v];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int64_t u0 = ustart[b], u1 = ustart[b + 1];
    for (int64_t c0 = u0; c0 < u1; c0 += LEAF64_UCHUNK) {
        const int nc = (int)min((int64_t)LEAF64_UCHUNK, u1 - c0);
        __syncthreads(); // L2T values written, previous chunk finished
        if (threadIdx.x == 0) {
            int run = 0;
            for (int e = 0; e < nc; ++e) {
                const int32_t s = usrc[c0 + e], term = uterm[c0 + e];
                fj0[e] = ls[s];
                fterm[e] = term;
                fpre[e] = run;
                run += (term == 0 && !free_on) ? 0 : (int)(ls[s + 1] - ls[s]);
            }
            fpre[nc] = run;
        }
        __syncthreads();
        const int tot = fpre[nc];
        for (int64_t i = lo + warp; i < hi; i += nwarp) {
            const double xi = xs[i], yi = ys[i];
            zd acc[LM_MAXV];
            for (int v = 0; v < nvec; ++v) acc[v] = zd{0.0, 0.0};
            int e = 0;
            for (int f = lane; f < tot; f += 32) {
                while (fpre[e + 1] <= f) ++e; // f < tot = fpre[nc] keeps e < nc
                const int64_t j = fj0[e] + (f - fpre[e]);
                const int term = fterm[e];
                zd gij;
                if (term == 0) {
                    if (j == i) continue;
                    const double r = hypot(xi - xs[j], yi - ys[j]);
                    gij = h0_free64(k * r); // (i/4) H0^(1)(k r)
                } else {
                    const double X = fabs(xi - xs[j]);
                    const double h = term == 1 ? -(yi + ys[j]) : yi + ys[j] + 2.0 * d;
                    gij = near_refl64(nq, term - 1, X, h, !pw); // segment added by k_near_pw64
                    const double ri = nq.rinf[term - 1];
                    if (ri != 0.0) gij = gij + ri * h0_free64(k * hypot(X, h)); // the wall's image, closed form
                }
                for (int v = 0; v < nvec; ++v) cfma(acc[v], gij, qs[(int64_t)v * n + j]);
            }
            for (int v = 0; v < nvec; ++v) {
                double re = acc[v].re, im = acc[v].im;
                for (int o = 16; o > 0; o >>= 1) {
                    re += __shfl_xor_sync(0xffffffffu, re, o);
                    im += __shfl_xor_sync(0xffffffffu, im, o);
                }
                if (lane == 0) us[(int64_t)v * n + i] = us[(int64_t)v * n + i] + zd{re, im};
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Segment part of the reflected direct terms, factorised per target leaf (FP64
// form of the mixed path's k_near_pw32).  On the fixed segment the folded
// integrand of a pair separates,
//   2 cos(lambda (x_i - x_j)) e^{-s2 h_ij} = sum_{s=+-1} e^{s i lambda (x_i - x_T)} E(y_i) e^{-s i lambda (x_j - x_T)} E(y_j),
// E(y) = e^{s2 y} (tt) or e^{-s2 (y + d)} (bb), x_T the target leaf centre:
// phase A sums the near sources into B_{n,s}[v], phase B evaluates them at the
// leaf's targets and adds to us.  One block per leaf of the top (and bottom) row.
// ---------------------------------------------------------------------------
#define PW64_SRC 64
size_t lm_near_pw64_smem(int nseg) { return (size_t)2 * nseg * LM_MAXV * sizeof(zd); }
#define PW64_SRC_SMEM (PW64_SRC * LM_MAXV * sizeof(zd) + 2 * PW64_SRC * sizeof(double))
// Phase A works per U entry through the source leaf's own coefficients: with
// c_s the source leaf centre, x_j - x_T = (x_j - c_s) + (c_s - x_T), so
//   C_{k,s}(S) = sum_{j in S} e^{-s i lambda_k (x_j - c_s)} E(y_j) q_j
// is formed once per interface leaf and apply (k_pw_src64), and each U entry
// adds e^{-s i lambda_k (c_s - x_T)} C_{k,s}(S): one exponential per node and
// entry instead of one per node and source point.  An interface leaf's tt (bb)
// sources are interface leaves themselves (the image adjacency is symmetric),
// so every source has its coefficients; pwidx maps a box to its slot.
template <class Geo>
__global__ void __launch_bounds__(256) k_pw_src64(Geo geo, double d, const double *xs, const double *ys,
                                                  const int64_t *ls, const int64_t *ustart, const int32_t *uterm,
                                                  NearQuadD nq, const zd *qs, int64_t n, int nvec, zd *C)
{
    extern __shared__ unsigned char smem[];
    const int nk = 2 * nq.nseg;
    zd *SQ = (zd *)smem;                              // [PW64_SRC][LM_MAXV]
    double *SX = (double *)(SQ + PW64_SRC * LM_MAXV); // [PW64_SRC]
    double *SY = SX + PW64_SRC;                       // [PW64_SRC]
    const int64_t slot = blockIdx.x, b = geo.id(slot);
    if (ls[b + 1] == ls[b]) return; // an empty leaf: its coefficients are never read
    double cs, ys_, ws;
    geo.centre(b, &cs, &ys_, &ws);
    for (int term = 1; term <= 2; ++term) {
        bool any = false;
        for (int64_t e = ustart[b]; e < ustart[b + 1]; ++e) any |= (uterm[e] == term);
        if (!any) continue; // block-uniform
        const int m = term - 1;
        zd *Cm = C + ((slot * 2 + m) * nk) * LM_MAXV;
        for (int k = threadIdx.x; k < nk; k += blockDim.x)
            for (int v = 0; v < nvec; ++v) Cm[k * LM_MAXV + v] = zd{0.0, 0.0};
        for (int64_t j0 = ls[b]; j0 < ls[b + 1]; j0 += PW64_SRC) {
            const int cnt = (int)min((int64_t)PW64_SRC, ls[b + 1] - j0);
            __syncthreads();
            for (int t = threadIdx.x; t < cnt * nvec; t += blockDim.x) {
                const int jj = t % cnt, v = t / cnt;
                SQ[jj * LM_MAXV + v] = qs[(int64_t)v * n + j0 + jj];
            }
            for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
                SX[t] = xs[j0 + t] - cs;
                SY[t] = ys[j0 + t];
            }
            __syncthreads();
            for (int k = threadIdx.x; k < nk; k += blockDim.x) {
                const zd lam = nq.seg_lam[k >> 1], s2 = nq.seg_s2[k >> 1];
                const double sg = (k & 1) ? -1.0 : 1.0;
                zd part[LM_MAXV];
                for (int v = 0; v < nvec; ++v) part[v] = zd{0.0, 0.0};
                for (int t = 0; t < cnt; ++t) {
                    const double x = SX[t], y = SY[t];
                    zd ex = {sg * lam.im * x, -sg * lam.re * x}; // -s i lambda (x_j - c_s)
                    ex = ex + (m == 0 ? y * s2 : -(y + d) * s2);
                    const zd f = cexpd(ex);
                    for (int v = 0; v < nvec; ++v) cfma(part[v], f, SQ[t * LM_MAXV + v]);
                }
                for (int v = 0; v < nvec; ++v) Cm[k * LM_MAXV + v] = Cm[k * LM_MAXV + v] + part[v];
            }
        }
    }
}

template <class Geo>
__global__ void __launch_bounds__(256) k_near_pw64(Geo geo, double d, const double *xs,
                                                   const double *ys, const int64_t *ls, const int64_t *ustart,
                                                   const int32_t *usrc, const int32_t *uterm, NearQuadD nq,
                                                   const zd *qs, const zd *C, const int32_t *pwidx, int64_t n,
                                                   int nvec, zd *us)
{
    extern __shared__ unsigned char smem[];
    const int nk = 2 * nq.nseg;
    zd *B = (zd *)smem;                              // [nk][LM_MAXV]
    const int64_t b = geo.id(blockIdx.x);
    if (ls[b + 1] == ls[b]) return; // no targets (block-uniform)
    double xT, yT, wT;
    geo.centre(b, &xT, &yT, &wT);
    for (int term = 1; term <= 2; ++term) {
        bool any = false;
        for (int64_t e = ustart[b]; e < ustart[b + 1]; ++e) any |= (uterm[e] == term);
        if (!any) continue; // block-uniform
        const int m = term - 1;
        const zd *W = nq.seg_w + (int64_t)m * nq.nseg;
        __syncthreads();
        for (int k = threadIdx.x; k < nk * LM_MAXV; k += blockDim.x) B[k] = zd{0.0, 0.0};
        __syncthreads();
        for (int64_t e = ustart[b]; e < ustart[b + 1]; ++e) {
            if (uterm[e] != term) continue;
            const int64_t s = usrc[e];
            if (ls[s + 1] == ls[s]) continue; // no sources (uniform over the block)
            double cs, ysc, wsc;
            geo.centre(s, &cs, &ysc, &wsc);
            const double dx = cs - xT;
            const zd *Cs = C + (((int64_t)pwidx[s] * 2 + m) * nk) * LM_MAXV;
            for (int k = threadIdx.x; k < nk; k += blockDim.x) {
                const zd lam = nq.seg_lam[k >> 1];
                const double sg = (k & 1) ? -1.0 : 1.0;
                const zd f = cexpd(zd{sg * lam.im * dx, -sg * lam.re * dx}); // -s i lambda (c_s - x_T)
                for (int v = 0; v < nvec; ++v) cfma(B[k * LM_MAXV + v], f, Cs[k * LM_MAXV + v]);
            }
        }
        __syncthreads();
        const int64_t lo = ls[b], cntT = ls[b + 1] - lo;
        for (int64_t t = threadIdx.x; t < cntT * nvec; t += blockDim.x) {
            const int64_t i = lo + t % cntT;
            const int v = (int)(t / cntT);
            const double x = xs[i] - xT, y = ys[i];
            zd acc = {0.0, 0.0};
            for (int k = 0; k < nk; ++k) {
                const zd lam = nq.seg_lam[k >> 1], s2 = nq.seg_s2[k >> 1];
                const double sg = (k & 1) ? -1.0 : 1.0;
                zd ex = {-sg * lam.im * x, sg * lam.re * x}; // s i lambda x
                ex = ex + (m == 0 ? y * s2 : -(y + d) * s2);
                cfma(acc, cexpd(ex) * W[k >> 1], B[k * LM_MAXV + v]);
            }
            us[(int64_t)v * n + i] = us[(int64_t)v * n + i] + acc;
        }
    }
}

// ---------------------------------------------------------------------------
// Target gradient of one reflected direct term: the value, d/dX and d/dh of
// the near-field quadrature of near_refl64 (segment: e^{+-i lam X} -> +-i lam,
// e^{-s2 h} -> -s2; tail: Z = E -> i lam E, -s2 E in P Re(Z) + i M Im(Z)).
// ---------------------------------------------------------------------------
__device__ void near_refl64_grad(const NearQuadD &q, int m, double X, double h, zd *val, zd *dX, zd *dh)
{
    zd a0 = {0.0, 0.0}, a1 = {0.0, 0.0}, a2 = {0.0, 0.0};
    const zd *W = q.seg_w + (int64_t)m * q.nseg;
    // an impedance wall: the h-derivative sums (sigma - 1 - 2 i beta / s2) s2, whose
    // integrand decays with e^{-lam h}; the caller adds the 2 i beta / s2 part in closed form
    const zd *Cs = q.seg_c ? q.seg_c + (int64_t)m * q.nseg : nullptr;
    for (int i = 0; i < q.nseg; ++i) {
        zd lam = q.seg_lam[i], s2 = q.seg_s2[i];
        double er = -s2.re * h, ei = -s2.im * h;
        zd e1 = cexpd(zd{er - lam.im * X, ei + lam.re * X});
        zd e2 = cexpd(zd{er + lam.im * X, ei - lam.re * X});
        zd we = W[i] * (e1 + e2);
        a0 = a0 + we;
        cfma(a1, W[i] * zd{-lam.im, lam.re}, e1 - e2);
        cfma(a2, -1.0 * s2, Cs ? we - Cs[i] * (e1 + e2) : we);
    }
    // the tail: one weight table on one ray, or (walls on both sides) single and multiple
    // reflections on their own rays, as in near_refl64; Ct (or null) the correction on Wt's rays
    auto tail = [&](const zd *Wt, const zd *Ct, int k) {
        const zd *tl = q.tail_lam + (int64_t)k * q.ntail, *ts = q.tail_s2 + (int64_t)k * q.ntail;
        const int64_t tot = (int64_t)q.nray * q.ntail;
        const int64_t o = (2 * m) * tot + (int64_t)k * q.ntail;
        const zd *tP = Wt + o, *tM = tP + tot;
        for (int i = 0; i < q.ntail; ++i) {
            zd lam = tl[i], s2 = ts[i];
            const zd e = cexpd(zd{-lam.im * X - s2.re * h, lam.re * X - s2.im * h});
            const zd P = tP[i], iM = zd{-tM[i].im, tM[i].re};
            const zd z1 = zd{-lam.im, lam.re} * e, z2 = -1.0 * (s2 * e); // i lam E, -s2 E
            a0 = a0 + e.re * P + e.im * iM;
            a1 = a1 + z1.re * P + z1.im * iM;
            if (Ct) {
                const zd cP = Ct[o + i], ciM = zd{-Ct[o + tot + i].im, Ct[o + tot + i].re};
                a2 = a2 + z2.re * (P - cP) + z2.im * (iM - ciM);
            } else {
                a2 = a2 + z2.re * P + z2.im * iM;
            }
        }
    };
    if (q.tail_w2) {
        if (!q.a_zero) tail(q.tail_w, q.tail_c, tail_ray(q, X, h));
        tail(q.tail_w2, nullptr, tail_ray(q, X, h + q.d2));
    } else {
        tail(q.tail_w, q.tail_c, tail_ray(q, X, h + q.hray));
    }
    *val = a0;
    *dX = a1;
    *dh = a2;
}

// ---------------------------------------------------------------------------
// Step 4 with the target gradient: u, du/dx, du/dy for nv <= GV vectors
// starting at v0, written straight to input order through perm.  Far field:
// the local expansion differentiated with (d/dx + i d/dy) J_n e^{i n t} =
// -k J_{n+1} e^{i(n+1)t} and (d/dx - i d/dy) J_n e^{i n t} = k J_{n-1}
// e^{i(n-1)t}; in scaled coefficients the shifts carry S(|n|)/S(|n -+ 1|).
// ---------------------------------------------------------------------------
#define GV 4
template <class Geo>
__global__ void __launch_bounds__(LEAF64_THREADS) k_leaf64_grad(Geo geo, int P, double k, double d, const double *xs, const double *ys,
                              const int64_t *ls, const int64_t *ustart, const int32_t *usrc,
                              const int32_t *uterm, NearQuadD nq, const zd *Lc, const zd *qs, int64_t n,
                              int v0, int nv, int free_on, const int64_t *perm, zd *u, zd *ux, zd *uy)
{
    const int64_t b = geo.id(blockIdx.x);
    double cx, cy, bw;
    geo.centre(b, &cx, &cy, &bw);
    const double sc = k * bw, hs = 0.5 * sc;
    const zd *Lb = Lc + b * (2 * P + 1) * LM_MAXV + v0;
    __shared__ int64_t fj0[LEAF64_UCHUNK];
    __shared__ int fpre[LEAF64_UCHUNK + 1];
    __shared__ int fterm[LEAF64_UCHUNK];
    for (int64_t i = ls[b] + threadIdx.x; i < ls[b + 1]; i += blockDim.x) {
        const double xi = xs[i], yi = ys[i];
        zd a[GV], dp[GV], dm[GV], gxa[GV], gya[GV]; // dp = (d/dx - i d/dy) u, dm = (d/dx + i d/dy) u
        for (int v = 0; v < GV; ++v) a[v] = dp[v] = dm[v] = zd{0.0, 0.0};
        {
            double rx = xi - cx, ry = yi - cy, r = hypot(rx, ry);
            double J[LM_MAXP + 2];
            bessel_j_scaled<double>(P + 1, k * r, sc, J);
            zd z = r > 0.0 ? zd{rx / r, ry / r} : zd{1.0, 0.0}; // e^{i theta}
            zd zp = {1.0, 0.0};
            for (int m = 0; m <= P + 1; ++m) {
                if (m > 0) zp = zp * z;
                const zd bp = J[m] * zp;                           // Jhat_m e^{i m t}
                const zd bn = ((m & 1) ? -J[m] : J[m]) * conj(zp); // Jhat_{-m} e^{-i m t}
                const double rdn = m >= 1 ? hs / m : 0.0;          // S(m)/S(m-1)
                const double rup = (m + 1) / hs;                   // S(m)/S(m+1)
                for (int v = 0; v < nv; ++v) {
                    const zd *Lv = Lb + P * LM_MAXV + v; // Lv[n * LM_MAXV] = Lhat_n
                    if (m <= P) cfma(a[v], bp, Lv[m * LM_MAXV]);
                    if (m >= 1 && m <= P) cfma(a[v], bn, Lv[-m * LM_MAXV]);
                    // dm = -k sum_n L_{n-1} J_n e^{i n t}: n = m, and n = -m (m >= 1, -m-1 >= -P)
                    if (m >= 1) cfma(dm[v], (-k * rdn) * bp, Lv[(m - 1) * LM_MAXV]);
                    else cfma(dm[v], (-k / hs) * bp, Lv[-LM_MAXV]);
                    if (m >= 1 && m <= P - 1) cfma(dm[v], (-k * rup) * bn, Lv[(-m - 1) * LM_MAXV]);
                    // dp = k sum_n L_{n+1} J_n e^{i n t}: n = m (m + 1 <= P), and n = -m (m >= 1)
                    if (m <= P - 1) cfma(dp[v], (k * rup) * bp, Lv[(m + 1) * LM_MAXV]);
                    if (m >= 1) cfma(dp[v], (k * rdn) * bn, Lv[(1 - m) * LM_MAXV]);
                }
            }
            for (int v = 0; v < GV; ++v) {
                gxa[v] = 0.5 * (dp[v] + dm[v]);
                const zd df = dp[v] - dm[v];
                gya[v] = zd{-0.5 * df.im, 0.5 * df.re}; // i (dp - dm) / 2
            }
        }
        const int64_t o = perm[i];
        for (int v = 0; v < nv; ++v) {
            if (u) u[(int64_t)v * n + o] = a[v];
            ux[(int64_t)v * n + o] = gxa[v];
            uy[(int64_t)v * n + o] = gya[v];
        }
    }
    // direct interactions: one warp per target over the flattened near sources (as k_leaf64)
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    const int64_t lo = ls[b], hi = ls[b + 1], u0 = ustart[b], u1 = ustart[b + 1];
    for (int64_t c0 = u0; c0 < u1; c0 += LEAF64_UCHUNK) {
        const int nc = (int)min((int64_t)LEAF64_UCHUNK, u1 - c0);
        __syncthreads(); // far-field values written, previous chunk finished
        if (threadIdx.x == 0) {
            int run = 0;
            for (int e = 0; e < nc; ++e) {
                const int32_t s = usrc[c0 + e], term = uterm[c0 + e];
                fj0[e] = ls[s];
                fterm[e] = term;
                fpre[e] = run;
                run += (term == 0 && !free_on) ? 0 : (int)(ls[s + 1] - ls[s]);
            }
            fpre[nc] = run;
        }
        __syncthreads();
        const int tot = fpre[nc];
        for (int64_t i = lo + warp; i < hi; i += nwarp) {
            const double xi = xs[i], yi = ys[i];
            zd a[GV], gxa[GV], gya[GV];
            for (int v = 0; v < GV; ++v) a[v] = gxa[v] = gya[v] = zd{0.0, 0.0};
            int e = 0;
            for (int f = lane; f < tot; f += 32) {
                while (fpre[e + 1] <= f) ++e; // f < tot = fpre[nc] keeps e < nc
                const int64_t j = fj0[e] + (f - fpre[e]);
                const int term = fterm[e];
                zd gv, gx, gy;
                const double Dx = xi - xs[j];
                if (term == 0) {
                    if (j == i) continue;
                    const double Dy = yi - ys[j], r = hypot(Dx, Dy);
                    zd h1;
                    h01_free64(k * r, &gv, &h1);    // (i/4) H0, (i/4) H1
                    const zd dr = (-k) * h1;          // d/dr (i/4) H0(k r) = (i/4)(-k) H1
                    gx = (Dx / r) * dr;
                    gy = (Dy / r) * dr;
                } else {
                    const double X = fabs(Dx);
                    const double h = term == 1 ? -(yi + ys[j]) : yi + ys[j] + 2.0 * d;
                    zd dX, dh;
                    near_refl64_grad(nq, term - 1, X, h, &gv, &dX, &dh);
                    const double ri = nq.rinf[term - 1];
                    if (ri != 0.0) { // the wall's image (i/4) H0(k rho), rho = |(X, h)|, and its derivatives
                        const double rho = hypot(X, h);
                        zd h0, h1;
                        h01_free64(k * rho, &h0, &h1);
                        const zd dr = (-k * ri / rho) * h1;
                        gv = gv + ri * h0;
                        dX = dX + X * dr;
                        dh = dh + h * dr + zd{0.0, -2.0 * nq.beta[term - 1]} * h0; // -2 i beta (i/4) H0
                    }
                    gx = (Dx > 0.0 ? 1.0 : (Dx < 0.0 ? -1.0 : 0.0)) * dX;
                    gy = (term == 1 ? -1.0 : 1.0) * dh; // dh/dy: -1 (tt), +1 (bb)
                }
                for (int v = 0; v < nv; ++v) {
                    const zd qj = qs[(int64_t)(v0 + v) * n + j];
                    cfma(a[v], gv, qj);
                    cfma(gxa[v], gx, qj);
                    cfma(gya[v], gy, qj);
                }
            }
            const int64_t o = perm[i];
            for (int v = 0; v < nv; ++v) {
                double r6[6] = {a[v].re, a[v].im, gxa[v].re, gxa[v].im, gya[v].re, gya[v].im};
                for (int c = 0; c < 6; ++c)
                    for (int off = 16; off > 0; off >>= 1) r6[c] += __shfl_xor_sync(0xffffffffu, r6[c], off);
                if (lane == 0) {
                    if (u) u[(int64_t)v * n + o] = u[(int64_t)v * n + o] + zd{r6[0], r6[1]};
                    ux[(int64_t)v * n + o] = ux[(int64_t)v * n + o] + zd{r6[2], r6[3]};
                    uy[(int64_t)v * n + o] = uy[(int64_t)v * n + o] + zd{r6[4], r6[5]};
                }
            }
        }
    }
}

static lm_status run_fp64(lm_tree_s *t, const zd *q, int nvec, zd *u, bool adjoint, zd *ux, zd *uy,
                          cudaStream_t st);

lm_status lm_run_apply(lm_tree_s *t, const zd *q, int nvec, zd *u, bool adjoint, cudaStream_t st)
{
    if (t->precision == LM_MIXED) return lm_run_apply_mixed(t, q, nvec, u, adjoint, false, st);
    return run_fp64(t, q, nvec, u, adjoint, nullptr, nullptr, st);
}

lm_status lm_run_apply_grad(lm_tree_s *t, const zd *q, int nvec, zd *u, zd *ux, zd *uy, cudaStream_t st)
{
    return run_fp64(t, q, nvec, u, false, ux, uy, st);
}

// FP64 driver of the adaptive tree: the same steps over the box lists of each level
static lm_status run_fp64_adaptive(lm_tree_s *t, const zd *q, int nvec, zd *u, bool adjoint, zd *ux, zd *uy,
                                   cudaStream_t st)
{
    const AdaptTree &A = t->at;
    const int L = t->L, P = t->p, np = 2 * P + 1;
    const int64_t n = t->n;
    const double k = t->med.k2;
    NearQuadD nq{t->nq.nseg, t->nq.nray, t->nq.ntail, t->nq.seg_lam, t->nq.seg_s2,
                 t->nq.seg_w, t->nq.tail_lam, t->nq.tail_s2, t->nq.tail_w, {t->nq.rinf[0], t->nq.rinf[1]}, t->nq.hray,
                 t->nq.tail_w2, t->nq.a_zero, 2.0 * t->med.d, nullptr, nullptr, {0.0, 0.0}};
    // the target gradient integrates its differentiated tails with the longer rule
    const NearQuadD nqg{t->nq.nseg,     t->nq.nray,       t->nq.ntail_g,   t->nq.seg_lam,
                        t->nq.seg_s2,   t->nq.seg_w,      t->nq.tail_lam_g, t->nq.tail_s2_g,
                        t->nq.tail_w_g, {t->nq.rinf[0], t->nq.rinf[1]}, t->nq.hray,
                        t->nq.tail_w2_g, t->nq.a_zero, 2.0 * t->med.d,
                        t->nq.seg_c, t->nq.tail_c_g, {t->nq.beta[0], t->nq.beta[1]}};
    const ListBoxes leaves{A.leaves, A.cx, A.cy, A.w}, pwl{A.pwleaves, A.cx, A.cy, A.w};
    const int free_on = t->med.opt.kernel == LM_KERNEL_G;
    for (int v0 = 0; v0 < nvec; v0 += LM_MAXV) {
        const int nv = std::min(LM_MAXV, nvec - v0);
        lm_phase_begin(t, PH_PERMUTE, st);
        k_permute_in<<<gridn(n, 256), 256, 0, st>>>(q + (int64_t)v0 * n, t->perm, n, nv, adjoint, t->qs);
        if (t->m2l_df) {
            LM_CUDA(cudaMemsetAsync(t->qexp, 0x80, sizeof(int), st)); // below any exponent
            k_qexp<<<std::min(1024, gridn(n * nv, 256)), 256, 0, st>>>(t->qs, n, nv, t->qexp);
        }
        lm_phase_end(t, PH_PERMUTE, st, t->m2l_df ? 2 : 1);
        // step 2: S2M at every leaf, M2M up the levels
        lm_phase_begin(t, PH_S2M, st);
        const size_t shm = (P2M_CHUNK * np + P2M_CHUNK * LM_MAXV) * sizeof(zd);
        k_p2m64_list<<<(unsigned)A.nleaf, p2m_threads(np * nv), shm, st>>>(leaves, P, k, t->xs, t->ys, t->leaf_start, t->qs, n, nv,
                                                           A.M);
        lm_phase_end(t, PH_S2M, st, 1);
        int nl = 0;
        lm_phase_begin(t, PH_M2M, st);
        for (int l = L - 1; l >= 0; --l) {
            const int64_t npar = A.nl_start[l + 1] - A.nl_start[l];
            if (npar == 0) continue;
            if (t->m2l_df)
                k_m2m_df<<<(unsigned)npar, df_threads(np * nv), np * nv * sizeof(float4), st>>>(
                    ListParents{A.nonleaf + A.nl_start[l], A.child}, P, nv, t->lev[l].m2mdf, A.M, t->qexp, A.M);
            else
                k_m2m64a<<<gridn(npar * np * nv, 128), 128, 0, st>>>(npar, A.nonleaf + A.nl_start[l], A.child, P,
                                                                     nv, t->lev[l].m2m, A.M);
            ++nl;
        }
        lm_phase_end(t, PH_M2M, st, nl);
        if (t->m2l_df) {
            lm_phase_begin(t, PH_M2L, st);
            k_m_df<<<gridn(A.nbox * np * nv, 256), 256, 0, st>>>(0, A.nbox, P, nv, A.M, t->qexp, A.Mdf);
            lm_phase_end(t, PH_M2L, st, 1);
        }
        // step 3: level by level, L2L from the parent then M2L from the V list
        for (int l = 0; l <= L; ++l) {
            const int64_t b0 = A.lev_start[l], nb = A.lev_start[l + 1] - b0;
            lm_phase_begin(t, PH_L2L, st);
            if (l == 0)
                LM_CUDA(cudaMemsetAsync(A.Lc, 0, nb * np * LM_MAXV * sizeof(zd), st));
            else if (t->m2l_df) {
                const int64_t npar = A.nl_start[l] - A.nl_start[l - 1]; // the parents of level l
                k_l2l_df<<<(unsigned)npar, df_threads(4 * np * nv), np * nv * sizeof(float4), st>>>(
                    ListParents{A.nonleaf + A.nl_start[l - 1], A.child}, P, nv, t->lev[l].l2ldf, A.Lc, t->qexp, A.Lc);
            } else
                k_l2l64a<<<gridn(nb * np * nv, 128), 128, 0, st>>>(b0, nb, A.parent, A.pos, P, nv, t->lev[l].l2l,
                                                                   A.Lc);
            lm_phase_end(t, PH_L2L, st, l > 0);
            lm_phase_begin(t, PH_M2L, st);
            if (A.lev_nv[l] > 0 && t->m2l_df && nv <= DF_TR_NV)
                k_m2l_df<true><<<gridn(nb * np * nv, 128), 128, 0, st>>>(
                    nb, P, nv, A.vstart + b0, A.vsrc, A.vslot, A.tabdft, A.Mdf, t->qexp, A.Lc + b0 * np * LM_MAXV);
            else if (A.lev_nv[l] > 0 && t->m2l_df)
                k_m2l_df<false><<<gridn(nb * np * nv, 128), 128, 0, st>>>(
                    nb, P, nv, A.vstart + b0, A.vsrc, A.vslot, A.tabdf, A.Mdf, t->qexp, A.Lc + b0 * np * LM_MAXV);
            else if (A.lev_nv[l] > 0)
                k_m2l64<<<gridn(nb * np * nv, 128), 128, 0, st>>>(nb, P, nv, A.vstart + b0, A.vsrc, A.vslot, A.tab,
                                                                  A.M, A.Lc + b0 * np * LM_MAXV);
            lm_phase_end(t, PH_M2L, st, A.lev_nv[l] > 0);
        }
        // step 4: L2T and the direct list at every leaf
        lm_phase_begin(t, PH_LEAF, st);
        if (ux) {
            const int64_t off = (int64_t)v0 * n;
            int ng = 0;
            for (int w0 = 0; w0 < nv; w0 += GV, ++ng)
                k_leaf64_grad<<<(unsigned)A.nleaf, LEAF64_THREADS, 0, st>>>(
                    leaves, P, k, t->med.d, t->xs, t->ys, t->leaf_start, t->ustart, t->usrc, t->uterm, nqg, A.Lc,
                    t->qs, n, w0, std::min(GV, nv - w0), free_on, t->perm, u ? u + off + (int64_t)w0 * n : nullptr,
                    ux + off + (int64_t)w0 * n, uy + off + (int64_t)w0 * n);
            lm_phase_end(t, PH_LEAF, st, ng);
            LM_CUDA(cudaGetLastError());
            continue;
        }
        const int pw = t->near_pw64 ? 1 : 0;
        k_leaf64<<<(unsigned)A.nleaf, LEAF64_THREADS, 0, st>>>(leaves, P, k, t->med.d, t->xs, t->ys, t->leaf_start, t->ustart,
                                                   t->usrc, t->uterm, nq, A.Lc, t->qs, n, nv, free_on, pw, t->us);
        if (pw && A.npw > 0) {
            k_pw_src64<<<(unsigned)A.npw, 256, PW64_SRC_SMEM, st>>>(pwl, t->med.d, t->xs, t->ys, t->leaf_start,
                                                                    t->ustart, t->uterm, nq, t->qs, n, nv, t->pwC);
            k_near_pw64<<<(unsigned)A.npw, 256, lm_near_pw64_smem(t->nq.nseg), st>>>(
                pwl, t->med.d, t->xs, t->ys, t->leaf_start, t->ustart, t->usrc, t->uterm, nq, t->qs, t->pwC, t->pwidx,
                n, nv, t->us);
        }
        lm_phase_end(t, PH_LEAF, st, (pw && A.npw > 0) ? 3 : 1);
        lm_phase_begin(t, PH_PERMUTE, st);
        k_permute_out<<<gridn(n, 256), 256, 0, st>>>(t->us, t->perm, n, nv, adjoint, u + (int64_t)v0 * n);
        lm_phase_end(t, PH_PERMUTE, st, 1);
        LM_CUDA(cudaGetLastError());
    }
    return LM_OK;
}

// FP64 driver; with ux set, step 4 also evaluates the target gradient and writes u, ux, uy
static lm_status run_fp64(lm_tree_s *t, const zd *q, int nvec, zd *u, bool adjoint, zd *ux, zd *uy,
                          cudaStream_t st)
{
    if (t->adaptive) return run_fp64_adaptive(t, q, nvec, u, adjoint, ux, uy, st);
    const int L = t->L, P = t->p, np = 2 * P + 1;
    const int64_t n = t->n;
    const double k = t->med.k2;
    NearQuadD nq{t->nq.nseg, t->nq.nray, t->nq.ntail, t->nq.seg_lam, t->nq.seg_s2,
                 t->nq.seg_w, t->nq.tail_lam, t->nq.tail_s2, t->nq.tail_w, {t->nq.rinf[0], t->nq.rinf[1]}, t->nq.hray,
                 t->nq.tail_w2, t->nq.a_zero, 2.0 * t->med.d, nullptr, nullptr, {0.0, 0.0}};
    // the target gradient integrates its differentiated tails with the longer rule
    const NearQuadD nqg{t->nq.nseg,     t->nq.nray,       t->nq.ntail_g,   t->nq.seg_lam,
                        t->nq.seg_s2,   t->nq.seg_w,      t->nq.tail_lam_g, t->nq.tail_s2_g,
                        t->nq.tail_w_g, {t->nq.rinf[0], t->nq.rinf[1]}, t->nq.hray,
                        t->nq.tail_w2_g, t->nq.a_zero, 2.0 * t->med.d,
                        t->nq.seg_c, t->nq.tail_c_g, {t->nq.beta[0], t->nq.beta[1]}};
    for (int v0 = 0; v0 < nvec; v0 += LM_MAXV) {
        const int nv = std::min(LM_MAXV, nvec - v0);
        lm_phase_begin(t, PH_PERMUTE, st);
        k_permute_in<<<gridn(n, 256), 256, 0, st>>>(q + (int64_t)v0 * n, t->perm, n, nv, adjoint, t->qs);
        if (t->m2l_df) {
            LM_CUDA(cudaMemsetAsync(t->qexp, 0x80, sizeof(int), st)); // below any exponent
            k_qexp<<<std::min(1024, gridn(n * nv, 256)), 256, 0, st>>>(t->qs, n, nv, t->qexp);
        }
        lm_phase_end(t, PH_PERMUTE, st, t->m2l_df ? 2 : 1);
        // step 2: upward pass
        lm_phase_begin(t, PH_S2M, st);
        {
            Level &lv = t->lev[L];
            LeafGeom g{lv.ncol, t->x0, lv.w};
            size_t shm = (P2M_CHUNK * np + P2M_CHUNK * LM_MAXV) * sizeof(zd);
            k_p2m64<<<(unsigned)lv.nbox, p2m_threads(np * nv), shm, st>>>(g, P, k, t->xs, t->ys, t->leaf_start, t->qs, n,
                                                        nv, lv.M);
        }
        lm_phase_end(t, PH_S2M, st, 1);
        if (L > 0) lm_phase_begin(t, PH_M2M, st);
        for (int l = L - 1; l >= 0; --l) {
            Level &lv = t->lev[l];
            int64_t tot = lv.nbox * np * nv;
            if (t->m2l_df)
                k_m2m_df<<<(unsigned)lv.nbox, df_threads(np * nv), np * nv * sizeof(float4), st>>>(
                    GridParents{lv.ncol}, P, nv, lv.m2mdf, t->lev[l + 1].M, t->qexp, lv.M);
            else
                k_m2m64<<<gridn(tot, 128), 128, 0, st>>>(lv.ncol, lv.nbox, P, nv, lv.m2m, t->lev[l + 1].M, lv.M);
        }
        if (L > 0) lm_phase_end(t, PH_M2M, st, L);
        if (t->m2l_df) {
            lm_phase_begin(t, PH_M2L, st);
            for (int l = 0; l <= L; ++l) {
                Level &lv = t->lev[l];
                k_m_df<<<gridn(lv.nbox * np * nv, 256), 256, 0, st>>>(0, lv.nbox, P, nv, lv.M, t->qexp, lv.Mdf);
            }
            lm_phase_end(t, PH_M2L, st, L + 1);
        }

        // step 3: downward pass
        for (int l = 0; l <= L; ++l) {
            Level &lv = t->lev[l];
            int64_t tot = lv.nbox * np * nv;
            lm_phase_begin(t, PH_L2L, st);
            if (l == 0)
                LM_CUDA(cudaMemsetAsync(lv.Lc, 0, lv.nbox * np * LM_MAXV * sizeof(zd), st));
            else if (t->m2l_df)
                k_l2l_df<<<(unsigned)t->lev[l - 1].nbox, df_threads(4 * np * nv), np * nv * sizeof(float4), st>>>(
                    GridParents{t->lev[l - 1].ncol}, P, nv, lv.l2ldf, t->lev[l - 1].Lc, t->qexp, lv.Lc);
            else
                k_l2l64<<<gridn(tot, 128), 128, 0, st>>>(lv.ncol, lv.nbox, P, nv, lv.l2l, t->lev[l - 1].Lc,
                                                         lv.Lc);
            lm_phase_end(t, PH_L2L, st, l > 0);
            lm_phase_begin(t, PH_M2L, st);
            if (lv.nv > 0 && t->m2l_df && nv <= DF_TR_NV)
                k_m2l_df<true><<<gridn(tot, 128), 128, 0, st>>>(lv.nbox, P, nv, lv.vstart, lv.vsrc, lv.vslot,
                                                                lv.tabdft, lv.Mdf, t->qexp, lv.Lc);
            else if (lv.nv > 0 && t->m2l_df)
                k_m2l_df<false><<<gridn(tot, 128), 128, 0, st>>>(lv.nbox, P, nv, lv.vstart, lv.vsrc, lv.vslot,
                                                                 lv.tabdf, lv.Mdf, t->qexp, lv.Lc);
            else if (lv.nv > 0)
                k_m2l64<<<gridn(tot, 128), 128, 0, st>>>(lv.nbox, P, nv, lv.vstart, lv.vsrc, lv.vslot, lv.tab,
                                                         lv.M, lv.Lc);
            lm_phase_end(t, PH_M2L, st, lv.nv > 0);
        }
        // step 4: evaluation
        const int free_on = t->med.opt.kernel == LM_KERNEL_G;
        lm_phase_begin(t, PH_LEAF, st);
        if (ux) {
            Level &lv = t->lev[L];
            LeafGeom g{lv.ncol, t->x0, lv.w};
            const int64_t off = (int64_t)v0 * n;
            int nl = 0;
            for (int w0 = 0; w0 < nv; w0 += GV, ++nl)
                k_leaf64_grad<<<(unsigned)lv.nbox, LEAF64_THREADS, 0, st>>>(
                    GridLeaves{g}, P, k, t->med.d, t->xs, t->ys, t->leaf_start, t->ustart, t->usrc, t->uterm, nqg, lv.Lc,
                    t->qs, n, w0, std::min(GV, nv - w0), free_on, t->perm,
                    u ? u + off + (int64_t)w0 * n : nullptr, ux + off + (int64_t)w0 * n,
                    uy + off + (int64_t)w0 * n);
            lm_phase_end(t, PH_LEAF, st, nl);
            LM_CUDA(cudaGetLastError());
            continue;
        }
        {
            Level &lv = t->lev[L];
            LeafGeom g{lv.ncol, t->x0, lv.w};
            const int pw = t->near_pw64 ? 1 : 0;
            k_leaf64<<<(unsigned)lv.nbox, LEAF64_THREADS, 0, st>>>(GridLeaves{g}, P, k, t->med.d, t->xs, t->ys, t->leaf_start,
                                                       t->ustart, t->usrc, t->uterm, nq, lv.Lc, t->qs, n,
                                                       nv, free_on, pw, t->us);
            if (pw) {
                const unsigned npw = (unsigned)(lv.nrow == 1 ? lv.ncol : 2 * lv.ncol);
                const EdgeRowLeaves er{g, lv.nrow};
                k_pw_src64<<<npw, 256, PW64_SRC_SMEM, st>>>(er, t->med.d, t->xs, t->ys, t->leaf_start, t->ustart,
                                                             t->uterm, nq, t->qs, n, nv, t->pwC);
                k_near_pw64<<<npw, 256, lm_near_pw64_smem(t->nq.nseg), st>>>(
                    er, t->med.d, t->xs, t->ys, t->leaf_start, t->ustart, t->usrc, t->uterm, nq, t->qs, t->pwC,
                    t->pwidx, n, nv, t->us);
            }
        }
        lm_phase_end(t, PH_LEAF, st, t->near_pw64 ? 3 : 1);
        lm_phase_begin(t, PH_PERMUTE, st);
        k_permute_out<<<gridn(n, 256), 256, 0, st>>>(t->us, t->perm, n, nv, adjoint, u + (int64_t)v0 * n);
        lm_phase_end(t, PH_PERMUTE, st, 1);
        LM_CUDA(cudaGetLastError());
    }
    return LM_OK;
}

// dynamic shared-memory limit of k_near_pw64 (raised, never lowered: shared by all trees)
lm_status lm_near_pw64_attr(size_t bytes)
{
    LM_CUDA(lm_raise_smem((const void *)k_near_pw64<EdgeRowLeaves>, LM_SMEM_NEAR_PW64, (int)bytes));
    LM_CUDA(lm_raise_smem((const void *)k_near_pw64<ListBoxes>, LM_SMEM_NEAR_PW64_A, (int)bytes));
    return LM_OK;
}

// double-float copies of the M2L tables, multipole buffers and the exponent slot (FP64 form)
lm_status lm_setup_df(lm_tree_s *t, cudaStream_t st)
{
    if (!t->m2l_df) return LM_OK;
    const int np = 2 * t->p + 1;
    LM_CUDA(cudaMalloc((void **)&t->qexp, sizeof(int)));
    t->bytes += sizeof(int);
    auto conv = [&](const zd *tab, int64_t ncls, float4 **out) -> lm_status {
        const int64_t cnt = std::max<int64_t>(1, ncls) * np * np;
        lm_status s = lm_dalloc(t, out, cnt);
        if (s != LM_OK) return s;
        k_tab_df<<<gridn(cnt, 256), 256, 0, st>>>(tab, cnt, *out);
        return LM_OK;
    };
    auto conv_t = [&](const zd *tab, int64_t ncls, float4 **out) -> lm_status {
        const int64_t cnt = std::max<int64_t>(1, ncls) * np * np;
        lm_status s = lm_dalloc(t, out, cnt);
        if (s != LM_OK) return s;
        k_tab_df_t<<<gridn(cnt, 256), 256, 0, st>>>(tab, cnt, np, *out);
        return LM_OK;
    };
    for (Level &lv : t->lev) {
        if (lv.m2m) {
            lm_status s = conv(lv.m2m, 4, &lv.m2mdf); // 4 child positions
            if (s != LM_OK) return s;
        }
        if (lv.l2l) {
            lm_status s = conv(lv.l2l, 4, &lv.l2ldf);
            if (s != LM_OK) return s;
        }
    }
    if (t->adaptive) {
        lm_status s = conv(t->at.tab, (int64_t)t->at.cls_term.size(), &t->at.tabdf);
        if (s == LM_OK) s = conv_t(t->at.tab, (int64_t)t->at.cls_term.size(), &t->at.tabdft);
        if (s != LM_OK) return s;
        s = lm_dalloc(t, &t->at.Mdf, (size_t)t->at.nbox * np * LM_MAXV);
        if (s != LM_OK) return s;
    } else {
        for (Level &lv : t->lev) {
            lm_status s = conv(lv.tab, (int64_t)lv.cls_term.size(), &lv.tabdf);
            if (s == LM_OK) s = conv_t(lv.tab, (int64_t)lv.cls_term.size(), &lv.tabdft);
            if (s != LM_OK) return s;
            s = lm_dalloc(t, &lv.Mdf, (size_t)lv.nbox * np * LM_MAXV);
            if (s != LM_OK) return s;
        }
    }
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

// slots of the interface leaves (the blocks of k_pw_src64 / k_near_pw64) and their
// per-apply plane-wave coefficients (FP64 form with the factorised segment)
lm_status lm_setup_pwsrc(lm_tree_s *t, cudaStream_t st)
{
    if (!t->near_pw64) return LM_OK;
    std::vector<int32_t> idx;
    int64_t npw;
    if (t->adaptive) {
        idx.assign(t->at.nbox, -1);
        npw = (int64_t)t->at.hpw.size();
        for (int64_t i = 0; i < npw; ++i) idx[t->at.hpw[i]] = (int32_t)i;
    } else {
        const Level &lv = t->lev[t->L];
        idx.assign(lv.nbox, -1);
        npw = lv.nrow == 1 ? lv.ncol : 2 * lv.ncol;
        for (int64_t i = 0; i < npw; ++i) { // the block order of EdgeRowLeaves
            const int64_t row = (lv.nrow == 1 || i < lv.ncol) ? 0 : lv.nrow - 1;
            idx[row * lv.ncol + i % lv.ncol] = (int32_t)i;
        }
    }
    lm_status s = lm_dalloc(t, &t->pwidx, idx.size());
    if (s != LM_OK) return s;
    LM_CUDA(cudaMemcpyAsync(t->pwidx, idx.data(), idx.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
    LM_CUDA(cudaStreamSynchronize(st)); // idx is a host temporary
    return lm_dalloc(t, &t->pwC, (size_t)std::max<int64_t>(1, npw) * 2 * 2 * t->nq.nseg * LM_MAXV);
}
