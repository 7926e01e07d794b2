// lmfmm_mixed.cu -- the mixed-precision apply (Algorithm 1, steps 2-4):
// translation and quadrature tables are built in FP64 (densities sigma(lambda),
// branch points, contour nodes, large exponential factors) and rounded to
// FP32; expansions, the M2L contraction and the near field run in FP32 with
// FP32 accumulation.  Points are handled in leaf-local FP32 coordinates so
// that close pairs keep their relative accuracy.
#include <algorithm>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "mixed_near.cuh"

#define MX_MAXP 24
bool lm_mixed_order_supported(int P);
static int gridm(int64_t n, int b) { return (int)((n + b - 1) / b); }

LM_HD zf f2(zd a) { return zf{(float)a.re, (float)a.im}; }

// Box geometry of the FP32 kernels.  Grid32: leaf i of the uniform leaf lattice
// (ncol columns of width w); List32: box ids[i] of the adaptive tree, with
// centres and widths from its arrays.  offset(t, s) = centre_t - centre_s.
struct Grid32 {
    int64_t ncol;
    float w;
    __device__ int64_t id(int64_t i) const { return i; }
    __device__ float width(int64_t) const { return w; }
    __device__ void offset(int64_t bt, int64_t bs, float &ox, float &oy) const
    {
        const int rt = (int)(bt / ncol), ct = (int)(bt % ncol), rs = (int)(bs / ncol), cs = (int)(bs % ncol);
        ox = (float)(ct - cs) * w;
        oy = -(float)(rt - rs) * w;
    }
};
struct EdgeGrid32 : Grid32 { // the leaves of the top row, then (nrow > 1) of the bottom row
    int64_t nrow;
    __device__ int64_t id(int64_t i) const { return ((nrow == 1 || i < ncol) ? 0 : nrow - 1) * ncol + i % ncol; }
};
struct List32 {
    const int32_t *ids;
    const double *bx, *by, *bw;
    __device__ int64_t id(int64_t i) const { return ids[i]; }
    __device__ float width(int64_t b) const { return (float)bw[b]; }
    __device__ void offset(int64_t bt, int64_t bs, float &ox, float &oy) const
    {
        ox = (float)(bx[bt] - bx[bs]);
        oy = (float)(by[bt] - by[bs]);
    }
};
// parents and their four children: the lattice one level down, or the adaptive tree's links
struct GridKids32 {
    int64_t ncol;
    __device__ int64_t parent(int64_t i) const { return i; }
    __device__ int64_t child(int64_t b, int pos) const
    {
        const int64_t r = b / ncol, c = b % ncol;
        return (2 * r + (pos >> 1)) * (2 * ncol) + 2 * c + (pos & 1);
    }
};
struct ListKids32 {
    const int32_t *ids, *kids;
    __device__ int64_t parent(int64_t i) const { return ids[i]; }
    __device__ int64_t child(int64_t b, int pos) const { return kids[4 * b + pos]; }
};
// boxes of a level and their parents: the lattice one level up, or the adaptive tree's links
struct GridPar32 {
    int64_t ncol;
    __device__ int64_t box(int64_t i) const { return i; }
    __device__ int64_t parent(int64_t b) const { return (b / ncol / 2) * (ncol / 2) + (b % ncol) / 2; }
    __device__ int pos(int64_t b) const { return (int)(((b / ncol) & 1) * 2 + ((b % ncol) & 1)); }
};
struct ListPar32 {
    int64_t b0;
    const int32_t *par, *cpos;
    __device__ int64_t box(int64_t i) const { return b0 + i; }
    __device__ int64_t parent(int64_t b) const { return par[b]; }
    __device__ int pos(int64_t b) const { return cpos[b]; }
};

// ---------------------------------------------------------------------------
// setup
// ---------------------------------------------------------------------------
__global__ void k_d2f(const zd *a, zf *b, int64_t n)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) b[i] = f2(a[i]);
}

// leaf-local coordinates (FP64 difference, then rounded) and absolute y in FP32
__global__ void k_local_coords(int64_t ncol, double x0, double w, const int64_t *ls, const double *xs,
                               const double *ys, float *xl, float *yl, float *y32)
{
    int64_t b = blockIdx.x;
    int64_t r = b / ncol, c = b % ncol;
    double cx = x0 + (c + 0.5) * w, cy = -(r + 0.5) * w;
    for (int64_t i = ls[b] + threadIdx.x; i < ls[b + 1]; i += blockDim.x) {
        xl[i] = (float)(xs[i] - cx);
        yl[i] = (float)(ys[i] - cy);
        y32[i] = (float)ys[i];
    }
}

// entries of the V list that the free-space stencil kernel does not cover
__global__ void k_rest(int l, int64_t nbox, const int64_t *vstart, const int32_t *vsrc,
                       const int32_t *vslot, const int32_t *vterm, int64_t *rstart, int32_t *rsrc,
                       int32_t *rslot, int pass)
{
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nbox) return;
    int64_t pos = pass ? rstart[b] : 0, cnt = 0;
    for (int64_t e = vstart[b]; e < vstart[b + 1]; ++e) {
        if (l > 0 && vterm[e] == 0) continue;
        if (pass) {
            rsrc[pos] = vsrc[e];
            rslot[pos] = vslot[e];
            ++pos;
        }
        ++cnt;
    }
    if (!pass) rstart[b] = cnt;
}
__global__ void k_scan64b(int64_t *c, int64_t m)
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

static size_t near_pw_smem(const lm_tree_s *t);
__global__ void k_inverse_perm(const int64_t *perm, int64_t n, int64_t *iperm);
template <class G>
__global__ void __launch_bounds__(256) k_near_pw32(G geo, float d, const float *xl, const float *y32,
                                                   const int64_t *ls, const int64_t *ustart, const int32_t *usrc,
                                                   const int32_t *uterm, NearQuadF nq, const zf *qs, zf *us);

#define TRYM(x)                      \
    do {                             \
        lm_status s_ = (x);          \
        if (s_ != LM_OK) return s_;  \
    } while (0)

template <typename A, typename B>
static lm_status conv(lm_tree_s *t, const A *src, B **dst, int64_t n, cudaStream_t st)
{
    TRYM(lm_dalloc(t, dst, n));
    k_d2f<<<gridm(n, 256), 256, 0, st>>>(src, *dst, n);
    return LM_OK;
}

static lm_status setup_mixed_points(lm_tree_s *t, cudaStream_t st);
lm_status lm_setup_mixed(lm_tree_s *t, cudaStream_t st)
{
    const int L = t->L, P = t->p, np = 2 * P + 1;
    if (P > MX_MAXP || !lm_mixed_order_supported(P)) {
        lm_set_error("build_tree: the mixed-precision path supports p in {4,6,8..14,16,18,20,24}");
        return LM_ENOTSUP;
    }
    for (int l = 0; l <= L; ++l) {
        Level &lv = t->lev[l];
        int ncls = (int)lv.cls_term.size();
        TRYM(conv(t, lv.tab, &lv.tab32, (int64_t)std::max(1, ncls) * np * np, st));
        if (lv.m2m) TRYM(conv(t, lv.m2m, &lv.m2m32, 4 * np * np, st));
        if (lv.l2l) TRYM(conv(t, lv.l2l, &lv.l2l32, 4 * np * np, st));
        TRYM(lm_dalloc(t, &lv.M32, lv.nbox * np * LM_MAXV));
        TRYM(lm_dalloc(t, &lv.L32, lv.nbox * np * LM_MAXV));
        std::vector<int32_t> sten(49, -1);
        for (int i = 0; i < ncls; ++i)
            if (lv.cls_term[i] == 0 && abs(lv.cls_dc[i]) <= 3 && abs(lv.cls_dr[i]) <= 3)
                sten[(lv.cls_dc[i] + 3) * 7 + lv.cls_dr[i] + 3] = i;
        TRYM(lm_dalloc(t, &lv.stencil, 49));
        LM_CUDA(cudaMemcpyAsync(lv.stencil, sten.data(), 49 * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        TRYM(lm_dalloc(t, &lv.rstart, lv.nbox + 1));
        k_rest<<<gridm(lv.nbox, 128), 128, 0, st>>>(l, lv.nbox, lv.vstart, lv.vsrc, lv.vslot, lv.vterm,
                                                     lv.rstart, nullptr, nullptr, 0);
        k_scan64b<<<1, 1024, 0, st>>>(lv.rstart, lv.nbox);
        LM_CUDA(cudaMemcpyAsync(&lv.nrest, lv.rstart + lv.nbox, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        LM_CUDA(cudaStreamSynchronize(st));
        // the stencil kernel assumes every free-space offset of an interior box has a table
        if (l > 0)
            for (int dc = -3; dc <= 3; ++dc)
                for (int dr = -3; dr <= 3; ++dr)
                    if ((abs(dc) > 1 || abs(dr) > 1) && sten[(dc + 3) * 7 + dr + 3] < 0 && lv.ncol > 6 &&
                        lv.nrow > 6) {
                        lm_set_error("build_tree: free-space class (%d, %d) missing at level %d", dc, dr, l);
                        return LM_ECUDA;
                    }
        TRYM(lm_dalloc(t, &lv.rsrc, lv.nrest));
        TRYM(lm_dalloc(t, &lv.rslot, lv.nrest));
        k_rest<<<gridm(lv.nbox, 128), 128, 0, st>>>(l, lv.nbox, lv.vstart, lv.vsrc, lv.vslot, lv.vterm,
                                                     lv.rstart, lv.rsrc, lv.rslot, 1);
        {
            // targets that have entries on this list
            std::vector<int64_t> hs(lv.nbox + 1);
            LM_CUDA(cudaMemcpyAsync(hs.data(), lv.rstart, (lv.nbox + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
            LM_CUDA(cudaStreamSynchronize(st));
            std::vector<int32_t> tg;
            for (int64_t b2 = 0; b2 < lv.nbox; ++b2)
                if (hs[b2 + 1] > hs[b2]) tg.push_back((int32_t)b2);
            lv.nrtgt = (int64_t)tg.size();
            TRYM(lm_dalloc(t, &lv.rtgt, tg.size()));
            if (!tg.empty())
                LM_CUDA(cudaMemcpyAsync(lv.rtgt, tg.data(), tg.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        }
    }
    const int64_t n = t->n;
    TRYM(lm_dalloc(t, &t->xl32, n));
    TRYM(lm_dalloc(t, &t->yl32, n));
    TRYM(lm_dalloc(t, &t->y32, n));
    {
        Level &lv = t->lev[L];
        k_local_coords<<<(unsigned)lv.nbox, 64, 0, st>>>(lv.ncol, t->x0, lv.w, t->leaf_start, t->xs, t->ys,
                                                          t->xl32, t->yl32, t->y32);
    }
    TRYM(setup_mixed_points(t, st));
    if (t->med.opt.tensor_m2l) TRYM(lm_setup_tc(t, st));
    if (t->tc_ready) TRYM(lm_setup_tt(t, st));
    TRYM(lm_setup_leaf_tt(t, st));
    for (Level &lv : t->lev) lv.m2l_impl = t->tc_ready ? 0 : 4;
    LM_CUDA(cudaGetLastError());
    LM_CUDA(cudaStreamSynchronize(st));
    return LM_OK;
}

// tree-order point data of the mixed form that does not depend on the tree kind:
// the inverse permutation, FP32 density / potential scratch and the FP32 near-field
// quadrature tables (the leaf-local coordinates are written by the caller)
static lm_status setup_mixed_points(lm_tree_s *t, cudaStream_t st)
{
    const int64_t n = t->n;
    TRYM(lm_dalloc(t, &t->iperm, n));
    k_inverse_perm<<<gridm(n, 256), 256, 0, st>>>(t->perm, n, t->iperm);
    TRYM(lm_dalloc(t, &t->qs32, n * LM_MAXV));
    TRYM(lm_dalloc(t, &t->us32, n * LM_MAXV));
    NearQuad &q = t->nq;
    TRYM(conv(t, q.seg_lam, &t->nq_seg_lam, q.nseg, st));
    TRYM(conv(t, q.seg_s2, &t->nq_seg_s2, q.nseg, st));
    TRYM(conv(t, q.seg_w, &t->nq_seg_w, 2 * q.nseg, st));
    int64_t nt = (int64_t)q.nray * q.ntail;
    TRYM(conv(t, q.tail_lam, &t->nq_tail_lam, nt, st));
    TRYM(conv(t, q.tail_s2, &t->nq_tail_s2, nt, st));
    TRYM(conv(t, q.tail_w, &t->nq_tail_w, 4 * nt, st));
    size_t shm = near_pw_smem(t);
    if (shm > 200 * 1024) {
        lm_set_error("build_tree: near-field segment of %d nodes is too long for the factorised kernel", q.nseg);
        return LM_ENOTSUP;
    }
    LM_CUDA(lm_raise_smem((const void *)k_near_pw32<EdgeGrid32>, LM_SMEM_NEAR_PW, (int)shm));
    LM_CUDA(lm_raise_smem((const void *)k_near_pw32<List32>, LM_SMEM_NEAR_PW_A, (int)shm));
    return LM_OK;
}

// leaf-local coordinates of the adaptive tree's leaves (box centres from its arrays)
__global__ void k_local_coords_list(const int32_t *leaves, const double *bx, const double *by, const int64_t *ls,
                                    const double *xs, const double *ys, float *xl, float *yl, float *y32)
{
    const int64_t b = leaves[blockIdx.x];
    const double cx = bx[b], cy = by[b];
    for (int64_t i = ls[b] + threadIdx.x; i < ls[b + 1]; i += blockDim.x) {
        xl[i] = (float)(xs[i] - cx);
        yl[i] = (float)(ys[i] - cy);
        y32[i] = (float)ys[i];
    }
}

// Mixed form of the adaptive tree (Algorithm 1 step 1, reading G14): FP32 copies of
// the cross-level M2L tables and of each level's M2M / L2L tables, FP32 expansions
// of every box, per level the boxes that have V entries, and the leaf-local points.
// The M2L runs on the staged CUDA-core contraction over the V list (any two levels);
// the leaf, S2M, M2M, L2L and segment kernels take the box lists as their geometry.
lm_status lm_setup_mixed_adaptive(lm_tree_s *t, cudaStream_t st)
{
    AdaptTree &A = t->at;
    const int L = t->L, P = t->p, np = 2 * P + 1;
    if (P > MX_MAXP || !lm_mixed_order_supported(P)) {
        lm_set_error("build_tree: the mixed-precision path supports p in {4,6,8..14,16,18,20,24}");
        return LM_ENOTSUP;
    }
    const int64_t ncls = (int64_t)A.cls_term.size();
    TRYM(conv(t, A.tab, &A.tab32, std::max<int64_t>(1, ncls) * np * np, st));
    for (int l = 0; l <= L; ++l) {
        Level &lv = t->lev[l];
        if (lv.m2m) TRYM(conv(t, lv.m2m, &lv.m2m32, 4 * np * np, st));
        if (lv.l2l) TRYM(conv(t, lv.l2l, &lv.l2l32, 4 * np * np, st));
    }
    TRYM(lm_dalloc(t, &A.M32, (size_t)A.nbox * np * LM_MAXV));
    TRYM(lm_dalloc(t, &A.L32, (size_t)A.nbox * np * LM_MAXV));
    {
        std::vector<int64_t> hs(A.nbox + 1);
        LM_CUDA(cudaMemcpyAsync(hs.data(), A.vstart, (A.nbox + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        LM_CUDA(cudaStreamSynchronize(st));
        A.m2l_tgt.assign(L + 1, nullptr);
        A.m2l_ntgt.assign(L + 1, 0);
        for (int l = 0; l <= L; ++l) {
            std::vector<int32_t> tg;
            for (int64_t b = A.lev_start[l]; b < A.lev_start[l + 1]; ++b)
                if (hs[b + 1] > hs[b]) tg.push_back((int32_t)b);
            A.m2l_ntgt[l] = (int64_t)tg.size();
            TRYM(lm_dalloc(t, &A.m2l_tgt[l], tg.size()));
            if (!tg.empty())
                LM_CUDA(cudaMemcpyAsync(A.m2l_tgt[l], tg.data(), tg.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                        st));
            LM_CUDA(cudaStreamSynchronize(st));
        }
    }
    const int64_t n = t->n;
    TRYM(lm_dalloc(t, &t->xl32, n));
    TRYM(lm_dalloc(t, &t->yl32, n));
    TRYM(lm_dalloc(t, &t->y32, n));
    if (A.nleaf > 0)
        k_local_coords_list<<<(unsigned)A.nleaf, 64, 0, st>>>(A.leaves, A.cx, A.cy, t->leaf_start, t->xs, t->ys,
                                                              t->xl32, t->yl32, t->y32);
    TRYM(setup_mixed_points(t, st));
    LM_CUDA(cudaGetLastError());
    LM_CUDA(cudaStreamSynchronize(st));
    return LM_OK;
}

void lm_free_mixed(lm_tree_s *t)
{
    lm_free_tt(t);
    lm_free_leaf_tt(t);
    {
        AdaptTree &A = t->at;
        void *ap[] = {A.tab32, A.M32, A.L32};
        for (void *p : ap)
            if (p) cudaFree(p);
        for (int32_t *p : A.m2l_tgt)
            if (p) cudaFree(p);
    }
    void *ptrs[] = {t->xl32, t->yl32, t->y32, t->qs32, t->us32, t->iperm, t->nq_seg_lam, t->nq_seg_s2, t->nq_seg_w,
                    t->nq_tail_lam, t->nq_tail_s2, t->nq_tail_w};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (Level &lv : t->lev) {
        void *lp[] = {lv.tab32, lv.m2m32, lv.l2l32, lv.M32, lv.L32, lv.stencil, lv.rstart, lv.rsrc, lv.rslot,
                      lv.rtgt};
        for (void *p : lp)
            if (p) cudaFree(p);
    }
}

// ---------------------------------------------------------------------------
// apply kernels (FP32)
// ---------------------------------------------------------------------------
// input order -> tree order: one thread per input point, coalesced reads of
// q[v][j], one 128-byte row written at the point's tree position
template <typename TIO>
__global__ void k_permute_in32(const TIO *q, const int64_t *iperm, int64_t n, int nvec, int conjugate, zf *qs,
                               uint32_t *qmax)
{
    __shared__ uint32_t red[32];
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    uint32_t m = 0;
    if (j < n) {
        const int64_t i = iperm[j];
        zf a[LM_MAXV];
#pragma unroll
        for (int v = 0; v < LM_MAXV; ++v) {
            a[v] = zf{0.f, 0.f};
            if (v < nvec) {
                const TIO b = q[(int64_t)v * n + j];
                a[v] = zf{(float)b.re, (float)(conjugate ? -b.im : b.im)};
            }
        }
        float4 *o = (float4 *)(qs + i * LM_MAXV);
#pragma unroll
        for (int v2 = 0; v2 < LM_MAXV / 2; ++v2)
            o[v2] = make_float4(a[2 * v2].re, a[2 * v2].im, a[2 * v2 + 1].re, a[2 * v2 + 1].im);
#pragma unroll
        for (int v = 0; v < LM_MAXV; ++v)
            m = max(m, max(__float_as_uint(a[v].re) & 0x7fffffffu, __float_as_uint(a[v].im) & 0x7fffffffu));
    }
    if (qmax) { // largest |component| of the densities (as bits of a non-negative float): one atomic per block
        m = __reduce_max_sync(0xffffffffu, m);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t mm = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = max(mm, red[w]);
            if (mm) atomicMax(qmax, mm);
        }
    }
}
// tree order -> input order: one thread per input point, one 128-byte row
// read at its tree position, coalesced writes of u[v][j]
template <typename TIO>
__global__ void k_permute_out32(const zf *us, const int64_t *iperm, int64_t n, int nvec, int conjugate, TIO *u)
{
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t i = iperm[j];
    const float4 *src = (const float4 *)(us + i * LM_MAXV);
    float4 a[LM_MAXV / 2];
#pragma unroll
    for (int v2 = 0; v2 < LM_MAXV / 2; ++v2) a[v2] = src[v2];
#pragma unroll
    for (int v = 0; v < LM_MAXV; ++v) {
        if (v < nvec) {
            const float4 t = a[v / 2];
            const float re = (v & 1) ? t.z : t.x, im = (v & 1) ? t.w : t.y;
            TIO b;
            b.re = re;
            b.im = conjugate ? -im : im;
            u[(int64_t)v * n + j] = b;
        }
    }
}
__global__ void k_inverse_perm(const int64_t *perm, int64_t n, int64_t *iperm)
{
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) iperm[perm[i]] = i;
}

// S2M in FP32 (Eq. (multipole_coef), scaled): one block per leaf
#define P2M32_CHUNK 32
template <class G>
__global__ void k_p2m32(G geo, int P, float k, const float *xl, const float *yl, const int64_t *ls,
                        const zf *qs, int nvs, zf *M)
{
    extern __shared__ unsigned char smem[];
    const int np = 2 * P + 1;
    zf *B = (zf *)smem;                        // [P2M32_CHUNK][np]
    zf *Q = B + P2M32_CHUNK * np;              // [P2M32_CHUNK][LM_MAXV]
    const int64_t b = geo.id(blockIdx.x);
    const int64_t lo = ls[b], hi = ls[b + 1];
    const float sc = k * geo.width(b);
    const int nent = np * nvs; // (order, vector) entries computed; M keeps 16 vector slots
    zf acc[8];
    for (int e = 0; e < 8; ++e) acc[e] = zf{0.f, 0.f};
    for (int64_t base = lo; base < hi; base += P2M32_CHUNK) {
        __syncthreads();
        int j = threadIdx.x;
        if (j < P2M32_CHUNK) {
            int64_t i = base + j;
            zf *row = B + j * np + P;
            if (i < hi) {
                float rx = xl[i], ry = yl[i], r = sqrtf(rx * rx + ry * ry);
                float J[MX_MAXP + 1];
                bessel_j_scaled<float>(P, k * r, sc, J);
                zf z = r > 0.f ? zf{rx / r, -ry / r} : zf{1.f, 0.f};
                zf zp = {1.f, 0.f};
                row[0] = zf{J[0], 0.f};
                for (int m = 1; m <= P; ++m) {
                    zp = zp * z;
                    row[m] = J[m] * zp;
                    float s = (m & 1) ? -J[m] : J[m];
                    row[-m] = s * conj(zp);
                }
            } else {
                for (int m = -P; m <= P; ++m) row[m] = zf{0.f, 0.f};
            }
        }
        for (int e = threadIdx.x; e < P2M32_CHUNK * LM_MAXV; e += blockDim.x) {
            int jj = e / LM_MAXV;
            int64_t i = base + jj;
            Q[e] = i < hi ? qs[i * LM_MAXV + e % LM_MAXV] : zf{0.f, 0.f};
        }
        __syncthreads();
        int cnt = (int)min((int64_t)P2M32_CHUNK, hi - base);
        for (int e = 0; e < 8; ++e) {
            int idx = threadIdx.x + e * blockDim.x;
            if (idx >= nent) break;
            int qi = idx / nvs, v = idx % nvs;
            zf s = acc[e];
            for (int jj = 0; jj < cnt; ++jj) cfmaf(s, B[jj * np + qi], Q[jj * LM_MAXV + v]);
            acc[e] = s;
        }
    }
    for (int e = 0; e < 8; ++e) {
        int idx = threadIdx.x + e * blockDim.x;
        if (idx >= nent) break;
        M[(b * np + idx / nvs) * LM_MAXV + idx % nvs] = acc[e];
    }
}

// S2M of the 16 vector slots (Eq. (multipole_coef), scaled) on the leaves of a
// uniform tree with k w <= 2: one warp per leaf, no recurrence.  Lane j forms
// the basis row of point j of a chunk of 32 from the ascending series of the
// scaled Bessel function (A&S 9.1.10 by Horner's rule to 8 terms; points lie
// within w/sqrt(2) of the centre, so t = (k r / 2)^2 <= 1/2 and the first
// dropped term is below 2e-14).  The lanes then own 2 orders x 4 vectors each.
// Orders m and -m share their products: with b = a + i c the basis value of
// order m >= 0 and q = x + i y a density, b q and conj(b) q follow from the
// four sums of a x, c y, a y and c x, and the basis of order -m is
// (-1)^m conj(b).
#define S2M16_NB 16 // orders 0 .. 15 per basis row (P <= 15)
#define S2M16_RS 18 // basis row stride in complex entries (144 bytes: 16-byte aligned rows)
template <int P>
__global__ void __launch_bounds__(128) k_s2m16(int64_t nbox, float w, float k, const float *xl, const float *yl,
                                               const int64_t *ls, const zf *qs, zf *M)
{
    static_assert(P < S2M16_NB, "basis rows hold orders 0 .. 15");
    constexpr int NP = 2 * P + 1;
    __shared__ __align__(16) zf Bs[4][32 * S2M16_RS];
    __shared__ __align__(16) float4 Qs[4][32 * LM_MAXV / 2];
    const int wp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t b = blockIdx.x * 4LL + wp;
    if (b >= nbox) return; // the warps of a block share no barrier
    const int64_t lo = ls[b], hi = ls[b + 1];
    const int og = lane >> 2, vg = lane & 3; // orders 2 og, 2 og + 1; vectors 4 vg .. 4 vg + 3
    zf *B = Bs[wp];
    float4 *Q = Qs[wp];
    const float iw = 1.0f / w, hk2 = 0.25f * k * k;
    float acc[2][4][4];
#pragma unroll
    for (int o = 0; o < 2; ++o)
#pragma unroll
        for (int v = 0; v < 4; ++v)
#pragma unroll
            for (int s = 0; s < 4; ++s) acc[o][v][s] = 0.f;
    for (int64_t base = lo; base < hi; base += 32) {
        const int cnt = (int)min((int64_t)32, hi - base);
        __syncwarp();
        {
            zf *row = B + lane * S2M16_RS;
            float rx = 0.f, ry = 0.f;
            if (lane < cnt) {
                rx = xl[base + lane];
                ry = yl[base + lane];
            }
            const float t = hk2 * fmaf(rx, rx, ry * ry);
            const zf z = {rx * iw, -ry * iw};
            zf pw = {lane < cnt ? 1.0f : 0.0f, 0.f};
#pragma unroll
            for (int m = 0; m < S2M16_NB; ++m) {
                if (m <= P) {
                    float sv = 1.0f;
#pragma unroll
                    for (int q = 8; q >= 1; --q) sv = fmaf(-t * (1.0f / (float)(q * (q + m))), sv, 1.0f);
                    row[m] = sv * pw;
                    pw = pw * z;
                } else {
                    row[m] = zf{0.f, 0.f};
                }
            }
        }
        const float4 *src = (const float4 *)(qs + base * LM_MAXV);
#pragma unroll
        for (int r = 0; r < LM_MAXV / 2; ++r) {
            const int e = lane + 32 * r;
            Q[e] = (e / (LM_MAXV / 2)) < cnt ? src[e] : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncwarp();
        for (int p = 0; p < cnt; ++p) {
            const float4 bb = *(const float4 *)(B + p * S2M16_RS + 2 * og);
            const float4 q0 = Q[p * (LM_MAXV / 2) + 2 * vg], q1 = Q[p * (LM_MAXV / 2) + 2 * vg + 1];
            const float br[2] = {bb.x, bb.z}, bi[2] = {bb.y, bb.w};
            const float qr[4] = {q0.x, q0.z, q1.x, q1.z}, qi[4] = {q0.y, q0.w, q1.y, q1.w};
#pragma unroll
            for (int o = 0; o < 2; ++o)
#pragma unroll
                for (int v = 0; v < 4; ++v) {
                    acc[o][v][0] = fmaf(br[o], qr[v], acc[o][v][0]);
                    acc[o][v][1] = fmaf(bi[o], qi[v], acc[o][v][1]);
                    acc[o][v][2] = fmaf(br[o], qi[v], acc[o][v][2]);
                    acc[o][v][3] = fmaf(bi[o], qr[v], acc[o][v][3]);
                }
        }
    }
#pragma unroll
    for (int o = 0; o < 2; ++o) {
        const int m = 2 * og + o;
        if (m > P) continue;
        float4 pos[2], neg[2];
        const float sg = (m & 1) ? -1.0f : 1.0f;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const float *a0 = acc[o][2 * h], *a1 = acc[o][2 * h + 1];
            pos[h] = make_float4(a0[0] - a0[1], a0[2] + a0[3], a1[0] - a1[1], a1[2] + a1[3]);
            neg[h] = make_float4(sg * (a0[0] + a0[1]), sg * (a0[2] - a0[3]), sg * (a1[0] + a1[1]),
                                 sg * (a1[2] - a1[3]));
        }
        float4 *dp = (float4 *)(M + (b * NP + P + m) * LM_MAXV + 4 * vg);
        dp[0] = pos[0];
        dp[1] = pos[1];
        if (m > 0) {
            float4 *dn = (float4 *)(M + (b * NP + P - m) * LM_MAXV + 4 * vg);
            dn[0] = neg[0];
            dn[1] = neg[1];
        }
    }
}

// the series S2M on the leaf level (16 vector slots, P <= 15, k w <= 2)
template <int P>
static void launch_s2m16(const Level &lv, float k, const lm_tree_s *t, cudaStream_t st)
{
    if constexpr (P < S2M16_NB)
        k_s2m16<P><<<(unsigned)((lv.nbox + 3) / 4), 128, 0, st>>>(lv.nbox, (float)lv.w, k, t->xl32, t->yl32,
                                                                  t->leaf_start, t->qs32, lv.M32);
}
static bool s2m16_ok(const lm_tree_s *t, int nvs)
{
    return nvs == LM_MAXV && t->p < S2M16_NB && (double)(float)t->med.k2 * t->lev[t->L].w <= 2.0;
}

// Free-space M2L over the fixed 27-offset stencil of the V list (levels >= 1).
// Boxes of one parity class share their offsets.  A block takes 16 boxes of
// one class; its threads form (row group of 4 orders) x (box, 4 vectors)
// tiles, so each staged translation entry feeds 4 columns and each source
// multipole quad feeds 4 orders.  Offset by offset the matrix is staged in
// shared memory (transposed: warp-uniform broadcast reads) and the gathered
// source multipoles stream from L2 as 32-byte vector loads.  Each offset's
// contraction accumulates in fresh registers before joining the sum.
// RG (orders per thread, hence the block's row tiling) is the tile shape the
// autotuner chooses among, together with the tensor-core kernel.
template <int NP, int RG>
__global__ void __launch_bounds__(64 * ((NP + RG - 1) / RG))
    k_m2l_stencil32(int64_t ncol, int64_t nrow, const int32_t *stencil, const zf *tab, const zf *M, zf *Lc)
{
    __shared__ zf At[NP * NP]; // At[q][p]
    const int cls = blockIdx.y;
    const int pc = cls & 1, pr = cls >> 1;
    const int64_t hc = ncol / 2, hr = nrow / 2;
    const int rg = threadIdx.x >> 6, cg = threadIdx.x & 63;
    const int lb = cg >> 2, vq = (cg & 3) * 4;
    const int64_t cidx = (int64_t)blockIdx.x * 16 + lb;
    const bool active = cidx < hc * hr;
    const int64_t c = 2 * (active ? cidx % hc : 0) + pc, r = 2 * (active ? cidx / hc : 0) + pr;
    const int p0 = rg * RG;
    zf acc[RG][4];
#pragma unroll
    for (int i = 0; i < RG; ++i)
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[i][u] = zf{0.f, 0.f};
    for (int dc = pc - 3; dc <= pc + 2; ++dc)
        for (int dr = pr - 3; dr <= pr + 2; ++dr) {
            if (dc >= -1 && dc <= 1 && dr >= -1 && dr <= 1) continue;
            const int slot = stencil[(dc + 3) * 7 + dr + 3];
            if (slot < 0) continue; // offset beyond the grid at this level
            __syncthreads();
            const zf *T = tab + (int64_t)slot * NP * NP;
            for (int e = threadIdx.x; e < NP * NP; e += blockDim.x) {
                int p = e / NP, q = e % NP;
                At[q * NP + p] = T[e];
            }
            __syncthreads();
            const int64_t cs = c - dc, rs = r - dr;
            if (!active || cs < 0 || cs >= ncol || rs < 0 || rs >= nrow) continue;
            const zf *m = M + (rs * ncol + cs) * NP * LM_MAXV + vq;
            zf tmp[RG][4];
#pragma unroll
            for (int i = 0; i < RG; ++i)
#pragma unroll
                for (int u = 0; u < 4; ++u) tmp[i][u] = zf{0.f, 0.f};
#pragma unroll 2
            for (int q = 0; q < NP; ++q) {
                const float4 m01 = *(const float4 *)(m + q * LM_MAXV);
                const float4 m23 = *(const float4 *)(m + q * LM_MAXV + 2);
                const zf mv[4] = {{m01.x, m01.y}, {m01.z, m01.w}, {m23.x, m23.y}, {m23.z, m23.w}};
                const zf *a = At + q * NP + p0;
#pragma unroll
                for (int i = 0; i < RG; ++i) {
                    if (p0 + i < NP) {
                        const zf ai = a[i];
#pragma unroll
                        for (int u = 0; u < 4; ++u) cfmaf(tmp[i][u], ai, mv[u]);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < RG; ++i)
#pragma unroll
                for (int u = 0; u < 4; ++u) acc[i][u] = acc[i][u] + tmp[i][u];
        }
    if (!active) return;
    zf *out = Lc + (r * ncol + c) * NP * LM_MAXV + vq;
#pragma unroll
    for (int i = 0; i < RG; ++i) {
        if (p0 + i >= NP) break;
        float4 *o = (float4 *)(out + (p0 + i) * LM_MAXV);
        float4 x0 = o[0], x1 = o[1];
        o[0] = make_float4(x0.x + acc[i][0].re, x0.y + acc[i][0].im, x0.z + acc[i][1].re, x0.w + acc[i][1].im);
        o[1] = make_float4(x1.x + acc[i][2].re, x1.y + acc[i][2].im, x1.z + acc[i][3].re, x1.w + acc[i][3].im);
    }
}

// terms of the J0/Y0 series needed for arguments up to xmax (truncation < 1e-9)
int lm_h0_terms(double xmax)
{
    if (xmax > 2.0) return 11;
    double t = 0.25 * xmax * xmax, a = 1.0;
    for (int m = 1; m <= 11; ++m) {
        a *= t / ((double)m * m);
        if (a * 3.1 < 1e-9) return m;
    }
    return 11;
}

// Segment part of the reflected direct terms, factorised per target leaf.
// On the fixed deformed segment the integrand of a pair separates,
//   2 cos(lambda (x_i - x_j)) e^{-s2 h_ij} = sum_{s=+-1} e^{s i lambda (x_i - x_T)} E(y_i) e^{-s i lambda (x_j - x_T)} E(y_j),
// E(y) = e^{s2 y} (tt) or e^{-s2 (y + d)} (bb), x_T the target leaf centre; so
// each leaf first sums its near sources into plane-wave coefficients
// B_{n,s} (phase A) and then evaluates them at its targets (phase B).
// One block per leaf in the top or bottom row; adds into us.
#define PW_SRC 128
template <class G>
__global__ void __launch_bounds__(256) k_near_pw32(G geo, float d, const float *xl,
                                                   const float *y32, const int64_t *ls, const int64_t *ustart,
                                                   const int32_t *usrc, const int32_t *uterm, NearQuadF nq,
                                                   const zf *qs, zf *us)
{
    extern __shared__ unsigned char smem[];
    const int nk = 2 * nq.nseg;
    zf *B = (zf *)smem;                         // [nk][LM_MAXV]
    zf *SQ = B + (size_t)nk * LM_MAXV;          // [PW_SRC][LM_MAXV]
    float *SX = (float *)(SQ + PW_SRC * LM_MAXV); // [PW_SRC]
    float *SY = SX + PW_SRC;                    // [PW_SRC]
    const int64_t b = geo.id(blockIdx.x);
    for (int term = 1; term <= 2; ++term) {
        bool any = false;
        for (int64_t e = ustart[b]; e < ustart[b + 1]; ++e) any |= (uterm[e] == term);
        if (!any) continue;
        const int m = term - 1;
        const zf *W = nq.seg_w + (int64_t)m * nq.nseg;
        for (int k = threadIdx.x; k < nk * LM_MAXV; k += blockDim.x) B[k] = zf{0.f, 0.f};
        // phase A: B_{n,s}[v] = sum_j q_j[v] e^{-s i lambda_n (x_j - x_T)} E_n(y_j), per source leaf
        for (int64_t e = ustart[b]; e < ustart[b + 1]; ++e) {
            if (uterm[e] != term) continue;
            const int64_t s = usrc[e];
            float ox, oy;
            geo.offset(s, b, ox, oy); // centre_s - centre_T
            for (int64_t j0 = ls[s]; j0 < ls[s + 1]; j0 += PW_SRC) {
                const int cnt = (int)min((int64_t)PW_SRC, ls[s + 1] - j0);
                __syncthreads();
                for (int t = threadIdx.x; t < cnt * LM_MAXV; t += blockDim.x) SQ[t] = qs[(j0 + t / LM_MAXV) * LM_MAXV + t % LM_MAXV];
                for (int t = threadIdx.x; t < cnt; t += blockDim.x) {
                    SX[t] = xl[j0 + t] + ox;
                    SY[t] = y32[j0 + t];
                }
                __syncthreads();
                for (int k = threadIdx.x; k < nk; k += blockDim.x) {
                    const zf lam = nq.seg_lam[k >> 1], s2 = nq.seg_s2[k >> 1];
                    const float sg = (k & 1) ? -1.f : 1.f;
                    zf part[LM_MAXV];
#pragma unroll
                    for (int v = 0; v < LM_MAXV; ++v) part[v] = zf{0.f, 0.f};
                    for (int t = 0; t < cnt; ++t) {
                        const float x = SX[t], y = SY[t];
                        float er = sg * lam.im * x, ei = -sg * lam.re * x;
                        if (m == 0) {
                            er += s2.re * y;
                            ei += s2.im * y;
                        } else {
                            er -= s2.re * (y + d);
                            ei -= s2.im * (y + d);
                        }
                        const float a = expf(er);
                        float sn, cs;
                        sincosf(ei, &sn, &cs);
                        const zf f = {a * cs, a * sn};
#pragma unroll
                        for (int v = 0; v < LM_MAXV; ++v) cfmaf(part[v], f, SQ[t * LM_MAXV + v]);
                    }
#pragma unroll
                    for (int v = 0; v < LM_MAXV; ++v) B[k * LM_MAXV + v] = B[k * LM_MAXV + v] + part[v];
                }
            }
        }
        __syncthreads();
        // phase B: u_i[v] += sum_{n,s} W_n e^{s i lambda_n (x_i - x_T)} E_n(y_i) B_{n,s}[v]
        const int64_t lo = ls[b], cntT = ls[b + 1] - lo;
        for (int64_t t = threadIdx.x; t < cntT * 4; t += blockDim.x) {
            const int64_t i = lo + t / 4;
            const int vq = (int)(t % 4) * 4;
            const float x = xl[i], y = y32[i];
            zf acc[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
            for (int k0 = 0; k0 < nk; k0 += 20) {
                zf part[4] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
                const int k1 = min(nk, k0 + 20);
                for (int k = k0; k < k1; ++k) {
                    const zf lam = nq.seg_lam[k >> 1], s2 = nq.seg_s2[k >> 1];
                    const float sg = (k & 1) ? -1.f : 1.f;
                    float er = -sg * lam.im * x, ei = sg * lam.re * x;
                    if (m == 0) {
                        er += s2.re * y;
                        ei += s2.im * y;
                    } else {
                        er -= s2.re * (y + d);
                        ei -= s2.im * (y + d);
                    }
                    const float a = expf(er);
                    float sn, cs;
                    sincosf(ei, &sn, &cs);
                    const zf g = zf{a * cs, a * sn} * W[k >> 1];
#pragma unroll
                    for (int v = 0; v < 4; ++v) cfmaf(part[v], g, B[k * LM_MAXV + vq + v]);
                }
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[v] = acc[v] + part[v];
            }
#pragma unroll
            for (int v = 0; v < 4; ++v) {
                zf o = us[i * LM_MAXV + vq + v];
                us[i * LM_MAXV + vq + v] = o + acc[v];
            }
        }
        __syncthreads();
    }
}

// Step 4 in FP32: L2T and S2T for every target of a leaf, one thread per
// target holding all 16 vectors.  The source leaves of the U list are
// streamed through shared memory in chunks of up to 64 points with
// double-buffered cp.async (coordinates and the 128-byte density rows), so
// the inner loop reads broadcast shared-memory rows while the next chunk
// is in flight.
#define LCAP 64
// ---------------------------------------------------------------------------
// Staged contraction of one output box: acc = sum over its entries e of
// T[slot(e)] M[src(e)], each (NP x NP) x (NP x 16 vectors).  Each entry's table
// and source coefficients are staged in shared memory with the next entry's
// copies in flight (double-buffered cp.async).  Thread (v, g) of 128 owns
// vector v and rows g, g + 8, g + 16, ...; each entry's sum is formed on its
// own before it is added (blocked FP32 accumulation).  Used by the rest-list
// M2L, M2M (4 child entries) and L2L (1 parent entry).
// ---------------------------------------------------------------------------
// NVS: vector slots computed (16, or 4 for the batched form's 4-vector applies);
// thread (v, g) of 128 owns vector v < NVS and rows g, g + NG, g + 2 NG, ...
template <int NP, int NVS = LM_MAXV>
struct Staged {
    static constexpr int NG = 128 / NVS; // row groups
    static constexpr int NR = (NP + NG - 1) / NG;
    // two buffers while they fit the 48 KB of static shared memory (all orders but p = 24)
    static constexpr int NB = 2 * (NP * NP + NP * LM_MAXV) * 8 <= 48 * 1024 ? 2 : 1;
};
template <int NP, int NVS, class EntryF>
__device__ __forceinline__ void staged_contract(int ne, EntryF entry, const zf *tab, const zf *M,
                                                zf (&acc)[Staged<NP, NVS>::NR], zf (*Ts)[NP * NP],
                                                zf (*Ms)[NP * LM_MAXV])
{
    constexpr int NR = Staged<NP, NVS>::NR, NB = Staged<NP, NVS>::NB, NG = Staged<NP, NVS>::NG;
    const int v = threadIdx.x & (NVS - 1), g = threadIdx.x / NVS;
    auto stage = [&](int e, int buf) {
        int slot;
        int64_t src;
        entry(e, &slot, &src);
        // table slots are NP*NP*8 bytes apart (8-byte aligned); coefficient rows are 16-byte aligned
        const zf *T = tab + (int64_t)slot * NP * NP;
        for (int i = threadIdx.x; i < NP * NP; i += blockDim.x) cp_async8(&Ts[buf][i], T + i);
        const zf *Mm = M + src * NP * LM_MAXV;
        for (int i = threadIdx.x; i < NP * NVS / 2; i += blockDim.x) {
            const int q = i / (NVS / 2), o = q * LM_MAXV + 2 * (i % (NVS / 2));
            cp_async16(&Ms[buf][o], Mm + o);
        }
    };
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = zf{0.f, 0.f};
    if (NB == 2 && ne > 0) {
        stage(0, 0);
        cp_commit();
    }
    for (int e = 0; e < ne; ++e) {
        const int buf = NB == 2 ? (e & 1) : 0;
        if (NB == 1) {
            stage(e, 0);
            cp_commit();
            cp_wait<0>();
        } else if (e + 1 < ne) {
            stage(e + 1, buf ^ 1);
            cp_commit();
            cp_wait<1>();
        } else {
            cp_wait<0>();
        }
        __syncthreads();
        zf tmp[NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) tmp[r] = zf{0.f, 0.f};
        const zf *Tb = Ts[buf];
        const zf *Mb = Ms[buf] + v;
#pragma unroll 4
        for (int q = 0; q < NP; ++q) {
            const zf m = Mb[q * LM_MAXV];
#pragma unroll
            for (int r = 0; r < NR; ++r) {
                const int p = g + NG * r;
                if (p < NP) cfmaf(tmp[r], Tb[p * NP + q], m);
            }
        }
#pragma unroll
        for (int r = 0; r < NR; ++r) acc[r] = acc[r] + tmp[r];
        __syncthreads(); // buffer `buf` is refilled by the stage of entry e + NB
    }
}

// Remaining V-list entries (level 0 and the image terms): one block per target
// box with such entries; adds into L
template <int NP, int NVS>
__global__ void __launch_bounds__(128) k_m2l_rest32(const int32_t *rtgt, const int64_t *rstart,
                                                    const int32_t *rsrc, const int32_t *rslot, const zf *tab,
                                                    const zf *M, zf *Lc)
{
    constexpr int NR = Staged<NP, NVS>::NR, NB = Staged<NP, NVS>::NB, NG = Staged<NP, NVS>::NG;
    __shared__ __align__(16) zf Ts[NB][NP * NP];
    __shared__ __align__(16) zf Ms[NB][NP * LM_MAXV];
    const int64_t b = rtgt[blockIdx.x];
    const int64_t e0 = rstart[b];
    auto entry = [&](int e, int *slot, int64_t *src) {
        *slot = rslot[e0 + e];
        *src = rsrc[e0 + e];
    };
    zf acc[NR];
    staged_contract<NP, NVS>((int)(rstart[b + 1] - e0), entry, tab, M, acc, Ts, Ms);
    const int v = threadIdx.x & (NVS - 1), g = threadIdx.x / NVS;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        const int p = g + NG * r;
        if (p < NP) {
            zf *o = Lc + (b * NP + p) * LM_MAXV + v;
            *o = *o + acc[r];
        }
    }
}

// M2M (Lemma M2M): a parent (this level) from its four children (level l + 1),
// table slot = child position (dy, dx); writes the parent's coefficients
template <int NP, int NVS, class K = GridKids32>
__global__ void __launch_bounds__(128) k_m2m32(K kids, const zf *tabs, const zf *Mc, zf *Mp)
{
    constexpr int NR = Staged<NP, NVS>::NR, NB = Staged<NP, NVS>::NB, NG = Staged<NP, NVS>::NG;
    __shared__ __align__(16) zf Ts[NB][NP * NP];
    __shared__ __align__(16) zf Ms[NB][NP * LM_MAXV];
    const int64_t b = kids.parent(blockIdx.x);
    auto entry = [&](int pos, int *slot, int64_t *src) {
        *slot = pos;
        *src = kids.child(b, pos);
    };
    zf acc[NR];
    staged_contract<NP, NVS>(4, entry, tabs, Mc, acc, Ts, Ms);
    const int v = threadIdx.x & (NVS - 1), g = threadIdx.x / NVS;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int p = g + NG * k;
        if (p < NP) Mp[(b * NP + p) * LM_MAXV + v] = acc[k];
    }
}

// L2L (Lemma L2L): a child (this level) from its parent (level l - 1), table
// slot = the child's position in the parent; writes the child's coefficients,
// or adds them (ACC) where the level's M2L has already written them
template <int NP, int NVS, bool ACC = false, class K = GridPar32>
__global__ void __launch_bounds__(128) k_l2l32(K par, const zf *tabs, const zf *Lp, zf *Lc, uint32_t *lmax)
{
    constexpr int NR = Staged<NP, NVS>::NR, NB = Staged<NP, NVS>::NB, NG = Staged<NP, NVS>::NG;
    __shared__ __align__(16) zf Ts[NB][NP * NP];
    __shared__ __align__(16) zf Ms[NB][NP * LM_MAXV];
    const int64_t b = par.box(blockIdx.x);
    auto entry = [&](int, int *slot, int64_t *src) {
        *slot = par.pos(b);
        *src = par.parent(b);
    };
    zf acc[NR];
    staged_contract<NP, NVS>(1, entry, tabs, Lp, acc, Ts, Ms);
    const int v = threadIdx.x & (NVS - 1), g = threadIdx.x / NVS;
    uint32_t m = 0;
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        const int p = g + NG * k;
        if (p < NP) {
            zf *o = Lc + (b * NP + p) * LM_MAXV + v;
            const zf r = ACC ? *o + acc[k] : acc[k];
            *o = r;
            m = max(m, max(__float_as_uint(r.re) & 0x7fffffffu, __float_as_uint(r.im) & 0x7fffffffu));
        }
    }
    if (lmax) { // largest |component| of the local expansions written (bits of a non-negative float)
        __shared__ uint32_t red[4];
        m = __reduce_max_sync(0xffffffffu, m);
        if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            const uint32_t mm = max(max(red[0], red[1]), max(red[2], red[3]));
            if (mm) atomicMax(lmax, mm);
        }
    }
}

struct LeafChunk {
    int e, j0, cnt;
};

#define LEAF32_MAXE 64   // U entries whose source ranges are staged for the chunk table
#define LEAF32_MAXCH 64  // chunks in the shared-memory chunk table
// A leaf's U list cut into chunks of at most LCAP source points, each (entry,
// first point, count).  Built once per leaf in shared memory: every thread
// reads one U entry's source range, thread 0 lays the chunks out in list order;
// a list of more than LEAF32_MAXCH chunks is enumerated on the fly instead.
struct LeafChunkTable {
    int cfirst[LEAF32_MAXE], ccount[LEAF32_MAXE];
    LeafChunk ctab[LEAF32_MAXCH];
    int nch, tabled;
};
__device__ __forceinline__ LeafChunk leaf_chunk_at(const int64_t *ls, const int32_t *usrc, int e0, int e1, int c)
{
    LeafChunk ch{-1, 0, 0};
    for (int e = e0; e < e1; ++e) {
        const int s = usrc[e], a0 = (int)ls[s], a1 = (int)ls[s + 1];
        const int nc = (a1 - a0 + LCAP - 1) / LCAP;
        if (c < nc) {
            ch.e = e;
            ch.j0 = a0 + c * LCAP;
            ch.cnt = min(LCAP, a1 - ch.j0);
            return ch;
        }
        c -= nc;
    }
    return ch;
}
// all threads of the block; ends with a barrier
__device__ __forceinline__ void leaf_chunk_build(LeafChunkTable &T, const int64_t *ls, const int32_t *usrc, int e0,
                                                 int e1)
{
    const int ne = e1 - e0;
    if (ne <= LEAF32_MAXE) {
        for (int t = threadIdx.x; t < ne; t += blockDim.x) {
            const int s = usrc[e0 + t];
            T.cfirst[t] = (int)ls[s];
            T.ccount[t] = (int)(ls[s + 1] - ls[s]);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            int n = 0;
            for (int t = 0; t < ne; ++t)
                for (int j = 0; j < T.ccount[t]; j += LCAP, ++n)
                    if (n < LEAF32_MAXCH) T.ctab[n] = LeafChunk{e0 + t, T.cfirst[t] + j, min(LCAP, T.ccount[t] - j)};
            T.nch = n;
            T.tabled = n <= LEAF32_MAXCH;
        }
    } else if (threadIdx.x == 0) {
        int n = 0;
        for (int e = e0; e < e1; ++e) {
            const int s = usrc[e];
            n += ((int)(ls[s + 1] - ls[s]) + LCAP - 1) / LCAP;
        }
        T.nch = n;
        T.tabled = 0;
    }
    __syncthreads();
}
__device__ __forceinline__ LeafChunk leaf_chunk(const LeafChunkTable &T, const int64_t *ls, const int32_t *usrc,
                                                int e0, int e1, int c)
{
    return T.tabled ? T.ctab[c] : leaf_chunk_at(ls, usrc, e0, e1, c);
}

// Step 4 in FP32: L2T (Eq. (local)) and S2T for every target of a leaf, one
// block per leaf, one thread per target.  The leaf's U list is cut into chunks
// of at most LCAP source points (tabled once in shared memory); each chunk's
// coordinates and densities are staged with cp.async, double-buffered, one
// barrier per chunk.  A chunk's sums are kept apart from the running totals
// (in shared memory) so that FP32 rounding grows with the chunk length, not the
// list length.  Free pairs take (i/4) H0 from its series, evaluated one pair
// ahead of the multiply-adds; reflected pairs add their tails (the segment part
// comes from k_near_pw32).
// NV: vectors computed (4 or 16); buffers keep the 16-vector layout.
// DEG > 0: every free near pair has t = (k r / 2)^2 <= 1 and the series of degree
// DEG meets the 1e-9 truncation bound (lm_h0_terms); DEG = 0: degree 8 and the far form.
#define LEAF32_THREADS 64
template <int P, int NV, int DEG = 0, class G = Grid32>
__global__ void __launch_bounds__(LEAF32_THREADS, 8) k_leaf32(G geo, float k, float d, const float *xl,
                                                  const float *yl, const float *y32, const int64_t *ls,
                                                  const int64_t *ustart, const int32_t *usrc, const int32_t *uterm,
                                                  NearQuadF nq, const zf *Lc, const zf *qs, zf *us, int nterms,
                                                  int free_on)
{
    constexpr int NP = 2 * P + 1;
    __shared__ __align__(16) zf sq[2][LCAP * LM_MAXV];
    __shared__ float sx[2][LCAP], sy[2][LCAP], sya[2][LCAP];
    __shared__ __align__(16) zf sacc[NV * LEAF32_THREADS]; // running sums per target and vector
    const int64_t b = geo.id(blockIdx.x);
    const float w = geo.width(b);
    const zf *Lb = Lc + b * NP * LM_MAXV;
    const int lo = (int)ls[b], hi = (int)ls[b + 1];
    const int e0 = (int)ustart[b], e1 = (int)ustart[b + 1];
    const float k24 = 0.25f * k * k;

    __shared__ LeafChunkTable ctable;
    leaf_chunk_build(ctable, ls, usrc, e0, e1);
    const int nch = ctable.nch;
    auto chunk = [&](int c) { return leaf_chunk(ctable, ls, usrc, e0, e1, c); };
    auto issue = [&](int c, int buf) {
        const LeafChunk ch = chunk(c);
        for (int t = threadIdx.x; t < ch.cnt * (NV / 2); t += blockDim.x) {
            const int j = t / (NV / 2), part = t % (NV / 2);
            cp_async16(&sq[buf][j * LM_MAXV + 2 * part], qs + (int64_t)(ch.j0 + j) * LM_MAXV + 2 * part);
        }
        for (int t = threadIdx.x; t < ch.cnt; t += blockDim.x) {
            cp_async4(&sx[buf][t], xl + ch.j0 + t);
            cp_async4(&sy[buf][t], yl + ch.j0 + t);
            cp_async4(&sya[buf][t], y32 + ch.j0 + t);
        }
    };

    for (int i0 = lo; i0 < hi; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        const bool act = i < hi;
        const float xi = act ? xl[i] : 0.f, yi = act ? yl[i] : 0.f, ya = act ? y32[i] : -0.5f;
        zf *sa = sacc + threadIdx.x; // this target's running sums, vector v at sa[v * LEAF32_THREADS]
        if (nch > 0) {
            issue(0, 0);
            cp_commit();
        }
        {
            zf acc[NV];
#pragma unroll
            for (int v = 0; v < NV; ++v) acc[v] = zf{0.f, 0.f};
            if (act) {
                float r = sqrtf(xi * xi + yi * yi);
                float J[P + 1];
                bessel_j_scaled<float>(P, k * r, k * w, J);
                zf z = r > 0.f ? zf{xi / r, yi / r} : zf{1.f, 0.f};
                zf zp = {1.f, 0.f};
#pragma unroll
                for (int v = 0; v < NV; ++v) cfmaf(acc[v], zf{J[0], 0.f}, Lb[P * LM_MAXV + v]);
                for (int m = 1; m <= P; ++m) {
                    zp = zp * z;
                    zf bp = J[m] * zp;
                    zf bn = ((m & 1) ? -J[m] : J[m]) * conj(zp);
#pragma unroll
                    for (int v = 0; v < NV; ++v) {
                        cfmaf(acc[v], bp, Lb[(P + m) * LM_MAXV + v]);
                        cfmaf(acc[v], bn, Lb[(P - m) * LM_MAXV + v]);
                    }
                }
            }
#pragma unroll
            for (int v = 0; v < NV; ++v) sa[v * LEAF32_THREADS] = acc[v];
        }
        for (int c = 0; c < nch; ++c) {
            const int buf = c & 1;
            // chunk c has landed; past this barrier every thread is done with chunk c - 1,
            // so its buffer takes chunk c + 1 (one barrier per chunk)
            cp_wait<0>();
            __syncthreads();
            if (c + 1 < nch) {
                issue(c + 1, buf ^ 1);
                cp_commit();
            }
            const LeafChunk ch = chunk(c);
            const int s = usrc[ch.e], term = uterm[ch.e];
            float ox, oy;
            geo.offset(b, s, ox, oy); // centre_t - centre_s
            if (act) {
                // the chunk's sums on the paired FP32 pipe: A_v = sum g.re q_v and B_v = sum g.im q_v,
                // each a (re, im) pair, so that g q_v = (A.x - B.y, A.y + B.x) at the end of the chunk
                float2 A[NV], B[NV];
#pragma unroll
                for (int v = 0; v < NV; ++v) A[v] = B[v] = make_float2(0.f, 0.f);
                auto mac = [&](zf g, int jj) {
                    const float2 gr = make_float2(g.re, g.re), gi = make_float2(g.im, g.im);
                    const float4 *qj = (const float4 *)&sq[buf][jj * LM_MAXV];
#pragma unroll
                    for (int v2 = 0; v2 < NV / 2; ++v2) {
                        const float4 t = qj[v2];
                        const float2 q0 = make_float2(t.x, t.y), q1 = make_float2(t.z, t.w);
                        A[2 * v2] = __ffma2_rn(gr, q0, A[2 * v2]);
                        B[2 * v2] = __ffma2_rn(gi, q0, B[2 * v2]);
                        A[2 * v2 + 1] = __ffma2_rn(gr, q1, A[2 * v2 + 1]);
                        B[2 * v2 + 1] = __ffma2_rn(gi, q1, B[2 * v2 + 1]);
                    }
                };
                if (term == 0 && free_on) {
                    const int self = i - ch.j0; // this target's slot in the chunk, if it is a source here
                    // the target relative to the source leaf's centre, once per chunk
                    const float xo = xi + ox, yo = yi + oy;
                    // software pipeline: the series of pair jj + 1 is evaluated in the same
                    // basic block as the multiply-adds of pair jj, so its serial Horner chain
                    // overlaps them; the rare far-argument branch comes after them.  Only the
                    // chunk that holds the target itself tests for the self term, which is
                    // excluded: a dummy t = 1 keeps the evaluation finite, the weight is zeroed.
                    auto pairs = [&](auto has_self) {
                        constexpr bool HS = decltype(has_self)::value;
                        auto targ = [&](int jj) {
                            const float dx = xo - sx[buf][jj], dy = yo - sy[buf][jj];
                            const float t2 = k24 * fmaf(dx, dx, dy * dy);
                            return (HS && jj == self) ? 1.0f : t2;
                        };
                        float tn = targ(0);
                        zf gn = DEG ? green_free32_series_d<DEG ? DEG : 8>(tn)
                                    : (tn <= 1.0f ? green_free32_series(tn) : green_free32_far(tn));
                        for (int jj = 0; jj < ch.cnt; ++jj) {
                            const zf g = (HS && jj == self) ? zf{0.f, 0.f} : gn;
                            tn = targ(min(jj + 1, ch.cnt - 1));
                            gn = DEG ? green_free32_series_d<DEG ? DEG : 8>(tn) : green_free32_series(tn);
                            mac(g, jj);
                            if (!DEG && tn > 1.0f) gn = green_free32_far(tn);
                        }
                    };
                    if (self >= 0 && self < ch.cnt)
                        pairs(std::true_type{});
                    else
                        pairs(std::false_type{});
                } else if (term != 0) {
                    for (int jj = 0; jj < ch.cnt; ++jj) {
                        // tail of a reflected direct term; its segment part is added by k_near_pw32
                        const float dx = (xi - sx[buf][jj]) + ox;
                        const float h = term == 1 ? -(ya + sya[buf][jj]) : ya + sya[buf][jj] + 2.0f * d;
                        mac(near_tail32(nq, term - 1, fabsf(dx), h), jj);
                    }
                }
#pragma unroll
                for (int v = 0; v < NV; ++v)
                    sa[v * LEAF32_THREADS] = sa[v * LEAF32_THREADS] + zf{A[v].x - B[v].y, A[v].y + B[v].x};
            }
        }
        __syncthreads(); // the next pass of targets refills buffer 0
        if (act) {
            float4 *o = (float4 *)(us + (int64_t)i * LM_MAXV);
#pragma unroll
            for (int v2 = 0; v2 < NV / 2; ++v2) {
                const zf a0 = sa[2 * v2 * LEAF32_THREADS], a1 = sa[(2 * v2 + 1) * LEAF32_THREADS];
                o[v2] = make_float4(a0.re, a0.im, a1.re, a1.im);
            }
        }
    }
}

// ---------------------------------------------------------------------------
template <int NP, int RG>
static void launch_stencil_rg(const Level &lv, cudaStream_t st)
{
    int64_t ncls = (lv.ncol / 2) * (lv.nrow / 2);
    dim3 g((unsigned)((ncls + 15) / 16), 4);
    k_m2l_stencil32<NP, RG><<<g, 64 * ((NP + RG - 1) / RG), 0, st>>>(lv.ncol, lv.nrow, lv.stencil, lv.tab32,
                                                                       lv.M32, lv.L32);
}
// rg = 2 only while the block stays within 1024 threads (2p + 1 <= 32)
template <int P>
static void launch_stencil(const Level &lv, cudaStream_t st, int rg)
{
    constexpr int NP = 2 * P + 1;
    if constexpr (NP <= 32) {
        if (rg == 2) return launch_stencil_rg<NP, 2>(lv, st);
    }
    if (rg == 8) return launch_stencil_rg<NP, 8>(lv, st);
    launch_stencil_rg<NP, 4>(lv, st);
}
// nvs: vector slots the apply computes (4 or 16)
template <int P>
static void launch_m2m(const Level &lv, const Level &child, cudaStream_t st, int nvs)
{
    constexpr int NP = 2 * P + 1;
    if (nvs == 4)
        k_m2m32<NP, 4><<<(unsigned)lv.nbox, 128, 0, st>>>(GridKids32{lv.ncol}, lv.m2m32, child.M32, lv.M32);
    else
        k_m2m32<NP, LM_MAXV><<<(unsigned)lv.nbox, 128, 0, st>>>(GridKids32{lv.ncol}, lv.m2m32, child.M32, lv.M32);
}
template <int P>
static void launch_l2l(const Level &lv, const Level &par, cudaStream_t st, int nvs)
{
    constexpr int NP = 2 * P + 1;
    if (nvs == 4)
        k_l2l32<NP, 4><<<(unsigned)lv.nbox, 128, 0, st>>>(GridPar32{lv.ncol}, lv.l2l32, par.L32, lv.L32, nullptr);
    else
        k_l2l32<NP, LM_MAXV><<<(unsigned)lv.nbox, 128, 0, st>>>(GridPar32{lv.ncol}, lv.l2l32, par.L32, lv.L32,
                                                                 nullptr);
}
// L2L of the tile-form apply: adds to the M2L's local expansions
template <int P>
static void launch_l2l_acc(const Level &lv, const Level &par, cudaStream_t st, int nvs, uint32_t *lmax)
{
    constexpr int NP = 2 * P + 1;
    if (nvs == 4)
        k_l2l32<NP, 4, true><<<(unsigned)lv.nbox, 128, 0, st>>>(GridPar32{lv.ncol}, lv.l2l32, par.L32, lv.L32, lmax);
    else
        k_l2l32<NP, LM_MAXV, true><<<(unsigned)lv.nbox, 128, 0, st>>>(GridPar32{lv.ncol}, lv.l2l32, par.L32,
                                                                       lv.L32, lmax);
}
template <int P>
static void launch_rest(const Level &lv, cudaStream_t st, int nvs)
{
    constexpr int NP = 2 * P + 1;
    if (nvs == 4)
        k_m2l_rest32<NP, 4><<<(unsigned)lv.nrtgt, 128, 0, st>>>(lv.rtgt, lv.rstart, lv.rsrc, lv.rslot, lv.tab32,
                                                              lv.M32, lv.L32);
    else
        k_m2l_rest32<NP, LM_MAXV><<<(unsigned)lv.nrtgt, 128, 0, st>>>(lv.rtgt, lv.rstart, lv.rsrc, lv.rslot,
                                                                    lv.tab32, lv.M32, lv.L32);
}
static bool tiles_ready(const lm_tree_s *t);
template <int P>
static void launch_leaf(lm_tree_s *t, const NearQuadF &nq, cudaStream_t st, int nv)
{
    if (nv > 4 && t->lf_ready && tiles_ready(t)) { // 16 vector slots: the multiply-adds on the tensor cores
        lm_launch_leaf_tt(t, nq, st);
        return;
    }
    const Level &lv = t->lev[t->L];
    // largest k r of a direct pair: two leaves apart diagonally
    const double xmax = t->med.k2 * lv.w * 2.0 * 1.4142135623730951 * 1.0001;
    const int nterms = lm_h0_terms(xmax);
    const int free_on = t->med.opt.kernel == LM_KERNEL_G;
    if (nv > 4 && xmax <= 2.0 && nterms <= 6) // short series, no far form (k2 w <= 0.7)
        k_leaf32<P, LM_MAXV, 6><<<(unsigned)lv.nbox, LEAF32_THREADS, 0, st>>>(
            Grid32{lv.ncol, (float)lv.w}, (float)t->med.k2, (float)t->med.d, t->xl32, t->yl32, t->y32, t->leaf_start,
            t->ustart, t->usrc, t->uterm, nq, lv.L32, t->qs32, t->us32, nterms, free_on);
    else if (nv <= 4) // the batched form's 4-vector applies: a quarter of the contraction
        k_leaf32<P, 4><<<(unsigned)lv.nbox, LEAF32_THREADS, 0, st>>>(Grid32{lv.ncol, (float)lv.w}, (float)t->med.k2, (float)t->med.d,
                                                         t->xl32, t->yl32, t->y32, t->leaf_start, t->ustart,
                                                         t->usrc, t->uterm, nq, lv.L32, t->qs32, t->us32, nterms,
                                                         free_on);
    else
        k_leaf32<P, LM_MAXV><<<(unsigned)lv.nbox, LEAF32_THREADS, 0, st>>>(Grid32{lv.ncol, (float)lv.w}, (float)t->med.k2,
                                                               (float)t->med.d, t->xl32, t->yl32, t->y32,
                                                               t->leaf_start, t->ustart, t->usrc, t->uterm, nq,
                                                               lv.L32, t->qs32, t->us32, nterms, free_on);
}

int lm_h0_terms(double xmax);
static size_t near_pw_smem(const lm_tree_s *t)
{
    return (size_t)2 * t->nq.nseg * LM_MAXV * sizeof(zf) + PW_SRC * LM_MAXV * sizeof(zf) + 2 * PW_SRC * sizeof(float);
}

#define MX_DISPATCH(P, FN, ...)                                           \
    switch (P) {                                                          \
    case 4: FN<4>(__VA_ARGS__); break;                                    \
    case 6: FN<6>(__VA_ARGS__); break;                                    \
    case 8: FN<8>(__VA_ARGS__); break;                                    \
    case 9: FN<9>(__VA_ARGS__); break;                                    \
    case 10: FN<10>(__VA_ARGS__); break;                                  \
    case 11: FN<11>(__VA_ARGS__); break;                                  \
    case 12: FN<12>(__VA_ARGS__); break;                                  \
    case 13: FN<13>(__VA_ARGS__); break;                                  \
    case 14: FN<14>(__VA_ARGS__); break;                                  \
    case 16: FN<16>(__VA_ARGS__); break;                                  \
    case 18: FN<18>(__VA_ARGS__); break;                                  \
    case 20: FN<20>(__VA_ARGS__); break;                                  \
    case 24: FN<24>(__VA_ARGS__); break;                                  \
    default: break;                                                       \
    }

bool lm_mixed_order_supported(int P)
{
    switch (P) {
    case 4: case 6: case 8: case 9: case 10: case 11: case 12: case 13: case 14: case 16: case 18: case 20:
    case 24: return true;
    default: return false;
    }
}

static NearQuadF nqf_of(const lm_tree_s *t)
{
    return NearQuadF{t->nq.nseg, t->nq.nray, t->nq.ntail, t->nq_seg_lam, t->nq_seg_s2, t->nq_seg_w, t->nq_tail_lam,
                     t->nq_tail_s2, t->nq_tail_w,
                     t->med.opt.top_bc != LM_BC_IMPEDANCE && t->med.opt.bottom_bc != LM_BC_IMPEDANCE,
                     {(float)t->nq.rinf[0], (float)t->nq.rinf[1]}, (float)t->nq.hray,
                     (float)(0.25 * t->med.k2 * t->med.k2)};
}

// the mixed apply on the adaptive tree: the steps of the uniform apply over box lists
template <int P>
static void launch_m2m_list(const AdaptTree &A, const Level &lv, int l, cudaStream_t st, int nvs)
{
    constexpr int NP = 2 * P + 1;
    const int64_t npar = A.nl_start[l + 1] - A.nl_start[l];
    if (npar == 0) return;
    const ListKids32 kids{A.nonleaf + A.nl_start[l], A.child};
    if (nvs == 4)
        k_m2m32<NP, 4, ListKids32><<<(unsigned)npar, 128, 0, st>>>(kids, lv.m2m32, A.M32, A.M32);
    else
        k_m2m32<NP, LM_MAXV, ListKids32><<<(unsigned)npar, 128, 0, st>>>(kids, lv.m2m32, A.M32, A.M32);
}
template <int P>
static void launch_l2l_list(const AdaptTree &A, const Level &lv, int l, cudaStream_t st, int nvs)
{
    constexpr int NP = 2 * P + 1;
    const int64_t b0 = A.lev_start[l], nb = A.lev_start[l + 1] - b0;
    if (nb == 0) return;
    const ListPar32 par{b0, A.parent, A.pos};
    if (nvs == 4)
        k_l2l32<NP, 4, false, ListPar32><<<(unsigned)nb, 128, 0, st>>>(par, lv.l2l32, A.L32, A.L32, nullptr);
    else
        k_l2l32<NP, LM_MAXV, false, ListPar32><<<(unsigned)nb, 128, 0, st>>>(par, lv.l2l32, A.L32, A.L32,
                                                                             nullptr);
}
template <int P>
static void launch_rest_list(const AdaptTree &A, int l, cudaStream_t st, int nvs)
{
    constexpr int NP = 2 * P + 1;
    if (A.m2l_ntgt[l] == 0) return;
    if (nvs == 4)
        k_m2l_rest32<NP, 4><<<(unsigned)A.m2l_ntgt[l], 128, 0, st>>>(A.m2l_tgt[l], A.vstart, A.vsrc, A.vslot,
                                                                       A.tab32, A.M32, A.L32);
    else
        k_m2l_rest32<NP, LM_MAXV><<<(unsigned)A.m2l_ntgt[l], 128, 0, st>>>(A.m2l_tgt[l], A.vstart, A.vsrc,
                                                                             A.vslot, A.tab32, A.M32, A.L32);
}
template <int P>
static void launch_leaf_list(lm_tree_s *t, const NearQuadF &nq, cudaStream_t st, int nv)
{
    const AdaptTree &A = t->at;
    const List32 leaves{A.leaves, A.cx, A.cy, A.w};
    const int free_on = t->med.opt.kernel == LM_KERNEL_G;
    if (nv <= 4)
        k_leaf32<P, 4, 0, List32><<<(unsigned)A.nleaf, LEAF32_THREADS, 0, st>>>(
            leaves, (float)t->med.k2, (float)t->med.d, t->xl32, t->yl32, t->y32, t->leaf_start, t->ustart, t->usrc,
            t->uterm, nq, A.L32, t->qs32, t->us32, 11, free_on);
    else
        k_leaf32<P, LM_MAXV, 0, List32><<<(unsigned)A.nleaf, LEAF32_THREADS, 0, st>>>(
            leaves, (float)t->med.k2, (float)t->med.d, t->xl32, t->yl32, t->y32, t->leaf_start, t->ustart, t->usrc,
            t->uterm, nq, A.L32, t->qs32, t->us32, 11, free_on);
}

static lm_status run_mixed_adaptive(lm_tree_s *t, const void *q, int nvec, void *u, bool adjoint, bool c64,
                                    cudaStream_t st)
{
    const AdaptTree &A = t->at;
    const int L = t->L, P = t->p, np = 2 * P + 1;
    const int64_t n = t->n;
    const float k = (float)t->med.k2;
    const NearQuadF nq = nqf_of(t);
    const List32 leaves{A.leaves, A.cx, A.cy, A.w}, pwl{A.pwleaves, A.cx, A.cy, A.w};
    for (int v0 = 0; v0 < nvec; v0 += LM_MAXV) {
        const int nv = std::min(LM_MAXV, nvec - v0);
        const int nvs = nv <= 4 ? 4 : LM_MAXV;
        lm_phase_begin(t, PH_PERMUTE, st);
        if (c64)
            k_permute_in32<zf><<<gridm(n, 256), 256, 0, st>>>((const zf *)q + (int64_t)v0 * n, t->iperm, n, nv,
                                                             adjoint, t->qs32, nullptr);
        else
            k_permute_in32<zd><<<gridm(n, 256), 256, 0, st>>>((const zd *)q + (int64_t)v0 * n, t->iperm, n, nv,
                                                             adjoint, t->qs32, nullptr);
        lm_phase_end(t, PH_PERMUTE, st, 1);
        lm_phase_begin(t, PH_S2M, st);
        if (A.nleaf > 0) {
            const size_t shm = (P2M32_CHUNK * np + P2M32_CHUNK * LM_MAXV) * sizeof(zf);
            k_p2m32<List32><<<(unsigned)A.nleaf, 128, shm, st>>>(leaves, P, k, t->xl32, t->yl32, t->leaf_start,
                                                                 t->qs32, nvs, A.M32);
        }
        lm_phase_end(t, PH_S2M, st, 1);
        if (L > 0) lm_phase_begin(t, PH_M2M, st);
        for (int l = L - 1; l >= 0; --l) MX_DISPATCH(P, launch_m2m_list, A, t->lev[l], l, st, nvs);
        if (L > 0) lm_phase_end(t, PH_M2M, st, L);
        for (int l = 0; l <= L; ++l) {
            lm_phase_begin(t, PH_L2L, st);
            if (l == 0) {
                const int64_t nb = A.lev_start[1] - A.lev_start[0];
                LM_CUDA(cudaMemsetAsync(A.L32 + A.lev_start[0] * np * LM_MAXV, 0, nb * np * LM_MAXV * sizeof(zf), st));
            } else {
                MX_DISPATCH(P, launch_l2l_list, A, t->lev[l], l, st, nvs);
            }
            lm_phase_end(t, PH_L2L, st, l > 0);
            lm_phase_begin(t, PH_M2L, st);
            MX_DISPATCH(P, launch_rest_list, A, l, st, nvs);
            lm_phase_end(t, PH_M2L, st, A.m2l_ntgt[l] > 0);
        }
        lm_phase_begin(t, PH_LEAF, st);
        if (A.nleaf > 0) MX_DISPATCH(P, launch_leaf_list, t, nq, st, nv);
        if (A.npw > 0)
            k_near_pw32<List32><<<(unsigned)A.npw, 256, near_pw_smem(t), st>>>(
                pwl, (float)t->med.d, t->xl32, t->y32, t->leaf_start, t->ustart, t->usrc, t->uterm, nq, t->qs32,
                t->us32);
        lm_phase_end(t, PH_LEAF, st, 1 + (A.npw > 0));
        lm_phase_begin(t, PH_PERMUTE, st);
        if (c64)
            k_permute_out32<zf><<<gridm(n, 256), 256, 0, st>>>(t->us32, t->iperm, n, nv, adjoint,
                                                              (zf *)u + (int64_t)v0 * n);
        else
            k_permute_out32<zd><<<gridm(n, 256), 256, 0, st>>>(t->us32, t->iperm, n, nv, adjoint,
                                                              (zd *)u + (int64_t)v0 * n);
        lm_phase_end(t, PH_PERMUTE, st, 1);
        LM_CUDA(cudaGetLastError());
    }
    return LM_OK;
}

// the tile-form M2L of all levels applies to this tree
static bool tiles_ready(const lm_tree_s *t)
{
    bool ok = t->tt_ready && !t->adaptive;
    for (int l = 1; l <= t->L && ok; ++l) ok = t->lev[l].m2l_impl == 0;
    return ok;
}
bool lm_mixed_tiles(const lm_tree_s *t, int nvec)
{
    return t->precision == LM_MIXED && nvec >= 1 && nvec <= LM_MAXV && tiles_ready(t);
}

lm_status lm_run_apply_mixed(lm_tree_s *t, const void *q, int nvec, void *u, bool adjoint, bool c64, cudaStream_t st,
                             int part)
{
    if (t->adaptive) return run_mixed_adaptive(t, q, nvec, u, adjoint, c64, st);
    if (part != 0 && !lm_mixed_tiles(t, nvec)) {
        lm_set_error("apply: a split apply needs the tile-form M2L and at most %d vectors", LM_MAXV);
        return LM_ENOTSUP;
    }
    const int L = t->L, P = t->p, np = 2 * P + 1;
    const int64_t n = t->n;
    const float k = (float)t->med.k2;
    const NearQuadF nq = nqf_of(t);
    const bool up = part != 2;
    for (int v0 = 0; v0 < nvec; v0 += LM_MAXV) {
        const int nv = std::min(LM_MAXV, nvec - v0);
        const int nvs = nv <= 4 ? 4 : LM_MAXV; // vector slots the contractions compute
        const bool tiles = tiles_ready(t);
        // the tensor-core leaf step takes the largest density and local-expansion components of
        // this block of vectors (power-of-two scales into FP16's range), found by permute and L2L
        const bool lft = nv > 4 && t->lf_ready && tiles;
        if (up) {
        if (lft) LM_CUDA(cudaMemsetAsync(t->lf_scl, 0, 2 * sizeof(uint32_t), st));
        lm_phase_begin(t, PH_PERMUTE, st);
        if (c64)
            k_permute_in32<zf><<<gridm(n, 256), 256, 0, st>>>((const zf *)q + (int64_t)v0 * n, t->iperm, n, nv,
                                                             adjoint, t->qs32, lft ? t->lf_scl : nullptr);
        else
            k_permute_in32<zd><<<gridm(n, 256), 256, 0, st>>>((const zd *)q + (int64_t)v0 * n, t->iperm, n, nv,
                                                             adjoint, t->qs32, lft ? t->lf_scl : nullptr);
        lm_phase_end(t, PH_PERMUTE, st, 1);
        lm_phase_begin(t, PH_S2M, st);
        {
            Level &lv = t->lev[L];
            if (s2m16_ok(t, nvs)) {
                MX_DISPATCH(P, launch_s2m16, lv, k, t, st);
            } else {
                size_t shm = (P2M32_CHUNK * np + P2M32_CHUNK * LM_MAXV) * sizeof(zf);
                k_p2m32<<<(unsigned)lv.nbox, 128, shm, st>>>(Grid32{lv.ncol, (float)lv.w}, P, k, t->xl32, t->yl32,
                                                             t->leaf_start, t->qs32, nvs, lv.M32);
            }
        }
        lm_phase_end(t, PH_S2M, st, 1);
        if (L > 0) lm_phase_begin(t, PH_M2M, st);
        for (int l = L - 1; l >= 0; --l) {
            MX_DISPATCH(P, launch_m2m, t->lev[l], t->lev[l + 1], st, nvs);
        }
        if (L > 0) lm_phase_end(t, PH_M2M, st, L);
        }
        // tile form: the M2L of every level in one launch (it writes L), then L2L adds
        if (tiles) {
            lm_phase_begin(t, PH_M2L, st);
            if (up) {
                lm_status s = lm_launch_msplit_tt(t, st, nvs);
                if (s != LM_OK) return s;
            }
            if (part == 0) {
                lm_status s = lm_launch_m2l_tt(t, st, nvs);
                if (s != LM_OK) return s;
            }
            lm_phase_end(t, PH_M2L, st, up + (part == 0));
            if (part == 1) continue;
            if (L > 0) lm_phase_begin(t, PH_L2L, st);
            for (int l = 1; l <= L; ++l)
                MX_DISPATCH(P, launch_l2l_acc, t->lev[l], t->lev[l - 1], st, nvs, (l == L && lft) ? t->lf_scl + 1 : nullptr);
            if (L > 0) lm_phase_end(t, PH_L2L, st, L);
        }
        for (int l = 0; l <= L && !tiles; ++l) {
            Level &lv = t->lev[l];
            lm_phase_begin(t, PH_L2L, st);
            if (l == 0)
                LM_CUDA(cudaMemsetAsync(lv.L32, 0, lv.nbox * np * LM_MAXV * sizeof(zf), st));
            else
                MX_DISPATCH(P, launch_l2l, lv, t->lev[l - 1], st, nvs);
            lm_phase_end(t, PH_L2L, st, l > 0);
            lm_phase_begin(t, PH_M2L, st);
            int launches = 0;
            if (l > 0) {
                if (lv.m2l_impl == 0 && t->tc_ready) {
                    lm_status s = lm_launch_m2l_tc(t, l, st, nvs);
                    if (s != LM_OK) return s;
                } else {
                    MX_DISPATCH(P, launch_stencil, lv, st, lv.m2l_impl > 0 ? lv.m2l_impl : 4);
                }
                ++launches;
            }
            if (lv.nrest > 0) {
                MX_DISPATCH(P, launch_rest, lv, st, nvs);
                ++launches;
            }
            lm_phase_end(t, PH_M2L, st, launches);
        }
        lm_phase_begin(t, PH_LEAF, st);
        MX_DISPATCH(P, launch_leaf, t, nq, st, nv);
        {
            const Level &lv = t->lev[L];
            const unsigned nb = (unsigned)(lv.nrow == 1 ? lv.ncol : 2 * lv.ncol);
            EdgeGrid32 eg;
            eg.ncol = lv.ncol;
            eg.w = (float)lv.w;
            eg.nrow = lv.nrow;
            k_near_pw32<<<nb, 256, near_pw_smem(t), st>>>(eg, (float)t->med.d, t->xl32,
                                                          t->y32, t->leaf_start, t->ustart, t->usrc, t->uterm, nq,
                                                          t->qs32, t->us32);
        }
        lm_phase_end(t, PH_LEAF, st, 2);
        lm_phase_begin(t, PH_PERMUTE, st);
        if (c64)
            k_permute_out32<zf><<<gridm(n, 256), 256, 0, st>>>(t->us32, t->iperm, n, nv, adjoint,
                                                              (zf *)u + (int64_t)v0 * n);
        else
            k_permute_out32<zd><<<gridm(n, 256), 256, 0, st>>>(t->us32, t->iperm, n, nv, adjoint,
                                                              (zd *)u + (int64_t)v0 * n);
        lm_phase_end(t, PH_PERMUTE, st, 1);
        LM_CUDA(cudaGetLastError());
    }
    return LM_OK;
}

// ---------------------------------------------------------------------------
// M2L autotuner: per level >= 1, time the free-space stencil with each tile
// shape -- the tcgen05 kernel (8 boxes x 16 vectors x 64 real orders) and the
// CUDA-core kernel with 2, 4 or 8 orders per thread (16 boxes x 4 vectors per
// row group) -- on the tree's own buffers (zeroed first: an apply rewrites
// them), one warm-up and three timed launches each, CUDA events on `st`, and
// keep the fastest.  choice[l] receives 0 (tensor cores) or the rows per
// thread; ms[l] its time per launch.
// ---------------------------------------------------------------------------
lm_status lm_autotune_mixed(lm_tree_s *t, cudaStream_t st, int *choice, float *ms)
{
    const int P = t->p, np = 2 * P + 1;
    cudaEvent_t e0, e1;
    LM_CUDA(cudaEventCreate(&e0));
    LM_CUDA(cudaEventCreate(&e1));
    lm_status status = LM_OK;
    for (int l = 0; l <= t->L && status == LM_OK; ++l) {
        Level &lv = t->lev[l];
        if (choice) choice[l] = -1;
        if (ms) ms[l] = 0.f;
        if (l == 0) continue; // level 0 has no stencil: its entries are on the rest list
        if (cudaMemsetAsync(lv.M32, 0, lv.nbox * np * LM_MAXV * sizeof(zf), st) != cudaSuccess ||
            cudaMemsetAsync(lv.L32, 0, lv.nbox * np * LM_MAXV * sizeof(zf), st) != cudaSuccess) {
            status = LM_ECUDA;
            break;
        }
        int cand[4], nc = 0;
        if (t->tc_ready) cand[nc++] = 0;
        if (np <= 32) cand[nc++] = 2;
        cand[nc++] = 4;
        cand[nc++] = 8;
        int best = cand[0];
        float best_ms = 1e30f;
        for (int ci = 0; ci < nc && status == LM_OK; ++ci) {
            lv.m2l_impl = cand[ci];
            auto run = [&]() -> lm_status {
                if (cand[ci] == 0) return lm_launch_m2l_tc(t, l, st, LM_MAXV);
                MX_DISPATCH(P, launch_stencil, lv, st, cand[ci]);
                return LM_OK;
            };
            status = run();
            if (status != LM_OK) break;
            cudaEventRecord(e0, st);
            for (int r = 0; r < 3 && status == LM_OK; ++r) status = run();
            cudaEventRecord(e1, st);
            if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
                lm_set_error("autotune: a candidate launch failed at level %d", l);
                status = LM_ECUDA;
                break;
            }
            float el = 0.f;
            cudaEventElapsedTime(&el, e0, e1);
            el /= 3.f;
            if (el < best_ms) {
                best_ms = el;
                best = cand[ci];
            }
        }
        lv.m2l_impl = best;
        if (choice) choice[l] = best;
        if (ms) ms[l] = best_ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return status;
}
