// internal.h -- host-side structures shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/lmfmm.h"
#include "common.cuh"

#define LM_MAXP 48      // largest supported expansion order p
#define LM_MAXV 16      // vectors per kernel pass
#define LM_MAXLEAF 8192 // largest leaf the tree builder sorts

void lm_set_error(const char *fmt, ...);

// Dynamic shared-memory limits are per kernel and per device, shared by every
// tree: raise one (never lower it) so that trees built earlier, with larger
// needs, still launch.  slot names the kernel in a small per-device cache.
enum { LM_SMEM_NEAR_PW = 0, LM_SMEM_IMAGE_M2L = 1, LM_SMEM_CROSS_M2L = 2, LM_SMEM_NEAR_PW64 = 3,
       LM_SMEM_IMAGE_M2L_A = 4, LM_SMEM_NEAR_PW64_A = 5, LM_SMEM_NEAR_PW_A = 6, LM_SMEM_SLOTS = 7 };
cudaError_t lm_raise_smem(const void *func, int slot, int bytes);

#define LM_CUDA(call)                                                                       \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess) {                                                            \
            lm_set_error("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, \
                         __LINE__);                                                         \
            return LM_ECUDA;                                                                \
        }                                                                                   \
    } while (0)

// leaf lattice of one level: ncol columns from x0, boxes of width w, row 0 touching y = 0
struct LeafGeom {
    int64_t ncol;
    double x0, w;
};
__device__ inline void leaf_centre(const LeafGeom &g, int64_t b, double *cx, double *cy)
{
    int64_t r = b / g.ncol, c = b % g.ncol;
    *cx = g.x0 + (c + 0.5) * g.w;
    *cy = -(r + 0.5) * g.w;
}

// Image row of source row r for term m at a level with nrow rows: free r;
// tt -1-r (mirror in y = 0); bb 2nrow-1-r (mirror in y = -d); tb r-2nrow
// (shift +2d); bt r+2nrow (shift -2d).
__host__ __device__ inline int64_t img_row(int term, int64_t r, int64_t nrow)
{
    switch (term) {
    case 0: return r;
    case 1: return -1 - r;
    case 2: return 2 * nrow - 1 - r;
    case 3: return r - 2 * nrow;
    default: return r + 2 * nrow;
    }
}

struct lm_medium_s {
    double k1, k2, k3, d;
    lm_options opt;
};

// Near-field quadrature (Sec. 4.2 alternative directions, Sec. 5 first
// contour) for the two image terms that reach the direct interactions
// (tt near y = 0, bb near y = -d).  All weights include 1/(4 pi).
struct NearQuad {
    int nseg;    // nodes on the deformed segment t in [0, c]
    int nray;    // number of tail rays (angles 0 .. pi/2)
    int ntail;   // nodes per ray
    double c;    // segment end
    // device arrays
    zd *seg_lam, *seg_s2, *seg_w;    // [nseg], [nseg], [2][nseg]: w * lambda' * sigma_m / s2 / 4pi
    zd *tail_lam, *tail_s2, *tail_w; // [nray][ntail], ..., [2 terms][P, M][nray][ntail] (see k_near_tail)
    // FP64 target gradient: the differentiated tails decay more slowly and take their own,
    // longer rule (ntail_g >= 64 points per ray), same layout
    int ntail_g;
    zd *tail_lam_g, *tail_s2_g, *tail_w_g;
    // wall media: the tables integrate sigma - rinf; each pair adds rinf (i/4) H0(k2 rho_image)
    double rinf[2];
    // Between two walls the remainder sigma - rinf is carried by the multiple reflections,
    // e^{-2 d s2}: images at height h + 2d.  Their integrand decays along the ray nearest
    // atan2(X, h + 2d), not along the north ray that a pair close to a wall would pick
    // from atan2(X, h), where e^{-2 d s2} only oscillates.  hray = 2d then, else 0.
    double hray;
    // FP64 with walls on both sides: tail_w holds the single reflection R - rinf (summed on
    // the ray of atan2(X, h); identically zero for Dirichlet / Neumann walls, a_zero) and
    // tail_w2 the multiple reflections sigma - R (ray of atan2(X, h + 2d)); same layout.
    bool split, a_zero;
    zd *tail_w2, *tail_w2_g;
    // FP64 with an impedance wall: weights of 2 i beta / s2 on the segment ([2][nseg]) and on
    // the gradient's tail rays (layout of tail_w_g), which the gradient's h-derivative
    // subtracts (imp_beta); beta = k2 alpha per wall, 0 without one
    zd *seg_c, *tail_c_g;
    double beta[2];
};

struct Level {
    int l;
    int64_t ncol, nrow, nbox;
    double w;
    // V list (target-major CSR): sources and table slots
    int64_t nv;
    int64_t *vstart; // [nbox + 1]
    int32_t *vsrc;   // [nv]
    int32_t *vslot;  // [nv]
    int32_t *vterm;  // [nv]
    // translation classes of this level (host copies) and their tables (device)
    std::vector<int> cls_term, cls_dc, cls_dr;
    zd *tab;         // [nclass][np][np] scaled M2L tables
    double *scale;   // [p + 1] S_l(n) = (k w_l / 2)^n / n!
    zd *m2m;         // [4][np][np]: child (level l+1) -> this level's box (l < L)
    zd *l2l;         // [4][np][np]: parent (level l-1) -> child at this level (l > 0)
    zd *M, *Lc;      // [nbox][np][LM_MAXV]
    // FP64 form, double-float M2L: tables and multipoles as (re hi, re lo, im hi, im lo)
    float4 *tabdf;   // [nclass][np][np]
    float4 *tabdft;  // the same, each table transposed ([q][p])
    float4 *Mdf;     // [nbox][np][LM_MAXV], scaled by 2^-qexp
    float4 *m2mdf, *l2ldf; // [4][np][np] copies of m2m, l2l
    // mixed-precision copies (FP32, rounded from the FP64 tables)
    zf *tab32;       // [nclass][np][np]
    zf *m2m32, *l2l32; // [4][np][np]
    zf *M32, *L32;   // [nbox][np][LM_MAXV]
    int32_t *stencil; // [7][7] class index of the free-space offset (dc, dr) + 3, or -1
    // entries not covered by the free-space stencil kernel (level 0, image terms)
    int64_t nrest;
    int64_t *rstart; // [nbox + 1]
    int32_t *rsrc, *rslot;
    int m2l_impl;    // free-space stencil M2L at this level: 0 tensor cores, else CUDA cores with
                     // this many orders per thread (set at build, changed by the autotuner)
    int64_t nrtgt;   // targets with entries on the rest list
    int32_t *rtgt;   // [nrtgt]
};

// Adaptive tree (Algorithm 1, step 1): boxes of every level in one array,
// numbered level by level and, within a level, by row * (R 2^l) + column.  A
// box holding more than leaf_target points above the depth limit has all four
// children; points are ordered by leaf, then input index (leaf_start then has
// one entry per box, empty for boxes that are not leaves).  Lists come from a
// dual traversal and hold entries between boxes of any two levels.
struct AdaptTree {
    int64_t nbox = 0, nleaf = 0, npw = 0;
    std::vector<int64_t> lev_start;  // [L + 2] boxes of level l: [lev_start[l], lev_start[l + 1])
    std::vector<int64_t> nl_start;   // [L + 1] non-leaf boxes of level l: nonleaf[nl_start[l] .. nl_start[l + 1])
    std::vector<int64_t> hbox;       // host copy [nbox][4]: level, column, row, leaf
    std::vector<int> cls_term, cls_lt, cls_ls; // V-list classes: term, target and source level,
    std::vector<int64_t> cls_dx, cls_dy;       // centre offsets in half-widths of the finer level
    double *cx = nullptr, *cy = nullptr, *w = nullptr; // [nbox] box centres and widths
    int32_t *parent = nullptr, *pos = nullptr;         // [nbox] parent id (-1 for roots), child position
    int32_t *child = nullptr;                          // [nbox][4] (-1 for leaves)
    int32_t *leaves = nullptr, *nonleaf = nullptr, *pwleaves = nullptr; // box id lists
    std::vector<int32_t> hpw;                          // host copy of pwleaves
    int64_t nv = 0;
    std::vector<int64_t> lev_nv;                       // [L + 1] V entries of the targets of level l
    int64_t *vstart = nullptr;                         // [nbox + 1] V list, target-major
    int32_t *vsrc = nullptr, *vslot = nullptr, *vterm = nullptr;
    zd *tab = nullptr;                                 // [nclass][np][np] scaled M2L tables
    zd *M = nullptr, *Lc = nullptr;                    // [nbox][np][LM_MAXV]
    float4 *tabdf = nullptr, *tabdft = nullptr, *Mdf = nullptr; // double-float copies (as Level)
    // mixed form: FP32 copies of the tables and expansions, and per level the boxes with V entries
    zf *tab32 = nullptr, *M32 = nullptr, *L32 = nullptr;
    std::vector<int32_t *> m2l_tgt;
    std::vector<int64_t> m2l_ntgt;
};

struct lm_tree_s {
    lm_medium_s med;
    int64_t n;
    int R, L, p, np;
    double x0;
    int64_t nleaf;
    int precision;
    int max_nvec;
    double *xs, *ys;     // tree order coordinates [n]
    int64_t *perm;       // [n] tree position -> input index
    int64_t *leaf_start; // [nleaf + 1]
    // U list (leaf level, target-major CSR)
    int64_t nu;
    int64_t *ustart;  // [nleaf + 1]
    int32_t *usrc;    // [nu]
    int32_t *uterm;   // [nu]
    std::vector<Level> lev;
    NearQuad nq;
    zd *qs, *us; // [LM_MAXV][n] tree-order scratch
    // mixed path
    float *xl32, *yl32, *y32; // leaf-local coordinates and absolute y, FP32 [n]
    int64_t *iperm;            // [n] input index -> tree position
    zf *qs32, *us32;           // [n][LM_MAXV]
    zf *nq_seg_lam, *nq_seg_s2, *nq_seg_w, *nq_tail_lam, *nq_tail_s2, *nq_tail_w;
    bool tc_ready; // tensor-core M2L tables built
    // tile form of the tensor-core M2L (16-vector applies): every V-list entry of every
    // level (free space and the four image terms) as (tile of 8 target boxes, entry) work
    bool tt_ready;
    // [0]: 16-vector form (tiles of 8 boxes), [1]: 4-vector form (tiles of 32 boxes)
    int64_t tt_ntile[2], tt_nent[2];
    void *tt_tiles[2], *tt_ents[2]; // device TtTile[tt_ntile], TtEnt[tt_nent]
    void *tt_lv[2];             // device level descriptors (TtLevel[L + 1]) of each form
    float *tt_tab;              // [classes of all levels][128 rows][64 K] FP16 hi/lo tables, canonical layout
                                // (4096 words per class)
    float *tt_msplit;           // [boxes of all levels + 1][1024 words] FP16 hi/lo multipoles (the 4-vector
                                // form packs 256 words per box in the same buffer), canonical layout
    uint32_t *tt_tmax;          // per level: largest component of its tables (float bits)
    uint32_t *tt_mmax;          // per level: largest multipole component of the apply (float bits)
    std::vector<int64_t> tt_tbase, tt_mbase; // per level: first table, first box
    int tt_grid;                // persistent CTAs (one per SM)
    int tt_poll_limit;          // polls of the first operand wait (-1: the library default)
    // tensor-core leaf step (16-vector applies on uniform trees)
    bool lf_ready;
    void *lf_pts;               // [n] float4 (x, y relative to the leaf centre, absolute y, 0)
    int32_t *lf_tot;            // [nleaf] U-list source points per leaf
    void *lf_ent;               // [nleaf][32] int4 (first point, points, U term, source leaf) per U entry
    uint32_t *lf_scl;           // [2] largest |component| of the apply's densities and leaf-level local
                                // expansions (float bits), for the FP16 scales
    int lf_grid;                // persistent CTAs (one per SM)
    int lf_poll_limit;          // polls of the MMA issuer's first wait (-1: the library default)
    bool near_pw64; // FP64 reflected near field: segment factorised per leaf (k_near_pw64)
    int32_t *pwidx; // [boxes of the leaf level / of the tree] slot of an interface leaf, or -1
    zd *pwC;        // [slots][2 terms][2 nseg][LM_MAXV] per-leaf segment coefficients (k_pw_src64)
    bool adaptive;  // boxes refined where the points are (AdaptTree), FP64 only
    AdaptTree at;
    int *dflag;  // device error flag
    bool m2l_df; // FP64 form: M2L contraction in double-float on the FP32 pipes
    int *qexp;   // device: binary exponent of the largest |density| component of the apply
    int64_t bytes;
    // phase profiling
    int prof_max, prof_used;
    std::vector<cudaEvent_t> prof_ev; // [prof_max][LM_NPHASE][2]
    int64_t prof_launch[8];
    int prof_occ[8];             // occurrences of each phase in the apply being recorded
    std::vector<int> prof_nocc;  // [prof_max][LM_NPHASE]
};

#define LM_NPHASE 7
enum { PH_PERMUTE = 0, PH_S2M, PH_M2M, PH_M2L, PH_L2L, PH_LEAF, PH_REFINE };
// record phase boundaries of the apply in progress (no-ops unless profiling)
void lm_phase_begin(lm_tree_s *t, int ph, cudaStream_t st);
void lm_phase_end(lm_tree_s *t, int ph, cudaStream_t st, int launches);
// bracket one apply for the phase profile (lmfmm_api.cu)
void lm_profile_apply_start(lm_tree_s *t);
void lm_profile_apply_stop(lm_tree_s *t);

// setup (lmfmm_setup.cu)
lm_status lm_setup_tree(lm_tree_s *t, const double *x, const double *y, cudaStream_t st);
lm_status lm_setup_tables(lm_tree_s *t, cudaStream_t st);
lm_status lm_setup_levels(lm_tree_s *t, int L, bool boxes, cudaStream_t st); // scales, M2M/L2L tables
lm_status lm_setup_near(lm_tree_s *t, cudaStream_t st);                      // near-field quadrature
// adaptive tree (lmfmm_adaptive.cu)
lm_status lm_setup_adaptive(lm_tree_s *t, const double *x, const double *y, cudaStream_t st);
lm_status lm_adaptive_lists_to_host(lm_tree_s *t, int which, std::vector<int64_t> &rows, cudaStream_t st);
void lm_free_adaptive(lm_tree_s *t);
lm_status lm_list_to_host(lm_tree_s *t, int which, int level, std::vector<int64_t> &rows,
                          cudaStream_t st);
void lm_free_tree_device(lm_tree_s *t);
// apply (lmfmm_apply.cu)
lm_status lm_run_apply(lm_tree_s *t, const zd *q, int nvec, zd *u, bool adjoint, cudaStream_t st);
size_t lm_near_pw64_smem(int nseg);
lm_status lm_near_pw64_attr(size_t bytes);
lm_status lm_setup_pwsrc(lm_tree_s *t, cudaStream_t st); // interface-leaf slots and coefficient buffer
lm_status lm_setup_df(lm_tree_s *t, cudaStream_t st); // double-float tables and multipole buffers
lm_status lm_run_apply_grad(lm_tree_s *t, const zd *q, int nvec, zd *u, zd *ux, zd *uy, cudaStream_t st);
// mixed precision (lmfmm_mixed.cu)
lm_status lm_setup_mixed(lm_tree_s *t, cudaStream_t st);
lm_status lm_setup_mixed_adaptive(lm_tree_s *t, cudaStream_t st);
lm_status lm_autotune_mixed(lm_tree_s *t, cudaStream_t st, int *choice, float *ms);
lm_status lm_run_apply_mixed(lm_tree_s *t, const void *q, int nvec, void *u, bool adjoint, bool c64, cudaStream_t st,
                             int part = 0);
void lm_free_mixed(lm_tree_s *t);
// tensor-core M2L (lmfmm_tc.cu)
lm_status lm_setup_tc(lm_tree_s *t, cudaStream_t st);
lm_status lm_launch_m2l_tc(lm_tree_s *t, int l, cudaStream_t st, int nvs); // nvs: 4 or 16 vector slots
// tile form (lmfmm_tc_tiles.cu): set-up, and the apply's multipole split + M2L of all levels
lm_status lm_setup_tt(lm_tree_s *t, cudaStream_t st);
lm_status lm_launch_m2l_tt(lm_tree_s *t, cudaStream_t st, int nvs); // nvs: 16 or 4 vector slots
lm_status lm_launch_msplit_tt(lm_tree_s *t, cudaStream_t st, int nvs);
// one tile-form M2L launch over the tiles of several trees (batched applies)
// tensor-core leaf step (lmfmm_leaf_tt.cu): L2T + S2T of 16-vector applies
struct NearQuadF;
lm_status lm_setup_leaf_tt(lm_tree_s *t, cudaStream_t st);
lm_status lm_launch_leaf_tt(lm_tree_s *t, const NearQuadF &nq, cudaStream_t st);
void lm_free_leaf_tt(lm_tree_s *t);
struct lm_tt_batch_s;
lm_status lm_tt_batch_build(lm_tree_s *const *trees, int count, int nvs, lm_tt_batch_s **out);
lm_status lm_tt_batch_launch(const lm_tt_batch_s *b, cudaStream_t st);
void lm_tt_batch_free(lm_tt_batch_s *b);
// the mixed apply in parts: 0 all; 1 up to the split multipoles (the tile M2L left out);
// 2 from L2L on (after a tile M2L of the tree has run).  Parts 1 and 2 need the tile
// form and at most 16 vectors.
bool lm_mixed_tiles(const lm_tree_s *t, int nvec);
void lm_free_tt(lm_tree_s *t);
template <typename T>
lm_status lm_dalloc(lm_tree_s *t, T **p, size_t count)
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
