/*
 * lmfmm.h -- C ABI of a GB300 (sm_103a) library that applies the 2-D
 * three-layer Helmholtz Green's function to complex density vectors with the
 * layered-media FMM of Cho & Huang, "Adapting free-space fast multipole method
 * for layered media Green's function: algorithm and analysis"
 * (arXiv:1902.08250).
 *
 * Medium (Sec. 3, Example 4): interfaces y = 0 and y = -d; wave numbers k1
 * (y > 0), k2 (-d < y < 0), k3 (y < -d).  Sources and targets are the same N
 * points, all in the middle layer.  The operator applied is
 *
 *   u_i = sum_{j != i} q_j (i/4) H0^(1)(k2 |x_i - x_j|) + sum_j q_j G_r(x_i, x_j)
 *
 * (Eq. (direct_sum) with the free-space part of Example 1 and the reflected
 * part G_r written, like Eq. (Green), as four image terms tt, bb, tb, bt of the
 * form Int e^{i lambda (x - x0)} e^{-s2 h_m} sigma_m(lambda) / (4 pi s2) d lambda,
 * s2 = sqrt(lambda^2 - k2^2) with Re s2 >= 0).  The free-space self term j = i
 * is excluded; the reflected self terms are included.
 *
 * Conventions shared by every entry point:
 *  - Device pointers are CUDA global-memory pointers on the current device.
 *    Complex arrays are interleaved (re, im) IEEE double, i.e. complex128,
 *    laid out [nvec][n] (vector-major, contiguous, no padding).
 *  - Host pointers are ordinary CPU memory.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    All device work of a call is enqueued on it; calls return without
 *    synchronising unless stated.
 *  - The caller owns every buffer it passes; the library never frees or
 *    retains caller buffers after a call returns.  Handles own their device
 *    memory (tables, tree arrays, expansion scratch), which is allocated by
 *    lm_build_tree and freed by lm_destroy_tree; lm_apply allocates nothing.
 *  - Every call returns an lm_status; on failure lm_last_error() returns a
 *    thread-local message.  Nothing aborts, traps or exits.
 */
#ifndef LMFMM_H
#define LMFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LM_OK = 0,
    LM_EINVAL = 1,   /* invalid argument: bad medium, point, size, alias */
    LM_ENOMEM = 2,   /* device or host allocation failed */
    LM_ECUDA = 3,    /* a CUDA runtime call failed */
    LM_ETIMEOUT = 4, /* a bounded device-side wait gave up */
    LM_ENOTSUP = 5   /* configuration outside what this build supports */
} lm_status;

typedef enum {
    LM_FP64 = 0, /* every step in IEEE double */
    LM_MIXED = 1 /* tables built in FP64 and rounded to FP32; expansions, M2L and
                    near field in FP32 with FP32 accumulation; p in {4, 6, 8..14, 16,
                    18, 20, 24} */
} lm_precision;

typedef struct {
    int p;           /* expansion order: coefficients -p..p (Sec. 4.1); 0 -> 20 */
    int depth;       /* quadtree depth below the d x d roots; -1 -> automatic */
    int leaf_target; /* automatic depth: from the least L with n <= leaf_target * R * 4^L, deeper
                        while sum(n_leaf^2)/n > 1.5 leaf_target (clustered points), keeping the
                        leaves fewer than twice the points; 0 -> 48 */
    int precision;   /* lm_precision */
    int max_nvec;    /* largest nvec one apply processes at once (larger nvec is
                        processed in chunks); 0 -> 16 */
    int seg_order;   /* near-field contour: Gauss-Legendre points per segment panel; 0 -> 16 (FP64), 10 (mixed) */
    int tail_order;  /* near-field tail: Gauss-Legendre points per ray; 0 -> 48 (FP64; 192 with an
                        impedance wall, whose reflection tends to 1 only like 1/lambda), 24 (mixed).
                        The FP64 target gradient (lm_apply_grad) integrates its differentiated
                        tails, which decay more slowly, with max(64, tail_order) points. */
    int tail_rays;   /* near-field tail: rays between the north and east directions; 0 -> 9 */
    int tensor_m2l;  /* mixed path, p <= 14: M2L on the tcgen05 tensor cores, FP32 accumulation
                        in tensor memory -- 16-vector applies on uniform trees: every level and
                        image term in one launch, FP16 hi/lo operands with a power-of-two scale
                        per level; 1-4 vectors: the free-space stencil per level, TF32 hi/lo;
                        1 on, 0 off */
    int kernel;      /* lm_kernel: the operator the tree applies; 0 -> LM_KERNEL_G */
    int autotune;    /* LM_MIXED: run lm_autotune at the end of lm_build_tree; 0 off (default) */
    int top_bc;      /* lm_boundary of the interface y = 0; 0 -> LM_BC_TRANSMISSION (layer 1, k1) */
    int bottom_bc;   /* lm_boundary of the interface y = -d; 0 -> LM_BC_TRANSMISSION (layer 3, k3) */
    double top_alpha;    /* LM_BC_IMPEDANCE at y = 0: alpha (real, finite) */
    double bottom_alpha; /* LM_BC_IMPEDANCE at y = -d: alpha */
    int adaptive;    /* 1: adaptive tree (Algorithm 1, step 1) -- a box holding more than
                        leaf_target points is split into its four children while its level is
                        below depth (-1 -> 14); boxes of different levels interact through
                        lists built by a dual traversal (see lm_build_tree).  Both precisions:
                        LM_MIXED trees run M2L between any two levels on the CUDA-core staged
                        contraction, the other steps on the box lists.  0 (default): uniform depth. */
    int m2l_fp64;    /* LM_FP64 trees: 1 runs the M2L, M2M and L2L contractions in IEEE FP64;
                        0 (default) runs them in double-float on the FP32 pipes -- each value a pair of
                        FP32 numbers (48-bit significand), exact products by fma and
                        error-free sums, densities scaled by a power of two per apply so
                        the expansions stay inside FP32's exponent range; about 1e-14
                        relative, and several times the FP64 pipe's rate on GB300. */
    int tensor_leaf; /* LM_MIXED uniform trees, p <= 14, applies of 5-16 vectors: the leaf step's
                        multiply-adds over the vectors (direct S2T pairs and L2T) on the tcgen05
                        tensor cores, the kernel values on the CUDA cores (FP16 hi/lo split of both
                        factors with power-of-two scales, FP32 accumulation); 1 on
                        (lm_options_default), 0 off */
} lm_options;

/* Other media (Sec. 3, Examples 2 and 3): an interface of the middle layer
 * may be a wall with a one-sided condition instead of a transmission to an
 * outer layer.  Its reflection coefficient replaces R_t or R_b:
 *   LM_BC_DIRICHLET  u = 0          R = -1
 *   LM_BC_NEUMANN    du/dn = 0      R = +1
 *   LM_BC_IMPEDANCE  du/dn - i k2 alpha u = 0, n the layer's outward normal:
 *                    R = (s2 + i k2 alpha)/(s2 - i k2 alpha), the image term
 *                    of Eq. (halfspace)
 * A half-space is a wall on top and k3 = k2 below (R_b = 0), with d any
 * depth below the points.  With a wall, k1 (or k3) is not used but must
 * still be finite and positive. */
typedef enum { LM_BC_TRANSMISSION = 0, LM_BC_DIRICHLET = 1, LM_BC_NEUMANN = 2, LM_BC_IMPEDANCE = 3 } lm_boundary;

typedef enum {
    LM_KERNEL_G = 0,     /* G = free space + reflected part (Sec. 3, Example 4; reading R1) */
    LM_KERNEL_DG_DD = 1  /* dG/dd at fixed points: the reflected part with each image density
                            sigma_m replaced by d/dd[sigma_m e^{-s2 c_m}] e^{s2 c_m}
                            = -2 s2 (E/(1-E) + [m != tt]) sigma_m, E = R_t R_b e^{-2 d s2},
                            c_m the d-dependent part of h_m (0 for tt, 2d otherwise); the free
                            part has no d and is left out.  Same FMM, same lists. */
} lm_kernel;

typedef struct lm_medium_s *lm_medium; /* opaque, library-owned */
typedef struct lm_tree_s *lm_tree;     /* opaque, library-owned */

typedef struct {
    int64_t n;        /* number of points */
    int R;            /* number of d x d roots along x */
    int depth;        /* L: leaves are at level L, width d 2^-L */
    int p;            /* expansion order */
    double x_origin;  /* left edge of the first root: floor(min x / d) d */
    int64_t nleaf;    /* R 4^L */
    int precision;    /* lm_precision */
    int max_nvec;
    int64_t device_bytes; /* device memory held by the tree handle */
    int64_t nbox;     /* boxes of every level (uniform: sum over l of R 4^l) */
    int adaptive;     /* 1 for an adaptive tree: depth is then its deepest level and
                         nleaf its number of leaves */
    int tensor_leaf;  /* 1 when applies of 5-16 vectors run the leaf step's multiply-adds on
                         the tensor cores (LM_MIXED uniform tree, tile-form M2L, p <= 14,
                         k2 w <= 2 at the leaves, lm_options.tensor_leaf set) */
} lm_tree_info;

/* Fill *opt with the defaults listed above. LM_EINVAL if opt is NULL. */
lm_status lm_options_default(lm_options *opt);

/*
 * create_medium -- the three-layer medium of Sec. 3, Example 4.
 *   k1, k2, k3: real wave numbers (> 0, finite); d: middle-layer thickness (> 0).
 *   opt: NULL for defaults; copied, not retained.
 *   out: receives a new handle (host object, no device work).
 * Errors: LM_EINVAL for a non-positive or non-finite parameter or bad option.
 */
lm_status lm_create_medium(double k1, double k2, double k3, double d, const lm_options *opt,
                           lm_medium *out);

/*
 * build_tree -- Algorithm 1, step 1: the adaptive hierarchical tree and the
 * precomputed tables.  Here the tree is a forest of R roots, each a d x d
 * square, tiling [x_origin, x_origin + R d) x (-d, 0), refined uniformly to
 * depth L; box edges lie on both interfaces.  Builds, on the device and on
 * `stream`: point keys and the tree order (sorted by leaf, ties by input
 * index), interaction lists (free space and the four image lattices), the
 * M2M / L2L / M2L translation tables (Lemmas M2M, M2L, L2L) and the
 * near-field Sommerfeld quadrature tables (Sec. 4.2, Sec. 5 first contour).
 *   x, y: device arrays of n doubles (point coordinates, input order); read
 *         during the call only.
 *   n >= 1.
 * Synchronises `stream` (host needs the x extent and a validity flag).
 *
 * With opt.adaptive = 1 the roots are refined only where the points are: a box
 * (level l, column c, row r) with more than leaf_target points and l < depth
 * has all four children; boxes are numbered level by level, within a level by
 * r * (R 2^l) + c; points are ordered by leaf number, then input index.  The
 * lists come from a dual traversal per term from every pair of roots: a target
 * box and the image of a source box (row mapped as for the uniform lists, at
 * the source's level) with max(|dx|, |dy|) >= w_t + w_s between centres are a
 * V entry (M2L between their levels); two leaves that are not are a U entry;
 * otherwise the larger box is split (both when the levels are equal).  This
 * tree and its lists are built on the host (the points are copied back once);
 * tables, lists and expansions are on the device.
 * Errors: LM_EINVAL if a point is non-finite or not strictly inside
 * -d < y < 0, or if the x extent needs more than 2^30 roots (checked in double
 * precision before the count becomes an integer); LM_ENOMEM; LM_ENOTSUP if a
 * leaf holds more than 8192 points; LM_ECUDA.
 */
lm_status lm_build_tree(lm_medium m, const double *x, const double *y, int64_t n, void *stream,
                        lm_tree *out);

/*
 * apply -- u = G q by the FMM (Algorithm 1, steps 2-4).
 *   q: device, complex128 [nvec][n] densities in input order.
 *   u: device, complex128 [nvec][n] output (overwritten), input order; must
 *      not overlap q.
 *   nvec >= 1.
 * Errors: LM_EINVAL (nvec < 1, NULL or overlapping buffers), LM_ECUDA.
 */
lm_status lm_apply(lm_tree t, const void *q, int nvec, void *u, void *stream);

/*
 * apply_adjoint -- w = G^H v.  The kernel is reciprocal, G(x, x0) = G(x0, x)
 * (Sec. 3: every term depends on x - x0 through lambda^2-even integrands and
 * on y, y0 symmetrically), so G^H v = conj(G conj(v)); the conjugations are
 * fused into the permutation kernels.  Arguments and errors as lm_apply.
 */
lm_status lm_apply_adjoint(lm_tree t, const void *v, int nvec, void *w, void *stream);

/* Geometry of a built tree (host struct). */
lm_status lm_get_tree_info(lm_tree t, lm_tree_info *info);

/*
 * tree_export -- copy the tree order to host memory (synchronises `stream`).
 *   perm: host int64[n], tree position -> input index (may be NULL).
 *   leaf_start: host int64[nleaf + 1], first tree position of each leaf (may be NULL);
 *               adaptive trees: int64[nbox + 1], the points of box b are tree positions
 *               leaf_start[b] .. leaf_start[b + 1] - 1 (none for a box that is not a leaf).
 */
lm_status lm_tree_export(lm_tree t, int64_t *perm, int64_t *leaf_start, void *stream);

/*
 * list_export -- copy one interaction list to host memory as rows of
 * (target box, term, source box), box id = row * (R 2^l) + column, term
 * 0 = free space, 1 = tt, 2 = bb, 3 = tb, 4 = bt; rows ordered by target,
 * then term, then source (Algorithm 1: the interaction list of step 3 and
 * the direct-interaction list of step 4).
 *   which: 0 = V list of `level` (0..L), 1 = U list (leaf level; level ignored).
 *   Adaptive trees: box ids are those of lm_box_export, which = 0 gives the V
 *   list of every level at once and `level` is ignored.
 *   out: host int64[3 * cap]; *count receives the full length (rows written:
 *   min(cap, *count)).  Synchronises `stream`.
 */
lm_status lm_list_export(lm_tree t, int which, int level, int64_t *out, int64_t cap,
                         int64_t *count, void *stream);

/*
 * box_export -- the boxes of a tree as rows (level, column, row, leaf) in box-id
 * order: level by level, within a level by row * (R 2^l) + column (the uniform
 * tree lists every box of every level; leaf = 1 at level L).
 *   boxes: host int64[4 * cap]; *count receives the number of boxes (rows
 *   written: min(cap, *count)).  Host-only; no device work.
 */
lm_status lm_box_export(lm_tree t, int64_t *boxes, int64_t cap, int64_t *count);

/*
 * adaptive_plan -- the host half of lm_build_tree with opt.adaptive = 1, from
 * HOST arrays and without device work (no GPU needed): validation, the grid of
 * roots, the adaptive boxes, the point order and the V and U lists, exactly as
 * the tree that lm_build_tree builds from the same points and options.
 *   x, y: host double[n], n >= 1; d > 0: the layer thickness; leaf_target >= 1;
 *   depth: the depth limit, -1 (14) or 0..14.
 *   x_origin, R, nbox, nv, nu: receive the grid and the counts (each may be NULL).
 *   boxes: int64[4 * box_cap], rows (level, column, row, leaf) in box-id order
 *   (min(box_cap, nbox) rows written); pstart: int64[nbox + 1], written only when
 *   box_cap >= nbox (may be NULL); perm: int64[n] (may be NULL).
 *   vrows / urows: int64[3 * v_cap] / [3 * u_cap], rows (target box, term, source
 *   box) sorted, min(cap, count) written; a cap of 0 with a NULL array asks only
 *   for the count.
 * Errors: LM_EINVAL for bad arguments or a point that is non-finite or not
 * strictly inside -d < y < 0; LM_ENOTSUP beyond 2^22 roots.
 */
lm_status lm_adaptive_plan(const double *x, const double *y, int64_t n, double d, int leaf_target, int depth,
                           double *x_origin, int *R, int64_t *nbox, int64_t *boxes, int64_t box_cap,
                           int64_t *perm, int64_t *pstart, int64_t *nv, int64_t *vrows, int64_t v_cap,
                           int64_t *nu, int64_t *urows, int64_t u_cap);

/*
 * m2l_table_export -- copy one M2L translation matrix A_pq (Lemma M2L for
 * term 1..4, the free-space translation for term 0), unscaled, p, q in
 * -P..P, to host memory as complex128 [(2P+1)][(2P+1)] (row p, column q).
 * The class is given by level, term, column offset dc = target col - source
 * col and row offset dr = target row - image row (image rows as in
 * lm_list_export's lists).  LM_EINVAL if that class is not in any list;
 * LM_ENOTSUP for an adaptive tree.
 * Synchronises `stream`.
 */
lm_status lm_m2l_table_export(lm_tree t, int level, int term, int dc, int dr, double *out,
                              void *stream);

/*
 * Phase profiling (instrumentation, no counterpart in the paper).  While
 * enabled, lm_apply records a pair of CUDA events around each phase on the
 * launching stream: 0 permute, 1 S2M, 2 M2M, 3 M2L, 4 L2L, 5 L2T + S2T,
 * 6 mixed-precision refinement.
 *   profile_begin: enable for at most max_applies applies (allocates host
 *     event handles only; LM_EINVAL if max_applies < 1).
 *   profile_end: synchronise on the recorded events, write per-phase total
 *     milliseconds and kernel-launch counts into host arrays of nphase
 *     entries (either may be NULL), and disable.  Applies beyond max_applies
 *     are not recorded.
 */
lm_status lm_profile_begin(lm_tree t, int max_applies);
lm_status lm_profile_end(lm_tree t, double *ms, int64_t *launches, int nphase, int *applies);

/*
 * Peak probe (instrumentation): time `iters` dependent-chain iterations of
 * one arithmetic unit on every SM and return the achieved operation rate.
 *   kind: 0 = FP64 FMA, 1 = FP32 FMA, 2 = FP32 sin/cos (SFU path), 3 = FP64 exp.
 *   *rate receives operations per second (an FMA counts 2 flops for kinds
 *   0 and 1, i.e. the value is FLOP/s).  Synchronises `stream`.
 */
lm_status lm_peak_probe(int kind, int64_t iters, void *stream, double *rate);

/*
 * tree_order_noalloc -- the tree order that lm_build_tree computes (points
 * sorted by leaf of the d x d strip forest refined to depth L, ties broken by
 * input index), computed without allocating any memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot allocate --
 * code that may only allocate at start-up (real-time or certified
 * pipelines), code running inside an allocator or memory-pool callback where
 * a nested cudaMalloc would re-enter the allocator, and processes whose
 * device memory is entirely reserved by another framework's caching
 * allocator.
 *   x, y: device arrays of n doubles (input order); 1 <= n <= 1,048,576.
 *   d > 0: root size (layer thickness); depth: 0..14, with R 4^depth <= 262,144 leaves.
 *   perm: device int64[n], receives tree position -> input index.
 *   leaf_start: device int64[leaf_cap]; receives nleaf + 1 = R 4^depth + 1
 *     offsets (LM_EINVAL, with *R and *x_origin set, if leaf_cap is smaller).
 *   x_origin, R: host outputs (left edge of the first root, number of roots).
 * Scratch: one file-scope device array of about 6.3 MB, resident on every GPU
 * that loads the library until the process exits.  The first call on a
 * device looks up that array's device address (cudaGetSymbolAddress) with
 * the device current, and caches it for the life of the process: after
 * cudaDeviceReset (or a reset of the primary context) the module is loaded
 * again, the array may move, and this entry point must not be called again
 * in that process.  The array is shared by all calls and keeps the last
 * call's contents (the counters are cleared at the start of each call), so
 * calls whose device work overlaps -- on different streams or threads --
 * race and must be serialised by the caller.  Calls no cudaMalloc or
 * cudaFree and no allocating library routine.  Synchronises `stream`.
 * Errors: LM_EINVAL for sizes beyond the limits above (the leaf count is
 * checked in double precision before any integer conversion, so a huge x
 * extent or a tiny d is rejected, not wrapped), a non-finite d, NULL
 * pointers or invalid points; LM_ENOTSUP if a leaf holds more than 8192
 * points; LM_ECUDA.
 */
lm_status lm_tree_order_noalloc(const double *x, const double *y, int64_t n, double d, int depth,
                                int64_t *perm, int64_t *leaf_start, int64_t leaf_cap, double *x_origin,
                                int *R, void *stream);

/*
 * Batched apply: the applies of `count` built trees -- each with its own
 * medium, size, expansion order and precision -- captured once into one CUDA
 * graph and replayed as a single launch.  Inside the graph the trees are
 * forked over up to 8 streams so that small instances run concurrently.
 *   batch_create: trees[i], q[i] (device, complex128 [nvec[i]][n_i]), u[i]
 *     (device, same layout, not overlapping q[i]) for i < count; c64 (host,
 *     nullable): c64[i] != 0 makes entry i's buffers complex64 (LM_MIXED trees).  The buffer
 *     addresses are bound at capture: every launch reads q[i] and writes u[i].
 *     The trees must be distinct and outlive the batch, and no other apply may
 *     use them while a launch is in flight.  Profiling must be off on them.
 *   batch_launch: enqueue the whole batch on `stream`.
 *   batch_info: the number of kernel launches one batch_launch makes (kernel
 *     nodes of the graph) and whether the batch runs one M2L launch over
 *     every tree (joint_m2l = 1: at least two LM_MIXED trees that all use the
 *     tile-form M2L at one expansion order and vector width); either output
 *     may be NULL.
 * Errors: LM_EINVAL for bad arguments, LM_ECUDA if capture or instantiation fails.
 */
typedef struct lm_batch_s *lm_batch;
lm_status lm_batch_create(const lm_tree *trees, int count, const void *const *q, const int *nvec,
                          void *const *u, const int *c64, lm_batch *out);
lm_status lm_batch_launch(lm_batch b, void *stream);
lm_status lm_batch_info(lm_batch b, int64_t *kernels, int *joint_m2l);
void lm_batch_destroy(lm_batch b);

/*
 * autotune -- choose, per level, the tile shape of the free-space M2L of an
 * LM_MIXED tree: the tcgen05 kernel (8 boxes x 16 vectors x 64 real orders
 * per tile) or the CUDA-core kernel with 2, 4 or 8 orders per thread (16
 * boxes x 4 vectors per row group), by timing each on the tree's own buffers
 * with CUDA events on `stream` (synchronises it).  The choice stays with the
 * tree.  choice, ms: host arrays of depth + 1 entries, or NULL; choice[l] =
 * -1 (no stencil at level 0), 0 (tensor cores) or the orders per thread;
 * ms[l] = the chosen kernel's time per launch.  On an LM_FP64 tree nothing
 * is tuned and every choice is -1.  Not to be called while an apply of the
 * tree is in flight.  Errors: LM_EINVAL (NULL tree), LM_ECUDA.
 */
lm_status lm_autotune(lm_tree t, void *stream, int *choice, float *ms);

/*
 * apply_c64, apply_adjoint_c64 -- lm_apply and lm_apply_adjoint with
 * complex64 (interleaved float re, im) densities and potentials, [nvec][n],
 * for LM_MIXED trees, whose arithmetic is FP32 already: halves the bytes moved
 * and copied per point.  Errors as lm_apply; LM_EINVAL on an LM_FP64 tree.
 */
lm_status lm_apply_c64(lm_tree t, const void *q, int nvec, void *u, void *stream);
lm_status lm_apply_adjoint_c64(lm_tree t, const void *v, int nvec, void *w, void *stream);

/*
 * apply_grad -- the field and its target gradient, FP64 trees only:
 *   u_i  = sum_j G(x_i, x_j) q_j                (as lm_apply)
 *   ux_i = sum_j d/dx G(x, x_j)|_{x = x_i} q_j  (sources held fixed)
 *   uy_i = sum_j d/dy G(x, x_j)|_{x = x_i} q_j
 * The far field differentiates the local expansion (Eq. (local)) with
 * (d/dx +- i d/dy) J_n(kr) e^{i n theta} = -+k J_{n+-1}(kr) e^{i (n+-1) theta};
 * the free near field uses (i/4)(-k) H1(k r); the reflected near field
 * multiplies the Sommerfeld integrand by i lambda (x) and -s2 dh_m/dy (y),
 * on tail rays of max(64, tail_order) points.  Beside a wall the image term
 * R_inf (i/4) H0(k2 rho) and its H1 derivatives are added in closed form; an
 * impedance wall (beta = k2 alpha) also moves the part 2 i beta / s2 of the
 * y-derivative's integrand into the closed form -2 i beta (i/4) H0(k2 rho).
 * With reciprocity this gives every coordinate gradient of a misfit: for
 * J(u), g = dJ/d(Re u) + i dJ/d(Im u), dJ/dx_j = Re[conj(g_j) ux(q)_j +
 * q_j ux(conj g)_j] (and the same in y).
 *   q: device [nvec][n] complex128, input order; u (may be NULL), ux, uy:
 *   device [nvec][n] complex128, input order, not overlapping q.
 * Errors: as lm_apply; LM_ENOTSUP on an LM_MIXED tree.
 */
lm_status lm_apply_grad(lm_tree t, const void *q, int nvec, void *u, void *ux, void *uy, void *stream);

/*
 * misfit_grad -- every gradient of a real misfit J(u), u = G(x, y, d) q, from
 * g = dJ/d(Re u) + i dJ/d(Im u) (device [nvec][n] complex128, input order),
 * assembled by the library's kernels on `stream`:
 *   gq = G^H g = conj(G conj g)                        (lm_apply_adjoint);
 *   gx_j = Re sum_v [conj(g_vj) dx(G q_v)_j + q_vj dx(G conj g_v)_j], gy_j
 *        the same in y: the target gradient at x_j (lm_apply_grad) over the
 *        stacked vectors [q; conj g], with G(a, b) = G(b, a) (Sec. 3)
 *        turning the target derivative into the source-point derivative;
 *   gd = Re sum_v sum_i conj(g_vi) (dG/dd q_v)_i, from dtree: a tree built over
 *        the same points with kernel = LM_KERNEL_DG_DD; reduced in a fixed
 *        order (reproducible).
 *   q, g: device [nvec][n] complex128.  gq: device [nvec][n] complex128; gx,
 *   gy: device double [n]; gd: device double [1]; any output may be NULL (not
 *   computed).  dtree: needed only for gd.  workspace: device memory of at
 *   least lm_misfit_grad_workspace bytes, owned by the caller and needed
 *   only for gx, gy or gd; the library allocates nothing here.
 * Errors: LM_EINVAL for NULL inputs, nvec < 1, a short workspace, overlapping
 * outputs or a missing / mismatched dtree; LM_ENOTSUP for gx or gy on an
 * LM_MIXED tree (the target gradient is FP64 only); LM_ECUDA.
 */
lm_status lm_misfit_grad_workspace(lm_tree t, int nvec, size_t *bytes);
lm_status lm_misfit_grad(lm_tree t, lm_tree dtree, const void *q, const void *g, int nvec, void *gq, double *gx,
                         double *gy, double *gd, void *workspace, size_t ws_bytes, void *stream);

/*
 * Cross-layer operator (Sec. 3, Example 4 as printed): sources in layer 1,
 * targets in the middle layer,
 *     u_i = sum_j q_j [g_2^t + g_2^b](x_i, x_j),
 * g_2^t, g_2^b with the printed densities sigma_2^t, sigma_2^b, through the
 * FMM with two wave numbers: multipoles in k1 about the source boxes, local
 * expansions in k2 about the target boxes (Sec. 2.1), on a source and a target
 * tree sharing one lattice of d x d roots.  The medium must have kernel
 * LM_KERNEL_G and transmission interfaces.  Precision LM_FP64: every step in
 * FP64.  LM_MIXED: tables and near-field quadrature built in FP64; expansions,
 * translations and multiply-adds in FP32 (tables rounded once), near kernel
 * values evaluated in FP64 and rounded.
 *   build_cross: xs, ys (device, [ns]) sources with 0 < ys < d; xt, yt
 *     (device, [nt]) targets with -d < yt < 0.  Copies what it needs.
 *   cross_apply: q device complex128 [nvec][ns]; u device complex128 [nvec][nt].
 *   cross_info: sizes and the shared lattice (any output may be NULL).
 * Errors: LM_EINVAL for bad points or arguments, LM_ENOTSUP for another
 * medium kind, LM_ENOMEM, LM_ECUDA.
 */
typedef struct lm_cross_s *lm_cross;
lm_status lm_build_cross(lm_medium m, const double *xs, const double *ys, int64_t ns, const double *xt,
                         const double *yt, int64_t nt, void *stream, lm_cross *out);
lm_status lm_cross_apply(lm_cross c, const void *q, int nvec, void *u, void *stream);
lm_status lm_cross_info(lm_cross c, int64_t *ns, int64_t *nt, int *R, int *depth, double *x_origin);
void lm_destroy_cross(lm_cross c);

/*
 * sync_status -- synchronise `stream` and report device-side failures of the
 * applies enqueued so far on tree t: LM_ETIMEOUT if a bounded wait inside a
 * tensor-core kernel gave up (the result of that apply is invalid), LM_OK
 * otherwise.  Clears the recorded failure.
 */
lm_status lm_sync_status(lm_tree t, void *stream);

/*
 * set_poll_limit -- failure-path check of the bounded waits (no counterpart
 * in the paper).  For the next 16-vector apply of an LM_MIXED tree that runs
 * the tile-form tensor-core M2L, the MMA issuer's first wait for its operands
 * polls at most `limit` times (0: gives up at once) before it reports a
 * timeout; every other wait, including the waits that let copies and MMAs in
 * flight finish before tensor memory is freed, keeps the library's limit.
 * The setting applies to one apply and is then cleared; limit < 0 clears it.
 * That apply's result is invalid and lm_sync_status returns LM_ETIMEOUT.
 * Errors: LM_EINVAL (NULL tree).
 */
lm_status lm_set_poll_limit(lm_tree t, int limit);

void lm_destroy_tree(lm_tree t);
void lm_destroy_medium(lm_medium m);
const char *lm_status_string(lm_status s);
const char *lm_last_error(void); /* thread-local; never NULL */

#ifdef __cplusplus
}
#endif
#endif
