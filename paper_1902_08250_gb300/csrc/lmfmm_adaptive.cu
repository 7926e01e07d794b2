// lmfmm_adaptive.cu -- Algorithm 1, step 1 with an adaptive hierarchical tree:
// the d x d roots of the strip forest are refined only where the points are.
//
// Reading of the paper's "adaptive hierarchical tree": a box (level l, column
// c, row r) holding more than s = leaf_target points at a level below the
// depth limit is split into all four of its children.  A point's cell at
// level l is (floor((x - x0)/w_l), floor(-y/w_l)), clamped to the lattice,
// w_l = d 2^-l, exactly as for the uniform tree.  Boxes are numbered level by
// level and, within a level, by r * (R 2^l) + c; points are ordered by the
// number of their leaf, then by input index.
//
// Lists by dual traversal, per term m (0 free, 1 tt, 2 bb, 3 tb, 4 bt), from
// every pair of roots: a target box and the image of a source box (its row
// mapped through img_row at the source's level) are well separated when the
// larger of |dx|, |dy| between their centres is at least w_t + w_s -- then the
// pair is a V entry (M2L, Lemma M2L or the free-space translation); otherwise
// two leaves make a U entry (direct interaction, step 4); otherwise the larger
// box is split (never a leaf; both when the levels are equal).  On a uniformly
// refined tree this reproduces the uniform V and U lists level by level.
//
// The build runs on the host (the tree is data-dependent and small next to
// the points); its tables, lists and expansions live on the device.
#include <math.h>
#include <string.h>
#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "internal.h"
#include "tables.cuh"

namespace {

struct HBox {
    int level;
    int64_t col, row;
    int64_t lo, hi; // range of the Morton-sorted points
    int32_t parent, kpos;
    int32_t child[4];
    bool leaf;
};

// bit j of v -> bit 2j
uint64_t spread_bits(uint64_t v)
{
    uint64_t r = 0;
    for (int j = 0; j < 32; ++j) r |= ((v >> j) & 1ull) << (2 * j);
    return r;
}

struct Builder {
    int64_t n;
    double d, x0;
    int R, Lmax, s;
    std::vector<uint64_t> key;   // sorted Morton keys at level Lmax
    std::vector<int64_t> order;  // input index of each sorted key
    std::vector<HBox> box;
    std::vector<int64_t> lev_start;

    int64_t find_range(uint64_t k) const
    {
        return std::lower_bound(key.begin(), key.end(), k) - key.begin();
    }

    void build(const std::vector<double> &x, const std::vector<double> &y)
    {
        const double wL = ldexp(d, -Lmax);
        const int64_t ncolL = (int64_t)R << Lmax, nrowL = (int64_t)1 << Lmax;
        std::vector<std::pair<uint64_t, int64_t>> kv(n);
        for (int64_t i = 0; i < n; ++i) {
            int64_t c = (int64_t)floor((x[i] - x0) / wL), r = (int64_t)floor(-y[i] / wL);
            c = std::min(std::max(c, (int64_t)0), ncolL - 1);
            r = std::min(std::max(r, (int64_t)0), nrowL - 1);
            const uint64_t root = (uint64_t)(c >> Lmax), cl = (uint64_t)(c - ((int64_t)root << Lmax));
            kv[i] = {(root << (2 * Lmax)) | (spread_bits((uint64_t)r) << 1) | spread_bits(cl), i};
        }
        std::sort(kv.begin(), kv.end());
        key.resize(n);
        order.resize(n);
        for (int64_t i = 0; i < n; ++i) {
            key[i] = kv[i].first;
            order[i] = kv[i].second;
        }
        box.clear();
        lev_start.assign(1, 0);
        for (int64_t c = 0; c < R; ++c) {
            HBox b{};
            b.level = 0;
            b.col = c;
            b.row = 0;
            b.lo = find_range((uint64_t)c << (2 * Lmax));
            b.hi = find_range((uint64_t)(c + 1) << (2 * Lmax));
            b.parent = -1;
            b.kpos = 0;
            b.leaf = true;
            for (int k = 0; k < 4; ++k) b.child[k] = -1;
            box.push_back(b);
        }
        lev_start.push_back((int64_t)box.size());
        for (int l = 0; l < Lmax; ++l) {
            const int64_t lo = lev_start[l], hi = lev_start[l + 1];
            const int sh = 2 * (Lmax - l - 1); // key bits below the children's level
            std::vector<HBox> next;
            for (int64_t b = lo; b < hi; ++b) {
                if (box[b].hi - box[b].lo <= s) continue;
                box[b].leaf = false;
                const uint64_t pre = key[box[b].lo] >> (sh + 2); // the box's own prefix
                for (int k = 0; k < 4; ++k) {
                    HBox ch{};
                    ch.level = l + 1;
                    ch.col = 2 * box[b].col + (k & 1);
                    ch.row = 2 * box[b].row + (k >> 1);
                    ch.lo = find_range(((pre << 2) + (uint64_t)k) << sh);
                    ch.hi = find_range(((pre << 2) + (uint64_t)(k + 1)) << sh);
                    ch.parent = (int32_t)b;
                    ch.kpos = k;
                    ch.leaf = true;
                    for (int j = 0; j < 4; ++j) ch.child[j] = -1;
                    next.push_back(ch);
                }
            }
            if (next.empty()) break;
            const int64_t ncol1 = (int64_t)R << (l + 1);
            std::sort(next.begin(), next.end(), [&](const HBox &a, const HBox &b) {
                return a.row * ncol1 + a.col < b.row * ncol1 + b.col;
            });
            for (const HBox &ch : next) {
                box[ch.parent].child[ch.kpos] = (int32_t)box.size();
                box.push_back(ch);
            }
            lev_start.push_back((int64_t)box.size());
        }
    }

    // separation of target t and the image of source s under term m, in half
    // widths of the finer of the two levels (exact integer arithmetic)
    void offsets(int64_t t, int64_t sb, int m, int64_t *dx2, int64_t *dy2, int64_t *lim) const
    {
        const HBox &A = box[t], &B = box[sb];
        const int lf = std::max(A.level, B.level);
        const int64_t SA = (int64_t)1 << (lf - A.level), SB = (int64_t)1 << (lf - B.level);
        const int64_t ri = img_row(m, B.row, (int64_t)1 << B.level);
        *dx2 = (2 * A.col + 1) * SA - (2 * B.col + 1) * SB;
        *dy2 = (2 * A.row + 1) * SA - (2 * ri + 1) * SB;
        *lim = 2 * (SA + SB);
    }
    bool separated(int64_t t, int64_t sb, int m) const
    {
        int64_t dx2, dy2, lim;
        offsets(t, sb, m, &dx2, &dy2, &lim);
        return std::max(dx2 < 0 ? -dx2 : dx2, dy2 < 0 ? -dy2 : dy2) >= lim;
    }

    void visit(int64_t t, int64_t sb, int m, std::vector<std::tuple<int64_t, int, int64_t>> &V,
               std::vector<std::tuple<int64_t, int, int64_t>> &U) const
    {
        if (separated(t, sb, m)) {
            V.emplace_back(t, m, sb);
            return;
        }
        const HBox &A = box[t], &B = box[sb];
        if (A.leaf && B.leaf) {
            U.emplace_back(t, m, sb);
            return;
        }
        if (A.leaf || (!B.leaf && B.level < A.level)) {
            for (int k = 0; k < 4; ++k) visit(t, B.child[k], m, V, U);
        } else if (B.leaf || A.level < B.level) {
            for (int k = 0; k < 4; ++k) visit(A.child[k], sb, m, V, U);
        } else {
            for (int k = 0; k < 4; ++k)
                for (int j = 0; j < 4; ++j) visit(A.child[k], B.child[j], m, V, U);
        }
    }
};

typedef std::vector<std::tuple<int64_t, int, int64_t>> Rows;

// The whole host side of the build: validates the points, sets the grid of
// roots, builds the boxes, the point order (by leaf, then input index) and the
// sorted V and U lists.  No device work.
lm_status plan(const double *hx, const double *hy, int64_t n, double d, int s, int Lmax, const char *who,
               Builder &B, std::vector<int64_t> &perm, std::vector<int64_t> &pstart, Rows &V, Rows &U)
{
    double mn = hx[0], mx = hx[0];
    for (int64_t i = 0; i < n; ++i) {
        if (!isfinite(hx[i]) || !isfinite(hy[i]) || !(hy[i] < 0.0) || !(hy[i] > -d)) {
            lm_set_error("%s: a point is non-finite or not strictly inside -d < y < 0", who);
            return LM_EINVAL;
        }
        mn = fmin(mn, hx[i]);
        mx = fmax(mx, hx[i]);
    }
    const double f0 = floor(mn / d), f1 = floor(mx / d);
    if (f1 - f0 + 1.0 > (double)(1 << 22)) {
        lm_set_error("%s: the points span more than 2^22 roots; not supported by the adaptive tree", who);
        return LM_ENOTSUP;
    }
    B.n = n;
    B.d = d;
    B.x0 = f0 * d;
    B.R = (int)(f1 - f0) + 1;
    B.Lmax = Lmax;
    B.s = s;
    std::vector<double> x(hx, hx + n), y(hy, hy + n);
    B.build(x, y);
    const int64_t nbox = (int64_t)B.box.size();
    if (nbox >= INT32_MAX / 4) {
        lm_set_error("%s: %lld boxes is beyond this build", who, (long long)nbox);
        return LM_ENOTSUP;
    }
    perm.resize(n);
    pstart.resize(nbox + 1);
    int64_t pos = 0;
    for (int64_t b = 0; b < nbox; ++b) {
        pstart[b] = pos;
        if (!B.box[b].leaf) continue;
        std::vector<int64_t> idx(B.order.begin() + B.box[b].lo, B.order.begin() + B.box[b].hi);
        std::sort(idx.begin(), idx.end());
        for (int64_t i : idx) perm[pos++] = i;
    }
    pstart[nbox] = pos;
    V.clear();
    U.clear();
    for (int64_t tb = 0; tb < B.R; ++tb)
        for (int64_t sb = 0; sb < B.R; ++sb)
            for (int m = 0; m < 5; ++m) B.visit(tb, sb, m, V, U);
    std::sort(V.begin(), V.end());
    std::sort(U.begin(), U.end());
    return LM_OK;
}

template <typename T>
lm_status upload(lm_tree_s *t, T **dst, const std::vector<T> &src, cudaStream_t st)
{
    lm_status s = lm_dalloc(t, dst, src.size());
    if (s != LM_OK) return s;
    if (!src.empty())
        LM_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return LM_OK;
}

} // namespace

// ---------------------------------------------------------------------------
// M2L tables of the adaptive lists.  A class is (term, target level lt, source
// level ls, centre offsets in half widths of the finer level); its table is
// scaled by S_lt(p) S_ls(q), S_l(n) = (k w_l / 2)^|n| / |n|!, so that it acts
// on the scaled multipole of the source box and yields the scaled local
// expansion of the target box.
//   free term: A_pq = (i/4) H_{q-p}(k rho) e^{i (q-p) theta}, (rho, theta) the
//              polar form of target centre - source centre (Rokhlin's translation);
//   image terms: Lemma M2L with dx = x_t - x_s and h the image height.
// ---------------------------------------------------------------------------
__global__ void k_free_m2l_a(double k, int P, const double *cdx, const double *cdy, const int *clt,
                             const int *cls, int ncls, const double *scales, zd *tab)
{
    const int np = 2 * P + 1;
    const int ci = blockIdx.y;
    if (ci >= ncls) return;
    const double cx = cdx[ci], cy = cdy[ci];
    const double rho = hypot(cx, cy), th = atan2(cy, cx);
    const double *st = scales + (int64_t)clt[ci] * (P + 1), *ss = scales + (int64_t)cls[ci] * (P + 1);
    zd *T = tab + (int64_t)ci * np * np;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < np * np; idx += gridDim.x * blockDim.x) {
        const int p = idx / np - P, q = idx % np - P;
        const int n = q - p, a = n < 0 ? -n : n;
        double jv = jn(a, k * rho), yv = yn(a, k * rho);
        if (n < 0 && (a & 1)) {
            jv = -jv;
            yv = -yv;
        }
        const double s = st[p < 0 ? -p : p] * ss[q < 0 ? -q : q];
        const zd h = {-0.25 * yv * s, 0.25 * jv * s}; // (i/4)(J + iY) S_t S_s
        const zd e = {cos(n * th), sin(n * th)};
        T[idx] = h * e;
    }
}

__global__ void __launch_bounds__(256) k_image_m2l_a(MediumD m, int P, const int *cterm, const double *cdx,
                                                     const double *ch, const int *clt, const int *cls,
                                                     int ncls, zd *tab, int *flag)
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
    const double sct = m.k2 * ldexp(m.d, -clt[ci]), scs = m.k2 * ldexp(m.d, -cls[ci]);
    m2l_table_body(sigf, km, kmin, m.k2, m.k2, P, sct, scs, tau, vs, cdx[ci], ch[ci], 0.0,
                   tab + (int64_t)ci * (2 * P + 1) * (2 * P + 1), flag);
}

#define TRY_A(x)                    \
    do {                            \
        lm_status s_ = (x);         \
        if (s_ != LM_OK) return s_; \
    } while (0)

lm_status lm_setup_adaptive(lm_tree_s *t, const double *x, const double *y, cudaStream_t st)
{
    const int64_t n = t->n;
    const double d = t->med.d;
    const int P = t->p, np = 2 * P + 1;
    AdaptTree &A = t->at;
    t->adaptive = true;
    TRY_A(lm_dalloc(t, &t->dflag, 4));
    LM_CUDA(cudaMemsetAsync(t->dflag, 0, 4 * sizeof(int), st));
    // points to the host
    std::vector<double> hx(n), hy(n);
    LM_CUDA(cudaMemcpyAsync(hx.data(), x, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaMemcpyAsync(hy.data(), y, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    Builder B;
    std::vector<int64_t> perm, pstart;
    Rows V, U;
    TRY_A(plan(hx.data(), hy.data(), n, d, t->med.opt.leaf_target, t->med.opt.depth >= 0 ? t->med.opt.depth : 14,
               "build_tree", B, perm, pstart, V, U));
    t->x0 = B.x0;
    t->R = B.R;
    const int64_t nbox = (int64_t)B.box.size();
    A.nbox = nbox;
    A.lev_start = B.lev_start;
    t->L = (int)A.lev_start.size() - 2;
    // boxes: geometry, links, point ranges; points in tree order
    std::vector<double> bcx(nbox), bcy(nbox), bw(nbox), xs(n), ys(n);
    std::vector<int32_t> par(nbox), pos(nbox), chl(4 * nbox), leaves, nonleaf;
    A.hbox.resize(4 * nbox);
    A.nl_start.assign(1, 0);
    for (int64_t b = 0; b < nbox; ++b) {
        const HBox &h = B.box[b];
        const double w = ldexp(d, -h.level);
        bw[b] = w;
        bcx[b] = t->x0 + (h.col + 0.5) * w;
        bcy[b] = -(h.row + 0.5) * w;
        par[b] = h.parent;
        pos[b] = (int32_t)((h.row & 1) * 2 + (h.col & 1));
        for (int k = 0; k < 4; ++k) chl[4 * b + k] = h.child[k];
        A.hbox[4 * b] = h.level;
        A.hbox[4 * b + 1] = h.col;
        A.hbox[4 * b + 2] = h.row;
        A.hbox[4 * b + 3] = h.leaf ? 1 : 0;
        if (h.leaf) leaves.push_back((int32_t)b);
    }
    for (int64_t i = 0; i < n; ++i) {
        xs[i] = hx[perm[i]];
        ys[i] = hy[perm[i]];
    }
    for (int l = 0; l <= t->L; ++l) {
        for (int64_t b = A.lev_start[l]; b < A.lev_start[l + 1]; ++b)
            if (!B.box[b].leaf) nonleaf.push_back((int32_t)b);
        A.nl_start.push_back((int64_t)nonleaf.size());
    }
    A.nleaf = (int64_t)leaves.size();
    t->nleaf = A.nleaf;
    // V classes and CSR
    std::map<std::tuple<int, int, int, int64_t, int64_t>, int> cmap;
    std::vector<int64_t> vstart(nbox + 1, 0);
    std::vector<int32_t> vsrc(V.size()), vslot(V.size()), vterm(V.size());
    for (size_t e = 0; e < V.size(); ++e) {
        const int64_t tb = std::get<0>(V[e]), sb = std::get<2>(V[e]);
        const int m = std::get<1>(V[e]);
        int64_t dx2, dy2, lim;
        B.offsets(tb, sb, m, &dx2, &dy2, &lim);
        auto key = std::make_tuple(m, B.box[tb].level, B.box[sb].level, dx2, dy2);
        auto it = cmap.find(key);
        int slot;
        if (it == cmap.end()) {
            slot = (int)cmap.size();
            cmap.emplace(key, slot);
            A.cls_term.push_back(m);
            A.cls_lt.push_back(B.box[tb].level);
            A.cls_ls.push_back(B.box[sb].level);
            A.cls_dx.push_back(dx2);
            A.cls_dy.push_back(dy2);
        } else {
            slot = it->second;
        }
        vstart[tb + 1]++;
        vsrc[e] = (int32_t)sb;
        vslot[e] = slot;
        vterm[e] = m;
    }
    for (int64_t b = 0; b < nbox; ++b) vstart[b + 1] += vstart[b];
    A.nv = (int64_t)V.size();
    A.lev_nv.resize(t->L + 1);
    for (int l = 0; l <= t->L; ++l) A.lev_nv[l] = vstart[A.lev_start[l + 1]] - vstart[A.lev_start[l]];
    // U list CSR; leaves with a reflected direct term get the factorised segment
    std::vector<int64_t> ustart(nbox + 1, 0);
    std::vector<int32_t> usrc(U.size()), uterm(U.size());
    std::vector<char> haspw(nbox, 0);
    for (size_t e = 0; e < U.size(); ++e) {
        const int64_t tb = std::get<0>(U[e]);
        const int m = std::get<1>(U[e]);
        if (m > 2) { // the tb / bt images lie at least d away: always separated at the roots
            lm_set_error("build_tree: internal error, a tb/bt pair reached the direct list");
            return LM_ECUDA;
        }
        ustart[tb + 1]++;
        usrc[e] = (int32_t)std::get<2>(U[e]);
        uterm[e] = m;
        if (m > 0) haspw[tb] = 1;
    }
    for (int64_t b = 0; b < nbox; ++b) ustart[b + 1] += ustart[b];
    t->nu = (int64_t)U.size();
    std::vector<int32_t> pwl;
    for (int64_t b = 0; b < nbox; ++b)
        if (haspw[b]) pwl.push_back((int32_t)b);
    A.npw = (int64_t)pwl.size();
    A.hpw = pwl;
    { // the factorised segment forms a source leaf's coefficients for the terms of its own entries, so
      // every tt (bb) source leaf must have a tt (bb) entry itself (the lists are symmetric per term)
        std::vector<char> hast(2 * (size_t)nbox, 0);
        for (const auto &r : U)
            if (std::get<1>(r) > 0) hast[2 * std::get<0>(r) + std::get<1>(r) - 1] = 1;
        for (const auto &r : U)
            if (std::get<1>(r) > 0 && !hast[2 * std::get<2>(r) + std::get<1>(r) - 1]) {
                lm_set_error("build_tree: internal error, a reflected source leaf lacks an entry of that term");
                return LM_ECUDA;
            }
    }
    // device copies
    TRY_A(upload(t, &A.cx, bcx, st));
    TRY_A(upload(t, &A.cy, bcy, st));
    TRY_A(upload(t, &A.w, bw, st));
    TRY_A(upload(t, &A.parent, par, st));
    TRY_A(upload(t, &A.pos, pos, st));
    TRY_A(upload(t, &A.child, chl, st));
    TRY_A(upload(t, &A.leaves, leaves, st));
    TRY_A(upload(t, &A.nonleaf, nonleaf, st));
    TRY_A(upload(t, &A.pwleaves, pwl, st));
    TRY_A(upload(t, &t->perm, perm, st));
    TRY_A(upload(t, &t->leaf_start, pstart, st));
    TRY_A(upload(t, &t->xs, xs, st));
    TRY_A(upload(t, &t->ys, ys, st));
    TRY_A(upload(t, &A.vstart, vstart, st));
    TRY_A(upload(t, &A.vsrc, vsrc, st));
    TRY_A(upload(t, &A.vslot, vslot, st));
    TRY_A(upload(t, &A.vterm, vterm, st));
    TRY_A(upload(t, &t->ustart, ustart, st));
    TRY_A(upload(t, &t->usrc, usrc, st));
    TRY_A(upload(t, &t->uterm, uterm, st));
    LM_CUDA(cudaStreamSynchronize(st)); // host vectors go out of scope
    // per-level scales and M2M / L2L tables, near-field quadrature
    TRY_A(lm_setup_levels(t, t->L, false, st));
    TRY_A(lm_setup_near(t, st));
    // class tables
    const int ncls = (int)A.cls_term.size();
    TRY_A(lm_dalloc(t, &A.tab, (size_t)std::max(1, ncls) * np * np));
    {
        MediumD md{t->med.k1,
                   t->med.k2,
                   t->med.k3,
                   d,
                   t->med.opt.kernel == LM_KERNEL_DG_DD,
                   {t->med.opt.top_bc, t->med.opt.bottom_bc},
                   {t->med.opt.top_alpha, t->med.opt.bottom_alpha}};
        std::vector<int> fidx, iidx;
        for (int i = 0; i < ncls; ++i) (A.cls_term[i] == 0 ? fidx : iidx).push_back(i);
        // free classes first, then image classes, each group in its own table range
        std::vector<int> cterm(ncls), clt(ncls), cls(ncls);
        std::vector<double> cdx(ncls), cdy(ncls);
        std::vector<int> ord;
        ord.insert(ord.end(), fidx.begin(), fidx.end());
        ord.insert(ord.end(), iidx.begin(), iidx.end());
        std::vector<int> newslot(ncls);
        for (int j = 0; j < ncls; ++j) {
            const int i = ord[j];
            newslot[i] = j;
            cterm[j] = A.cls_term[i];
            clt[j] = A.cls_lt[i];
            cls[j] = A.cls_ls[i];
            const double hw = ldexp(d, -std::max(A.cls_lt[i], A.cls_ls[i]) - 1); // half width, finer level
            cdx[j] = (double)A.cls_dx[i] * hw;
            // free term: y_t - y_s = -dy2 hw; image terms: h = |dy2| hw
            cdy[j] = A.cls_term[i] == 0 ? -(double)A.cls_dy[i] * hw : fabs((double)A.cls_dy[i]) * hw;
        }
        // renumber the classes so that the table order is the launch order
        {
            std::vector<int> t_term(ncls), t_lt(ncls), t_ls(ncls);
            std::vector<int64_t> t_dx(ncls), t_dy(ncls);
            for (int i = 0; i < ncls; ++i) {
                const int j = newslot[i];
                t_term[j] = A.cls_term[i];
                t_lt[j] = A.cls_lt[i];
                t_ls[j] = A.cls_ls[i];
                t_dx[j] = A.cls_dx[i];
                t_dy[j] = A.cls_dy[i];
            }
            A.cls_term.swap(t_term);
            A.cls_lt.swap(t_lt);
            A.cls_ls.swap(t_ls);
            A.cls_dx.swap(t_dx);
            A.cls_dy.swap(t_dy);
            for (auto &s : vslot) s = newslot[s];
            LM_CUDA(cudaMemcpyAsync(A.vslot, vslot.data(), vslot.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                                    st));
        }
        const int nf = (int)fidx.size(), ni = (int)iidx.size();
        int *dint;
        double *ddbl, *dsc;
        TRY_A(lm_dalloc(t, &dint, 3 * (size_t)ncls + 1));
        TRY_A(lm_dalloc(t, &ddbl, 2 * (size_t)ncls + 1));
        TRY_A(lm_dalloc(t, &dsc, (size_t)(t->L + 1) * (P + 1)));
        std::vector<int> hint;
        hint.insert(hint.end(), cterm.begin(), cterm.end());
        hint.insert(hint.end(), clt.begin(), clt.end());
        hint.insert(hint.end(), cls.begin(), cls.end());
        std::vector<double> hdbl;
        hdbl.insert(hdbl.end(), cdx.begin(), cdx.end());
        hdbl.insert(hdbl.end(), cdy.begin(), cdy.end());
        if (ncls > 0) {
            LM_CUDA(cudaMemcpyAsync(dint, hint.data(), hint.size() * sizeof(int), cudaMemcpyHostToDevice, st));
            LM_CUDA(cudaMemcpyAsync(ddbl, hdbl.data(), hdbl.size() * sizeof(double), cudaMemcpyHostToDevice, st));
        }
        for (int l = 0; l <= t->L; ++l)
            LM_CUDA(cudaMemcpyAsync(dsc + (size_t)l * (P + 1), t->lev[l].scale, (P + 1) * sizeof(double),
                                    cudaMemcpyDeviceToDevice, st));
        if (md.deriv) // the free part does not depend on d: its tables stay zero
            LM_CUDA(cudaMemsetAsync(A.tab, 0, (size_t)std::max(1, ncls) * np * np * sizeof(zd), st));
        if (nf > 0 && !md.deriv) {
            dim3 g((np * np + 255) / 256, nf);
            k_free_m2l_a<<<g, 256, 0, st>>>(t->med.k2, P, ddbl, ddbl + ncls, dint + ncls, dint + 2 * ncls, nf, dsc,
                                            A.tab);
        }
        if (ni > 0) {
            const size_t shm = (2 * TB_CHUNK * np + TB_CHUNK) * sizeof(zd);
            LM_CUDA(lm_raise_smem((const void *)k_image_m2l_a, LM_SMEM_IMAGE_M2L_A, (int)shm));
            k_image_m2l_a<<<ni, 256, shm, st>>>(md, P, dint + nf, ddbl + nf, ddbl + ncls + nf, dint + ncls + nf,
                                                dint + 2 * ncls + nf, ni, A.tab + (size_t)nf * np * np, t->dflag);
        }
        LM_CUDA(cudaGetLastError());
        LM_CUDA(cudaStreamSynchronize(st));
        cudaFree(dint);
        cudaFree(ddbl);
        cudaFree(dsc);
        t->bytes -= (3 * (size_t)ncls + 1) * sizeof(int) + (2 * (size_t)ncls + 1 + (size_t)(t->L + 1) * (P + 1)) *
                                                               sizeof(double);
    }
    // expansions and tree-order scratch
    TRY_A(lm_dalloc(t, &A.M, (size_t)nbox * np * LM_MAXV));
    TRY_A(lm_dalloc(t, &A.Lc, (size_t)nbox * np * LM_MAXV));
    TRY_A(lm_dalloc(t, &t->qs, (size_t)LM_MAXV * n));
    TRY_A(lm_dalloc(t, &t->us, (size_t)LM_MAXV * n));
    int hflag = 0;
    LM_CUDA(cudaMemcpyAsync(&hflag, t->dflag, sizeof(int), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    if (hflag & 8) {
        lm_set_error("build_tree: expansion order too large for the table builder");
        return LM_ENOTSUP;
    }
    if (hflag & 16) {
        lm_set_error("build_tree: a layered M2L table overflowed; lower p");
        return LM_ENOTSUP;
    }
    if (t->precision == LM_MIXED) return lm_setup_mixed_adaptive(t, st);
    return lm_setup_df(t, st);
}

// V (which = 0, every level) or U (which = 1) rows (target box, term, source box)
lm_status lm_adaptive_lists_to_host(lm_tree_s *t, int which, std::vector<int64_t> &rows, cudaStream_t st)
{
    AdaptTree &A = t->at;
    const int64_t nb = A.nbox, ne = which ? t->nu : A.nv;
    const int64_t *start = which ? t->ustart : A.vstart;
    const int32_t *src = which ? t->usrc : A.vsrc, *term = which ? t->uterm : A.vterm;
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

void lm_free_adaptive(lm_tree_s *t)
{
    AdaptTree &A = t->at;
    void *ptrs[] = {A.cx,     A.cy,     A.w,      A.parent, A.pos,   A.child, A.leaves, A.nonleaf,
                    A.pwleaves, A.vstart, A.vsrc, A.vslot,  A.vterm, A.tab,   A.M,      A.Lc,
                    A.tabdf,  A.tabdft, A.Mdf};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    A = AdaptTree();
}

extern "C" lm_status lm_adaptive_plan(const double *x, const double *y, int64_t n, double d, int leaf_target,
                                      int depth, double *x_origin, int *R, int64_t *nbox, int64_t *boxes,
                                      int64_t box_cap, int64_t *perm, int64_t *pstart, int64_t *nv,
                                      int64_t *vrows, int64_t v_cap, int64_t *nu, int64_t *urows, int64_t u_cap)
{
    if (!x || !y || n < 1 || !isfinite(d) || !(d > 0.0) || leaf_target < 1 || depth < -1 || depth > 14 ||
        box_cap < 0 || v_cap < 0 || u_cap < 0 || (box_cap > 0 && !boxes) || (v_cap > 0 && !vrows) ||
        (u_cap > 0 && !urows)) {
        lm_set_error("adaptive_plan: bad argument");
        return LM_EINVAL;
    }
    Builder B;
    std::vector<int64_t> hperm, hpstart;
    Rows V, U;
    lm_status s = plan(x, y, n, d, leaf_target, depth >= 0 ? depth : 14, "adaptive_plan", B, hperm, hpstart, V, U);
    if (s != LM_OK) return s;
    const int64_t nb = (int64_t)B.box.size();
    if (x_origin) *x_origin = B.x0;
    if (R) *R = B.R;
    if (nbox) *nbox = nb;
    if (nv) *nv = (int64_t)V.size();
    if (nu) *nu = (int64_t)U.size();
    for (int64_t b = 0; b < std::min(nb, box_cap); ++b) {
        const HBox &h = B.box[b];
        boxes[4 * b] = h.level;
        boxes[4 * b + 1] = h.col;
        boxes[4 * b + 2] = h.row;
        boxes[4 * b + 3] = h.leaf ? 1 : 0;
    }
    if (perm) memcpy(perm, hperm.data(), n * sizeof(int64_t));
    if (pstart && box_cap >= nb) memcpy(pstart, hpstart.data(), (nb + 1) * sizeof(int64_t));
    auto put = [](const Rows &L, int64_t *out, int64_t cap) {
        for (int64_t e = 0; e < std::min((int64_t)L.size(), cap); ++e) {
            out[3 * e] = std::get<0>(L[e]);
            out[3 * e + 1] = std::get<1>(L[e]);
            out[3 * e + 2] = std::get<2>(L[e]);
        }
    };
    put(V, vrows, v_cap);
    put(U, urows, u_cap);
    return LM_OK;
}
