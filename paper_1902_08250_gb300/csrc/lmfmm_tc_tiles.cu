// lmfmm_tc_tiles.cu -- the M2L of every level, free space and the four image
// terms of Lemma M2L (Sec. 2.1), on the 5th-generation tensor cores (tcgen05,
// kind::tf32) as one persistent launch, for applies of 16 density vectors.
//
// Work is cut into tiles of 8 target boxes that lie in one row of one level,
// in steps of 2 columns (one parity class; level 0: consecutive roots).  For
// every V-list entry of its boxes a tile holds one (table slot, column offset
// dc, source row) item, with a mask of the boxes that have it.  The 8 boxes'
// sources of an item lie in one row, dc columns to the left of their targets.
//
// One item is one MMA chain in real-block form:
//     D[128 x 256] = A[128 x 64] . B[256 x 64]^T,
//   A rows 0..63   the table's TF32 hi part, rows 64..127 its lo part (real-block
//                  rows [Re L_p; Im L_p], 2(2p+1) <= 64, zero-padded),
//   B rows         8 boxes x (16 vectors of the multipoles' hi part, 16 of the
//                  lo part), K = 64 real input orders (zero-padded).
// So D holds hi*hi + hi*lo in rows 0..63 and lo*hi + lo*lo in rows 64..127,
// every product of the TF32 split; the four sums per output are added in
// registers.  Tables are split once at set-up, multipoles once per apply by
// k_msplit, both into the canonical K-major layout the MMA reads (8-row x
// 16-byte core matrices, K-adjacent ones 128 B apart, 8-row groups 2 KB apart),
// so staging an item is 9 plain bulk copies (32 KB table + 8 x 8 KB boxes) and
// no thread touches operand data.  M = 128 and N = 256 keep the shared-memory
// operand reads at 96 B per tensor-core clock.
//
// Roles (10 warps, one CTA per SM, persistent over tiles):
//   warp 8  producer: loads 32 entries at a time across its lanes; lane 0
//           waits for a free stage and issues the bulk copies, which complete
//           on the stage's `full` barrier;
//   warp 9  MMA issuer: waits for the stage and for a free accumulator, issues
//           the 8 MMAs, commits them to the stage's `empty` and the
//           accumulator's `tfull` barrier;
//   warps 0-7 epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 of
//           boxes 4 (w / 4) .. + 3, adds each item's D into registers (each
//           entry summed on its own, blocked accumulation), and frees the
//           accumulator.  At the end of a tile the lo-part rows go through
//           shared memory to their hi-part rows, and the tile's local
//           expansions are written, coalesced, over L (this launch sets L;
//           L2L adds to it afterwards).
// Two shared-memory stages and two tensor-memory accumulators (2 x 256
// columns) let copies, MMAs and the epilogue of consecutive items overlap.
// Every wait is bounded; a role that gives up sets the CTA's abort word and
// the launch's error flag, the others stop at their next wait, copies and
// MMAs in flight are waited for (bounded) and tensor memory is freed.
#include <algorithm>
#include <map>
#include <tuple>
#include <vector>

#include "internal.h"
#include "tc_common.cuh"

#define TT_BOXES 8                                   // target boxes per tile
#define TT_K 64                                      // real input orders per item (zero-padded)
#define TT_TAB_FLOATS (128 * TT_K)                   // one split table: 64 hi + 64 lo rows
#define TT_BOX_FLOATS (32 * TT_K)                    // one split box: 16 hi + 16 lo vector rows
#define TT_STAGE_TAB (TT_TAB_FLOATS * 4)             // 32 KB
#define TT_STAGE ((TT_TAB_FLOATS + TT_BOXES * TT_BOX_FLOATS) * 4) // 96 KB
#define TT_NSTAGE 2
#define TT_EPI_WARPS 8
#define TT_THREADS ((TT_EPI_WARPS + 2) * 32)         // + producer + MMA warp
#define TT_MAXLEV 16
#define TT_CB_STRIDE 33                              // floats per (box, order) row of the combine buffer

struct TtTile {
    int32_t level, row, c0, cstride, nbox, e0, e1, pad;
};
struct TtEnt {
    int32_t slot, dc, rs;
    uint32_t mask; // bit j: target box j of the tile has this entry
};
struct TtLevels {
    int64_t ncol[TT_MAXLEV];
    int64_t mbase[TT_MAXLEV]; // first box of the level in the split multipoles
    int64_t tbase[TT_MAXLEV]; // first table of the level in the split tables
    const zf *M[TT_MAXLEV];   // multipoles [nbox][NP][16]
    zf *L[TT_MAXLEV];         // local expansions [nbox][NP][16]
};

template <int NP>
struct TtSmem {
    static constexpr int CB_OFF = TT_NSTAGE * TT_STAGE;
    static constexpr int CB_BYTES = (TT_BOXES * NP * TT_CB_STRIDE * 4 + 15) / 16 * 16;
    static constexpr int BAR_OFF = CB_OFF + CB_BYTES;
    static constexpr int BYTES = BAR_OFF + 8 * 8 + 16;
};

// TF32 split: hi rounded to nearest (11 significant bits), lo = x - hi (exact in
// FP32) rounded the same way, so the tensor core reads both exactly
__device__ __forceinline__ void tt_split(float x, float &hi, float &lo)
{
    hi = tf32_rna(x);
    lo = tf32_rna(__fsub_rn(x, hi));
}

// ---------------------------------------------------------------------------
// operand preparation
// ---------------------------------------------------------------------------
// Tables of one level -> real-block A operands: row r < NP is Re L_r with
// (Re T, -Im T) at K = 2q, 2q + 1; row NP + r is Im L_r with (Im T, Re T).
// hi part in rows 0..63, lo part (T - hi, split again) in rows 64..127.
// One thread per (class, row 0..63, K chunk of 4).
__global__ void k_tsplit(const zd *tab, int ncls, int NP, float *out)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)ncls * 64 * 16) return;
    const int c = (int)(t & 15), r = (int)((t >> 4) & 63);
    const int64_t cls = t >> 10;
    float hv[4], lv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int k = 4 * c + i, q = k >> 1, im = k & 1;
        double v = 0.0;
        if (r < 2 * NP && q < NP) {
            const int p = r < NP ? r : r - NP;
            const zd a = tab[(cls * NP + p) * NP + q];
            v = r < NP ? (im ? -a.im : a.re) : (im ? a.re : a.im);
        }
        hv[i] = tf32_rna((float)v);
        lv[i] = tf32_rna((float)(v - (double)hv[i]));
    }
    float *o = out + cls * TT_TAB_FLOATS;
    *(float4 *)(o + tc_off(r, 4 * c) / 4) = make_float4(hv[0], hv[1], hv[2], hv[3]);
    *(float4 *)(o + tc_off(64 + r, 4 * c) / 4) = make_float4(lv[0], lv[1], lv[2], lv[3]);
}

// Multipoles of every level -> B operands, one 8 KB block per box: [hi v0-7 |
// hi v8-15 | lo v0-7 | lo v8-15], each an 8-row x 64-K group of core matrices
// (2 KB).  One thread per (box, K chunk of 4 = orders 2c, 2c + 1, vector);
// a warp reads two orders' 16 vectors (256 B) and writes two 128-B rows.
template <int NP>
__global__ void k_msplit(TtLevels lv, int nlev, int64_t ntot, float *out)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ntot * 256) return;
    const int v = (int)(t & 15), c = (int)((t >> 4) & 15);
    const int64_t gb = t >> 8;
    int l = 0;
    while (l + 1 < nlev && gb >= lv.mbase[l + 1]) ++l;
    const zf *m = lv.M[l] + (gb - lv.mbase[l]) * NP * LM_MAXV + v;
    float x[4];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        const int q = 2 * c + h;
        const zf z = q < NP ? m[q * LM_MAXV] : zf{0.f, 0.f};
        x[2 * h] = z.re;
        x[2 * h + 1] = z.im;
    }
    float4 hi, lo;
    tt_split(x[0], hi.x, lo.x);
    tt_split(x[1], hi.y, lo.y);
    tt_split(x[2], hi.z, lo.z);
    tt_split(x[3], hi.w, lo.w);
    float *o = out + gb * TT_BOX_FLOATS + (v >> 3) * 512 + c * 32 + (v & 7) * 4;
    *(float4 *)o = hi;
    *(float4 *)(o + 1024) = lo;
}

// ---------------------------------------------------------------------------
// the persistent tile kernel
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tt_fail(volatile int *abort_s, int *err)
{
    *abort_s = 1;
    atomicOr(err, 1);
}

// first_limit >= 0: poll limit of the MMA issuer's first operand wait (the
// timeout path's test); otherwise every wait polls up to TC_WAIT_LIMIT times
template <int NP>
__global__ void __launch_bounds__(TT_THREADS, 1)
    k_m2l_tt(const TtTile *tiles, int ntiles, const TtEnt *ents, TtLevels lv, const float *msplit,
             const float *tabs, int64_t zero_box, int *err, int first_limit)
{
    using S = TtSmem<NP>;
    extern __shared__ __align__(1024) unsigned char smem[];
    float *cb = (float *)(smem + S::CB_OFF);
    uint64_t *bars = (uint64_t *)(smem + S::BAR_OFF);
    uint32_t *tslot = (uint32_t *)(bars + 8);
    volatile int *abort_s = (volatile int *)(tslot + 1);
    volatile int *stop_s = abort_s + 1;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bfull = smem_u32(bars), bempty = bfull + 16, btfull = bfull + 32, btempty = bfull + 48;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < 2; ++i) {
            mbar_init(bfull + 8 * i, 1);
            mbar_init(bempty + 8 * i, 1);
            mbar_init(btfull + 8 * i, 1);
            mbar_init(btempty + 8 * i, TT_EPI_WARPS);
        }
        *abort_s = *(volatile int *)err; // an earlier CTA gave up: do no work
        *stop_s = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(512));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;

    if (warp == TT_EPI_WARPS) {
        // ---- producer: the warp loads 32 entries at a time (one per lane, in parallel) and
        // lane 0 takes them by shuffle, waits for stages and issues the copies ----
        uint32_t it = 0;
        int last[2] = {-1, -1}; // last item copied into each stage (lane 0)
        bool stop = false;
        for (int tile = blockIdx.x; tile < ntiles && !stop; tile += gridDim.x) {
            const TtTile T = tiles[tile];
            const int64_t ncol = lv.ncol[T.level], mb = lv.mbase[T.level];
            const float *tb = tabs + lv.tbase[T.level] * TT_TAB_FLOATS;
            for (int base = T.e0; base < T.e1 && !stop; base += 32) {
                const int cnt = min(32, T.e1 - base);
                TtEnt mine = lane < cnt ? ents[base + lane] : TtEnt{0, 0, 0, 0u};
                for (int i = 0; i < cnt; ++i, ++it) {
                    const TtEnt E = {__shfl_sync(0xffffffffu, mine.slot, i), __shfl_sync(0xffffffffu, mine.dc, i),
                                     __shfl_sync(0xffffffffu, mine.rs, i), __shfl_sync(0xffffffffu, mine.mask, i)};
                    if (lane == 0) {
                        const int s = it & 1;
                        if (!mbar_wait_lim(bempty + 8 * s, ((it >> 1) & 1) ^ 1, TC_WAIT_LIMIT, abort_s, err)) {
                            tt_fail(abort_s, err);
                        } else {
                            const uint32_t st = sbase + s * TT_STAGE, fb = bfull + 8 * s;
                            mbar_expect_tx(fb, TT_STAGE);
                            bulk_g2s(st, tb + (int64_t)E.slot * TT_TAB_FLOATS, TT_STAGE_TAB, fb);
#pragma unroll 1
                            for (int j = 0; j < TT_BOXES; ++j) {
                                int64_t src = zero_box;
                                if (j < T.nbox && ((E.mask >> j) & 1u))
                                    src = mb + (int64_t)E.rs * ncol + T.c0 + (int64_t)j * T.cstride - E.dc;
                                bulk_g2s(st + TT_STAGE_TAB + j * TT_BOX_FLOATS * 4, msplit + src * TT_BOX_FLOATS,
                                         TT_BOX_FLOATS * 4, fb);
                            }
                            last[s] = (int)it;
                        }
                    }
                    stop = __shfl_sync(0xffffffffu, (int)(*abort_s != 0), 0) != 0;
                    if (stop) break;
                }
            }
        }
        // copies in flight land before the CTA's shared memory is released
        if (lane == 0)
            for (int s = 0; s < 2; ++s)
                if (last[s] >= 0) mbar_wait_lim(bfull + 8 * s, (last[s] >> 1) & 1, TC_WAIT_LIMIT, nullptr, nullptr);
        __syncwarp();
    } else if (warp == TT_EPI_WARPS + 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            const uint32_t idesc = tc_idesc_mn(128, 256);
            uint32_t it = 0;
            int last = -1;
            for (int tile = blockIdx.x; tile < ntiles && !*abort_s; tile += gridDim.x) {
                const TtTile T = tiles[tile];
                for (int e = T.e0; e < T.e1; ++e, ++it) {
                    const int s = it & 1; // stage and accumulator
                    const uint32_t ph = (it >> 1) & 1;
                    const int lim = (it == 0 && first_limit >= 0) ? first_limit : TC_WAIT_LIMIT;
                    if (!mbar_wait_lim(bfull + 8 * s, ph, lim, abort_s, err) ||
                        !mbar_wait_lim(btempty + 8 * s, ph ^ 1, TC_WAIT_LIMIT, abort_s, err)) {
                        tt_fail(abort_s, err);
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a = sbase + s * TT_STAGE, b = a + TT_STAGE_TAB, d = tmem + 256u * s;
#pragma unroll
                    for (int kk = 0; kk < TT_K / 8; ++kk)
                        tc_mma(d, tc_desc(a + kk * 256), tc_desc(b + kk * 256), idesc, kk > 0 ? 1u : 0u);
                    tc_commit(bempty + 8 * s);
                    tc_commit(btfull + 8 * s);
                    last = (int)it;
                }
            }
            // MMAs in flight complete before tensor memory is freed
            if (last >= 0)
                mbar_wait_lim(btfull + 8 * (last & 1), (last >> 1) & 1, TC_WAIT_LIMIT, nullptr, nullptr);
        }
        __syncwarp();
    } else {
        // ---- epilogue ----
        const int Q = warp & 3, H = warp >> 2;
        const int n = 32 * Q + lane, r = n & 63; // accumulator row; real-block row
        const bool rowok = r < 2 * NP;
        const int p = r < NP ? r : r - NP, reim = r < NP ? 0 : 1;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * Q) << 16) + 128u * H;
        uint32_t it = 0;
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const TtTile T = tiles[tile];
            float acc[4][16];
#pragma unroll
            for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                for (int v = 0; v < 16; ++v) acc[jj][v] = 0.f;
            bool bad = *abort_s != 0;
            for (int e = T.e0; e < T.e1; ++e, ++it) {
                if (bad) continue;
                const int s = it & 1;
                if (!mbar_wait_lim(btfull + 8 * s, (it >> 1) & 1, TC_WAIT_LIMIT, abort_s, err)) {
                    tt_fail(abort_s, err);
                    bad = true;
                    continue;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
                for (int jj = 0; jj < 4; ++jj) {
                    float v[32];
                    tc_ld32(lane_base + 256u * s + 32u * jj, v);
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[jj][i] += v[i] + v[16 + i];
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncwarp();
                if (lane == 0) mbar_arrive(btempty + 8 * s);
            }
            // one decision for all epilogue warps: taken by warp 0, read after the barrier
            if (threadIdx.x == 0) *stop_s = *abort_s;
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (*stop_s) break;
            if (n >= 64 && rowok)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                    for (int v = 0; v < 16; ++v) cb[((4 * H + jj) * NP + p) * TT_CB_STRIDE + 2 * v + reim] = acc[jj][v];
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (n < 64 && rowok)
#pragma unroll
                for (int jj = 0; jj < 4; ++jj)
#pragma unroll
                    for (int v = 0; v < 16; ++v) cb[((4 * H + jj) * NP + p) * TT_CB_STRIDE + 2 * v + reim] += acc[jj][v];
            asm volatile("bar.sync 1, 256;" ::: "memory");
            float *Lg = (float *)lv.L[T.level];
            const int64_t rowbase = (int64_t)T.row * lv.ncol[T.level] + T.c0;
            for (int x = threadIdx.x; x < T.nbox * NP * 32; x += TT_EPI_WARPS * 32) {
                const int jp = x >> 5, f = x & 31, j = jp / NP, pp = jp - j * NP;
                const int64_t box = rowbase + (int64_t)j * T.cstride;
                Lg[(box * NP + pp) * 32 + f] = cb[jp * TT_CB_STRIDE + f];
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
#define TT_TRY(x)                    \
    do {                             \
        lm_status s_ = (x);          \
        if (s_ != LM_OK) return s_;  \
    } while (0)

static TtLevels tt_levels(const lm_tree_s *t)
{
    TtLevels lv{};
    for (int l = 0; l <= t->L; ++l) {
        lv.ncol[l] = t->lev[l].ncol;
        lv.mbase[l] = t->tt_mbase[l];
        lv.tbase[l] = t->tt_tbase[l];
        lv.M[l] = t->lev[l].M32;
        lv.L[l] = t->lev[l].L32;
    }
    return lv;
}

template <int NP>
static lm_status tt_attr()
{
    LM_CUDA(cudaFuncSetAttribute(k_m2l_tt<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, TtSmem<NP>::BYTES));
    return LM_OK;
}

template <int NP>
static lm_status tt_launch(lm_tree_s *t, cudaStream_t st)
{
    const TtLevels lv = tt_levels(t);
    const int64_t ntot = t->tt_mbase[t->L + 1];
    k_msplit<NP><<<(unsigned)((ntot * 256 + 255) / 256), 256, 0, st>>>(lv, t->L + 1, ntot, t->tt_msplit);
    const int first = t->tt_poll_limit;
    t->tt_poll_limit = -1; // a test limit applies to one launch
    k_m2l_tt<NP><<<t->tt_grid, TT_THREADS, TtSmem<NP>::BYTES, st>>>(
        (const TtTile *)t->tt_tiles, (int)t->tt_ntile, (const TtEnt *)t->tt_ents, lv, t->tt_msplit, t->tt_tab, ntot,
        t->dflag + 1, first);
    return LM_OK;
}

#define TT_SWITCH(P, FN, ...)            \
    switch (P) {                         \
    case 4: return FN<9>(__VA_ARGS__);   \
    case 6: return FN<13>(__VA_ARGS__);  \
    case 8: return FN<17>(__VA_ARGS__);  \
    case 9: return FN<19>(__VA_ARGS__);  \
    case 10: return FN<21>(__VA_ARGS__); \
    case 11: return FN<23>(__VA_ARGS__); \
    case 12: return FN<25>(__VA_ARGS__); \
    case 13: return FN<27>(__VA_ARGS__); \
    case 14: return FN<29>(__VA_ARGS__); \
    default: break;                      \
    }

template <int NP>
static int tt_bytes_np()
{
    return TtSmem<NP>::BYTES;
}
static int tt_bytes(int p)
{
    TT_SWITCH(p, tt_bytes_np);
    return 0;
}
static lm_status tt_set_attr(int p)
{
    TT_SWITCH(p, tt_attr);
    lm_set_error("tensor-core M2L tiles: order %d not instantiated", p);
    return LM_ENOTSUP;
}

// Set-up of the tile form: split tables, the split-multipole buffer (one zero
// box at the end for masked sources) and the tile / entry lists built on the
// host from the V lists of every level.  Leaves tt_ready false (the per-level
// kernels then run) where the form does not apply.
lm_status lm_setup_tt(lm_tree_s *t, cudaStream_t st)
{
    const int L = t->L, np = 2 * t->p + 1;
    t->tt_ready = false;
    t->tt_poll_limit = -1;
    if (!t->tc_ready || 2 * np > TT_K || L + 1 > TT_MAXLEV || t->adaptive) return LM_OK;
    int dev = 0;
    LM_CUDA(cudaGetDevice(&dev));
    int nsm = 0;
    LM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    int optin = 0;
    LM_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    const int need = tt_bytes(t->p);
    if (need == 0 || need > optin) return LM_OK; // order not instantiated, or too little shared memory
    t->tt_tbase.assign(L + 2, 0);
    t->tt_mbase.assign(L + 2, 0);
    for (int l = 0; l <= L; ++l) {
        t->tt_tbase[l + 1] = t->tt_tbase[l] + (int64_t)t->lev[l].cls_term.size();
        t->tt_mbase[l + 1] = t->tt_mbase[l] + t->lev[l].nbox;
    }
    TT_TRY(lm_dalloc(t, &t->tt_tab, (size_t)std::max<int64_t>(1, t->tt_tbase[L + 1]) * TT_TAB_FLOATS));
    TT_TRY(lm_dalloc(t, &t->tt_msplit, (size_t)(t->tt_mbase[L + 1] + 1) * TT_BOX_FLOATS));
    LM_CUDA(cudaMemsetAsync(t->tt_msplit + t->tt_mbase[L + 1] * TT_BOX_FLOATS, 0, TT_BOX_FLOATS * sizeof(float), st));
    for (int l = 0; l <= L; ++l) {
        const int ncls = (int)t->lev[l].cls_term.size();
        if (ncls == 0) continue;
        const int64_t nt = (int64_t)ncls * 1024;
        k_tsplit<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(t->lev[l].tab, ncls, np,
                                                               t->tt_tab + t->tt_tbase[l] * TT_TAB_FLOATS);
    }
    // tiles and entries
    std::vector<TtTile> tiles;
    std::vector<TtEnt> ents;
    for (int l = 0; l <= L; ++l) {
        const Level &lv = t->lev[l];
        std::vector<int64_t> hs(lv.nbox + 1);
        std::vector<int32_t> hsrc(std::max<int64_t>(1, lv.nv)), hslot(std::max<int64_t>(1, lv.nv));
        LM_CUDA(cudaMemcpyAsync(hs.data(), lv.vstart, (lv.nbox + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        if (lv.nv > 0) {
            LM_CUDA(cudaMemcpyAsync(hsrc.data(), lv.vsrc, lv.nv * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            LM_CUDA(cudaMemcpyAsync(hslot.data(), lv.vslot, lv.nv * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        }
        LM_CUDA(cudaStreamSynchronize(st));
        const int64_t ncol = lv.ncol, nrow = lv.nrow;
        const int cstride = l == 0 ? 1 : 2, npar = l == 0 ? 1 : 2;
        const int64_t ncl = ncol / cstride; // boxes of one parity in a row (ncol is even at l >= 1)
        for (int64_t r = 0; r < nrow; ++r)
            for (int pc = 0; pc < npar; ++pc)
                for (int64_t i0 = 0; i0 < ncl; i0 += TT_BOXES) {
                    TtTile T{l, (int32_t)r, (int32_t)(i0 * cstride + pc), cstride,
                             (int32_t)std::min<int64_t>(TT_BOXES, ncl - i0), (int32_t)ents.size(), 0, 0};
                    std::map<std::tuple<int32_t, int32_t, int32_t>, uint32_t> m;
                    for (int j = 0; j < T.nbox; ++j) {
                        const int64_t c = T.c0 + (int64_t)j * cstride, b = r * ncol + c;
                        for (int64_t e = hs[b]; e < hs[b + 1]; ++e) {
                            const int64_t s = hsrc[e];
                            const int32_t dc = (int32_t)(c - s % ncol), rs = (int32_t)(s / ncol);
                            m[std::make_tuple(hslot[e], dc, rs)] |= 1u << j;
                        }
                    }
                    for (const auto &kv : m)
                        ents.push_back(TtEnt{std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                                             kv.second});
                    T.e1 = (int32_t)ents.size();
                    tiles.push_back(T);
                }
    }
    if (ents.size() > (size_t)INT32_MAX || tiles.size() > (size_t)INT32_MAX) return LM_OK;
    t->tt_ntile = (int64_t)tiles.size();
    t->tt_nent = (int64_t)ents.size();
    TtTile *dt = nullptr;
    TtEnt *de = nullptr;
    TT_TRY(lm_dalloc(t, &dt, tiles.size()));
    TT_TRY(lm_dalloc(t, &de, std::max<size_t>(1, ents.size())));
    t->tt_tiles = dt;
    t->tt_ents = de;
    LM_CUDA(cudaMemcpyAsync(dt, tiles.data(), tiles.size() * sizeof(TtTile), cudaMemcpyHostToDevice, st));
    if (!ents.empty())
        LM_CUDA(cudaMemcpyAsync(de, ents.data(), ents.size() * sizeof(TtEnt), cudaMemcpyHostToDevice, st));
    LM_CUDA(cudaStreamSynchronize(st));
    t->tt_grid = std::max(1, std::min<int>(nsm, (int)tiles.size()));
    TT_TRY(tt_set_attr(t->p));
    t->tt_ready = true;
    return LM_OK;
}

lm_status lm_launch_m2l_tt(lm_tree_s *t, cudaStream_t st)
{
    TT_SWITCH(t->p, tt_launch, t, st);
    lm_set_error("tensor-core M2L tiles: order %d not instantiated", t->p);
    return LM_ENOTSUP;
}

void lm_free_tt(lm_tree_s *t)
{
    void *ptrs[] = {t->tt_tiles, t->tt_ents, t->tt_tab, t->tt_msplit};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    t->tt_tiles = t->tt_ents = nullptr;
    t->tt_tab = t->tt_msplit = nullptr;
}
