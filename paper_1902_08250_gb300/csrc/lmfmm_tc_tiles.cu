// lmfmm_tc_tiles.cu -- the M2L of every level, free space and the four image
// terms of Lemma M2L (Sec. 2.1), on the 5th-generation tensor cores (tcgen05,
// kind::f16 with FP32 accumulation) as one persistent launch, for applies of
// 16 density vectors (and, in the batched form, of 4).
//
// Work is cut into tiles of 8 target boxes that lie in one row of one level,
// in steps of 2 columns (one parity class; level 0: consecutive roots).  For
// every V-list entry of its boxes a tile holds one (table slot, column offset
// dc, source row) item, with a mask of the boxes that have it.  The 8 boxes'
// sources of an item lie in one row, dc columns to the left of their targets.
//
// One item adds one product in real-block form:
//     D[128 x 256] += A[128 x 64] . B[256 x 64]^T,
//   A rows 0..63   the table's FP16 hi part, rows 64..127 its lo part (real-block
//                  rows [Re L_p; Im L_p], 2(2p+1) <= 64, zero-padded),
//   B rows         8 boxes x (16 vectors of the multipoles' hi part, 16 of the
//                  lo part), K = 64 real input orders (zero-padded).
// So D holds hi*hi + hi*lo in rows 0..63 and lo*hi + lo*lo in rows 64..127,
// every product of the split; the four sums per output are added in registers.
// FP16 hi/lo keeps 22 significant bits, as TF32 hi/lo did, in half the bytes.
// Its range is met by powers of two: the tables of each level are scaled so
// that their largest component lies in [2^14, 2^15) (found at set-up by
// k_tmax), the multipoles of each level the same way (found per apply by
// k_mmax); the epilogue multiplies the sums by the inverse of the two scales,
// which is exact.  Components below 2^-24 of the largest one of their level
// fall into FP16's subnormal range: their absolute error stays below 2^-39 of
// that largest component.
// Tables are split once at set-up, multipoles once per apply by k_msplit, both
// into the canonical K-major layout the MMA reads (8-row x 16-byte core
// matrices, K-adjacent ones 128 B apart, 8-row groups 1 KB apart), so staging
// an item is 9 plain bulk copies (16 KB table + 8 x 4 KB boxes) and no thread
// touches operand data.
//
// Roles (10 warps, one CTA per SM, persistent over tiles):
//   warp 8  producer: loads 32 entries at a time across its lanes; lane 0
//           waits for a free stage and issues the bulk copies, which complete
//           on the stage's `full` barrier;
//   warp 9  MMA issuer: takes a tile's items in groups of up to TT_G = 8, all
//           of one group into one accumulator: waits for a free accumulator,
//           then per item for its stage, issues the 4 MMAs and commits them to
//           the stage's `empty` barrier; at the end of a group it commits to
//           the accumulator's `tfull` barrier;
//   warps 0-7 epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. + 31 of
//           boxes 4 (w / 4) .. + 3 once per group, adds it into registers
//           (blocked accumulation: groups of 8 entries summed on their own),
//           and frees the accumulator.  At the end of a tile the lo-part rows go through
//           shared memory to their hi-part rows, and the tile's local
//           expansions are written, coalesced, over L (this launch sets L;
//           L2L adds to it afterwards).
// Four shared-memory stages and two tensor-memory accumulators (2 x 256
// columns) let copies, MMAs and the epilogue of consecutive items overlap.
// Every wait is bounded; a role that gives up sets the CTA's abort word and
// the launch's error flag, the others stop at their next wait, copies and
// MMAs in flight are waited for (bounded) and tensor memory is freed.
#include <algorithm>
#include <map>
#include <tuple>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "tc_common.cuh"

#include <cuda_fp16.h>

#define TT_K 64                                      // real input orders per item (zero-padded)
#define TT_ROW (TT_K * 2)                            // bytes of one FP16 operand row
#define TT_TAB_FLOATS (128 * TT_ROW / 4)             // one split table (64 hi + 64 lo rows), in 4-byte words
#define TT_STAGE_TAB (TT_TAB_FLOATS * 4)             // 16 KB
#define TT_STAGE (TT_STAGE_TAB + 256 * TT_ROW)       // 48 KB: the table and 256 operand rows
#define TT_NSTAGE 4
#define TT_NBAR (2 * TT_NSTAGE + 4)                  // full / empty per stage, tfull / tempty per accumulator
#define TT_SMAX 14                                   // largest component scaled into [2^14, 2^15)
#define TT_G 4                                       // items of one tile summed in one accumulator
#define TT_EPI_WARPS 8
#define TT_THREADS ((TT_EPI_WARPS + 2) * 32)         // + producer + MMA warp
#define TT_MAXLEV 16

// NV vectors per box: a box is 2 NV operand rows ([hi v0..NV-1 | lo v0..NV-1]); a tile
// holds TB = 128 / NV boxes (8 boxes of 16 vectors, or 32 of 4), N = 256 either way
template <int NV>
struct TtShape {
    static constexpr int TB = 128 / NV;              // boxes per tile
    static constexpr int BOX_FLOATS = 2 * NV * TT_ROW / 4; // one split box, in 4-byte words
    static constexpr int CB_STRIDE = 2 * NV + 1;     // floats per (box, order) row of the combine buffer
    static constexpr int BPL = 32 / (2 * NV);        // boxes per 32-column tensor-memory load
};

struct TtTile {
    int32_t level, row, c0, cstride, nbox, e0, e1, pad; // level: index into the launch's level descriptors
};
struct TtEnt {
    int32_t slot, dc, rs;
    uint32_t mask; // bit j: target box j of the tile has this entry
};
// one level of one tree as the tile kernels see it
struct TtLevel {
    int64_t ncol;      // columns of the level
    int64_t mstart;    // first box of the level in its tree's split-multipole buffer
    const zf *M;       // multipoles [nbox][NP][16]
    zf *L;             // local expansions [nbox][NP][16]
    const float *tab;  // the level's first split table
    float *ms;         // the level's first split box
    const uint32_t *tmax; // the largest component of the level's tables (float bits)
    uint32_t *mmax;       // the level's largest multipole component (float bits), per apply
};

template <int NP, int NV>
struct TtSmem {
    static constexpr int CB_OFF = TT_NSTAGE * TT_STAGE;
    static constexpr int CB_BYTES = (TtShape<NV>::TB * NP * TtShape<NV>::CB_STRIDE * 4 + 15) / 16 * 16;
    static constexpr int BAR_OFF = CB_OFF + CB_BYTES;
    static constexpr int BYTES = BAR_OFF + TT_NBAR * 8 + 16;
};

// byte offset of element (row, k) of a K-major no-swizzle FP16 operand with K = 64:
// 8-row x 16-byte core matrices, K-adjacent ones 128 B apart, 8-row groups 1 KB apart
__host__ __device__ __forceinline__ uint32_t tt_off(int row, int k)
{
    return (uint32_t)((row >> 3) * (8 * TT_ROW) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}
__device__ __forceinline__ uint64_t tt_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;           // LBO: K-direction core-matrix stride
    d |= (uint64_t)((8 * TT_ROW) >> 4) << 32;  // SBO: 8-row-group stride
    d |= (uint64_t)1 << 46;
    return d;
}
// instruction descriptor of kind::f16: D = F32, A = B = F16, both K-major, M x N
__host__ __device__ constexpr uint32_t tt_idesc(int m, int n)
{
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void tt_mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
                 "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
// power-of-two scale exponent that puts the largest component (float bits) in
// [2^14, 2^15); kept within [-126, 126] so that the scale and its inverse are normal
__host__ __device__ __forceinline__ int tt_scale_exp(uint32_t mxbits)
{
    const int e = mxbits ? (int)((mxbits >> 23) & 0xff) - 127 : 0;
    const int es = TT_SMAX - e;
    return es < -126 ? -126 : (es > 126 ? 126 : es);
}
__device__ __forceinline__ float tt_pow2(int e) { return __uint_as_float((uint32_t)(e + 127) << 23); }
// position of box (r, c) in a level's split-multipole buffer: within each row the
// even columns, then the odd ones (levels >= 1, cstride 2), so that the sources of a
// tile's boxes at one entry are consecutive; level 0 (cstride 1) keeps the box order
__host__ __device__ __forceinline__ int64_t tt_pos(int64_t r, int64_t c, int64_t ncol, int cstride)
{
    return cstride == 2 ? r * ncol + (c & 1) * (ncol >> 1) + (c >> 1) : r * ncol + c;
}
// x -> FP16 hi (nearest) and lo = x - hi (nearest), packed two by two
__device__ __forceinline__ void tt_split2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *(const uint32_t *)&h;
    lo = *(const uint32_t *)&l;
}

// ---------------------------------------------------------------------------
// operand preparation
// ---------------------------------------------------------------------------
// The largest real or imaginary part over all table classes of one level, as
// float bits by atomicMax into the level's word (zeroed before).  One block per class.
__global__ void k_tmax(const zd *tab, int ncls, int NP, uint32_t *tmax)
{
    __shared__ uint32_t red[8];
    const int64_t cls = blockIdx.x;
    uint32_t m = 0;
    for (int i = threadIdx.x; i < NP * NP; i += blockDim.x) {
        const zd a = tab[cls * NP * NP + i];
        m = max(m, __float_as_uint(fmaxf(fabsf((float)a.re), fabsf((float)a.im))));
    }
    m = __reduce_max_sync(0xffffffffu, m); // non-negative floats: bits order as values
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t mm = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = max(mm, red[w]);
        if (mm) atomicMax(tmax, mm);
    }
}
// Tables of one level -> real-block A operands: row r < NP is Re L_r with
// (Re T, -Im T) at K = 2q, 2q + 1; row NP + r is Im L_r with (Im T, Re T).
// Scaled by the level's power of two, hi part in rows 0..63, lo part (the
// remainder, in FP64, rounded) in rows 64..127.  One thread per (class,
// row 0..63, K chunk of 8).
__global__ void k_tsplit(const zd *tab, int ncls, int NP, const uint32_t *tmax, float *out)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= (int64_t)ncls * 64 * 8) return;
    const int c = (int)(t & 7), r = (int)((t >> 3) & 63);
    const int64_t cls = t >> 9;
    const double sc = (double)tt_pow2(tt_scale_exp(*tmax));
    uint32_t hv[4], lv[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        double v2[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int k = 8 * c + 2 * i + h, q = k >> 1, im = k & 1;
            double v = 0.0;
            if (r < 2 * NP && q < NP) {
                const int p = r < NP ? r : r - NP;
                const zd a = tab[(cls * NP + p) * NP + q];
                v = r < NP ? (im ? -a.im : a.re) : (im ? a.re : a.im);
            }
            v2[h] = v * sc;
        }
        const __half2 hh = __floats2half2_rn((float)v2[0], (float)v2[1]);
        const float2 hf = __half22float2(hh);
        const __half2 ll = __floats2half2_rn((float)(v2[0] - (double)hf.x), (float)(v2[1] - (double)hf.y));
        hv[i] = *(const uint32_t *)&hh;
        lv[i] = *(const uint32_t *)&ll;
    }
    unsigned char *o = (unsigned char *)(out + cls * TT_TAB_FLOATS);
    *(uint4 *)(o + tt_off(r, 8 * c)) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
    *(uint4 *)(o + tt_off(64 + r, 8 * c)) = make_uint4(lv[0], lv[1], lv[2], lv[3]);
}

// The largest multipole component of each level (the first NV vector slots), as
// float bits by atomicMax into the level's word (zeroed before).  Grid (chunks,
// levels): block (x, l) reads part of level l's multipoles, 16 bytes per thread
// and step, and adds one atomic.
template <int NP, int NV>
__global__ void __launch_bounds__(256) k_mmax(const TtLevel *lv, int nlev, int64_t ntot)
{
    __shared__ uint32_t red[8];
    const int l = blockIdx.y;
    const int64_t nb = (l + 1 < nlev ? lv[l + 1].mstart : ntot) - lv[l].mstart;
    const int64_t n = nb * NP * (NV / 2);
    const zf *M = lv[l].M;
    uint32_t m = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    // four independent 16-byte loads in flight per thread and step
    for (int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t0 < n; t0 += 4 * stride) {
        float4 x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t t = t0 + u * stride;
            x[u] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (t < n) x[u] = *(const float4 *)(M + (t / (NV / 2)) * LM_MAXV + 2 * (int)(t % (NV / 2)));
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
            m = max(m, max(max(__float_as_uint(x[u].x) & 0x7fffffffu, __float_as_uint(x[u].y) & 0x7fffffffu),
                           max(__float_as_uint(x[u].z) & 0x7fffffffu, __float_as_uint(x[u].w) & 0x7fffffffu)));
    }
    m = __reduce_max_sync(0xffffffffu, m);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t mm = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) mm = max(mm, red[w]);
        if (mm) atomicMax(lv[l].mmax, mm);
    }
}

// Multipoles of every level of one tree -> B operands, one block of 2 NV rows per
// box: [hi v0..NV-1 | lo v0..NV-1] x 64 K in the canonical layout (8-row groups of
// 1 KB), scaled by the level's power of two.  One thread per (box, K chunk of 8 =
// orders 4c .. 4c + 3, vector).
template <int NP, int NV>
__global__ void k_msplit(const TtLevel *lv, int nlev, int64_t ntot)
{
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= ntot * 8 * NV) return;
    const int v = (int)(t % NV), c = (int)((t / NV) & 7);
    const int64_t gb = t / (8 * NV);
    int l = 0;
    while (l + 1 < nlev && gb >= lv[l + 1].mstart) ++l;
    const int64_t b = gb - lv[l].mstart;
    const float sc = tt_pow2(tt_scale_exp(*lv[l].mmax));
    const zf *m = lv[l].M + b * NP * LM_MAXV + v;
    uint32_t hv[4], lo[4];
#pragma unroll
    for (int h = 0; h < 4; ++h) {
        const int q = 4 * c + h;
        const zf z = q < NP ? m[q * LM_MAXV] : zf{0.f, 0.f};
        tt_split2(z.re * sc, z.im * sc, hv[h], lo[h]);
    }
    const int64_t ncol = lv[l].ncol;
    unsigned char *o =
        (unsigned char *)(lv[l].ms + tt_pos(b / ncol, b % ncol, ncol, l == 0 ? 1 : 2) * TtShape<NV>::BOX_FLOATS);
    *(uint4 *)(o + tt_off(v, 8 * c)) = make_uint4(hv[0], hv[1], hv[2], hv[3]);
    *(uint4 *)(o + tt_off(NV + v, 8 * c)) = make_uint4(lo[0], lo[1], lo[2], lo[3]);
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
template <int NP, int NV>
__global__ void __launch_bounds__(TT_THREADS, 1)
    k_m2l_tt(const TtTile *tiles, int ntiles, const TtEnt *ents, const TtLevel *lvs, const float *zero_box,
             int *err, int first_limit)
{
    using S = TtSmem<NP, NV>;
    using Sh = TtShape<NV>;
    extern __shared__ __align__(1024) unsigned char smem[];
    float *cb = (float *)(smem + S::CB_OFF);
    uint64_t *bars = (uint64_t *)(smem + S::BAR_OFF);
    uint32_t *tslot = (uint32_t *)(bars + TT_NBAR);
    volatile int *abort_s = (volatile int *)(tslot + 1);
    volatile int *stop_s = abort_s + 1;
    const uint32_t sbase = smem_u32(smem);
    const uint32_t bfull = smem_u32(bars), bempty = bfull + 8 * TT_NSTAGE, btfull = bfull + 16 * TT_NSTAGE,
                   btempty = btfull + 16;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int i = 0; i < TT_NSTAGE; ++i) {
            mbar_init(bfull + 8 * i, 1);
            mbar_init(bempty + 8 * i, 1);
        }
        for (int i = 0; i < 2; ++i) {
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
        int last[TT_NSTAGE]; // last item copied into each stage (lane 0)
#pragma unroll
        for (int s = 0; s < TT_NSTAGE; ++s) last[s] = -1;
        bool stop = false;
        for (int tile = blockIdx.x; tile < ntiles && !stop; tile += gridDim.x) {
            const TtTile T = tiles[tile];
            const TtLevel &lv = lvs[T.level];
            const int64_t ncol = lv.ncol;
            const float *tb = lv.tab, *ms = lv.ms;
            for (int base = T.e0; base < T.e1 && !stop; base += 32) {
                const int cnt = min(32, T.e1 - base);
                TtEnt mine = lane < cnt ? ents[base + lane] : TtEnt{0, 0, 0, 0u};
                for (int i = 0; i < cnt; ++i, ++it) {
                    const TtEnt E = {__shfl_sync(0xffffffffu, mine.slot, i), __shfl_sync(0xffffffffu, mine.dc, i),
                                     __shfl_sync(0xffffffffu, mine.rs, i), __shfl_sync(0xffffffffu, mine.mask, i)};
                    if (lane == 0) {
                        const int s = (int)(it % TT_NSTAGE);
                        if (!mbar_wait_lim(bempty + 8 * s, ((it / TT_NSTAGE) & 1) ^ 1, TC_WAIT_LIMIT, abort_s, err)) {
                            tt_fail(abort_s, err);
                        } else {
                            const uint32_t st = sbase + s * TT_STAGE, fb = bfull + 8 * s;
                            mbar_expect_tx(fb, TT_STAGE);
                            bulk_g2s(st, tb + (int64_t)E.slot * TT_TAB_FLOATS, TT_STAGE_TAB, fb);
                            const uint32_t full = T.nbox >= 32 ? 0xffffffffu : (1u << T.nbox) - 1u;
                            int j0 = 0;
                            if (E.mask == full) {
                                // every box of the tile has the entry: its sources are consecutive
                                // in the buffer, one copy
                                const float *src =
                                    ms + tt_pos(E.rs, T.c0 - E.dc, ncol, T.cstride) * Sh::BOX_FLOATS;
                                bulk_g2s(st + TT_STAGE_TAB, src, T.nbox * Sh::BOX_FLOATS * 4, fb);
                                j0 = T.nbox;
                            }
#pragma unroll 1
                            for (int j = j0; j < Sh::TB; ++j) {
                                const float *src = zero_box;
                                if (j < T.nbox && ((E.mask >> j) & 1u))
                                    src = ms + tt_pos(E.rs, T.c0 + (int64_t)j * T.cstride - E.dc, ncol, T.cstride) *
                                                   Sh::BOX_FLOATS;
                                bulk_g2s(st + TT_STAGE_TAB + j * Sh::BOX_FLOATS * 4, src, Sh::BOX_FLOATS * 4, fb);
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
            for (int s = 0; s < TT_NSTAGE; ++s)
                if (last[s] >= 0)
                    mbar_wait_lim(bfull + 8 * s, (last[s] / TT_NSTAGE) & 1, TC_WAIT_LIMIT, nullptr, nullptr);
        __syncwarp();
    } else if (warp == TT_EPI_WARPS + 1) {
        // ---- MMA issuer ----
        if (lane == 0) {
            const uint32_t idesc = tt_idesc(128, 256);
            uint32_t it = 0, gc = 0; // items, groups of up to TT_G items of one tile
            int lastg = -1;
            bool stop = false;
            for (int tile = blockIdx.x; tile < ntiles && !stop && !*abort_s; tile += gridDim.x) {
                const TtTile T = tiles[tile];
                for (int g0 = T.e0; g0 < T.e1 && !stop; g0 += TT_G, ++gc) {
                    const int g1 = min(T.e1, g0 + TT_G), ac = (int)(gc & 1);
                    if (!mbar_wait_lim(btempty + 8 * ac, ((gc >> 1) & 1) ^ 1, TC_WAIT_LIMIT, abort_s, err)) {
                        tt_fail(abort_s, err);
                        stop = true;
                        break;
                    }
                    const uint32_t d = tmem + 256u * ac;
                    int issued = 0;
                    for (int e = g0; e < g1; ++e, ++it, ++issued) {
                        const int s = (int)(it % TT_NSTAGE);
                        const int lim = (it == 0 && first_limit >= 0) ? first_limit : TC_WAIT_LIMIT;
                        if (!mbar_wait_lim(bfull + 8 * s, (it / TT_NSTAGE) & 1, lim, abort_s, err)) {
                            tt_fail(abort_s, err);
                            stop = true;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        const uint32_t a = sbase + s * TT_STAGE, b = a + TT_STAGE_TAB;
                        // K = 16 per MMA (two 128-byte core matrices along K); the group's items
                        // add into one accumulator
#pragma unroll
                        for (int kk = 0; kk < TT_K / 16; ++kk)
                            tt_mma(d, tt_desc(a + kk * 256), tt_desc(b + kk * 256), idesc,
                                   (e > g0 || kk > 0) ? 1u : 0u);
                        tc_commit(bempty + 8 * s);
                    }
                    // (after a failed wait too: the drain below then covers every MMA issued)
                    if (issued > 0) {
                        tc_commit(btfull + 8 * ac);
                        lastg = (int)gc;
                    }
                    if (stop) break;
                }
            }
            // MMAs in flight complete before tensor memory is freed
            if (lastg >= 0)
                mbar_wait_lim(btfull + 8 * (lastg & 1), (lastg >> 1) & 1, TC_WAIT_LIMIT, nullptr, nullptr);
        }
        __syncwarp();
    } else {
        // ---- epilogue: warp (quadrant Q, half H) holds accumulator rows 32 Q .. + 31 of
        // boxes H TB/2 .. + TB/2 - 1 (128 columns) ----
        constexpr int HB = Sh::TB / 2; // boxes per warp
        const int Q = warp & 3, H = warp >> 2;
        const int n = 32 * Q + lane, r = n & 63; // accumulator row; real-block row
        const bool rowok = r < 2 * NP;
        const int p = r < NP ? r : r - NP, reim = r < NP ? 0 : 1;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * Q) << 16) + 128u * H;
        uint32_t gc = 0; // groups of up to TT_G items, as the MMA issuer counts them
        for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
            const TtTile T = tiles[tile];
            const TtLevel &lv = lvs[T.level];
            // undoes the level's table and multipole scales (the bits k_tsplit and k_msplit read)
            const float f = tt_pow2(-tt_scale_exp(*lv.tmax)) * tt_pow2(-tt_scale_exp(*lv.mmax));
            float acc[HB][NV];
#pragma unroll
            for (int jj = 0; jj < HB; ++jj)
#pragma unroll
                for (int v = 0; v < NV; ++v) acc[jj][v] = 0.f;
            bool bad = *abort_s != 0;
            for (int g0 = T.e0; g0 < T.e1; g0 += TT_G, ++gc) {
                if (bad) continue;
                const int s = (int)(gc & 1);
                if (!mbar_wait_lim(btfull + 8 * s, (gc >> 1) & 1, TC_WAIT_LIMIT, abort_s, err)) {
                    tt_fail(abort_s, err);
                    bad = true;
                    continue;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                // two 32-column loads in flight per wait
#pragma unroll
                for (int ld = 0; ld < 4; ld += 2) {
                    float v[2][32];
                    tc_ld32x2(lane_base + 256u * s + 32u * ld, v[0], v[1]);
#pragma unroll
                    for (int h = 0; h < 2; ++h)
#pragma unroll
                        for (int b4 = 0; b4 < Sh::BPL; ++b4)
#pragma unroll
                            for (int k = 0; k < NV; ++k)
                                acc[(ld + h) * Sh::BPL + b4][k] =
                                    fmaf(v[h][2 * NV * b4 + k] + v[h][2 * NV * b4 + NV + k], f,
                                         acc[(ld + h) * Sh::BPL + b4][k]);
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
                for (int jj = 0; jj < HB; ++jj)
#pragma unroll
                    for (int v = 0; v < NV; ++v)
                        cb[((HB * H + jj) * NP + p) * Sh::CB_STRIDE + 2 * v + reim] = acc[jj][v];
            asm volatile("bar.sync 1, 256;" ::: "memory");
            if (n < 64 && rowok)
#pragma unroll
                for (int jj = 0; jj < HB; ++jj)
#pragma unroll
                    for (int v = 0; v < NV; ++v)
                        cb[((HB * H + jj) * NP + p) * Sh::CB_STRIDE + 2 * v + reim] += acc[jj][v];
            asm volatile("bar.sync 1, 256;" ::: "memory");
            float *Lg = (float *)lv.L;
            const int64_t rowbase = (int64_t)T.row * lv.ncol + T.c0;
            for (int x = threadIdx.x; x < T.nbox * NP * 2 * NV; x += TT_EPI_WARPS * 32) {
                const int jp = x / (2 * NV), f = x % (2 * NV), j = jp / NP, pp = jp - j * NP;
                const int64_t box = rowbase + (int64_t)j * T.cstride;
                Lg[(box * NP + pp) * 2 * LM_MAXV + f] = cb[jp * Sh::CB_STRIDE + f];
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

// the level descriptors of one tree for one vector form (NV = 16: 8 KB per split box,
// NV = 4: 2 KB), in host memory
static std::vector<TtLevel> tt_levels(const lm_tree_s *t, int nv)
{
    const int64_t bf = nv == 16 ? TtShape<16>::BOX_FLOATS : TtShape<4>::BOX_FLOATS;
    std::vector<TtLevel> lv(t->L + 1);
    for (int l = 0; l <= t->L; ++l)
        lv[l] = TtLevel{t->lev[l].ncol,
                        t->tt_mbase[l],
                        t->lev[l].M32,
                        t->lev[l].L32,
                        t->tt_tab + t->tt_tbase[l] * TT_TAB_FLOATS,
                        t->tt_msplit + t->tt_mbase[l] * bf,
                        t->tt_tmax + l,
                        t->tt_mmax + l};
    return lv;
}

template <int NP, int NV>
static lm_status tt_attr()
{
    LM_CUDA(cudaFuncSetAttribute(k_m2l_tt<NP, NV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 TtSmem<NP, NV>::BYTES));
    return LM_OK;
}
template <int NP>
static lm_status tt_attr_np()
{
    lm_status s = tt_attr<NP, 16>();
    return s == LM_OK ? tt_attr<NP, 4>() : s;
}

// split the multipoles of every level of one tree (one launch)
template <int NP, int NV>
static void tt_msplit_launch(const lm_tree_s *t, const void *lv, cudaStream_t st)
{
    const int64_t ntot = t->tt_mbase[t->L + 1];
    int64_t nbmax = 1;
    for (int l = 0; l <= t->L; ++l) nbmax = std::max(nbmax, t->tt_mbase[l + 1] - t->tt_mbase[l]);
    const int64_t nx = std::max<int64_t>(1, std::min<int64_t>((nbmax * NP * (NV / 2) + 2047) / 2048, 2048));
    k_mmax<NP, NV><<<dim3((unsigned)nx, (unsigned)(t->L + 1)), 256, 0, st>>>((const TtLevel *)lv, t->L + 1, ntot);
    k_msplit<NP, NV><<<(unsigned)((ntot * 8 * NV + 255) / 256), 256, 0, st>>>((const TtLevel *)lv, t->L + 1, ntot);
}

template <int NP>
static lm_status tt_msplit(lm_tree_s *t, cudaStream_t st, int nvs)
{
    LM_CUDA(cudaMemsetAsync(t->tt_mmax, 0, (t->L + 1) * sizeof(uint32_t), st));
    if (nvs == LM_MAXV)
        tt_msplit_launch<NP, 16>(t, t->tt_lv[0], st);
    else
        tt_msplit_launch<NP, 4>(t, t->tt_lv[1], st);
    return LM_OK;
}

template <int NP>
static lm_status tt_launch(lm_tree_s *t, cudaStream_t st, int nvs)
{
    const int f = nvs == LM_MAXV ? 0 : 1;
    const int first = t->tt_poll_limit;
    t->tt_poll_limit = -1; // a test limit applies to one launch
    const float *zero = t->tt_msplit + t->tt_mbase[t->L + 1] * TtShape<16>::BOX_FLOATS;
    if (f == 0)
        k_m2l_tt<NP, 16><<<t->tt_grid, TT_THREADS, TtSmem<NP, 16>::BYTES, st>>>(
            (const TtTile *)t->tt_tiles[0], (int)t->tt_ntile[0], (const TtEnt *)t->tt_ents[0],
            (const TtLevel *)t->tt_lv[0], zero, t->dflag + 1, first);
    else
        k_m2l_tt<NP, 4><<<t->tt_grid, TT_THREADS, TtSmem<NP, 4>::BYTES, st>>>(
            (const TtTile *)t->tt_tiles[1], (int)t->tt_ntile[1], (const TtEnt *)t->tt_ents[1],
            (const TtLevel *)t->tt_lv[1], zero, t->dflag + 1, first);
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
    return std::max(TtSmem<NP, 16>::BYTES, TtSmem<NP, 4>::BYTES);
}
static int tt_bytes(int p)
{
    TT_SWITCH(p, tt_bytes_np);
    return 0;
}
static lm_status tt_set_attr(int p)
{
    TT_SWITCH(p, tt_attr_np);
    lm_set_error("tensor-core M2L tiles: order %d not instantiated", p);
    return LM_ENOTSUP;
}

// Tiles of tb class-consecutive boxes over every level, from the host copies of the
// V lists: per tile the union of its boxes' entries, each with the mask of boxes that have it
static void tt_build_tiles(const std::vector<std::vector<int64_t>> &vs, const std::vector<std::vector<int32_t>> &vsrc,
                           const std::vector<std::vector<int32_t>> &vslot, const lm_tree_s *t, int tb,
                           std::vector<TtTile> &tiles, std::vector<TtEnt> &ents)
{
    for (int l = 0; l <= t->L; ++l) {
        const Level &lv = t->lev[l];
        const int64_t ncol = lv.ncol, nrow = lv.nrow;
        const int cstride = l == 0 ? 1 : 2, npar = l == 0 ? 1 : 2;
        const int64_t ncl = ncol / cstride; // boxes of one parity in a row (ncol is even at l >= 1)
        for (int64_t r = 0; r < nrow; ++r)
            for (int pc = 0; pc < npar; ++pc)
                for (int64_t i0 = 0; i0 < ncl; i0 += tb) {
                    TtTile T{l, (int32_t)r, (int32_t)(i0 * cstride + pc), cstride,
                             (int32_t)std::min<int64_t>(tb, ncl - i0), (int32_t)ents.size(), 0, 0};
                    std::map<std::tuple<int32_t, int32_t, int32_t>, uint32_t> m;
                    for (int j = 0; j < T.nbox; ++j) {
                        const int64_t c = T.c0 + (int64_t)j * cstride, b = r * ncol + c;
                        for (int64_t e = vs[l][b]; e < vs[l][b + 1]; ++e) {
                            const int64_t src = vsrc[l][e];
                            const int32_t dc = (int32_t)(c - src % ncol), rs = (int32_t)(src / ncol);
                            m[std::make_tuple(vslot[l][e], dc, rs)] |= 1u << j;
                        }
                    }
                    for (const auto &kv : m)
                        ents.push_back(TtEnt{std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first),
                                             kv.second});
                    T.e1 = (int32_t)ents.size();
                    tiles.push_back(T);
                }
    }
}

template <typename T>
static lm_status tt_upload(lm_tree_s *t, const std::vector<T> &h, void **out, cudaStream_t st)
{
    T *d = nullptr;
    TT_TRY(lm_dalloc(t, &d, std::max<size_t>(1, h.size())));
    *out = d;
    if (!h.empty()) LM_CUDA(cudaMemcpyAsync(d, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return LM_OK;
}

// Set-up of the tile form: split tables, the split-multipole buffer (sized for the
// 16-vector form, with one zero box at the end for masked sources), the level
// descriptors of both vector forms and their tile / entry lists, built on the host
// from the V lists of every level.  Leaves tt_ready false (the per-level kernels
// then run) where the form does not apply.
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
    const int64_t bf16 = TtShape<16>::BOX_FLOATS;
    TT_TRY(lm_dalloc(t, &t->tt_tab, (size_t)std::max<int64_t>(1, t->tt_tbase[L + 1]) * TT_TAB_FLOATS));
    TT_TRY(lm_dalloc(t, &t->tt_msplit, (size_t)(t->tt_mbase[L + 1] + 1) * bf16));
    TT_TRY(lm_dalloc(t, &t->tt_tmax, (size_t)(L + 1)));
    TT_TRY(lm_dalloc(t, &t->tt_mmax, (size_t)(L + 1)));
    LM_CUDA(cudaMemsetAsync(t->tt_msplit + t->tt_mbase[L + 1] * bf16, 0, bf16 * sizeof(float), st));
    LM_CUDA(cudaMemsetAsync(t->tt_tmax, 0, (L + 1) * sizeof(uint32_t), st));
    LM_CUDA(cudaMemsetAsync(t->tt_mmax, 0, (L + 1) * sizeof(uint32_t), st));
    for (int l = 0; l <= L; ++l) {
        const int ncls = (int)t->lev[l].cls_term.size();
        if (ncls == 0) continue;
        k_tmax<<<(unsigned)ncls, 256, 0, st>>>(t->lev[l].tab, ncls, np, t->tt_tmax + l);
        const int64_t nt = (int64_t)ncls * 512;
        k_tsplit<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(t->lev[l].tab, ncls, np, t->tt_tmax + l,
                                                               t->tt_tab + t->tt_tbase[l] * TT_TAB_FLOATS);
    }
    // host copies of the V lists
    std::vector<std::vector<int64_t>> vs(L + 1);
    std::vector<std::vector<int32_t>> vsrc(L + 1), vslot(L + 1);
    for (int l = 0; l <= L; ++l) {
        const Level &lv = t->lev[l];
        vs[l].resize(lv.nbox + 1);
        vsrc[l].resize(std::max<int64_t>(1, lv.nv));
        vslot[l].resize(std::max<int64_t>(1, lv.nv));
        LM_CUDA(cudaMemcpyAsync(vs[l].data(), lv.vstart, (lv.nbox + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
        if (lv.nv > 0) {
            LM_CUDA(cudaMemcpyAsync(vsrc[l].data(), lv.vsrc, lv.nv * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
            LM_CUDA(cudaMemcpyAsync(vslot[l].data(), lv.vslot, lv.nv * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
        }
    }
    LM_CUDA(cudaStreamSynchronize(st));
    int64_t maxtiles = 0;
    for (int f = 0; f < 2; ++f) {
        std::vector<TtTile> tiles;
        std::vector<TtEnt> ents;
        tt_build_tiles(vs, vsrc, vslot, t, f == 0 ? TtShape<16>::TB : TtShape<4>::TB, tiles, ents);
        if (ents.size() > (size_t)INT32_MAX || tiles.size() > (size_t)INT32_MAX) return LM_OK;
        t->tt_ntile[f] = (int64_t)tiles.size();
        t->tt_nent[f] = (int64_t)ents.size();
        TT_TRY(tt_upload(t, tiles, &t->tt_tiles[f], st));
        TT_TRY(tt_upload(t, ents, &t->tt_ents[f], st));
        TT_TRY(tt_upload(t, tt_levels(t, f == 0 ? 16 : 4), &t->tt_lv[f], st));
        maxtiles = std::max(maxtiles, t->tt_ntile[f]);
    }
    LM_CUDA(cudaStreamSynchronize(st));
    t->tt_grid = std::max(1, (int)std::min<int64_t>(nsm, maxtiles));
    TT_TRY(tt_set_attr(t->p));
    t->tt_ready = true;
    return LM_OK;
}

lm_status lm_launch_msplit_tt(lm_tree_s *t, cudaStream_t st, int nvs)
{
    TT_SWITCH(t->p, tt_msplit, t, st, nvs);
    lm_set_error("tensor-core M2L tiles: order %d not instantiated", t->p);
    return LM_ENOTSUP;
}

lm_status lm_launch_m2l_tt(lm_tree_s *t, cudaStream_t st, int nvs)
{
    TT_SWITCH(t->p, tt_launch, t, st, nvs);
    lm_set_error("tensor-core M2L tiles: order %d not instantiated", t->p);
    return LM_ENOTSUP;
}

// ---------------------------------------------------------------------------
// one launch over the tiles of many trees (batched applies)
// ---------------------------------------------------------------------------
struct lm_tt_batch_s {
    int p = 0, nvs = 0, grid = 0;
    int64_t ntile = 0;
    TtTile *tiles = nullptr;
    TtEnt *ents = nullptr;
    TtLevel *lv = nullptr;
    const float *zero = nullptr;
    int *err = nullptr;
};

template <typename T>
static lm_status tt_fetch(const void *d, int64_t n, std::vector<T> &h)
{
    h.resize(n);
    if (n > 0) LM_CUDA(cudaMemcpy(h.data(), d, n * sizeof(T), cudaMemcpyDeviceToHost));
    return LM_OK;
}

// Concatenates the trees' tile and entry lists of one vector form into one work
// list: a tile's level index is offset into the concatenated level descriptors,
// its entry range into the concatenated entries.  Every tree must have the tile
// form ready with the same p.  A timeout of the launch is reported on trees[0].
lm_status lm_tt_batch_build(lm_tree_s *const *trees, int count, int nvs, lm_tt_batch_s **out)
{
    *out = nullptr;
    const int f = nvs == LM_MAXV ? 0 : 1;
    std::vector<TtTile> tiles;
    std::vector<TtEnt> ents;
    std::vector<TtLevel> lv;
    for (int i = 0; i < count; ++i) {
        const lm_tree_s *t = trees[i];
        std::vector<TtTile> ht;
        std::vector<TtEnt> he;
        std::vector<TtLevel> hl;
        TT_TRY(tt_fetch(t->tt_tiles[f], t->tt_ntile[f], ht));
        TT_TRY(tt_fetch(t->tt_ents[f], t->tt_nent[f], he));
        TT_TRY(tt_fetch(t->tt_lv[f], t->L + 1, hl));
        const int32_t eoff = (int32_t)ents.size(), loff = (int32_t)lv.size();
        for (TtTile T : ht) {
            T.level += loff;
            T.e0 += eoff;
            T.e1 += eoff;
            tiles.push_back(T);
        }
        ents.insert(ents.end(), he.begin(), he.end());
        lv.insert(lv.end(), hl.begin(), hl.end());
        if (ents.size() > (size_t)INT32_MAX || tiles.size() > (size_t)INT32_MAX) {
            lm_set_error("batch_create: too many M2L tiles for one launch");
            return LM_ENOTSUP;
        }
    }
    int dev = 0, nsm = 0;
    LM_CUDA(cudaGetDevice(&dev));
    LM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    lm_tt_batch_s *b = new (std::nothrow) lm_tt_batch_s();
    if (!b) {
        lm_set_error("batch_create: host allocation failed");
        return LM_ENOMEM;
    }
    b->p = trees[0]->p;
    b->nvs = nvs;
    b->ntile = (int64_t)tiles.size();
    b->grid = std::max(1, (int)std::min<int64_t>(nsm, b->ntile));
    b->zero = trees[0]->tt_msplit + trees[0]->tt_mbase[trees[0]->L + 1] * TtShape<16>::BOX_FLOATS;
    b->err = trees[0]->dflag + 1;
    auto up = [&](auto &v, auto **d) -> lm_status {
        using T = typename std::remove_reference<decltype(v)>::type::value_type;
        cudaError_t e = cudaMalloc((void **)d, std::max<size_t>(1, v.size()) * sizeof(T));
        if (e != cudaSuccess) {
            lm_set_error("batch_create: cudaMalloc failed: %s", cudaGetErrorString(e));
            return LM_ENOMEM;
        }
        if (!v.empty()) LM_CUDA(cudaMemcpy(*d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
        return LM_OK;
    };
    lm_status s = up(tiles, &b->tiles);
    if (s == LM_OK) s = up(ents, &b->ents);
    if (s == LM_OK) s = up(lv, &b->lv);
    if (s != LM_OK) {
        lm_tt_batch_free(b);
        return s;
    }
    *out = b;
    return LM_OK;
}

template <int NP>
static lm_status tt_batch_launch(const lm_tt_batch_s *b, cudaStream_t st)
{
    if (b->nvs == LM_MAXV)
        k_m2l_tt<NP, 16><<<b->grid, TT_THREADS, TtSmem<NP, 16>::BYTES, st>>>(b->tiles, (int)b->ntile, b->ents, b->lv,
                                                                          b->zero, b->err, -1);
    else
        k_m2l_tt<NP, 4><<<b->grid, TT_THREADS, TtSmem<NP, 4>::BYTES, st>>>(b->tiles, (int)b->ntile, b->ents, b->lv,
                                                                        b->zero, b->err, -1);
    return LM_OK;
}

lm_status lm_tt_batch_launch(const lm_tt_batch_s *b, cudaStream_t st)
{
    TT_SWITCH(b->p, tt_batch_launch, b, st);
    lm_set_error("tensor-core M2L tiles: order %d not instantiated", b->p);
    return LM_ENOTSUP;
}

void lm_tt_batch_free(lm_tt_batch_s *b)
{
    if (!b) return;
    void *ptrs[] = {b->tiles, b->ents, b->lv};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    delete b;
}

void lm_free_tt(lm_tree_s *t)
{
    for (int f = 0; f < 2; ++f) {
        void *ptrs[] = {t->tt_tiles[f], t->tt_ents[f], t->tt_lv[f]};
        for (void *p : ptrs)
            if (p) cudaFree(p);
        t->tt_tiles[f] = t->tt_ents[f] = t->tt_lv[f] = nullptr;
    }
    if (t->tt_tab) cudaFree(t->tt_tab);
    if (t->tt_msplit) cudaFree(t->tt_msplit);
    if (t->tt_tmax) cudaFree(t->tt_tmax);
    if (t->tt_mmax) cudaFree(t->tt_mmax);
    t->tt_tab = t->tt_msplit = nullptr;
    t->tt_tmax = t->tt_mmax = nullptr;
}
