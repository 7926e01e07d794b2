// lmfmm_tc.cu -- the free-space M2L stencil on the 5th-generation tensor
// cores (tcgen05, kind::tf32), mixed-precision path.
//
// In real-block form the M2L of one offset is
//     [Re L; Im L] += [[Ar, -Ai], [Ai, Ar]] [Re M; Im M],
// a real (2p+1)-by-(2p+1) block matrix (2(2p+1) <= 64) applied to the source
// multipoles of every (box, vector) column.  One CTA takes 8 target boxes of
// one parity class x 16 vectors = 128 rows: D[128 x 64] (rows = columns of
// the problem, 64 = padded real orders) lives in tensor memory and
// accumulates K = 64 per offset over all 27 offsets of the class.  Operands
// are staged in shared memory in the canonical K-major no-swizzle layout
// (8-row x 16-byte core matrices; K-adjacent core matrices 128 B apart,
// 8-row groups 2 KB apart).  Each operand is split into TF32 hi + lo parts
// and D += Ahi Bhi + Ahi Blo + Alo Bhi, which keeps FP32-level accuracy.
// One elected thread issues the MMAs and commits them to an mbarrier; every
// wait on it is bounded and reports a timeout through the error flag.
#include <stdint.h>

#include "internal.h"

#define TC_ROWS 128 // MMA M: 8 boxes x 16 vectors
#define TC_N 64     // MMA N: real orders, padded
#define TC_K 64     // K per offset
#define TC_TILE_A (TC_ROWS * TC_K * 4)   // bytes of one A operand (hi or lo)
#define TC_TILE_B (TC_N * TC_K * 4)      // bytes of one B operand
#define TC_PAD 0                         // no slack after the tiles
#define TC_SMEM (2 * TC_TILE_A + 2 * TC_TILE_B + TC_PAD + 64)

#include "tc_common.cuh"

// Real-block TF32 hi/lo images of the stencil tables, already in the shared
// layout (row n = real output order, k = real input order).
__global__ void k_tc_tables(int P, const zd *tab, const int32_t *slots, int nslot, float *rb)
{
    const int np = 2 * P + 1;
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= nslot * TC_N * TC_K) return;
    int s = e / (TC_N * TC_K), n = (e / TC_K) % TC_N, k = e % TC_K;
    // K is interleaved (k = 2q + part, part 0 = Re M_q, 1 = Im M_q) so that an
    // operand row is the complex multipole vector as consecutive floats;
    // N is [Re L_0..Re L_{np-1}, Im L_0..Im L_{np-1}, padding]
    double v = 0.0;
    if (n < 2 * np && k < 2 * np) {
        const int q = k >> 1, im_in = k & 1;
        const zd a = tab[((int64_t)slots[s] * np + (n % np)) * np + q];
        if (n < np) v = im_in ? -a.im : a.re;
        else v = im_in ? a.re : a.im;
    }
    float hi = tf32_rna((float)v);
    float lo = tf32_rna((float)(v - (double)hi));
    float *dst = rb + (size_t)s * 2 * (TC_N * TC_K);
    dst[tc_off(n, k) / 4] = hi;
    dst[TC_N * TC_K + tc_off(n, k) / 4] = lo;
}

template <int NP>
__global__ void __launch_bounds__(128, 2) k_m2l_tc(int64_t ncol, int64_t nrow, const int32_t *rbslot,
                                                   const float *rb, const zf *M, zf *Lc, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *Ahi = smem, *Alo = smem + TC_TILE_A;
    unsigned char *Bhi = smem + 2 * TC_TILE_A, *Blo = Bhi + TC_TILE_B;
    uint64_t *mbar = (uint64_t *)(smem + 2 * TC_TILE_A + 2 * TC_TILE_B + TC_PAD);
    uint32_t *tslot = (uint32_t *)(mbar + 1);

    // an earlier CTA timed out: this apply is already invalid (decided block-wide)
    if (__syncthreads_or(*(const volatile int *)err != 0)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cls = blockIdx.y, pc = cls & 1, pr = cls >> 1;
    const int64_t hc = ncol / 2, hr = nrow / 2;
    // this thread's row of the A operand: box lb of the tile, vector v
    const int lb = tid >> 4, v = tid & 15;
    const int64_t cidx = (int64_t)blockIdx.x * 8 + lb;
    const bool active = cidx < hc * hr;
    const int64_t c = 2 * (active ? cidx % hc : 0) + pc, r = 2 * (active ? cidx / hc : 0) + pr;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(64));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc_idesc_mn(TC_ROWS, TC_N);
    const uint32_t mb = smem_u32(mbar);
    uint32_t phase = 0;
    bool ok = true;
    int issued = 0;
    // running sum of the offsets' contributions for this thread's row; each
    // offset accumulates in tensor memory from zero and is folded in here
    // once complete (blocked accumulation keeps FP32 rounding short)
    float acc[TC_N];
#pragma unroll
    for (int j = 0; j < TC_N; ++j) acc[j] = 0.f;

    for (int dc = pc - 3; dc <= pc + 2 && ok; ++dc)
        for (int dr = pr - 3; dr <= pr + 2 && ok; ++dr) {
            if (dc >= -1 && dc <= 1 && dr >= -1 && dr <= 1) continue;
            const int s = rbslot[(dc + 3) * 7 + dr + 3];
            if (s < 0) continue; // offset beyond the grid at this level
            if (issued > 0) {
                // the previous offset's MMAs must finish before the operands are overwritten
                ok = __syncthreads_and(mbar_wait(mb, phase, err)); // block-uniform decision
                phase ^= 1;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (!ok) break;
                float dv[16];
#pragma unroll
                for (int j = 0; j < TC_N / 16; ++j) {
                    tc_ld16(tmem + ((uint32_t)(32 * warp) << 16) + 16 * j, dv);
#pragma unroll
                    for (int i = 0; i < 16; ++i) acc[16 * j + i] += dv[i];
                }
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncthreads(); // D is read by every warp before the next offset overwrites it
            }
            // B operand: the offset's table, hi and lo images (16 KB each)
            const uint4 *src = (const uint4 *)(rb + (size_t)s * 2 * (TC_N * TC_K));
            uint4 *bdst = (uint4 *)Bhi;
            for (int i = tid; i < 2 * TC_TILE_B / 16; i += 128) bdst[i] = src[i];
            // A operand: this row's gathered source multipoles, split hi/lo
            const int64_t cs = c - dc, rs = r - dr;
            const bool valid = active && cs >= 0 && cs < ncol && rs >= 0 && rs < nrow;
            const zf *m = M + (rs * ncol + cs) * NP * LM_MAXV + v;
            const int row = tid;
            // all of the row's loads first (independent, in flight together), then split and store
            zf x[NP];
#pragma unroll
            for (int q = 0; q < NP; ++q) x[q] = valid ? m[q * LM_MAXV] : zf{0.f, 0.f};
#pragma unroll
            for (int q2 = 0; q2 < (NP + 1) / 2; ++q2) {
                const zf a = x[2 * q2], b = (2 * q2 + 1 < NP) ? x[2 * q2 + 1] : zf{0.f, 0.f};
                float4 h, l;
                h.x = tf32_rna(a.re); h.y = tf32_rna(a.im); h.z = tf32_rna(b.re); h.w = tf32_rna(b.im);
                l.x = tf32_rna(a.re - h.x); l.y = tf32_rna(a.im - h.y);
                l.z = tf32_rna(b.re - h.z); l.w = tf32_rna(b.im - h.w);
                *(float4 *)(Ahi + tc_off(row, 4 * q2)) = h;
                *(float4 *)(Alo + tc_off(row, 4 * q2)) = l;
            }
            if (issued == 0)
                for (int k = 4 * ((NP + 1) / 2); k < TC_K; k += 4) {
                    *(float4 *)(Ahi + tc_off(row, k)) = make_float4(0.f, 0.f, 0.f, 0.f);
                    *(float4 *)(Alo + tc_off(row, k)) = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t ah = smem_u32(Ahi), al = smem_u32(Alo), bh = smem_u32(Bhi), bl = smem_u32(Blo);
#pragma unroll
                for (int kk = 0; kk < TC_K / 8; ++kk) {
                    const uint32_t o = kk * 256; // 8 TF32 = two 16-byte core matrices along K
                    // small terms first, then hi*hi; the first MMA of an offset starts from zero
                    tc_mma(tmem, tc_desc(ah + o), tc_desc(bl + o), idesc, kk > 0 ? 1u : 0u);
                    tc_mma(tmem, tc_desc(al + o), tc_desc(bh + o), idesc, 1u);
                    tc_mma(tmem, tc_desc(ah + o), tc_desc(bh + o), idesc, 1u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb)
                             : "memory");
            }
            ++issued;
        }
    if (issued > 0 && ok) {
        ok = __syncthreads_and(mbar_wait(mb, phase, err));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (ok && issued > 0) {
        // last offset; D row (32 warp + lane) = (box, vector), columns = real orders
        float dv[16];
#pragma unroll
        for (int j = 0; j < TC_N / 16; ++j) {
            tc_ld16(tmem + ((uint32_t)(32 * warp) << 16) + 16 * j, dv);
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[16 * j + i] += dv[i];
        }
        const int row = 32 * warp + lane;
        const int lb2 = row >> 4, v2 = row & 15;
        const int64_t cidx2 = (int64_t)blockIdx.x * 8 + lb2;
        if (cidx2 < hc * hr) {
            const int64_t c2 = 2 * (cidx2 % hc) + pc, r2 = 2 * (cidx2 / hc) + pr;
            zf *out = Lc + (r2 * ncol + c2) * NP * LM_MAXV + v2;
#pragma unroll
            for (int p = 0; p < NP; ++p) {
                zf o = out[p * LM_MAXV];
                out[p * LM_MAXV] = zf{o.re + acc[p], o.im + acc[NP + p]};
            }
        }
    }
    if (!ok && tid == 0) atomicOr(err, 1);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64));
}

static lm_status lm_attr_tc(int P);

// ---------------------------------------------------------------------------
lm_status lm_setup_tc(lm_tree_s *t, cudaStream_t st)
{
    const int P = t->p, np = 2 * P + 1;
    if (2 * np > TC_K) return LM_OK; // orders beyond the tensor-core tile: CUDA-core stencil only
    {
        lm_status sa = lm_attr_tc(P);
        if (sa != LM_OK) return sa;
    }
    for (int l = 1; l <= t->L; ++l) {
        Level &lv = t->lev[l];
        std::vector<int32_t> slots, map(49, -1);
        for (size_t i = 0; i < lv.cls_term.size(); ++i)
            if (lv.cls_term[i] == 0 && abs(lv.cls_dc[i]) <= 3 && abs(lv.cls_dr[i]) <= 3) {
                map[(lv.cls_dc[i] + 3) * 7 + lv.cls_dr[i] + 3] = (int32_t)slots.size();
                slots.push_back((int32_t)i);
            }
        if (slots.empty()) continue;
        int32_t *dslots;
        if (lm_dalloc(t, &dslots, slots.size()) != LM_OK) return LM_ENOMEM;
        if (lm_dalloc(t, &lv.rb, slots.size() * 2 * TC_N * TC_K) != LM_OK) return LM_ENOMEM;
        if (lm_dalloc(t, &lv.rbslot, 49) != LM_OK) return LM_ENOMEM;
        LM_CUDA(cudaMemcpyAsync(dslots, slots.data(), slots.size() * 4, cudaMemcpyHostToDevice, st));
        LM_CUDA(cudaMemcpyAsync(lv.rbslot, map.data(), 49 * 4, cudaMemcpyHostToDevice, st));
        int64_t tot = (int64_t)slots.size() * TC_N * TC_K;
        k_tc_tables<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(P, lv.tab, dslots, (int)slots.size(), lv.rb);
        LM_CUDA(cudaStreamSynchronize(st));
        cudaFree(dslots);
        t->bytes -= slots.size() * 4;
    }
    t->tc_ready = true;
    return LM_OK;
}

template <int NP>
static lm_status attr_tc_np()
{
    LM_CUDA(cudaFuncSetAttribute(k_m2l_tc<NP>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    return LM_OK;
}

template <int NP>
static lm_status launch_tc_np(lm_tree_s *t, const Level &lv, cudaStream_t st)
{
    int64_t ncls = (lv.ncol / 2) * (lv.nrow / 2);
    dim3 g((unsigned)((ncls + 7) / 8), 4);
    k_m2l_tc<NP><<<g, 128, TC_SMEM, st>>>(lv.ncol, lv.nrow, lv.rbslot, lv.rb, lv.M32, lv.L32, t->dflag + 1);
    return LM_OK;
}

#define TC_SWITCH(P, FN, ...)                    \
    switch (P) {                                 \
    case 4: return FN<9>(__VA_ARGS__);           \
    case 6: return FN<13>(__VA_ARGS__);          \
    case 8: return FN<17>(__VA_ARGS__);          \
    case 9: return FN<19>(__VA_ARGS__);          \
    case 10: return FN<21>(__VA_ARGS__);         \
    case 11: return FN<23>(__VA_ARGS__);         \
    case 12: return FN<25>(__VA_ARGS__);         \
    case 13: return FN<27>(__VA_ARGS__);         \
    case 14: return FN<29>(__VA_ARGS__);         \
    default: break;                              \
    }

// kernel attributes are set once at set-up, never while an apply may be captured
static lm_status lm_attr_tc(int P)
{
    TC_SWITCH(P, attr_tc_np);
    lm_set_error("tensor-core M2L: order %d not instantiated", P);
    return LM_ENOTSUP;
}

lm_status lm_launch_m2l_tc(lm_tree_s *t, int l, cudaStream_t st)
{
    const Level &lv = t->lev[l];
    TC_SWITCH(t->p, launch_tc_np, t, lv, st);
    lm_set_error("tensor-core M2L: order %d not instantiated", t->p);
    return LM_ENOTSUP;
}
