// lmfmm_tc.cu -- the free-space M2L stencil on the 5th-generation tensor
// cores (tcgen05, kind::tf32), mixed-precision path.
//
// In real-block form the M2L of one offset is
//     [Re L; Im L] += [[Ar, -Ai], [Ai, Ar]] [Re M; Im M],
// a real 2(2p+1)-square block matrix (2(2p+1) <= 64) applied to the source
// multipoles of every (box, vector) column.  One CTA takes 8 target boxes of
// one parity class x 16 vectors = 128 rows (or, for applies of at most 4
// vectors, 32 boxes x 4 vectors): D[128 x 64] (rows = columns of the problem,
// 64 = padded real orders) accumulates K = 64 per offset in tensor memory,
// over the (up to) 27 offsets of the class.
//
// Operands are staged in shared memory in the canonical K-major no-swizzle
// layout (8-row x 16-byte core matrices; K-adjacent core matrices 128 B apart,
// 8-row groups 2 KB apart), each split into TF32 hi + lo parts so that
// D += Ahi Bhi + Ahi Blo + Alo Bhi keeps FP32-level accuracy.  A is gathered
// from the source multipoles (two threads per row, one half of K each); B is
// expanded in shared memory from the offset's complex FP32 table (6.7 KB at
// p = 14, L2-resident) with consecutive threads on consecutive rows of one
// 16-byte chunk column, so neither operand's stores conflict.  The next
// offset's global loads are issued before the wait for the current MMAs;
// 256 threads and 96 KB per CTA keep two CTAs (16 warps) on each SM, so one
// CTA's staging overlaps the other's MMAs.  Each offset accumulates from zero
// and is folded into registers (blocked accumulation).  One elected thread
// issues the MMAs and commits them to an mbarrier; every wait on it is
// bounded and reports a timeout through the error flag.
#include <stdint.h>

#include "internal.h"

#define TC_ROWS 128 // MMA M: 8 boxes x 16 vectors
#define TC_N 64     // MMA N: real orders, padded
#define TC_K 64     // K per offset
#define TC_THREADS 256
#define TC_TILE_A (TC_ROWS * TC_K * 4) // bytes of one A operand (hi or lo)
#define TC_TILE_B (TC_N * TC_K * 4)    // bytes of one B operand
#define TC_STAGE (2 * TC_TILE_A + 2 * TC_TILE_B)
#define TC_TAIL 64 // mbarrier, tensor-memory slot
#define TC_SMEM (TC_STAGE + TC_TAIL)

#include "tc_common.cuh"

// TF32 hi/lo split: hi by the Veltkamp construction (x rounded to 11 significant
// bits, exact in TF32), lo = x - hi exactly; IEEE operations without contraction
__device__ __forceinline__ void tf32_split(float x, float &hi, float &lo)
{
    const float t = __fmul_rn(x, 8193.0f); // 2^13 + 1
    hi = __fsub_rn(t, __fsub_rn(t, x));
    lo = __fsub_rn(x, hi);
}

// the thread's share of one offset's operands, held in registers between the
// global loads and the shared-memory stores
// B work item t = tid + TC_THREADS j: table row p = t % NP, K chunk J = t / NP
// (entries q = 2J, 2J + 1), so that consecutive threads store consecutive rows
// of one 16-byte chunk column (conflict-free, like the A rows)
template <int NP>
struct TcRaw {
    static constexpr int NJ = (NP + 1) / 2; // K chunks holding table entries
    static constexpr int NBI = (NP * NJ + TC_THREADS - 1) / TC_THREADS;
    zf a[16];     // A: multipoles q = 16 h .. 16 h + 15 of this thread's row (zero past NP)
    zf b[NBI][2]; // B: T[p][2J], T[p][2J + 1] of the thread's items
};

template <int NP>
__device__ __forceinline__ void tc_load(TcRaw<NP> &x, const zf *M, const zf *T, int64_t ncol, int64_t nrow,
                                        bool active, int64_t c, int64_t r, int dc, int dr, int v, int h, int tid)
{
    const int64_t cs = c - dc, rs = r - dr;
    const bool valid = active && cs >= 0 && cs < ncol && rs >= 0 && rs < nrow;
    const zf *m = M + (rs * ncol + cs) * NP * LM_MAXV + v;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        const int q = 16 * h + j;
        x.a[j] = (valid && q < NP) ? m[q * LM_MAXV] : zf{0.f, 0.f};
    }
#pragma unroll
    for (int j = 0; j < TcRaw<NP>::NBI; ++j) {
        const int t = tid + TC_THREADS * j, p = t % NP, J = t / NP;
        const bool in = J < TcRaw<NP>::NJ;
        x.b[j][0] = in ? T[p * NP + 2 * J] : zf{0.f, 0.f};
        x.b[j][1] = (in && 2 * J + 1 < NP) ? T[p * NP + 2 * J + 1] : zf{0.f, 0.f};
    }
}

// split into TF32 hi/lo and store into one stage (A row `row`, chunks 8h..8h+7;
// B real-block entries of the thread's table elements)
template <int NP>
__device__ __forceinline__ void tc_store(const TcRaw<NP> &x, unsigned char *stage, int row, int h, int tid)
{
    unsigned char *Ahi = stage, *Alo = stage + TC_TILE_A;
    unsigned char *Bhi = stage + 2 * TC_TILE_A, *Blo = Bhi + TC_TILE_B;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const zf a = x.a[2 * j], b = x.a[2 * j + 1];
        float4 hv, lv;
        tf32_split(a.re, hv.x, lv.x);
        tf32_split(a.im, hv.y, lv.y);
        tf32_split(b.re, hv.z, lv.z);
        tf32_split(b.im, hv.w, lv.w);
        const uint32_t o = tc_off(row, 4 * (8 * h + j)); // K interleaved: k = 2q + (0 re, 1 im)
        *(float4 *)(Ahi + o) = hv;
        *(float4 *)(Alo + o) = lv;
    }
#pragma unroll
    for (int j = 0; j < TcRaw<NP>::NBI; ++j) {
        const int t = tid + TC_THREADS * j, p = t % NP, J = t / NP;
        if (J >= TcRaw<NP>::NJ) break;
        // row p (Re L_p): (a.re, -a.im) at k = 2q, 2q + 1; row NP + p (Im L_p): (a.im, a.re)
        const zf a = x.b[j][0], b = x.b[j][1];
        float ar, ai, br, bi, lar, lai, lbr, lbi;
        tf32_split(a.re, ar, lar);
        tf32_split(a.im, ai, lai);
        tf32_split(b.re, br, lbr);
        tf32_split(b.im, bi, lbi);
        const uint32_t o1 = tc_off(p, 4 * J), o2 = tc_off(NP + p, 4 * J);
        *(float4 *)(Bhi + o1) = make_float4(ar, -ai, br, -bi);
        *(float4 *)(Blo + o1) = make_float4(lar, -lai, lbr, -lbi);
        *(float4 *)(Bhi + o2) = make_float4(ai, ar, bi, br);
        *(float4 *)(Blo + o2) = make_float4(lai, lar, lbi, lbr);
    }
}

// 24 MMAs of one offset into accumulator `dt` (small terms first, then hi*hi;
// the first starts from zero)
__device__ __forceinline__ void tc_issue(uint32_t dt, const unsigned char *stage, uint32_t idesc)
{
    const uint32_t ah = smem_u32(stage), al = ah + TC_TILE_A, bh = ah + 2 * TC_TILE_A, bl = bh + TC_TILE_B;
#pragma unroll
    for (int kk = 0; kk < TC_K / 8; ++kk) {
        const uint32_t o = kk * 256; // 8 TF32 = two 16-byte core matrices along K
        tc_mma(dt, tc_desc(ah + o), tc_desc(bl + o), idesc, kk > 0 ? 1u : 0u);
        tc_mma(dt, tc_desc(al + o), tc_desc(bh + o), idesc, 1u);
        tc_mma(dt, tc_desc(ah + o), tc_desc(bh + o), idesc, 1u);
    }
}


// VB: log2 of the vector slots per box in a tile (4: 8 boxes x 16 vectors; 2: 32 boxes x 4 vectors)
template <int NP, int VB>
__global__ void __launch_bounds__(TC_THREADS, 2) k_m2l_tc(int64_t ncol, int64_t nrow, const int32_t *stencil,
                                                         const zf *tab, const zf *M, zf *Lc, int *err)
{
    constexpr int BOXES = TC_ROWS >> VB, VMASK = (1 << VB) - 1;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char *stage = smem;
    uint64_t *mbar = (uint64_t *)(smem + TC_STAGE);
    uint32_t *tslot = (uint32_t *)(mbar + 1);

    if (__syncthreads_or(*(const volatile int *)err != 0)) return;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int cls = blockIdx.y, pc = cls & 1, pr = cls >> 1;
    const int64_t hc = ncol / 2, hr = nrow / 2;
    const int row = tid & (TC_ROWS - 1), h = tid >> 7;
    const int lb = row >> VB, v = row & VMASK;
    const int64_t cidx = (int64_t)blockIdx.x * BOXES + lb;
    const bool active = cidx < hc * hr;
    const int64_t c = 2 * (active ? cidx % hc : 0) + pc, r = 2 * (active ? cidx / hc : 0) + pr;
    const int quad = warp & 3, chalf = warp >> 2;

    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(64));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    for (int i = tid; i < 2 * TC_TILE_B / 16; i += TC_THREADS)
        ((uint4 *)(stage + 2 * TC_TILE_A))[i] = make_uint4(0u, 0u, 0u, 0u);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = tc_idesc_mn(TC_ROWS, TC_N);
    const uint32_t mb = smem_u32(mbar);
    uint32_t phase = 0;
    bool ok = true;
    int issued = 0;
    float acc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) acc[j] = 0.f;
    auto fold = [&]() {
        float dv[16];
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            tc_ld16(tmem + ((uint32_t)(32 * quad) << 16) + 32u * (uint32_t)chalf + 16u * j, dv);
#pragma unroll
            for (int i = 0; i < 16; ++i) acc[16 * j + i] += dv[i];
        }
    };
    TcRaw<NP> x;
    for (int dc = pc - 3; dc <= pc + 2 && ok; ++dc)
        for (int dr = pr - 3; dr <= pr + 2 && ok; ++dr) {
            if (dc >= -1 && dc <= 1 && dr >= -1 && dr <= 1) continue;
            const int s = stencil[(dc + 3) * 7 + dr + 3];
            if (s < 0) continue;
            tc_load<NP>(x, M, tab + (int64_t)s * NP * NP, ncol, nrow, active, c, r, dc, dr, v, h, tid);
            if (issued > 0) {
                ok = __syncthreads_and(mbar_wait(mb, phase, err));
                phase ^= 1;
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                if (!ok) break;
                fold();
                asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                __syncthreads();
            }
            tc_store<NP>(x, stage, row, h, tid);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncthreads();
            if (tid == 0) {
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                tc_issue(tmem, stage, idesc);
                tc_commit(mb);
            }
            ++issued;
        }
    if (issued > 0 && ok) {
        ok = __syncthreads_and(mbar_wait(mb, phase, err));
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (ok && issued > 0) {
        fold();
        const int orow = 32 * quad + lane;
        const int lb2 = orow >> VB, v2 = orow & VMASK;
        const int64_t cidx2 = (int64_t)blockIdx.x * BOXES + lb2;
        if (cidx2 < hc * hr) {
            const int64_t c2 = 2 * (cidx2 % hc) + pc, r2 = 2 * (cidx2 / hc) + pr;
            float *out = (float *)(Lc + (r2 * ncol + c2) * NP * LM_MAXV + v2);
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int n = 32 * chalf + j;
                if (n < NP) out[2 * LM_MAXV * n] += acc[j];
                else if (n < 2 * NP) out[2 * LM_MAXV * (n - NP) + 1] += acc[j];
            }
        }
    }
    if (!ok && tid == 0) atomicOr(err, 1);
    if (!ok && issued > 0) mbar_wait(mb, phase, nullptr); // let an MMA in flight finish (bounded)
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(64));
}

// ---------------------------------------------------------------------------
template <int NP>
static lm_status attr_tc_np()
{
    LM_CUDA(cudaFuncSetAttribute(k_m2l_tc<NP, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    LM_CUDA(cudaFuncSetAttribute(k_m2l_tc<NP, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM));
    return LM_OK;
}

template <int NP>
static lm_status launch_tc_np(lm_tree_s *t, const Level &lv, cudaStream_t st, int nvs)
{
    const int64_t ncls = (lv.ncol / 2) * (lv.nrow / 2);
    if (nvs == 4) {
        dim3 g((unsigned)((ncls + 31) / 32), 4);
        k_m2l_tc<NP, 2><<<g, TC_THREADS, TC_SMEM, st>>>(lv.ncol, lv.nrow, lv.stencil, lv.tab32, lv.M32, lv.L32,
                                                         t->dflag + 1);
    } else {
        dim3 g((unsigned)((ncls + 7) / 8), 4);
        k_m2l_tc<NP, 4><<<g, TC_THREADS, TC_SMEM, st>>>(lv.ncol, lv.nrow, lv.stencil, lv.tab32, lv.M32, lv.L32,
                                                         t->dflag + 1);
    }
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

static lm_status lm_attr_tc(int P)
{
    TC_SWITCH(P, attr_tc_np);
    lm_set_error("tensor-core M2L: order %d not instantiated", P);
    return LM_ENOTSUP;
}

// kernel attributes are set once at set-up, never while an apply may be captured;
// the kernel reads the FP32 stencil tables and their (dc, dr) map directly
lm_status lm_setup_tc(lm_tree_s *t, cudaStream_t)
{
    const int np = 2 * t->p + 1;
    if (2 * np > TC_K) return LM_OK; // orders beyond the tensor-core tile: CUDA-core stencil only
    lm_status s = lm_attr_tc(t->p);
    if (s == LM_OK) t->tc_ready = true;
    return s;
}

lm_status lm_launch_m2l_tc(lm_tree_s *t, int l, cudaStream_t st, int nvs)
{
    const Level &lv = t->lev[l];
    TC_SWITCH(t->p, launch_tc_np, t, lv, st, nvs);
    lm_set_error("tensor-core M2L: order %d not instantiated", t->p);
    return LM_ENOTSUP;
}
