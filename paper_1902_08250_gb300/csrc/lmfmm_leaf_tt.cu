// lmfmm_leaf_tt.cu -- step 4 of the mixed-precision apply for 16 density vectors
// on uniform trees: the L2T evaluation of the local expansion (Eq. (local)) and
// the direct S2T interactions of the U list, with the multiply-adds over the
// vectors on the 5th-generation tensor cores (tcgen05, kind::f16 with FP32
// accumulation), as one persistent launch.
//
// For the targets of one leaf (a pass of up to 64 of them) both parts are one
// complex product
//     U[t][v] = sum_j G[t][j] Q[j][v],
// j over the leaf's U-list source points (free space: G = (i/4) H0(k2 r), the
// self pair excluded; reflected terms: their tails, the segment part coming from
// k_near_pw32), cut into chunks of 64, and in a last chunk over the orders
// n = -p..p (G the scaled J_|n|(k2 r) e^{i n theta} basis, Q the leaf's local
// expansion).  In real form, with K = (j, re / im) and N = (part h of Q's FP16
// split, output re / im, vector v):
//     D[t][(h, o, v)] = sum_k A[t][k] B[(h, o, v)][k],
//     A[t][(j, re)] = Re G,  A[t][(j, im)] = Im G,
//     B[(h, re, v)] = (Re Q_h, -Im Q_h),  B[(h, im, v)] = (Im Q_h, Re Q_h)  at (j, re), (j, im).
// A's rows 0..63 hold G's hi part for the 64 target slots and rows 64..127 its lo
// part, so one MMA chain per chunk (M = 128, N = 64, K = 128) forms every product
// of the split; the four sums of an output are added in registers, each chunk's D
// on its own (blocked accumulation).  The CUDA cores evaluate G (the kernel values
// are the expensive part) and no thread multiplies over the vectors.
//
// Roles (16 warps, one CTA per SM, persistent over the leaves):
//   warp 0     producer: tables the leaf's flattened U-list sources once per
//              leaf; per chunk its lanes write each source's record (offset of
//              the source leaf, point, U term), and the lane at the start of
//              each run of consecutive points bulk-copies the run's densities
//              (rows of 128 B) and coordinates (rows of 16 B), or lane 0 the
//              leaf's local expansion;
//   warps 1, 3 converters: split a stage's densities into the B operand
//              (canonical K-major layout, hi/lo parts, real-block signs), 8
//              vectors each; warp 1 also turns the records into coordinates;
//   warp 2     MMA issuer, owner of the tensor memory;
//   warps 4-11 kernel values: warp 4 + g evaluates G for target slots
//              32 (g & 1) .. + 31 and the chunk's sources 16 (g >> 1) .. + 15 and
//              stores their hi and lo rows of A;
//   warps 12-15 epilogue: warp 12 + Q reads tensor-memory lanes 32 Q .. + 31 of
//              each chunk's accumulator; at the end of a pass the lo-part rows
//              meet their hi-part rows in shared memory and the potentials are
//              written.
// Four source stages, two A buffers and four accumulators (4 x 64 columns) let
// copies, conversion, kernel values, MMAs and the epilogue of consecutive chunks
// overlap; every role loads the next leaf's counts while it serves the current
// one.  Every wait is bounded: a role that gives up sets the CTA's abort word and
// the launch's error flag, the others stop at their next wait (the epilogue
// warps, which share a named barrier, decide together once per pass), copies and
// MMAs in flight are waited for (bounded) and the tensor memory is freed.
#include <algorithm>

#include "internal.h"
#include "mixed_near.cuh"
#include "tc_common.cuh"
#include <cuda_fp16.h>

#define LF_CH 64                          // sources per chunk: K = 128 real columns
#define LF_K (2 * LF_CH)
#define LF_TGT 64                         // target slots per pass
#define LF_NS 4                           // source stages
#define LF_NA 2                           // A buffers
#define LF_ND 4                           // accumulators (64 tensor-memory columns each)
#define LF_GW 8                           // kernel-value warps
#define LF_JS 16                          // sources (order slots) per kernel-value thread and chunk
#define LF_RB 4                           // of which one round of evaluations takes LF_RB
#define LF_EPI0 (4 + LF_GW)               // first epilogue warp (a multiple of 4)
#define LF_THREADS ((LF_EPI0 + 4) * 32)
#define LF_MAXE 32                        // U entries of a leaf (one per producer lane)
#define LF_A_BYTES (128 * LF_K * 2)       // 32 KB: FP16
#define LF_B_BYTES (64 * LF_K * 2)        // 16 KB
#define LF_GSCALE 1024.0f                 // kernel values enter A multiplied by 2^10
#define LF_Q_BYTES (LF_CH * LM_MAXV * 8)  // 8 KB: rows of 16 complex densities
#define LF_RAW_BYTES (LF_Q_BYTES + LF_CH * 16) // + coordinate rows (x, y local; y absolute; 0)
#define LF_XS 33                          // floats per target row of the exchange buffer

// one stage's sources as the kernel-value warps read them, one 16-byte record each:
// (x, y relative to the target leaf's centre, absolute y, code = point << 2 | U term;
// an empty slot has point -1).  The producer writes the offsets centre_t - centre_s
// into x, y and the converter turns them into coordinates.
struct LfMeta {
    float4 src[LF_CH];
    int32_t n, pad[3]; // sources in the chunk (orders in the L2T chunk)
};
#define LF_MAXT 1024 // flattened U-list sources of a leaf tabled by the producer

template <int P>
struct LfSmem {
    static constexpr int A_OFF = 0;
    static constexpr int B_OFF = A_OFF + LF_NA * LF_A_BYTES;
    static constexpr int RAW_OFF = B_OFF + LF_NS * LF_B_BYTES;
    static constexpr int META_OFF = RAW_OFF + LF_NS * LF_RAW_BYTES;
    static constexpr int XCH_OFF = META_OFF + LF_NS * (int)sizeof(LfMeta);
    static constexpr int ETAB_OFF = XCH_OFF + 2 * LF_TGT * LF_XS * 4;
    static constexpr int TAB_OFF = ETAB_OFF + 6 * (LF_MAXE + 1) * 4;
    static constexpr int BAR_OFF = (TAB_OFF + LF_MAXT * 5 + 7) / 8 * 8;
    static constexpr int NBAR = 3 * LF_NS + 2 * LF_NA + 2 * LF_ND;
    static constexpr int BYTES = BAR_OFF + NBAR * 8 + 16;
};

// Operands are FP16 pairs: x = hi + lo with hi = fp16(x) and lo = fp16(x - hi), 22
// significant bits together; both factors are scaled by powers of two into FP16's range
// first (kernel values by 2^10; densities, and local expansions, so that the apply's largest
// component lies in [2^14, 2^15)), and the epilogue undoes the scales exactly.  Components
// below 2^-24 of that largest one lose relative precision (FP16 subnormals): their absolute
// error stays below 2^-39 of it.
// Byte offset of element (row, k) of a K-major no-swizzle FP16 operand with K = LF_K:
// 8-row x 16-byte core matrices, K-adjacent ones 128 B apart, 8-row groups LF_K * 16 B apart.
__host__ __device__ __forceinline__ uint32_t lf_off(int row, int k)
{
    return (uint32_t)((row >> 3) * (LF_K * 16) + (k >> 3) * 128 + (row & 7) * 16 + (k & 7) * 2);
}
__device__ __forceinline__ uint64_t lf_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFF) >> 4);
    d |= (uint64_t)(128 >> 4) << 16;   // LBO: K-direction core-matrix stride
    d |= (uint64_t)((LF_K * 16) >> 4) << 32; // SBO: 8-row-group stride
    d |= (uint64_t)1 << 46;
    return d;
}
// instruction descriptor of kind::f16: D = F32, A = B = F16, both K-major, M x N
__host__ __device__ constexpr uint32_t lf_idesc(int m, int n)
{
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void lf_mma(uint32_t dtmem, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc)
{
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dtmem),
                 "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
}
// (a, b) -> FP16 hi and lo pairs, each packed in 32 bits (a in the low half)
__device__ __forceinline__ void lf_split2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    const __half2 h = __floats2half2_rn(a, b);
    const float2 hf = __half22float2(h);
    const __half2 l = __floats2half2_rn(a - hf.x, b - hf.y);
    hi = *(const uint32_t *)&h;
    lo = *(const uint32_t *)&l;
}

__device__ __forceinline__ void lf_fail(volatile int *abort_s, int *err)
{
    *abort_s = 1;
    atomicOr(err, 1);
}

// bounded wait on an mbarrier phase: each poll parks the thread in the hardware for
// up to LF_SUSPEND_NS (it wakes as soon as the phase completes), so waiting warps take
// no issue slots from the working ones; gives up after `limit` polls, or early once
// the CTA's abort word or the launch's error flag is set
#define LF_SUSPEND_NS 20000
#define LF_WAIT_LIMIT (1 << 15)
__device__ __forceinline__ bool lf_wait(uint32_t addr, uint32_t parity, int limit, const volatile int *abort_s,
                                        const volatile int *err)
{
    {
        uint32_t done; // the phase is usually complete already: a non-blocking test first
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(done)
                     : "r"(addr), "r"(parity)
                     : "memory");
        if (done) return true;
    }
    for (int i = 0; i < limit; ++i) {
        uint32_t ok;
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}\n"
                     : "=r"(ok)
                     : "r"(addr), "r"(parity), "r"(LF_SUSPEND_NS)
                     : "memory");
        if (ok) return true;
        if (abort_s && *abort_s) return false;
        if ((i & 63) == 63 && err && *err) return false;
    }
    return false;
}

// S (i/4) H0(x) with S = LF_GSCALE, t = x^2/4 <= 1, from the ascending series of J0 and
// Y0 (A&S 9.1.12-13) to degree DEG, the constant factors folded into the coefficients:
//   im = S J0 / 4,   re = -S Y0 / 4 = -(2/pi)(ln(t)/2 + gamma) im + S/(2 pi) sum_m H_m c_m t^m,
// c_m = (-1)^m/(m!)^2, H_m the harmonic numbers; ln t from the hardware log2.
template <int DEG>
__device__ __forceinline__ zf lf_h0s(float t)
{
    static_assert(DEG >= 5 && DEG <= 8, "series degree");
    constexpr float S4 = 0.25f * LF_GSCALE, K1 = LF_GSCALE * 0.15915494309189535f; // S/4, S/(2 pi)
    constexpr float c[9] = {1.0f, -1.0f, 0.25f, -2.77777778e-02f, 1.73611111e-03f, -6.94444444e-05f,
                            1.92901235e-06f, -3.93675989e-08f, 6.15118733e-10f};
    constexpr float e[9] = {0.0f, -1.0f, 0.375f, -5.09259259e-02f, 3.61689815e-03f, -1.58564815e-04f,
                            4.72608025e-06f, -1.02074560e-07f, 1.67180484e-09f};
    const float2 tt = make_float2(t, t);
    float2 pp = make_float2(S4 * c[DEG], K1 * e[DEG]);
#pragma unroll
    for (int m = DEG - 1; m >= 1; --m) pp = __ffma2_rn(pp, tt, make_float2(S4 * c[m], K1 * e[m]));
    const float im = fmaf(pp.x, t, S4);
    const float sh = pp.y * t;
    // -(2/pi)(ln(t)/2 + gamma) = a1 log2(t) + b1
    constexpr float a1 = -0.63661977236758134f * 0.5f * 0.69314718055994531f;
    constexpr float b1 = -0.63661977236758134f * 0.57721566490153286f;
    const float wc = fmaf(a1, __log2f(t), b1);
    return zf{fmaf(wc, im, sh), im};
}

// L2T basis of the order slots E .. E + NS - 1 (slot P + n <-> order n) for a target at
// (x, y) relative to its leaf centre, zeta = (x + i y) / w, t = (k r / 2)^2:
//   n >= 0: s_n(t) zeta^n,   n < 0: (-1)^|n| s_|n|(t) conj(zeta)^|n|,
// s_m(t) = sum_j (-t)^j m! / (j! (j + m)!) = J_m(k r) / ((k r / 2)^m / m!), the scaled
// Bessel function of the local expansion (Eq. (local)), from its ascending series
// (A&S 9.1.10) by Horner's rule to j = 8 (first dropped term < 2e-14 for t <= 1/2).
template <int P, int E, int NS>
__device__ __forceinline__ void lf_basis(float xs, float ys, float t, zf *gv)
{
    constexpr int NP = 2 * P + 1;
    zf pw[P + 1];
    pw[0] = zf{1.f, 0.f};
#pragma unroll
    for (int m = 1; m <= P; ++m) pw[m] = pw[m - 1] * zf{xs, ys};
#pragma unroll
    for (int ii = 0; ii < NS; ++ii) {
        const int j = E + ii, n = j - P, a = n < 0 ? -n : n;
        if (j >= NP) {
            gv[ii] = zf{0.f, 0.f};
            continue;
        }
        float sv = 1.0f;
#pragma unroll
        for (int q = 8; q >= 1; --q) sv = fmaf(-t * (1.0f / (float)(q * (q + a))), sv, 1.0f);
        const zf z = n >= 0 ? pw[a] : conj(pw[a]);
        gv[ii] = (((n < 0 && (a & 1)) ? -sv : sv) * LF_GSCALE) * z;
    }
}

// named barrier over `nthreads` threads that returns the OR of their predicates
// (one decision for warps that must keep meeting at the same barriers)
__device__ __forceinline__ bool lf_bar_or(int id, int nthreads, bool p)
{
    uint32_t r;
    asm volatile("{\n\t.reg .pred q, s;\n\tsetp.ne.u32 q, %1, 0;\n\tbar.red.or.pred s, %2, %3, q;\n\t"
                 "selp.u32 %0, 1, 0, s;\n\t}\n"
                 : "=r"(r)
                 : "r"((uint32_t)p), "r"(id), "r"(nthreads)
                 : "memory");
    return r != 0;
}

// per leaf: its U-list source points (the length of its flattened source list)
__global__ void k_lf_tot(const int64_t *ls, const int64_t *ustart, const int32_t *usrc, int64_t nleaf,
                         int32_t *tot)
{
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int64_t T = 0;
    for (int64_t e = ustart[b]; e < ustart[b + 1]; ++e) T += ls[usrc[e] + 1] - ls[usrc[e]];
    tot[b] = (int32_t)T;
}
// per (leaf, entry slot < LF_MAXE): (first point, points, U term, source leaf) of the entry;
// zeros past the leaf's entries (and the free-term entries of a dG/dd tree would be dropped)
__global__ void k_lf_ent(const int64_t *ls, const int64_t *ustart, const int32_t *usrc, const int32_t *uterm,
                         int64_t nleaf, int4 *ent)
{
    const int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (x >= nleaf * LF_MAXE) return;
    const int64_t b = x / LF_MAXE, e = x % LF_MAXE, e0 = ustart[b];
    int4 r = make_int4(0, 0, 0, 0);
    if (e0 + e < ustart[b + 1]) {
        const int s = usrc[e0 + e];
        r = make_int4((int)ls[s], (int)(ls[s + 1] - ls[s]), uterm[e0 + e], s);
    }
    ent[x] = r;
}

// a leaf's target range and U-list length, loaded one leaf ahead by every role
struct LfLeaf {
    int lo, hi, T;
};
__device__ __forceinline__ LfLeaf lf_leaf(const int64_t *ls, const int32_t *tot, int64_t b, int64_t nleaf)
{
    if (b >= nleaf) return LfLeaf{0, 0, 0};
    return LfLeaf{(int)ls[b], (int)ls[b + 1], tot[b]};
}

// per point: (x, y) relative to its leaf's centre and absolute y, one 16-byte row
__global__ void k_lf_pts(const float *xl, const float *yl, const float *y32, int64_t n, float4 *pts)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) pts[i] = make_float4(xl[i], yl[i], y32[i], 0.f);
}

// first_limit >= 0: poll limit of the MMA issuer's first wait (the timeout path's test)
template <int P, int DEG>
__global__ void __launch_bounds__(LF_THREADS, 1)
    k_leaf_tt(int64_t nleaf, int64_t ncol, float w, float k, float d, const float *xl, const float *yl,
              const float *y32, const float4 *pts, const int64_t *ls, const int4 *ent, const int32_t *tot,
              const uint32_t *scl, NearQuadF nq, const zf *Lc,
              const zf *qs, zf *us, int *err, int first_limit)
{
    constexpr int NP = 2 * P + 1;
    static_assert(2 * NP <= 64, "the local expansion's orders must fit one chunk");
    using S = LfSmem<P>;
    extern __shared__ __align__(1024) unsigned char smem[];
    LfMeta *meta = (LfMeta *)(smem + S::META_OFF);
    float *xch = (float *)(smem + S::XCH_OFF);
    int32_t *eterm = (int32_t *)(smem + S::ETAB_OFF);
    int32_t *epref = eterm + (LF_MAXE + 1), *ebase = epref + (LF_MAXE + 1);
    float *eox = (float *)(ebase + (LF_MAXE + 1)), *eoy = eox + (LF_MAXE + 1);
    int32_t *tpi = (int32_t *)(smem + S::TAB_OFF);            // [LF_MAXT] point of flattened source g
    uint8_t *te = (uint8_t *)(tpi + LF_MAXT);                 // [LF_MAXT] its entry
    uint64_t *bars = (uint64_t *)(smem + S::BAR_OFF);
    uint32_t *tslot = (uint32_t *)(bars + S::NBAR);
    volatile int *abort_s = (volatile int *)(tslot + 1);
    const uint32_t sbase = smem_u32(smem);
    const uint32_t b0 = smem_u32(bars);
    // barriers: rfull (copies landed), bfull (B converted, meta ready), sempty (stage free),
    // afull (A stored), aempty (A read), dfull (accumulator written), dempty (accumulator read)
    auto rfull = [&](int s) { return b0 + 8u * s; };
    auto bfull = [&](int s) { return b0 + 8u * (LF_NS + s); };
    auto sempty = [&](int s) { return b0 + 8u * (2 * LF_NS + s); };
    auto afull = [&](int a) { return b0 + 8u * (3 * LF_NS + a); };
    auto aempty = [&](int a) { return b0 + 8u * (3 * LF_NS + LF_NA + a); };
    auto dfull = [&](int a) { return b0 + 8u * (3 * LF_NS + 2 * LF_NA + a); };
    auto dempty = [&](int a) { return b0 + 8u * (3 * LF_NS + 2 * LF_NA + LF_ND + a); };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // A buffers start as zeros: rows of empty target slots are read by the MMA
    for (int i = threadIdx.x; i < LF_NA * LF_A_BYTES / 16; i += LF_THREADS)
        ((float4 *)(smem + S::A_OFF))[i] = make_float4(0.f, 0.f, 0.f, 0.f);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    if (threadIdx.x == 0) {
        for (int s = 0; s < LF_NS; ++s) {
            mbar_init(rfull(s), 1);
            mbar_init(bfull(s), 2);
            mbar_init(sempty(s), 1 + LF_GW);
        }
        for (int a = 0; a < LF_NA; ++a) {
            mbar_init(afull(a), LF_GW);
            mbar_init(aempty(a), 1);
        }
        for (int a = 0; a < LF_ND; ++a) {
            mbar_init(dfull(a), 1);
            mbar_init(dempty(a), 4);
        }
        *abort_s = *(volatile int *)err; // an earlier launch or CTA gave up: do no work
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 2) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                     "r"(256));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = *tslot;
    const float kh = 0.5f * k;
    // power-of-two scales 2^(14 - e) of the densities ([0]) and the local expansions ([1]), e the
    // binary exponent of the largest component, and their inverses
    float scq[2], invq[2];
#pragma unroll
    for (int z = 0; z < 2; ++z) {
        const uint32_t mx = scl[z];
        const int e = mx ? (int)(mx >> 23) - 127 : 0;
        const int es = min(127, max(-126, 14 - e));
        scq[z] = __uint_as_float((uint32_t)(es + 127) << 23);
        invq[z] = __uint_as_float((uint32_t)(127 - es) << 23);
    }

    if (warp == 0) {
        // ---------------- producer ----------------
        uint32_t cc = 0;
        int last[LF_NS]; // last chunk copied into each stage (lane 0)
#pragma unroll
        for (int s = 0; s < LF_NS; ++s) last[s] = -1;
        bool stop = *abort_s != 0;
        LfLeaf nx = lf_leaf(ls, tot, blockIdx.x, nleaf);
        int4 nrec = blockIdx.x < nleaf ? ent[blockIdx.x * LF_MAXE + lane] : make_int4(0, 0, 0, 0);
        for (int64_t b = blockIdx.x; b < nleaf && !stop; b += gridDim.x) {
            const LfLeaf cu = nx;
            const int4 rec = nrec;
            nx = lf_leaf(ls, tot, b + gridDim.x, nleaf); // in flight while this leaf is served
            if (b + gridDim.x < nleaf) nrec = ent[(b + gridDim.x) * LF_MAXE + lane];
            const int lo = cu.lo, hi = cu.hi;
            if (hi <= lo) continue;
            // this lane's U entry (zeros past the leaf's entries)
            const int base = rec.x, cnt = rec.y, term = rec.z, src = rec.w;
            int incl = cnt;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
            }
            const int T = __shfl_sync(0xffffffffu, incl, 31);
            {
                const int64_t rt = b / ncol, ct = b % ncol, rs = src / ncol, cs = src % ncol;
                eox[lane] = (float)(ct - cs) * w; // centre_t - centre_s
                eoy[lane] = -(float)(rt - rs) * w;
            }
            eterm[lane] = term;
            ebase[lane] = base;
            epref[lane + 1] = incl;
            if (lane == 0) epref[0] = 0;
            __syncwarp();
            const bool tabled = T <= LF_MAXT;
            if (tabled) {
                // the entries with points, one after the other (their data by shuffle)
                for (uint32_t live = __ballot_sync(0xffffffffu, cnt > 0); live; live &= live - 1) {
                    const int e = __ffs(live) - 1;
                    const int p0 = __shfl_sync(0xffffffffu, incl - cnt, e), ce = __shfl_sync(0xffffffffu, cnt, e);
                    const int be = __shfl_sync(0xffffffffu, base, e);
                    for (int k2 = lane; k2 < ce; k2 += 32) {
                        tpi[p0 + k2] = be + k2;
                        te[p0 + k2] = (uint8_t)e;
                    }
                }
                __syncwarp();
            }
            const int nreg = (T + LF_CH - 1) / LF_CH, nch = nreg + 1;
            for (int i0 = lo; i0 < hi && !stop; i0 += LF_TGT) {
                for (int c = 0; c < nch; ++c, ++cc) {
                    const int s = (int)(cc % LF_NS);
                    int ok = 1;
                    if (lane == 0)
                        ok = lf_wait(sempty(s), ((cc / LF_NS) & 1) ^ 1, LF_WAIT_LIMIT, abort_s, err);
                    ok = __shfl_sync(0xffffffffu, ok, 0);
                    if (!ok) {
                        if (lane == 0) lf_fail(abort_s, err);
                        stop = true;
                        break;
                    }
                    LfMeta &m = meta[s];
                    const uint32_t raw = sbase + S::RAW_OFF + s * LF_RAW_BYTES;
                    if (c < nreg) {
                        const int g0 = c * LF_CH, n = min(LF_CH, T - g0);
                        // slots lane and 32 + lane: point, meta record, start of a run of consecutive points
                        int pi[2], last0 = -2;
                        uint32_t starts[2];
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int slot = 32 * h + lane;
                            const bool valid = slot < n;
                            int e = 0;
                            pi[h] = -1;
                            if (valid) {
                                const int g = g0 + slot;
                                if (tabled) {
                                    pi[h] = tpi[g];
                                    e = te[g];
                                } else {
                                    while (epref[e + 1] <= g) ++e;
                                    pi[h] = ebase[e] + (g - epref[e]);
                                }
                            }
                            m.src[slot] = valid ? make_float4(eox[e], eoy[e], 0.f, __int_as_float((pi[h] << 2) | eterm[e]))
                                                : make_float4(0.f, 0.f, 0.f, __int_as_float(-4));
                            int prev = __shfl_up_sync(0xffffffffu, pi[h], 1);
                            if (lane == 0) prev = last0; // slot 31 before slot 32; none before slot 0
                            starts[h] = __ballot_sync(0xffffffffu, valid && pi[h] != prev + 1);
                            last0 = __shfl_sync(0xffffffffu, pi[0], 31);
                        }
                        if (lane == 0) m.n = n;
                        __syncwarp();
                        if (lane == 0) mbar_expect_tx(rfull(s), (uint32_t)n * (LM_MAXV * 8 + 16));
                        __syncwarp();
                        // runs of consecutive points: the lane at a run's first slot copies its densities and
                        // coordinates (the copies of a chunk are issued in parallel)
                        const uint64_t st64 = (uint64_t)starts[0] | ((uint64_t)starts[1] << 32);
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int r = 32 * h + lane;
                            if ((st64 >> r) & 1) {
                                const uint64_t after = r < 63 ? st64 >> (r + 1) : 0;
                                const int r1 = after ? r + __ffsll((long long)after) : n;
                                const uint32_t len = (uint32_t)(r1 - r);
                                bulk_g2s(raw + (uint32_t)r * LM_MAXV * 8, qs + (int64_t)pi[h] * LM_MAXV, len * LM_MAXV * 8,
                                         rfull(s));
                                bulk_g2s(raw + LF_Q_BYTES + (uint32_t)r * 16, pts + pi[h], len * 16, rfull(s));
                            }
                        }
                    } else {
                        // the L2T chunk: the leaf's local expansion, orders as sources
                        if (lane == 0) {
                            m.n = NP;
                            mbar_expect_tx(rfull(s), NP * LM_MAXV * 8);
                            bulk_g2s(raw, Lc + b * NP * LM_MAXV, NP * LM_MAXV * 8, rfull(s));
                        }
                    }
                    if (lane == 0) last[s] = (int)cc;
                    stop = __shfl_sync(0xffffffffu, (int)(*abort_s != 0), 0) != 0;
                    if (stop) break;
                }
            }
        }
        // copies in flight land before the CTA's shared memory is released
        if (lane == 0)
            for (int s = 0; s < LF_NS; ++s)
                if (last[s] >= 0)
                    lf_wait(rfull(s), (last[s] / LF_NS) & 1, LF_WAIT_LIMIT, nullptr, nullptr);
        __syncwarp();
    } else if (warp == 1 || warp == 3) {
        // ---------------- converters: warp 1 vectors 0..7 (and the coordinates), warp 3 vectors 8..15 ----------------
        uint32_t cc = 0;
        bool stop = *abort_s != 0;
        const int cw = warp == 1 ? 0 : 1, v = 8 * cw + (lane & 7), kbp = lane >> 3;
        LfLeaf nx = lf_leaf(ls, tot, blockIdx.x, nleaf);
        for (int64_t b = blockIdx.x; b < nleaf && !stop; b += gridDim.x) {
            const LfLeaf cu = nx;
            nx = lf_leaf(ls, tot, b + gridDim.x, nleaf);
            const int lo = cu.lo, hi = cu.hi;
            if (hi <= lo) continue;
            const int nreg = (cu.T + LF_CH - 1) / LF_CH, nch = nreg + 1;
            for (int i0 = lo; i0 < hi && !stop; i0 += LF_TGT) {
                for (int c = 0; c < nch; ++c, ++cc) {
                    const int s = (int)(cc % LF_NS);
                    if (!lf_wait(rfull(s), (cc / LF_NS) & 1, LF_WAIT_LIMIT, abort_s, err)) {
                        lf_fail(abort_s, err);
                        stop = true;
                        break;
                    }
                    LfMeta &m = meta[s];
                    const int n = m.n;
                    const zf *raw = (const zf *)(smem + S::RAW_OFF + s * LF_RAW_BYTES);
                    if (cw == 0 && c < nreg) { // coordinates relative to the target leaf: X = x_s - (centre_t - centre_s)
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int slot = 32 * h + lane;
                            const float4 pt = slot < n ? ((const float4 *)(raw + LF_CH * LM_MAXV))[slot]
                                                       : make_float4(0.f, 0.f, 0.f, 0.f);
                            const float4 o = m.src[slot];
                            m.src[slot] = make_float4(kh * (pt.x - o.x), kh * (pt.y - o.y), pt.z, o.w);
                        }
                    }
                    unsigned char *B = smem + S::B_OFF + s * LF_B_BYTES;
                    const float sc = scq[c < nreg ? 0 : 1];
                    // K block kb holds sources 4 kb .. 4 kb + 3 (real, imaginary part each)
#pragma unroll
                    for (int kb = kbp; kb < LF_CH / 4; kb += 4) {
                        uint32_t h[2][4], l[2][4]; // [output re / im][source]
#pragma unroll
                        for (int jj = 0; jj < 4; ++jj) {
                            const int j = 4 * kb + jj;
                            const zf q = j < n ? raw[j * LM_MAXV + v] : zf{0.f, 0.f};
                            const float qr = q.re * sc, qi = q.im * sc;
                            uint32_t hr, lr, hi2, li2;
                            lf_split2(qr, -qi, hr, lr);  // out re: (Re Q, -Im Q)
                            lf_split2(qi, qr, hi2, li2); // out im: (Im Q, Re Q)
                            h[0][jj] = hr;
                            h[1][jj] = hi2;
                            l[0][jj] = lr;
                            l[1][jj] = li2;
                        }
                        const int kk = 8 * kb;
                        *(uint4 *)(B + lf_off(v, kk)) = make_uint4(h[0][0], h[0][1], h[0][2], h[0][3]);
                        *(uint4 *)(B + lf_off(16 + v, kk)) = make_uint4(h[1][0], h[1][1], h[1][2], h[1][3]);
                        *(uint4 *)(B + lf_off(32 + v, kk)) = make_uint4(l[0][0], l[0][1], l[0][2], l[0][3]);
                        *(uint4 *)(B + lf_off(48 + v, kk)) = make_uint4(l[1][0], l[1][1], l[1][2], l[1][3]);
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(bfull(s));
                    stop = *abort_s != 0;
                    if (stop) break;
                }
            }
        }
        __syncwarp();
    } else if (warp == 2) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = lf_idesc(128, 64);
            const uint64_t adesc0 = lf_desc(sbase + S::A_OFF), bdesc0 = lf_desc(sbase + S::B_OFF);
            uint32_t cc = 0;
            int last = -1;
            bool stop = *abort_s != 0;
            LfLeaf nx = lf_leaf(ls, tot, blockIdx.x, nleaf);
            for (int64_t b = blockIdx.x; b < nleaf && !stop; b += gridDim.x) {
                const LfLeaf cu = nx;
                nx = lf_leaf(ls, tot, b + gridDim.x, nleaf);
                const int lo = cu.lo, hi = cu.hi;
                if (hi <= lo) continue;
                const int nch = (cu.T + LF_CH - 1) / LF_CH + 1;
                for (int i0 = lo; i0 < hi && !stop; i0 += LF_TGT) {
                    for (int c = 0; c < nch; ++c, ++cc) {
                        const int s = (int)(cc % LF_NS), a = (int)(cc % LF_NA), dn = (int)(cc % LF_ND);
                        const uint32_t pa = (cc / LF_NA) & 1, pd = (cc / LF_ND) & 1;
                        const int lim = (cc == 0 && first_limit >= 0) ? first_limit : LF_WAIT_LIMIT;
                        if (!lf_wait(bfull(s), (cc / LF_NS) & 1, lim, abort_s, err) ||
                            !lf_wait(afull(a), pa, LF_WAIT_LIMIT, abort_s, err) ||
                            !lf_wait(dempty(dn), pd ^ 1, LF_WAIT_LIMIT, abort_s, err)) {
                            lf_fail(abort_s, err);
                            stop = true;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                        // K steps of 16 advance both start addresses by 256 B: 16 in the descriptors'
                        // address field (addresses < 256 KB, so the field does not carry)
                        const uint64_t da = adesc0 + (uint64_t)(a * (LF_A_BYTES >> 4));
                        const uint64_t db = bdesc0 + (uint64_t)(s * (LF_B_BYTES >> 4));
                        const uint32_t dd = tmem + 64u * dn;
#pragma unroll
                        for (int kk = 0; kk < LF_K / 16; ++kk)
                            lf_mma(dd, da + 16u * kk, db + 16u * kk, idesc, kk > 0 ? 1u : 0u);
                        tc_commit(sempty(s));
                        tc_commit(aempty(a));
                        tc_commit(dfull(dn));
                        last = (int)cc;
                    }
                }
            }
            // MMAs in flight complete before the tensor memory is freed
            if (last >= 0)
                lf_wait(dfull(last % LF_ND), (last / LF_ND) & 1, LF_WAIT_LIMIT, nullptr, nullptr);
        }
        __syncwarp();
    } else if (warp >= 4 && warp < LF_EPI0) {
        // ---------------- kernel values ----------------
        const int g = warp - 4, part = g >> 1, t = 32 * (g & 1) + lane;
        const int j0 = LF_JS * part;
        uint32_t cc = 0;
        bool bad = *abort_s != 0;
        LfLeaf nx = lf_leaf(ls, tot, blockIdx.x, nleaf);
        int pre_i0 = -1; // the pass whose target row is prefetched, and the row
        float4 pre_pt = make_float4(0.f, 0.f, 0.f, 0.f);
        for (int64_t b = blockIdx.x; b < nleaf && !bad; b += gridDim.x) {
            const LfLeaf cu = nx;
            nx = lf_leaf(ls, tot, b + gridDim.x, nleaf);
            const int lo = cu.lo, hi = cu.hi;
            if (hi <= lo) continue;
            const int nreg = (cu.T + LF_CH - 1) / LF_CH, nch = nreg + 1;
            for (int i0 = lo; i0 < hi && !bad; i0 += LF_TGT) {
                const int i = i0 + t;
                const bool act = i < hi;
                const float4 pt = i0 == pre_i0 ? pre_pt : (act ? pts[i] : make_float4(0.f, 0.f, 0.f, 0.f));
                {
                    // the next pass's target row, in flight while this pass is served
                    const int n0 = i0 + LF_TGT < hi ? i0 + LF_TGT : nx.lo, nh = i0 + LF_TGT < hi ? hi : nx.hi;
                    pre_i0 = n0;
                    pre_pt = n0 + t < nh ? pts[n0 + t] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
                const float xi = pt.x, yi = pt.y, ya = pt.z;
                const float xk = kh * xi, yk = kh * yi;
                for (int c = 0; c < nch; ++c, ++cc) {
                    const int s = (int)(cc % LF_NS), a = (int)(cc % LF_NA);
                    if (!lf_wait(bfull(s), (cc / LF_NS) & 1, LF_WAIT_LIMIT, abort_s, err) ||
                        !lf_wait(aempty(a), ((cc / LF_NA) & 1) ^ 1, LF_WAIT_LIMIT, abort_s, err)) {
                        lf_fail(abort_s, err);
                        bad = true;
                        break;
                    }
                    unsigned char *A = smem + S::A_OFF + a * LF_A_BYTES;
                    if (act) {
                        // this thread's LF_JS sources (or order slots) in rounds of LF_RB
#pragma unroll 1
                        for (int hb = 0; hb < LF_JS / LF_RB; ++hb) {
                            const int jb = j0 + LF_RB * hb;
                            zf gv[LF_RB];
                            if (c < nreg) {
                                // coordinates in units of 2/k, so that t = (k r / 2)^2 = dx^2 + dy^2; slots past
                                // the chunk's sources hold zeros (finite values; B is zero there)
                                const LfMeta &m = meta[s];
                                float tv[LF_RB];
                                bool special = false;
#pragma unroll
                                for (int ii = 0; ii < LF_RB; ++ii) {
                                    const float4 r4 = m.src[jb + ii];
                                    const float dx = xk - r4.x, dy = yk - r4.y;
                                    tv[ii] = fmaf(dx, dx, dy * dy);
                                    special |= ((__float_as_int(r4.w) & 3) != 0) | (!DEG && tv[ii] > 1.0f);
                                }
#pragma unroll
                                for (int ii = 0; ii < LF_RB; ++ii) gv[ii] = lf_h0s<DEG ? DEG : 8>(tv[ii]);
                                if (!special) {
                                    // t = 0: the self pair (and points that coincide) is left out
#pragma unroll
                                    for (int ii = 0; ii < LF_RB; ++ii)
                                        if (tv[ii] == 0.f) gv[ii] = zf{0.f, 0.f};
                                } else {
#pragma unroll
                                    for (int ii = 0; ii < LF_RB; ++ii) {
                                        const float4 r4 = m.src[jb + ii]; // read again: the rare path
                                        const int term = __float_as_int(r4.w) & 3;
                                        if (term != 0) { // tail of a reflected direct term
                                            const float X = fabsf(xk - r4.x) * (1.0f / kh);
                                            const float h = term == 1 ? -(ya + r4.z) : ya + r4.z + 2.0f * d;
                                            const zf tl = near_tail32(nq, term - 1, X, h);
                                            gv[ii] = zf{tl.re * LF_GSCALE, tl.im * LF_GSCALE};
                                        } else if (tv[ii] == 0.f) {
                                            gv[ii] = zf{0.f, 0.f};
                                        } else if (!DEG && tv[ii] > 1.0f) {
                                            const zf fr = green_free32_far(tv[ii]);
                                            gv[ii] = zf{fr.re * LF_GSCALE, fr.im * LF_GSCALE};
                                        }
                                    }
                                }
                            } else {
                                // the L2T chunk: order slots jb .. jb + LF_RB - 1 (a compile-time set per case)
                                const float xs = xi / w, ys = yi / w, tt = fmaf(xk, xk, yk * yk);
                                switch (jb / LF_RB) {
                                case 0: lf_basis<P, 0, LF_RB>(xs, ys, tt, gv); break;
                                case 1: lf_basis<P, LF_RB, LF_RB>(xs, ys, tt, gv); break;
                                case 2: lf_basis<P, 2 * LF_RB, LF_RB>(xs, ys, tt, gv); break;
                                case 3: lf_basis<P, 3 * LF_RB, LF_RB>(xs, ys, tt, gv); break;
#if LF_RB == 4
                                case 4: lf_basis<P, 16, 4>(xs, ys, tt, gv); break;
                                case 5: lf_basis<P, 20, 4>(xs, ys, tt, gv); break;
                                case 6: lf_basis<P, 24, 4>(xs, ys, tt, gv); break;
                                case 7: lf_basis<P, 28, 4>(xs, ys, tt, gv); break;
#endif
                                default: // slots past 2 P + 1 <= 29 hold zeros
#pragma unroll
                                    for (int ii = 0; ii < LF_RB; ++ii) gv[ii] = zf{0.f, 0.f};
                                    break;
                                }
                            }
                            // hi and lo rows of this target slot: one 16-byte store per 4 sources and part
#pragma unroll
                            for (int m4 = 0; m4 < LF_RB / 4; ++m4) {
                                uint32_t h[4], l[4];
#pragma unroll
                                for (int jj = 0; jj < 4; ++jj)
                                    lf_split2(gv[4 * m4 + jj].re, gv[4 * m4 + jj].im, h[jj], l[jj]);
                                const int kk = 2 * (jb + 4 * m4);
                                *(uint4 *)(A + lf_off(t, kk)) = make_uint4(h[0], h[1], h[2], h[3]);
                                *(uint4 *)(A + lf_off(64 + t, kk)) = make_uint4(l[0], l[1], l[2], l[3]);
                            }
                        }
                    }
                    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive(afull(a));
                        mbar_arrive(sempty(s));
                    }
                }
            }
        }
    } else if (warp >= LF_EPI0) {
        // ---------------- epilogue ----------------
        const int Q = warp & 3, t = 32 * (Q & 1) + lane;
        const uint32_t lane_base = tmem + ((uint32_t)(32 * Q) << 16);
        uint32_t cc = 0, pp = 0;
        bool bad = false;
        LfLeaf nx = lf_leaf(ls, tot, blockIdx.x, nleaf);
        for (int64_t b = blockIdx.x; b < nleaf; b += gridDim.x) {
            const LfLeaf cu = nx;
            nx = lf_leaf(ls, tot, b + gridDim.x, nleaf);
            const int lo = cu.lo, hi = cu.hi;
            if (hi <= lo) continue;
            const int nch = (cu.T + LF_CH - 1) / LF_CH + 1;
            for (int i0 = lo; i0 < hi; i0 += LF_TGT, ++pp) {
                float acc[32];
#pragma unroll
                for (int m = 0; m < 32; ++m) acc[m] = 0.f;
                for (int c = 0; c < nch; ++c, ++cc) {
                    if (bad) continue;
                    const int a = (int)(cc % LF_ND);
                    if (!lf_wait(dfull(a), (cc / LF_ND) & 1, LF_WAIT_LIMIT, abort_s, err)) {
                        lf_fail(abort_s, err);
                        bad = true;
                        continue;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const float f = invq[c < nch - 1 ? 0 : 1] * (1.0f / LF_GSCALE);
#pragma unroll
                    for (int q4 = 0; q4 < 4; ++q4) { // columns (part of Q, out, vector), 16 at a time
                        float v[16];
                        tc_ld16(lane_base + 64u * a + 16u * q4, v);
#pragma unroll
                        for (int m = 0; m < 16; ++m) acc[16 * (q4 & 1) + m] = fmaf(v[m], f, acc[16 * (q4 & 1) + m]);
                    }
                    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
                    __syncwarp();
                    if (lane == 0) mbar_arrive(dempty(a));
                }
                // lanes 64 .. 127 (G's lo part) pass their sums to lanes 0 .. 63
                float *xc = xch + (pp & 1) * LF_TGT * LF_XS + t * LF_XS;
                if (Q >= 2)
#pragma unroll
                    for (int m = 0; m < 32; ++m) xc[m] = acc[m];
                bad = lf_bar_or(2, 128, bad || *abort_s != 0);
                if (bad) break;
                const int i = i0 + t;
                if (Q < 2 && i < hi) {
#pragma unroll
                    for (int m = 0; m < 32; ++m) acc[m] += xc[m];
                    float4 *o = (float4 *)(us + (int64_t)i * LM_MAXV);
#pragma unroll
                    for (int v2 = 0; v2 < LM_MAXV / 2; ++v2)
                        o[v2] = make_float4(acc[2 * v2], acc[16 + 2 * v2], acc[2 * v2 + 1], acc[16 + 2 * v2 + 1]);
                }
            }
            if (bad) break;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 2) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256));
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int lm_h0_terms(double xmax);

#define LF_SWITCH(P, FN, ...)            \
    switch (P) {                         \
    case 4: return FN<4>(__VA_ARGS__);   \
    case 6: return FN<6>(__VA_ARGS__);   \
    case 8: return FN<8>(__VA_ARGS__);   \
    case 9: return FN<9>(__VA_ARGS__);   \
    case 10: return FN<10>(__VA_ARGS__); \
    case 11: return FN<11>(__VA_ARGS__); \
    case 12: return FN<12>(__VA_ARGS__); \
    case 13: return FN<13>(__VA_ARGS__); \
    case 14: return FN<14>(__VA_ARGS__); \
    default: break;                      \
    }

template <int P>
static lm_status lf_attr()
{
    LM_CUDA(cudaFuncSetAttribute(k_leaf_tt<P, 6>, cudaFuncAttributeMaxDynamicSharedMemorySize, LfSmem<P>::BYTES));
    LM_CUDA(cudaFuncSetAttribute(k_leaf_tt<P, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, LfSmem<P>::BYTES));
    return LM_OK;
}

static lm_status lf_set_attr(int p)
{
    LF_SWITCH(p, lf_attr);
    lm_set_error("tensor-core leaf step: order %d not instantiated", p);
    return LM_ENOTSUP;
}

// Enables the tensor-core leaf step for a uniform mixed-precision tree of the free
// kernel whose order has an instantiation and whose leaves have at most LF_MAXE U entries.
lm_status lm_setup_leaf_tt(lm_tree_s *t, cudaStream_t st)
{
    t->lf_ready = false;
    t->lf_poll_limit = -1;
    if (!t->tc_ready || t->adaptive || !t->med.opt.tensor_leaf || t->med.opt.kernel != LM_KERNEL_G) return LM_OK;
    bool inst = false;
    switch (t->p) {
    case 4: case 6: case 8: case 9: case 10: case 11: case 12: case 13: case 14: inst = true; break;
    default: break;
    }
    // the L2T basis series holds for k2 w <= 2 (t = (k2 r / 2)^2 <= 1/2 inside a leaf)
    if (!inst || t->L < 1 || t->n >= ((int64_t)1 << 29) || t->med.k2 * t->lev[t->L].w > 2.0) return LM_OK;
    std::vector<int64_t> us(t->nleaf + 1);
    LM_CUDA(cudaMemcpyAsync(us.data(), t->ustart, us.size() * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    LM_CUDA(cudaStreamSynchronize(st));
    for (int64_t b = 0; b < t->nleaf; ++b)
        if (us[b + 1] - us[b] > LF_MAXE) return LM_OK;
    int dev = 0, nsm = 0;
    LM_CUDA(cudaGetDevice(&dev));
    LM_CUDA(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    t->lf_grid = (int)std::max<int64_t>(1, std::min<int64_t>(nsm, t->nleaf));
    const lm_status s = lf_set_attr(t->p);
    if (s != LM_OK) return s;
    if (!t->lf_pts) {
        LM_CUDA(cudaMalloc((void **)&t->lf_pts, (size_t)std::max<int64_t>(1, t->n) * sizeof(float4)));
        t->bytes += (int64_t)std::max<int64_t>(1, t->n) * sizeof(float4);
    }
    if (!t->lf_ent) {
        LM_CUDA(cudaMalloc((void **)&t->lf_ent, (size_t)t->nleaf * LF_MAXE * sizeof(int4)));
        t->bytes += t->nleaf * LF_MAXE * (int64_t)sizeof(int4);
    }
    if (!t->lf_scl) {
        LM_CUDA(cudaMalloc((void **)&t->lf_scl, 2 * sizeof(uint32_t)));
        t->bytes += 2 * sizeof(uint32_t);
    }
    if (!t->lf_tot) {
        LM_CUDA(cudaMalloc((void **)&t->lf_tot, (size_t)t->nleaf * sizeof(int32_t)));
        t->bytes += t->nleaf * (int64_t)sizeof(int32_t);
    }
    k_lf_pts<<<(unsigned)((t->n + 255) / 256), 256, 0, st>>>(t->xl32, t->yl32, t->y32, t->n, (float4 *)t->lf_pts);
    k_lf_tot<<<(unsigned)((t->nleaf + 255) / 256), 256, 0, st>>>(t->leaf_start, t->ustart, t->usrc, t->nleaf,
                                                                  t->lf_tot);
    k_lf_ent<<<(unsigned)((t->nleaf * LF_MAXE + 255) / 256), 256, 0, st>>>(t->leaf_start, t->ustart, t->usrc,
                                                                          t->uterm, t->nleaf, (int4 *)t->lf_ent);
    LM_CUDA(cudaGetLastError());
    t->lf_ready = true;
    return LM_OK;
}

template <int P>
static lm_status lf_launch(lm_tree_s *t, const NearQuadF &nq, cudaStream_t st)
{
    const Level &lv = t->lev[t->L];
    const double xmax = t->med.k2 * lv.w * 2.0 * 1.4142135623730951 * 1.0001; // largest k r of a near pair
    const int nterms = lm_h0_terms(xmax);
    const int first = t->lf_poll_limit;
    t->lf_poll_limit = -1; // a test limit applies to one launch
    if (xmax <= 2.0 && nterms <= 6)
        k_leaf_tt<P, 6><<<t->lf_grid, LF_THREADS, LfSmem<P>::BYTES, st>>>(
            t->nleaf, lv.ncol, (float)lv.w, (float)t->med.k2, (float)t->med.d, t->xl32, t->yl32, t->y32,
            (const float4 *)t->lf_pts, t->leaf_start, (const int4 *)t->lf_ent, t->lf_tot, t->lf_scl, nq, lv.L32,
            t->qs32,
            t->us32, t->dflag + 1, first);
    else
        k_leaf_tt<P, 0><<<t->lf_grid, LF_THREADS, LfSmem<P>::BYTES, st>>>(
            t->nleaf, lv.ncol, (float)lv.w, (float)t->med.k2, (float)t->med.d, t->xl32, t->yl32, t->y32,
            (const float4 *)t->lf_pts, t->leaf_start, (const int4 *)t->lf_ent, t->lf_tot, t->lf_scl, nq, lv.L32,
            t->qs32,
            t->us32, t->dflag + 1, first);
    LM_CUDA(cudaGetLastError());
    return LM_OK;
}

void lm_free_leaf_tt(lm_tree_s *t)
{
    cudaFree(t->lf_pts);
    cudaFree(t->lf_tot);
    cudaFree(t->lf_scl);
    cudaFree(t->lf_ent);
    t->lf_ent = nullptr;
    t->lf_pts = nullptr;
    t->lf_tot = nullptr;
    t->lf_scl = nullptr;
    t->lf_ready = false;
}

lm_status lm_launch_leaf_tt(lm_tree_s *t, const NearQuadF &nq, cudaStream_t st)
{
    LF_SWITCH(t->p, lf_launch, t, nq, st);
    lm_set_error("tensor-core leaf step: order %d not instantiated", t->p);
    return LM_ENOTSUP;
}
