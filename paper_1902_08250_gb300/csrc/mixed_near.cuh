// mixed_near.cuh -- FP32 pieces of the mixed-precision near field shared by
// the leaf kernels: the free-space kernel (i/4) H0 from its series, the
// reflected tails (Sec. 4.2 alternative directions) and a complex FMA.
#pragma once
#include "internal.h"

// asynchronous global -> shared copies (cp.async), completed per commit group
__device__ __forceinline__ void cp_async4(void *sdst, const void *gsrc)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_async16(void *sdst, const void *gsrc)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc)
                 : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void cp_async8(void *sdst, const void *gsrc)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(sdst)),
                 "l"(gsrc)
                 : "memory");
}


__device__ __forceinline__ void cfmaf(zf &a, zf b, zf c)
{
    a.re = fmaf(b.re, c.re, fmaf(-b.im, c.im, a.re));
    a.im = fmaf(b.re, c.im, fmaf(b.im, c.re, a.im));
}

// (i/4) H0^(1)(x) in FP32 as a function of t = x^2/4.  For t <= 1 (x <= 2)
// the ascending series of J0 and Y0 (Abramowitz & Stegun 9.1.12, 9.1.13),
//   J0 = sum_m c_m t^m,  c_m = (-1)^m/(m!)^2,
//   Y0 = (2/pi) [ (ln(x/2) + gamma) J0 - sum_{m>=1} H_m c_m t^m ],  ln(x/2) = ln(t)/2,
// H_m the harmonic numbers, are evaluated by Horner's rule to degree 8
// (truncation < 1e-11); no square root is needed.  Larger x use the
// library's j0f / y0f.
// the series branch alone (valid for t <= 1; finite for any t > 0)
__device__ __forceinline__ zf green_free32_series(float t)
{
    // c_m and H_m c_m for m = 8 .. 1, from the series definitions
    const float c8 = 6.15118733e-10f, c7 = -3.93675989e-08f, c6 = 1.92901235e-06f, c5 = -6.94444444e-05f,
                c4 = 1.73611111e-03f, c3 = -2.77777778e-02f, c2 = 0.25f, c1 = -1.0f;
    const float e8 = 1.67180484e-09f, e7 = -1.02074560e-07f, e6 = 4.72608025e-06f, e5 = -1.58564815e-04f,
                e4 = 3.61689815e-03f, e3 = -5.09259259e-02f, e2 = 0.375f, e1 = -1.0f;
    const float2 tt = make_float2(t, t);
    float2 pp = __ffma2_rn(make_float2(c8, e8), tt, make_float2(c7, e7));
    pp = __ffma2_rn(pp, tt, make_float2(c6, e6));
    pp = __ffma2_rn(pp, tt, make_float2(c5, e5));
    pp = __ffma2_rn(pp, tt, make_float2(c4, e4));
    pp = __ffma2_rn(pp, tt, make_float2(c3, e3));
    pp = __ffma2_rn(pp, tt, make_float2(c2, e2));
    pp = __ffma2_rn(pp, tt, make_float2(c1, e1));
    const float j = fmaf(pp.x, t, 1.0f);
    const float sh = pp.y * t;
    // MUFU logarithm: absolute error ~1e-7, well inside the 1e-6 budget
    const float y = 0.63661977236758134f * (fmaf(0.5f, __logf(t), 0.57721566490153286f) * j - sh);
    return zf{-0.25f * y, 0.25f * j};
}
// The same series truncated at degree DEG (5..8), for leaves whose near pairs all
// have t <= t_max with the first dropped term below 1e-9 (lm_h0_terms).
template <int DEG>
__device__ __forceinline__ zf green_free32_series_d(float t)
{
    static_assert(DEG >= 5 && DEG <= 8, "series degree");
    constexpr float c[9] = {1.0f, -1.0f, 0.25f, -2.77777778e-02f, 1.73611111e-03f, -6.94444444e-05f,
                            1.92901235e-06f, -3.93675989e-08f, 6.15118733e-10f};
    constexpr float e[9] = {0.0f, -1.0f, 0.375f, -5.09259259e-02f, 3.61689815e-03f, -1.58564815e-04f,
                            4.72608025e-06f, -1.02074560e-07f, 1.67180484e-09f};
    const float2 tt = make_float2(t, t);
    float2 pp = make_float2(c[DEG], e[DEG]);
#pragma unroll
    for (int m = DEG - 1; m >= 1; --m) pp = __ffma2_rn(pp, tt, make_float2(c[m], e[m]));
    const float j = fmaf(pp.x, t, 1.0f);
    const float sh = pp.y * t;
    const float y = 0.63661977236758134f * (fmaf(0.5f, __logf(t), 0.57721566490153286f) * j - sh);
    return zf{-0.25f * y, 0.25f * j};
}
// t > 1: the library's j0f / y0f
static __device__ __noinline__ zf green_free32_far(float t)
{
    const float x = 2.0f * sqrtf(t);
    return zf{-0.25f * y0f(x), 0.25f * j0f(x)};
}
__device__ __forceinline__ zf green_free32_t(float t)
{
    return t <= 1.0f ? green_free32_series(t) : green_free32_far(t);
}

struct NearQuadF {
    int nseg, nray, ntail;
    const zf *seg_lam, *seg_s2, *seg_w, *tail_lam, *tail_s2, *tail_w;
    int sym; // sigma(conj lambda) = conj(sigma(lambda)) (no impedance wall): the tail is real
    float rinf[2]; // wall limit of sigma_tt, sigma_bb: the tables hold sigma - rinf (refl_inf)
    float hray;    // added to h when the tail ray is chosen (see NearQuad)
    float k24;     // k2^2 / 4, for the wall image's closed form
};
// Tail of one reflected direct term (tt: m = 0, bb: m = 1) for a pair at
// horizontal distance X and image height h: the rays lambda = c + t e^{i phi_k}
// nearest the steepest-descent direction atan2(X, h) (Sec. 4.2, alternative
// directions); 2 Re is taken because sigma(conj lambda) = conj(sigma(lambda)).
// Kept out of line: inlined into k_leaf32 it pushes the kernel to its
// 128-register cap and slows the free-space loop by 9 % (measured).
static __device__ __noinline__ zf near_tail32(const NearQuadF &q, int m, float X, float h)
{
    int k = q.nray > 1 ? (int)rintf(atan2f(X, h + q.hray) * (q.nray - 1) * 0.63661977236758134f) : 0;
    const zf *tl = q.tail_lam + (int64_t)k * q.ntail, *ts = q.tail_s2 + (int64_t)k * q.ntail;
    const int64_t tot = (int64_t)q.nray * q.ntail;
    const zf *tP = q.tail_w + (2 * m) * tot + (int64_t)k * q.ntail, *tM = tP + tot;
    float re = 0.f, im = 0.f; // sum P Re(E) + i M Im(E)
    if (q.rinf[m] != 0.f) { // a wall's image (i/4) H0(k rho), rho = |(X, h)|, in closed form
        const zf img = q.rinf[m] * green_free32_t(q.k24 * fmaf(X, X, h * h));
        re = img.re;
        im = img.im;
    }
    if (q.sym) { // P real, M imaginary: only the real part of the tail survives
        for (int i = 0; i < q.ntail; ++i) {
            zf lam = tl[i], s2 = ts[i];
            float a = expf(-lam.im * X - s2.re * h), sn, cs;
            sincosf(lam.re * X - s2.im * h, &sn, &cs);
            re += a * (tP[i].re * cs - tM[i].im * sn);
        }
        return zf{re, im};
    }
    for (int i = 0; i < q.ntail; ++i) {
        zf lam = tl[i], s2 = ts[i];
        float a = expf(-lam.im * X - s2.re * h), sn, cs;
        sincosf(lam.re * X - s2.im * h, &sn, &cs);
        const zf P = tP[i], M = tM[i];
        re += a * (P.re * cs - M.im * sn);
        im += a * (P.im * cs + M.re * sn);
    }
    return zf{re, im};
}

