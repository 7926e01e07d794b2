// common.cuh -- complex arithmetic, the square-root branch and Bessel
// recurrences shared by the library's kernels (device and host-device code).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#define LM_HD __host__ __device__ __forceinline__

template <typename T>
struct cpx {
    T re, im;
};
typedef cpx<double> zd;
typedef cpx<float> zf;

template <typename T> LM_HD cpx<T> mk(T r, T i) { return cpx<T>{r, i}; }
template <typename T> LM_HD cpx<T> operator+(cpx<T> a, cpx<T> b) { return {a.re + b.re, a.im + b.im}; }
template <typename T> LM_HD cpx<T> operator-(cpx<T> a, cpx<T> b) { return {a.re - b.re, a.im - b.im}; }
template <typename T> LM_HD cpx<T> operator-(cpx<T> a) { return {-a.re, -a.im}; }
template <typename T> LM_HD cpx<T> operator*(cpx<T> a, cpx<T> b)
{
    return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename T> LM_HD cpx<T> operator*(T s, cpx<T> a) { return {s * a.re, s * a.im}; }
template <typename T> LM_HD cpx<T> operator*(cpx<T> a, T s) { return {s * a.re, s * a.im}; }
template <typename T> LM_HD cpx<T> &operator+=(cpx<T> &a, cpx<T> b)
{
    a.re += b.re;
    a.im += b.im;
    return a;
}
template <typename T> LM_HD cpx<T> conj(cpx<T> a) { return {a.re, -a.im}; }
template <typename T> LM_HD T abs2(cpx<T> a) { return a.re * a.re + a.im * a.im; }
// fused a += b * c
template <typename T> LM_HD void cfma(cpx<T> &a, cpx<T> b, cpx<T> c)
{
    a.re = fma(b.re, c.re, fma(-b.im, c.im, a.re));
    a.im = fma(b.re, c.im, fma(b.im, c.re, a.im));
}
LM_HD zd cdiv(zd a, zd b)
{
    // Smith's algorithm (scaled division without overflow for moderate ranges)
    if (fabs(b.re) >= fabs(b.im)) {
        double r = b.im / b.re, den = b.re + b.im * r;
        return {(a.re + a.im * r) / den, (a.im - a.re * r) / den};
    } else {
        double r = b.re / b.im, den = b.re * r + b.im;
        return {(a.re * r + a.im) / den, (a.im * r - a.re) / den};
    }
}
LM_HD zd cexpd(zd z)
{
    double e = exp(z.re), s, c;
    sincos(z.im, &s, &c);
    return {e * c, e * s};
}
LM_HD zd csqrtd(zd z)
{
    // principal square root
    double r = hypot(z.re, z.im);
    if (r == 0.0) return {0.0, 0.0};
    double t = sqrt(0.5 * (r + fabs(z.re)));
    if (z.re >= 0.0) return {t, 0.5 * z.im / t};
    return {0.5 * fabs(z.im) / t, copysign(t, z.im)};
}
// Branch of s = sqrt(lambda^2 - k^2) (Sec. 3, Eq. (Green)): s = -i r with
// r = sqrt(k^2 - lambda^2), Im r >= 0 (Re r >= 0 when Im r = 0); Re s >= 0.
LM_HD zd sbranch(zd lam, double k)
{
    zd z = {k * k - (lam.re * lam.re - lam.im * lam.im), -2.0 * lam.re * lam.im};
    zd r = csqrtd(z);
    if (r.im < 0.0 || (r.im == 0.0 && r.re < 0.0)) r = -r;
    return {r.im, -r.re}; // -i * r
}

// Number of orders above nmax at which Miller's backward recurrence starts (even).
LM_HD int miller_start(int nmax, double x)
{
    int ns = nmax + 16 + (int)(2.0 * x) + (int)sqrt(40.0 * (nmax + 1));
    return ns + (ns & 1);
}

// Scaled Bessel values Jhat_n(x) = J_n(x) / S(n), n = 0..nmax, with
// S(n) = (sc/2)^n / n!, by Miller's backward recurrence written for the
// scaled sequence,
//     Jhat_{n-1} = (sc/x) Jhat_n - sc^2 / (4 n (n+1)) Jhat_{n+1},
// normalised with Neumann's identity J_0 + 2 sum_m J_{2m} = 1, accumulated
// in the same scaled form.  Values are O(1) for x <= sc whatever n is, so
// the routine works in FP32 as well as FP64.  x >= 0.
template <typename T>
__device__ __forceinline__ void bessel_j_scaled(int nmax, T x, T sc, T *out)
{
    if (x < (T)1e-3 * (sc < (T)1 ? sc : (T)1)) {
        // two terms of the power series: Jhat_n = (x/sc)^n (1 - x^2 / (4 (n+1)))
        T r = x / sc, pw = (T)1;
        for (int n = 0; n <= nmax; ++n) {
            out[n] = pw * ((T)1 - x * x / ((T)4 * (T)(n + 1)));
            pw *= r;
        }
        return;
    }
    const T big = sizeof(T) == 8 ? (T)1e250 : (T)1e30;
    const int ns = miller_start(nmax, (double)x);
    const T ax = sc / x, sc2 = sc * sc * (T)0.25;
    T jn1 = (T)0, jn = (T)1;
    T acc = (T)2; // ns is even: 2 * Jhat_ns * S(ns)/S(ns)
    for (int n = ns; n >= 1; --n) {
        T jm = ax * jn - sc2 / ((T)n * (T)(n + 1)) * jn1;
        acc = acc * (sc / ((T)2 * (T)n));
        if (((n - 1) & 1) == 0) acc += (n - 1 == 0 ? (T)1 : (T)2) * jm;
        jn1 = jn;
        jn = jm;
        if (n - 1 <= nmax) out[n - 1] = jm;
        if (jn > big || jn < -big) {
            const T s = (T)1 / big;
            jn *= s;
            jn1 *= s;
            acc *= s;
            for (int m = n - 1; m <= nmax; ++m) out[m] *= s;
        }
    }
    const T f = (T)1 / acc;
    for (int n = 0; n <= nmax; ++n) out[n] *= f;
}
