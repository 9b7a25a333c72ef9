// asm_sweep.cuh -- the chain kernel of blocked modes sampling (Ghanem & Koch,
// arXiv:1912.01379, Sec. IV.B-C) for sm_103a.
//
// Layout.  A team of S lanes (S a power of two, S <= 32) runs one chain; a warp
// runs 32/S chains.  While a block is visited, the team keeps the block's part
// of the chain state f in registers: lane s holds the 16-byte vectors
// k*S + s (k < KV) of the block.  Mode rows (V, and the masked reciprocals
// R = -1/V that give the bounds of Eq. modeLimits) are read as 16-byte vectors
// from a CTA-shared ring of move records; every chain of the same problem reads
// the same rows at the same time.  The tracked residual r~ = g~ - K~ f and the block's
// projections c_j = U_j^T r~ live in shared memory.
//
// One move of mode j (Sec. IV.B, "sample e_i' from a univariate Gaussian ...
// truncated to the interval for which f' >= 0"):
//   [lo, hi]  = interval of delta from the previous pass (team minima of the
//               bound keys, see BoundKey)
//   delta     ~ N(c_j/d_j, 1/d_j^2) on [lo, hi] by the inverse CDF (flat if d_j = 0)
//   pass      f += delta V_j, clamp at 0, and the bounds of mode j+1 in the same
//             sweep over the registers
//   w_j       = dres_j delta  (the residual moves by -w_j U_j, dres_j = |K~_b V_j|;
//               c_j is not needed again)
// Block entry computes c = U_b^T r~, block exit applies r~ -= U_b w.
#pragma once

#include <cuda_runtime.h>
#include <type_traits>
#include <math_constants.h>

#include "asm_internal.h"

namespace asmgb {

// --------------------------------------------------------------------------
// Philox4x64-10 (Salmon et al., SC'11): counter-based, so every move's uniform
// is a pure function of (seed, move, sweep, chain, problem).
// --------------------------------------------------------------------------
__device__ __forceinline__ void philox4x64_10(unsigned long long &c0, unsigned long long &c1,
                                              unsigned long long &c2, unsigned long long &c3,
                                              unsigned long long k0, unsigned long long k1)
{
    const unsigned long long M0 = 0xD2E7470EE14C6C93ull, M1 = 0xCA5A826395121157ull;
    const unsigned long long W0 = 0x9E3779B97F4A7C15ull, W1 = 0xBB67AE8584CAA73Bull;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k0 += W0; k1 += W1; }
        const unsigned long long hi0 = __umul64hi(M0, c0), lo0 = M0 * c0;
        const unsigned long long hi1 = __umul64hi(M1, c2), lo1 = M1 * c2;
        const unsigned long long y0 = hi1 ^ c1 ^ k0, y2 = hi0 ^ c3 ^ k1;
        c0 = y0; c1 = lo1; c2 = y2; c3 = lo0;
    }
}

// u in (0,1) on the grid (k + 1/2) 2^-52 (FP64) or (k + 1/2) 2^-23 (FP32, the
// top 23 bits of the same word); 1 - u is exact in both.
template <class T> __device__ __forceinline__ T uniform_from(unsigned long long w);
template <> __device__ __forceinline__ double uniform_from<double>(unsigned long long w)
{
    return ((double)(w >> 12) + 0.5) * 0x1p-52;
}
template <> __device__ __forceinline__ float uniform_from<float>(unsigned long long w)
{
    return ((float)(unsigned)(w >> 41) + 0.5f) * 0x1p-23f;
}

// --------------------------------------------------------------------------
// precision-overloaded math (CUDA math library calls)
// --------------------------------------------------------------------------
__device__ __forceinline__ double m_fma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float m_fma(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double m_max(double a, double b) { return fmax(a, b); }
__device__ __forceinline__ float m_max(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double m_min(double a, double b) { return fmin(a, b); }
__device__ __forceinline__ float m_min(float a, float b) { return fminf(a, b); }
__device__ __forceinline__ double m_phi(double x) { return normcdf(x); }
__device__ __forceinline__ float m_phi(float x) { return normcdff(x); }
__device__ __forceinline__ double m_phiinv(double p) { return normcdfinv(p); }
__device__ __forceinline__ float m_phiinv(float p) { return normcdfinvf(p); }
__device__ __forceinline__ double m_erfcx(double x) { return erfcx(x); }
__device__ __forceinline__ float m_erfcx(float x) { return erfcxf(x); }
__device__ __forceinline__ double m_log(double x) { return log(x); }
__device__ __forceinline__ float m_log(float x) { return logf(x); }
__device__ __forceinline__ double m_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float m_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double m_exp(double x) { return exp(x); }
__device__ __forceinline__ float m_exp(float x) { return expf(x); }
__device__ __forceinline__ double m_expm1(double x) { return expm1(x); }
__device__ __forceinline__ float m_expm1(float x) { return expm1f(x); }
__device__ __forceinline__ double m_abs(double x) { return fabs(x); }
__device__ __forceinline__ float m_abs(float x) { return fabsf(x); }

template <class T> struct TailTraits;
// far: with both standardized bounds beyond +-far, Phi(a) and 1 - Phi(b) are
// below half an ulp of the smallest uniform (2^-53 resp. 2^-24), so
// (1-u) Phi(a) + u Phi(b) rounds to u: Phi(-12) = 1.8e-33 < 2^-107 and
// Phi(-10) = 7.6e-24 < 2^-49.
template <> struct TailTraits<double> {
    static constexpr double tol = 1e-14;
    static constexpr int nmax = 40;
    static constexpr double far = 12.0;
};
template <> struct TailTraits<float> {
    static constexpr float tol = 2e-6f;
    static constexpr int nmax = 16;
    static constexpr float far = 10.0f;
};

// x ~ N(0,1) restricted to [a, a + w], a >= 0, 0 < w <= inf, by Q(x) = (1-u)Q(a) + uQ(b),
// b = a + w.  The width comes in as w, formed from the interval's ends before they are
// standardised: b - a of two standardised ends far in the tail cancels (a = 35 and
// w = 0.03 leave w with a relative error of 2^-24 a / w = 7e-5 in FP32).
// Returns the offset y = x - a.  The equation in y,
//   log Q(a + y) - log Q(a) = dt,  dt = log((1-u) + u Q(b)/Q(a)),
// is solved by Newton's method on log Q (concave, so the iterates are monotone
// after the first step), with Q(b)/Q(a) formed through erfcx to keep narrow
// intervals accurate.  The start is the exponential tail's inverse for a >= 5
// and, below, y = -Phi^{-1}(q) - a with q = (1-u)Q(a) + uQ(b): accurate to a
// few ulp of a, which FP32 keeps; in FP64 the offset form refines it so that y
// keeps its relative accuracy however small it is.
template <class T>
__device__ __forceinline__ T right_tail(T a, T w, T u, int &capped)
{
    const T b = a + w;
    const T kRsqrt2 = T(0.70710678118654752440);
    const T kSqrtPiOver2 = T(1.25331413731550025121);
    constexpr bool kRefine = sizeof(T) == 8;
    T y;
    if (a < T(5)) {
        const T qa = m_phi(-a);
        const T qb = isinf(b) ? T(0) : m_phi(-b);
        const T q = (T(1) - u) * qa + u * qb;
        y = -m_phiinv(q) - a;
    }
    if (a >= T(5) || (kRefine && a > T(0))) {
        const T exa = m_erfcx(a * kRsqrt2);
        T r = T(0), em = T(-1);
        if (!isinf(b)) {
            const T lr = m_log(m_erfcx(b * kRsqrt2) / exa) - T(0.5) * w * (a + b);
            r = m_exp(lr);
            em = m_expm1(lr);
        }
        const T dt = r < T(0.5) ? m_log((T(1) - u) + u * r) : m_log1p(u * em);
        if (a >= T(5)) y = -dt / a;
        int it = 0;
        for (; it < TailTraits<T>::nmax; ++it) {
            const T exy = m_erfcx((a + y) * kRsqrt2);
            const T g = m_log(exy / exa) - y * (a + T(0.5) * y) - dt;
            const T step = -g * exy * kSqrtPiOver2;   // g / g', g' = -sqrt(2/pi)/erfcx
            y -= step;
            if (m_abs(step) <= TailTraits<T>::tol * (y + T(1) / a)) break;
        }
        if (it == TailTraits<T>::nmax) ++capped;
    }
    y = m_max(y, T(0));
    y = m_min(y, w);
    return y;
}

// Gauss-Legendre rule on [-1, 1] (symmetric half: nodes x > 0 and weights;
// values of numpy.polynomial.legendre.leggauss).  8 points for FP64 (relative
// error ~2e-16 on the narrow intervals below), 4 points for FP32 (~2e-10).
template <class T> struct GaussLegendre;
template <> struct GaussLegendre<double> {
    static constexpr int half = 4;
    __device__ static constexpr double x(int i)
    {
        return i == 0 ? 0.18343464249564978 : i == 1 ? 0.525532409916329 : i == 2 ? 0.7966664774136267
                                                                                 : 0.9602898564975362;
    }
    __device__ static constexpr double w(int i)
    {
        return i == 0 ? 0.36268378337836166 : i == 1 ? 0.3137066458778869 : i == 2 ? 0.22238103445337443
                                                                                  : 0.10122853629037706;
    }
    static constexpr double tol = 4e-16;
    static constexpr int nmax = 40;
};
template <> struct GaussLegendre<float> {
    static constexpr int half = 2;
    __device__ static constexpr float x(int i) { return i == 0 ? 0.33998104358485626f : 0.8611363115940526f; }
    __device__ static constexpr float w(int i) { return i == 0 ? 0.6521451548625464f : 0.34785484513745357f; }
    static constexpr float tol = 4e-7f;
    static constexpr int nmax = 12;
};

// I(t) = int_0^t exp(-a s - s^2/2) ds (the CDF of N(0,1) on [a, a+w] from a,
// unnormalised) by Gauss-Legendre; accurate while t (|a| + t) <= 1/2.
template <class T>
__device__ __forceinline__ T narrow_cdf(T a, T t)
{
    using GL = GaussLegendre<T>;
    const T h = T(0.5) * t;
    T acc = T(0);
#pragma unroll
    for (int i = 0; i < GL::half; ++i) {
        const T s1 = h * (T(1) - GL::x(i)), s2 = h * (T(1) + GL::x(i));
        acc += GL::w(i) * (m_exp(-s1 * (a + T(0.5) * s1)) + m_exp(-s2 * (a + T(0.5) * s2)));
    }
    return h * acc;
}

// Narrow interval (w (|a| + w) <= 1/2, the Gaussian nearly flat across it):
// solve I(t) = u I(w) by Newton's method.  The start is the inverse CDF of the
// exponential law whose rate is the log-density's slope at the interval's
// midpoint, lam = a + w/2: the neglected curvature changes the log-density by
// at most w^2/8 across the interval, so one or two steps converge where the
// flat start t = u w needed four.  The offset t from the lower end keeps its
// relative accuracy however narrow the interval is.
// In FP32 the start is the answer when w^2 / 8, the curvature's bound on the
// relative error of the exponential law's CDF, lies below 2^-23 (w <= 6e-4: the
// weak modes whose intervals are a tiny fraction of their Gaussian's width),
// and one Newton step is when w <= 0.2: Newton's error is quadratic in the
// start's, which is below w^2/12 relative, and one step leaves at most 1.5e-7
// relative over the narrow regime with w <= 0.2 (measured against the root of
// a 64-point rule at 4 million (a, w, u)), below the FP32 tolerance.
template <class T>
__device__ __forceinline__ T narrow_offset(T a, T w, T u, int &capped)
{
    using GL = GaussLegendre<T>;
    const T lam = a + T(0.5) * w;
    const T x = lam * w;
    T t = m_abs(x) < T(1e-3) ? u * w * (T(1) - T(0.5) * x * (T(1) - u))   // the series for small lam w
                             : -m_log1p(u * m_expm1(-x)) / lam;
    t = m_min(m_max(t, T(0)), w);
    if (sizeof(T) == 4 && w * w <= T(4e-7)) return t;
    const T target = u * narrow_cdf(a, w);
    if (sizeof(T) == 4 && w <= T(0.2)) {
        const T step = (narrow_cdf(a, t) - target) / m_exp(-t * (a + T(0.5) * t));
        return m_min(m_max(t - step, T(0)), w);
    }
    int it = 0;
    for (; it < GL::nmax; ++it) {
        const T step = (narrow_cdf(a, t) - target) / m_exp(-t * (a + T(0.5) * t));
        t = m_min(m_max(t - step, T(0)), w);
        if (m_abs(step) <= GL::tol * t || t == T(0)) break;
    }
    if (it == GL::nmax) ++capped;
    return t;
}

// delta ~ N(c/d, 1/d^2) restricted to [lo, hi] (lo < hi), by the inverse CDF at u.
// In standard units x = d delta - c the interval is [a, b] = [d lo - c, d hi - c].
// Each branch returns delta in the form that keeps delta - lo (or hi - delta)
// accurate relative to hi - lo.
template <class T>
__device__ __forceinline__ T tn_step(T c, T d, T invd, T lo, T hi, T u, int &capped)
{
    const T a = m_fma(lo, d, -c);
    const T b = m_fma(hi, d, -c);
    const T wid = (hi - lo) * d;
    T delta;
    if (isfinite(wid) && wid * (m_abs(a) + wid) <= T(0.5)) {
        delta = lo + invd * narrow_offset(a, wid, u, capped);
    } else if (a >= T(0)) {
        delta = lo + invd * right_tail(a, wid, u, capped);
    } else if (b <= T(0)) {
        delta = hi - invd * right_tail(-b, wid, T(1) - u, capped);
    } else if (a < -TailTraits<T>::far && b > TailTraits<T>::far) {
        // the truncation is below the resolution of u: the untruncated inverse CDF
        const T x = u <= T(0.5) ? m_phiinv(u) : -m_phiinv(T(1) - u);
        delta = (x + c) * invd;
    } else {
        const T p = (T(1) - u) * m_phi(a) + u * m_phi(b);
        T x;
        if (p <= T(0.5)) {
            x = m_phiinv(p);
        } else {
            x = -m_phiinv((T(1) - u) * m_phi(-a) + u * m_phi(-b));
        }
        delta = (x + c) * invd;
    }
    return m_min(m_max(delta, lo), hi);
}

// --------------------------------------------------------------------------
// 16-byte vector loads through the read-only path
// --------------------------------------------------------------------------
template <class T> struct VecOf;
template <> struct VecOf<float> { static constexpr int n = 4; };
template <> struct VecOf<double> { static constexpr int n = 2; };

__device__ __forceinline__ void ldv(const float *p, float (&o)[4])
{
    const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void ldv(const double *p, double (&o)[2])
{
    const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
    o[0] = v.x; o[1] = v.y;
}

// Bound keys.  With x >= +0 and R = -1/V (NaN where V is left out of the
// bounds), t = x R is <= -0 exactly when V > 0 (a lower-bound candidate for
// the step) and >= +0 when V < 0 (an upper-bound candidate).  Read as integers
// of the same width, the largest lower candidate is the SIGNED minimum of the
// bit patterns of all t (negative floats order by magnitude, above every
// negative the -inf of the initial key) and the smallest upper candidate the
// UNSIGNED minimum (negative floats and NaN lie above +inf).  One multiply and
// two integer minima per element, one R row instead of two.
template <class T> struct BoundKey;
template <> struct BoundKey<float> {
    using S = int;
    using U = unsigned;
    static constexpr S lo0 = (S)0xff800000;   // -inf
    static constexpr U hi0 = 0x7f800000u;     // +inf
    static __device__ __forceinline__ S bits(float x) { return __float_as_int(x); }
    static __device__ __forceinline__ float lo_of(S k) { return __int_as_float(k); }
    static __device__ __forceinline__ float hi_of(U k) { return __uint_as_float(k); }
};
template <> struct BoundKey<double> {
    using S = long long;
    using U = unsigned long long;
    static constexpr S lo0 = (S)0xfff0000000000000ull;
    static constexpr U hi0 = 0x7ff0000000000000ull;
    static __device__ __forceinline__ S bits(double x) { return __double_as_longlong(x); }
    static __device__ __forceinline__ double lo_of(S k) { return __longlong_as_double(k); }
    static __device__ __forceinline__ double hi_of(U k) { return __longlong_as_double((long long)k); }
};
template <class T>
__device__ __forceinline__ void key_update(typename BoundKey<T>::S &lk, typename BoundKey<T>::U &hk, T t)
{
    const typename BoundKey<T>::S k = BoundKey<T>::bits(t);
    lk = k < lk ? k : lk;
    const typename BoundKey<T>::U ku = (typename BoundKey<T>::U)k;
    hk = ku < hk ? ku : hk;
}

// One 16-byte chunk of the pass: x = max(f + delta V, +0), f = x, and the keys
// of t = x R into two accumulator pairs (even and odd element), so that the
// chain of integer minima is half as long.  The minima are exact, so the keys
// do not depend on the grouping.  FP32: the products and the fused
// multiply-adds in packed pairs (one instruction per two elements, each
// element rounded as by the scalar instruction).
template <class T>
struct Keys {
    typename BoundKey<T>::S l0, l1;
    typename BoundKey<T>::U h0, h1;
    __device__ __forceinline__ void reset()
    {
        l0 = l1 = BoundKey<T>::lo0;
        h0 = h1 = BoundKey<T>::hi0;
    }
    __device__ __forceinline__ void fold(typename BoundKey<T>::S &lk, typename BoundKey<T>::U &hk) const
    {
        lk = l1 < l0 ? l1 : l0;
        hk = h1 < h0 ? h1 : h0;
    }
};
__device__ __forceinline__ void pass_chunk(float (&f)[4], float delta, const float (&vv)[4], const float (&rr)[4],
                                           Keys<float> &kk)
{
    const float2 d2 = make_float2(delta, delta);
    float2 a = __ffma2_rn(d2, make_float2(vv[0], vv[1]), make_float2(f[0], f[1]));
    float2 b = __ffma2_rn(d2, make_float2(vv[2], vv[3]), make_float2(f[2], f[3]));
    a.x = fmaxf(a.x, 0.0f);
    a.y = fmaxf(a.y, 0.0f);
    b.x = fmaxf(b.x, 0.0f);
    b.y = fmaxf(b.y, 0.0f);
    f[0] = a.x; f[1] = a.y; f[2] = b.x; f[3] = b.y;
    const float2 ta = __fmul2_rn(a, make_float2(rr[0], rr[1]));
    const float2 tb = __fmul2_rn(b, make_float2(rr[2], rr[3]));
    key_update<float>(kk.l0, kk.h0, ta.x);
    key_update<float>(kk.l1, kk.h1, ta.y);
    key_update<float>(kk.l0, kk.h0, tb.x);
    key_update<float>(kk.l1, kk.h1, tb.y);
}
__device__ __forceinline__ void pass_chunk(double (&f)[2], double delta, const double (&vv)[2],
                                           const double (&rr)[2], Keys<double> &kk)
{
    double x0 = fmax(fma(delta, vv[0], f[0]), 0.0);
    double x1 = fmax(fma(delta, vv[1], f[1]), 0.0);
    f[0] = x0;
    f[1] = x1;
    key_update<double>(kk.l0, kk.h0, x0 * rr[0]);
    key_update<double>(kk.l1, kk.h1, x1 * rr[1]);
}
// Keys alone (the first mode of a block: f is unchanged, t = f R).
__device__ __forceinline__ void key_chunk(const float (&f)[4], const float (&rr)[4], Keys<float> &kk)
{
    const float2 ta = __fmul2_rn(make_float2(f[0], f[1]), make_float2(rr[0], rr[1]));
    const float2 tb = __fmul2_rn(make_float2(f[2], f[3]), make_float2(rr[2], rr[3]));
    key_update<float>(kk.l0, kk.h0, ta.x);
    key_update<float>(kk.l1, kk.h1, ta.y);
    key_update<float>(kk.l0, kk.h0, tb.x);
    key_update<float>(kk.l1, kk.h1, tb.y);
}
__device__ __forceinline__ void key_chunk(const double (&f)[2], const double (&rr)[2], Keys<double> &kk)
{
    key_update<double>(kk.l0, kk.h0, f[0] * rr[0]);
    key_update<double>(kk.l1, kk.h1, f[1] * rr[1]);
}

// The lane's bound keys of a block's first mode from f (>= +0, so that
// max(f + 0 V, +0) = f and the pass reduces to the products) and that mode's R
// row, read from global memory.
template <class T, int KV>
__device__ __forceinline__ void first_keys(const T (&f)[KV][VecOf<T>::n], const T *__restrict__ rrow, int kcnt,
                                           int sl, int S, typename BoundKey<T>::S &lk,
                                           typename BoundKey<T>::U &hk)
{
    constexpr int VEC = VecOf<T>::n;
    Keys<T> kk;
    kk.reset();
#pragma unroll
    for (int k = 0; k < KV; ++k) {
        if (k < kcnt) {
            T rr[VEC];
            ldv(rrow + VEC * (k * S + sl), rr);
            key_chunk(f[k], rr, kk);
        }
    }
    kk.fold(lk, hk);
}

// --------------------------------------------------------------------------
// bulk copies (TMA engine) and mbarriers, inline PTX
// --------------------------------------------------------------------------
__device__ __forceinline__ unsigned smem_addr(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_test_wait(unsigned long long *bar, unsigned parity)
{
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait: gives up after `limit` polls (each poll may suspend briefly).
__device__ __forceinline__ bool mbar_wait(unsigned long long *bar, unsigned parity, int limit)
{
    for (int i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
// Consumer-side wait: a non-blocking test first (the record has usually
// landed long before it is needed), then the suspending wait, bounded.
__device__ __forceinline__ bool mbar_wait_ready(unsigned long long *bar, unsigned parity, int limit)
{
    if (mbar_test_wait(bar, parity)) return true;
    return mbar_wait(bar, parity, limit);
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, unsigned bytes, unsigned long long *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}


// Team-wide bounds from the lanes' keys: signed and unsigned integer minima
// (FP32: one redux instruction each; FP64: a butterfly of shuffles).
__device__ __forceinline__ void team_bounds(int lk, unsigned hk, float &lo, float &hi, int S, int team_base)
{
    const unsigned mask = S == 32 ? 0xffffffffu : (((1u << S) - 1u) << team_base);
    lo = __int_as_float(__reduce_min_sync(mask, lk));
    hi = __uint_as_float(__reduce_min_sync(mask, hk));
}
__device__ __forceinline__ void team_bounds(long long lk, unsigned long long hk, double &lo, double &hi, int S, int)
{
    for (int off = 1; off < S; off <<= 1) {
        const long long l2 = __shfl_xor_sync(0xffffffffu, lk, off);
        const unsigned long long h2 = __shfl_xor_sync(0xffffffffu, hk, off);
        lk = l2 < lk ? l2 : lk;
        hk = h2 < hk ? h2 : hk;
    }
    lo = __longlong_as_double(lk);
    hi = __longlong_as_double((long long)hk);
}

// 16-byte vector loads from shared memory
__device__ __forceinline__ void lds_v(const float *p, float (&o)[4])
{
    const float4 v = *reinterpret_cast<const float4 *>(p);
    o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void lds_v(const double *p, double (&o)[2])
{
    const double2 v = *reinterpret_cast<const double2 *>(p);
    o[0] = v.x; o[1] = v.y;
}

// f += delta * V (clamped at +0) and the lane's bound keys of the next mode,
// rows read from a shared-memory stage.
// The caller loads chunk 0 (v0, r0) ahead of the draw; kcnt >= 1.  The pass
// covers chunks 0 .. KK-1; with CHK each is tested against kcnt, without it
// all KK are present (kcnt == KK), so the loop has no branch.
template <class T, int KV, int KK = KV, bool CHK = true>
__device__ __forceinline__ void fused_pass_smem(T (&f)[KV][VecOf<T>::n], T delta, const T (&v0)[VecOf<T>::n],
                                                const T (&r0)[VecOf<T>::n], const T *vrow, const T *rrow,
                                                int kcnt, int sl, int S, typename BoundKey<T>::S &lk,
                                                typename BoundKey<T>::U &hk)
{
    constexpr int VEC = VecOf<T>::n;
    static_assert(KK >= 1 && KK <= KV, "chunk count");
    Keys<T> kk;
    kk.reset();
#pragma unroll
    for (int k = 0; k < KK; ++k) {
        if (!CHK || k < kcnt) {
            const int idx = VEC * (k * S + sl);
            if (k == 0) {
                pass_chunk(f[0], delta, v0, r0, kk);
            } else {
                T vv[VEC], rr[VEC];
                lds_v(vrow + idx, vv);
                lds_v(rrow + idx, rr);
                pass_chunk(f[k], delta, vv, rr, kk);
            }
        }
    }
    kk.fold(lk, hk);
}

// --------------------------------------------------------------------------
// Position in the stream of moves of a launch (sweep, level, block, mode).
// --------------------------------------------------------------------------
struct MoveCursor {
    long long s, s_end;     // sweep, end of the launch's range
    int bi, j;              // block within the level, mode within the block
    int nb;                 // blocks of the level
    const BlockDesc *bd;    // blocks of the level
    BlockDesc B;            // the current block (a copy)
    bool done;
};

// The launch's sweep range, read from the device control block.
struct SweepRange {
    long long sweep0, nsweeps, burn_in;
};

// A warp's position in the record ring: records seen (g), stage and phase
// (kept incrementally: no division per move).
struct RingPos {
    unsigned g;             // stages in this launch (< 2^32: one launch is at most 64 sweeps)
    int slot;
    unsigned phase;
    unsigned ug;            // block visits whose U went through the two U stages
};

// Bytes of block B's U in its staging layout, and whether it goes through the U stages.
template <class T>
__device__ __forceinline__ unsigned u_stage_bytes(const BlockDesc &B)
{
    return (unsigned)((((size_t)B.np * B.usr * sizeof(T)) + 15) / 16 * 16);
}
template <class T>
__device__ __forceinline__ bool u_staged(const LaunchShape &sh, const BlockDesc &B)
{
    return sh.ubytes > 0 && u_stage_bytes<T>(B) <= (unsigned)sh.ubytes;
}

__device__ __forceinline__ void ring_next(RingPos &r, int depth)
{
    ++r.g;
    if (++r.slot == depth) {
        r.slot = 0;
        r.phase ^= 1u;
    }
}

__device__ __forceinline__ int level_of_sweep(long long s, unsigned long long seed, unsigned long long pid,
                                              int n_levels)
{
    unsigned long long l0 = ~0ull, l1 = (unsigned long long)s, l2 = 0ull, l3 = pid;
    philox4x64_10(l0, l1, l2, l3, seed, 0ull);
    int level = (int)(uniform_from<double>(l0) * n_levels);
    return level >= n_levels ? n_levels - 1 : level;
}

template <class T>
__device__ __forceinline__ void cursor_start_sweep(MoveCursor &c, const SweepParams<T> &p)
{
    const int level = level_of_sweep(c.s, p.seed, p.problem_id, p.n_levels);
    c.nb = p.level_nblocks[level];
    c.bd = p.blocks + p.level_first[level];
    c.bi = 0;
    c.j = 0;
    c.B = c.bd[0];
}

template <class T>
__device__ __forceinline__ void cursor_advance(MoveCursor &c, const SweepParams<T> &p, int n = 1)
{
    if ((c.j += n) < c.B.n) return;
    c.j = 0;
    if (++c.bi < c.nb) {
        c.B = c.bd[c.bi];
        return;
    }
    if (++c.s >= c.s_end) {
        c.done = true;
        return;
    }
    cursor_start_sweep(c, p);
}

__device__ __forceinline__ void mbar_arrive(unsigned long long *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}
// Arrival by lane 0 of the warp only, as a predicated instruction (no branch).
__device__ __forceinline__ void mbar_arrive_lane0(unsigned long long *bar, int lane)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.eq.s32 p, %1, 0;\n\t"
        "@p mbarrier.arrive.shared::cta.b64 _, [%0];\n\t}" ::"r"(smem_addr(bar)),
        "r"(lane)
        : "memory");
}

// --------------------------------------------------------------------------
// The producer warp: one bulk copy per stage of up to sh.rps consecutive move
// records of one block into the ring, after every consumer warp has released
// the slot's previous stage.  The ring position runs on across the CTA's items.
// --------------------------------------------------------------------------
template <class T>
__device__ __forceinline__ void produce(const SweepParams<T> &p, const LaunchShape &sh, const SweepRange &rg,
                                        unsigned long long *full, unsigned long long *empty,
                                        unsigned char *stages, unsigned long long *ufull, unsigned long long *uempty,
                                        unsigned char *ubuf, RingPos &rp, bool &failed)
{
    if ((threadIdx.x & 31) != 0 || rg.nsweeps <= 0 || failed || sh.stall) return;
    const int D = sh.depth;
    MoveCursor c;
    c.s = rg.sweep0;
    c.s_end = rg.sweep0 + rg.nsweeps;
    c.done = false;
    cursor_start_sweep(c, p);
    const unsigned g0 = rp.g, ug0 = rp.ug;
    while (!c.done) {
        // a block visit starts: its U into the next U stage (after that stage's previous
        // U has been released by every consumer warp)
        if (c.j == 0 && u_staged<T>(sh, c.B)) {
            const unsigned us = rp.ug & 1u;
            if (rp.ug >= 2u && !mbar_wait(uempty + us, ((rp.ug >> 1) & 1u) ^ 1u, sh.wait_limit)) {
                failed = true;
                break;
            }
            const unsigned ubytes = u_stage_bytes<T>(c.B);
            mbar_expect_tx(ufull + us, ubytes);
            bulk_g2s(ubuf + (size_t)us * sh.ubytes, p.pd.Us + c.B.offUs, ubytes, ufull + us);
            ++rp.ug;
        }
        // the slot's previous stage (phase ^ 1) must have been released
        if (rp.g >= (unsigned)D && !mbar_wait(empty + rp.slot, rp.phase ^ 1u, sh.wait_limit)) {
            failed = true;
            break;
        }
        const int nrec = min(sh.rps, c.B.n - c.j);   // records of this stage (a stage stays in its block)
        const unsigned bytes = (unsigned)(nrec * c.B.recstride * sizeof(T));
        mbar_expect_tx(full + rp.slot, bytes);
        bulk_g2s(stages + (size_t)rp.slot * sh.stage_bytes, p.pd.rec + c.B.offRec + (size_t)c.j * c.B.recstride,
                 bytes, full + rp.slot);
        ring_next(rp, D);
        cursor_advance(c, p, nrec);
    }
    if (failed) {
        // the copies already issued must land before the CTA may exit
        const unsigned g = rp.g;
        const unsigned from = g > g0 + (unsigned)D ? g - D : g0;
        for (unsigned k = from; k < g; ++k)
            mbar_wait(full + (k % (unsigned)D), (k / (unsigned)D) & 1u, sh.wait_limit);
        const unsigned ufrom = rp.ug > ug0 + 2u ? rp.ug - 2u : ug0;
        for (unsigned k = ufrom; k < rp.ug; ++k) mbar_wait(ufull + (k & 1u), (k >> 1) & 1u, sh.wait_limit);
        atomicAdd(&p.counters->timeouts, 1ull);
    }
}

// --------------------------------------------------------------------------
// A consumer warp: its team(s) of S lanes run the chains of chain group
// `group` (consumers x 32/S chains) of problem p for the launch's sweeps.
// WIDE: the block entry/exit projections keep sixteen loads in flight instead
// of eight (same accumulation order); it pays in the kernels budgeted for two
// CTAs per SM and costs a little in the 255-register ones.
// --------------------------------------------------------------------------
template <class T, int KV, bool PRIOR, bool WIDE>
__device__ __forceinline__ void consume(const SweepParams<T> &p, const LaunchShape &sh, const SweepRange &rg,
                                        int group, unsigned char *smem_raw, unsigned long long *full,
                                        unsigned long long *empty, unsigned char *stages, unsigned long long *ufull,
                                        unsigned long long *uempty, unsigned char *ubuf, RingPos &rp, bool &failed)
{
    constexpr int VEC = VecOf<T>::n;
    if (failed) return;
    const int lane = threadIdx.x & 31;
    const int wcta = threadIdx.x >> 5;
    const int D = sh.depth;
    const int S = sh.S;
    const int TW = 32 / S;
    const int team = lane / S;
    const int sl = lane - team * S;
    const int team_base = team * S;
    const long long gwarp = (long long)group * sh.consumers + wcta;
    const long long q_raw = gwarp * TW + team;
    const bool active = q_raw < p.chains;
    const long long q = active ? q_raw : (long long)p.chains - 1;  // idle teams shadow a real chain, write nothing

    // per team in shared memory: c (cpad), w (cpad), r~ (mpad), the uniforms of the
    // current window of 4S moves and, where they fit (npad > 0), the sums of f and f^2
    // over this launch's kept sweeps (FP32; at most one refresh period of terms)
    T *csm = reinterpret_cast<T *>(smem_raw) + (size_t)(wcta * TW + team) * sh.team_words;
    T *wsm = csm + sh.cpad;
    T *rsm = wsm + sh.cpad;
    T *usm = rsm + sh.mpad;   // 4S uniforms of the draws, then 4S of the prior's acceptances
    // FP32 chain state: the kept-sweep sums of the current kBinSweeps-sweep block (aligned
    // to absolute sweep indices) in FP32, added to the FP64 sums when the block closes.
    // Between launches they wait in the workspace (P1, P2); during one they live in shared
    // memory where they fit, else in the workspace -- the same arithmetic in the same order
    // either way, so results do not depend on where a run is split into calls.
    // FP64 chain state: straight into the FP64 sums.
    constexpr bool psums = sizeof(T) == 4;
    const bool kept_here = psums && rg.burn_in < rg.sweep0 + rg.nsweeps;
    T *P1q = psums ? reinterpret_cast<T *>(p.P1) + (size_t)q * p.ldF : nullptr;
    T *P2q = psums ? reinterpret_cast<T *>(p.P2) + (size_t)q * p.ldF : nullptr;
    T *p1sm = sh.npad ? usm + 8 * S : P1q;
    T *p2sm = sh.npad ? p1sm + sh.npad : P2q;
    if (kept_here && sh.npad)
        for (int n = sl; n < p.N; n += S) {
            p1sm[n] = P1q[n];
            p2sm[n] = P2q[n];
        }
    T *Rq = p.R + (size_t)q * p.ldR;
    for (int m = sl; m < p.M; m += S) rsm[m] = Rq[m];
    T *Fq = p.F + (size_t)q * p.ldF;
    double *S1q = p.S1 + (size_t)q * p.N;
    double *S2q = p.S2 + (size_t)q * p.N;
    __syncwarp();

    T f[KV][VEC];
    unsigned n_deg = 0, n_zero = 0, n_bad = 0, n_rej = 0;   // per launch: at most 64 sweeps of moves
    const bool trace = p.steptrace != nullptr;   // step-size trace of Fig. MCsteps (diagnostic)
    int capped = 0;
    const long long s_end = rg.sweep0 + rg.nsweeps;
    for (long long s = rg.sweep0; s < s_end && !failed; ++s) {
        // level of this sweep: same for every chain of the problem (Sec. IV.C)
        const int level = level_of_sweep(s, p.seed, p.problem_id, p.n_levels);
        const bool keep = s >= rg.burn_in;
        int win = 0, win_end = -1;  // window [win, win_end) of moves whose uniforms are in usm
        const int nb = p.level_nblocks[level];
        const BlockDesc *bd = p.blocks + p.level_first[level];
        T sd2 = T(0), sf2 = T(0);   // this lane's |f(s+1) - f(s)|^2 and |f(s)|^2 (trace only)

        for (int bi = 0; bi < nb && !failed; ++bi) {
            const BlockDesc B = bd[bi];
            const int kcnt = (B.n + VEC * S - 1) / (VEC * S);
            // entry: the block's f into registers
#pragma unroll
            for (int k = 0; k < KV; ++k)
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    const int nl = VEC * (k * S + sl) + v;
                    f[k][v] = (k < kcnt && nl < B.n) ? Fq[B.start + nl] : T(0);
                }
            // U of this block: from its U stage once the producer's copy has landed, else
            // from global memory
            const bool ust = u_staged<T>(sh, B);
            const T *Us = nullptr;
            if (ust) {
                bool ok = mbar_test_wait(ufull + (rp.ug & 1u), (rp.ug >> 1) & 1u);
                if (__any_sync(0xffffffffu, !ok)) {
                    ok = ok || mbar_wait(ufull + (rp.ug & 1u), (rp.ug >> 1) & 1u, sh.wait_limit);
                    if (__any_sync(0xffffffffu, !ok)) {   // decided warp-wide
                        failed = true;
                        break;
                    }
                }
                Us = reinterpret_cast<const T *>(ubuf + (size_t)(rp.ug & 1u) * sh.ubytes);
            }
            // c = U_b^T r~ (lanes split the modes; eight (WIDE: sixteen) loads in flight, eight
            // partial sums, partial sum i taking the terms m = i mod 8 in increasing m; the
            // same sums in the same order from the U stage)
            const T *Um = p.pd.Um + B.offU;
            if (ust) {
                // two of the lane's modes at a time (j, j + S): two independent chains of sums
                // (one at a time in the widest register tiles, whose registers hold f)
                for (int j = sl; j < B.np; j += (KV <= 8 ? 2 : 1) * S) {
                    const bool two = KV <= 8 && j + S < B.np;
                    const T *u = Us + (size_t)j * B.usr;
                    const T *u2 = Us + (size_t)(two ? j + S : j) * B.usr;
                    T a[8], b[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) a[i] = b[i] = T(0);
                    int m = 0;
                    for (; m + 7 < p.M; m += 8) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const T r = rsm[m + i];
                            a[i] = m_fma(u[m + i], r, a[i]);
                            b[i] = m_fma(u2[m + i], r, b[i]);
                        }
                    }
                    for (; m < p.M; ++m) {
                        a[0] = m_fma(u[m], rsm[m], a[0]);
                        b[0] = m_fma(u2[m], rsm[m], b[0]);
                    }
                    csm[j] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
                    if (two) csm[j + S] = ((b[0] + b[1]) + (b[2] + b[3])) + ((b[4] + b[5]) + (b[6] + b[7]));
                }
            } else
            for (int j = sl; j < B.np; j += S) {
                T a[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = T(0);
                int m = 0;
                if constexpr (WIDE) {
                    for (; m + 15 < p.M; m += 16) {
                        T x[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) x[i] = __ldg(Um + (size_t)(m + i) * B.np + j);
#pragma unroll
                        for (int i = 0; i < 16; ++i) a[i & 7] = m_fma(x[i], rsm[m + i], a[i & 7]);
                    }
                }
                for (; m + 7 < p.M; m += 8) {
                    T x[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) x[i] = __ldg(Um + (size_t)(m + i) * B.np + j);
#pragma unroll
                    for (int i = 0; i < 8; ++i) a[i] = m_fma(x[i], rsm[m + i], a[i]);
                }
                for (; m < p.M; ++m) a[0] = m_fma(__ldg(Um + (size_t)m * B.np + j), rsm[m], a[0]);
                csm[j] = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
            }
            __syncwarp();

            typename BoundKey<T>::S lk;
            typename BoundKey<T>::U hk;
            first_keys<T, KV>(f, p.pd.R + B.offR, kcnt, sl, S, lk, hk);  // keys of mode 0
            // The block's moves.  Where the lane's chunk count is 1 (blocks of at most
            // VEC*S points) or KV (every chunk present) it is a compile-time constant and
            // the move loop tests no chunk; the uniforms are refilled once per window of
            // 4S moves, outside the loop over the window's moves.
            auto block_moves = [&](auto chunks) {
                constexpr int KC = decltype(chunks)::value;   // 0: kcnt chunks, each tested
                constexpr int KK = KC ? KC : KV;
                constexpr bool CHK = KC == 0;
                int jr = 0;                        // record of move j within its ring stage
                const T *stb = nullptr;            // the stage holding move j's record
                for (int j = 0; j < B.n && !failed;) {
                    // uniform of move t: word t%4 of Philox(ctr = {t/4, s, q, problem}); the 4S
                    // uniforms of a window come from one Philox call per lane (lane sl: ctr
                    // win/4 + sl, moves win + 4 sl + 0..3)
                    const int t0 = B.start + j;
                    if (t0 >= win_end) {
                        win = (t0 / (4 * S)) * (4 * S);
                        win_end = win + 4 * S;
                        unsigned long long c0 = (unsigned long long)(win >> 2) + (unsigned long long)sl;
                        unsigned long long c1 = (unsigned long long)s, c2 = (unsigned long long)q + p.chain_offset,
                                           c3 = p.problem_id;
                        philox4x64_10(c0, c1, c2, c3, p.seed, 0ull);
                        __syncwarp();   // the previous window is read by every lane
                        usm[4 * sl] = uniform_from<T>(c0);
                        usm[4 * sl + 1] = uniform_from<T>(c1);
                        usm[4 * sl + 2] = uniform_from<T>(c2);
                        usm[4 * sl + 3] = uniform_from<T>(c3);
                        if constexpr (PRIOR) {   // acceptance uniforms: ctr {t/4, s, q, problem xor 2^63}
                            c0 = (unsigned long long)(win >> 2) + (unsigned long long)sl;
                            c1 = (unsigned long long)s;
                            c2 = (unsigned long long)q + p.chain_offset;
                            c3 = p.problem_id ^ (1ull << 63);
                            philox4x64_10(c0, c1, c2, c3, p.seed, 0ull);
                            usm[4 * S + 4 * sl] = uniform_from<T>(c0);
                            usm[4 * S + 4 * sl + 1] = uniform_from<T>(c1);
                            usm[4 * S + 4 * sl + 2] = uniform_from<T>(c2);
                            usm[4 * S + 4 * sl + 3] = uniform_from<T>(c3);
                        }
                        __syncwarp();
                    }
                    // the stage of the next record: usually landed long ago (one test, one vote
                    // per stage of sh.rps moves)
                    if (jr == 0) {
                        bool ok = mbar_test_wait(full + rp.slot, rp.phase);
                        if (__any_sync(0xffffffffu, !ok)) {
                            ok = ok || mbar_wait(full + rp.slot, rp.phase, sh.wait_limit);
                            if (__any_sync(0xffffffffu, !ok)) {   // decided warp-wide
                                failed = true;
                                break;
                            }
                        }
                        stb = reinterpret_cast<const T *>(stages + (size_t)rp.slot * sh.stage_bytes);
                    }
                    // this segment's moves: up to the end of the window, of the stage or of the block
                    const int jbeg = j, jend = min(min(B.n, win_end - B.start), j + (sh.rps - jr));
                    const T *st = stb + (size_t)jr * B.recstride;
                    for (; j < jend; ++j, st += B.recstride) {
                        // what does not depend on the bounds first: c_j and the uniform
                        const T cj = j < B.np ? csm[j] : T(0);
                        const int t = B.start + j;
                        const T u = usm[t - win];
                        const T dj = st[2 * B.rs], ij = st[2 * B.rs + 1];
                        T v0[VEC], r0[VEC];   // chunk 0 of the pass: independent of the draw, loaded first
                        lds_v(st + VEC * sl, v0);
                        lds_v(st + B.rs + VEC * sl, r0);

                        T lo, hi;
                        team_bounds(lk, hk, lo, hi, S, team_base);
                        // degenerate interval: no move; zero mode: flat on [lo, hi] (both bounds
                        // finite: set-up rejects zero modes that do not change sign); else the
                        // truncated Gaussian.  The branch is on the record's d_j, which is known
                        // long before the bounds, so the flat path is one FMA and a select.
                        const bool open = hi > lo;
                        T delta;
                        if (dj == T(0)) {
                            delta = open ? m_fma(u, hi - lo, lo) : T(0);
                            n_zero += open ? 1u : 0u;
                        } else {
                            delta = open ? tn_step<T>(cj, dj, ij, lo, hi, u, capped) : T(0);
                            const bool fin = isfinite(delta);
                            n_bad += fin ? 0u : 1u;
                            delta = fin ? delta : T(0);
                        }
                        n_deg += open ? 0u : 1u;
                        if constexpr (PRIOR) if (delta != T(0)) {
                            // gamma prior (Eq. compat): the draw is a proposal, accepted with
                            // probability min(1, prod ((f + delta V)_+ / f)^(a - 1)) over the block
                            T lsum = T(0);
                            unsigned zflags = 0u;   // 1: a proposed value is 0, 2: a current value is 0
#pragma unroll
                            for (int k = 0; k < KV; ++k) {
                                if (k < kcnt) {
                                    T vv[VEC];
                                    if (k == 0) {
#pragma unroll
                                        for (int v = 0; v < VEC; ++v) vv[v] = v0[v];
                                    } else {
                                        lds_v(st + VEC * (k * S + sl), vv);
                                    }
#pragma unroll
                                    for (int v = 0; v < VEC; ++v) {
                                        const int nl = VEC * (k * S + sl) + v;
                                        if (nl < B.n) {
                                            const T am1 = __ldg(p.prior_am1 + B.start + nl);
                                            if (am1 != T(0)) {
                                                const T x0 = f[k][v];
                                                const T x1 = m_max(m_fma(delta, vv[v], x0), T(0));
                                                if (x1 == T(0)) zflags |= 1u;
                                                else if (x0 == T(0)) zflags |= 2u;
                                                else lsum += am1 * (m_log(x1) - m_log(x0));
                                            }
                                        }
                                    }
                                }
                            }
                            for (int off = 1; off < S; off <<= 1) {
                                lsum += __shfl_xor_sync(0xffffffffu, lsum, off);
                                zflags |= __shfl_xor_sync(0xffffffffu, zflags, off);
                            }
                            const T lr = (zflags & 1u) ? -CUDART_INF_F : (zflags & 2u) ? CUDART_INF_F : lsum;
                            const T ua = usm[4 * S + (t - win)];
                            if (!(m_log(ua) < lr)) {
                                delta = T(0);
                                ++n_rej;
                            }
                        }
                        fused_pass_smem<T, KV, KK, CHK>(f, delta, v0, r0, st, st + B.rs, kcnt, sl, S, lk, hk);
                        // the residual moves by K~_b V_j delta = dres_j delta U_j (dres = d for a
                        // Gaussian mode, |K~_b V_j| for one sampled flat)
                        if (j < B.np && sl == 0) wsm[j] = st[2 * B.rs + 2] * delta;
                    }
                    // release the stage to the producer after its last record (one arrival per warp)
                    jr += j - jbeg;
                    if (jr == sh.rps || j == B.n) {
                        __syncwarp();
                        mbar_arrive_lane0(empty + rp.slot, lane);
                        ring_next(rp, D);
                        jr = 0;
                    }
                }
            };
            if (kcnt == 1) {
                block_moves(std::integral_constant<int, 1>{});
            } else if constexpr (KV > 1) {
                if (kcnt == KV)
                    block_moves(std::integral_constant<int, KV>{});
                else
                    block_moves(std::integral_constant<int, 0>{});
            }
            if (failed) break;
            __syncwarp();
            // exit: r~ -= U_b w (lanes split the data points; eight (WIDE: sixteen) loads in
            // flight, eight partial sums as at entry; the same from the U stage)
            const T *Ut = p.pd.Ut + B.offU;
            if (ust) {
                // two of the lane's data points at a time (m, m + S; one in the widest tiles)
                for (int m = sl; m < p.M; m += (KV <= 8 ? 2 : 1) * S) {
                    const bool two = KV <= 8 && m + S < p.M;
                    const int m2 = two ? m + S : m;
                    T a[8], b[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) a[i] = b[i] = T(0);
                    int j = 0;
                    for (; j + 7 < B.np; j += 8) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            const T w = wsm[j + i];
                            const T *u = Us + (size_t)(j + i) * B.usr;
                            a[i] = m_fma(u[m], w, a[i]);
                            b[i] = m_fma(u[m2], w, b[i]);
                        }
                    }
                    for (; j < B.np; ++j) {
                        a[0] = m_fma(Us[(size_t)j * B.usr + m], wsm[j], a[0]);
                        b[0] = m_fma(Us[(size_t)j * B.usr + m2], wsm[j], b[0]);
                    }
                    rsm[m] -= ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
                    if (two) rsm[m + S] -= ((b[0] + b[1]) + (b[2] + b[3])) + ((b[4] + b[5]) + (b[6] + b[7]));
                }
                // release the U stage to the producer (one arrival per warp)
                __syncwarp();
                mbar_arrive_lane0(uempty + (rp.ug & 1u), lane);
                ++rp.ug;
            } else
            for (int m = sl; m < p.M; m += S) {
                T a[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) a[i] = T(0);
                int j = 0;
                if constexpr (WIDE) {
                    for (; j + 15 < B.np; j += 16) {
                        T x[16];
#pragma unroll
                        for (int i = 0; i < 16; ++i) x[i] = __ldg(Ut + (size_t)(j + i) * p.M + m);
#pragma unroll
                        for (int i = 0; i < 16; ++i) a[i & 7] = m_fma(x[i], wsm[j + i], a[i & 7]);
                    }
                }
                for (; j + 7 < B.np; j += 8) {
                    T x[8];
#pragma unroll
                    for (int i = 0; i < 8; ++i) x[i] = __ldg(Ut + (size_t)(j + i) * p.M + m);
#pragma unroll
                    for (int i = 0; i < 8; ++i) a[i] = m_fma(x[i], wsm[j + i], a[i]);
                }
                for (; j < B.np; ++j) a[0] = m_fma(__ldg(Ut + (size_t)j * p.M + m), wsm[j], a[0]);
                rsm[m] -= ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
            }
            // write the block back and accumulate the kept sweep
#pragma unroll
            for (int k = 0; k < KV; ++k)
#pragma unroll
                for (int v = 0; v < VEC; ++v) {
                    const int nl = VEC * (k * S + sl) + v;
                    if (active && k < kcnt && nl < B.n) {
                        const int n = B.start + nl;
                        if (trace) {
                            const T old = Fq[n], dlt = f[k][v] - old;
                            sd2 = m_fma(dlt, dlt, sd2);
                            sf2 = m_fma(old, old, sf2);
                        }
                        Fq[n] = f[k][v];
                        if (keep) {
                            if constexpr (psums) {
                                p1sm[n] += f[k][v];
                                p2sm[n] = m_fma(f[k][v], f[k][v], p2sm[n]);
                            } else {
                                const double x = (double)f[k][v];
                                S1q[n] += x;
                                S2q[n] += x * x;
                            }
                        }
                    }
                    // one chunk's sums at a time: keeps the compiler from holding every
                    // chunk's loaded sums in registers at once (the widest tiles spilled)
                    if (v + 1 == VEC) asm volatile("" ::: "memory");
                }
            __syncwarp();
        }
        if (trace && !failed) {   // Delta_s = |f(s+1) - f(s)| / |f(s)| of this chain, summed over chains
            for (int off = 1; off < S; off <<= 1) {
                sd2 += __shfl_xor_sync(0xffffffffu, sd2, off);
                sf2 += __shfl_xor_sync(0xffffffffu, sf2, off);
            }
            if (active && sl == 0 && s < p.trace_cap && sf2 > T(0))
                atomicAdd(p.steptrace + s, sqrt((double)sd2 / (double)sf2));
        }
    }
    if (failed) {
        if (lane == 0) atomicAdd(&p.counters->timeouts, 1ull);
        return;
    }
    if (active) {
        for (int m = sl; m < p.M; m += S) Rq[m] = rsm[m];
        if (kept_here) {
            if ((rg.sweep0 + rg.nsweeps) % kBinSweeps == 0) {   // the block closes: into the FP64 sums
                for (int n = sl; n < p.N; n += S) {
                    S1q[n] += (double)p1sm[n];
                    S2q[n] += (double)p2sm[n];
                    P1q[n] = P2q[n] = T(0);
                }
            } else if (sh.npad) {   // the block continues in a later launch
                for (int n = sl; n < p.N; n += S) {
                    P1q[n] = p1sm[n];
                    P2q[n] = p2sm[n];
                }
            }
        }
        if (sl == 0) {
            if (n_deg) atomicAdd(&p.counters->degenerate, (unsigned long long)n_deg);
            if (n_zero) atomicAdd(&p.counters->zero_mode, (unsigned long long)n_zero);
            if (n_bad) atomicAdd(&p.counters->nonfinite, (unsigned long long)n_bad);
            if (n_rej) atomicAdd(&p.counters->prior_rejections, (unsigned long long)n_rej);
            if (capped) atomicAdd(&p.counters->tail_capped, (unsigned long long)capped);
        }
    }
}

// --------------------------------------------------------------------------
// the persistent sweep kernel: the sweeps [ctrl->sweep0, + ctrl->nsweeps) of
// every work item (problem, chain group).  Warps 0 .. consumers-1 run chains;
// warp `consumers` produces the move records.  CTAs pull items from
// ctrl->queue.  One problem (BATCH = false): its parameters are the launch's
// grid constant p0.  Several: each item's parameters are copied from probs
// into shared memory.
// --------------------------------------------------------------------------
template <class T, int KV, bool BATCH, int MINB, bool PRIOR>
__global__ void __launch_bounds__(32 * (kMaxConsumers + 1), MINB) sweep_kernel(const __grid_constant__ SweepParams<T> p0,
                                                    const SweepParams<T> *__restrict__ probs,
                                                    const WorkItem *__restrict__ items, RunCtrl *ctrl,
                                                    const __grid_constant__ LaunchShape shape)
{
    __shared__ SweepParams<T> sp;
    __shared__ SweepRange rg;
    __shared__ int s_item;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned long long *full = reinterpret_cast<unsigned long long *>(smem_raw + shape.off_full);
    unsigned long long *empty = reinterpret_cast<unsigned long long *>(smem_raw + shape.off_empty);
    unsigned char *stages = smem_raw + shape.off_stages;
    unsigned long long *ufull = reinterpret_cast<unsigned long long *>(smem_raw + shape.off_ubar);
    unsigned long long *uempty = ufull + 2;
    unsigned char *ubuf = smem_raw + shape.off_ubuf;
    const int wcta = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        for (int i = 0; i < shape.depth; ++i) {
            mbar_init(full + i, 1);
            mbar_init(empty + i, (unsigned)shape.consumers);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(ufull + i, 1);
            mbar_init(uempty + i, (unsigned)shape.consumers);
        }
        fence_mbar_init();
        fence_proxy_async_smem();
        rg.sweep0 = ctrl->sweep0;
        rg.nsweeps = ctrl->nsweeps;
        rg.burn_in = ctrl->burn_in;
    }
    RingPos rp{0u, 0, 0u, 0u};
    bool failed = false;
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(&ctrl->queue, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= shape.n_items) break;
        const WorkItem w = items[it];
        if constexpr (BATCH) {
            if (threadIdx.x == 0) sp = probs[w.problem];
            __syncthreads();
        }
        const SweepParams<T> &p = BATCH ? sp : p0;
        if (wcta == shape.consumers)
            produce(p, shape, rg, full, empty, stages, ufull, uempty, ubuf, rp, failed);
        else
            consume<T, KV, PRIOR, (MINB > 1)>(p, shape, rg, w.group, smem_raw, full, empty, stages, ufull, uempty,
                                             ubuf, rp, failed);
        __syncthreads();   // the item is finished before sp and s_item change
    }
}

template <class T, int KV, bool BATCH, int MINB, bool PRIOR>
cudaError_t launch_sweep_kernel(const SweepParams<T> &p0, const SweepParams<T> *probs, const WorkItem *items,
                                RunCtrl *ctrl, const LaunchShape &shape, int ctas, cudaStream_t stream)
{
    const size_t smem = (size_t)shape.off_stages + (size_t)shape.depth * shape.stage_bytes;
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<T, KV, BATCH, MINB, PRIOR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    sweep_kernel<T, KV, BATCH, MINB, PRIOR><<<(unsigned)ctas, 32 * (shape.consumers + 1), smem, stream>>>(p0, probs, items, ctrl,
                                                                                             shape);
    return cudaGetLastError();
}

template <class T, int KV, bool BATCH, int MINB, bool PRIOR>
int sweep_ctas_per_sm(const LaunchShape &shape)
{
    const size_t smem = (size_t)shape.off_stages + (size_t)shape.depth * shape.stage_bytes;
    if (cudaFuncSetAttribute(sweep_kernel<T, KV, BATCH, MINB, PRIOR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
        cudaSuccess)
        return 0;
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<T, KV, BATCH, MINB, PRIOR>, 32 * (shape.consumers + 1),
                                                      smem) != cudaSuccess)
        return 0;
    return n;
}

// dispatch over the register tile (kv) and the batch flag, for one residency
// MINB (CTAs per SM the registers are budgeted for) and prior flag
template <class T, int MINB, bool PRIOR, int... KVs>
struct SweepDispatch {
    static cudaError_t launch(const SweepParams<T> &p0, const SweepParams<T> *probs, const WorkItem *items,
                              RunCtrl *ctrl, const LaunchShape &shape, int kv, bool batch, int ctas, cudaStream_t s)
    {
        cudaError_t e = cudaErrorInvalidValue;
        ((kv == KVs ? (e = batch ? launch_sweep_kernel<T, KVs, true, MINB, PRIOR>(p0, probs, items, ctrl, shape, ctas, s)
                                 : launch_sweep_kernel<T, KVs, false, MINB, PRIOR>(p0, probs, items, ctrl, shape, ctas, s),
                       0)
                    : 0),
         ...);
        return e;
    }
    static int per_sm(const LaunchShape &shape, int kv, bool batch)
    {
        int n = 0;
        ((kv == KVs ? (n = batch ? sweep_ctas_per_sm<T, KVs, true, MINB, PRIOR>(shape)
                                 : sweep_ctas_per_sm<T, KVs, false, MINB, PRIOR>(shape),
                       0)
                    : 0),
         ...);
        return n;
    }
};

}  // namespace asmgb
