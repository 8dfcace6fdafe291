// df.cuh -- double-float ("float-float") arithmetic and Stockham FFT stages
// on it, for the FA_PREC_MIXED shift search.
//
// A value is an unevaluated sum h + l of two floats with |l| <= ulp(h)/2
// (about 48 significant bits).  The operations are the classical error-free
// transformations: Knuth's two-sum, Dekker's fast-two-sum for ordered
// operands, and the exact product split a*b = p + fma(a, b, -p).  Every FP32
// operation is written with an explicit round-to-nearest intrinsic so that the
// compiler can neither contract nor reassociate them.  Additions are the
// "sloppy" double-float sum (one two-sum on the high parts): its error is
// bounded by a few 2^-48 times |x| + |y|, which is the form of error bound an
// FFT analysis needs (errors relative to the magnitudes being combined).
//
// All of this runs on the FP32 pipe, which on this part is 62x the FP64
// rate; a radix-4 butterfly costs ~290 FP32 instructions against 24 FP64.
#pragma once

#include "fa_internal.cuh"

namespace fa {

struct dfl {
    float h, l;
};

__device__ __forceinline__ dfl two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ dfl fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl df_add(dfl x, dfl y)
{
    const dfl s = two_sum(x.h, y.h);
    return fast_two_sum(s.h, __fadd_rn(s.l, __fadd_rn(x.l, y.l)));
}

__device__ __forceinline__ dfl df_sub(dfl x, dfl y) { return df_add(x, dfl{-y.h, -y.l}); }

// a b + s c d (s = +1 or -1), with the high products split exactly
template <int S>
__device__ __forceinline__ dfl df_dot2(dfl a, dfl b, dfl c, dfl d)
{
    const float p1 = __fmul_rn(a.h, b.h);
    const float e1 = __fmaf_rn(a.h, b.h, -p1);
    const float p2 = __fmul_rn(c.h, d.h);
    const float e2 = __fmaf_rn(c.h, d.h, -p2);
    const dfl s = two_sum(p1, S > 0 ? p2 : -p2);
    float err = __fadd_rn(S > 0 ? __fadd_rn(e1, e2) : __fsub_rn(e1, e2), s.l);
    err = __fmaf_rn(a.h, b.l, err);
    err = __fmaf_rn(a.l, b.h, err);
    err = __fmaf_rn(S > 0 ? c.h : -c.h, d.l, err);
    err = __fmaf_rn(S > 0 ? c.l : -c.l, d.h, err);
    return fast_two_sum(s.h, err);
}

// a b (the leading product split exactly by FMA; about 2^-47 relative)
__device__ __forceinline__ dfl df_mul(dfl a, dfl b)
{
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return fast_two_sum(p, e);
}

// 1/x for x != 0: the FP32 reciprocal of the leading part and one Newton step
// r0 + r0 (1 - x r0), its residual formed by FMA (1 - x.h r0 is exact to
// 2^-48, x r0 being within 2^-23 of 1); about 2^-46 relative
__device__ __forceinline__ dfl df_rcp(dfl x)
{
    const float r0 = __frcp_rn(x.h);
    const float e = __fmaf_rn(-x.l, r0, __fmaf_rn(-x.h, r0, 1.0f));
    return fast_two_sum(r0, __fmul_rn(r0, e));
}

// float -> double from the bits (zero and subnormal floats give 0): no FP64
// conversion instruction
__device__ __forceinline__ double df_widen(float f)
{
    const unsigned u = __float_as_uint(f);
    const unsigned ef = (u >> 23) & 0xff;
    if (ef == 0) return 0.0;
    const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
    return __longlong_as_double((long long)(sign | ((unsigned long long)(ef - 127 + 1023) << 52) |
                                            ((unsigned long long)(u & 0x7fffff) << 29)));
}
// h + l in FP64 (one FP64 add)
__device__ __forceinline__ double df_to_double(dfl x) { return df_widen(x.h) + df_widen(x.l); }

__device__ __forceinline__ dfl df_neg(dfl x) { return {-x.h, -x.l}; }
__device__ __forceinline__ dfl df_twice(dfl x) { return {__fmul_rn(2.0f, x.h), __fmul_rn(2.0f, x.l)}; }

// complex double-float, stored in shared memory as float4 (re.h, re.l, im.h, im.l)
struct cdf {
    dfl re, im;
};

__device__ __forceinline__ cdf ld4(const float4& v) { return {{v.x, v.y}, {v.z, v.w}}; }
__device__ __forceinline__ float4 st4(const cdf& c) { return make_float4(c.re.h, c.re.l, c.im.h, c.im.l); }
__device__ __forceinline__ cdf cadd(cdf a, cdf b) { return {df_add(a.re, b.re), df_add(a.im, b.im)}; }
__device__ __forceinline__ cdf csub(cdf a, cdf b) { return {df_sub(a.re, b.re), df_sub(a.im, b.im)}; }
// a w
__device__ __forceinline__ cdf cmul_df(cdf a, cdf w)
{
    return {df_dot2<-1>(a.re, w.re, a.im, w.im), df_dot2<+1>(a.re, w.im, a.im, w.re)};
}
// a conj(b)
__device__ __forceinline__ cdf cmulc_df(cdf a, cdf b)
{
    return {df_dot2<+1>(a.re, b.re, a.im, b.im), df_dot2<-1>(a.im, b.re, a.re, b.im)};
}

// double -> double-float without FP64 instructions: the high part keeps the
// top 24 significand bits (truncated), the low part the remaining 29 bits
// rounded to 24, both rebuilt from the integer bits.  Exact to 2^-47
// relative for |v| in [2^-74, 2^128); the low part is dropped below 2^-74 and
// magnitudes below 2^-126 flush to zero.  (Inputs here are unit-length curves.)
__device__ __forceinline__ dfl split_d(double v)
{
    const long long b = __double_as_longlong(v);
    const int e = (int)((b >> 52) & 0x7ff);
    const int fe = e - 1023 + 127;  // float exponent field of v
    if (fe <= 0 || fe >= 255) return {0.f, 0.f};
    const unsigned sign = (unsigned)((unsigned long long)b >> 32) & 0x80000000u;
    const float hi = __uint_as_float(sign | ((unsigned)fe << 23) | (unsigned)((b >> 29) & 0x7fffff));
    if (fe < 53) return {hi, 0.f};
    const int m = (int)(b & 0x1fffffff);  // remaining significand bits, < 2^29
    // lo = m * 2^(e - 1075); the float exponent field of 2^(e - 1075) is fe - 52
    const float scale = __uint_as_float((unsigned)(fe - 52) << 23);
    const float lo = __fmul_rn(__int2float_rn(m), scale);
    return {hi, sign ? -lo : lo};
}
__device__ __forceinline__ cdf split_c(double2 v) { return {split_d(v.x), split_d(v.y)}; }
__device__ __forceinline__ cdf split_c(float2 v) { return {{v.x, 0.f}, {v.y, 0.f}}; }

// order-preserving 64-bit key of a non-negative double-float
__device__ __forceinline__ long long df_key(dfl x)
{
    const unsigned lb = __float_as_uint(x.l);
    const unsigned lo = (lb & 0x80000000u) ? ~lb : (lb | 0x80000000u);
    return (long long)(((unsigned long long)__float_as_uint(x.h) << 31) | (lo >> 1));
}

// |c|^2 in double-float
__device__ __forceinline__ dfl cnorm2(cdf c) { return df_dot2<+1>(c.re, c.re, c.im, c.im); }

__device__ __forceinline__ void bfly4_df(cdf& v0, cdf& v1, cdf& v2, cdf& v3)
{
    const cdf a0 = cadd(v0, v2), a1 = csub(v0, v2), a2 = cadd(v1, v3), a3 = csub(v1, v3);
    v0 = cadd(a0, a2);
    v2 = csub(a0, a2);
    v1 = {df_add(a1.re, a3.im), df_sub(a1.im, a3.re)};  // a1 - i a3
    v3 = {df_sub(a1.re, a3.im), df_add(a1.im, a3.re)};  // a1 + i a3
}

// ----- Stockham stages (same structure as fft_stages.cuh), W = W_N[k] table --
template <int LOGN>
__device__ __forceinline__ void stage2_two_df(float4* X1, float4* X2, int t)
{
    constexpr int N = 1 << LOGN, Q = N / 4, H = N / 2;
    const cdf a = ld4(X1[t]), b = ld4(X1[t + H]), c = ld4(X1[t + Q]), d = ld4(X1[t + Q + H]);
    const cdf e = ld4(X2[t]), f = ld4(X2[t + H]), g = ld4(X2[t + Q]), k = ld4(X2[t + Q + H]);
    __syncthreads();
    X1[2 * t] = st4(cadd(a, b)); X1[2 * t + 1] = st4(csub(a, b));
    X1[2 * (t + Q)] = st4(cadd(c, d)); X1[2 * (t + Q) + 1] = st4(csub(c, d));
    X2[2 * t] = st4(cadd(e, f)); X2[2 * t + 1] = st4(csub(e, f));
    X2[2 * (t + Q)] = st4(cadd(g, k)); X2[2 * (t + Q) + 1] = st4(csub(g, k));
    __syncthreads();
}

template <int LOGN, int NS>
__device__ __forceinline__ void stage4_two_df(float4* X1, float4* X2, int t,
                                              const float4* __restrict__ W)
{
    constexpr int N = 1 << LOGN, Q = N / 4;
    cdf a0 = ld4(X1[t]), a1 = ld4(X1[t + Q]), a2 = ld4(X1[t + 2 * Q]), a3 = ld4(X1[t + 3 * Q]);
    cdf b0 = ld4(X2[t]), b1 = ld4(X2[t + Q]), b2 = ld4(X2[t + 2 * Q]), b3 = ld4(X2[t + 3 * Q]);
    const int k = t & (NS - 1);
    if constexpr (NS > 1) {
        constexpr int STR = N / (4 * NS);
        const cdf w1 = ld4(__ldg(W + k * STR)), w2 = ld4(__ldg(W + 2 * k * STR)),
                  w3 = ld4(__ldg(W + 3 * k * STR));
        a1 = cmul_df(a1, w1); a2 = cmul_df(a2, w2); a3 = cmul_df(a3, w3);
        b1 = cmul_df(b1, w1); b2 = cmul_df(b2, w2); b3 = cmul_df(b3, w3);
    }
    bfly4_df(a0, a1, a2, a3);
    bfly4_df(b0, b1, b2, b3);
    __syncthreads();
    const int idx = (t - k) * 4 + k;
    X1[idx] = st4(a0); X1[idx + NS] = st4(a1); X1[idx + 2 * NS] = st4(a2); X1[idx + 3 * NS] = st4(a3);
    X2[idx] = st4(b0); X2[idx + NS] = st4(b1); X2[idx + 2 * NS] = st4(b2); X2[idx + 3 * NS] = st4(b3);
    __syncthreads();
}

template <int LOGN, int NS>
__device__ __forceinline__ void fft_two_df_from(float4* X1, float4* X2, int t,
                                                const float4* __restrict__ W)
{
    if constexpr (NS < (1 << LOGN)) {
        stage4_two_df<LOGN, NS>(X1, X2, t, W);
        fft_two_df_from<LOGN, NS * 4>(X1, X2, t, W);
    }
}

template <int LOGN>
__device__ __forceinline__ void fft_two_df(float4* X1, float4* X2, int t, const float4* __restrict__ W)
{
    if constexpr (LOGN & 1) {
        stage2_two_df<LOGN>(X1, X2, t);
        fft_two_df_from<LOGN, 2>(X1, X2, t, W);
    } else {
        fft_two_df_from<LOGN, 1>(X1, X2, t, W);
    }
}

template <int LOGN, int NS, bool PROD, bool LAST>
__device__ __forceinline__ void stage4_one_df(float4* X1, const float4* X2, int t,
                                              const float4* __restrict__ W, cdf (&y)[4])
{
    constexpr int N = 1 << LOGN, Q = N / 4;
    cdf v0 = ld4(X1[t]), v1 = ld4(X1[t + Q]), v2 = ld4(X1[t + 2 * Q]), v3 = ld4(X1[t + 3 * Q]);
    if constexpr (PROD) {
        v0 = cmulc_df(v0, ld4(X2[t])); v1 = cmulc_df(v1, ld4(X2[t + Q]));
        v2 = cmulc_df(v2, ld4(X2[t + 2 * Q])); v3 = cmulc_df(v3, ld4(X2[t + 3 * Q]));
    }
    const int k = t & (NS - 1);
    if constexpr (NS > 1) {
        constexpr int STR = N / (4 * NS);
        v1 = cmul_df(v1, ld4(__ldg(W + k * STR)));
        v2 = cmul_df(v2, ld4(__ldg(W + 2 * k * STR)));
        v3 = cmul_df(v3, ld4(__ldg(W + 3 * k * STR)));
    }
    bfly4_df(v0, v1, v2, v3);
    if constexpr (LAST) {
        y[0] = v0; y[1] = v1; y[2] = v2; y[3] = v3;
    } else {
        __syncthreads();
        const int idx = (t - k) * 4 + k;
        X1[idx] = st4(v0); X1[idx + NS] = st4(v1); X1[idx + 2 * NS] = st4(v2); X1[idx + 3 * NS] = st4(v3);
        __syncthreads();
    }
}

template <int LOGN>
__device__ __forceinline__ void stage2_prod_df(float4* X1, const float4* X2, int t)
{
    constexpr int N = 1 << LOGN, Q = N / 4, H = N / 2;
    const cdf a = cmulc_df(ld4(X1[t]), ld4(X2[t])), b = cmulc_df(ld4(X1[t + H]), ld4(X2[t + H]));
    const cdf c = cmulc_df(ld4(X1[t + Q]), ld4(X2[t + Q]));
    const cdf d = cmulc_df(ld4(X1[t + Q + H]), ld4(X2[t + Q + H]));
    __syncthreads();
    X1[2 * t] = st4(cadd(a, b)); X1[2 * t + 1] = st4(csub(a, b));
    X1[2 * (t + Q)] = st4(cadd(c, d)); X1[2 * (t + Q) + 1] = st4(csub(c, d));
    __syncthreads();
}

template <int LOGN, int NS>
__device__ __forceinline__ void fft_one_df_from(float4* X, int t, const float4* __restrict__ W,
                                                cdf (&y)[4])
{
    constexpr int N = 1 << LOGN;
    if constexpr (NS * 4 == N) {
        stage4_one_df<LOGN, NS, false, true>(X, nullptr, t, W, y);
    } else {
        stage4_one_df<LOGN, NS, false, false>(X, nullptr, t, W, y);
        fft_one_df_from<LOGN, NS * 4>(X, t, W, y);
    }
}

// y[q] = N c(t + qQ) in double-float from the spectra X1, X2 (X1 overwritten)
template <int LOGN>
__device__ __forceinline__ void fft_corr_df(float4* X1, const float4* X2, int t,
                                            const float4* __restrict__ W, cdf (&y)[4])
{
    if constexpr (LOGN & 1) {
        stage2_prod_df<LOGN>(X1, X2, t);
        fft_one_df_from<LOGN, 2>(X1, t, W, y);
    } else if constexpr (LOGN == 2) {
        stage4_one_df<LOGN, 1, true, true>(X1, X2, t, W, y);
    } else {
        stage4_one_df<LOGN, 1, true, false>(X1, X2, t, W, y);
        fft_one_df_from<LOGN, 4>(X1, t, W, y);
    }
}

}  // namespace fa
