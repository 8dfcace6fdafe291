// fft_stages.cuh -- Stockham radix-4 FFT stages in shared memory, generic over
// the element type (double2 for the FP64 search, float2 for the FP32 search of
// FA_PREC_MIXED).  One thread group of Q = N/4 threads per transform pair;
// every CTA-wide barrier is taken by all groups of the CTA together.
//
// Stage with sub-transform size NS (Stockham autosort, radix 4): thread t
// reads x[t + rQ], r = 0..3, applies the twiddles W_N^{r k N/(4 NS)} with
// k = t mod NS, and writes the radix-4 outputs to ((t - k)*4 + k) + q NS.  When
// log2 N is odd one radix-2 stage (NS = 1) comes first.  Twiddled butterflies
// use the FMA form (four FMA butterflies of 6 FMA each, see fbfly_v).
#pragma once

#include "fa_internal.cuh"

namespace fa {

template <typename V> struct Scalar;
template <> struct Scalar<double2> { using T = double; };
template <> struct Scalar<float2> { using T = float; };

template <typename V>
__device__ __forceinline__ V mk2(typename Scalar<V>::T x, typename Scalar<V>::T y)
{
    V v;
    v.x = x;
    v.y = y;
    return v;
}

// sign flip of m when fb, by integer XOR on the sign bit (no FP instruction)
__device__ __forceinline__ double flip_if(double m, bool fb)
{
    return __longlong_as_double(__double_as_longlong(m) ^ ((unsigned long long)fb << 63));
}
__device__ __forceinline__ float flip_if(float m, bool fb)
{
    return __int_as_float(__float_as_int(m) ^ ((unsigned)fb << 31));
}

// (a, b) <- (a + w b, a - w b), w = (m, rho) in FMA form (see fa_handle::tf64)
template <typename V>
__device__ __forceinline__ void fbfly_v(V& a, V& b, V t, bool fb)
{
    using T = typename Scalar<V>::T;
    const T m = t.x, rho = t.y;
    const T U = fb ? b.x : b.y;
    const T V_ = fb ? b.y : b.x;
    const T tx = fma(-rho, U, V_);
    const T ty = fma(rho, V_, U);
    const T mx = flip_if(m, fb);
    b = mk2<V>(fma(-mx, tx, a.x), fma(-m, ty, a.y));
    a = mk2<V>(fma(mx, tx, a.x), fma(m, ty, a.y));
}

template <typename V>
__device__ __forceinline__ V add_v(V a, V b) { return mk2<V>(a.x + b.x, a.y + b.y); }
template <typename V>
__device__ __forceinline__ V sub_v(V a, V b) { return mk2<V>(a.x - b.x, a.y - b.y); }
// a * conj(b)
template <typename V>
__device__ __forceinline__ V mulc_v(V a, V b)
{
    return mk2<V>(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}

template <typename V>
__device__ __forceinline__ void bfly4_plain(V& v0, V& v1, V& v2, V& v3)
{
    const V a0 = add_v(v0, v2), a1 = sub_v(v0, v2), a2 = add_v(v1, v3), a3 = sub_v(v1, v3);
    v0 = add_v(a0, a2);
    v2 = sub_v(a0, a2);
    v1 = mk2<V>(a1.x + a3.y, a1.y - a3.x);  // a1 - i a3
    v3 = mk2<V>(a1.x - a3.y, a1.y + a3.x);  // a1 + i a3
}

// Twiddles W^e1, W^2e1 and -i W^e1 = W^(e1 + N/4) with their storage forms.
template <typename V>
struct Tw4v {
    V t1, t2, t3;
    bool f1, f2, f3;
};

template <int N, typename V>
__device__ __forceinline__ Tw4v<V> load_tw4v(const V* __restrict__ T, int e1)
{
    Tw4v<V> w;
    const int e2 = 2 * e1, e3 = e1 + N / 4;
    w.t1 = __ldg(T + e1); w.t2 = __ldg(T + e2); w.t3 = __ldg(T + e3);
    w.f1 = tw_form_b(e1, N); w.f2 = tw_form_b(e2, N); w.f3 = tw_form_b(e3, N);
    return w;
}

// Twiddled radix-4 butterfly in FMA form: (A, B) = v0 +- w^2 v2,
// (C, D) = v1 +- w^2 v3, y0/y2 = A +- w C, y1/y3 = B -+ i w D.
template <typename V>
__device__ __forceinline__ void bfly4_fma(V& v0, V& v1, V& v2, V& v3, const Tw4v<V>& w)
{
    fbfly_v(v0, v2, w.t2, w.f2);
    fbfly_v(v1, v3, w.t2, w.f2);
    fbfly_v(v0, v1, w.t1, w.f1);
    fbfly_v(v2, v3, w.t3, w.f3);
    const V t = v1;
    v1 = v2;
    v2 = t;
}

// Radix-2 stage (NS = 1) on two buffers: butterflies j = t and j = t + Q.
template <int LOGN, typename V>
__device__ __forceinline__ void stage2_two(V* X1, V* X2, int t)
{
    constexpr int N = 1 << LOGN, Q = N / 4, H = N / 2;
    const V a = X1[t], b = X1[t + H], c = X1[t + Q], d = X1[t + Q + H];
    const V e = X2[t], f = X2[t + H], g = X2[t + Q], k = X2[t + Q + H];
    __syncthreads();
    X1[2 * t] = add_v(a, b); X1[2 * t + 1] = sub_v(a, b);
    X1[2 * (t + Q)] = add_v(c, d); X1[2 * (t + Q) + 1] = sub_v(c, d);
    X2[2 * t] = add_v(e, f); X2[2 * t + 1] = sub_v(e, f);
    X2[2 * (t + Q)] = add_v(g, k); X2[2 * (t + Q) + 1] = sub_v(g, k);
    __syncthreads();
}

template <int LOGN, int NS, typename V>
__device__ __forceinline__ void stage4_two(V* X1, V* X2, int t, const V* __restrict__ W)
{
    constexpr int N = 1 << LOGN, Q = N / 4;
    V a0 = X1[t], a1 = X1[t + Q], a2 = X1[t + 2 * Q], a3 = X1[t + 3 * Q];
    V b0 = X2[t], b1 = X2[t + Q], b2 = X2[t + 2 * Q], b3 = X2[t + 3 * Q];
    const int k = t & (NS - 1);
    if constexpr (NS > 1) {
        const Tw4v<V> w = load_tw4v<N>(W, k * (N / (4 * NS)));
        bfly4_fma(a0, a1, a2, a3, w);
        bfly4_fma(b0, b1, b2, b3, w);
    } else {
        bfly4_plain(a0, a1, a2, a3);
        bfly4_plain(b0, b1, b2, b3);
    }
    __syncthreads();
    const int idx = (t - k) * 4 + k;
    X1[idx] = a0; X1[idx + NS] = a1; X1[idx + 2 * NS] = a2; X1[idx + 3 * NS] = a3;
    X2[idx] = b0; X2[idx + NS] = b1; X2[idx + 2 * NS] = b2; X2[idx + 3 * NS] = b3;
    __syncthreads();
}

template <int LOGN, int NS, typename V>
__device__ __forceinline__ void fft_two_from(V* X1, V* X2, int t, const V* __restrict__ W)
{
    if constexpr (NS < (1 << LOGN)) {
        stage4_two<LOGN, NS>(X1, X2, t, W);
        fft_two_from<LOGN, NS * 4>(X1, X2, t, W);
    }
}

// In-place forward DFT of X1 and X2 (N = 2^LOGN each).
template <int LOGN, typename V>
__device__ __forceinline__ void fft_two(V* X1, V* X2, int t, const V* __restrict__ W)
{
    if constexpr (LOGN & 1) {
        stage2_two<LOGN>(X1, X2, t);
        fft_two_from<LOGN, 2>(X1, X2, t, W);
    } else {
        fft_two_from<LOGN, 1>(X1, X2, t, W);
    }
}

// Radix-4 stage on X1 alone.  PROD: inputs are X1 * conj(X2).  LAST: the
// outputs stay in registers, y[q] at s = t + qQ.
template <int LOGN, int NS, bool PROD, bool LAST, typename V>
__device__ __forceinline__ void stage4_one(V* X1, const V* X2, int t, const V* __restrict__ W,
                                           V (&y)[4])
{
    constexpr int N = 1 << LOGN, Q = N / 4;
    V v0 = X1[t], v1 = X1[t + Q], v2 = X1[t + 2 * Q], v3 = X1[t + 3 * Q];
    if constexpr (PROD) {
        v0 = mulc_v(v0, X2[t]); v1 = mulc_v(v1, X2[t + Q]);
        v2 = mulc_v(v2, X2[t + 2 * Q]); v3 = mulc_v(v3, X2[t + 3 * Q]);
    }
    const int k = t & (NS - 1);
    if constexpr (NS > 1)
        bfly4_fma(v0, v1, v2, v3, load_tw4v<N>(W, k * (N / (4 * NS))));
    else
        bfly4_plain(v0, v1, v2, v3);
    if constexpr (LAST) {
        y[0] = v0; y[1] = v1; y[2] = v2; y[3] = v3;
    } else {
        __syncthreads();
        const int idx = (t - k) * 4 + k;
        X1[idx] = v0; X1[idx + NS] = v1; X1[idx + 2 * NS] = v2; X1[idx + 3 * NS] = v3;
        __syncthreads();
    }
}

// Radix-2 first stage of the correlation transform, inputs X1 * conj(X2).
template <int LOGN, typename V>
__device__ __forceinline__ void stage2_prod(V* X1, const V* X2, int t)
{
    constexpr int N = 1 << LOGN, Q = N / 4, H = N / 2;
    const V a = mulc_v(X1[t], X2[t]), b = mulc_v(X1[t + H], X2[t + H]);
    const V c = mulc_v(X1[t + Q], X2[t + Q]), d = mulc_v(X1[t + Q + H], X2[t + Q + H]);
    __syncthreads();
    X1[2 * t] = add_v(a, b); X1[2 * t + 1] = sub_v(a, b);
    X1[2 * (t + Q)] = add_v(c, d); X1[2 * (t + Q) + 1] = sub_v(c, d);
    __syncthreads();
}

template <int LOGN, int NS, typename V>
__device__ __forceinline__ void fft_one_from(V* X, int t, const V* __restrict__ W, V (&y)[4])
{
    constexpr int N = 1 << LOGN;
    if constexpr (NS * 4 == N) {
        stage4_one<LOGN, NS, false, true>(X, (const V*)nullptr, t, W, y);
    } else {
        stage4_one<LOGN, NS, false, false>(X, (const V*)nullptr, t, W, y);
        fft_one_from<LOGN, NS * 4>(X, t, W, y);
    }
}

// y[q] = N c(t + qQ) with c(s) = sum_k z1[k] conj(z2[k+s]) from the spectra in
// X1 = DFT(z1), X2 = DFT(z2): the forward DFT of X1 * conj(X2) (the
// convolution theorem); X1 is overwritten.
template <int LOGN, typename V>
__device__ __forceinline__ void fft_corr(V* X1, const V* X2, int t, const V* __restrict__ W,
                                         V (&y)[4])
{
    if constexpr (LOGN & 1) {
        stage2_prod<LOGN>(X1, X2, t);
        fft_one_from<LOGN, 2>(X1, t, W, y);
    } else if constexpr (LOGN == 2) {
        stage4_one<LOGN, 1, true, true>(X1, X2, t, W, y);
    } else {
        stage4_one<LOGN, 1, true, false>(X1, X2, t, W, y);
        fft_one_from<LOGN, 4>(X1, t, W, y);
    }
}

}  // namespace fa
