// cta_ops.cuh -- CTA-wide building blocks shared by the persistent kernels:
// a runtime-size in-place FFT in shared memory and CTA reductions.
#pragma once

#include "fa_internal.cuh"
#include "fft_stages.cuh"

namespace fa {

// In-place forward DFT of X[0, B), B = 2^logb in [4, BMAX], by a group of T
// threads whose local index is tid (Stockham stages as in fft_stages.cuh with
// runtime sizes; each thread holds its butterflies in registers between the
// two barriers).  The barriers are CTA-wide: every group of the CTA calls it
// at the same time with the same B.
template <int T, int BMAX>
__device__ void fft_rt_g(double2* X, int logb, const double2* __restrict__ Wf, int tid)
{
    constexpr int MAX4 = (BMAX / 4 + T - 1) / T;  // radix-4 butterflies per thread (at most)
    const int B = 1 << logb, Q = B >> 2, H = B >> 1;
    double2 v[MAX4][4];  // one register block for both stage kinds
    int ns = 1;
    if (logb & 1) {
        // radix-2 butterflies j = tid + i T, i < 2 MAX4, kept in v[i/2][2(i%2) .. +1]
#pragma unroll
        for (int i = 0; i < 2 * MAX4; ++i) {
            const int j = tid + i * T;
            if (j < H) {
                const double2 a = X[j], b = X[j + H];
                v[i >> 1][2 * (i & 1)] = add_v(a, b);
                v[i >> 1][2 * (i & 1) + 1] = sub_v(a, b);
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < 2 * MAX4; ++i) {
            const int j = tid + i * T;
            if (j < H) { X[2 * j] = v[i >> 1][2 * (i & 1)]; X[2 * j + 1] = v[i >> 1][2 * (i & 1) + 1]; }
        }
        __syncthreads();
        ns = 2;
    }
    for (; ns < B; ns <<= 2) {
#pragma unroll
        for (int i = 0; i < MAX4; ++i) {
            const int j = tid + i * T;
            if (j < Q) {
                v[i][0] = X[j]; v[i][1] = X[j + Q]; v[i][2] = X[j + 2 * Q]; v[i][3] = X[j + 3 * Q];
                const int k = j & (ns - 1);
                if (ns > 1) {
                    const int e1 = k * (B / (4 * ns)), e2 = 2 * e1, e3 = e1 + Q;
                    Tw4v<double2> w;
                    w.t1 = __ldg(Wf + e1); w.t2 = __ldg(Wf + e2); w.t3 = __ldg(Wf + e3);
                    w.f1 = tw_form_b(e1, B); w.f2 = tw_form_b(e2, B); w.f3 = tw_form_b(e3, B);
                    bfly4_fma(v[i][0], v[i][1], v[i][2], v[i][3], w);
                } else {
                    bfly4_plain(v[i][0], v[i][1], v[i][2], v[i][3]);
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int i = 0; i < MAX4; ++i) {
            const int j = tid + i * T;
            if (j < Q) {
                const int k = j & (ns - 1);
                const int idx = (j - k) * 4 + k;
                X[idx] = v[i][0]; X[idx + ns] = v[i][1]; X[idx + 2 * ns] = v[i][2];
                X[idx + 3 * ns] = v[i][3];
            }
        }
        __syncthreads();
    }
}

// the whole CTA (T threads) as one group
template <int T, int BMAX>
__device__ __forceinline__ void fft_rt(double2* X, int logb, const double2* __restrict__ Wf)
{
    fft_rt_g<T, BMAX>(X, logb, Wf, threadIdx.x);
}

template <int T>
__device__ __forceinline__ void cta_argmax(long long& key, int& idx, long long* sk, int* si)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const long long k2 = __shfl_xor_sync(0xffffffffu, key, off);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, off);
        if (key_better(k2, i2, key, idx)) { key = k2; idx = i2; }
    }
    if ((threadIdx.x & 31) == 0) { sk[threadIdx.x >> 5] = key; si[threadIdx.x >> 5] = idx; }
    __syncthreads();
    key = sk[0];
    idx = si[0];
#pragma unroll
    for (int w = 1; w < T / 32; ++w)
        if (key_better(sk[w], si[w], key, idx)) { key = sk[w]; idx = si[w]; }
    __syncthreads();
}

// CTA sum of a double2 (partials in shared memory, FP64 adds on warp 0)
template <int T>
__device__ __forceinline__ double2 cta_sum(double2 v, double2* part)
{
    part[threadIdx.x] = v;
    __syncthreads();
    if (threadIdx.x < 32) {
        double2 s = part[threadIdx.x];
        for (int i = threadIdx.x + 32; i < T; i += 32) { s.x += part[i].x; s.y += part[i].y; }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
            s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
        }
        if (threadIdx.x == 0) part[T] = s;
    }
    __syncthreads();
    const double2 r = part[T];
    __syncthreads();
    return r;
}

}  // namespace fa
