// align_common.cuh -- thread-group geometry and group reductions shared by
// the pair-alignment kernels (align_fft.cu, align_df_impl.cuh).  A "group" is
// the Q = N/4 threads that work on one pair; a CTA holds G groups.
#pragma once

#include "fa_internal.cuh"

namespace fa {

template <int LOGN>
struct Geo {
    static constexpr int N = 1 << LOGN;
    static constexpr int Q = N / 4;                   // threads per pair
    static constexpr int G = Q >= 128 ? 1 : 128 / Q;  // pairs per CTA
    static constexpr int T = G * Q;                   // threads per CTA
    static constexpr int W = Q >= 32 ? Q / 32 : 1;    // warps per pair
};

// Group-wide argmax of (key, idx); every thread of the group gets the result.
template <int Q>
__device__ __forceinline__ void group_argmax(long long& key, int& idx, long long* sk, int* si,
                                             int g, int t)
{
    constexpr int WID = Q < 32 ? Q : 32;
#pragma unroll
    for (int off = WID / 2; off > 0; off >>= 1) {
        const long long k2 = __shfl_xor_sync(0xffffffffu, key, off);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, off);
        if (key_better(k2, i2, key, idx)) { key = k2; idx = i2; }
    }
    if constexpr (Q > 32) {
        constexpr int W = Q / 32;
        if ((t & 31) == 0) { sk[g * W + (t >> 5)] = key; si[g * W + (t >> 5)] = idx; }
        __syncthreads();
        key = sk[g * W];
        idx = si[g * W];
#pragma unroll
        for (int i = 1; i < W; ++i)
            if (key_better(sk[g * W + i], si[g * W + i], key, idx)) {
                key = sk[g * W + i];
                idx = si[g * W + i];
            }
        __syncthreads();
    }
}

// Group-wide sum of a double2: partials go to shared memory and the first
// warp of the group adds them (FP64 adds on one warp only).  Result in out
// (shared), valid after the trailing __syncthreads.
template <int Q>
__device__ __forceinline__ void group_sum(double2 v, double2* part, double2* out, int g, int t)
{
    part[t] = v;
    __syncthreads();
    if constexpr (Q <= 32) {
        if (t == 0) {
            double2 s = part[0];
            for (int i = 1; i < Q; ++i) { s.x += part[i].x; s.y += part[i].y; }
            out[g] = s;
        }
    } else {
        if (t < 32) {
            double2 s = part[t];
            for (int i = t + 32; i < Q; i += 32) { s.x += part[i].x; s.y += part[i].y; }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
                s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
            }
            if (t == 0) out[g] = s;
        }
    }
    __syncthreads();
}


}  // namespace fa
