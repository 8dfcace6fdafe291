// align_fft.cu -- FA_FFT / FA_PREC_FP64: Algorithm 2 of the paper with the
// convolution theorem, one thread group per curve pair, all in FP64.
//
// Per pair (N = 2^LOGN nodes, Q = N/4 threads):
//   1. Z1 = DFT(z1), Z2 = DFT(z2): Stockham radix-4 stages in shared memory
//      (one radix-2 stage first when LOGN is odd), both curves per stage.
//   2. P = Z1 * conj(Z2) formed in registers by the first stage of a third
//      forward transform, so that DFT(P)[s] = N c(s) with
//      c(s) = sum_k z1[k] conj(z2[k+s])  (Sec. 2, convolution theorem; the
//      complex form of the four real correlations A_kj(t_m) of Eq. A-mtx).
//   3. The last stage keeps its outputs in registers and reduces
//      argmax_s |c(s)|^2 (smallest s on exact ties) -- the loop over t0 of
//      Algorithm 2, where the per-shift Kabsch SVD collapses to |c(s)|.
//   4. c(s*) by its O(N) sum, theta = arg c(s*), energy of Eq. disc-energy by
//      its definition (Algorithm 1 in closed form at the winning shift).
//
// The path is bound by the FP64 pipe (about 2 DFMA per clock per SM on this
// part), so the design minimises FP64 instructions: twiddles come from a
// table in FMA form (every twiddled radix-4 butterfly is 24 DFMA), index
// arithmetic and the argmax compare are integer, and block reductions run
// their FP64 adds on one warp only.
#include "fa_internal.cuh"

namespace fa {
namespace {

__device__ __forceinline__ void bfly4(double2& v0, double2& v1, double2& v2, double2& v3)
{
    const double2 a0 = make_double2(v0.x + v2.x, v0.y + v2.y);
    const double2 a1 = make_double2(v0.x - v2.x, v0.y - v2.y);
    const double2 a2 = make_double2(v1.x + v3.x, v1.y + v3.y);
    const double2 a3 = make_double2(v1.x - v3.x, v1.y - v3.y);
    v0 = make_double2(a0.x + a2.x, a0.y + a2.y);
    v2 = make_double2(a0.x - a2.x, a0.y - a2.y);
    v1 = make_double2(a1.x + a3.y, a1.y - a3.x);  // a1 - i a3
    v3 = make_double2(a1.x - a3.y, a1.y + a3.x);  // a1 + i a3
}

// Radix-4 butterfly with twiddles W^e1, W^2e1, W^3e1 on v1, v2, v3, in FMA form:
// (A, B) = v0 +- w^2 v2, (C, D) = v1 +- w^2 v3, y0/y2 = A +- w C, y1/y3 = B -+ i w D,
// i.e. four FMA butterflies (24 DFMA) instead of three complex products plus
// sixteen additions (28 instructions).  -i w = W^(e1 + N/4).
struct Tw4 {
    double2 t1, t2, t3;
    bool f1, f2, f3;
};

template <int N>
__device__ __forceinline__ Tw4 load_tw4(const double2* __restrict__ T, int e1)
{
    Tw4 w;
    const int e2 = 2 * e1, e3 = e1 + N / 4;
    w.t1 = __ldg(T + e1); w.t2 = __ldg(T + e2); w.t3 = __ldg(T + e3);
    w.f1 = tw_form_b(e1, N); w.f2 = tw_form_b(e2, N); w.f3 = tw_form_b(e3, N);
    return w;
}

__device__ __forceinline__ void bfly4_tw(double2& v0, double2& v1, double2& v2, double2& v3,
                                         const Tw4& w)
{
    fbfly(v0, v2, w.t2, w.f2);  // v0 = A, v2 = B
    fbfly(v1, v3, w.t2, w.f2);  // v1 = C, v3 = D
    fbfly(v0, v1, w.t1, w.f1);  // v0 = y0, v1 = y2
    fbfly(v2, v3, w.t3, w.f3);  // v2 = y1, v3 = y3
    const double2 t = v1;
    v1 = v2;
    v2 = t;
}

template <int LOGN>
struct Geo {
    static constexpr int N = 1 << LOGN;
    static constexpr int Q = N / 4;                   // threads per pair
    static constexpr int G = Q >= 128 ? 1 : 128 / Q;  // pairs per CTA
    static constexpr int T = G * Q;                   // threads per CTA
    static constexpr int W = Q >= 32 ? Q / 32 : 1;    // warps per pair
};

// Radix-2 stage (Ns = 1) on both buffers: butterflies j = t and j = t + Q.
template <int LOGN>
__device__ __forceinline__ void stage2_two(double2* X1, double2* X2, int t)
{
    constexpr int N = 1 << LOGN, Q = N / 4, H = N / 2;
    const double2 a = X1[t], b = X1[t + H], c = X1[t + Q], d = X1[t + Q + H];
    const double2 e = X2[t], f = X2[t + H], g = X2[t + Q], k = X2[t + Q + H];
    __syncthreads();
    X1[2 * t] = make_double2(a.x + b.x, a.y + b.y);
    X1[2 * t + 1] = make_double2(a.x - b.x, a.y - b.y);
    X1[2 * (t + Q)] = make_double2(c.x + d.x, c.y + d.y);
    X1[2 * (t + Q) + 1] = make_double2(c.x - d.x, c.y - d.y);
    X2[2 * t] = make_double2(e.x + f.x, e.y + f.y);
    X2[2 * t + 1] = make_double2(e.x - f.x, e.y - f.y);
    X2[2 * (t + Q)] = make_double2(g.x + k.x, g.y + k.y);
    X2[2 * (t + Q) + 1] = make_double2(g.x - k.x, g.y - k.y);
    __syncthreads();
}

// Radix-4 Stockham stage with sub-transform size NS on both buffers.
template <int LOGN, int NS>
__device__ __forceinline__ void stage4_two(double2* X1, double2* X2, int t,
                                           const double2* __restrict__ W)
{
    constexpr int N = 1 << LOGN, Q = N / 4;
    double2 a0 = X1[t], a1 = X1[t + Q], a2 = X1[t + 2 * Q], a3 = X1[t + 3 * Q];
    double2 b0 = X2[t], b1 = X2[t + Q], b2 = X2[t + 2 * Q], b3 = X2[t + 3 * Q];
    const int k = t & (NS - 1);
    if constexpr (NS > 1) {
        const Tw4 w = load_tw4<N>(W, k * (N / (4 * NS)));
        bfly4_tw(a0, a1, a2, a3, w);
        bfly4_tw(b0, b1, b2, b3, w);
    } else {
        bfly4(a0, a1, a2, a3);
        bfly4(b0, b1, b2, b3);
    }
    __syncthreads();
    const int idx = (t - k) * 4 + k;
    X1[idx] = a0; X1[idx + NS] = a1; X1[idx + 2 * NS] = a2; X1[idx + 3 * NS] = a3;
    X2[idx] = b0; X2[idx + NS] = b1; X2[idx + 2 * NS] = b2; X2[idx + 3 * NS] = b3;
    __syncthreads();
}

template <int LOGN, int NS>
__device__ __forceinline__ void fft_two_from(double2* X1, double2* X2, int t,
                                             const double2* __restrict__ W)
{
    if constexpr (NS < (1 << LOGN)) {
        stage4_two<LOGN, NS>(X1, X2, t, W);
        fft_two_from<LOGN, NS * 4>(X1, X2, t, W);
    }
}

template <int LOGN>
__device__ __forceinline__ void fft_two(double2* X1, double2* X2, int t,
                                        const double2* __restrict__ W)
{
    if constexpr (LOGN & 1) {
        stage2_two<LOGN>(X1, X2, t);
        fft_two_from<LOGN, 2>(X1, X2, t, W);
    } else {
        fft_two_from<LOGN, 1>(X1, X2, t, W);
    }
}

// Radix-4 stage on X1 alone.  PROD: the inputs are X1 * conj(X2) (the
// spectrum product).  LAST: outputs stay in registers (y[q] = c at s = t+qQ).
template <int LOGN, int NS, bool PROD, bool LAST>
__device__ __forceinline__ void stage4_one(double2* X1, const double2* X2, int t,
                                           const double2* __restrict__ W, double2 (&y)[4])
{
    constexpr int N = 1 << LOGN, Q = N / 4;
    double2 v0 = X1[t], v1 = X1[t + Q], v2 = X1[t + 2 * Q], v3 = X1[t + 3 * Q];
    if constexpr (PROD) {
        v0 = cmulc(v0, X2[t]); v1 = cmulc(v1, X2[t + Q]);
        v2 = cmulc(v2, X2[t + 2 * Q]); v3 = cmulc(v3, X2[t + 3 * Q]);
    }
    const int k = t & (NS - 1);
    if constexpr (NS > 1)
        bfly4_tw(v0, v1, v2, v3, load_tw4<N>(W, k * (N / (4 * NS))));
    else
        bfly4(v0, v1, v2, v3);
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
template <int LOGN>
__device__ __forceinline__ void stage2_prod(double2* X1, const double2* X2, int t)
{
    constexpr int N = 1 << LOGN, Q = N / 4, H = N / 2;
    const double2 a = cmulc(X1[t], X2[t]), b = cmulc(X1[t + H], X2[t + H]);
    const double2 c = cmulc(X1[t + Q], X2[t + Q]), d = cmulc(X1[t + Q + H], X2[t + Q + H]);
    __syncthreads();
    X1[2 * t] = make_double2(a.x + b.x, a.y + b.y);
    X1[2 * t + 1] = make_double2(a.x - b.x, a.y - b.y);
    X1[2 * (t + Q)] = make_double2(c.x + d.x, c.y + d.y);
    X1[2 * (t + Q) + 1] = make_double2(c.x - d.x, c.y - d.y);
    __syncthreads();
}

template <int LOGN, int NS>
__device__ __forceinline__ void fft_one_from(double2* X, int t, const double2* __restrict__ W,
                                             double2 (&y)[4])
{
    constexpr int N = 1 << LOGN;
    if constexpr (NS * 4 == N) {
        stage4_one<LOGN, NS, false, true>(X, nullptr, t, W, y);
    } else {
        stage4_one<LOGN, NS, false, false>(X, nullptr, t, W, y);
        fft_one_from<LOGN, NS * 4>(X, t, W, y);
    }
}

// y[q] = N c(t + qQ) with c(s) = sum_k z1[k] conj(z2[k+s]), from the spectra in X1, X2.
template <int LOGN>
__device__ __forceinline__ void fft_corr(double2* X1, const double2* X2, int t,
                                         const double2* __restrict__ W, double2 (&y)[4])
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

template <int LOGN, typename ZT>
__global__ void __launch_bounds__(Geo<LOGN>::T)
    align_fft_kernel(const ZT* __restrict__ z1, const ZT* __restrict__ z2, int64_t P,
                     const double2* __restrict__ W, int32_t* __restrict__ shift,
                     double* __restrict__ theta, double* __restrict__ energy,
                     int8_t* __restrict__ status)
{
    using Gm = Geo<LOGN>;
    constexpr int N = Gm::N, Q = Gm::Q, G = Gm::G;
    extern __shared__ __align__(16) double2 smem[];
    double2* X1 = smem + (size_t)(threadIdx.x / Q) * 2 * N;
    double2* X2 = X1 + N;
    double2* bcast = smem + (size_t)G * 2 * N;          // [G] : (cos, sin) of theta
    double2* sums = bcast + G;                           // [G]
    long long* sk = reinterpret_cast<long long*>(sums + G);  // [G*W]
    int* si = reinterpret_cast<int*>(sk + G * Gm::W);        // [G*W]
    int* bad = si + G * Gm::W;                               // [G]

    const int g = threadIdx.x / Q;
    const int t = threadIdx.x % Q;
    const int64_t pair = (int64_t)blockIdx.x * G + g;
    const bool valid = pair < P;
    const ZT* p1 = z1 + (valid ? pair : 0) * N;
    const ZT* p2 = z2 + (valid ? pair : 0) * N;

    if (t == 0) bad[g] = 0;
    __syncthreads();
    bool nf = false;
    double2 a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        a[r] = valid ? ld_z(p1, t + r * Q) : make_double2(0.0, 0.0);
        b[r] = valid ? ld_z(p2, t + r * Q) : make_double2(0.0, 0.0);
        nf |= !finite2(a[r]) || !finite2(b[r]);
        X1[t + r * Q] = a[r];
        X2[t + r * Q] = b[r];
    }
    if (nf) bad[g] = 1;
    __syncthreads();

    fft_two<LOGN>(X1, X2, t, W);
    double2 y[4];
    fft_corr<LOGN>(X1, X2, t, W, y);

    long long key = -1;
    int idx = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double m = fma(y[q].x, y[q].x, y[q].y * y[q].y);
        const long long kq = __double_as_longlong(m);
        const int s = t + q * Q;
        if (key_better(kq, s, key, idx)) { key = kq; idx = s; }
    }
    group_argmax<Q>(key, idx, sk, si, g, t);
    const int sbest = idx;

    // c(s*) by its O(N) definition (inputs re-read from L1/L2)
    double2 c = make_double2(0.0, 0.0);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        b[r] = valid ? ld_z(p2, (t + r * Q + sbest) & (N - 1)) : make_double2(0.0, 0.0);
        c.x = fma(a[r].x, b[r].x, fma(a[r].y, b[r].y, c.x));
        c.y = fma(a[r].y, b[r].x, fma(-a[r].x, b[r].y, c.y));
    }
    __syncthreads();  // the last stage's shared-memory reads are done: X1 is free
    group_sum<Q>(c, X1, sums, g, t);
    if (t == 0) {
        const double2 cs = sums[g];
        const double r = sqrt(fma(cs.x, cs.x, cs.y * cs.y));
        bcast[g] = r > 0.0 ? make_double2(cs.x / r, cs.y / r) : make_double2(1.0, 0.0);
    }
    __syncthreads();
    const double2 rot = bcast[g];
    double e = 0.0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const double rx = fma(rot.x, b[r].x, -rot.y * b[r].y);
        const double ry = fma(rot.y, b[r].x, rot.x * b[r].y);
        const double dx = a[r].x - rx, dy = a[r].y - ry;
        e = fma(dx, dx, e);
        e = fma(dy, dy, e);
    }
    const double2 csum = sums[g];
    __syncthreads();  // everyone has read sums[g] before it is overwritten
    group_sum<Q>(make_double2(e, 0.0), X1, sums, g, t);
    if (t == 0 && valid) {
        if (bad[g]) {
            shift[pair] = -1;
            theta[pair] = __longlong_as_double(0x7ff8000000000000LL);
            energy[pair] = __longlong_as_double(0x7ff8000000000000LL);
            status[pair] = FA_STATUS_NONFINITE;
        } else {
            shift[pair] = sbest;
            theta[pair] = atan2(csum.y, csum.x);
            energy[pair] = sums[g].x * (1.0 / N);
            status[pair] = FA_STATUS_OK;
        }
    }
}

template <int LOGN, typename ZT>
int launch_one(const fa_handle* h, const void* z1, const void* z2, int64_t P, int32_t* shift,
               double* theta, double* energy, int8_t* status, cudaStream_t st)
{
    using Gm = Geo<LOGN>;
    const size_t smem = (size_t)Gm::G * 2 * Gm::N * sizeof(double2) + 2 * Gm::G * sizeof(double2) +
                        (size_t)Gm::G * Gm::W * (sizeof(long long) + sizeof(int)) +
                        Gm::G * sizeof(int);
    auto kern = align_fft_kernel<LOGN, ZT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "align_fft: cudaFuncSetAttribute");
    }
    const int64_t blocks = (P + Gm::G - 1) / Gm::G;
    kern<<<(unsigned)blocks, Gm::T, smem, st>>>(static_cast<const ZT*>(z1),
                                                static_cast<const ZT*>(z2), P, h->tf64[LOGN],
                                                shift, theta, energy, status);
    return cuda_error(cudaGetLastError(), "align_fft launch");
}

template <typename ZT>
int dispatch(const fa_handle* h, const void* z1, const void* z2, int64_t P, int logn,
             int32_t* shift, double* theta, double* energy, int8_t* status, cudaStream_t st)
{
    switch (logn) {
#define FA_CASE(L) \
    case L: return launch_one<L, ZT>(h, z1, z2, P, shift, theta, energy, status, st);
        FA_CASE(2) FA_CASE(3) FA_CASE(4) FA_CASE(5) FA_CASE(6) FA_CASE(7) FA_CASE(8) FA_CASE(9)
        FA_CASE(10) FA_CASE(11) FA_CASE(12)
#undef FA_CASE
    }
    return set_error(FA_ERR_UNSUPPORTED, "align_fft: unsupported N");
}

}  // namespace

int launch_align_fft(const fa_handle* h, const void* z1, const void* z2, int64_t P, int logn,
                     int ztype, int32_t* shift, double* theta, double* energy, int8_t* status,
                     cudaStream_t st)
{
    if (P == 0) return FA_OK;
    if (ztype == FA_Z_F64)
        return dispatch<double2>(h, z1, z2, P, logn, shift, theta, energy, status, st);
    return dispatch<float2>(h, z1, z2, P, logn, shift, theta, energy, status, st);
}

}  // namespace fa
