// align_df_impl.cuh -- FA_PREC_MIXED: the shift search of Algorithm 2 in
// double-float arithmetic on the FP32 pipe, c(s*), theta and the energy in
// FP64 (fa_align_pairs and fa_align_all_pairs).
//
// The three transforms (DFT z1, DFT z2, DFT(Z1 conj Z2) = N c(s)) run in
// double-float (df.cuh, ~48-bit significands).  Each output then carries an
// error of at most a few units of 2^-47 times log2 N times the 1-norm of the
// transform's input, i.e. about 1e-13 of max_s |c(s)| for N <= 4096: the
// argmax of |c|^2 can only differ from the exact one between shifts whose
// energies agree to ~1e-14, far inside the 1e-9 tie tolerance.  At the
// winning shift c(s*) is summed in FP64 (4N DFMA), theta = arg c(s*), and the
// energy of Eq. disc-energy is evaluated directly in FP64 (8N instructions) --
// the only FP64 work per pair, against ~104k for the all-FP64 search at
// N = 1024.
//
// The kernels are instantiated per transform size in separate translation
// units (align_df_*.cu), which keeps the parallel build short.
#pragma once

#include "align_common.cuh"
#include "df.cuh"

namespace fa {
namespace {

// FP64 tail shared by the pair and all-pairs kernels: c(s*) by its sum, the
// rotation, the energy.  a[r] = z1[t + rQ]; z2 is read at (t + rQ + s*) mod N.
template <int LOGN, typename ZT>
__device__ __forceinline__ void fp64_tail(const double2 (&a)[4], const ZT* p2, bool valid, int sbest,
                                          double2* part, double2* sums, double2* bcast, int g, int t,
                                          double2& csum, double& esum)
{
    using Gm = Geo<LOGN>;
    constexpr int N = Gm::N, Q = Gm::Q;
    double2 b[4];
    double2 c = make_double2(0.0, 0.0);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        b[r] = valid ? ld_z(p2, (t + r * Q + sbest) & (N - 1)) : make_double2(0.0, 0.0);
        c.x = fma(a[r].x, b[r].x, fma(a[r].y, b[r].y, c.x));
        c.y = fma(a[r].y, b[r].x, fma(-a[r].x, b[r].y, c.y));
    }
    __syncthreads();  // the transform's shared-memory reads are done
    group_sum<Q>(c, part, sums, g, t);
    if (t == 0) {
        const double2 cs = sums[g];
        const double rr = sqrt(fma(cs.x, cs.x, cs.y * cs.y));
        bcast[g] = rr > 0.0 ? make_double2(cs.x / rr, cs.y / rr) : make_double2(1.0, 0.0);
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
    csum = sums[g];
    __syncthreads();
    group_sum<Q>(make_double2(e, 0.0), part, sums, g, t);
    esum = sums[g].x;
}

template <int LOGN>
struct DfSmem {
    using Gm = Geo<LOGN>;
    static constexpr size_t bytes = (size_t)Gm::G * 2 * Gm::N * sizeof(float4) +
                                    2 * Gm::G * sizeof(double2) +
                                    (size_t)Gm::G * Gm::W * (sizeof(long long) + sizeof(int)) +
                                    Gm::G * sizeof(int);
};

template <int LOGN, typename ZT>
__global__ void __launch_bounds__(Geo<LOGN>::T)
    align_df_kernel(const ZT* __restrict__ z1, const ZT* __restrict__ z2, int64_t P,
                    const float4* __restrict__ W, int32_t* __restrict__ shift,
                    double* __restrict__ theta, double* __restrict__ energy,
                    int8_t* __restrict__ status)
{
    using Gm = Geo<LOGN>;
    constexpr int N = Gm::N, Q = Gm::Q, G = Gm::G;
    extern __shared__ __align__(16) float4 smem4[];
    const int g = threadIdx.x / Q;
    const int t = threadIdx.x % Q;
    float4* X1 = smem4 + (size_t)g * 2 * N;
    float4* X2 = X1 + N;
    double2* part = reinterpret_cast<double2*>(X1);  // reused after the transforms
    double2* sums = reinterpret_cast<double2*>(smem4 + (size_t)G * 2 * N);  // [G]
    double2* bcast = sums + G;                                                // [G]
    long long* sk = reinterpret_cast<long long*>(bcast + G);                  // [G*W]
    int* si = reinterpret_cast<int*>(sk + G * Gm::W);                         // [G*W]
    int* bad = si + G * Gm::W;                                                // [G]

    const int64_t pair = (int64_t)blockIdx.x * G + g;
    const bool valid = pair < P;
    const ZT* p1 = z1 + (valid ? pair : 0) * N;
    const ZT* p2 = z2 + (valid ? pair : 0) * N;
    if (t == 0) bad[g] = 0;
    __syncthreads();
    bool nf = false;
    double2 a[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        a[r] = valid ? ld_z(p1, t + r * Q) : make_double2(0.0, 0.0);
        const double2 b = valid ? ld_z(p2, t + r * Q) : make_double2(0.0, 0.0);
        nf |= !finite2(a[r]) || !finite2(b);
        X1[t + r * Q] = st4(split_c(a[r]));
        X2[t + r * Q] = st4(split_c(b));
    }
    if (nf) bad[g] = 1;
    __syncthreads();
    fft_two_df<LOGN>(X1, X2, t, W);
    cdf y[4];
    fft_corr_df<LOGN>(X1, X2, t, W, y);
    long long key = -1;
    int idx = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const long long kq = df_key(cnorm2(y[q]));
        if (key_better(kq, t + q * Q, key, idx)) { key = kq; idx = t + q * Q; }
    }
    group_argmax<Q>(key, idx, sk, si, g, t);
    double2 csum;
    double esum;
    fp64_tail<LOGN>(a, p2, valid, idx, part, sums, bcast, g, t, csum, esum);
    if (t == 0 && valid) {
        if (bad[g]) {
            shift[pair] = -1;
            theta[pair] = __longlong_as_double(0x7ff8000000000000LL);
            energy[pair] = __longlong_as_double(0x7ff8000000000000LL);
            status[pair] = FA_STATUS_NONFINITE;
        } else {
            shift[pair] = idx;
            theta[pair] = atan2(csum.y, csum.x);
            energy[pair] = esum * (1.0 / N);
            status[pair] = FA_STATUS_OK;
        }
    }
}

// ----------------------------------------------------------- all pairs ----
template <int LOGN, typename ZT>
__global__ void __launch_bounds__(Geo<LOGN>::T)
    spectra_df_kernel(const ZT* __restrict__ z, int64_t M, const float4* __restrict__ W,
                      float4* __restrict__ spec, int8_t* __restrict__ status,
                      int32_t* __restrict__ shift, double* __restrict__ theta,
                      double* __restrict__ energy)
{
    using Gm = Geo<LOGN>;
    constexpr int N = Gm::N, Q = Gm::Q, G = Gm::G;
    extern __shared__ __align__(16) float4 smem4[];
    const int g = threadIdx.x / Q;
    const int t = threadIdx.x % Q;
    float4* X1 = smem4 + (size_t)g * 2 * N;
    float4* X2 = X1 + N;
    int* bad = reinterpret_cast<int*>(smem4 + (size_t)G * 2 * N);  // [2G]
    const int64_t m1 = 2 * ((int64_t)blockIdx.x * G + g), m2 = m1 + 1;
    const bool v1 = m1 < M, v2 = m2 < M;
    if (t == 0) { bad[2 * g] = 0; bad[2 * g + 1] = 0; }
    __syncthreads();
    bool nf1 = false, nf2 = false;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const double2 a = v1 ? ld_z(z + m1 * N, t + r * Q) : make_double2(0.0, 0.0);
        const double2 b = v2 ? ld_z(z + m2 * N, t + r * Q) : make_double2(0.0, 0.0);
        nf1 |= !finite2(a);
        nf2 |= !finite2(b);
        X1[t + r * Q] = st4(split_c(a));
        X2[t + r * Q] = st4(split_c(b));
    }
    if (nf1) bad[2 * g] = 1;
    if (nf2) bad[2 * g + 1] = 1;
    __syncthreads();
    fft_two_df<LOGN>(X1, X2, t, W);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if (v1) spec[m1 * N + t + r * Q] = X1[t + r * Q];
        if (v2) spec[m2 * N + t + r * Q] = X2[t + r * Q];
    }
    if (t == 0) {
        if (v1) {
            status[m1] = bad[2 * g] ? FA_STATUS_NONFINITE : FA_STATUS_OK;
            const int64_t d = m1 * M + m1;
            shift[d] = 0; theta[d] = 0.0; energy[d] = 0.0;
        }
        if (v2) {
            status[m2] = bad[2 * g + 1] ? FA_STATUS_NONFINITE : FA_STATUS_OK;
            const int64_t d = m2 * M + m2;
            shift[d] = 0; theta[d] = 0.0; energy[d] = 0.0;
        }
    }
}

__device__ __forceinline__ int64_t tri_start(int64_t i, int64_t M) { return i * (2 * M - i - 1) / 2; }

template <int LOGN, typename ZT>
__global__ void __launch_bounds__(Geo<LOGN>::T)
    allpairs_df_kernel(const ZT* __restrict__ z, int64_t M, const float4* __restrict__ spec,
                       const float4* __restrict__ W, const int8_t* __restrict__ cstatus,
                       int32_t* __restrict__ shift, double* __restrict__ theta,
                       double* __restrict__ energy)
{
    using Gm = Geo<LOGN>;
    constexpr int N = Gm::N, Q = Gm::Q, G = Gm::G;
    extern __shared__ __align__(16) float4 smem4[];
    const int g = threadIdx.x / Q;
    const int t = threadIdx.x % Q;
    float4* X1 = smem4 + (size_t)g * 2 * N;
    float4* X2 = X1 + N;
    double2* part = reinterpret_cast<double2*>(X1);
    double2* sums = reinterpret_cast<double2*>(smem4 + (size_t)G * 2 * N);
    double2* bcast = sums + G;
    long long* sk = reinterpret_cast<long long*>(bcast + G);
    int* si = reinterpret_cast<int*>(sk + G * Gm::W);

    const int64_t npairs = M * (M - 1) / 2;
    const int64_t q = (int64_t)blockIdx.x * G + g;
    const bool valid = q < npairs;
    int64_t i = 0, j = 1;
    if (valid) {
        const float af = (float)(2 * M - 1);
        int64_t e = (int64_t)floorf(0.5f * (af - sqrtf(fmaxf(af * af - 8.0f * (float)q, 0.f))));
        e = max((int64_t)0, min(e, M - 2));
        while (e > 0 && tri_start(e, M) > q) --e;
        while (e < M - 2 && tri_start(e + 1, M) <= q) ++e;
        i = e;
        j = q - tri_start(i, M) + i + 1;
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        X1[t + r * Q] = valid ? spec[i * N + t + r * Q] : make_float4(0.f, 0.f, 0.f, 0.f);
        X2[t + r * Q] = valid ? spec[j * N + t + r * Q] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncthreads();
    cdf y[4];
    fft_corr_df<LOGN>(X1, X2, t, W, y);
    long long key = -1;
    int idx = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const long long kq = df_key(cnorm2(y[r]));
        if (key_better(kq, t + r * Q, key, idx)) { key = kq; idx = t + r * Q; }
    }
    group_argmax<Q>(key, idx, sk, si, g, t);
    double2 a[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) a[r] = valid ? ld_z(z + i * N, t + r * Q) : make_double2(0.0, 0.0);
    double2 csum;
    double esum;
    fp64_tail<LOGN>(a, z + j * N, valid, idx, part, sums, bcast, g, t, csum, esum);
    if (t == 0 && valid) {
        const int64_t ij = i * M + j, ji = j * M + i;
        if (cstatus[i] != FA_STATUS_OK || cstatus[j] != FA_STATUS_OK) {
            const double qn = __longlong_as_double(0x7ff8000000000000LL);
            shift[ij] = shift[ji] = -1;
            theta[ij] = theta[ji] = qn;
            energy[ij] = energy[ji] = qn;
        } else {
            const double th = atan2(csum.y, csum.x);
            const double en = esum * (1.0 / N);
            shift[ij] = idx;
            theta[ij] = th;
            energy[ij] = en;
            shift[ji] = idx ? N - idx : 0;
            theta[ji] = (th == 3.141592653589793) ? th : -th;
            energy[ji] = en;
        }
    }
}

template <typename K>
int set_smem(K kern, size_t smem, const char* what)
{
    if (smem <= 48 * 1024) return FA_OK;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    return e == cudaSuccess ? FA_OK : cuda_error(e, what);
}

template <int LOGN, typename ZT>
int launch_pairs(const fa_handle* h, const void* z1, const void* z2, int64_t P, int32_t* shift,
                 double* theta, double* energy, int8_t* status, cudaStream_t st)
{
    using Gm = Geo<LOGN>;
    const size_t smem = DfSmem<LOGN>::bytes;
    auto kern = align_df_kernel<LOGN, ZT>;
    int rc = set_smem(kern, smem, "align_df: cudaFuncSetAttribute");
    if (rc != FA_OK) return rc;
    kern<<<(unsigned)((P + Gm::G - 1) / Gm::G), Gm::T, smem, st>>>(
        static_cast<const ZT*>(z1), static_cast<const ZT*>(z2), P, h->tdf[LOGN], shift, theta,
        energy, status);
    return cuda_error(cudaGetLastError(), "align_df launch");
}

template <int LOGN, typename ZT>
int launch_all(const fa_handle* h, const void* z, int64_t M, float4* spec, int8_t* status,
               int32_t* shift, double* theta, double* energy, cudaStream_t st)
{
    using Gm = Geo<LOGN>;
    const ZT* zz = static_cast<const ZT*>(z);
    const float4* W = h->tdf[LOGN];
    {
        const size_t smem = (size_t)Gm::G * 2 * Gm::N * sizeof(float4) + 2 * Gm::G * sizeof(int);
        auto kern = spectra_df_kernel<LOGN, ZT>;
        int rc = set_smem(kern, smem, "spectra_df: cudaFuncSetAttribute");
        if (rc != FA_OK) return rc;
        const int64_t groups = (M + 1) / 2;
        kern<<<(unsigned)((groups + Gm::G - 1) / Gm::G), Gm::T, smem, st>>>(zz, M, W, spec, status,
                                                                            shift, theta, energy);
        rc = cuda_error(cudaGetLastError(), "spectra_df launch");
        if (rc != FA_OK) return rc;
    }
    const int64_t npairs = M * (M - 1) / 2;
    if (npairs == 0) return FA_OK;
    const size_t smem = DfSmem<LOGN>::bytes;
    auto kern = allpairs_df_kernel<LOGN, ZT>;
    int rc = set_smem(kern, smem, "allpairs_df: cudaFuncSetAttribute");
    if (rc != FA_OK) return rc;
    kern<<<(unsigned)((npairs + Gm::G - 1) / Gm::G), Gm::T, smem, st>>>(zz, M, spec, W, status,
                                                                         shift, theta, energy);
    return cuda_error(cudaGetLastError(), "allpairs_df launch");
}

}  // namespace

#define FA_DF_PAIRS_CASE(L)                                                                   \
    case L:                                                                                   \
        return f64 ? launch_pairs<L, double2>(h, z1, z2, P, shift, theta, energy, status, st) \
                   : launch_pairs<L, float2>(h, z1, z2, P, shift, theta, energy, status, st);
#define FA_DF_ALL_CASE(L)                                                                     \
    case L:                                                                                   \
        return f64 ? launch_all<L, double2>(h, z, M, spec, status, shift, theta, energy, st)  \
                   : launch_all<L, float2>(h, z, M, spec, status, shift, theta, energy, st);

}  // namespace fa
