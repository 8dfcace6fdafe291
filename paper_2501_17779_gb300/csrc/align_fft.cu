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
//      its definition (Algorithm 1 in closed form at the winning shift).  The
//      sum for c(s*) runs in float-float (about 2^-46 of the summed
//      magnitudes: theta far inside its 1e-10 bound, and the energy, summed
//      in FP64 at that angle, moves only at second order in the angle's error)
//      for pairs whose largest coordinate lies in [2^-40, 2^40], in FP64
//      otherwise; the energy stays FP64, whose 53 bits the difference of two
//      nearly aligned curves needs.
//
// The path is bound by the FP64 pipe (about 2 DFMA per clock per SM on this
// part), so the design minimises FP64 instructions: twiddles come from a
// table in FMA form (every twiddled radix-4 butterfly is 24 DFMA), index
// arithmetic and the argmax compare are integer, and block reductions run
// their FP64 adds on one warp only.
#include "fa_internal.cuh"
#include "align_common.cuh"
#include "df.cuh"
#include "fft_stages.cuh"

namespace fa {
namespace {

// Resident CTAs per SM requested from the compiler for CTAs of <= 256
// threads: 3 (a register cap of ~85 per thread; at N = 1024 measured 1.6 %
// faster than 2 despite a small spill).  Larger CTAs keep the compiler's choice.
#ifndef FA_ALIGN_MIN_BLOCKS
#define FA_ALIGN_MIN_BLOCKS 3
#endif
template <int T>
constexpr int align_min_blocks() { return T <= 256 ? FA_ALIGN_MIN_BLOCKS : 1; }

// biased exponent field of a double (integer instructions)
__device__ __forceinline__ int bexp(double x) { return (int)((__double_as_longlong(x) >> 52) & 0x7ff); }

template <int LOGN, typename ZT>
__global__ void __launch_bounds__(Geo<LOGN>::T, align_min_blocks<Geo<LOGN>::T>())
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
    int* emx = bad + G;  // [G] largest biased exponent of the pair's coordinates

    const int g = threadIdx.x / Q;
    const int t = threadIdx.x % Q;
    const int64_t pair = (int64_t)blockIdx.x * G + g;
    const bool valid = pair < P;
    const ZT* p1 = z1 + (valid ? pair : 0) * N;
    const ZT* p2 = z2 + (valid ? pair : 0) * N;

    if (t == 0) { bad[g] = 0; emx[g] = 0; }
    __syncthreads();
    bool nf = false;
    int ex = 0;
    double2 a[4], b[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        a[r] = valid ? ld_z(p1, t + r * Q) : make_double2(0.0, 0.0);
        b[r] = valid ? ld_z(p2, t + r * Q) : make_double2(0.0, 0.0);
        nf |= !finite2(a[r]) || !finite2(b[r]);
        ex = max(ex, max(max(bexp(a[r].x), bexp(a[r].y)), max(bexp(b[r].x), bexp(b[r].y))));
        X1[t + r * Q] = a[r];
        X2[t + r * Q] = b[r];
    }
    if (nf) bad[g] = 1;
    atomicMax(&emx[g], ex);
    __syncthreads();
    const bool dfc = emx[g] > 1023 - 40 && emx[g] < 1023 + 40;  // the same for the whole group

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
    for (int r = 0; r < 4; ++r) b[r] = valid ? ld_z(p2, (t + r * Q + sbest) & (N - 1)) : make_double2(0.0, 0.0);
    if (dfc) {
        cdf cd{{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const cdf u = split_c(a[r]), v = split_c(b[r]);
            cd.re = df_add(cd.re, df_dot2<+1>(u.re, v.re, u.im, v.im));
            cd.im = df_add(cd.im, df_dot2<-1>(u.im, v.re, u.re, v.im));
        }
        c = make_double2(df_to_double(cd.re), df_to_double(cd.im));
    } else {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            c.x = fma(a[r].x, b[r].x, fma(a[r].y, b[r].y, c.x));
            c.y = fma(a[r].y, b[r].x, fma(-a[r].x, b[r].y, c.y));
        }
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
                        2 * Gm::G * sizeof(int);
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
