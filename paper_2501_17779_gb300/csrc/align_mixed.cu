// align_mixed.cu -- FA_FFT with FA_PREC_MIXED: the shift search of
// Algorithm 2 in FP32, every shift that FP32 cannot rule out re-scored in
// FP64, theta and the energy in FP64.  Results satisfy the same bounds as the
// all-FP64 path; the FP64 instruction count per pair drops from ~104k to
// ~(4N per candidate + 8N).
//
// Per pair (N = 2^LOGN, Q = N/4 threads):
//   1. z1, z2 (FP64, or complex64 widened) are rounded to float and both
//      transformed, then c~(s) = DFT(Z1 conj Z2) in FP32 (same Stockham stages
//      as the FP64 path, float twiddles in FMA form).
//   2. Rigorous FP32 error bound.  With u = 2^-24, every |c~(s)| is within
//          delta = u (K N ||z1|| ||z2|| + 4 M),   K = 2 (24 log2 N + 53),
//      of the exact |N c(s)| (M = max_s |c~(s)|): input rounding (2u), the two
//      forward transforms (2-norm error <= 8u (log2 N + 2) each, Higham's
//      bound for Cooley-Tukey), the spectrum product (3u), and the third
//      transform, whose error at every output is bounded by its per-level
//      rounding times the 1-norm of its input, ||P||_1 <= ||Z1|| ||Z2|| =
//      N ||z1|| ||z2|| (Parseval); the magnitude adds 4uM; the factor 2 is a
//      safety margin.  The exact maximiser s* then satisfies
//      |c~(s*)| >= |c(s*)| - delta >= |c(s_M)| - delta >= M - 2 delta, so every
//      shift with |c~(s)| >= M - 2 delta is a candidate and s* is among them.
//   3. Each candidate's c(s) = sum_k z1[k] conj(z2[k+s]) is summed in FP64
//      (4 DFMA per node); the largest |c|^2 wins (smallest s on exact ties).
//   4. theta = arg c(s*), energy by its definition (Eq. disc-energy), FP64.
//   Pairs with more than KMAX candidates are flagged and finished by the FP64
//   kernel in a second launch that skips every other pair.
#include <type_traits>

#include "align_common.cuh"
#include "fft_stages.cuh"

namespace fa {
namespace {

constexpr int CB = 4;                     // candidates re-scored per pass
// More candidates than this cost more in FP64 (4N each) than the all-FP64
// transforms of the pair; such pairs (near-circles, near-symmetric shapes,
// whose |c(s)| is nearly flat in s) are handed to the FP64 kernel instead.
constexpr int KMAX = 16;
constexpr float kU = 5.9604644775390625e-8f;  // 2^-24

template <int LOGN>
struct MixSmem {
    // per CTA, after the G group buffers (X1, X2 float2 [N] each, cand int [N])
    static constexpr int N = 1 << LOGN, G = Geo<LOGN>::G, W = Geo<LOGN>::W;
    static constexpr size_t group_bytes = (size_t)N * (2 * sizeof(float2) + sizeof(int));
    static constexpr size_t bytes = (size_t)G * group_bytes
                                    + G * CB * sizeof(double2)      // candidate totals
                                    + 3 * G * sizeof(double2)       // best c, rotation, sums
                                    + G * W * 4 * sizeof(float)     // float reductions
                                    + 2 * G * sizeof(int);          // candidate count, bad flag
};

template <int LOGN, typename ZT>
__global__ void __launch_bounds__(Geo<LOGN>::T)
    align_mixed_kernel(const ZT* __restrict__ z1, const ZT* __restrict__ z2, int64_t P,
                       const float2* __restrict__ Tf, int32_t* __restrict__ shift,
                       double* __restrict__ theta, double* __restrict__ energy,
                       int8_t* __restrict__ status)
{
    using Gm = Geo<LOGN>;
    using Sm = MixSmem<LOGN>;
    constexpr int N = Gm::N, Q = Gm::Q, G = Gm::G, W = Gm::W;
    extern __shared__ __align__(16) unsigned char smem[];
    const int g = threadIdx.x / Q;
    const int t = threadIdx.x % Q;
    unsigned char* gb = smem + (size_t)g * Sm::group_bytes;
    float2* X1 = reinterpret_cast<float2*>(gb);
    float2* X2 = X1 + N;
    int* cand = reinterpret_cast<int*>(X2 + N);
    double2* part = reinterpret_cast<double2*>(gb);  // reuses X1/X2: [CB][Q] or [Q]
    double2* tot = reinterpret_cast<double2*>(smem + (size_t)G * Sm::group_bytes);  // [G][CB]
    double2* bestc = tot + G * CB;   // [G]
    double2* rot = bestc + G;        // [G]
    double2* sums = rot + G;         // [G]
    float* fr = reinterpret_cast<float*>(sums + G);  // [G][W][4]
    int* cnt = reinterpret_cast<int*>(fr + G * W * 4);  // [G]
    int* bad = cnt + G;                                  // [G]

    const int64_t pair = (int64_t)blockIdx.x * G + g;
    const bool valid = pair < P;
    const ZT* p1 = z1 + (valid ? pair : 0) * N;
    const ZT* p2 = z2 + (valid ? pair : 0) * N;

    if (t == 0) { bad[g] = 0; cnt[g] = 0; }
    __syncthreads();
    bool nf = false;
    double2 a[4];
    float n1 = 0.f, n2 = 0.f;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        a[r] = valid ? ld_z(p1, t + r * Q) : make_double2(0.0, 0.0);
        const double2 b = valid ? ld_z(p2, t + r * Q) : make_double2(0.0, 0.0);
        nf |= !finite2(a[r]) || !finite2(b);
        const float2 af = make_float2((float)a[r].x, (float)a[r].y);
        const float2 bf = make_float2((float)b.x, (float)b.y);
        X1[t + r * Q] = af;
        X2[t + r * Q] = bf;
        n1 = fmaf(af.x, af.x, fmaf(af.y, af.y, n1));
        n2 = fmaf(bf.x, bf.x, fmaf(bf.y, bf.y, n2));
    }
    if (nf) bad[g] = 1;
    __syncthreads();

    fft_two<LOGN>(X1, X2, t, Tf);
    float2 y[4];
    fft_corr<LOGN>(X1, X2, t, Tf, y);
    float m[4];
    float mx = 0.f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        m[q] = sqrtf(fmaf(y[q].x, y[q].x, y[q].y * y[q].y));
        mx = fmaxf(mx, m[q]);
    }
    // group reduction: max |c~|, sum |z1|^2, sum |z2|^2 (FP32)
    {
        constexpr int WID = Q < 32 ? Q : 32;
#pragma unroll
        for (int off = WID / 2; off > 0; off >>= 1) {
            mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, off));
            n1 += __shfl_xor_sync(0xffffffffu, n1, off);
            n2 += __shfl_xor_sync(0xffffffffu, n2, off);
        }
        if constexpr (Q > 32) {
            if ((t & 31) == 0) {
                float* f = fr + (g * W + (t >> 5)) * 4;
                f[0] = mx; f[1] = n1; f[2] = n2;
            }
            __syncthreads();
            mx = 0.f; n1 = 0.f; n2 = 0.f;
            for (int w = 0; w < W; ++w) {
                const float* f = fr + (g * W + w) * 4;
                mx = fmaxf(mx, f[0]); n1 += f[1]; n2 += f[2];
            }
        }
    }
    const float delta = kU * (2.0f * (24.0f * LOGN + 53.0f) * (float)N * sqrtf(n1 * n2) + 4.0f * mx);
    const float tau = mx - 2.0f * delta;
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (valid && m[q] >= tau) cand[atomicAdd(&cnt[g], 1)] = t + q * Q;
    __syncthreads();
    int maxcnt = 0;
#pragma unroll
    for (int i = 0; i < G; ++i) maxcnt = max(maxcnt, cnt[i] <= KMAX ? cnt[i] : 0);
    const bool retry = cnt[g] > KMAX;
    const int ncand = retry ? 0 : cnt[g];

    // FP64 re-score of the candidates, CB at a time
    long long bkey = -1;
    int bs = 0;
    double2 bc = make_double2(0.0, 0.0);
    for (int base = 0; base < maxcnt; base += CB) {
#pragma unroll
        for (int c = 0; c < CB; ++c) {
            const int s = (base + c < ncand) ? cand[base + c] : -1;
            double2 acc = make_double2(0.0, 0.0);
            if (s >= 0 && valid) {
#pragma unroll
                for (int r = 0; r < 4; ++r) {
                    const double2 b = ld_z(p2, (t + r * Q + s) & (N - 1));
                    acc.x = fma(a[r].x, b.x, fma(a[r].y, b.y, acc.x));
                    acc.y = fma(a[r].y, b.x, fma(-a[r].x, b.y, acc.y));
                }
            }
            part[c * Q + t] = acc;
        }
        __syncthreads();
        if constexpr (Q <= 32) {
            for (int c = t; c < CB; c += Q) {
                double2 sacc = part[c * Q];
                for (int i = 1; i < Q; ++i) { sacc.x += part[c * Q + i].x; sacc.y += part[c * Q + i].y; }
                tot[g * CB + c] = sacc;
            }
        } else {
            const int w = t >> 5, lane = t & 31;
            for (int c = w; c < CB; c += W) {
                double2 sacc = part[c * Q + lane];
                for (int i = lane + 32; i < Q; i += 32) {
                    sacc.x += part[c * Q + i].x;
                    sacc.y += part[c * Q + i].y;
                }
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    sacc.x += __shfl_xor_sync(0xffffffffu, sacc.x, off);
                    sacc.y += __shfl_xor_sync(0xffffffffu, sacc.y, off);
                }
                if (lane == 0) tot[g * CB + c] = sacc;
            }
        }
        __syncthreads();
        if (t == 0) {
#pragma unroll
            for (int c = 0; c < CB; ++c) {
                if (base + c >= ncand) break;
                const double2 v = tot[g * CB + c];
                const long long k = __double_as_longlong(fma(v.x, v.x, v.y * v.y));
                const int s = cand[base + c];
                if (key_better(k, s, bkey, bs)) { bkey = k; bs = s; bc = v; }
            }
        }
        __syncthreads();
    }
    if (t == 0) {
        bestc[g] = bc;
        const double r = sqrt(fma(bc.x, bc.x, bc.y * bc.y));
        rot[g] = r > 0.0 ? make_double2(bc.x / r, bc.y / r) : make_double2(1.0, 0.0);
        cnt[g] = bs;  // broadcast the winning shift
    }
    __syncthreads();
    const int sbest = cnt[g];
    const double2 rt = rot[g];
    double e = 0.0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const double2 b = valid ? ld_z(p2, (t + r * Q + sbest) & (N - 1)) : make_double2(0.0, 0.0);
        const double rx = fma(rt.x, b.x, -rt.y * b.y);
        const double ry = fma(rt.y, b.x, rt.x * b.y);
        const double dx = a[r].x - rx, dy = a[r].y - ry;
        e = fma(dx, dx, e);
        e = fma(dy, dy, e);
    }
    group_sum<Q>(make_double2(e, 0.0), part, sums, g, t);
    if (t == 0 && valid) {
        if (retry && !bad[g]) {
            status[pair] = kStatusRetryFP64;  // finished by the FP64 kernel
        } else if (bad[g]) {
            shift[pair] = -1;
            theta[pair] = __longlong_as_double(0x7ff8000000000000LL);
            energy[pair] = __longlong_as_double(0x7ff8000000000000LL);
            status[pair] = FA_STATUS_NONFINITE;
        } else {
            const double2 c = bestc[g];
            shift[pair] = sbest;
            theta[pair] = atan2(c.y, c.x);
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
    const size_t smem = MixSmem<LOGN>::bytes;
    auto kern = align_mixed_kernel<LOGN, ZT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "align_mixed: cudaFuncSetAttribute");
    }
    const int64_t blocks = (P + Gm::G - 1) / Gm::G;
    kern<<<(unsigned)blocks, Gm::T, smem, st>>>(static_cast<const ZT*>(z1),
                                                static_cast<const ZT*>(z2), P, h->tf32[LOGN],
                                                shift, theta, energy, status);
    int rc = cuda_error(cudaGetLastError(), "align_mixed launch");
    if (rc != FA_OK) return rc;
    // pairs flagged kStatusRetryFP64 are searched again in FP64 (same stream)
    return launch_align_fft_retry(h, z1, z2, P, LOGN, std::is_same<ZT, double2>::value
                                  ? FA_Z_F64 : FA_Z_F32, shift, theta, energy, status, st);
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
    return set_error(FA_ERR_UNSUPPORTED, "align_mixed: unsupported N");
}

}  // namespace

int launch_align_mixed(const fa_handle* h, const void* z1, const void* z2, int64_t P, int logn,
                       int ztype, int32_t* shift, double* theta, double* energy, int8_t* status,
                       cudaStream_t st)
{
    if (P == 0) return FA_OK;
    if (ztype == FA_Z_F64)
        return dispatch<double2>(h, z1, z2, P, logn, shift, theta, energy, status, st);
    return dispatch<float2>(h, z1, z2, P, logn, shift, theta, energy, status, st);
}

}  // namespace fa
