// align_direct.cu -- FA_DIRECT: the O(N^2) search the paper compares its FFT
// method against (Sec. 2: for every t0, A(t0) by its O(N) sum, then Kabsch),
// written as a fair FP64 GPU baseline.
//
// One CTA per pair.  Both curves sit in shared memory; thread t owns the S
// consecutive shifts s0 = t*S .. s0+S-1 and accumulates
//     c(s) = sum_k z1[k] conj(z2[(k+s) mod N])
// with 4 DFMA per (k, s) -- the minimum for a complex multiply-accumulate.
// The per-shift Kabsch solve collapses to |c(s)| (max over SO(2) of
// tr(R A^T) = |c|), so the best shift maximises |c(s)|^2 (smallest s on exact
// ties); theta = arg c(s*) and the energy of Eq. disc-energy is evaluated
// directly at s*.
#include "fa_internal.cuh"

namespace fa {
namespace {

constexpr int kT = 256;

template <typename ZT, int S>
__global__ void __launch_bounds__(kT)
    align_direct_kernel(const ZT* __restrict__ z1, const ZT* __restrict__ z2, int64_t P, int N,
                        int32_t* __restrict__ shift, double* __restrict__ theta,
                        double* __restrict__ energy, int8_t* __restrict__ status)
{
    extern __shared__ __align__(16) double2 sm[];
    double2* A = sm;                 // z1, N entries
    double2* B = sm + N;             // z2, N entries
    double2* red = sm + 2 * N;       // [kT] FP64 partials
    long long* rk = reinterpret_cast<long long*>(red + kT);  // [kT/32]
    int* ri = reinterpret_cast<int*>(rk + kT / 32);          // [kT/32]
    int* flag = ri + kT / 32;                                // [2]: nonfinite, winner slot

    const int64_t pair = blockIdx.x;
    const int t = threadIdx.x;
    const ZT* p1 = z1 + pair * N;
    const ZT* p2 = z2 + pair * N;
    if (t == 0) flag[0] = 0;
    __syncthreads();
    bool nf = false;
    for (int k = t; k < N; k += kT) {
        const double2 a = ld_z(p1, k), b = ld_z(p2, k);
        nf |= !finite2(a) || !finite2(b);
        A[k] = a;
        B[k] = b;
    }
    if (nf) flag[0] = 1;
    __syncthreads();

    const int s0 = t * S;
    double2 acc[S];
#pragma unroll
    for (int j = 0; j < S; ++j) acc[j] = make_double2(0.0, 0.0);
    if (s0 < N) {
        for (int k = 0; k < N; ++k) {
            const double2 a = A[k];
            int m = k + s0;
            if (m >= N) m -= N;
#pragma unroll
            for (int j = 0; j < S; ++j) {
                const double2 b = B[m];
                acc[j].x = fma(a.x, b.x, fma(a.y, b.y, acc[j].x));
                acc[j].y = fma(a.y, b.x, fma(-a.x, b.y, acc[j].y));
                if (++m == N) m = 0;
            }
        }
    }
    long long key = -1;
    int idx = 0;
#pragma unroll
    for (int j = 0; j < S; ++j) {
        if (s0 + j < N) {
            const long long kq = __double_as_longlong(fma(acc[j].x, acc[j].x, acc[j].y * acc[j].y));
            if (key_better(kq, s0 + j, key, idx)) { key = kq; idx = s0 + j; }
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const long long k2 = __shfl_xor_sync(0xffffffffu, key, off);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, off);
        if (key_better(k2, i2, key, idx)) { key = k2; idx = i2; }
    }
    if ((t & 31) == 0) { rk[t >> 5] = key; ri[t >> 5] = idx; }
    __syncthreads();
    key = rk[0];
    idx = ri[0];
#pragma unroll
    for (int w = 1; w < kT / 32; ++w)
        if (key_better(rk[w], ri[w], key, idx)) { key = rk[w]; idx = ri[w]; }
    const int sbest = idx;
    // the owner of s* publishes c(s*)
    if (sbest >= s0 && sbest < s0 + S) {
#pragma unroll
        for (int j = 0; j < S; ++j)
            if (s0 + j == sbest) red[0] = acc[j];
    }
    __syncthreads();
    const double2 c = red[0];
    if (t == 0) {
        const double r = sqrt(fma(c.x, c.x, c.y * c.y));
        red[1] = r > 0.0 ? make_double2(c.x / r, c.y / r) : make_double2(1.0, 0.0);
    }
    __syncthreads();
    const double2 rot = red[1];
    __syncthreads();
    double e = 0.0;
    for (int k = t; k < N; k += kT) {
        const double2 a = A[k];
        int m = k + sbest;
        if (m >= N) m -= N;
        const double2 b = B[m];
        const double rx = fma(rot.x, b.x, -rot.y * b.y);
        const double ry = fma(rot.y, b.x, rot.x * b.y);
        const double dx = a.x - rx, dy = a.y - ry;
        e = fma(dx, dx, e);
        e = fma(dy, dy, e);
    }
    red[t] = make_double2(e, 0.0);
    __syncthreads();
    if (t < 32) {
        double s = red[t].x;
        for (int i = t + 32; i < kT; i += 32) s += red[i].x;
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
        if (t == 0) {
            if (flag[0]) {
                shift[pair] = -1;
                theta[pair] = __longlong_as_double(0x7ff8000000000000LL);
                energy[pair] = __longlong_as_double(0x7ff8000000000000LL);
                status[pair] = FA_STATUS_NONFINITE;
            } else {
                shift[pair] = sbest;
                theta[pair] = atan2(c.y, c.x);
                energy[pair] = s / (double)N;
                status[pair] = FA_STATUS_OK;
            }
        }
    }
}

template <typename ZT, int S>
int launch_s(const void* z1, const void* z2, int64_t P, int N, int32_t* shift, double* theta,
             double* energy, int8_t* status, cudaStream_t st)
{
    const size_t smem = (size_t)2 * N * sizeof(double2) + kT * sizeof(double2) +
                        (kT / 32) * (sizeof(long long) + sizeof(int)) + 2 * sizeof(int);
    auto kern = align_direct_kernel<ZT, S>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "align_direct: cudaFuncSetAttribute");
    }
    kern<<<(unsigned)P, kT, smem, st>>>(static_cast<const ZT*>(z1), static_cast<const ZT*>(z2), P,
                                        N, shift, theta, energy, status);
    return cuda_error(cudaGetLastError(), "align_direct launch");
}

template <typename ZT>
int dispatch(const void* z1, const void* z2, int64_t P, int N, int32_t* shift, double* theta,
             double* energy, int8_t* status, cudaStream_t st)
{
    const int need = (N + kT - 1) / kT;
    if (need <= 1) return launch_s<ZT, 1>(z1, z2, P, N, shift, theta, energy, status, st);
    if (need <= 2) return launch_s<ZT, 2>(z1, z2, P, N, shift, theta, energy, status, st);
    if (need <= 4) return launch_s<ZT, 4>(z1, z2, P, N, shift, theta, energy, status, st);
    if (need <= 8) return launch_s<ZT, 8>(z1, z2, P, N, shift, theta, energy, status, st);
    return launch_s<ZT, 16>(z1, z2, P, N, shift, theta, energy, status, st);
}

}  // namespace

int launch_align_direct(const fa_handle* h, const void* z1, const void* z2, int64_t P, int N,
                        int ztype, int32_t* shift, double* theta, double* energy, int8_t* status,
                        cudaStream_t st)
{
    (void)h;
    if (P == 0) return FA_OK;
    if (ztype == FA_Z_F64) return dispatch<double2>(z1, z2, P, N, shift, theta, energy, status, st);
    return dispatch<float2>(z1, z2, P, N, shift, theta, energy, status, st);
}

}  // namespace fa
