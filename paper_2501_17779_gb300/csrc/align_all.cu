// align_all.cu -- fa_align_all_pairs: the alignment of every ordered pair of
// M curves (the all-pairs matrix), FP64.
//
// Each curve's spectrum Z_m = DFT(z_m) is computed once (spectra_kernel, two
// curves per thread group) into the caller's workspace; then one thread group
// per unordered pair i < j forms Z_i conj(Z_j) in the first stage of a forward
// transform, giving N c_ij(s) = N sum_k z_i[k] conj(z_j[k+s]) for all s
// (Sec. 2, convolution theorem), takes argmax_s |c_ij(s)|^2 (smallest s on
// exact ties), recomputes c_ij(s*) by its O(N) sum, and evaluates theta and
// the energy of Eq. disc-energy directly.  The pair (j, i) follows from the
// symmetry of the energy: shift (N - s) mod N, angle -theta, the same energy.
// Per pair the FFT work is one transform instead of three.
#include "align_common.cuh"
#include "fft_stages.cuh"

namespace fa {
namespace {

template <int LOGN, typename ZT>
__global__ void __launch_bounds__(Geo<LOGN>::T)
    spectra_kernel(const ZT* __restrict__ z, int64_t M, const double2* __restrict__ W,
                   double2* __restrict__ spec, int8_t* __restrict__ status,
                   int32_t* __restrict__ shift, double* __restrict__ theta,
                   double* __restrict__ energy)
{
    using Gm = Geo<LOGN>;
    constexpr int N = Gm::N, Q = Gm::Q, G = Gm::G;
    extern __shared__ __align__(16) double2 smem[];
    const int g = threadIdx.x / Q;
    const int t = threadIdx.x % Q;
    double2* X1 = smem + (size_t)g * 2 * N;
    double2* X2 = X1 + N;
    int* bad = reinterpret_cast<int*>(smem + (size_t)G * 2 * N);  // [2G]
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
        X1[t + r * Q] = a;
        X2[t + r * Q] = b;
    }
    if (nf1) bad[2 * g] = 1;
    if (nf2) bad[2 * g + 1] = 1;
    __syncthreads();
    fft_two<LOGN>(X1, X2, t, W);
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

// start of row i of the upper triangle in the pair enumeration
__device__ __forceinline__ int64_t tri_start(int64_t i, int64_t M) { return i * (2 * M - i - 1) / 2; }

template <int LOGN, typename ZT>
__global__ void __launch_bounds__(Geo<LOGN>::T)
    allpairs_kernel(const ZT* __restrict__ z, int64_t M, const double2* __restrict__ spec,
                    const double2* __restrict__ W, const int8_t* __restrict__ cstatus,
                    int32_t* __restrict__ shift, double* __restrict__ theta,
                    double* __restrict__ energy)
{
    using Gm = Geo<LOGN>;
    constexpr int N = Gm::N, Q = Gm::Q, G = Gm::G;
    extern __shared__ __align__(16) double2 smem[];
    const int g = threadIdx.x / Q;
    const int t = threadIdx.x % Q;
    double2* X1 = smem + (size_t)g * 2 * N;
    double2* X2 = X1 + N;
    double2* sums = smem + (size_t)G * 2 * N;                  // [G]
    double2* bcast = sums + G;                                  // [G]
    long long* sk = reinterpret_cast<long long*>(bcast + G);    // [G*W]
    int* si = reinterpret_cast<int*>(sk + G * Gm::W);           // [G*W]

    const int64_t npairs = M * (M - 1) / 2;
    const int64_t q = (int64_t)blockIdx.x * G + g;
    const bool valid = q < npairs;
    int64_t i = 0, j = 1;
    if (valid) {
        // invert q = start(i) + (j - i - 1): FP32 estimate, then integer correction
        const float a = (float)(2 * M - 1);
        int64_t e = (int64_t)floorf(0.5f * (a - sqrtf(fmaxf(a * a - 8.0f * (float)q, 0.f))));
        e = max((int64_t)0, min(e, M - 2));
        while (e > 0 && tri_start(e, M) > q) --e;
        while (e < M - 2 && tri_start(e + 1, M) <= q) ++e;
        i = e;
        j = q - tri_start(i, M) + i + 1;
    }
    const double2* Zi = spec + i * N;
    const double2* Zj = spec + j * N;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        X1[t + r * Q] = valid ? Zi[t + r * Q] : make_double2(0.0, 0.0);
        X2[t + r * Q] = valid ? Zj[t + r * Q] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    double2 y[4];
    fft_corr<LOGN>(X1, X2, t, W, y);
    long long key = -1;
    int idx = 0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const long long kq = __double_as_longlong(fma(y[r].x, y[r].x, y[r].y * y[r].y));
        if (key_better(kq, t + r * Q, key, idx)) { key = kq; idx = t + r * Q; }
    }
    group_argmax<Q>(key, idx, sk, si, g, t);
    const int sbest = idx;
    const ZT* zi = z + i * N;
    const ZT* zj = z + j * N;
    double2 a[4], b[4];
    double2 c = make_double2(0.0, 0.0);
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        a[r] = valid ? ld_z(zi, t + r * Q) : make_double2(0.0, 0.0);
        b[r] = valid ? ld_z(zj, (t + r * Q + sbest) & (N - 1)) : make_double2(0.0, 0.0);
        c.x = fma(a[r].x, b[r].x, fma(a[r].y, b[r].y, c.x));
        c.y = fma(a[r].y, b[r].x, fma(-a[r].x, b[r].y, c.y));
    }
    __syncthreads();  // X1 is free for the reductions
    group_sum<Q>(c, X1, sums, g, t);
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
    const double2 csum = sums[g];
    __syncthreads();
    group_sum<Q>(make_double2(e, 0.0), X1, sums, g, t);
    if (t == 0 && valid) {
        const int64_t ij = i * M + j, ji = j * M + i;
        if (cstatus[i] != FA_STATUS_OK || cstatus[j] != FA_STATUS_OK) {
            const double qn = __longlong_as_double(0x7ff8000000000000LL);
            shift[ij] = shift[ji] = -1;
            theta[ij] = theta[ji] = qn;
            energy[ij] = energy[ji] = qn;
        } else {
            const double th = atan2(csum.y, csum.x);
            const double en = sums[g].x * (1.0 / N);
            shift[ij] = sbest;
            theta[ij] = th;
            energy[ij] = en;
            shift[ji] = sbest ? N - sbest : 0;
            theta[ji] = (th == 3.141592653589793) ? th : -th;  // keep (-pi, pi]
            energy[ji] = en;
        }
    }
}

template <int LOGN, typename ZT>
int launch_spec(const fa_handle* h, const void* z, int64_t M, double2* spec, int8_t* status,
                int32_t* shift, double* theta, double* energy, cudaStream_t st)
{
    using Gm = Geo<LOGN>;
    const double2* W = h->tf64[LOGN];
    const ZT* zz = static_cast<const ZT*>(z);
    {
        const size_t smem = (size_t)Gm::G * 2 * Gm::N * sizeof(double2) + 2 * Gm::G * sizeof(int);
        auto kern = spectra_kernel<LOGN, ZT>;
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 (int)smem);
            if (e != cudaSuccess) return cuda_error(e, "spectra: cudaFuncSetAttribute");
        }
        const int64_t groups = (M + 1) / 2;
        kern<<<(unsigned)((groups + Gm::G - 1) / Gm::G), Gm::T, smem, st>>>(zz, M, W, spec, status,
                                                                            shift, theta, energy);
        return cuda_error(cudaGetLastError(), "spectra launch");
    }
}

template <int LOGN, typename ZT>
int launch_all(const fa_handle* h, const void* z, int64_t M, double2* spec, int8_t* status,
               int32_t* shift, double* theta, double* energy, cudaStream_t st)
{
    using Gm = Geo<LOGN>;
    const double2* W = h->tf64[LOGN];
    const ZT* zz = static_cast<const ZT*>(z);
    {
        const int rc = launch_spec<LOGN, ZT>(h, z, M, spec, status, shift, theta, energy, st);
        if (rc != FA_OK) return rc;
    }
    const int64_t npairs = M * (M - 1) / 2;
    if (npairs == 0) return FA_OK;
    const size_t smem = (size_t)Gm::G * 2 * Gm::N * sizeof(double2) + 2 * Gm::G * sizeof(double2) +
                        (size_t)Gm::G * Gm::W * (sizeof(long long) + sizeof(int));
    auto kern = allpairs_kernel<LOGN, ZT>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return cuda_error(e, "allpairs: cudaFuncSetAttribute");
    }
    const int64_t blocks = (npairs + Gm::G - 1) / Gm::G;
    kern<<<(unsigned)blocks, Gm::T, smem, st>>>(zz, M, spec, W, status, shift, theta, energy);
    return cuda_error(cudaGetLastError(), "allpairs launch");
}

template <typename ZT>
int dispatch(const fa_handle* h, const void* z, int64_t M, int logn, double2* spec,
             int8_t* status, int32_t* shift, double* theta, double* energy, cudaStream_t st)
{
    switch (logn) {
#define FA_CASE(L) \
    case L: return launch_all<L, ZT>(h, z, M, spec, status, shift, theta, energy, st);
        FA_CASE(2) FA_CASE(3) FA_CASE(4) FA_CASE(5) FA_CASE(6) FA_CASE(7) FA_CASE(8) FA_CASE(9)
        FA_CASE(10) FA_CASE(11) FA_CASE(12)
#undef FA_CASE
    }
    return set_error(FA_ERR_UNSUPPORTED, "align_all_pairs: unsupported N");
}

}  // namespace

size_t align_all_ws_bytes(int64_t M, int N) { return (size_t)M * (size_t)N * sizeof(double2); }

int launch_spectra(const fa_handle* h, const void* z, int64_t M, int logn, int ztype,
                   double2* spec, int8_t* status, int32_t* shift, double* theta, double* energy,
                   cudaStream_t st)
{
    if (M == 0) return FA_OK;
    switch (logn) {
#define FA_CASE(L)                                                                          \
    case L:                                                                                 \
        return ztype == FA_Z_F64                                                            \
                   ? launch_spec<L, double2>(h, z, M, spec, status, shift, theta, energy, st) \
                   : launch_spec<L, float2>(h, z, M, spec, status, shift, theta, energy, st);
        FA_CASE(2) FA_CASE(3) FA_CASE(4) FA_CASE(5) FA_CASE(6) FA_CASE(7) FA_CASE(8) FA_CASE(9)
        FA_CASE(10) FA_CASE(11) FA_CASE(12)
#undef FA_CASE
    }
    return set_error(FA_ERR_UNSUPPORTED, "spectra: unsupported N");
}

int launch_align_all(const fa_handle* h, const void* z, int64_t M, int logn, int ztype, void* ws,
                     int8_t* status, int32_t* shift, double* theta, double* energy,
                     cudaStream_t st)
{
    if (M == 0) return FA_OK;
    double2* spec = static_cast<double2*>(ws);
    if (ztype == FA_Z_F64)
        return dispatch<double2>(h, z, M, logn, spec, status, shift, theta, energy, st);
    return dispatch<float2>(h, z, M, logn, spec, status, shift, theta, energy, st);
}

}  // namespace fa
