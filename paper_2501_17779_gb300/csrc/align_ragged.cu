// align_ragged.cu -- fa_align_pairs_ragged: rigid alignment (Algorithm 2) of
// pairs with different node counts n_p in ONE persistent launch, FP64.
//
// Transform length.  For n a power of two the cyclic correlation
// c(s) = sum_k z1[k] conj(z2[(k+s) mod n]) is computed with transforms of
// length L = n.  Otherwise it is the exact linear correlation of
//     a[k] = z1[k] (k < n), 0 (n <= k < L)   and   b[m] = z2[m mod n] (m < 2n), 0
// with L = the power of two >= 2n: for s < n every index k+s < 2n <= L, so the
// length-L cyclic correlation DFT(A conj(B)) / L equals c(s) -- no chirps.
//
// Sub-transforms.  Shared memory holds one array of B = min(L, 4096) complex
// doubles.  For L = R B (R = 2 or 4) the first radix-R decimation-in-frequency
// stage is applied on the fly while loading: y_q[t] = W_L^{qt} sum_r
// x[t + rB] W_R^{qr}, and X[Rm + q] = DFT_B(y_q)[m].  The spectrum product is
// taken per q, F_q = DFT_B(Z1_q conj Z2_q), and the shifts that are needed
// are recombined by the matching decimation-in-time step
//     L c(s) = sum_q W_L^{qs} F_q[s mod B],   s < n.
// Z1_q and F_q live in a per-CTA slice of the workspace (L2 resident).
//
// Scheduling.  ragged_keys_kernel buckets the pairs by log2 L (invalid sizes
// are answered there), ragged_order_kernel writes a work list ordered by
// decreasing L (longest first keeps the tail short), and the persistent CTAs
// pop items from it with one atomic counter.  Every step is a plain launch or
// a memset on the caller's stream, so the sequence can be captured in a CUDA
// graph.  The CTA size (256, 512 or 1024 threads) is the tunable, chosen by
// fa_align_pairs_ragged_autotune from timed runs on the caller's batch.
#include <algorithm>

#include "fa_internal.cuh"
#include "fft_stages.cuh"
#include "cta_ops.cuh"

namespace fa {
namespace {

constexpr int BMAX = 4096;       // largest shared-memory sub-transform
constexpr int LOG_BMAX = 12;
constexpr int kBuckets = 16;     // log2 L in [2, 14]; kBuckets-1 unused
constexpr int kCounterBytes = 256;

struct RaggedCounters {
    int hist[kBuckets];
    int cursor[kBuckets];
    int head;
};

__device__ __forceinline__ int ilog2(int x) { return 31 - __clz(x); }

// transform length for n nodes (0 when unsupported)
__device__ __forceinline__ int ragged_len(int n)
{
    if (n < 4 || n > kMaxRaggedN) return 0;
    if ((n & (n - 1)) == 0) return n;
    return 1 << (ilog2(2 * n - 1) + 1);
}

__global__ void ragged_keys_kernel(const int64_t* __restrict__ off, int64_t P, int max_n,
                                   RaggedCounters* __restrict__ cnt, int32_t* __restrict__ shift,
                                   double* __restrict__ theta, double* __restrict__ energy,
                                   int8_t* __restrict__ status)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int64_t n64 = off[p + 1] - off[p];
    const int n = (n64 > 0 && n64 <= kMaxRaggedN) ? (int)n64 : 0;
    const int L = (n <= max_n) ? ragged_len(n) : 0;
    if (L == 0) {
        shift[p] = -1;
        theta[p] = __longlong_as_double(0x7ff8000000000000LL);
        energy[p] = __longlong_as_double(0x7ff8000000000000LL);
        status[p] = FA_STATUS_BAD_SIZE;
        return;
    }
    atomicAdd(&cnt->hist[ilog2(L)], 1);
}

__global__ void ragged_order_kernel(const int64_t* __restrict__ off, int64_t P, int max_n,
                                    RaggedCounters* __restrict__ cnt, int* __restrict__ order)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= P) return;
    const int64_t n64 = off[p + 1] - off[p];
    const int n = (n64 > 0 && n64 <= kMaxRaggedN) ? (int)n64 : 0;
    const int L = (n <= max_n) ? ragged_len(n) : 0;
    if (L == 0) return;
    const int b = ilog2(L);
    int pos = 0;
    for (int k = b + 1; k < kBuckets; ++k) pos += cnt->hist[k];
    order[pos + atomicAdd(&cnt->cursor[b], 1)] = (int)p;
}

// y_q[t] = W_L^{qt} sum_{r<R} x[t + rB] W_R^{qr} into X, where x is the padded
// sequence of one curve: x[k] = z[k] for k < n (KIND 0), or z[k mod n] for
// k < 2n (KIND 1, the periodic extension), zero beyond.
template <int T, int KIND, typename ZT>
__device__ void load_dif(double2* X, const ZT* __restrict__ z, int n, int L, int B, int R, int q,
                         const double2* __restrict__ WL)
{
    const int lim = (KIND == 0) ? n : 2 * n;
    for (int t = threadIdx.x; t < B; t += T) {
        double2 acc = make_double2(0.0, 0.0);
        for (int r = 0; r < R; ++r) {
            const int k = t + r * B;
            double2 x = make_double2(0.0, 0.0);
            if (k < lim) x = ld_z(z, (KIND == 0 || k < n) ? k : k - n);
            // times W_R^{qr} = (-i)^{4qr/R}, R in {1, 2, 4}
            const int e = (q * r * (4 / R)) & 3;  // power of -i
            if (e == 0) { acc.x += x.x; acc.y += x.y; }
            else if (e == 1) { acc.x += x.y; acc.y -= x.x; }
            else if (e == 2) { acc.x -= x.x; acc.y -= x.y; }
            else { acc.x -= x.y; acc.y += x.x; }
        }
        if (q > 0) acc = cmul(acc, __ldg(WL + q * t));
        X[t] = acc;
    }
}

struct RaggedArgs {
    const void* z1;
    const void* z2;
    const int64_t* off;
    int64_t P;
    int max_n;
    RaggedCounters* cnt;
    const int* order;
    double2* slots;         // per-CTA scratch: 2 * Lmax complex doubles each
    int64_t slot_elems;     // 2 * Lmax
    int32_t* shift;
    double* theta;
    double* energy;
    int8_t* status;
};

struct Tables {
    const double2* tf[LOG_BMAX + 1];      // FMA-form twiddles for B <= 4096
    const double2* tw[kMaxRaggedLogL + 1];  // W_L^k for L <= 16384
};

template <int T, typename ZT>
__global__ void __launch_bounds__(T)
    ragged_kernel(const __grid_constant__ RaggedArgs a, const __grid_constant__ Tables tb)
{
    extern __shared__ __align__(16) double2 smem[];
    double2* X = smem;                       // [BMAX]
    double2* part = smem + BMAX;             // [T + 1]
    long long* sk = reinterpret_cast<long long*>(part + T + 1);  // [T/32]
    int* si = reinterpret_cast<int*>(sk + T / 32);               // [T/32]
    int* item = si + T / 32;                                     // [2]
    const ZT* Z1 = static_cast<const ZT*>(a.z1);
    const ZT* Z2 = static_cast<const ZT*>(a.z2);
    double2* Zs = a.slots + (int64_t)blockIdx.x * a.slot_elems;  // Z1_q parts [L]
    double2* Fs = Zs + a.slot_elems / 2;                          // F_q parts [L]
    int total = 0;
    for (int b = 0; b < kBuckets; ++b) total += a.cnt->hist[b];

    for (;;) {
        if (threadIdx.x == 0) item[0] = atomicAdd(&a.cnt->head, 1);
        __syncthreads();
        const int it = item[0];
        __syncthreads();
        if (it >= total) break;
        const int p = a.order[it];
        const int64_t o = a.off[p];
        const int n = (int)(a.off[p + 1] - o);
        const ZT* z1 = Z1 + o;
        const ZT* z2 = Z2 + o;
        int L = n;
        if ((n & (n - 1)) != 0) L = 1 << (ilog2(2 * n - 1) + 1);
        const int logL = ilog2(L);
        const int logb = min(logL, LOG_BMAX);
        const int B = 1 << logb, R = L >> logb;
        const double2* Wf = tb.tf[logb];
        const double2* WL = tb.tw[logL];

        // non-finite inputs
        bool nf = false;
        for (int k = threadIdx.x; k < n; k += T) nf |= !finite2(ld_z(z1, k)) || !finite2(ld_z(z2, k));
        const bool bad = __syncthreads_or(nf);
        if (bad) {
            if (threadIdx.x == 0) {
                a.shift[p] = -1;
                a.theta[p] = __longlong_as_double(0x7ff8000000000000LL);
                a.energy[p] = __longlong_as_double(0x7ff8000000000000LL);
                a.status[p] = FA_STATUS_NONFINITE;
            }
            continue;
        }
        // spectra of the padded curve 1, one DIF part at a time
        for (int q = 0; q < R; ++q) {
            load_dif<T, 0>(X, z1, n, L, B, R, q, WL);
            __syncthreads();
            fft_rt<T, BMAX>(X, logb, Wf);
            for (int m = threadIdx.x; m < B; m += T) Zs[q * B + m] = X[m];
            __syncthreads();
        }
        // per part: spectrum of curve 2, product, correlation transform
        for (int q = 0; q < R; ++q) {
            load_dif<T, 1>(X, z2, n, L, B, R, q, WL);
            __syncthreads();
            fft_rt<T, BMAX>(X, logb, Wf);
            for (int m = threadIdx.x; m < B; m += T) X[m] = cmulc(Zs[q * B + m], X[m]);
            __syncthreads();
            fft_rt<T, BMAX>(X, logb, Wf);
            if (q < R - 1)
                for (int m = threadIdx.x; m < B; m += T) Fs[q * B + m] = X[m];
            __syncthreads();
        }
        // L c(s) = sum_q W_L^{qs} F_q[s mod B] for s < n; F_{R-1} is still in X
        long long key = -1;
        int idx = 0;
        for (int s = threadIdx.x; s < n; s += T) {
            const int sm = s & (B - 1);
            double2 c = X[sm];
            if (R > 1) {
                c = cmul(c, __ldg(WL + (((R - 1) * s) & (L - 1))));
                for (int q = 0; q < R - 1; ++q) {
                    double2 f = Fs[q * B + sm];
                    if (q > 0) f = cmul(f, __ldg(WL + ((q * s) & (L - 1))));
                    c.x += f.x;
                    c.y += f.y;
                }
            }
            const long long kq = __double_as_longlong(fma(c.x, c.x, c.y * c.y));
            if (key_better(kq, s, key, idx)) { key = kq; idx = s; }
        }
        cta_argmax<T>(key, idx, sk, si);
        const int sbest = idx;
        // c(s*) by its O(n) sum, theta, energy by its definition
        double2 c = make_double2(0.0, 0.0);
        for (int k = threadIdx.x; k < n; k += T) {
            const double2 u = ld_z(z1, k);
            int m = k + sbest;
            if (m >= n) m -= n;
            const double2 v = ld_z(z2, m);
            c.x = fma(u.x, v.x, fma(u.y, v.y, c.x));
            c.y = fma(u.y, v.x, fma(-u.x, v.y, c.y));
        }
        c = cta_sum<T>(c, part);
        const double rr = sqrt(fma(c.x, c.x, c.y * c.y));
        const double2 rot = rr > 0.0 ? make_double2(c.x / rr, c.y / rr) : make_double2(1.0, 0.0);
        double e = 0.0;
        for (int k = threadIdx.x; k < n; k += T) {
            const double2 u = ld_z(z1, k);
            int m = k + sbest;
            if (m >= n) m -= n;
            const double2 v = ld_z(z2, m);
            const double rx = fma(rot.x, v.x, -rot.y * v.y);
            const double ry = fma(rot.y, v.x, rot.x * v.y);
            const double dx = u.x - rx, dy = u.y - ry;
            e = fma(dx, dx, e);
            e = fma(dy, dy, e);
        }
        const double2 es = cta_sum<T>(make_double2(e, 0.0), part);
        if (threadIdx.x == 0) {
            a.shift[p] = sbest;
            a.theta[p] = atan2(c.y, c.x);
            a.energy[p] = es.x / (double)n;
            a.status[p] = FA_STATUS_OK;
        }
    }
}

template <int T>
constexpr size_t ragged_smem() { return (size_t)BMAX * 16 + (T + 1) * 16 + (T / 32) * 12 + 16; }

template <int T, typename ZT>
int launch_t(const fa_handle* h, const RaggedArgs& a, const Tables& tb, int grid, cudaStream_t st)
{
    ragged_kernel<T, ZT><<<grid, T, ragged_smem<T>(), st>>>(a, tb);
    return cuda_error(cudaGetLastError(), "ragged launch");
}

// longest transform over all node counts n <= max_n: a non-power-of-two n just
// below a power of two needs the power of two >= 2n - 1
int64_t lmax_for(int max_n)
{
    int64_t L = 4;
    while (L < 2 * (int64_t)max_n - 1) L <<= 1;
    return L;
}

inline size_t a256(size_t b) { return (b + 255) & ~(size_t)255; }

}  // namespace

int ragged_grid(const fa_handle* h, int T)
{
    int per_sm = 1;
    cudaError_t e = cudaSuccess;
    switch (T) {
        case 1024: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ragged_kernel<1024, double2>, 1024, ragged_smem<1024>()); break;
        case 512: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ragged_kernel<512, double2>, 512, ragged_smem<512>()); break;
        default: e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ragged_kernel<256, double2>, 256, ragged_smem<256>()); break;
    }
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return per_sm * h->num_sms;
}

int ragged_set_attributes()
{
    const void* ks[] = {(const void*)ragged_kernel<1024, double2>, (const void*)ragged_kernel<1024, float2>,
                        (const void*)ragged_kernel<256, double2>, (const void*)ragged_kernel<256, float2>,
                        (const void*)ragged_kernel<512, double2>, (const void*)ragged_kernel<512, float2>};
    const size_t sm[] = {ragged_smem<1024>(), ragged_smem<1024>(), ragged_smem<256>(),
                         ragged_smem<256>(), ragged_smem<512>(), ragged_smem<512>()};
    for (int i = 0; i < 6; ++i) {
        cudaError_t e = cudaFuncSetAttribute(ks[i], cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm[i]);
        if (e != cudaSuccess) return cuda_error(e, "ragged: cudaFuncSetAttribute");
    }
    return FA_OK;
}

size_t ragged_ws_bytes(const fa_handle* h, int64_t P, int max_n)
{
    const int grid = std::max(ragged_grid(h, 1024), std::max(ragged_grid(h, 256), ragged_grid(h, 512)));
    const int64_t L = lmax_for(max_n);
    return a256(kCounterBytes) + a256((size_t)P * sizeof(int)) +
           (size_t)grid * 2 * (size_t)L * sizeof(double2);
}

int launch_align_ragged(const fa_handle* h, const void* z1, const void* z2, const int64_t* off,
                        int64_t P, int max_n, int ztype, int threads, int32_t* shift,
                        double* theta, double* energy, int8_t* status, void* ws,
                        cudaStream_t st)
{
    if (P == 0) return FA_OK;
    char* w = static_cast<char*>(ws);
    RaggedCounters* cnt = reinterpret_cast<RaggedCounters*>(w);
    int* order = reinterpret_cast<int*>(w + a256(kCounterBytes));
    double2* slots = reinterpret_cast<double2*>(w + a256(kCounterBytes) + a256((size_t)P * sizeof(int)));
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(RaggedCounters), st);
    if (e != cudaSuccess) return cuda_error(e, "ragged: memset");
    const unsigned nb = (unsigned)((P + 255) / 256);
    ragged_keys_kernel<<<nb, 256, 0, st>>>(off, P, max_n, cnt, shift, theta, energy, status);
    ragged_order_kernel<<<nb, 256, 0, st>>>(off, P, max_n, cnt, order);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "ragged: keys/order launch");
    RaggedArgs a;
    a.z1 = z1; a.z2 = z2; a.off = off; a.P = P; a.max_n = max_n; a.cnt = cnt; a.order = order;
    a.slots = slots; a.slot_elems = 2 * lmax_for(max_n);
    a.shift = shift; a.theta = theta; a.energy = energy; a.status = status;
    Tables tb;
    for (int i = 0; i <= LOG_BMAX; ++i) tb.tf[i] = (i >= kMinLogN) ? h->tf64[i] : nullptr;
    for (int i = 0; i <= kMaxRaggedLogL; ++i) tb.tw[i] = (i >= kMinLogN) ? h->tw64[i] : nullptr;
    const int T = (threads == 1024 || threads == 512) ? threads : 256;
    const int grid = ragged_grid(h, T);
    const bool f64 = ztype == FA_Z_F64;
    if (T == 1024) return f64 ? launch_t<1024, double2>(h, a, tb, grid, st) : launch_t<1024, float2>(h, a, tb, grid, st);
    if (T == 512) return f64 ? launch_t<512, double2>(h, a, tb, grid, st) : launch_t<512, float2>(h, a, tb, grid, st);
    return f64 ? launch_t<256, double2>(h, a, tb, grid, st) : launch_t<256, float2>(h, a, tb, grid, st);
}

}  // namespace fa
