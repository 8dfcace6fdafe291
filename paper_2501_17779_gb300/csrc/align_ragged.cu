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
// graph.  Each bucket's plan (CTA size, pairs per CTA, or a cluster of CTAs
// per pair) is the tunable, chosen by fa_align_pairs_ragged_autotune from
// timed runs on the caller's batch.
#include <cooperative_groups.h>

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
    int bhead[kBuckets];  // per bucket: items handed out so far
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
// k < 2n (KIND 1, the periodic extension), zero beyond.  Only the nonzero
// inputs are added (terms r < ceil(lim / B), and within them k < lim: both
// conditions are uniform over all but one warp), and y_q[t] = 0 for t >= lim
// skips the twiddle.
template <int T, int KIND, typename ZT>
__device__ void load_dif(double2* X, const ZT* __restrict__ z, int n, int L, int B, int R, int q,
                         const double2* __restrict__ WL, int tl)
{
    const int lim = (KIND == 0) ? n : 2 * n;
    const int rmax = min(R, (lim + B - 1) / B);
    for (int t = tl; t < B; t += T) {
        double2 acc = make_double2(0.0, 0.0);
        if (t < lim) {
            acc = ld_z(z, (KIND == 0 || t < n) ? t : t - n);
            for (int r = 1; r < rmax; ++r) {
                const int k = t + r * B;
                if (k >= lim) break;
                const double2 x = ld_z(z, (KIND == 0 || k < n) ? k : k - n);
                // times W_R^{qr} = (-i)^{4qr/R}, R in {2, 4}
                const int e = (q * r * (4 / R)) & 3;  // power of -i
                if (e == 0) { acc.x += x.x; acc.y += x.y; }
                else if (e == 1) { acc.x += x.y; acc.y -= x.x; }
                else if (e == 2) { acc.x -= x.x; acc.y -= x.y; }
                else { acc.x -= x.y; acc.y += x.x; }
            }
            if (q > 0) acc = cmul(acc, __ldg(WL + q * t));
        }
        X[t] = acc;
    }
}

struct RaggedArgs {
    const void* z1;
    const void* z2;
    const int64_t* off;
    int64_t P;
    int max_n;
    int bucket;             // log2 L of the pairs this launch processes
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

// ---- reductions over a group of TG threads (local index tl) ----------------
// Every group of the CTA calls them at the same time (their barriers are
// CTA-wide); sk/si/part are the group's own slices of shared memory.
template <int TG>
__device__ __forceinline__ void grp_argmax(long long& key, int& idx, long long* sk, int* si, int tl)
{
    constexpr int W = TG < 32 ? TG : 32;
#pragma unroll
    for (int off = W / 2; off > 0; off >>= 1) {
        const long long k2 = __shfl_xor_sync(0xffffffffu, key, off, W);
        const int i2 = __shfl_xor_sync(0xffffffffu, idx, off, W);
        if (key_better(k2, i2, key, idx)) { key = k2; idx = i2; }
    }
    if constexpr (TG > 32) {
        if ((tl & 31) == 0) { sk[tl >> 5] = key; si[tl >> 5] = idx; }
        __syncthreads();
        key = sk[0];
        idx = si[0];
#pragma unroll
        for (int w = 1; w < TG / 32; ++w)
            if (key_better(sk[w], si[w], key, idx)) { key = sk[w]; idx = si[w]; }
        __syncthreads();
    }
}

template <int TG>
__device__ __forceinline__ double2 grp_sum(double2 v, double2* part, int tl)
{
    part[tl] = v;
    __syncthreads();
    if constexpr (TG >= 32) {
        if (tl < 32) {
            double2 s = part[tl];
            for (int i = tl + 32; i < TG; i += 32) { s.x += part[i].x; s.y += part[i].y; }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                s.x += __shfl_xor_sync(0xffffffffu, s.x, off);
                s.y += __shfl_xor_sync(0xffffffffu, s.y, off);
            }
            if (tl == 0) part[TG] = s;
        }
    } else {
        if (tl == 0) {
            double2 s = part[0];
            for (int i = 1; i < TG; ++i) { s.x += part[i].x; s.y += part[i].y; }
            part[TG] = s;
        }
    }
    __syncthreads();
    const double2 r = part[TG];
    __syncthreads();
    return r;
}

// Plan of one bucket: T threads per CTA, G pairs per CTA (T / G threads per
// pair).  G = 1 handles every length (L > 4096 by the radix-R split); G >= 2
// keeps both spectra of each pair in shared memory, so G L <= 2048.
template <int T, int G>
constexpr int grp_lmax() { return G == 1 ? (1 << kMaxRaggedLogL) : BMAX / (2 * G); }

template <int T, int G, typename ZT>
__global__ void __launch_bounds__(T)
    ragged_kernel(const __grid_constant__ RaggedArgs a, const __grid_constant__ Tables tb)
{
    constexpr int TG = T / G;
    constexpr int SW = TG >= 32 ? TG / 32 : 1;  // argmax slots per group
    extern __shared__ __align__(16) double2 smem[];
    double2* X = smem;                                          // [BMAX]
    double2* part_all = smem + BMAX;                            // [G][TG + 1]
    long long* sk_all = reinterpret_cast<long long*>(part_all + G * (TG + 1));  // [G][SW]
    int* si_all = reinterpret_cast<int*>(sk_all + G * SW);                     // [G][SW]
    int* item = si_all + G * SW;                                               // [1 + G]
    const int g = threadIdx.x / TG, tl = threadIdx.x % TG;
    double2* part = part_all + g * (TG + 1);
    long long* sk = sk_all + g * SW;
    int* si = si_all + g * SW;
    int* badf = item + 1;
    const ZT* Z1 = static_cast<const ZT*>(a.z1);
    const ZT* Z2 = static_cast<const ZT*>(a.z2);
    double2* Zs = a.slots + (int64_t)blockIdx.x * a.slot_elems;  // Z1_q parts [L] (G = 1)
    double2* Fs = Zs + a.slot_elems / 2;                          // F_q parts [L] (G = 1)
    const int b = a.bucket;
    const int count = a.cnt->hist[b];
    int start = 0;
    for (int k = b + 1; k < kBuckets; ++k) start += a.cnt->hist[k];
    const int L = 1 << b, logL = b;
    const int logb = min(logL, LOG_BMAX);
    const int B = 1 << logb, R = L >> logb;  // R > 1 only for G = 1
    const double2* Wf = tb.tf[logb];
    const double2* WL = tb.tw[logL];

    for (;;) {
        if (threadIdx.x == 0) item[0] = atomicAdd(&a.cnt->bhead[b], G);
        if (threadIdx.x < G) badf[threadIdx.x] = 0;
        __syncthreads();
        const int base = item[0];
        __syncthreads();
        if (base >= count) break;
        const bool valid = base + g < count;
        const int p = valid ? a.order[start + base + g] : 0;
        const int64_t o = valid ? a.off[p] : 0;
        const int n = valid ? (int)(a.off[p + 1] - o) : 0;
        const ZT* z1 = Z1 + o;
        const ZT* z2 = Z2 + o;

        // non-finite inputs: that pair is answered with NaNs and computed on
        // zeros (its group still takes part in every barrier)
        bool nf = false;
        for (int k = tl; k < n; k += TG) nf |= !finite2(ld_z(z1, k)) || !finite2(ld_z(z2, k));
        if (nf) badf[g] = 1;
        __syncthreads();
        const bool bad = badf[g] != 0;
        const int nn = bad ? 0 : n;  // the node count the transforms see

        long long key = -1;
        int idx = 0;
        if constexpr (G == 1) {
            // spectra of the padded curve 1, one DIF part at a time
            for (int q = 0; q < R; ++q) {
                load_dif<T, 0>(X, z1, nn, L, B, R, q, WL, tl);
                __syncthreads();
                fft_rt_g<T, BMAX>(X, logb, Wf, tl);
                for (int m = tl; m < B; m += T) Zs[q * B + m] = X[m];
                __syncthreads();
            }
            // per part: spectrum of curve 2, product, correlation transform
            for (int q = 0; q < R; ++q) {
                load_dif<T, 1>(X, z2, nn, L, B, R, q, WL, tl);
                __syncthreads();
                fft_rt_g<T, BMAX>(X, logb, Wf, tl);
                for (int m = tl; m < B; m += T) X[m] = cmulc(Zs[q * B + m], X[m]);
                __syncthreads();
                fft_rt_g<T, BMAX>(X, logb, Wf, tl);
                if (q < R - 1)
                    for (int m = tl; m < B; m += T) Fs[q * B + m] = X[m];
                __syncthreads();
            }
            // L c(s) = sum_q W_L^{qs} F_q[s mod B] for s < n (F_{R-1} is still
            // in X), as the matching radix-R decimation-in-time step: for m < B,
            // G_q = W_L^{qm} F_q[m] and L c(m + jB) = sum_q W_R^{qj} G_q, only
            // for the j with m + jB < n
            auto take = [&](double2 c, int s) {
                const long long kq = __double_as_longlong(fma(c.x, c.x, c.y * c.y));
                if (key_better(kq, s, key, idx)) { key = kq; idx = s; }
            };
            const int mlim = min(B, nn);
            if (R == 1) {
                for (int s = tl; s < nn; s += T) take(X[s], s);
            } else if (R == 2) {
                for (int m = tl; m < mlim; m += T) {
                    const double2 g0 = Fs[m], g1 = cmul(X[m], __ldg(WL + m));
                    take(make_double2(g0.x + g1.x, g0.y + g1.y), m);
                    if (m + B < nn) take(make_double2(g0.x - g1.x, g0.y - g1.y), m + B);
                }
            } else {
                for (int m = tl; m < mlim; m += T) {
                    const double2 g0 = Fs[m];
                    const double2 g1 = cmul(Fs[B + m], __ldg(WL + m));
                    const double2 g2 = cmul(Fs[2 * B + m], __ldg(WL + 2 * m));
                    const double2 g3 = cmul(X[m], __ldg(WL + 3 * m));
                    const double2 a0 = make_double2(g0.x + g2.x, g0.y + g2.y);
                    const double2 a1 = make_double2(g0.x - g2.x, g0.y - g2.y);
                    const double2 b0 = make_double2(g1.x + g3.x, g1.y + g3.y);
                    const double2 b1 = make_double2(g1.x - g3.x, g1.y - g3.y);
                    // W_4^{qj} = (-i)^{qj}: j = 0: a0 + b0; 1: a1 - i b1; 2: a0 - b0; 3: a1 + i b1
                    take(make_double2(a0.x + b0.x, a0.y + b0.y), m);
                    if (m + B < nn) take(make_double2(a1.x + b1.y, a1.y - b1.x), m + B);
                    if (m + 2 * B < nn) take(make_double2(a0.x - b0.x, a0.y - b0.y), m + 2 * B);
                    if (m + 3 * B < nn) take(make_double2(a1.x - b1.y, a1.y + b1.x), m + 3 * B);
                }
            }
        } else {
            // both spectra of each pair in shared memory (L <= BMAX / (2G))
            double2* Xg = X + (size_t)g * 2 * (BMAX / (2 * G));
            double2* Yg = Xg + BMAX / (2 * G);
            load_dif<TG, 0>(Xg, z1, nn, L, L, 1, 0, WL, tl);
            load_dif<TG, 1>(Yg, z2, nn, L, L, 1, 0, WL, tl);
            __syncthreads();
            fft_rt_g<TG, BMAX / (2 * G)>(Xg, logb, Wf, tl);
            fft_rt_g<TG, BMAX / (2 * G)>(Yg, logb, Wf, tl);
            for (int m = tl; m < L; m += TG) Xg[m] = cmulc(Xg[m], Yg[m]);
            __syncthreads();
            fft_rt_g<TG, BMAX / (2 * G)>(Xg, logb, Wf, tl);
            for (int s = tl; s < nn; s += TG) {
                const double2 c = Xg[s];
                const long long kq = __double_as_longlong(fma(c.x, c.x, c.y * c.y));
                if (key_better(kq, s, key, idx)) { key = kq; idx = s; }
            }
        }
        grp_argmax<TG>(key, idx, sk, si, tl);
        const int sbest = idx;
        // c(s*) by its O(n) sum, theta, energy by its definition
        double2 c = make_double2(0.0, 0.0);
        for (int k = tl; k < nn; k += TG) {
            const double2 u = ld_z(z1, k);
            int m = k + sbest;
            if (m >= nn) m -= nn;
            const double2 v = ld_z(z2, m);
            c.x = fma(u.x, v.x, fma(u.y, v.y, c.x));
            c.y = fma(u.y, v.x, fma(-u.x, v.y, c.y));
        }
        c = grp_sum<TG>(c, part, tl);
        const double rr = sqrt(fma(c.x, c.x, c.y * c.y));
        const double2 rot = rr > 0.0 ? make_double2(c.x / rr, c.y / rr) : make_double2(1.0, 0.0);
        double e = 0.0;
        for (int k = tl; k < nn; k += TG) {
            const double2 u = ld_z(z1, k);
            int m = k + sbest;
            if (m >= nn) m -= nn;
            const double2 v = ld_z(z2, m);
            const double rx = fma(rot.x, v.x, -rot.y * v.y);
            const double ry = fma(rot.y, v.x, rot.x * v.y);
            const double dx = u.x - rx, dy = u.y - ry;
            e = fma(dx, dx, e);
            e = fma(dy, dy, e);
        }
        const double2 es = grp_sum<TG>(make_double2(e, 0.0), part, tl);
        if (tl == 0 && valid) {
            if (bad) {
                a.shift[p] = -1;
                a.theta[p] = __longlong_as_double(0x7ff8000000000000LL);
                a.energy[p] = __longlong_as_double(0x7ff8000000000000LL);
                a.status[p] = FA_STATUS_NONFINITE;
            } else {
                a.shift[p] = sbest;
                a.theta[p] = atan2(c.y, c.x);
                a.energy[p] = es.x / (double)n;
                a.status[p] = FA_STATUS_OK;
            }
        }
    }
}

// ---- one pair per thread-block cluster (L = R BMAX, R = 2 or 4) -------------
// CTA q of the cluster computes DIF part q of both spectra and F_q =
// DFT_B(Z1_q conj Z2_q), all in its own shared memory (no global slots); the
// recombination L c(s) = sum_q W_L^{qs} F_q[s mod B] reads the other CTAs' F_q
// through distributed shared memory, each CTA taking a 1/R share of the
// shifts; the argmax, c(s*) and the energy are reduced over the cluster in
// rank order.  Every CTA of a cluster takes the same branches and reaches every
// cluster barrier (the pair index is read from rank 0 and the non-finite test
// is repeated by every rank on the whole curves).
struct ClusterShared {
    long long key;  // this rank's best |c|^2 key
    double2 c;      // this rank's share of c(s*)
    double e;       // this rank's share of the energy sum
    int idx;        // shift of key
    int item;       // the pair's position in the bucket (rank 0)
    int bad;
};

template <int T>
constexpr size_t ragged_cluster_smem()
{
    return (size_t)2 * BMAX * 16 + (size_t)(T + 1) * 16 + (size_t)(T / 32) * 12 + 16 +
           sizeof(ClusterShared);
}

template <int T, int R, typename ZT>
__global__ void __launch_bounds__(T, 1)
    ragged_cluster_kernel(const __grid_constant__ RaggedArgs a, const __grid_constant__ Tables tb)
{
    namespace cg = cooperative_groups;
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank();
    extern __shared__ __align__(16) double2 smem[];
    double2* Z = smem;                  // [BMAX] curve 1's part q, then its spectrum
    double2* X = Z + BMAX;              // [BMAX] curve 2's part q, the product, then F_q
    double2* part = X + BMAX;           // [T + 1] CTA sums
    long long* sk = reinterpret_cast<long long*>(part + T + 1);  // [T / 32]
    int* si = reinterpret_cast<int*>(sk + T / 32);               // [T / 32]
    ClusterShared* sh = reinterpret_cast<ClusterShared*>(
        (reinterpret_cast<uintptr_t>(si + T / 32) + 15) & ~uintptr_t(15));
    const int tid = threadIdx.x;
    const ZT* Z1 = static_cast<const ZT*>(a.z1);
    const ZT* Z2 = static_cast<const ZT*>(a.z2);
    const int b = a.bucket;
    const int count = a.cnt->hist[b];
    int start = 0;
    for (int k = b + 1; k < kBuckets; ++k) start += a.cnt->hist[k];
    const int L = 1 << b;
    constexpr int B = BMAX;
    const double2* Wf = tb.tf[LOG_BMAX];
    const double2* WL = tb.tw[b];
    const double2* F[R];
    ClusterShared* shr[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        F[r] = cluster.map_shared_rank(X, r);
        shr[r] = cluster.map_shared_rank(sh, r);
    }

    for (;;) {
        if (q == 0 && tid == 0) sh->item = atomicAdd(&a.cnt->bhead[b], 1);
        cluster.sync();
        const int item = shr[0]->item;
        cluster.sync();  // every rank has read rank 0's value before it changes
        if (item >= count) break;
        const int p = a.order[start + item];
        const int64_t o = a.off[p];
        const int n = (int)(a.off[p + 1] - o);
        const ZT* z1 = Z1 + o;
        const ZT* z2 = Z2 + o;
        if (tid == 0) sh->bad = 0;
        __syncthreads();
        bool nf = false;
        for (int k = tid; k < n; k += T) nf |= !finite2(ld_z(z1, k)) || !finite2(ld_z(z2, k));
        if (nf) sh->bad = 1;
        __syncthreads();
        const bool bad = sh->bad != 0;
        const int nn = bad ? 0 : n;

        // part q of both spectra, the product, F_q
        load_dif<T, 0>(Z, z1, nn, L, B, R, q, WL, tid);
        __syncthreads();
        fft_rt<T, BMAX>(Z, LOG_BMAX, Wf);
        load_dif<T, 1>(X, z2, nn, L, B, R, q, WL, tid);
        __syncthreads();
        fft_rt<T, BMAX>(X, LOG_BMAX, Wf);
        for (int m = tid; m < B; m += T) X[m] = cmulc(Z[m], X[m]);
        __syncthreads();
        fft_rt<T, BMAX>(X, LOG_BMAX, Wf);
        cluster.sync();  // every F_q is complete

        // this rank's shifts: L c(s) = sum_r W_L^{rs} F_r[s mod B]
        const int share = (nn + R - 1) / R;
        const int s0 = q * share, s1 = min(nn, s0 + share);
        long long key = -1;
        int idx = 0;
        for (int s = s0 + tid; s < s1; s += T) {
            const int sm = s & (B - 1);
            double2 c = F[0][sm];
#pragma unroll
            for (int r = 1; r < R; ++r) {
                const double2 f = cmul(F[r][sm], __ldg(WL + ((r * s) & (L - 1))));
                c.x += f.x;
                c.y += f.y;
            }
            const long long kq = __double_as_longlong(fma(c.x, c.x, c.y * c.y));
            if (key_better(kq, s, key, idx)) { key = kq; idx = s; }
        }
        cta_argmax<T>(key, idx, sk, si);
        if (tid == 0) { sh->key = key; sh->idx = idx; }
        cluster.sync();
        long long bk = -1;
        int sbest = 0;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const long long kr = shr[r]->key;
            const int ir = shr[r]->idx;
            if (key_better(kr, ir, bk, sbest)) { bk = kr; sbest = ir; }
        }

        // c(s*) and the energy by their definitions, k split over the ranks
        const int k0 = s0, k1 = s1;
        double2 c = make_double2(0.0, 0.0);
        for (int k = k0 + tid; k < k1; k += T) {
            const double2 u = ld_z(z1, k);
            int m = k + sbest;
            if (m >= nn) m -= nn;
            const double2 v = ld_z(z2, m);
            c.x = fma(u.x, v.x, fma(u.y, v.y, c.x));
            c.y = fma(u.y, v.x, fma(-u.x, v.y, c.y));
        }
        c = cta_sum<T>(c, part);
        if (tid == 0) sh->c = c;
        cluster.sync();
        double2 cs = make_double2(0.0, 0.0);
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const double2 cr = shr[r]->c;
            cs.x += cr.x;
            cs.y += cr.y;
        }
        const double rr = sqrt(fma(cs.x, cs.x, cs.y * cs.y));
        const double2 rot = rr > 0.0 ? make_double2(cs.x / rr, cs.y / rr) : make_double2(1.0, 0.0);
        double e = 0.0;
        for (int k = k0 + tid; k < k1; k += T) {
            const double2 u = ld_z(z1, k);
            int m = k + sbest;
            if (m >= nn) m -= nn;
            const double2 v = ld_z(z2, m);
            const double rx = fma(rot.x, v.x, -rot.y * v.y);
            const double ry = fma(rot.y, v.x, rot.x * v.y);
            const double dx = u.x - rx, dy = u.y - ry;
            e = fma(dx, dx, e);
            e = fma(dy, dy, e);
        }
        const double2 es = cta_sum<T>(make_double2(e, 0.0), part);
        if (tid == 0) sh->e = es.x;
        cluster.sync();
        if (q == 0 && tid == 0) {
            if (bad) {
                a.shift[p] = -1;
                a.theta[p] = __longlong_as_double(0x7ff8000000000000LL);
                a.energy[p] = __longlong_as_double(0x7ff8000000000000LL);
                a.status[p] = FA_STATUS_NONFINITE;
            } else {
                double et = 0.0;
#pragma unroll
                for (int r = 0; r < R; ++r) et += shr[r]->e;
                a.shift[p] = sbest;
                a.theta[p] = atan2(cs.y, cs.x);
                a.energy[p] = et / (double)n;
                a.status[p] = FA_STATUS_OK;
            }
        }
    }
}

template <int T, int G>
constexpr size_t ragged_smem()
{
    constexpr int TG = T / G, SW = TG >= 32 ? TG / 32 : 1;
    return (size_t)BMAX * 16 + (size_t)G * (TG + 1) * 16 + (size_t)G * SW * 12 + 4 * (1 + G) + 16;
}

// the plans compiled in: (T, G); G = -R for one pair per cluster of R CTAs
struct PlanDesc { int T, G; };
constexpr PlanDesc kPlans[] = {{256, 1}, {512, 1}, {1024, 1}, {128, 2}, {256, 2}, {512, 2},
                               {128, 4}, {256, 4}, {512, 4}, {256, 8}, {256, 16},
                               {256, -2}, {512, -2}, {256, -4}, {512, -4}};
constexpr int kNPlans = sizeof(kPlans) / sizeof(kPlans[0]);

template <int T, int G>
const void* kernel_ptr(bool f64)
{
    if constexpr (G < 0)
        return f64 ? (const void*)ragged_cluster_kernel<T, -G, double2>
                   : (const void*)ragged_cluster_kernel<T, -G, float2>;
    else
        return f64 ? (const void*)ragged_kernel<T, G, double2> : (const void*)ragged_kernel<T, G, float2>;
}
template <int T, int G>
constexpr size_t plan_smem()
{
    if constexpr (G < 0) return ragged_cluster_smem<T>();
    else return ragged_smem<T, G>();
}

// f(kernel pointer, smem bytes) for plan i
template <typename F>
auto with_plan(int i, bool f64, F&& f)
{
    switch (i) {
#define FA_PLAN(k, T_, G_) \
    case k: return f(kernel_ptr<T_, G_>(f64), plan_smem<T_, G_>(), T_);
        FA_PLAN(0, 256, 1) FA_PLAN(1, 512, 1) FA_PLAN(2, 1024, 1) FA_PLAN(3, 128, 2)
        FA_PLAN(4, 256, 2) FA_PLAN(5, 512, 2) FA_PLAN(6, 128, 4) FA_PLAN(7, 256, 4)
        FA_PLAN(8, 512, 4) FA_PLAN(9, 256, 8) FA_PLAN(10, 256, 16)
        FA_PLAN(11, 256, -2) FA_PLAN(12, 512, -2) FA_PLAN(13, 256, -4) FA_PLAN(14, 512, -4)
#undef FA_PLAN
    }
    return f(kernel_ptr<256, 1>(f64), ragged_smem<256, 1>(), 256);
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

// launch configuration of a cluster plan (grid filled in by the caller)
cudaLaunchConfig_t cluster_config(int T, size_t smem, int R, cudaStream_t st, cudaLaunchAttribute* attr)
{
    cudaLaunchConfig_t cfg = {};
    cfg.blockDim = dim3((unsigned)T);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    attr->id = cudaLaunchAttributeClusterDimension;
    attr->val.clusterDim.x = (unsigned)R;
    attr->val.clusterDim.y = 1;
    attr->val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cfg;
}

int plan_grid(const fa_handle* h, int i)
{
    if (kPlans[i].G < 0) {
        // clusters that can be resident at once, R CTAs each
        const int R = -kPlans[i].G;
        int nc = 0;
        const cudaError_t e = with_plan(i, true, [&](const void* k, size_t smem, int T) {
            cudaLaunchAttribute attr;
            cudaLaunchConfig_t cfg = cluster_config(T, smem, R, nullptr, &attr);
            cfg.gridDim = dim3((unsigned)(R * (h->num_sms > 0 ? h->num_sms : 1)));
            return cudaOccupancyMaxActiveClusters(&nc, k, &cfg);
        });
        if (e != cudaSuccess || nc < 1) nc = 1;
        return nc * R;
    }
    int per_sm = 1;
    const cudaError_t e = with_plan(i, true, [&](const void* k, size_t smem, int T) {
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, T, smem);
    });
    if (e != cudaSuccess || per_sm < 1) per_sm = 1;
    return per_sm * h->num_sms;
}

Tables make_tables(const fa_handle* h)
{
    Tables tb;
    for (int i = 0; i <= LOG_BMAX; ++i) tb.tf[i] = (i >= kMinLogN) ? h->tf64[i] : nullptr;
    for (int i = 0; i <= kMaxRaggedLogL; ++i) tb.tw[i] = (i >= kMinLogN) ? h->tw64[i] : nullptr;
    return tb;
}

int launch_bucket(const fa_handle* h, RaggedArgs a, const Tables& tb, int bucket, int plan,
                  bool f64, cudaStream_t st)
{
    a.bucket = bucket;
    const int grid = plan_grid(h, plan);
    const int R = kPlans[plan].G < 0 ? -kPlans[plan].G : 1;
    const cudaError_t e = with_plan(plan, f64, [&](const void* k, size_t smem, int T) {
        void* args[] = {(void*)&a, (void*)&tb};
        if (R == 1) return cudaLaunchKernel(k, dim3((unsigned)grid), dim3((unsigned)T), args, smem, st);
        cudaLaunchAttribute attr;
        cudaLaunchConfig_t cfg = cluster_config(T, smem, R, st, &attr);
        cfg.gridDim = dim3((unsigned)grid);
        return cudaLaunchKernelExC(&cfg, k, args);
    });
    return cuda_error(e, "ragged launch");
}

}  // namespace

int ragged_num_plans() { return kNPlans; }
int ragged_plan_threads(int i) { return (i >= 0 && i < kNPlans) ? kPlans[i].T : 0; }
int ragged_plan_group(int i) { return (i >= 0 && i < kNPlans) ? kPlans[i].G : 0; }

// can plan i run transforms of length 2^bucket?
bool ragged_plan_fits(int i, int bucket)
{
    if (i < 0 || i >= kNPlans) return false;
    const int G = kPlans[i].G, L = 1 << bucket;
    if (G == 1) return true;
    if (G < 0) return L == -G * BMAX;  // a cluster of R CTAs: exactly R parts of BMAX
    return L <= BMAX / (2 * G) && kPlans[i].T / G <= L;
}

int ragged_default_plan(int bucket)
{
    const int L = 1 << bucket;
    if (L <= 128) return 10;   // 16 pairs of 16 threads
    if (L <= 256) return 9;    // 8 pairs of 32 threads
    if (L <= 512) return 7;    // 4 pairs of 64 threads
    if (L <= 1024) return 4;   // 2 pairs of 128 threads
    return 0;                  // one pair of 256 threads
}

int ragged_set_attributes()
{
    for (int i = 0; i < kNPlans; ++i)
        for (int f = 0; f < 2; ++f) {
            const cudaError_t e = with_plan(i, f == 0, [&](const void* k, size_t smem, int) {
                return cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            });
            if (e != cudaSuccess) return cuda_error(e, "ragged: cudaFuncSetAttribute");
        }
    return FA_OK;
}

size_t ragged_ws_bytes(const fa_handle* h, int64_t P, int max_n)
{
    int grid = 1;
    for (int i = 0; i < kNPlans; ++i)
        if (kPlans[i].G == 1) grid = std::max(grid, plan_grid(h, i));
    const int64_t L = lmax_for(max_n);
    return a256(kCounterBytes) + a256((size_t)P * sizeof(int)) +
           (size_t)grid * 2 * (size_t)L * sizeof(double2);
}

int ragged_max_bucket(int max_n)
{
    int b = 2;
    while ((1ll << b) < lmax_for(max_n)) ++b;
    return b;
}

// counters, bucket histogram and the longest-first work list
int ragged_prepare(const int64_t* off, int64_t P, int max_n, void* ws, int32_t* shift,
                   double* theta, double* energy, int8_t* status, cudaStream_t st)
{
    char* w = static_cast<char*>(ws);
    RaggedCounters* cnt = reinterpret_cast<RaggedCounters*>(w);
    int* order = reinterpret_cast<int*>(w + a256(kCounterBytes));
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(RaggedCounters), st);
    if (e != cudaSuccess) return cuda_error(e, "ragged: memset");
    const unsigned nb = (unsigned)((P + 255) / 256);
    ragged_keys_kernel<<<nb, 256, 0, st>>>(off, P, max_n, cnt, shift, theta, energy, status);
    ragged_order_kernel<<<nb, 256, 0, st>>>(off, P, max_n, cnt, order);
    return cuda_error(cudaGetLastError(), "ragged: keys/order launch");
}

// the bucket counts of the last ragged_prepare (device -> host, synchronises)
int ragged_hist(void* ws, int* hist, cudaStream_t st)
{
    RaggedCounters c;
    cudaError_t e = cudaMemcpyAsync(&c, ws, sizeof(RaggedCounters), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "ragged: histogram");
    for (int b = 0; b < kBuckets; ++b) hist[b] = c.hist[b];
    return FA_OK;
}

int ragged_run_bucket(const fa_handle* h, const void* z1, const void* z2, const int64_t* off,
                      int64_t P, int max_n, int ztype, int bucket, int plan, int32_t* shift,
                      double* theta, double* energy, int8_t* status, void* ws, bool reset,
                      cudaStream_t st)
{
    char* w = static_cast<char*>(ws);
    RaggedCounters* cnt = reinterpret_cast<RaggedCounters*>(w);
    if (reset) {
        const cudaError_t e = cudaMemsetAsync(&cnt->bhead[bucket], 0, sizeof(int), st);
        if (e != cudaSuccess) return cuda_error(e, "ragged: memset");
    }
    RaggedArgs a;
    a.z1 = z1; a.z2 = z2; a.off = off; a.P = P; a.max_n = max_n; a.cnt = cnt;
    a.order = reinterpret_cast<int*>(w + a256(kCounterBytes));
    a.slots = reinterpret_cast<double2*>(w + a256(kCounterBytes) + a256((size_t)P * sizeof(int)));
    a.slot_elems = 2 * lmax_for(max_n);
    a.shift = shift; a.theta = theta; a.energy = energy; a.status = status;
    return launch_bucket(h, a, make_tables(h), bucket, plan, ztype == FA_Z_F64, st);
}

int launch_align_ragged(const fa_handle* h, const void* z1, const void* z2, const int64_t* off,
                        int64_t P, int max_n, int ztype, int32_t* shift, double* theta,
                        double* energy, int8_t* status, void* ws, cudaStream_t st)
{
    if (P == 0) return FA_OK;
    int rc = ragged_prepare(off, P, max_n, ws, shift, theta, energy, status, st);
    if (rc != FA_OK) return rc;
    // longest transforms first (their launch's tail is covered by the next)
    for (int b = ragged_max_bucket(max_n); b >= kMinLogN; --b) {
        rc = ragged_run_bucket(h, z1, z2, off, P, max_n, ztype, b, h->ragged_plan[b], shift, theta,
                               energy, status, ws, false, st);
        if (rc != FA_OK) return rc;
    }
    return FA_OK;
}

}  // namespace fa
