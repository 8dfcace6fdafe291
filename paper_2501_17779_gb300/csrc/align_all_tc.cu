// align_all_tc.cu -- fa_align_all_pairs with the shift search on the tensor
// cores: the DFT of every cross-spectrum as one dense GEMM (tcgen05), the
// best 8 shifts per pair kept in the epilogue, those 8 re-scored exactly, and
// theta / energy at the winner.
//
// For curves i < j with spectra Z = DFT(z) (Sec. 2, convolution theorem),
//   c_ij(s) = sum_k z_i[k] conj(z_j[k+s]) = (1/N) sum_f P_ij[f] e^{-2 pi i f s / N},
//   P_ij[f] = Z_i[f] conj(Z_j[f]),
// so the correlations of all pairs are the product of the matrix of
// cross-spectra (one row per pair, 2N real columns: Re P, Im P per f) with a
// fixed real DFT matrix B (2N x 2N: columns Re c(s), Im c(s)):
//   Re c = sum_f Re P cos + Im P sin,   Im c = sum_f Im P cos - Re P sin
// (angle 2 pi f s / N).  C[i,j,s] is never stored: each CTA holds 128 pairs
// (one i, 128 consecutive j) in tensor memory, 128 shifts (256 columns) at a
// time, and keeps every pair's 8 largest |c(s)|^2 (smallest s first on ties)
// in registers.
//
// Precision variants (operands rounded to the tensor core's input type, float32
// accumulation in tensor memory):
//   BF16X3  each operand as bfloat16 hi + lo pieces, products hi hi + hi lo +
//           lo hi (about 16 significant bits)
//   FP16X3  the same with float16 pieces (about 22 bits; the cross-spectra
//           are scaled by 2^14 so that their pieces stay in float16 range)
//   TF32    one TF32 product (about 11 bits)
//   TF32X3  TF32 hi + lo pieces, three products (about 21 bits)
// The 8 candidates of each pair are then re-scored by their direct O(N)
// correlation, summed exactly on a fixed grid with float32 remainders (about
// 40 bits for complex64 input; float-float otherwise),
// the largest |c(s)|^2 wins (smallest s on ties), theta = arg c(s*) and the
// energy of Eq. disc-energy by its definition, both at FP64-bound accuracy.
//
// GEMM kernel: one CTA of 448 threads per SM, persistent over (i, j-tile)
// tiles from an atomic counter; per tile, per 128-shift column block, the
// 2N-long contraction runs in chunks of 64 bytes per row (32 f16 or 16 tf32
// elements) through four shared-memory stages.  Warps 0-7 form the 128
// cross-spectrum rows of each chunk (FP32 from the complex64 spectra, split
// into pieces, several lanes per row so that their loads are coalesced); one
// lane of warp 12 issues the MMAs, one lane of warp 13 bulk-copies
// (cp.async.bulk, completion on an mbarrier) the pre-tiled DFT blocks as far
// ahead as the stages allow; warps 8-11 read the
// finished accumulators and keep each pair's best 8 shifts, while the MMAs of
// the next column block run into the other accumulator.  The epilogue warps run
// their own tile loop (the others synchronise per tile on a named barrier), so
// the last column block of a tile is read while the next tile's MMAs start.  All waits are
// bounded; a wait that runs out sets an error flag that turns every output of
// the call into NaN.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <type_traits>

#include "align_common.cuh"
#include "df.cuh"
#include "umma.cuh"

namespace fa {
namespace {

constexpr int kTcT = 128;           // pairs per tile = TMEM lanes
constexpr int kTcProducers = 256;   // warps 0-7 form the operand rows
constexpr int kEpiWarp0 = kTcProducers / 32;   // warps 8-11 read the accumulators
constexpr int kIssuerWarp = kEpiWarp0 + 4;      // warp 12 issues the MMAs
constexpr int kCopyWarp = kIssuerWarp + 1;      // warp 13 copies the DFT blocks
constexpr int kTcThreads = 32 * (kCopyWarp + 1);
constexpr int kRowB = 64;      // bytes per operand row per K chunk
constexpr int kStages = 4;
constexpr int kCand = 8;       // candidate shifts kept per pair
constexpr float kPScale = 16384.0f;  // 2^14: cross-spectra scale (float16 range)

template <int V>
struct TcVar;
// MARGIN: a candidate whose GEMM |c|^2 is below (1 - MARGIN) times the best
// one's cannot be the maximum when the GEMM's relative error on |c|^2 is at
// most eps with MARGIN >= 2 eps (the best candidate is then >= (1 - eps) T and
// the largest value seen <= (1 + eps) T, T the true maximum), so it is not
// re-scored.  eps is about 6e-5 for bfloat16 pieces (16 bits) and 2e-6 for
// float16 / TF32 pieces (21-22 bits); the margins below are 65x and 250x that.
// Plain TF32 (11 bits) re-scores all 8.
template <>
struct TcVar<FA_PREC_TC_BF16X3> {
    static constexpr int ES = 2, NP = 2;
    static constexpr uint32_t FMT = 1;  // bfloat16 (kind::f16)
    static constexpr bool TF32 = false;
    static constexpr float MARGIN = 1.0f / 256.0f;
};
template <>
struct TcVar<FA_PREC_TC_FP16X3> {
    static constexpr int ES = 2, NP = 2;
    static constexpr uint32_t FMT = 0;  // float16 (kind::f16)
    static constexpr bool TF32 = false;
    static constexpr float MARGIN = 1.0f / 2048.0f;
};
template <>
struct TcVar<FA_PREC_TC_TF32> {
    static constexpr int ES = 4, NP = 1;
    static constexpr uint32_t FMT = 2;  // tf32 (kind::tf32)
    static constexpr bool TF32 = true;
    static constexpr float MARGIN = 2.0f;  // keeps every candidate
};
template <>
struct TcVar<FA_PREC_TC_TF32X3> {
    static constexpr int ES = 4, NP = 2;
    static constexpr uint32_t FMT = 2;
    static constexpr bool TF32 = true;
    static constexpr float MARGIN = 1.0f / 2048.0f;
};

// round a float to TF32 (10 fraction bits), to nearest even
__device__ __forceinline__ uint32_t tf32_rn(float x)
{
    uint32_t u = __float_as_uint(x);
    if ((u & 0x7f800000u) == 0x7f800000u) return u;
    u += 0xfffu + ((u >> 13) & 1u);
    return u & 0xffffe000u;
}

// x as NP pieces of the variant's element type (bit patterns, 16 or 32 bits)
template <int V>
__device__ __forceinline__ void to_pieces(float x, uint32_t& hi, uint32_t& lo)
{
    using T = TcVar<V>;
    if constexpr (T::TF32) {
        hi = tf32_rn(x);
        lo = T::NP > 1 ? tf32_rn(__fsub_rn(x, __uint_as_float(hi))) : 0u;
    } else if constexpr (T::FMT == 1) {
        const __nv_bfloat16 h = __float2bfloat16_rn(x);
        hi = __bfloat16_as_ushort(h);
        lo = __bfloat16_as_ushort(__float2bfloat16_rn(__fsub_rn(x, __bfloat162float(h))));
    } else {
        const __half h = __float2half_rn(x);
        hi = __half_as_ushort(h);
        lo = __half_as_ushort(__float2half_rn(__fsub_rn(x, __half2float(h))));
    }
}

// x0, x1 as two packed 16-bit pieces each (hi = x0 | x1 << 16 rounded, lo the
// rounded remainders), for the variants with 16-bit operands
template <int V>
__device__ __forceinline__ void to_pieces2(float x0, float x1, uint32_t& hi, uint32_t& lo)
{
    using T = TcVar<V>;
    static_assert(!T::TF32, "16-bit variants only");
    if constexpr (T::FMT == 1) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x0, x1);
        const float2 hf = __bfloat1622float2(h);
        const __nv_bfloat162 l = __floats2bfloat162_rn(__fsub_rn(x0, hf.x), __fsub_rn(x1, hf.y));
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    } else {
        const __half2 h = __floats2half2_rn(x0, x1);
        const float2 hf = __half22float2(h);
        const __half2 l = __floats2half2_rn(__fsub_rn(x0, hf.x), __fsub_rn(x1, hf.y));
        hi = *reinterpret_cast<const uint32_t*>(&h);
        lo = *reinterpret_cast<const uint32_t*>(&l);
    }
}

// start of row i of the upper triangle in the pair enumeration
__device__ __forceinline__ int64_t tri_start_tc(int64_t i, int64_t M) { return i * (2 * M - i - 1) / 2; }

// sum_{a=1}^{n} ceil(a / 128): the j-tiles of rows i' < i are F(M-1) - F(M-1-i)
__host__ __device__ __forceinline__ int64_t ceil_sum128(int64_t n)
{
    if (n <= 0) return 0;
    // sum_{a=1}^{n} ceil(a/q) = sum_{b=0}^{n-1} (floor(b/q) + 1)
    const int64_t q = 128, k = (n - 1) / q;  // floor((n-1)/q)
    return n + q * k * (k - 1) / 2 + k * (n - 1 - q * k + 1);
}

// ---- the pre-tiled DFT matrix ------------------------------------------------
// Block (cb, kc) holds column block cb (256 columns: Re c(s), Im c(s) for
// s = 128 cb .. 128 cb + 127) and K chunk kc (64 bytes per row), NP pieces,
// each piece 256 rows x 64 bytes in the K-major core-matrix layout, so that
// one bulk copy fills a stage.
template <int V, int LOGN>
__global__ void dft_tab_kernel(uint8_t* __restrict__ tab)
{
    using T = TcVar<V>;
    constexpr int N = 1 << LOGN, KC = kRowB / T::ES, NK = 2 * N / KC;
    constexpr size_t PIECE = (size_t)256 * kRowB, BLOCK = PIECE * T::NP;
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // (cb, kc, row, k)
    const int64_t total = (int64_t)(N / 128) * NK * 256 * KC;
    if (e >= total) return;
    const int k = (int)(e % KC);
    const int row = (int)((e / KC) % 256);
    const int kc = (int)((e / (KC * 256)) % NK);
    const int cb = (int)(e / ((int64_t)KC * 256 * NK));
    const int s = cb * 128 + (row & 127);
    const int kg = kc * KC + k;  // global contraction index: 2 f + (0: Re P, 1: Im P)
    const int f = kg >> 1;
    double sn, cs;
    sincospi(2.0 * (double)((f * s) & (N - 1)) / (double)N, &sn, &cs);
    double v;
    if (row < 128) v = (kg & 1) ? sn : cs;   // Re c: Re P cos + Im P sin
    else v = (kg & 1) ? cs : -sn;            // Im c: Im P cos - Re P sin
    uint32_t hi, lo;
    to_pieces<V>((float)v, hi, lo);
    uint8_t* blk = tab + ((size_t)cb * NK + kc) * BLOCK;
    const uint32_t off = umma::tile_off(row, k * T::ES, kRowB);
    if constexpr (T::ES == 2) {
        *reinterpret_cast<uint16_t*>(blk + off) = (uint16_t)hi;
        if (T::NP > 1) *reinterpret_cast<uint16_t*>(blk + PIECE + off) = (uint16_t)lo;
    } else {
        *reinterpret_cast<uint32_t*>(blk + off) = hi;
        if (T::NP > 1) *reinterpret_cast<uint32_t*>(blk + PIECE + off) = lo;
    }
}

// complex64 spectra scaled by 1/N (Fourier coefficients, |Z/N| <= max|z|)
template <int LOGN>
__global__ void spec32_kernel(const double2* __restrict__ spec, int64_t n, float2* __restrict__ out)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    const double2 v = spec[e];
    constexpr double s = 1.0 / (double)(1 << LOGN);
    out[e] = make_float2((float)(v.x * s), (float)(v.y * s));
}

__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* mbar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            umma::smem_u32(dst)),
        "l"(__cvta_generic_to_global(src)), "r"(bytes), "r"(umma::smem_u32(mbar))
        : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(umma::smem_u32(mbar)),
                 "r"(bytes)
                 : "memory");
}

// ---- the GEMM + top-8 kernel --------------------------------------------------
// Warp roles: warps 0-7 produce the cross-spectrum operand rows, warps 8-11
// read the accumulators (TMEM lane = pair), lane 0 of warp 12 issues the MMAs
// and lane 0 of warp 13 copies the DFT blocks.  Per stage: b_full (copy landed), a_full (the
// 256 producers stored their rows), mma_done (the stage's MMAs finished, it
// may be overwritten).  Two accumulators of 256 columns alternate between
// column blocks: acc_full[b] (block finished) and tmem_empty[b] (its 128
// readers are done).
template <int V, int LOGN>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_search_kernel(const float2* __restrict__ spec, int64_t M, const uint8_t* __restrict__ tab,
                     uint16_t* __restrict__ cand, unsigned long long* __restrict__ next,
                     int* __restrict__ err)
{
    using T = TcVar<V>;
    constexpr int N = 1 << LOGN, KC = kRowB / T::ES, NK = 2 * N / KC, KF = KC / 2;
    constexpr int NCB = N / 128;  // column blocks of 128 shifts
    constexpr size_t A_PIECE = (size_t)128 * kRowB, B_PIECE = (size_t)256 * kRowB;
    constexpr size_t STAGE = (A_PIECE + B_PIECE) * T::NP;
    constexpr uint32_t B_BYTES = (uint32_t)(B_PIECE * T::NP);
    constexpr uint32_t ID = umma::idesc(128, 256, T::FMT);
    constexpr int NT = T::NP == 2 ? 3 : 1;
    constexpr int LPR = KF / 2;                // producer lanes per operand row
    constexpr int RPP = kTcProducers / LPR;    // rows per producer pass
    constexpr int NPASS = kTcT / RPP;          // passes per chunk
    static_assert(NPASS * RPP == kTcT && 32 % LPR == 0, "producer mapping");
    extern __shared__ __align__(1024) uint8_t smem[];
    float2* zi_s = reinterpret_cast<float2*>(smem + kStages * STAGE);                  // [N]
    uint64_t* b_full = reinterpret_cast<uint64_t*>(smem + kStages * STAGE + N * 8);    // [kStages]
    uint64_t* a_full = b_full + kStages;                                               // [kStages]
    uint64_t* mma_done = a_full + kStages;                                             // [kStages]
    uint64_t* acc_full = mma_done + kStages;                                           // [2]
    uint64_t* tmem_empty = acc_full + 2;                                               // [2]
    uint64_t* tinfo = tmem_empty + 2;                                                  // [2]
    uint32_t* s_taddr = reinterpret_cast<uint32_t*>(tinfo + 2);
    volatile int* s_abort = reinterpret_cast<volatile int*>(s_taddr + 1);
    volatile long long* s_tile = reinterpret_cast<volatile long long*>(s_taddr + 2);
    volatile long long* s_tring = s_tile + 1;                                          // [2]
    float* escr = reinterpret_cast<float*>(const_cast<long long*>(s_tring + 2));      // [4][32][33]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int prow = tid / LPR, sub = tid % LPR;  // producers: row in a pass, frequency pair

    if (tid == 0) {
        for (int s = 0; s < kStages; ++s) {
            umma::mbar_init(&b_full[s], 1);
            umma::mbar_init(&a_full[s], kTcProducers);
            umma::mbar_init(&mma_done[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            umma::mbar_init(&acc_full[b], 1);
            umma::mbar_init(&tmem_empty[b], kTcT);
            umma::mbar_init(&tinfo[b], 1);
        }
        *s_abort = 0;
        umma::fence_mbar_init();
    }
    if (warp == 0) umma::tmem_alloc(s_taddr, 512);
    umma::tc_fence_before();
    __syncthreads();
    umma::tc_fence_after();
    const uint32_t tmem = *s_taddr;
    const int64_t total_tiles = ceil_sum128(M - 1);
    int64_t g = 0, cbg = 0;  // chunks (producers, issuer) and column blocks (epilogue, issuer) so far
    int64_t copied = 0;      // DFT blocks copied so far (the copier)
    auto fail = [&]() {
        *s_abort = 1;
        atomicExch(err, 1);
    };

    if (warp >= kEpiWarp0 && warp < kIssuerWarp) {
        // ---- epilogue warps: their own tile loop, one tile behind at most.
        // The tile comes through a two-slot ring (tinfo: one arrival per tile
        // from thread 0); the issuer cannot run more than two column blocks
        // ahead of this loop (it waits for tmem_empty), so a slot is never
        // rewritten before it is read.
        float* xs = escr + (size_t)(warp - kEpiWarp0) * 32 * 33 + lane * 33;
        for (int64_t tau = 0;; ++tau) {
            if (!umma::mbar_wait(&tinfo[tau & 1], (uint32_t)(tau >> 1) & 1)) { fail(); break; }
            const int64_t t = s_tring[tau & 1];
            if (t >= total_tiles) break;
            // tile -> (i, j-tile): largest i with tiles_before(i) <= t
            int64_t lo = 0, hi = M - 2;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (ceil_sum128(M - 1) - ceil_sum128(M - 1 - mid) <= t) lo = mid; else hi = mid - 1;
            }
            const int64_t i = lo;
            const int64_t j0 = i + 1 + 128 * (t - (ceil_sum128(M - 1) - ceil_sum128(M - 1 - i)));
            // ---- epilogue: TMEM lane = pair row ----
            const int row = (warp - kEpiWarp0) * 32 + lane;
            float best[kCand];
            int bs[kCand];
#pragma unroll
            for (int q = 0; q < kCand; ++q) { best[q] = -1.0f; bs[q] = 0; }
            // a value below (1 - MARGIN) times the largest seen so far can never
            // be among the candidates kept at the end (the largest only grows),
            // so it is not inserted; the kept set is the same as without the
            // test, and the insertions (a serial chain) become rare
            float top = -1.0f;
            bool ok = true;
            for (int cb = 0; cb < NCB && ok; ++cb) {
                const int buf = (int)(cbg & 1);
                if (!umma::mbar_wait(&acc_full[buf], (uint32_t)(cbg >> 1) & 1)) { fail(); ok = false; break; }
                umma::tc_fence_after();
#pragma unroll 1
                for (int c0 = 0; c0 < 128; c0 += 32) {
                    float re[32], im[32];
                    const uint32_t base = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(buf * 256);
                    umma::tmem_ld32(base + (uint32_t)c0, re);
                    umma::tmem_ld32(base + (uint32_t)(128 + c0), im);
                    float m = top;
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        re[q] = __fmaf_rn(re[q], re[q], __fmul_rn(im[q], im[q]));
                        m = fmaxf(m, re[q]);
                    }
                    top = m;
                    const float thr = fmaxf(best[kCand - 1], __fmul_rn(top, 1.0f - T::MARGIN));
                    // the values that may enter, staged in this lane's row of
                    // shared memory and inserted in shift order: the warp
                    // iterates as often as its busiest lane, not once per
                    // value some lane needs
                    unsigned msk = 0u;
#pragma unroll
                    for (int q = 0; q < 32; ++q) {
                        xs[q] = re[q];
                        msk |= (re[q] > best[kCand - 1] && re[q] >= thr) ? (1u << q) : 0u;
                    }
                    while (msk) {
                        const int q = __ffs(msk) - 1;
                        msk &= msk - 1;
                        float x = xs[q];
                        int sx = cb * 128 + c0 + q;
#pragma unroll
                        for (int r = 0; r < kCand; ++r) {
                            if (x > best[r]) {
                                const float tv = best[r];
                                const int ts = bs[r];
                                best[r] = x; bs[r] = sx;
                                x = tv; sx = ts;
                            }
                        }
                    }
                    __syncwarp();  // converged again for the next tcgen05.ld
                }
                umma::tc_fence_before();
                umma::mbar_arrive(&tmem_empty[buf]);
                ++cbg;
            }
            if (ok && j0 + row < M && !*s_abort) {
                const int64_t j = j0 + row;
                // candidates that can still be the maximum (see TcVar::MARGIN); the
                // count rides in bits 12-15 of the first entry (shifts < 4096)
                int keep = 0;
#pragma unroll
                for (int q = 0; q < kCand; ++q)
                    keep += best[q] >= __fmul_rn(best[0], 1.0f - T::MARGIN) ? 1 : 0;
                keep = max(keep, 1);
                uint4 w;
                w.x = (uint32_t)bs[0] | ((uint32_t)keep << 12) | ((uint32_t)bs[1] << 16);
                w.y = (uint32_t)bs[2] | ((uint32_t)bs[3] << 16);
                w.z = (uint32_t)bs[4] | ((uint32_t)bs[5] << 16);
                w.w = (uint32_t)bs[6] | ((uint32_t)bs[7] << 16);
                *reinterpret_cast<uint4*>(cand + ((size_t)i * M + j) * kCand) = w;
            }
            if (!ok) break;
        }
    } else {
        // ---- producers, MMA issuer and copier: tiles from the counter,
        // synchronised among themselves by a named barrier (the epilogue warps
        // keep their own pace); thread 0 alone decides when to stop, so that
        // every one of these warps leaves the loop together
        constexpr unsigned kMain = kTcThreads - 32 * (kIssuerWarp - kEpiWarp0);
        auto main_sync = [&]() { asm volatile("bar.sync 1, %0;" ::"r"(kMain) : "memory"); };
        for (int64_t tau = 0;; ++tau) {
            if (tid == 0) {
                const long long tt = *s_abort ? (long long)total_tiles : (long long)atomicAdd(next, 1ull);
                *s_tile = tt;
                s_tring[tau & 1] = tt;
                umma::mbar_arrive(&tinfo[tau & 1]);
            }
            main_sync();
            const int64_t t = *s_tile;
            if (t >= total_tiles) break;
            // tile -> (i, j-tile): largest i with tiles_before(i) <= t
            int64_t lo = 0, hi = M - 2;
            while (lo < hi) {
                const int64_t mid = (lo + hi + 1) >> 1;
                if (ceil_sum128(M - 1) - ceil_sum128(M - 1 - mid) <= t) lo = mid; else hi = mid - 1;
            }
            const int64_t i = lo;
            const int64_t j0 = i + 1 + 128 * (t - (ceil_sum128(M - 1) - ceil_sum128(M - 1 - i)));
            if (warp < kEpiWarp0)
                for (int k = tid; k < N; k += kTcProducers) {
                    // curve i's spectrum times the cross-spectrum scale (a power of
                    // two: the products below round exactly as if scaled after)
                    const float2 v = spec[i * N + k];
                    zi_s[k] = make_float2(v.x * kPScale, v.y * kPScale);
                }
            main_sync();
            if (warp < kEpiWarp0) {
                // ---- producers ----
                // Operand rows are formed LPR lanes per pair, two frequencies per
                // lane (one 16-byte load), so that a warp's load covers LPR * 16
                // contiguous bytes of each of 32 / LPR rows; pass q handles rows
                // q RPP + tid / LPR.
                const float4* zrow[NPASS];
#pragma unroll
                for (int q = 0; q < NPASS; ++q) {
                    const int64_t j = j0 + q * RPP + prow;
                    zrow[q] = reinterpret_cast<const float4*>(spec + (j < M ? j : i) * N) + sub;
                }
                // this thread's spectrum values of the next two chunks
                float4 zb[NPASS], zb2[NPASS];
#pragma unroll
                for (int q = 0; q < NPASS; ++q) {
                    zb[q] = zrow[q][0];
                    zb2[q] = zrow[q][(1 % NK) * (KF / 2)];
                }
                const float4* zi4 = reinterpret_cast<const float4*>(zi_s) + sub;
                // this thread's byte offsets in an operand stage, one per pass
                uint32_t soff[NPASS];
#pragma unroll
                for (int q = 0; q < NPASS; ++q) soff[q] = umma::tile_off(q * RPP + prow, sub * 4 * T::ES, kRowB);
                // One K chunk: wait for its stage, form and store this thread's
                // operand pieces from zbuf, signal, then load the chunk two ahead
                // into zbuf (K chunks wrap to the first ones for the next column
                // block).  The loads come after the proxy fence, which would
                // otherwise wait for them.
                auto produce = [&](int kc, float4 (&zbuf)[NPASS]) -> bool {
                    const int st = (int)(g % kStages);
                    const uint32_t use = (uint32_t)(g / kStages);
                    uint8_t* sa = smem + st * STAGE;
                    if (*s_abort) return false;
                    if (use > 0 && !umma::mbar_wait(&mma_done[st], (use - 1) & 1)) { fail(); return false; }
                    // frequencies kc KF + 2 sub, + 1 of curve i (pre-scaled)
                    const float4 a = zi4[kc * (KF / 2)];
#pragma unroll
                    for (int q = 0; q < NPASS; ++q) {
                        const float4 b = zbuf[q];
                        const float v0 = __fmaf_rn(a.x, b.x, __fmul_rn(a.y, b.y));
                        const float v1 = __fmaf_rn(a.y, b.x, -__fmul_rn(a.x, b.y));
                        const float v2 = __fmaf_rn(a.z, b.z, __fmul_rn(a.w, b.w));
                        const float v3 = __fmaf_rn(a.w, b.z, -__fmul_rn(a.z, b.w));
                        if constexpr (T::ES == 2) {
                            uint32_t h01, l01, h23, l23;
                            to_pieces2<V>(v0, v1, h01, l01);
                            to_pieces2<V>(v2, v3, h23, l23);
                            *reinterpret_cast<uint2*>(sa + soff[q]) = make_uint2(h01, h23);
                            *reinterpret_cast<uint2*>(sa + A_PIECE + soff[q]) = make_uint2(l01, l23);
                        } else {
                            uint32_t ph[4], pl[4];
                            to_pieces<V>(v0, ph[0], pl[0]);
                            to_pieces<V>(v1, ph[1], pl[1]);
                            to_pieces<V>(v2, ph[2], pl[2]);
                            to_pieces<V>(v3, ph[3], pl[3]);
                            *reinterpret_cast<uint4*>(sa + soff[q]) = make_uint4(ph[0], ph[1], ph[2], ph[3]);
                            if (T::NP > 1)
                                *reinterpret_cast<uint4*>(sa + A_PIECE + soff[q]) =
                                    make_uint4(pl[0], pl[1], pl[2], pl[3]);
                        }
                    }
                    umma::fence_async_smem();
                    umma::mbar_arrive(&a_full[st]);
                    const int fn = ((kc + 2) % NK) * (KF / 2);
#pragma unroll
                    for (int q = 0; q < NPASS; ++q) zbuf[q] = zrow[q][fn];
                    ++g;
                    return true;
                };
                // two chunks per trip: the buffers trade roles without copies
                bool ok = true;
                for (int cb = 0; cb < NCB && ok; ++cb)
                    for (int kc = 0; kc < NK && ok; kc += 2) ok = produce(kc, zb) && produce(kc + 1, zb2);
            } else if (warp == kIssuerWarp && lane == 0) {
                // ---- the MMA issuer: chunk c as soon as its operands are in.
                // Chunk c of the tile is column block c / NK, K chunk c % NK.
                constexpr int NC = NCB * NK;
                for (int c = 0; c < NC && !*s_abort; ++c, ++g) {
                    const int kc = c % NK;
                    const int buf = (int)(cbg & 1);
                    const int st = (int)(g % kStages);
                    const uint32_t use = (uint32_t)(g / kStages);
                    if (kc == 0 && cbg >= 2 &&
                        !umma::mbar_wait(&tmem_empty[buf], (uint32_t)((cbg >> 1) - 1) & 1)) {
                        fail();
                        break;
                    }
                    if (!umma::mbar_wait(&b_full[st], use & 1) || !umma::mbar_wait(&a_full[st], use & 1)) {
                        fail();
                        break;
                    }
                    umma::tc_fence_after();
                    const uint32_t a0 = umma::smem_u32(smem + st * STAGE);
                    const uint32_t b0 = a0 + (uint32_t)(A_PIECE * T::NP);
                    constexpr int PA[3] = {0, 0, 1}, PB[3] = {0, 1, 0};
#pragma unroll
                    for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
                        for (int tt = 0; tt < NT; ++tt) {
                            const uint64_t ad = umma::sdesc(a0 + (uint32_t)(PA[tt] * A_PIECE) + ks * 256,
                                                            128, kRowB * 8);
                            const uint64_t bd = umma::sdesc(b0 + (uint32_t)(PB[tt] * B_PIECE) + ks * 256,
                                                            128, kRowB * 8);
                            const uint32_t acc = (kc > 0 || ks > 0 || tt > 0) ? 1u : 0u;
                            if constexpr (T::TF32) umma::mma_tf32(tmem + buf * 256, ad, bd, ID, acc);
                            else umma::mma_f16(tmem + buf * 256, ad, bd, ID, acc);
                        }
                    }
                    umma::mma_commit(&mma_done[st]);
                    if (kc == NK - 1) {
                        umma::mma_commit(&acc_full[buf]);
                        ++cbg;
                    }
                }
            } else if (warp == kCopyWarp && lane == 0) {
                // ---- the DFT-block copier: block c (= chunk c of the tile) into
                // the stage of chunk c as soon as the MMAs of chunk c - kStages are
                // done with it, so copies run up to kStages chunks ahead
                constexpr int NC = NCB * NK;
                for (int c = 0; c < NC && !*s_abort; ++c, ++g) {
                    const int st = (int)(g % kStages);
                    const uint32_t use = (uint32_t)(g / kStages);
                    if (use > 0 && !umma::mbar_wait(&mma_done[st], (use - 1) & 1)) { fail(); break; }
                    mbar_expect_tx(&b_full[st], B_BYTES);
                    bulk_g2s(smem + st * STAGE + A_PIECE * T::NP, tab + (size_t)c * B_BYTES, B_BYTES,
                             &b_full[st]);
                    ++copied;
                }
            }
        }
    }
    // copies started and never consumed (only after an abort) land before
    // the CTA may exit: the copier waits for its own copies
    if (warp == kCopyWarp && lane == 0) {
        const int64_t first = copied > kStages ? copied - kStages : 0;
        for (int64_t gg = first; gg < copied; ++gg)
            if (!umma::mbar_wait(&b_full[gg % kStages], (uint32_t)(gg / kStages) & 1)) atomicExch(err, 1);
    }
    // every MMA this CTA issued has finished before the tensor memory is freed
    if (warp == kIssuerWarp && lane == 0 && g > 0 && !*s_abort) {
        const int64_t gl = g - 1;
        if (!umma::mbar_wait(&mma_done[gl % kStages], (uint32_t)(gl / kStages) & 1)) atomicExch(err, 1);
    }
    umma::tc_fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, 512);
}

// ---- re-score of the candidates, theta and energy (one warp per pair) --------
template <typename ZT>
__device__ __forceinline__ cdf ld_df(const ZT* p, int64_t k) { return split_c(p[k]); }

__device__ __forceinline__ dfl shfl_df(dfl v, int off)
{
    return {__shfl_xor_sync(0xffffffffu, v.h, off), __shfl_xor_sync(0xffffffffu, v.l, off)};
}

// one pair's re-score by a whole warp: the best candidate shift, c(s*) and the
// energy in float-float (every lane ends with the same values)
struct Rescored {
    int s;
    dfl cre, cim, e;
};

template <int LOGN, typename ZT>
__device__ __forceinline__ Rescored rescore_pair(const ZT* __restrict__ z, int64_t i, int64_t j,
                                                 int64_t M, const uint16_t* __restrict__ cand,
                                                 int lane)
{
    constexpr int N = 1 << LOGN, R = N / 32;
    const int64_t ij = i * M + j;
    const ZT* zi = z + i * N;
    const ZT* zj = z + j * N;
    const uint4 cw = *reinterpret_cast<const uint4*>(cand + (size_t)ij * kCand);
    long long bkey = -1;
    int sbest = 0;
    cdf cbest{{0.f, 0.f}, {0.f, 0.f}};
    const int keep = (int)((cw.x >> 12) & 15u);
    auto cand_shift = [&](int c) {
        const uint32_t w = c < 2 ? cw.x : c < 4 ? cw.y : c < 6 ? cw.z : cw.w;
        return (int)((w >> (16 * (c & 1))) & 0xfffu) & (N - 1);
    };
    auto take = [&](const cdf& acc, int s) {
        const long long key = df_key(cnorm2(acc));
        if (key > bkey || (key == bkey && s < sbest)) { bkey = key; sbest = s; cbest = acc; }
    };
    bool done = false;
    if constexpr (std::is_same<ZT, float2>::value) {
        // complex64 inputs.  Each product a b is split on a fixed grid: the
        // running sum T <- fl(a b + T), started at T0 = 1.5 2^k, takes the
        // part of a b on the grid of ulp(T) exactly (T_new - T is exact by
        // Sterbenz's lemma, as |a b| < 2^(k-1) <= T / 2), and the remainder
        // fl(a b - (T_new - T)), at most half a grid step u = 2^(k-23), is
        // recovered by one FMA and summed in float32.  Cauchy-Schwarz bounds the
        // sum of |a b| over a correlation by |z_i| |z_j| <= 2^(k-1), so T stays
        // in [2^k, 2^(k+1)] and the lanes' grid parts add exactly; the
        // remainders' rounding errors are typically of order 2^(k-40) (at most
        // about 2^(k-30)).  Four float32 operations per product instead of the
        // ten of a float-float sum.
        float2 ui[R];
        float ni = 0.f, nj = 0.f;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            ui[r] = zi[lane + 32 * r];
            const float2 v = zj[lane + 32 * r];
            ni = __fmaf_rn(ui[r].x, ui[r].x, __fmaf_rn(ui[r].y, ui[r].y, ni));
            nj = __fmaf_rn(v.x, v.x, __fmaf_rn(v.y, v.y, nj));
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            ni += __shfl_xor_sync(0xffffffffu, ni, off);
            nj += __shfl_xor_sync(0xffffffffu, nj, off);
        }
        // 4 |z_i| |z_j| (float32 rounding of the norms is far inside the
        // factor 2 of headroom); 2^k <= q < 2^(k+1)
        const float q = __fmul_rn(4.0f, __fmul_rn(__fsqrt_rn(ni), __fsqrt_rn(nj)));
        if (q >= 0x1p-60f && q <= 0x1p+100f) {
            const float T0 = __uint_as_float((__float_as_uint(q) & 0x7f800000u) | 0x00400000u);
#pragma unroll 1
            for (int c = 0; c < keep; ++c) {
                const int s = cand_shift(c);
                float tr = T0, ti = T0, lr = 0.f, li = 0.f;
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float2 v = zj[(lane + 32 * r + s) & (N - 1)];
                    const float2 a = ui[r];
                    float t = __fmaf_rn(a.x, v.x, tr);
                    lr = __fadd_rn(lr, __fmaf_rn(a.x, v.x, __fsub_rn(tr, t)));
                    tr = t;
                    t = __fmaf_rn(a.y, v.y, tr);
                    lr = __fadd_rn(lr, __fmaf_rn(a.y, v.y, __fsub_rn(tr, t)));
                    tr = t;
                    t = __fmaf_rn(a.y, v.x, ti);
                    li = __fadd_rn(li, __fmaf_rn(a.y, v.x, __fsub_rn(ti, t)));
                    ti = t;
                    t = __fmaf_rn(-a.x, v.y, ti);
                    li = __fadd_rn(li, __fmaf_rn(-a.x, v.y, __fsub_rn(ti, t)));
                    ti = t;
                }
                float gr = __fsub_rn(tr, T0), gi = __fsub_rn(ti, T0);  // exact
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) {
                    gr = __fadd_rn(gr, __shfl_xor_sync(0xffffffffu, gr, off));  // exact
                    gi = __fadd_rn(gi, __shfl_xor_sync(0xffffffffu, gi, off));  // exact
                    lr = __fadd_rn(lr, __shfl_xor_sync(0xffffffffu, lr, off));
                    li = __fadd_rn(li, __shfl_xor_sync(0xffffffffu, li, off));
                }
                take(cdf{two_sum(gr, lr), two_sum(gi, li)}, s);
            }
            done = true;
        }
    }
    if (!done) {
        // any input, any scale: products and sums in float-float
#pragma unroll 1
        for (int c = 0; c < keep; ++c) {
            const int s = cand_shift(c);
            cdf acc{{0.f, 0.f}, {0.f, 0.f}};
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const cdf b = ld_df(zj, (lane + 32 * r + s) & (N - 1));
                // a conj(b)
                const cdf ar = ld_df(zi, lane + 32 * r);
                acc.re = df_add(acc.re, df_dot2<+1>(ar.re, b.re, ar.im, b.im));
                acc.im = df_add(acc.im, df_dot2<-1>(ar.im, b.re, ar.re, b.im));
            }
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                acc.re = df_add(acc.re, shfl_df(acc.re, off));
                acc.im = df_add(acc.im, shfl_df(acc.im, off));
            }
            take(acc, s);
        }
    }
    // the rotation e^{i theta} = c / |c| in float-float (every lane holds the
    // reduced c(s*); FP64 only for theta itself, on one lane below)
    dfl rx{1.f, 0.f}, ry{0.f, 0.f};
    {
        const dfl n2 = cnorm2(cbest);
        if (n2.h > 0.f) {
            const float s0 = __fsqrt_rn(n2.h);
            const float pp = __fmul_rn(s0, s0), pe = __fmaf_rn(s0, s0, -pp);
            const float res = __fadd_rn(__fsub_rn(__fsub_rn(n2.h, pp), pe), n2.l);
            const dfl r = fast_two_sum(s0, __fmul_rn(res, __fdiv_rn(0.5f, s0)));  // |c|
            const float r0 = __fdiv_rn(1.0f, r.h);
            const float q = __fmul_rn(r.h, r0), qe = __fmaf_rn(r.h, r0, -q);
            const float e1 = __fsub_rn(__fsub_rn(1.0f, q), __fmaf_rn(r.l, r0, qe));
            const dfl inv = fast_two_sum(r0, __fmul_rn(r0, e1));  // 1/|c|
            rx = df_mul(cbest.re, inv);
            ry = df_mul(cbest.im, inv);
        }
    }
    // energy h sum_k |z_i[k] - e^{i theta} z_j[k + s*]|^2 in float-float
    dfl e{0.f, 0.f};
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const cdf b = ld_df(zj, (lane + 32 * r + sbest) & (N - 1));
        const dfl bxr = df_dot2<-1>(rx, b.re, ry, b.im);  // Re(e^{i theta} b)
        const dfl byr = df_dot2<+1>(ry, b.re, rx, b.im);  // Im(e^{i theta} b)
        const cdf ar = ld_df(zi, lane + 32 * r);
        const dfl dx = df_sub(ar.re, bxr), dy = df_sub(ar.im, byr);
        e = df_add(e, df_dot2<+1>(dx, dx, dy, dy));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) e = df_add(e, shfl_df(e, off));
    Rescored out;
    out.s = sbest;
    out.cre = cbest.re;
    out.cim = cbest.im;
    out.e = e;
    return out;
}

// One warp per pair: the re-score in float-float by all lanes, then theta
// (FP64 atan2) and the outputs by lane 0.  (Handing each lane a different
// pair's FP64 finish, 32 pairs per warp, measured slower: fewer warps in
// flight for the FP32 work that dominates.)
template <int LOGN, typename ZT>
__global__ void __launch_bounds__(256)
    tc_rescore_kernel(const ZT* __restrict__ z, int64_t M, const uint16_t* __restrict__ cand,
                      const int8_t* __restrict__ cstatus, const int* __restrict__ err,
                      int32_t* __restrict__ shift, double* __restrict__ theta,
                      double* __restrict__ energy)
{
    constexpr int N = 1 << LOGN;
    const int lane = threadIdx.x & 31;
    const int64_t npairs = M * (M - 1) / 2;
    const int64_t q = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (q >= npairs) return;
    int64_t i, j;
    {
        const float a = (float)(2 * M - 1);
        int64_t e = (int64_t)floorf(0.5f * (a - sqrtf(fmaxf(a * a - 8.0f * (float)q, 0.f))));
        e = max((int64_t)0, min(e, M - 2));
        while (e > 0 && tri_start_tc(e, M) > q) --e;
        while (e < M - 2 && tri_start_tc(e + 1, M) <= q) ++e;
        i = e;
        j = q - tri_start_tc(i, M) + i + 1;
    }
    const int64_t ij = i * M + j, ji = j * M + i;
    if (cstatus[i] != FA_STATUS_OK || cstatus[j] != FA_STATUS_OK || *err) {
        if (lane == 0) {
            const double qn = __longlong_as_double(0x7ff8000000000000LL);
            shift[ij] = shift[ji] = -1;
            theta[ij] = theta[ji] = qn;
            energy[ij] = energy[ji] = qn;
        }
        return;
    }
    const Rescored r = rescore_pair<LOGN, ZT>(z, i, j, M, cand, lane);
    if (lane == 0) {
        const double cx = (double)r.cre.h + (double)r.cre.l;
        const double cy = (double)r.cim.h + (double)r.cim.l;
        const double th = atan2(cy, cx);
        const double en = ((double)r.e.h + (double)r.e.l) * (1.0 / N);
        shift[ij] = r.s;
        theta[ij] = th;
        energy[ij] = en;
        shift[ji] = r.s ? N - r.s : 0;
        theta[ji] = (th == 3.141592653589793) ? th : -th;
        energy[ji] = en;
    }
}

struct TcLayout {
    size_t spec64, spec32, tab, cand, ctrl, total;
};

template <int V, int LOGN>
TcLayout tc_layout(int64_t M)
{
    using T = TcVar<V>;
    constexpr int N = 1 << LOGN, KC = kRowB / T::ES, NK = 2 * N / KC;
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    TcLayout L;
    size_t o = 0;
    L.spec64 = o; o = al(o + (size_t)M * N * sizeof(double2));
    L.spec32 = o; o = al(o + (size_t)M * N * sizeof(float2));
    L.tab = o; o = al(o + (size_t)(N / 128) * NK * 256 * kRowB * T::NP);
    L.cand = o; o = al(o + (size_t)M * M * kCand * sizeof(uint16_t));
    L.ctrl = o; o += 256;
    L.total = o;
    return L;
}

template <int V, int LOGN, typename ZT>
int launch_tc(const fa_handle* h, const void* z, int64_t M, void* ws, int8_t* status,
              int32_t* shift, double* theta, double* energy, cudaStream_t st)
{
    using T = TcVar<V>;
    constexpr int N = 1 << LOGN, KC = kRowB / T::ES, NK = 2 * N / KC;
    const TcLayout L = tc_layout<V, LOGN>(M);
    uint8_t* base = static_cast<uint8_t*>(ws);
    double2* spec64 = reinterpret_cast<double2*>(base + L.spec64);
    float2* spec32 = reinterpret_cast<float2*>(base + L.spec32);
    uint8_t* tab = base + L.tab;
    uint16_t* cand = reinterpret_cast<uint16_t*>(base + L.cand);
    unsigned long long* next = reinterpret_cast<unsigned long long*>(base + L.ctrl);
    int* err = reinterpret_cast<int*>(base + L.ctrl + 8);
    int rc = launch_spectra(h, z, M, LOGN, std::is_same<ZT, float2>::value ? FA_Z_F32 : FA_Z_F64,
                            spec64, status, shift, theta, energy, st);
    if (rc != FA_OK) return rc;
    if (M < 2) return FA_OK;
    cudaError_t e = cudaMemsetAsync(base + L.ctrl, 0, 16, st);
    if (e != cudaSuccess) return cuda_error(e, "all-pairs tc: memset");
    const int64_t ns = M * N;
    spec32_kernel<LOGN><<<(unsigned)((ns + 255) / 256), 256, 0, st>>>(spec64, ns, spec32);
    const int64_t ntab = (int64_t)(N / 128) * NK * 256 * KC;
    dft_tab_kernel<V, LOGN><<<(unsigned)((ntab + 255) / 256), 256, 0, st>>>(tab);
    rc = cuda_error(cudaGetLastError(), "all-pairs tc: setup launch");
    if (rc != FA_OK) return rc;
    constexpr size_t STAGE = (size_t)(128 + 256) * kRowB * T::NP;
    const size_t smem = kStages * STAGE + (size_t)N * 8 + (3 * kStages + 6) * 8 + 48 +
                        (size_t)4 * 32 * 33 * sizeof(float);
    auto kern = tc_search_kernel<V, LOGN>;
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "all-pairs tc: cudaFuncSetAttribute");
    const int64_t tiles = ceil_sum128(M - 1);
    const int grid = (int)std::min<int64_t>(tiles, (int64_t)(h->num_sms > 0 ? h->num_sms : 1));
    kern<<<grid, kTcThreads, smem, st>>>(spec32, M, tab, cand, next, err);
    rc = cuda_error(cudaGetLastError(), "all-pairs tc: search launch");
    if (rc != FA_OK) return rc;
    const int64_t npairs = M * (M - 1) / 2;
    tc_rescore_kernel<LOGN, ZT><<<(unsigned)((npairs * 32 + 255) / 256), 256, 0, st>>>(
        static_cast<const ZT*>(z), M, cand, status, err, shift, theta, energy);
    return cuda_error(cudaGetLastError(), "all-pairs tc: rescore launch");
}

template <int V, typename ZT>
int dispatch_tc(const fa_handle* h, const void* z, int64_t M, int logn, void* ws, int8_t* status,
                int32_t* shift, double* theta, double* energy, cudaStream_t st)
{
    switch (logn) {
    case 8: return launch_tc<V, 8, ZT>(h, z, M, ws, status, shift, theta, energy, st);
    case 9: return launch_tc<V, 9, ZT>(h, z, M, ws, status, shift, theta, energy, st);
    }
    return set_error(FA_ERR_UNSUPPORTED, "fa_align_all_pairs: the tensor-core search needs N = 256 or 512");
}

template <int V>
int dispatch_tc_z(const fa_handle* h, const void* z, int64_t M, int logn, int ztype, void* ws,
                  int8_t* status, int32_t* shift, double* theta, double* energy, cudaStream_t st)
{
    if (ztype == FA_Z_F64)
        return dispatch_tc<V, double2>(h, z, M, logn, ws, status, shift, theta, energy, st);
    return dispatch_tc<V, float2>(h, z, M, logn, ws, status, shift, theta, energy, st);
}

}  // namespace

size_t align_all_tc_ws_bytes(int64_t M, int logn, int prec)
{
    auto pick = [&](auto v) -> size_t {
        constexpr int V = decltype(v)::value;
        if (logn == 8) return tc_layout<V, 8>(M).total;
        if (logn == 9) return tc_layout<V, 9>(M).total;
        return 0;
    };
    switch (prec) {
    case FA_PREC_TC_BF16X3: return pick(std::integral_constant<int, FA_PREC_TC_BF16X3>{});
    case FA_PREC_TC_FP16X3: return pick(std::integral_constant<int, FA_PREC_TC_FP16X3>{});
    case FA_PREC_TC_TF32: return pick(std::integral_constant<int, FA_PREC_TC_TF32>{});
    case FA_PREC_TC_TF32X3: return pick(std::integral_constant<int, FA_PREC_TC_TF32X3>{});
    }
    return 0;
}

int launch_align_all_tc(const fa_handle* h, const void* z, int64_t M, int logn, int ztype, int prec,
                        void* ws, int8_t* status, int32_t* shift, double* theta, double* energy,
                        cudaStream_t st)
{
    if (M == 0) return FA_OK;
    switch (prec) {
    case FA_PREC_TC_BF16X3:
        return dispatch_tc_z<FA_PREC_TC_BF16X3>(h, z, M, logn, ztype, ws, status, shift, theta, energy, st);
    case FA_PREC_TC_FP16X3:
        return dispatch_tc_z<FA_PREC_TC_FP16X3>(h, z, M, logn, ztype, ws, status, shift, theta, energy, st);
    case FA_PREC_TC_TF32:
        return dispatch_tc_z<FA_PREC_TC_TF32>(h, z, M, logn, ztype, ws, status, shift, theta, energy, st);
    case FA_PREC_TC_TF32X3:
        return dispatch_tc_z<FA_PREC_TC_TF32X3>(h, z, M, logn, ztype, ws, status, shift, theta, energy, st);
    }
    return set_error(FA_ERR_INVALID_ARG, "fa_align_all_pairs: unknown precision");
}

}  // namespace fa
