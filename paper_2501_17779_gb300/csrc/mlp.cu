// mlp.cu -- the k-NN candidate-pruning network and the retrieval helpers.
//
// Not part of the paper: Sec. 3 computes elastic distances; pruning the
// candidates of a k-NN query by a learned embedding of rotation- and
// shift-invariant Fourier magnitudes is this library's addition, with the
// exact elastic distance as its fallback and as the measure of its recall.
//
// Network 64 -> 256 -> 256 -> 64 (ReLU, ReLU, linear); weights used in
// bfloat16 (float32 master copies for Adam), biases, activations and
// accumulation in float32.  Every layer product (forward, back-propagated
// gradients, weight gradients) runs on the tensor cores (tc_gemm_kernel:
// tcgen05.mma from shared-memory descriptors, float32 accumulators in tensor
// memory, float32 operands as three bfloat16 pieces) with the bias/ReLU/mask
// epilogues fused; weight gradients reduce over the batch with a
// deterministic split-K.
//
// Retrieval: squared embedding distances (a tiled SIMT kernel with a
// subtract-square inner step, also used for the bias gradients' column sums),
// and a per-row radix selection of the k
// smallest keys (8-bit digits over the order-preserving bit pattern, ordered
// compaction, bitonic sort of the k survivors by (key, position)).
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <vector>

#include <type_traits>

#include "cta_ops.cuh"
#include "fa_internal.cuh"
#include "fft_stages.cuh"
#include "umma.cuh"

struct fa_mlp {
    fa_handle* h = nullptr;
    float* p = nullptr;           // float32 master parameters (flat)
    __nv_bfloat16* pb = nullptr;  // bfloat16 copy used by the layers
    float* m = nullptr;           // Adam moments
    float* v = nullptr;
    float* g = nullptr;           // gradient of the last fa_mlp_pair_grad
    int64_t t = 0;                // Adam step count
    void* ws = nullptr;           // activations and split-K partials
    size_t ws_bytes = 0;
    int* tc_err = nullptr;        // set by a tensor-core GEMM whose wait timed out
};

namespace fa {

// parameter layout (flat, row-major): W1 [256][64], b1 [256], W2 [256][256],
// b2 [256], W3 [64][256], b3 [64]
constexpr int kDin = 64, kDh = 256, kDout = 64;
constexpr int64_t kOffW1 = 0, kOffB1 = kOffW1 + kDh * kDin, kOffW2 = kOffB1 + kDh,
                  kOffB2 = kOffW2 + kDh * kDh, kOffW3 = kOffB2 + kDh,
                  kOffB3 = kOffW3 + kDout * kDh, kNParams = kOffB3 + kDout;

namespace {

__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }

enum { OP_MUL = 0, OP_SQDIFF = 1 };
enum { EPI_NONE = 0, EPI_BIAS_RELU = 1, EPI_BIAS = 2, EPI_MASK = 3 };

template <typename TA, typename TB>
struct GemmArgs {
    int64_t M, N, K, kc;      // kc: k range per split (blockIdx.z)
    const TA* A;
    int64_t sam, sak;
    const TB* B;
    int64_t sbk, sbn;
    float* C;                 // [splits][M][N] when split, else [M][N] with scm, scn
    int64_t scm, scn;
    const float* bias;        // [N]
    const float* mask;        // [M][N] (scm, scn strides)
};

// C(m, n) = sum_k op(A(m, k), B(k, n)) + epilogue
template <typename TA, typename TB, int OP, int EPI>
__global__ void __launch_bounds__(256) gemm_kernel(const __grid_constant__ GemmArgs<TA, TB> g)
{
    constexpr int BM = 64, BN = 64, BK = 16;
    __shared__ float As[BK][BM + 4];
    __shared__ float Bs[BK][BN + 4];
    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
    const int64_t kb = (int64_t)blockIdx.z * g.kc;
    const int64_t ke = kb + g.kc < g.K ? kb + g.kc : g.K;
    float acc[4][4] = {};
    for (int64_t k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            const int e = tid + r * 256;
            const int mm = e >> 4, kk = e & 15;
            const int64_t m = m0 + mm, k = k0 + kk;
            As[kk][mm] = (m < g.M && k < ke) ? to_f(g.A[m * g.sam + k * g.sak]) : 0.0f;
            const int kk2 = e >> 6, nn = e & 63;
            const int64_t k2 = k0 + kk2, n = n0 + nn;
            Bs[kk2][nn] = (k2 < ke && n < g.N) ? to_f(g.B[k2 * g.sbk + n * g.sbn]) : 0.0f;
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) a[i] = As[kk][ty * 4 + i];
#pragma unroll
            for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx * 4 + j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    if constexpr (OP == OP_MUL) {
                        acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
                    } else {
                        const float d = a[i] - b[j];
                        acc[i][j] = fmaf(d, d, acc[i][j]);
                    }
                }
        }
        __syncthreads();
    }
    float* C = g.C + (int64_t)blockIdx.z * g.M * g.N;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int64_t m = m0 + ty * 4 + i;
        if (m >= g.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int64_t n = n0 + tx * 4 + j;
            if (n >= g.N) continue;
            float v = acc[i][j];
            if constexpr (EPI == EPI_BIAS_RELU) v = fmaxf(v + g.bias[n], 0.0f);
            if constexpr (EPI == EPI_BIAS) v += g.bias[n];
            if constexpr (EPI == EPI_MASK) v = g.mask[m * g.scm + n * g.scn] > 0.0f ? v : 0.0f;
            C[m * g.scm + n * g.scn] = v;
        }
    }
}

// ---- the same products on the tensor cores (tcgen05) ------------------------
// C(m, n) = sum_k A(m, k) B(k, n) + epilogue, A float32, B bfloat16 (the
// weights, exact) or float32.  float32 operands enter as three bfloat16
// pieces (hi + mid + lo = the float exactly), bfloat16 weights as one; the
// MMAs take the piece products that matter at float32 precision (hi hi, hi
// mid, mid hi, hi lo, mid mid, lo hi for two float operands: the dropped ones
// are below 2^-25 of the product) and accumulate in float32 in tensor memory.
// One CTA of 128 threads per 128-row tile and split (blockIdx.z), the whole N
// (64 or 256 columns) in one accumulator; the K range in chunks of 32, two
// shared-memory stages: all threads convert and store chunk c + 1 while the
// tensor core multiplies chunk c.  Thread 0 issues the MMAs; a commit per
// chunk arrives on that stage's mbarrier, which the threads wait on (bounded)
// before they overwrite the stage.  Epilogue: warp w reads accumulator lanes
// 32w..32w+31 (its rows), 32 columns at a time.
constexpr int kTcThreads = 128;
constexpr int kTcKC = 32;  // K chunk (elements)

template <typename TB>
__host__ __device__ constexpr int tc_bpieces() { return std::is_same<TB, float>::value ? 3 : 1; }

template <int NT, typename TB>
__host__ __device__ constexpr size_t tc_smem_bytes()
{
    return 2 * (size_t)(3 * 128 + tc_bpieces<TB>() * NT) * kTcKC * 2 + 64;
}

__device__ __forceinline__ void tc_store_pieces(uint8_t* base, size_t piece_bytes, int r, int k,
                                                float x, int npieces)
{
    const uint32_t off = umma::tile_off(r, 2 * k, 2 * kTcKC);
    if (npieces == 1) {
        *reinterpret_cast<uint16_t*>(base + off) = __bfloat16_as_ushort(__float2bfloat16_rn(x));
        return;
    }
    uint16_t h, m, l;
    umma::split3_bf16(x, h, m, l);
    *reinterpret_cast<uint16_t*>(base + off) = h;
    *reinterpret_cast<uint16_t*>(base + piece_bytes + off) = m;
    *reinterpret_cast<uint16_t*>(base + 2 * piece_bytes + off) = l;
}

template <typename TB, int NT, int EPI>
__global__ void __launch_bounds__(kTcThreads, 1)
    tc_gemm_kernel(const __grid_constant__ GemmArgs<float, TB> g, int* __restrict__ err)
{
    constexpr int BP = tc_bpieces<TB>();
    constexpr int NTERMS = BP == 3 ? 6 : 3;
    constexpr size_t A_PIECE = (size_t)128 * kTcKC * 2, B_PIECE = (size_t)NT * kTcKC * 2;
    constexpr size_t STAGE = 3 * A_PIECE + BP * B_PIECE;
    constexpr uint32_t TCOLS = NT < 32 ? 32 : NT;
    constexpr uint32_t ID = umma::idesc(128, NT, umma::kFmtBF16);
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + 2 * STAGE);
    uint32_t* s_taddr = reinterpret_cast<uint32_t*>(smem + 2 * STAGE + 16);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int64_t m0 = (int64_t)blockIdx.x * 128, n0 = (int64_t)blockIdx.y * NT;
    const int64_t kb = (int64_t)blockIdx.z * g.kc;
    const int64_t ke = kb + g.kc < g.K ? kb + g.kc : g.K;
    const int nchunks = ke > kb ? (int)((ke - kb + kTcKC - 1) / kTcKC) : 0;

    if (tid == 0) {
        umma::mbar_init(&mbar[0], 1);
        umma::mbar_init(&mbar[1], 1);
        umma::fence_mbar_init();
    }
    if (warp == 0) umma::tmem_alloc(s_taddr, TCOLS);
    umma::tc_fence_before();
    __syncthreads();
    umma::tc_fence_after();
    const uint32_t tmem = *s_taddr;
    bool ok = true;

    for (int c = 0; c < nchunks && ok; ++c) {
        const int st = c & 1;
        uint8_t* sa = smem + st * STAGE;
        uint8_t* sb = sa + 3 * A_PIECE;
        // the stage's previous MMAs (chunk c - 2) must be done before it is
        // overwritten; every thread waits, and all agree on the outcome
        if (c >= 2) ok = __syncthreads_and(umma::mbar_wait(&mbar[st], ((c - 2) >> 1) & 1) ? 1 : 0);
        if (!ok) break;
        const int64_t k0 = kb + (int64_t)c * kTcKC;
        // A chunk: 128 rows x 32 k.  Row-major A: eight consecutive k per task,
        // two float4 loads and one 16-byte store per piece; otherwise one
        // element per task, the unit-stride index fastest (coalesced).
        if (g.sak == 1) {
            for (int e = tid; e < 128 * (kTcKC / 8); e += kTcThreads) {
                const int r = e / (kTcKC / 8), kg = e % (kTcKC / 8);
                const int64_t m = m0 + r, kk = k0 + kg * 8;
                float x[8];
                const float* src = g.A + m * g.sam + kk;
                if (m < g.M && kk + 8 <= ke && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
                    const float4 u = *reinterpret_cast<const float4*>(src);
                    const float4 v = *reinterpret_cast<const float4*>(src + 4);
                    x[0] = u.x; x[1] = u.y; x[2] = u.z; x[3] = u.w;
                    x[4] = v.x; x[5] = v.y; x[6] = v.z; x[7] = v.w;
                } else {
#pragma unroll
                    for (int q = 0; q < 8; ++q) x[q] = (m < g.M && kk + q < ke) ? src[q] : 0.0f;
                }
                uint16_t h[8], md[8], l[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) umma::split3_bf16(x[q], h[q], md[q], l[q]);
                const uint32_t off = umma::tile_off(r, kg * 16, 2 * kTcKC);
                auto pack = [](const uint16_t* v) {
                    return make_uint4(v[0] | ((uint32_t)v[1] << 16), v[2] | ((uint32_t)v[3] << 16),
                                      v[4] | ((uint32_t)v[5] << 16), v[6] | ((uint32_t)v[7] << 16));
                };
                *reinterpret_cast<uint4*>(sa + off) = pack(h);
                *reinterpret_cast<uint4*>(sa + A_PIECE + off) = pack(md);
                *reinterpret_cast<uint4*>(sa + 2 * A_PIECE + off) = pack(l);
            }
        } else {
            for (int e = tid; e < 128 * kTcKC; e += kTcThreads) {
                const int r = e % 128, k = e / 128;
                const int64_t m = m0 + r, kk = k0 + k;
                const float x = (m < g.M && kk < ke) ? g.A[m * g.sam + kk * g.sak] : 0.0f;
                tc_store_pieces(sa, A_PIECE, r, k, x, 3);
            }
        }
        // B chunk: NT rows (n) x 32 k.  bfloat16 weights stored with k
        // contiguous: eight at a time, copied as they are (one piece)
        if (BP == 1 && g.sbk == 1) {
            for (int e = tid; e < NT * (kTcKC / 8); e += kTcThreads) {
                const int n = e / (kTcKC / 8), kg = e % (kTcKC / 8);
                const int64_t nn = n0 + n, kk = k0 + kg * 8;
                const TB* src = g.B + kk + nn * g.sbn;
                uint4 v = make_uint4(0u, 0u, 0u, 0u);
                if (nn < g.N && kk + 8 <= ke && (reinterpret_cast<uintptr_t>(src) & 15) == 0) {
                    v = *reinterpret_cast<const uint4*>(src);
                } else {
                    uint16_t t[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        t[q] = (nn < g.N && kk + q < ke)
                                   ? __bfloat16_as_ushort(__float2bfloat16_rn(to_f(src[q])))
                                   : (uint16_t)0;
                    v = make_uint4(t[0] | ((uint32_t)t[1] << 16), t[2] | ((uint32_t)t[3] << 16),
                                   t[4] | ((uint32_t)t[5] << 16), t[6] | ((uint32_t)t[7] << 16));
                }
                *reinterpret_cast<uint4*>(sb + umma::tile_off(n, kg * 16, 2 * kTcKC)) = v;
            }
        } else {
            for (int e = tid; e < NT * kTcKC; e += kTcThreads) {
                int n, k;
                if (g.sbk == 1) { n = e / kTcKC; k = e % kTcKC; } else { n = e % NT; k = e / NT; }
                const int64_t nn = n0 + n, kk = k0 + k;
                const float x = (nn < g.N && kk < ke) ? to_f(g.B[kk * g.sbk + nn * g.sbn]) : 0.0f;
                tc_store_pieces(sb, B_PIECE, n, k, x, BP);
            }
        }
        umma::fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            umma::tc_fence_after();
            const uint32_t a0 = umma::smem_u32(sa), b0 = umma::smem_u32(sb);
            constexpr int TA_[6] = {0, 0, 1, 0, 1, 2}, TB_[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
            for (int ks = 0; ks < kTcKC / 16; ++ks) {
#pragma unroll
                for (int t = 0; t < NTERMS; ++t) {
                    const int pa = BP == 3 ? TA_[t] : t, pb = BP == 3 ? TB_[t] : 0;
                    const uint64_t ad = umma::sdesc(a0 + (uint32_t)(pa * A_PIECE) + ks * 256, 128,
                                                    kTcKC * 2 * 8);
                    const uint64_t bd = umma::sdesc(b0 + (uint32_t)(pb * B_PIECE) + ks * 256, 128,
                                                    kTcKC * 2 * 8);
                    umma::mma_f16(tmem, ad, bd, ID, (c > 0 || ks > 0 || t > 0) ? 1u : 0u);
                }
            }
            umma::mma_commit(&mbar[st]);
        }
    }
    if (ok && nchunks > 0)
        ok = __syncthreads_and(
                 umma::mbar_wait(&mbar[(nchunks - 1) & 1], ((nchunks - 1) >> 1) & 1) ? 1 : 0) != 0;
    umma::tc_fence_after();
    if (!ok) {
        if (tid == 0) atomicExch(err, 1);
    } else {
        float* C = g.C + (int64_t)blockIdx.z * g.M * g.N;
        const int64_t m = m0 + warp * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < NT; c0 += 32) {
            float v[32];
            if (nchunks > 0) {
                umma::tmem_ld32(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
            } else {
#pragma unroll
                for (int j = 0; j < 32; ++j) v[j] = 0.0f;
            }
            if (m < g.M) {
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int64_t n = n0 + c0 + j;
                    if (n >= g.N) continue;
                    float x = v[j];
                    if constexpr (EPI == EPI_BIAS_RELU) x = fmaxf(x + g.bias[n], 0.0f);
                    if constexpr (EPI == EPI_BIAS) x += g.bias[n];
                    if constexpr (EPI == EPI_MASK) x = g.mask[m * g.scm + n * g.scn] > 0.0f ? x : 0.0f;
                    C[m * g.scm + n * g.scn] = x;
                }
            }
        }
    }
    umma::tc_fence_before();
    __syncthreads();
    if (warp == 0) umma::tmem_dealloc(tmem, TCOLS);
}

template <typename TB, int NT, int EPI>
int tc_gemm(const GemmArgs<float, TB>& a, int splits, int* err, cudaStream_t st)
{
    if (a.M == 0 || a.N == 0) return FA_OK;
    GemmArgs<float, TB> g = a;
    g.kc = (a.K + splits - 1) / splits;
    g.kc = (g.kc + kTcKC - 1) / kTcKC * kTcKC;
    auto kern = tc_gemm_kernel<TB, NT, EPI>;
    constexpr size_t smem = tc_smem_bytes<NT, TB>();
    const cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)smem);
    if (e != cudaSuccess) return cuda_error(e, "tc_gemm: cudaFuncSetAttribute");
    const dim3 grid((unsigned)((a.M + 127) / 128), (unsigned)((a.N + NT - 1) / NT), (unsigned)splits);
    kern<<<grid, kTcThreads, smem, st>>>(g, err);
    return cuda_error(cudaGetLastError(), "tc_gemm launch");
}

template <typename TA, typename TB, int OP, int EPI>
int gemm(const GemmArgs<TA, TB>& a, int splits, cudaStream_t st)
{
    if (a.M == 0 || a.N == 0) return FA_OK;
    GemmArgs<TA, TB> g = a;
    g.kc = (a.K + splits - 1) / splits;
    g.kc = (g.kc + 15) / 16 * 16;
    const dim3 grid((unsigned)((a.N + 63) / 64), (unsigned)((a.M + 63) / 64), (unsigned)splits);
    gemm_kernel<TA, TB, OP, EPI><<<grid, 256, 0, st>>>(g);
    return cuda_error(cudaGetLastError(), "gemm launch");
}

// out[i] = sum_z part[z][i], z in order (deterministic)
__global__ void split_sum_kernel(const float* __restrict__ part, int splits, int64_t n,
                                 float* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.0f;
    for (int z = 0; z < splits; ++z) s += part[(int64_t)z * n + i];
    out[i] = s;
}

__global__ void gather_rows_kernel(const float* __restrict__ X, const int64_t* __restrict__ pi,
                                   const int64_t* __restrict__ pj, int64_t P, int64_t rows,
                                   float* __restrict__ Xp, int* __restrict__ bad)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= 2 * P * kDin) return;
    const int64_t r = e / kDin, c = e - r * kDin;
    int64_t src = r < P ? pi[r] : pj[r - P];
    if (src < 0 || src >= rows) { atomicOr(bad, 1); src = 0; }
    Xp[e] = X[src * kDin + c];
}

__global__ void fill_kernel(float* p, int64_t n, float v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}

// one warp per pair: loss term and dL/dy for both embeddings
__global__ void pair_loss_kernel(const float* __restrict__ Y, int64_t P, const float* __restrict__ d,
                                 float* __restrict__ gY, float* __restrict__ lossp)
{
    const int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (p >= P) return;
    const float* a = Y + p * kDout;
    const float* b = Y + (P + p) * kDout;
    const float d0 = a[lane] - b[lane], d1 = a[lane + 32] - b[lane + 32];
    float s = fmaf(d0, d0, d1 * d1);
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    const float r = sqrtf(s + 1e-12f);
    const float dd = d[p];
    const float w = 1.0f / ((dd + 0.05f) * (dd + 0.05f));
    const float e = r - dd;
    const float coef = (2.0f / (float)P) * w * e / r;
    gY[p * kDout + lane] = coef * d0;
    gY[p * kDout + lane + 32] = coef * d1;
    gY[(P + p) * kDout + lane] = -coef * d0;
    gY[(P + p) * kDout + lane + 32] = -coef * d1;
    if (lane == 0) lossp[p] = w * e * e;
}

// mean of n values by one CTA (fixed order: strided partials, tree)
__global__ void mean_kernel(const float* __restrict__ x, int64_t n, float* __restrict__ out)
{
    __shared__ float part[256];
    float s = 0.0f;
    for (int64_t i = threadIdx.x; i < n; i += 256) s += x[i];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = part[0] / (float)n;
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, __nv_bfloat16* __restrict__ pb, int64_t n,
                            float lr, float bc1, float bc2)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = 0.9f * m[i] + 0.1f * gi;
    const float vi = 0.999f * v[i] + 0.001f * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
    p[i] = pi;
    pb[i] = __float2bfloat16_rn(pi);
}

__global__ void to_bf16_kernel(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) pb[i] = __float2bfloat16_rn(p[i]);
}

// ------------------------------------------------------------ descriptors --
// log |Z[f]|, Z = DFT(z)/N, f = 1..F then -1..-F, one CTA per curve
template <int T, int NMAX>
__global__ void __launch_bounds__(T) descriptor_kernel(const double2* __restrict__ z, int64_t M,
                                                       int N, int logn, int F,
                                                       const double2* __restrict__ tf,
                                                       float* __restrict__ out)
{
    extern __shared__ __align__(16) double2 X[];
    const int64_t c = blockIdx.x;
    for (int k = threadIdx.x; k < N; k += T) X[k] = z[c * N + k];
    __syncthreads();
    fft_rt<T, NMAX>(X, logn, tf);
    for (int e = threadIdx.x; e < 2 * F; e += T) {
        const int f = e < F ? e + 1 : N - (e - F + 1);
        const double2 v = X[f];
        const double mag = sqrt(v.x * v.x + v.y * v.y) / (double)N;
        out[c * 2 * F + e] = (float)log(mag + 1e-30);
    }
}

// per column: mean and 1/std (population) over M rows; one CTA per column
__global__ void column_stats_kernel(const float* __restrict__ X, int64_t M, int D,
                                    float* __restrict__ mean, float* __restrict__ inv_std)
{
    __shared__ double part[256];
    const int col = blockIdx.x;
    double s = 0.0;
    for (int64_t r = threadIdx.x; r < M; r += 256) s += X[r * D + col];
    part[threadIdx.x] = s;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    const double mu = part[0] / (double)M;
    __syncthreads();
    double q = 0.0;
    for (int64_t r = threadIdx.x; r < M; r += 256) {
        const double d = X[r * D + col] - mu;
        q += d * d;
    }
    part[threadIdx.x] = q;
    __syncthreads();
    for (int w = 128; w > 0; w >>= 1) {
        if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double var = part[0] / (double)M;
        mean[col] = (float)mu;
        inv_std[col] = var > 0.0 ? (float)(1.0 / sqrt(var)) : 1.0f;
    }
}

__global__ void standardize_kernel(float* __restrict__ X, int64_t M, int D,
                                   const float* __restrict__ mean, const float* __restrict__ inv_std)
{
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= M * D) return;
    const int c = (int)(e % D);
    X[e] = (X[e] - mean[c]) * inv_std[c];
}

// -------------------------------------------------------------- select k --
// order-preserving unsigned images of the keys (NaN sorts last)
__device__ __forceinline__ unsigned long long key_bits(float x)
{
    unsigned u = __float_as_uint(x);
    if ((u & 0x7fffffffu) > 0x7f800000u) return 0xffffffffull;
    u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    return u;
}
__device__ __forceinline__ unsigned long long key_bits(double x)
{
    unsigned long long u = (unsigned long long)__double_as_longlong(x);
    if ((u & 0x7fffffffffffffffull) > 0x7ff0000000000000ull) return ~0ull;
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}

template <int T>
__device__ __forceinline__ int block_excl_scan(int v, int* sw, int& total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, x, off);
        if (lane >= off) x += y;
    }
    if (lane == 31) sw[w] = x;
    __syncthreads();
    if (threadIdx.x == 0) {
        int run = 0;
        for (int i = 0; i < T / 32; ++i) { const int c = sw[i]; sw[i] = run; run += c; }
        sw[T / 32] = run;
    }
    __syncthreads();
    const int r = sw[w] + x - v;
    total = sw[T / 32];
    __syncthreads();
    return r;
}

// per row: positions of the k smallest keys, ascending by (key, position); k <= 256 <= T
template <typename K, int BITS>
__global__ void __launch_bounds__(256) select_k_kernel(const K* __restrict__ keys, int64_t C, int k,
                                                      int64_t* __restrict__ out_pos,
                                                      K* __restrict__ out_key)
{
    constexpr int T = 256;
    __shared__ unsigned hist[256];
    __shared__ unsigned long long s_want, s_mask;
    __shared__ int s_need;
    __shared__ int sw[T / 32 + 1];
    __shared__ unsigned long long ck[256];
    __shared__ long long cp[256];
    const K* kr = keys + (int64_t)blockIdx.x * C;
    unsigned long long want = 0, mask = 0;
    int need = k;  // rank (1-based) of the k-th smallest among the keys matching `want`
    for (int shift = BITS - 8; shift >= 0; shift -= 8) {
        hist[threadIdx.x] = 0;
        __syncthreads();
        for (int64_t i = threadIdx.x; i < C; i += T) {
            const unsigned long long u = key_bits(kr[i]);
            if ((u & mask) == want) atomicAdd(&hist[(u >> shift) & 255], 1u);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            unsigned cum = 0;
            int b = 0;
            for (; b < 255; ++b) {
                if (cum + hist[b] >= (unsigned)need) break;
                cum += hist[b];
            }
            s_need = need - (int)cum;
            s_want = want | ((unsigned long long)b << shift);
            s_mask = mask | (255ull << shift);
        }
        __syncthreads();
        want = s_want;
        mask = s_mask;
        need = s_need;
        __syncthreads();
    }
    // ordered compaction: every key below the k-th, then the first `need` equal to it
    int n_sel = 0, n_eq = 0;
    for (int64_t base = 0; base < C; base += T) {
        const int64_t i = base + threadIdx.x;
        unsigned long long u = 0;
        bool lt = false, eq = false;
        if (i < C) {
            u = key_bits(kr[i]);
            lt = u < want;
            eq = u == want;
        }
        int teq;
        const int req = block_excl_scan<T>(eq ? 1 : 0, sw, teq);
        const bool sel = lt || (eq && n_eq + req < need);
        int tsel;
        const int rs = block_excl_scan<T>(sel ? 1 : 0, sw, tsel);
        if (sel && n_sel + rs < 256) {
            ck[n_sel + rs] = u;
            cp[n_sel + rs] = i;
        }
        n_sel += tsel;
        n_eq += teq;
    }
    // bitonic sort of the k survivors by (key image, position); padding sorts last
    if (threadIdx.x >= k) { ck[threadIdx.x] = ~0ull; cp[threadIdx.x] = 0x7fffffffffffffffLL; }
    __syncthreads();
    for (int size = 2; size <= 256; size <<= 1)
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const int i = threadIdx.x, j = i ^ stride;
            if (j > i) {
                const bool up = (i & size) == 0;
                const unsigned long long ki = ck[i], kj = ck[j];
                const long long pi = cp[i], pj = cp[j];
                const bool gt = ki > kj || (ki == kj && pi > pj);
                if (gt == up) { ck[i] = kj; ck[j] = ki; cp[i] = pj; cp[j] = pi; }
            }
            __syncthreads();
        }
    if (threadIdx.x < k) {
        const long long p = cp[threadIdx.x];
        out_pos[(int64_t)blockIdx.x * k + threadIdx.x] = p;
        if (out_key) out_key[(int64_t)blockIdx.x * k + threadIdx.x] = kr[p];
    }
}

// host-side Gaussian initialisation (SplitMix64 + Box-Muller)
struct SplitMix {
    uint64_t s;
    uint64_t next()
    {
        uint64_t z = (s += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        return z ^ (z >> 31);
    }
    double uniform() { return ((next() >> 11) + 0.5) * (1.0 / 9007199254740992.0); }
    double normal()
    {
        const double u1 = uniform(), u2 = uniform();
        return std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2);
    }
};

int ensure_mlp_ws(fa_mlp* m, size_t need)
{
    if (m->ws_bytes >= need) return FA_OK;
    if (m->ws) cudaFree(m->ws);
    m->ws = nullptr;
    m->ws_bytes = 0;
    const cudaError_t e = cudaMalloc(&m->ws, need);
    if (e != cudaSuccess) return cuda_error(e, "fa_mlp workspace");
    m->ws_bytes = need;
    return FA_OK;
}

constexpr int kSplits = 64;

inline size_t al(size_t x) { return (x + 255) & ~size_t(255); }

int refresh_bf16(fa_mlp* m, cudaStream_t st)
{
    to_bf16_kernel<<<(unsigned)((kNParams + 255) / 256), 256, 0, st>>>(m->p, m->pb, kNParams);
    return cuda_error(cudaGetLastError(), "bf16 copy");
}

// forward of B rows of X into H1, H2, Y
int mlp_forward_into(const fa_mlp* m, const float* X, int64_t B, float* H1, float* H2, float* Y,
                     cudaStream_t st)
{
    using G = GemmArgs<float, __nv_bfloat16>;
    G g{};
    g.M = B; g.N = kDh; g.K = kDin; g.A = X; g.sam = kDin; g.sak = 1;
    g.B = m->pb + kOffW1; g.sbk = 1; g.sbn = kDin; g.C = H1; g.scm = kDh; g.scn = 1;
    g.bias = m->p + kOffB1;
    int rc = tc_gemm<__nv_bfloat16, 64, EPI_BIAS_RELU>(g, 1, m->tc_err, st);
    if (rc != FA_OK) return rc;
    g.K = kDh; g.A = H1; g.sam = kDh; g.B = m->pb + kOffW2; g.sbn = kDh; g.C = H2;
    g.bias = m->p + kOffB2;
    rc = tc_gemm<__nv_bfloat16, 64, EPI_BIAS_RELU>(g, 1, m->tc_err, st);
    if (rc != FA_OK) return rc;
    g.N = kDout; g.A = H2; g.B = m->pb + kOffW3; g.sbn = kDh; g.C = Y; g.scm = kDout;
    g.bias = m->p + kOffB3;
    return tc_gemm<__nv_bfloat16, 64, EPI_BIAS>(g, 1, m->tc_err, st);
}

// dW (out x in) = gH^T X over R rows, and db = column sums of gH, through the
// split-K partials in `part`
int weight_grad(const float* gH, int64_t R, int out, const float* X, int in, float* dW,
                float* db, const float* ones, float* part, int* tc_err, cudaStream_t st)
{
    GemmArgs<float, float> g{};
    g.M = out; g.N = in; g.K = R; g.A = gH; g.sam = 1; g.sak = out; g.B = X; g.sbk = in; g.sbn = 1;
    g.C = part; g.scm = in; g.scn = 1;
    int rc = tc_gemm<float, 64, EPI_NONE>(g, kSplits, tc_err, st);
    if (rc != FA_OK) return rc;
    split_sum_kernel<<<(unsigned)((out * in + 255) / 256), 256, 0, st>>>(part, kSplits,
                                                                        (int64_t)out * in, dW);
    rc = cuda_error(cudaGetLastError(), "split sum");
    if (rc != FA_OK) return rc;
    GemmArgs<float, float> b{};
    b.M = 1; b.N = out; b.K = R; b.A = ones; b.sam = 0; b.sak = 1; b.B = gH; b.sbk = out;
    b.sbn = 1; b.C = part; b.scm = out; b.scn = 1;
    rc = gemm<float, float, OP_MUL, EPI_NONE>(b, kSplits, st);
    if (rc != FA_OK) return rc;
    split_sum_kernel<<<(unsigned)((out + 255) / 256), 256, 0, st>>>(part, kSplits, out, db);
    return cuda_error(cudaGetLastError(), "split sum");
}

}  // namespace
}  // namespace fa

using namespace fa;

extern "C" {

int64_t fa_mlp_num_params(void) { return kNParams; }

int fa_mlp_create(fa_handle* h, uint64_t seed, fa_mlp** out)
{
    if (!h || !out) return set_error(FA_ERR_INVALID_ARG, "fa_mlp_create: null argument");
    *out = nullptr;
    DeviceGuard g(h->device);
    if (g.rc != FA_OK) return g.rc;
    fa_mlp* m = new fa_mlp();
    m->h = h;
    const size_t fb = sizeof(float) * kNParams;
    cudaError_t e = cudaMalloc(&m->p, fb);
    if (e == cudaSuccess) e = cudaMalloc(&m->m, fb);
    if (e == cudaSuccess) e = cudaMalloc(&m->v, fb);
    if (e == cudaSuccess) e = cudaMalloc(&m->g, fb);
    if (e == cudaSuccess) e = cudaMalloc(&m->pb, sizeof(__nv_bfloat16) * kNParams);
    if (e == cudaSuccess) e = cudaMalloc(&m->tc_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(m->tc_err, 0, sizeof(int));
    if (e != cudaSuccess) {
        fa_mlp_destroy(m);
        return cuda_error(e, "fa_mlp_create");
    }
    // He initialisation of the weights, zero biases
    std::vector<float> p(kNParams, 0.0f);
    SplitMix rng{seed};
    auto init = [&](int64_t off, int rows, int cols, double gain) {
        const double s = gain * std::sqrt(2.0 / cols);
        for (int64_t i = 0; i < (int64_t)rows * cols; ++i) p[off + i] = (float)(s * rng.normal());
    };
    init(kOffW1, kDh, kDin, 1.0);
    init(kOffW2, kDh, kDh, 1.0);
    // the output layer starts small: embedding distances of order 0.1, the
    // scale of the elastic distances they are trained on
    init(kOffW3, kDout, kDh, 0.01);
    *out = m;
    return fa_mlp_set_params(m, p.data());
}

int fa_mlp_destroy(fa_mlp* m)
{
    if (!m) return FA_OK;
    DeviceGuard g(m->h->device);
    cudaFree(m->p); cudaFree(m->m); cudaFree(m->v); cudaFree(m->g); cudaFree(m->pb);
    cudaFree(m->tc_err);
    if (m->ws) cudaFree(m->ws);
    delete m;
    return FA_OK;
}

int fa_mlp_set_params(fa_mlp* m, const float* params)
{
    if (!m || !params) return set_error(FA_ERR_INVALID_ARG, "fa_mlp_set_params: null argument");
    DeviceGuard g(m->h->device);
    if (g.rc != FA_OK) return g.rc;
    const size_t fb = sizeof(float) * kNParams;
    cudaError_t e = cudaMemcpy(m->p, params, fb, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemset(m->m, 0, fb);
    if (e == cudaSuccess) e = cudaMemset(m->v, 0, fb);
    if (e == cudaSuccess) e = cudaMemset(m->g, 0, fb);
    if (e != cudaSuccess) return cuda_error(e, "fa_mlp_set_params");
    m->t = 0;
    const int rc = refresh_bf16(m, 0);
    if (rc != FA_OK) return rc;
    return cuda_error(cudaDeviceSynchronize(), "fa_mlp_set_params");
}

int fa_mlp_get_params(fa_mlp* m, float* params)
{
    if (!m || !params) return set_error(FA_ERR_INVALID_ARG, "fa_mlp_get_params: null argument");
    DeviceGuard g(m->h->device);
    if (g.rc != FA_OK) return g.rc;
    return cuda_error(cudaMemcpy(params, m->p, sizeof(float) * kNParams, cudaMemcpyDeviceToHost),
                      "fa_mlp_get_params");
}

int fa_mlp_forward(fa_mlp* m, const float* X, int64_t B, float* Y, void* stream)
{
    if (!m) return set_error(FA_ERR_INVALID_ARG, "fa_mlp_forward: null handle");
    if (B < 0) return set_error(FA_ERR_INVALID_ARG, "fa_mlp_forward: negative batch");
    if (B == 0) return FA_OK;
    if (B > (1 << 21)) return set_error(FA_ERR_UNSUPPORTED, "fa_mlp_forward: batch too large");
    if (!X || !Y) return set_error(FA_ERR_INVALID_ARG, "fa_mlp_forward: null pointer");
    DeviceGuard g(m->h->device);
    if (g.rc != FA_OK) return g.rc;
    const size_t need = 2 * al(sizeof(float) * (size_t)B * kDh);
    int rc = ensure_mlp_ws(m, need);
    if (rc != FA_OK) return rc;
    float* H1 = static_cast<float*>(m->ws);
    float* H2 = reinterpret_cast<float*>(static_cast<char*>(m->ws) + al(sizeof(float) * B * kDh));
    return mlp_forward_into(m, X, B, H1, H2, Y, static_cast<cudaStream_t>(stream));
}

int fa_mlp_pair_grad(fa_mlp* m, const float* X, int64_t rows, const int64_t* pi,
                     const int64_t* pj, const float* d, int64_t P, float* loss, float* grad,
                     void* stream)
{
    if (!m) return set_error(FA_ERR_INVALID_ARG, "fa_mlp_pair_grad: null handle");
    if (P <= 0 || rows <= 0)
        return set_error(FA_ERR_INVALID_ARG, "fa_mlp_pair_grad: empty batch");
    // the GEMM grid's second dimension holds 2P / 64 row tiles (<= 65535)
    if (P > (1 << 20)) return set_error(FA_ERR_UNSUPPORTED, "fa_mlp_pair_grad: batch too large");
    if (!X || !pi || !pj || !d || !loss)
        return set_error(FA_ERR_INVALID_ARG, "fa_mlp_pair_grad: null pointer");
    DeviceGuard dg(m->h->device);
    if (dg.rc != FA_OK) return dg.rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int64_t R = 2 * P;
    const size_t sx = al(sizeof(float) * R * kDin), sh = al(sizeof(float) * R * kDh),
                 so = al(sizeof(float) * R * kDout), sp = al(sizeof(float) * P),
                 sr = al(sizeof(float) * R), spart = al(sizeof(float) * kSplits * kDh * kDh);
    const size_t need = sx + 4 * sh + 2 * so + sp + sr + spart + 256;
    int rc = ensure_mlp_ws(m, need);
    if (rc != FA_OK) return rc;
    char* w = static_cast<char*>(m->ws);
    float* Xp = reinterpret_cast<float*>(w); w += sx;
    float* H1 = reinterpret_cast<float*>(w); w += sh;
    float* H2 = reinterpret_cast<float*>(w); w += sh;
    float* gH2 = reinterpret_cast<float*>(w); w += sh;
    float* gH1 = reinterpret_cast<float*>(w); w += sh;
    float* Y = reinterpret_cast<float*>(w); w += so;
    float* gY = reinterpret_cast<float*>(w); w += so;
    float* lp = reinterpret_cast<float*>(w); w += sp;
    float* ones = reinterpret_cast<float*>(w); w += sr;
    float* part = reinterpret_cast<float*>(w); w += spart;
    int* bad = reinterpret_cast<int*>(w);
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_error(e, "fa_mlp_pair_grad memset");
    gather_rows_kernel<<<(unsigned)((R * kDin + 255) / 256), 256, 0, st>>>(X, pi, pj, P, rows, Xp,
                                                                          bad);
    fill_kernel<<<(unsigned)((R + 255) / 256), 256, 0, st>>>(ones, R, 1.0f);
    rc = cuda_error(cudaGetLastError(), "gather");
    if (rc != FA_OK) return rc;
    rc = mlp_forward_into(m, Xp, R, H1, H2, Y, st);
    if (rc != FA_OK) return rc;
    pair_loss_kernel<<<(unsigned)((P * 32 + 255) / 256), 256, 0, st>>>(Y, P, d, gY, lp);
    mean_kernel<<<1, 256, 0, st>>>(lp, P, loss);
    rc = cuda_error(cudaGetLastError(), "pair loss");
    if (rc != FA_OK) return rc;
    // layer 3
    rc = weight_grad(gY, R, kDout, H2, kDh, m->g + kOffW3, m->g + kOffB3, ones, part, m->tc_err,
                     st);
    if (rc != FA_OK) return rc;
    {
        GemmArgs<float, __nv_bfloat16> g{};
        g.M = R; g.N = kDh; g.K = kDout; g.A = gY; g.sam = kDout; g.sak = 1;
        g.B = m->pb + kOffW3; g.sbk = kDh; g.sbn = 1; g.C = gH2; g.scm = kDh; g.scn = 1;
        g.mask = H2;
        rc = tc_gemm<__nv_bfloat16, 64, EPI_MASK>(g, 1, m->tc_err, st);
        if (rc != FA_OK) return rc;
    }
    // layer 2
    rc = weight_grad(gH2, R, kDh, H1, kDh, m->g + kOffW2, m->g + kOffB2, ones, part, m->tc_err,
                     st);
    if (rc != FA_OK) return rc;
    {
        GemmArgs<float, __nv_bfloat16> g{};
        g.M = R; g.N = kDh; g.K = kDh; g.A = gH2; g.sam = kDh; g.sak = 1;
        g.B = m->pb + kOffW2; g.sbk = kDh; g.sbn = 1; g.C = gH1; g.scm = kDh; g.scn = 1;
        g.mask = H1;
        rc = tc_gemm<__nv_bfloat16, 64, EPI_MASK>(g, 1, m->tc_err, st);
        if (rc != FA_OK) return rc;
    }
    // layer 1
    rc = weight_grad(gH1, R, kDh, Xp, kDin, m->g + kOffW1, m->g + kOffB1, ones, part, m->tc_err,
                     st);
    if (rc != FA_OK) return rc;
    if (grad) {
        e = cudaMemcpyAsync(grad, m->g, sizeof(float) * kNParams, cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return cuda_error(e, "fa_mlp_pair_grad copy");
    }
    int hbad = 0, htc = 0;
    e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&htc, m->tc_err, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "fa_mlp_pair_grad");
    if (htc) return set_error(FA_ERR_CUDA, "fa_mlp_pair_grad: a tensor-core wait timed out");
    if (hbad) return set_error(FA_ERR_INVALID_ARG, "fa_mlp_pair_grad: pair index out of range");
    return FA_OK;
}

int fa_mlp_adam_step(fa_mlp* m, float lr, void* stream)
{
    if (!m) return set_error(FA_ERR_INVALID_ARG, "fa_mlp_adam_step: null handle");
    if (!(lr > 0.0f)) return set_error(FA_ERR_INVALID_ARG, "fa_mlp_adam_step: lr must be > 0");
    DeviceGuard g(m->h->device);
    if (g.rc != FA_OK) return g.rc;
    m->t += 1;
    const float bc1 = (float)(1.0 - std::pow(0.9, (double)m->t));
    const float bc2 = (float)(1.0 - std::pow(0.999, (double)m->t));
    adam_kernel<<<(unsigned)((kNParams + 255) / 256), 256, 0, static_cast<cudaStream_t>(stream)>>>(
        m->p, m->g, m->m, m->v, m->pb, kNParams, lr, bc1, bc2);
    return cuda_error(cudaGetLastError(), "adam launch");
}

int fa_fourier_descriptors(fa_handle* h, const double* z, int64_t M, int32_t N, int32_t F,
                           float* out, void* stream)
{
    if (!h) return set_error(FA_ERR_INVALID_ARG, "fa_fourier_descriptors: null handle");
    if (M < 0) return set_error(FA_ERR_INVALID_ARG, "fa_fourier_descriptors: negative count");
    int logn = -1;
    for (int L = 3; L <= 10; ++L)
        if (N == (1 << L)) logn = L;
    if (logn < 0)
        return set_error(FA_ERR_UNSUPPORTED,
                         "fa_fourier_descriptors: N must be a power of two in [8, 1024]");
    if (F < 1 || 2 * F >= N)
        return set_error(FA_ERR_INVALID_ARG, "fa_fourier_descriptors: need 1 <= F < N/2");
    if (M == 0) return FA_OK;
    if (!z || !out) return set_error(FA_ERR_INVALID_ARG, "fa_fourier_descriptors: null pointer");
    DeviceGuard g(h->device);
    if (g.rc != FA_OK) return g.rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t smem = sizeof(double2) * (size_t)N;
    if (N <= 256)
        descriptor_kernel<128, 256><<<(unsigned)M, 128, smem, st>>>(
            reinterpret_cast<const double2*>(z), M, N, logn, F, h->tf64[logn], out);
    else
        descriptor_kernel<128, 1024><<<(unsigned)M, 128, smem, st>>>(
            reinterpret_cast<const double2*>(z), M, N, logn, F, h->tf64[logn], out);
    return cuda_error(cudaGetLastError(), "descriptor launch");
}

int fa_column_stats(fa_handle* h, const float* X, int64_t M, int32_t D, float* mean,
                    float* inv_std, void* stream)
{
    if (!h || !X || !mean || !inv_std || M <= 0 || D <= 0)
        return set_error(FA_ERR_INVALID_ARG, "fa_column_stats: bad argument");
    DeviceGuard g(h->device);
    if (g.rc != FA_OK) return g.rc;
    column_stats_kernel<<<(unsigned)D, 256, 0, static_cast<cudaStream_t>(stream)>>>(X, M, D, mean,
                                                                                    inv_std);
    return cuda_error(cudaGetLastError(), "column stats launch");
}

int fa_standardize(fa_handle* h, float* X, int64_t M, int32_t D, const float* mean,
                   const float* inv_std, void* stream)
{
    if (!h || !X || !mean || !inv_std || M < 0 || D <= 0)
        return set_error(FA_ERR_INVALID_ARG, "fa_standardize: bad argument");
    if (M == 0) return FA_OK;
    DeviceGuard g(h->device);
    if (g.rc != FA_OK) return g.rc;
    standardize_kernel<<<(unsigned)((M * D + 255) / 256), 256, 0,
                         static_cast<cudaStream_t>(stream)>>>(X, M, D, mean, inv_std);
    return cuda_error(cudaGetLastError(), "standardize launch");
}

int fa_embed_sqdist(fa_handle* h, const float* A, int64_t Q, const float* B, int64_t G,
                    int32_t D, float* out, void* stream)
{
    if (!h || Q < 0 || G < 0 || D <= 0)
        return set_error(FA_ERR_INVALID_ARG, "fa_embed_sqdist: bad argument");
    if (Q == 0 || G == 0) return FA_OK;
    if (Q > (1 << 21) || G > ((int64_t)1 << 36))
        return set_error(FA_ERR_UNSUPPORTED, "fa_embed_sqdist: too many rows");
    if (!A || !B || !out) return set_error(FA_ERR_INVALID_ARG, "fa_embed_sqdist: null pointer");
    DeviceGuard dg(h->device);
    if (dg.rc != FA_OK) return dg.rc;
    GemmArgs<float, float> g{};
    g.M = Q; g.N = G; g.K = D; g.A = A; g.sam = D; g.sak = 1; g.B = B; g.sbk = 1; g.sbn = D;
    g.C = out; g.scm = G; g.scn = 1;
    return gemm<float, float, OP_SQDIFF, EPI_NONE>(g, 1, static_cast<cudaStream_t>(stream));
}

int fa_select_k(fa_handle* h, const void* keys, int32_t key_type, int64_t rows, int64_t C,
                int32_t k, int64_t* out_pos, void* out_keys, void* stream)
{
    if (!h) return set_error(FA_ERR_INVALID_ARG, "fa_select_k: null handle");
    if (key_type != FA_KEY_F32 && key_type != FA_KEY_F64)
        return set_error(FA_ERR_INVALID_ARG, "fa_select_k: unknown key type");
    if (rows < 0 || k < 1 || k > 256 || C < k)
        return set_error(FA_ERR_INVALID_ARG, "fa_select_k: need 1 <= k <= min(256, C)");
    if (rows == 0) return FA_OK;
    if (rows > (int64_t)1 << 31)
        return set_error(FA_ERR_UNSUPPORTED, "fa_select_k: too many rows");
    if (!keys || !out_pos) return set_error(FA_ERR_INVALID_ARG, "fa_select_k: null pointer");
    DeviceGuard g(h->device);
    if (g.rc != FA_OK) return g.rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (key_type == FA_KEY_F32)
        select_k_kernel<float, 32><<<(unsigned)rows, 256, 0, st>>>(
            static_cast<const float*>(keys), C, k, out_pos, static_cast<float*>(out_keys));
    else
        select_k_kernel<double, 64><<<(unsigned)rows, 256, 0, st>>>(
            static_cast<const double*>(keys), C, k, out_pos, static_cast<double*>(out_keys));
    return cuda_error(cudaGetLastError(), "select_k launch");
}

}  // extern "C"
