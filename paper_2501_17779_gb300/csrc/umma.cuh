// umma.cuh -- fifth-generation tensor core (tcgen05) primitives for sm_103a,
// written as inline PTX: tensor-memory allocation, shared-memory matrix
// descriptors, the instruction descriptor, MMA issue and commit, tensor-memory
// loads, mbarriers with bounded waits, and the proxy fences between them.
//
// Operand layout used throughout: K-major, no swizzle.  A tile of R rows by KC
// elements (KC a multiple of 8 for 16-bit types, of 4 for 32-bit) is stored as
// 8-row x 16-byte "core matrices", each 128 contiguous bytes (row r % 8 at
// byte 16 (r % 8)); core matrix (r / 8, kb) of the tile starts at byte
// ((r / 8) (KC_bytes / 16) + kb) 128.  In a descriptor the leading-dimension
// byte offset is then 128 (the next core matrix along K) and the
// stride-dimension byte offset KC_bytes * 8 (the next 8-row group).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace fa {
namespace umma {

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// byte offset of element (r, k) of a K-major core-matrix tile whose rows are
// row_bytes long (row_bytes = KC * element size, a multiple of 16)
__host__ __device__ __forceinline__ uint32_t tile_off(int r, int kbyte, int row_bytes)
{
    return (uint32_t)(((r >> 3) * (row_bytes >> 4) + (kbyte >> 4)) * 128 + (r & 7) * 16 + (kbyte & 15));
}

// Shared-memory matrix descriptor: start address >> 4 in bits 0-13, leading
// byte offset >> 4 in 16-29, stride byte offset >> 4 in 32-45, the fixed
// version bits 46-48 = 0b001, base offset 0, swizzle mode 0 (none).
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor: D format F32 (bits 4-5 = 1), A and B formats
// (bits 7-9, 10-12: 1 = BF16 for kind::f16, 2 = TF32 for kind::tf32), both
// K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t idesc(int M, int N, uint32_t ab_format)
{
    return (1u << 4) | (ab_format << 7) | (ab_format << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}
constexpr uint32_t kFmtBF16 = 1;
constexpr uint32_t kFmtTF32 = 2;

// ---- tensor memory (one warp, all lanes) -----------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
                 : "memory");
}

// ---- MMA issue (one thread) --------------------------------------------------
// D[tmem] (+)= A[smem] * B[smem]^T, M x N x 16 (kind::f16) or M x N x 8 (kind::tf32)
__device__ __forceinline__ void mma_f16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id,
                                        uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t id,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(id), "r"(accumulate)
        : "memory");
}
// the mbarrier receives one arrival once every MMA this thread issued so far
// has completed (and its shared-memory operands may be overwritten)
__device__ __forceinline__ void mma_commit(uint64_t* mbar)
{
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(mbar))
        : "memory");
}

// ---- fences ------------------------------------------------------------------
// generic-proxy shared-memory writes made visible to the tensor core
__device__ __forceinline__ void fence_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// ---- mbarriers -------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(count)
                 : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(mbar)) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Waits for the phase of the given parity to complete; gives up after about
// 2^22 polls, all but the first 256 followed by a 256 ns sleep (well over a
// second, far beyond any MMA) and returns false, so that a wrong arrival count
// can never hang the GPU: the caller then records an error and leaves cleanly.
// The first polls do not sleep: in a pipeline the phase usually completes
// within a few hundred cycles, and a sleep would add its whole length.
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity)
{
    for (uint32_t i = 0; i < (1u << 22); ++i) {
        if (mbar_test(mbar, parity)) return true;
        if (i >= 256) __nanosleep(256);
    }
    return false;
}

// ---- tensor memory -> registers (one warp: its 32 lanes, 32 columns) --------
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// float -> three bfloat16 pieces hi + mid + lo (each the round-to-nearest
// bfloat16 of what the previous ones leave): exactly x for every float whose
// exponent keeps the pieces normal, since each piece takes 8 more significand
// bits and a float has 24.
__device__ __forceinline__ void split3_bf16(float x, uint16_t& h, uint16_t& m, uint16_t& l)
{
    const __nv_bfloat16 bh = __float2bfloat16_rn(x);
    const float r1 = __fsub_rn(x, __bfloat162float(bh));
    const __nv_bfloat16 bm = __float2bfloat16_rn(r1);
    const float r2 = __fsub_rn(r1, __bfloat162float(bm));
    const __nv_bfloat16 bl = __float2bfloat16_rn(r2);
    h = __bfloat16_as_ushort(bh);
    m = __bfloat16_as_ushort(bm);
    l = __bfloat16_as_ushort(bl);
}

}  // namespace umma
}  // namespace fa
