// Blackwell 5th-generation tensor-core helpers (tcgen05, inline PTX) for the DFT-as-GEMM variant.
//
// One thread issues tcgen05.mma with both operands in shared memory (UMMA matrix descriptors,
// no swizzle; B K-major, A K-major or MN-major), the FP32 accumulator lives in tensor memory
// (TMEM), completion is
// signalled on an mbarrier through tcgen05.commit, and the four warps of a warpgroup read the
// accumulator rows back with tcgen05.ld (warp w owns TMEM lanes 32w .. 32w+31).
//
// Operand layout ("core matrices"): an R x K operand of 16-bit elements is stored as 8-row x
// 8-element core matrices of 128 contiguous bytes (row i of a core matrix at byte 16 i). Core
// matrix (g, c) (row group g, element group c) sits at byte (g * K/8 + c) * 128. In descriptor
// terms: leading-dimension byte offset (between core matrices along K) = 128, stride-dimension
// byte offset (between 8-row groups) = K/8 * 128.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include "vbw_common.cuh"

namespace vbw {

__device__ __forceinline__ uint32_t tc_smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Byte offset of element (row, k) of an R x K core-matrix operand (16-bit elements).
__host__ __device__ constexpr uint32_t core_offset(int row, int k, int K)
{
    return (uint32_t)(((row >> 3) * (K >> 3) + (k >> 3)) * 128 + (row & 7) * 16 + (k & 7) * 2);
}

// UMMA shared-memory matrix descriptor: start address, leading / stride byte offsets (all >> 4),
// descriptor version 1 (sm_100 family), base offset 0, no swizzle.
__device__ __forceinline__ uint64_t umma_desc(const void* base, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((tc_smem_u32(base) >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// The same descriptor from a 32-bit shared-memory address.
__device__ __forceinline__ uint64_t umma_desc_u32(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of tcgen05.mma kind::f16: FP32 accumulator, A and B both BF16 (bf16 =
// true) or both FP16, both K-major, shape M x N (M in {64, 128}, N a multiple of 8 up to 256).
// Bit 15 set makes A MN-major (the caller ORs it in).
__host__ __device__ constexpr uint32_t umma_idesc(bool bf16, int M, int N)
{
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
           ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst_smem, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_u32(dst_smem)),
                 "r"(ncols)
                 : "memory");
}

__device__ __forceinline__ void tmem_relinquish()
{
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

// D[tmem] (+)= A[smem] * B[smem]; issued by one thread.
__device__ __forceinline__ void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
        ::"r"(d_tmem), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on bar once every tcgen05 operation this thread issued before has completed.
__device__ __forceinline__ void umma_commit(uint64_t* bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     tc_smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 32 consecutive TMEM columns of this thread's lane (warp-wide, 32x32b shape), waited.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---- 16-bit rounding of single values (the GEMM test hook; the OLS kernel splits pairs of
// values into pieces with packed conversions, ols_tc.cuh)
template <bool BF16>
struct Half16;
template <>
struct Half16<true> {
    using T = __nv_bfloat16;
    __device__ static T from(float v) { return __float2bfloat16_rn(v); }
    __device__ static float to(T v) { return __bfloat162float(v); }
};
template <>
struct Half16<false> {
    using T = __half;
    __device__ static T from(float v) { return __float2half_rn(v); }
    __device__ static float to(T v) { return __half2float(v); }
};

}  // namespace vbw
