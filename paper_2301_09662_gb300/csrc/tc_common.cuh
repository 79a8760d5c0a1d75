// Operand layouts and helpers shared by the tensor-core imaging kernels
// (tc_dual64.cu, tc_pair128.cu): 128 x 128 16-bit operand parts in the
// canonical no-swizzle layouts of tcgen05 shared-memory descriptors, the
// instruction descriptors of kind::f16, and the hi + lo operand split.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdint>

namespace epic {
namespace tcc {

constexpr uint32_t kPart = 128u * 128u * 2u;    // one 128 x 128 16-bit operand part (32 KB)
constexpr uint32_t kLBO = 128;                  // K-adjacent core matrices
constexpr uint32_t kSBO = 2048;                 // M/N-adjacent core matrices (16 along K x 128 B)

// byte offset of (row/col n, k) in the MN-major canonical layout (8 consecutive n per 16 bytes)
__host__ __device__ constexpr uint32_t mn_off(int n, int k)
{
    return static_cast<uint32_t>((n >> 3) * kSBO + (k >> 3) * kLBO + (k & 7) * 16 + (n & 7) * 2);
}

// byte offset of (row, k) in the K-major canonical layout of one 128 x 128 part
// (8 consecutive k per 16 bytes, core matrices of 8 rows)
__host__ __device__ constexpr uint32_t k_off(int row, int k)
{
    return static_cast<uint32_t>((row >> 3) * kSBO + (k >> 3) * kLBO + (row & 7) * 16 + (k & 7) * 2);
}

// kind::f16 instruction descriptor: FP32 accumulate, A and B both FP16 or both
// BF16, both K-major (idesc_kk) or B MN-major (idesc_kmn), shape M x N
__host__ __device__ constexpr uint32_t idesc_kk(int M, int N, bool bf16)
{
    return (1u << 4) | ((bf16 ? 1u : 0u) << 7) | ((bf16 ? 1u : 0u) << 10) |
           (static_cast<uint32_t>(N >> 3) << 17) | (static_cast<uint32_t>(M >> 4) << 24);
}
__host__ __device__ constexpr uint32_t idesc_kmn(int M, int N, bool bf16) { return idesc_kk(M, N, bf16) | (1u << 16); }

// (a, b) rounded to a 16-bit pair hi; with SPLIT, lo = what hi leaves of them,
// rounded once more (a in the low half of each word)
template <bool BF16, bool SPLIT>
__device__ __forceinline__ void split_pair(float a, float b, uint32_t &hi, uint32_t &lo)
{
    if constexpr (BF16) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        if constexpr (SPLIT) {
            const float2 back = __bfloat1622float2(h);
            const __nv_bfloat162 l = __floats2bfloat162_rn(a - back.x, b - back.y);
            lo = *reinterpret_cast<const uint32_t *>(&l);
        }
    } else {
        const __half2 h = __floats2half2_rn(a, b);
        hi = *reinterpret_cast<const uint32_t *>(&h);
        if constexpr (SPLIT) {
            const float2 back = __half22float2(h);
            const __half2 l = __floats2half2_rn(a - back.x, b - back.y);
            lo = *reinterpret_cast<const uint32_t *>(&l);
        }
    }
}

// D(tmem) (+)= A(tmem) x B(smem)^T
__device__ __forceinline__ void mma_ts(uint32_t d_tmem, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d_tmem),
        "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(accumulate)
        : "memory");
}

}  // namespace tcc
}  // namespace epic
