// Fifth-generation tensor-core (tcgen05) primitives in inline PTX: TMEM
// allocation, shared-memory matrix descriptors for K-major tiles with the
// 128-byte swizzle, BF16 MMAs with FP32 accumulation in TMEM, commit to an
// mbarrier, accumulator loads, and the operand splits that give FP32
// accuracy from the reduced-precision inputs.  The operand tile layout is
// described with the BF16 helpers below.
#pragma once

#include <cuda_bf16.h>

#include <cstdint>

#include "tma.cuh"

namespace phylo {
namespace tc {

// Shared-memory matrix descriptor: start address, stride between 8-row
// groups 1024 bytes, fixed version bits, 128-byte swizzle.
__device__ __forceinline__ uint64_t desc(uint32_t saddr) {
  return ((uint64_t)((saddr & 0x3FFFF) >> 4)) | ((uint64_t)1 << 16) |
         ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Arrive on `bar` once every previously issued MMA of this thread is done.
__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Generic-proxy writes to shared memory made visible to the tensor core.
__device__ __forceinline__ void fence_smem_for_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Warp-wide TMEM allocation of `cols` columns; the address lands in *slot.
__device__ __forceinline__ void alloc(uint32_t* slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_addr(slot)),
               "r"(cols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void dealloc(uint32_t tmem, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols)
               : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's row (warp w of
// the block reads TMEM lanes 32w..32w+31).
__device__ __forceinline__ void ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 consecutive FP32 accumulator columns of this thread's row.
__device__ __forceinline__ void ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
        "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
        "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
        "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// ---------------------------------------------------------------------------
// BF16 operands (kind::f16).  A BF16 tile row is 128 bytes = 64 elements,
// so K = 64 is one swizzle atom: element (row, k) sits in 16-byte chunk
// k / 8 of the row, stored at chunk (k / 8) ^ (row % 8).  One MMA consumes
// K = 16 (32 bytes); k-step kk starts kk * 32 bytes into the row.
// ---------------------------------------------------------------------------

// Byte offset of element (row, k) of a BF16 tile.
__device__ __forceinline__ uint32_t b16_off(int row, int k) {
  return (uint32_t)(row * 128 + ((((k >> 3) ^ (row & 7))) << 4) + (k & 7) * 2);
}

// Byte offset of the 16-byte chunk holding k = 8j..8j+7 of row `row`.
__device__ __forceinline__ uint32_t b16_chunk(int row, int j) {
  return (uint32_t)(row * 128 + ((j ^ (row & 7)) << 4));
}

// Instruction descriptor: BF16 x BF16 -> FP32, both operands K-major.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b,
                                         uint32_t idesc, int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// D[128 x N] = A[128 x 64] B[N x 64]' with A = A0 + A1 + A2 and
// B = B0 + B1 + B2 split into BF16 terms of decreasing magnitude (each
// about 2^-8 of the previous one): the six products of order up to 2^-16,
// A0B0 + A0B1 + A1B0 + A0B2 + A1B1 + A2B0, give FP32 accuracy; the dropped
// ones are below 2^-24 relative.  a[t], b[t] are the shared addresses of
// the term tiles (A: 128 rows, B: N rows).  One thread issues.
template <int N>
__device__ __forceinline__ void mma_split_bf16x3(uint32_t d_tmem, const uint32_t (&a)[3],
                                                 const uint32_t (&b)[3]) {
  constexpr uint32_t id = idesc_bf16(128, N);
  constexpr int pa[6] = {0, 0, 1, 0, 1, 2};
  constexpr int pb[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
  for (int p = 0; p < 6; ++p)
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
      mma_bf16(d_tmem, desc(a[pa[p]] + kk * 32), desc(b[pb[p]] + kk * 32), id,
               (p | kk) ? 1 : 0);
}

// The same six products accumulated onto D (accumulate = true) or
// overwriting it: one K-block of a K-tiled contraction.
template <int N>
__device__ __forceinline__ void mma_split_bf16x3_acc(uint32_t d_tmem, const uint32_t (&a)[3],
                                                     const uint32_t (&b)[3], bool accumulate) {
  constexpr uint32_t id = idesc_bf16(128, N);
  constexpr int pa[6] = {0, 0, 1, 0, 1, 2};
  constexpr int pb[6] = {0, 1, 0, 2, 1, 0};
#pragma unroll
  for (int p = 0; p < 6; ++p)
#pragma unroll
    for (int kk = 0; kk < 4; ++kk)
      mma_bf16(d_tmem, desc(a[pa[p]] + kk * 32), desc(b[pb[p]] + kk * 32), id,
               (accumulate || p || kk) ? 1 : 0);
}

// Split 8 FP32 values into three BF16 terms x = t0 + t1 + t2 (each term
// the round-to-nearest BF16 of the remainder so far; the remainders are
// exact in FP32) and store the three 16-byte chunks of row `row`, chunk j.
__device__ __forceinline__ void put_split3(unsigned char* t0, unsigned char* t1,
                                           unsigned char* t2, int row, int j,
                                           const float (&x)[8]) {
  uint32_t w[3][4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    float a = x[2 * i], b = x[2 * i + 1];
#pragma unroll
    for (int t = 0; t < 3; ++t) {
      const __nv_bfloat162 h = __floats2bfloat162_rn(a, b);
      const float2 f = __bfloat1622float2(h);
      a = __fsub_rn(a, f.x);
      b = __fsub_rn(b, f.y);
      w[t][i] = *reinterpret_cast<const uint32_t*>(&h);
    }
  }
  const uint32_t off = b16_chunk(row, j);
  *reinterpret_cast<uint4*>(t0 + off) = make_uint4(w[0][0], w[0][1], w[0][2], w[0][3]);
  *reinterpret_cast<uint4*>(t1 + off) = make_uint4(w[1][0], w[1][1], w[1][2], w[1][3]);
  *reinterpret_cast<uint4*>(t2 + off) = make_uint4(w[2][0], w[2][1], w[2][2], w[2][3]);
}

// Element (row, k) of a three-term BF16 tile set, reassembled in FP32.
__device__ __forceinline__ float get_split3(const unsigned char* t0, const unsigned char* t1,
                                            const unsigned char* t2, int row, int k) {
  const uint32_t off = b16_off(row, k);
  const float a = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(t0 + off));
  const float b = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(t1 + off));
  const float c = __bfloat162float(*reinterpret_cast<const __nv_bfloat16*>(t2 + off));
  return (a + b) + c;
}

}  // namespace tc
}  // namespace phylo
