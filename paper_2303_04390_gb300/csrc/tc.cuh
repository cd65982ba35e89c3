// Fifth-generation tensor-core (tcgen05) primitives in inline PTX: TMEM
// allocation, shared-memory matrix descriptors for K-major tiles with the
// 128-byte swizzle, TF32 MMAs with FP32 accumulation in TMEM, commit to an
// mbarrier, and accumulator loads.
//
// Tile convention: a tile has `rows` rows (M or N) and K = 64 FP32 values
// per row, stored as two 128-byte-wide swizzle atoms along K (k in [0,32)
// and [32,64)), each atom `rows` x 128 bytes, rows at 128-byte stride, the
// 16-byte chunk j of row m stored at chunk j ^ (m % 8).  Atoms are
// 1024-byte aligned.  One MMA consumes K = 8 (32 bytes) of every row: the
// k-step kk starts at atom kk / 4, byte kk % 4 * 32 within the row.
#pragma once

#include <cstdint>

#include "tma.cuh"

namespace phylo {
namespace tc {

constexpr int kK = 64;  // contraction length (padded states)

// Byte offset of element (row, k) of a tile with `rows` rows.
__device__ __forceinline__ uint32_t sw_off(int row, int k, int rows) {
  const int atom = k >> 5, chunk = (k >> 2) & 7, within = k & 3;
  return (uint32_t)(atom * rows * 128 + row * 128 + ((chunk ^ (row & 7)) << 4) +
                    within * 4);
}

// Byte offset of the 16-byte chunk holding k = 4j..4j+3 of row `row`.
__device__ __forceinline__ uint32_t sw_chunk(int row, int j, int rows) {
  return (uint32_t)((j >> 3) * rows * 128 + row * 128 + (((j & 7) ^ (row & 7)) << 4));
}

// Shared-memory matrix descriptor: start address, stride between 8-row
// groups 1024 bytes, fixed version bits, 128-byte swizzle.
__device__ __forceinline__ uint64_t desc(uint32_t saddr) {
  return ((uint64_t)((saddr & 0x3FFFF) >> 4)) | ((uint64_t)1 << 16) |
         ((uint64_t)(1024 >> 4) << 32) | (1ull << 46) | (2ull << 61);
}

// Instruction descriptor: TF32 x TF32 -> FP32, both operands K-major.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t a, uint64_t b,
                                         uint32_t idesc, int accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(accumulate));
}

// D[128 x N] (+)= A[128 x 64] B[N x 64]' with A = Ahi + Alo and
// B = Bhi + Blo: the three products Ahi Bhi + Ahi Blo + Alo Bhi (the
// Alo Blo term is below FP32 resolution).  One thread issues.
template <int N>
__device__ __forceinline__ void mma_split3(uint32_t d_tmem, uint32_t a_hi, uint32_t a_lo,
                                           uint32_t b_hi, uint32_t b_lo) {
  constexpr uint32_t id = idesc_tf32(128, N);
  int first = 1;
#pragma unroll
  for (int pass = 0; pass < 3; ++pass) {
    const uint32_t a = pass == 2 ? a_lo : a_hi;
    const uint32_t b = pass == 1 ? b_lo : b_hi;
#pragma unroll
    for (int kk = 0; kk < 8; ++kk) {
      const uint32_t oa = (uint32_t)((kk >> 2) * 128 * 128 + (kk & 3) * 32);
      const uint32_t ob = (uint32_t)((kk >> 2) * N * 128 + (kk & 3) * 32);
      mma_tf32(d_tmem, desc(a + oa), desc(b + ob), id, first ? 0 : 1);
      first = 0;
    }
  }
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

// Round to TF32 (nearest, ties away), as an FP32 bit pattern.
__device__ __forceinline__ float tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Split 4 FP32 values into TF32 hi and exact remainder lo and store both
// chunks of row `row`, chunk j of a tile.
__device__ __forceinline__ void put_split4(unsigned char* hi_tile, unsigned char* lo_tile,
                                           int row, int j, int rows, float4 v) {
  float4 h = make_float4(tf32_hi(v.x), tf32_hi(v.y), tf32_hi(v.z), tf32_hi(v.w));
  float4 l = make_float4(v.x - h.x, v.y - h.y, v.z - h.z, v.w - h.w);
  const uint32_t off = sw_chunk(row, j, rows);
  *reinterpret_cast<float4*>(hi_tile + off) = h;
  *reinterpret_cast<float4*>(lo_tile + off) = l;
}

// Element (row, k) of a split tile, reassembled (hi + lo is the FP32 value).
__device__ __forceinline__ float get_split(const unsigned char* hi_tile,
                                           const unsigned char* lo_tile, int row, int k,
                                           int rows) {
  const uint32_t off = sw_off(row, k, rows);
  return *reinterpret_cast<const float*>(hi_tile + off) +
         *reinterpret_cast<const float*>(lo_tile + off);
}

}  // namespace tc
}  // namespace phylo
