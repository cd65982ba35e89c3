// FP32 level kernels for 21..64 states (codon models) on the tensor cores.
//
// Arithmetic of Eq. 2 (with Eq. 3 at the root) and Eq. 4 with the fused
// Eq. 8 ratio, per (node, tile of 128 patterns, category r):
//   post:  U_x = p_x P_x'            (x = the internal children)
//          p_k = U_i o U_j
//   pre:   [U_x | V_x] = p_x [P_x ; dP_x]'
//          a_i = q_k o U_j,  a_j = q_k o U_i
//          num_x = a_x . V_x,  den = a_i . U_i      (per pattern)
//          q_i = a_i P_i,  q_j = a_j P_j             (internal children)
// Every product with a partial tile is a 128 x N x 64 contraction issued as
// tcgen05.mma kind::tf32 with FP32 accumulation in TMEM.  FP32 accuracy
// comes from splitting both operands into TF32 hi and remainder lo and
// summing Ahi Bhi + Ahi Blo + Alo Bhi (three passes).  Operand tiles are
// written to shared memory in the K-major 128-byte-swizzle layout of
// tc.cuh.  After each contraction one thread per pattern reads its
// accumulator row back from TMEM, so the products, the Eq. 8 dot products,
// the ratio and the rescale are thread-local.
//
// Rescaling on this path is per (node, pattern, category): each vector gets
// its own power of two, and the exponents are kept per category.  This lets
// each category finish before the next begins, which keeps TMEM and shared
// memory within one CTA.  The exponents are combined where categories meet:
// in the root's log-likelihood and in the Eq. 8 ratio (sums over r taken
// relative to the largest exponent).
//   ep[node][r][c]: cumulative post-order exponent of p_node,r,c
//   eq[node][r][c]: cumulative pre-order exponent of q_node,r,c
// A tip child contributes exponent 0 and a compact tip selects a column of
// the staged matrix instead of a contraction.
//
// Every wait on an mbarrier is bounded; on expiry the kernel raises
// ERR_TIMEOUT, frees its TMEM and returns.
#pragma once

#include "tc.cuh"

namespace phylo {

constexpr int kTcRows = 128;     // patterns per tile (MMA M)
constexpr int kTcThreads = 128;  // one thread per pattern row

// Shared memory (bytes), 1024-byte aligned regions:
//   post: A (p tile, hi+lo 64 KB) | B_i (P_i hi+lo 32 KB) | B_j (32 KB)
//   pre:  A (64 KB) | Bc_i ([P_i; dP_i] hi+lo 64 KB) | Bc_j (64 KB)
constexpr uint32_t kTileBytes128 = 128 * 256;  // 128 rows x 64 FP32
constexpr uint32_t kTileBytes64 = 64 * 256;
constexpr size_t kTcPostSmem = 1024 + 2 * kTileBytes128 + 4 * kTileBytes64;
constexpr size_t kTcPreSmem = 1024 + 2 * kTileBytes128 + 4 * kTileBytes128;

__device__ __forceinline__ float pow2i(int d) {  // 2^d for d <= 0 (0 below 2^-126)
  return d < -126 ? 0.f : __uint_as_float((unsigned)(127 + d) << 23);
}

// Bounded wait; on timeout raise the flag (once per block).
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity, int* err) {
  const bool ok = mbar_wait(bar, parity);
  if (!ok && threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
  return ok;
}

// Stage the rows [row0, row0 + 64) of a tile from the 64 x 64 row-major
// FP32 matrix M (hi/lo split).
__device__ __forceinline__ void stage_matrix(unsigned char* hi, unsigned char* lo, int rows,
                                             int row0, const float* __restrict__ M) {
  for (int i = threadIdx.x; i < 64 * 16; i += kTcThreads) {
    const int s = i >> 4, j = i & 15;
    const float4 v = __ldg(reinterpret_cast<const float4*>(M + s * 64) + j);
    tc::put_split4(hi, lo, row0 + s, j, rows, v);
  }
}

// Stage M' (64 x 64): row t holds column t of M.
__device__ __forceinline__ void stage_matrix_t(unsigned char* hi, unsigned char* lo,
                                               const float* __restrict__ M) {
  for (int i = threadIdx.x; i < 64 * 16; i += kTcThreads) {
    const int t = i >> 4, j = i & 15;
    const float4 v = make_float4(__ldg(M + (4 * j) * 64 + t), __ldg(M + (4 * j + 1) * 64 + t),
                                 __ldg(M + (4 * j + 2) * 64 + t), __ldg(M + (4 * j + 3) * 64 + t));
    tc::put_split4(hi, lo, t, j, 64, v);
  }
}

// Stage this thread's row of a partial tile: 64 FP32 from src (or zeros).
__device__ __forceinline__ void stage_row(unsigned char* hi, unsigned char* lo, int row,
                                          const float* __restrict__ src, bool valid) {
#pragma unroll 4
  for (int j = 0; j < 16; ++j) {
    const float4 v = valid ? __ldg(reinterpret_cast<const float4*>(src) + j)
                           : make_float4(0.f, 0.f, 0.f, 0.f);
    tc::put_split4(hi, lo, row, j, kTcRows, v);
  }
}

struct TcChild {
  int b;
  bool compact;  // tip with a compact state
  bool tipvec;   // tip with a partial vector
  bool internal;
};

__device__ __forceinline__ TcChild tc_child(const LevelArgs<float>& a, int b, bool compact) {
  TcChild c;
  c.b = b;
  c.compact = compact;
  c.internal = b >= a.n_tips;
  c.tipvec = !c.internal && !compact;
  return c;
}

__device__ __forceinline__ const float* child_row(const LevelArgs<float>& a, const TcChild& x,
                                                  int c, int r) {
  const int C = a.n_patterns;
  if (x.internal)
    return a.post + (((size_t)(x.b - a.n_tips) * C + c) * a.n_cat + r) * 64;
  return a.tip_partials + ((size_t)x.b * C + c) * 64;
}

// 16 accumulator columns (or a compact tip's matrix column from the staged
// split tile; rows_tile = rows of that tile, row0 = its first row for this
// matrix).
__device__ __forceinline__ void child_chunk(const TcChild& x, int y, int S, uint32_t taddr,
                                            const unsigned char* hi, const unsigned char* lo,
                                            int rows_tile, int row0, int s0, float (&u)[16]) {
  if (!x.compact) {
    tc::ld16(taddr, u);
    return;
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int s = s0 + i;
    u[i] = y < S ? tc::get_split(hi, lo, row0 + s, y, rows_tile) : (s < S ? 1.f : 0.f);
  }
}

// ---------------------------------------------------------------------------
// Post-order level (Eq. 2; Eq. 3 at the root)
// ---------------------------------------------------------------------------
template <typename T>  // float only; a template so that it is emitted where used
__global__ void __launch_bounds__(kTcThreads) post_tc_kernel(LevelArgs<T> a) {
  static_assert(std::is_same<T, float>::value, "tensor-core path is FP32");
  extern __shared__ unsigned char smraw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  unsigned char* A_hi = base;
  unsigned char* A_lo = A_hi + kTileBytes128;
  unsigned char* B_hi[2] = {A_lo + kTileBytes128, A_lo + kTileBytes128 + 2 * kTileBytes64};
  unsigned char* B_lo[2] = {B_hi[0] + kTileBytes64, B_hi[1] + kTileBytes64};
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ double lred[kTcThreads / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int4 d = a.level_desc[blockIdx.y];
  const int k = d.x;
  const TcChild xs[2] = {tc_child(a, d.y, d.w & kDescFlagCompact0),
                         tc_child(a, d.z, d.w & kDescFlagCompact1)};
  const int c0 = blockIdx.x * kTcRows, c = c0 + tid;
  const bool valid = c < C;
  const int estr = a.escale_stride;
  if (warp == 0) tc::alloc(&tmem_slot, 128);
  if (tid == 0) mbar_init_fenced(&bar, 1);
  int y[2] = {0, 0};
  for (int x = 0; x < 2; ++x)
    if (xs[x].compact && valid) y[x] = a.tip_states[(size_t)xs[x].b * a.state_stride + c];
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  uint32_t parity = 0;
  bool ok = true;
  // running log-likelihood sum of the root (value, exponent)
  float lsum = 0.f;
  int lexp = INT_MIN / 2;
  for (int r = 0; r < R && ok; ++r) {
    for (int x = 0; x < 2; ++x)
      stage_matrix(B_hi[x], B_lo[x], 64, 0, a.P + ((size_t)xs[x].b * R + r) * 4096);
    for (int x = 0; x < 2 && ok; ++x) {
      if (xs[x].compact) continue;
      stage_row(A_hi, A_lo, tid, child_row(a, xs[x], valid ? c : c0, r), valid);
      tc::fence_smem_for_async();
      __syncthreads();
      tc::fence_after();
      if (tid == 0) {
        tc::mma_split3<64>(tmem + 64 * x, smem_addr(A_hi), smem_addr(A_lo), smem_addr(B_hi[x]),
                           smem_addr(B_lo[x]));
        tc::commit(&bar);
      }
      ok = __syncthreads_and(tc_wait(&bar, parity, a.err));
      parity ^= 1u;
      tc::fence_after();
    }
    if (!ok) break;
    __syncthreads();  // staged matrices visible for compact-tip columns
    // epilogue: p = U_i o U_j in registers, its max, then scale and store
    float p[64];
    float m = 0.f;
#pragma unroll
    for (int s0 = 0; s0 < 64; s0 += 16) {
      float ui[16], uj[16];
      child_chunk(xs[0], y[0], S, trow + 0 + s0, B_hi[0], B_lo[0], 64, 0, s0, ui);
      child_chunk(xs[1], y[1], S, trow + 64 + s0, B_hi[1], B_lo[1], 64, 0, s0, uj);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        p[s0 + i] = ui[i] * uj[i];
        m = fmaxf(m, fabsf(p[s0 + i]));
      }
    }
    // An all-zero vector is legitimate for one category (its terms vanish
    // wherever it is used); the root flags a pattern whose categories all
    // vanish.
    int e = 0;
    if (valid) {
      if (!isfinite(m)) atomicOr(a.err, ERR_ZERO_PARTIAL);
      else if (m > 0.f) (void)frexpf(m, &e);
      e = max(e, -126);  // 2^-e stays finite for a subnormal maximum
    }
    const float f = ldexpf(1.f, -e);
    int E = e;
    if (valid)
      for (int x = 0; x < 2; ++x)
        if (xs[x].internal)
          E += a.escale[((size_t)(xs[x].b - a.n_tips) * R + r) * estr + c];
    float pi_dot = 0.f;
    if (k != a.root) {
      if (valid) {
        float* out = a.post + (((size_t)(k - a.n_tips) * C + c) * R + r) * 64;
#pragma unroll
        for (int i = 0; i < 64; i += 4)
          *reinterpret_cast<float4*>(out + i) =
              make_float4(p[i] * f, p[i + 1] * f, p[i + 2] * f, p[i + 3] * f);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 64; ++i)
        if (i < S) pi_dot = fmaf(a.root_pit[i], p[i] * f, pi_dot);
    }
    if (k != a.root) {
      if (valid) a.escale[((size_t)(k - a.n_tips) * R + r) * estr + c] = E;
    } else if (valid && pi_dot != 0.f) {
      // L_c = sum_r w_r 2^E_r (pi' p_r): running sum relative to the largest E
      const float term = a.cat_wt[r] * pi_dot;
      if (E > lexp) {
        lsum = lsum * pow2i(lexp - E) + term;
        lexp = E;
      } else {
        lsum += term * pow2i(E - lexp);
      }
    }
    tc::fence_before();
    __syncthreads();  // TMEM and shared tiles are reused by the next category
    tc::fence_after();
  }
  if (ok && k == a.root) {
    double term = 0.0;
    if (valid) {
      if (!(lsum > 0.f) || !isfinite(lsum)) atomicOr(a.err, ERR_ZERO_PARTIAL);
      term = (double)a.pattern_wt[c] *
             (log((double)lsum) + (double)lexp * 0.69314718055994530942);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) term += __shfl_down_sync(kFull, term, o);
    if (lane == 0) lred[warp] = term;
    __syncthreads();
    if (tid == 0) {
      double l = 0.0;
      for (int w = 0; w < kTcThreads / 32; ++w) l += lred[w];
      a.lpart[blockIdx.x] = l;
    }
  }
  if (!ok && tid == 0) (void)mbar_wait(&bar, parity ^ 1u);  // bounded drain
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, 128);
}

// ---------------------------------------------------------------------------
// Pre-order level (Eq. 4) with the fused gradient (Eqs. 7, 8)
// ---------------------------------------------------------------------------
template <typename T>  // float only
__global__ void __launch_bounds__(kTcThreads) pre_tc_kernel(LevelArgs<T> a) {
  static_assert(std::is_same<T, float>::value, "tensor-core path is FP32");
  extern __shared__ unsigned char smraw[];
  unsigned char* base = reinterpret_cast<unsigned char*>(
      (reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  // A: 128-row tile (children's p, later the two 64-row P' tiles)
  unsigned char* A_hi = base;
  unsigned char* A_lo = A_hi + kTileBytes128;
  // Bc_x: [P_x; dP_x] as a 128-row tile; later a_x as an A operand
  unsigned char* C_hi[2] = {A_lo + kTileBytes128, A_lo + 3 * kTileBytes128};
  unsigned char* C_lo[2] = {C_hi[0] + kTileBytes128, C_hi[1] + kTileBytes128};
  unsigned char* T_hi[2] = {A_hi, A_hi + kTileBytes64};  // P_x' tiles (64 rows)
  unsigned char* T_lo[2] = {A_lo, A_lo + kTileBytes64};
  __shared__ uint64_t bar;
  __shared__ uint32_t tmem_slot;
  __shared__ F2 red[kTcThreads / 32][2];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int4 d = a.level_desc[blockIdx.y];
  const int k = d.x;
  const TcChild xs[2] = {tc_child(a, d.y, d.w & kDescFlagCompact0),
                         tc_child(a, d.z, d.w & kDescFlagCompact1)};
  const int c0 = blockIdx.x * kTcRows, c = c0 + tid;
  const bool valid = c < C;
  const int estr = a.escale_stride;
  const bool root = k == a.root;
  if (warp == 0) tc::alloc(&tmem_slot, 256);
  if (tid == 0) mbar_init_fenced(&bar, 1);
  int y[2] = {0, 0};
  for (int x = 0; x < 2; ++x)
    if (xs[x].compact && valid) y[x] = a.tip_states[(size_t)xs[x].b * a.state_stride + c];
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  uint32_t parity = 0;
  bool ok = true;
  // running Eq. 8 sums over categories, relative to exponent gexp
  float Ni = 0.f, Nj = 0.f, Dn = 0.f;
  int gexp = INT_MIN / 2;
  for (int r = 0; r < R && ok; ++r) {
    // ---- [U_x | V_x] = p_x [P_x ; dP_x]' ----
    for (int x = 0; x < 2; ++x) {
      const size_t mo = ((size_t)xs[x].b * R + r) * 4096;
      stage_matrix(C_hi[x], C_lo[x], 128, 0, a.P + mo);
      stage_matrix(C_hi[x], C_lo[x], 128, 64, a.dP + mo);
    }
    for (int x = 0; x < 2 && ok; ++x) {
      if (xs[x].compact) continue;
      stage_row(A_hi, A_lo, tid, child_row(a, xs[x], valid ? c : c0, r), valid);
      tc::fence_smem_for_async();
      __syncthreads();
      tc::fence_after();
      if (tid == 0) {
        tc::mma_split3<128>(tmem + 128 * x, smem_addr(A_hi), smem_addr(A_lo),
                            smem_addr(C_hi[x]), smem_addr(C_lo[x]));
        tc::commit(&bar);
      }
      ok = __syncthreads_and(tc_wait(&bar, parity, a.err));
      parity ^= 1u;
      tc::fence_after();
    }
    if (!ok) break;
    __syncthreads();  // staged matrices visible for compact-tip columns
    // exponent of this category's products at node k
    int E = 0;
    if (valid) {
      if (!root) E += a.pre_escale[((size_t)(k - a.n_tips) * R + r) * estr + c];
      for (int x = 0; x < 2; ++x)
        if (xs[x].internal) E += a.escale[((size_t)(xs[x].b - a.n_tips) * R + r) * estr + c];
    }
    // ---- epilogue 1: a_i, a_j, the Eq. 8 terms; a_x staged as an A operand ----
    const float* qrow = (!root && valid)
                            ? a.pre + (((size_t)(k - a.n_tips) * C + c) * R + r) * 64
                            : nullptr;
    float ni = 0.f, nj = 0.f, dn = 0.f;
#pragma unroll 1
    for (int s0 = 0; s0 < 64; s0 += 16) {
      float ui[16], vi[16], uj[16], vj[16], q[16];
      child_chunk(xs[0], y[0], S, trow + 0 + s0, C_hi[0], C_lo[0], 128, 0, s0, ui);
      child_chunk(xs[0], y[0], S, trow + 64 + s0, C_hi[0], C_lo[0], 128, 64, s0, vi);
      child_chunk(xs[1], y[1], S, trow + 128 + s0, C_hi[1], C_lo[1], 128, 0, s0, uj);
      child_chunk(xs[1], y[1], S, trow + 192 + s0, C_hi[1], C_lo[1], 128, 64, s0, vj);
      if (xs[0].compact && y[0] >= S)
        for (int i = 0; i < 16; ++i) vi[i] = 0.f;  // gap: d/dt of the all-ones vector
      if (xs[1].compact && y[1] >= S)
        for (int i = 0; i < 16; ++i) vj[i] = 0.f;
#pragma unroll
      for (int i = 0; i < 16; i += 4) {
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (qrow) v = __ldg(reinterpret_cast<const float4*>(qrow + s0 + i));
        else if (root && valid) {
          v.x = s0 + i < S ? a.root_pit[s0 + i] : 0.f;
          v.y = s0 + i + 1 < S ? a.root_pit[s0 + i + 1] : 0.f;
          v.z = s0 + i + 2 < S ? a.root_pit[s0 + i + 2] : 0.f;
          v.w = s0 + i + 3 < S ? a.root_pit[s0 + i + 3] : 0.f;
        }
        q[i] = v.x; q[i + 1] = v.y; q[i + 2] = v.z; q[i + 3] = v.w;
      }
      float ai[16], aj[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        ai[i] = q[i] * uj[i];
        aj[i] = q[i] * ui[i];
        ni = fmaf(ai[i], vi[i], ni);
        nj = fmaf(aj[i], vj[i], nj);
        dn = fmaf(ai[i], ui[i], dn);
      }
      // a_x becomes the A operand of q_x = a_x P_x (its Bc_x tile is no
      // longer read: an internal child's U, V came from TMEM)
#pragma unroll
      for (int i = 0; i < 16; i += 4) {
        if (xs[0].internal)
          tc::put_split4(C_hi[0], C_lo[0], tid, (s0 + i) >> 2, 128,
                         make_float4(ai[i], ai[i + 1], ai[i + 2], ai[i + 3]));
        if (xs[1].internal)
          tc::put_split4(C_hi[1], C_lo[1], tid, (s0 + i) >> 2, 128,
                         make_float4(aj[i], aj[i + 1], aj[i + 2], aj[i + 3]));
      }
    }
    // a category whose terms all vanish carries an arbitrary exponent: skip it
    if (valid && (ni != 0.f || nj != 0.f || dn != 0.f)) {
      const float w = a.cat_wt[r];
      if (E > gexp) {
        const float sc = pow2i(gexp - E);
        Ni = Ni * sc + w * ni;
        Nj = Nj * sc + w * nj;
        Dn = Dn * sc + w * dn;
        gexp = E;
      } else {
        const float sc = pow2i(E - gexp);
        Ni += w * ni * sc;
        Nj += w * nj * sc;
        Dn += w * dn * sc;
      }
    }
    // ---- q_x = a_x P_x for the internal children ----
    const bool any_int = xs[0].internal || xs[1].internal;
    if (any_int) {
      for (int x = 0; x < 2; ++x)
        if (xs[x].internal)
          stage_matrix_t(T_hi[x], T_lo[x], a.P + ((size_t)xs[x].b * R + r) * 4096);
      tc::fence_smem_for_async();
      tc::fence_before();
      __syncthreads();
      tc::fence_after();
      if (tid == 0) {
        for (int x = 0; x < 2; ++x)
          if (xs[x].internal)
            tc::mma_split3<64>(tmem + 64 * x, smem_addr(C_hi[x]), smem_addr(C_lo[x]),
                               smem_addr(T_hi[x]), smem_addr(T_lo[x]));
        tc::commit(&bar);
      }
      ok = __syncthreads_and(tc_wait(&bar, parity, a.err));
      parity ^= 1u;
      tc::fence_after();
      if (!ok) break;
      for (int x = 0; x < 2; ++x) {
        if (!xs[x].internal) continue;
        float v[64];
        float m = 0.f;
#pragma unroll
        for (int s0 = 0; s0 < 64; s0 += 16) {
          float w16[16];
          tc::ld16(trow + 64 * x + s0, w16);
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            v[s0 + i] = w16[i];
            m = fmaxf(m, fabsf(w16[i]));
          }
        }
        int e = 0;
        if (valid) {
          if (!isfinite(m)) atomicOr(a.err, ERR_ZERO_PARTIAL);
          else if (m > 0.f) (void)frexpf(m, &e);
          e = max(e, -126);  // 2^-e stays finite for a subnormal maximum
        }
        const float f = ldexpf(1.f, -e);
        if (valid) {
          const size_t slot = (size_t)(xs[x].b - a.n_tips);
          float* out = a.pre + ((slot * C + c) * R + r) * 64;
#pragma unroll
          for (int i = 0; i < 64; i += 4)
            *reinterpret_cast<float4*>(out + i) =
                make_float4(v[i] * f, v[i + 1] * f, v[i + 2] * f, v[i + 3] * f);
          // q_x = P_x' (q_k o u_sibling): exponents of q_k and of the sibling
          const int sib = 1 - x;
          int eq = e + (root ? 0 : a.pre_escale[((size_t)(k - a.n_tips) * R + r) * estr + c]);
          if (xs[sib].internal)
            eq += a.escale[((size_t)(xs[sib].b - a.n_tips) * R + r) * estr + c];
          a.pre_escale[(slot * R + r) * estr + c] = eq;
        }
      }
    }
    tc::fence_before();
    __syncthreads();  // TMEM and shared tiles are reused by the next category
    tc::fence_after();
  }
  F2 gi = {0.f, 0.f}, gj = {0.f, 0.f};
  if (ok && valid) {
    if (!(Dn > 0.f) || !isfinite(Dn)) {
      atomicOr(a.err, ERR_BAD_RATIO);
    } else {
      const float W = a.pattern_wt[c];
      gi = Acc<float>::prod(W, Ni / Dn);
      gj = Acc<float>::prod(W, Nj / Dn);
    }
  }
  if (ok) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      gi = f2_add(gi, Acc<float>::shfl_down(gi, o));
      gj = f2_add(gj, Acc<float>::shfl_down(gj, o));
    }
    if (lane == 0) { red[warp][0] = gi; red[warp][1] = gj; }
  }
  tc::fence_before();
  __syncthreads();
  if (ok && tid == 0) {
    for (int w = 1; w < kTcThreads / 32; ++w) {
      gi = f2_add(gi, red[w][0]);
      gj = f2_add(gj, red[w][1]);
    }
    a.gpart[(size_t)xs[0].b * a.n_tiles + blockIdx.x] = Acc<float>::to_double(gi);
    a.gpart[(size_t)xs[1].b * a.n_tiles + blockIdx.x] = Acc<float>::to_double(gj);
  }
  if (!ok && tid == 0) (void)mbar_wait(&bar, parity ^ 1u);  // bounded drain
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, 256);
}

template <typename T = float>
inline cudaError_t launch_tc64(const LevelArgs<float>& a, bool post, cudaStream_t st) {
  dim3 grid(a.n_tiles, a.n_level);
  if (post)
    post_tc_kernel<float><<<grid, kTcThreads, kTcPostSmem, st>>>(a);
  else
    pre_tc_kernel<float><<<grid, kTcThreads, kTcPreSmem, st>>>(a);
  return cudaGetLastError();
}

template <typename T = float>
inline cudaError_t prepare_tc64() {
  cudaError_t e = cudaFuncSetAttribute(post_tc_kernel<float>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kTcPostSmem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(pre_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kTcPreSmem);
}

}  // namespace phylo
