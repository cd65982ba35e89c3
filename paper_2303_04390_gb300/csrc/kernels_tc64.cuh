// FP32 kernels for 21..64 states (codon models) on the tensor cores.
//
// The post-order pass stores, for every non-root node x that has stored
// partials, U_x = P_x p_x -- the factor node x contributes to its parent in
// Eq. 2 -- rather than p_x; a node's own p is formed from its children's U
// when its step runs.  Per (node k with children i, j; tile of 128
// patterns; category r):
//   post:  p_k = U_i o U_j  (rescaled),  U_k = p_k P_k'       (Eq. 2)
//   root:  L_c = sum_r w_r pi' (U_i o U_j)                      (Eq. 3)
//   pre, per child x with sibling y (Eq. 4 with the Eq. 8 terms):
//          a_x = q_k o U_y,   den = a_x . U_x
//          [q_x | W_x] = a_x [P_x | Q]
//          num_x = gamma_r W_x . U_x
// The numerator is Eq. 8's gamma_r q_x' Q p_x with q_x = P_x' a_x (Eq. 4):
// q_x' Q p_x = a_x' P_x Q p_x = (a_x' Q)(P_x p_x) = W_x . U_x, because
// P_x = exp(gamma_r t_x Q) (Eq. 1) commutes with Q.
// Each step is therefore one contraction of a 128-pattern tile with a
// 64 x 64 (post) or two 64 x 64 (pre) matrices, and U costs the post-order
// pass the same bytes that storing p did.
//
// The contractions are tcgen05.mma kind::f16 on BF16 operands with FP32
// accumulation in TMEM.  FP32 accuracy comes from splitting each operand
// into three BF16 terms and summing the six products of order up to 2^-16
// (tc.cuh); BF16 MMAs run at eight times the TF32 rate on this GPU.  The
// vector work (products, maxima, dot products, the splits) runs in the
// cooperative layout of coalesced row transfers, and each accumulator row
// is read back from TMEM by the thread that owns that row.
//
// Matrices.  The transition-matrix kernel of this path writes, per (branch,
// r), the operand tiles the level kernels consume, already split and in the
// K-major 128-byte-swizzle layout of tc.cuh, so a level kernel stages one
// with a single 1-D bulk copy (cp.async.bulk):
//   [P: term 0 | 1 | 2][P': term 0 | 1 | 2][P' in FP32]
// Q' (rows = columns of Q) comes from the host once per model.  A compact
// tip's U_x is its column of P, read from the FP32 P'; a gap selects the
// all-ones vector, whose Eq. 8 numerator is zero.
//
// Rescaling is per (node, pattern, category): each CTA handles one category
// of one tile, so categories are independent until Eqs. 3 and 8 combine
// them.  The pre-order CTAs write their per-category Eq. 8 terms (w_r gamma_r
// num_i, w_r gamma_r num_j, w_r den, exponent) and a final kernel forms the
// ratios, with sums over r taken relative to the largest exponent.
//   escale[node][r][c]:     cumulative exponent of p_node (and of U_node)
//   pre_escale[node][r][c]: cumulative exponent of q_node
// A tip contributes exponent 0.
//
// Every wait on an mbarrier is bounded; on expiry the kernel raises
// ERR_TIMEOUT, waits (bounded) for its copies and MMAs in flight, frees its
// TMEM and returns.
#pragma once

#include <climits>

#include "tc.cuh"

namespace phylo {

constexpr int kTcRows = kTcTilePatterns;  // patterns per tile (MMA M)
// Level kernels: two threads per pattern row, thread t owning row t % 128
// and columns [32h, 32h + 32) with h = t / 128.  Warp w reads TMEM lanes
// 32 (w % 4) .. 32 (w % 4) + 31, which are exactly its rows.
constexpr int kTcThreads = 2 * kTcRows;
static_assert(kTcRows == 128, "one accumulator lane per pattern row");

constexpr uint32_t kTerm128 = 128 * 128;  // one BF16 term of a 128 x 64 tile
constexpr uint32_t kTerm64 = 64 * 128;    // one BF16 term of a 64 x 64 tile
constexpr uint32_t kOp128 = 3 * kTerm128;  // three-term 128-row operand
constexpr uint32_t kOp64 = 3 * kTerm64;    // three-term 64-row operand
// Matrix tiles of one (branch, r) in the workspace: P (rows = rows of P)
// and P' (rows = columns of P) as three-term BF16 operands, then P' again in
// FP32 for the compact-tip lookups (row y = column y of P).
constexpr uint32_t kUnitP = 0, kUnitPt = kOp64, kUnitPt32 = 2 * kOp64;
static_assert(kTcUnitBytes == 2 * kOp64 + 64 * 64 * 4, "matrix tile block size");
static_assert(kTcQtBytes == kOp64, "Q' operand size");

// Dynamic shared memory (+1024 for the alignment of the swizzled tiles):
//   post: p_k (128-row operand, later the U_k staging) | P_k (64 rows)
//   pre:  a_x (128-row operand, later the W_x staging) | P_x' | Q' (64 rows
//         each; later the q_x staging)
constexpr size_t kPostUSmem = 1024 + kOp128 + kOp64;
// Resident CTAs per SM the post-order kernel's registers are bounded for
// (its shared memory admits three; bounding the registers for three spills and measured slower).
#ifndef PHYLO_POST_U_BLOCKS
#define PHYLO_POST_U_BLOCKS 2
#endif
// FP32 P' of one (branch, r): the compact-tip lookup table, staged by bulk copy.
constexpr uint32_t kPt32Bytes = 64 * 64 * 4;
constexpr size_t kPreUSmem = 1024 + kOp128 + 2 * kOp64;

__device__ __forceinline__ float pow2i(int d) {  // 2^d for d <= 0 (0 below 2^-126)
  return d < -126 ? 0.f : __uint_as_float((unsigned)(127 + d) << 23);
}

__device__ __forceinline__ unsigned char* align1024(unsigned char* p) {
  return reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(p) + 1023) &
                                          ~(uintptr_t)1023);
}

// Bounded wait on an mbarrier phase, agreed by the whole block; on timeout
// raise the flag and record the phase still pending.
__device__ __forceinline__ bool tc_block_wait(uint64_t* bar, uint32_t& parity, int& pending,
                                              int* err) {
  const bool mine = mbar_wait(bar, parity);
  const bool ok = __syncthreads_and(mine);
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
    pending = (int)parity;
  }
  parity ^= 1u;
  tc::fence_after();
  return ok;
}

// Cooperative, coalesced access to a 128-row tile of 64-float rows (row
// c0 + m at base + (c0 + m) * stride): in iteration it (0..3) lane l of
// warp w handles row 32 it + 4 w + l / 8 and floats 8 (l % 8) .. + 7, so a
// warp instruction touches 4 rows in full rather than 32 rows in part.
__device__ __forceinline__ int coop_row(int it) {
  return 32 * it + 4 * (int)(threadIdx.x >> 5) + (int)((threadIdx.x & 31) >> 3);
}

__device__ __forceinline__ void coop_load(float4 (&v)[8], const float* __restrict__ base,
                                          size_t stride, int c0, int C) {
  const int j = threadIdx.x & 7;
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int c = c0 + coop_row(it);
    if (c < C) {
      const float4* src = reinterpret_cast<const float4*>(base + (size_t)c * stride + 8 * j);
      v[2 * it] = __ldg(src);
      v[2 * it + 1] = __ldg(src + 1);
    } else {
      v[2 * it] = v[2 * it + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
}

// Split a cooperatively loaded tile into the three BF16 term tiles of a
// 128-row operand at `op`.
__device__ __forceinline__ void coop_put(unsigned char* op, const float4 (&v)[8]) {
  const int j = threadIdx.x & 7;
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const float x[8] = {v[2 * it].x, v[2 * it].y, v[2 * it].z, v[2 * it].w,
                        v[2 * it + 1].x, v[2 * it + 1].y, v[2 * it + 1].z, v[2 * it + 1].w};
    tc::put_split3(op, op + kTerm128, op + 2 * kTerm128, coop_row(it), j, x);
  }
}

// Row staging in shared memory for coalesced transfers: [128][kStageLd]
// floats (the 4-float pad keeps both access patterns free of bank
// conflicts).
constexpr int kStageLd = 68;
constexpr uint32_t kStageBytes = kTcRows * kStageLd * 4;

// Thread (row, h) writes its half row (32 values times f) to the staging.
__device__ __forceinline__ void stage_half(float* st, int row, int h, const float (&p)[32],
                                           float f) {
#pragma unroll
  for (int i = 0; i < 32; i += 4)
    *reinterpret_cast<float4*>(st + row * kStageLd + 32 * h + i) =
        make_float4(p[i] * f, p[i + 1] * f, p[i + 2] * f, p[i + 3] * f);
}

// Coalesced store of the staged rows: a quarter warp writes one 128-byte
// half row per instruction.
__device__ __forceinline__ void coop_store(float* __restrict__ base, size_t stride, int c0,
                                           int C, const float* st) {
  const int jj = threadIdx.x & 7;
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int row = coop_row(it), c = c0 + row;
    if (c < C) {
      float* dst = base + (size_t)c * stride;
      *reinterpret_cast<float4*>(dst + 4 * jj) =
          *reinterpret_cast<const float4*>(st + row * kStageLd + 4 * jj);
      *reinterpret_cast<float4*>(dst + 32 + 4 * jj) =
          *reinterpret_cast<const float4*>(st + row * kStageLd + 32 + 4 * jj);
    }
  }
}

// Shared addresses of the three terms of an operand.
__device__ __forceinline__ void term_addrs(const unsigned char* op, uint32_t term,
                                           uint32_t (&t)[3]) {
  const uint32_t a = smem_addr(op);
  t[0] = a;
  t[1] = a + term;
  t[2] = a + 2 * term;
}

struct TcChild {
  int b;
  bool compact;  // tip with a compact state
  bool internal;
};

__device__ __forceinline__ TcChild tc_child(int n_tips, int b, bool compact) {
  return TcChild{b, compact, b >= n_tips};
}

__device__ __forceinline__ const unsigned char* unit_tiles(const LevelArgs<float>& a, int b,
                                                           int r) {
  return reinterpret_cast<const unsigned char*>(a.P) +
         ((size_t)b * a.n_cat + r) * kTcUnitBytes;
}

// ---------------------------------------------------------------------------
// Transition matrices (Eq. 1) in double-float arithmetic
// ---------------------------------------------------------------------------
// P - I = V diag(e^{lambda gamma t} - 1) Vinv.  The exponentials come from
// FP64; the contraction runs on the FP32 pipe with every value held as an
// unevaluated sum hi + lo of two floats (Dekker's double-float arithmetic:
// products split exactly with fmaf, sums with Knuth's TwoSum), about 48
// significant bits, which keeps the small off-diagonal entries of short
// branches accurate to FP32 despite the cancellation in the sum over
// eigenvalues.  The results are rounded once to FP32 and written as the
// split operand tiles and the FP32 P'.  V and Vinv arrive as double-float
// tables built on the host.  (dP is not needed on this path: the pre-order
// step uses dP = gamma Q P through Q.)
struct DF {
  float h, l;
};

__device__ __forceinline__ DF df_from(double x) {
  const float h = (float)x;
  return DF{h, (float)(x - (double)h)};
}

// a * b with the low part carried to first order (unnormalised).
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float h = __fmul_rn(a.h, b.h);
  float l = __fmaf_rn(a.h, b.h, -h);
  l = __fmaf_rn(a.h, b.l, l);
  l = __fmaf_rn(a.l, b.h, l);
  return DF{h, l};
}

// acc += a * b
__device__ __forceinline__ void df_fma(DF& acc, DF a, DF b) {
  const DF p = df_mul(a, b);
  const float s = __fadd_rn(acc.h, p.h);
  const float bb = __fsub_rn(s, acc.h);
  const float e = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bb)), __fsub_rn(p.h, bb));
  acc.h = s;
  acc.l = __fadd_rn(acc.l, __fadd_rn(e, p.l));
}

// FP32 value of acc (+ 1 when `one`), rounded once.
__device__ __forceinline__ float df_round(DF acc, bool one) {
  if (!one) return __fadd_rn(acc.h, acc.l);
  const float s = __fadd_rn(acc.h, 1.f);
  const float bb = __fsub_rn(s, acc.h);
  const float e = __fadd_rn(__fsub_rn(acc.h, __fsub_rn(s, bb)), __fsub_rn(1.f, bb));
  return __fadd_rn(s, __fadd_rn(e, acc.l));
}

// Store 4 consecutive elements (k = k0..k0+3, k0 % 4 == 0) of row `row` of
// a three-term BF16 operand at `op` with term stride `term`.
__device__ __forceinline__ void put_split3_4(unsigned char* op, uint32_t term, int row, int k0,
                                             float4 v) {
  float x[4] = {v.x, v.y, v.z, v.w};
  const uint32_t off = tc::b16_off(row, k0);
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(x[0], x[1]);
    const __nv_bfloat162 h1 = __floats2bfloat162_rn(x[2], x[3]);
    const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
    x[0] = __fsub_rn(x[0], f0.x);
    x[1] = __fsub_rn(x[1], f0.y);
    x[2] = __fsub_rn(x[2], f1.x);
    x[3] = __fsub_rn(x[3], f1.y);
    *reinterpret_cast<uint2*>(op + t * term + off) =
        make_uint2(*reinterpret_cast<const uint32_t*>(&h0), *reinterpret_cast<const uint32_t*>(&h1));
  }
}

// Writes the 4 x 4 block P[s0 + i][t0 + j] = B[i][j] of one (branch, r) unit
// in its three forms: P rows, P' rows (split) and P' rows in FP32.
__device__ __forceinline__ void put_pblock(unsigned char* unit, int s0, int t0,
                                           const float (&B)[4][4]) {
  float* pt32 = reinterpret_cast<float*>(unit + kUnitPt32);
#pragma unroll
  for (int i = 0; i < 4; ++i)
    put_split3_4(unit + kUnitP, kTerm64, s0 + i, t0,
                 make_float4(B[i][0], B[i][1], B[i][2], B[i][3]));
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const float4 col = make_float4(B[0][j], B[1][j], B[2][j], B[3][j]);
    put_split3_4(unit + kUnitPt, kTerm64, t0 + j, s0, col);
    *reinterpret_cast<float4*>(pt32 + (t0 + j) * 64 + s0) = col;
  }
}

constexpr int kPmatTcThreads = 256;  // one 4 x 4 block of (s, t) per thread
struct PmatTcSmem {
  float vt_h[64][64], vt_l[64][64];  // V transposed: [m][s]
  float vi_h[64][64], vi_l[64][64];  // Vinv: [m][t]
  float pi_h[64], pi_l[64];          // root distribution (reversible form)
  DF e[64];
  uint64_t bar;
};
static_assert(offsetof(PmatTcSmem, e) == kEigenSplitFloats * sizeof(float),
              "the staged table is the host's eigen split");
constexpr size_t kPmatTcSmem = sizeof(PmatTcSmem);

template <typename T>  // float only
__global__ void __launch_bounds__(kPmatTcThreads) pmat_tc_kernel(PmatArgs a) {
  static_assert(std::is_same<T, float>::value, "tensor-core path is FP32");
  extern __shared__ __align__(16) unsigned char smraw[];
  PmatTcSmem& sm = *reinterpret_cast<PmatTcSmem*>(smraw);
  const int S = a.n_states, R = a.n_cat;
  const int unit = blockIdx.x, b = unit / R, r = unit % R;
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init_fenced(&sm.bar, 1);
    mbar_expect_tx(&sm.bar, (uint32_t)(kEigenSplitFloats * sizeof(float)));
    bulk_g2s(&sm.vt_h[0][0], a.vsplit, (uint32_t)(kEigenSplitFloats * sizeof(float)), &sm.bar);
  }
  if (tid < 64) {
    double e = 0.0;
    if (tid < S) {
      double t = a.t[b];
      if (!(t >= 0.0) || !isfinite(t)) {
        if (tid == 0 && r == 0) atomicOr(a.err, ERR_BAD_LENGTH);
        t = 0.0;
      }
      e = expm1(a.lambda[tid] * a.rates[r] * t);
    }
    sm.e[tid] = df_from(e);
  }
  __syncthreads();  // barrier initialised, exponentials staged
  const bool ok = __syncthreads_and(mbar_wait(&sm.bar, 0));
  if (!ok) {  // bounded drain, then give up on this unit
    if (tid == 0) {
      atomicOr(a.err, ERR_TIMEOUT);
      (void)mbar_wait(&sm.bar, 0);
    }
    return;
  }
  unsigned char* base = static_cast<unsigned char*>(a.P) + (size_t)unit * kTcUnitBytes;
  if (a.reversible) {
    // Vinv[m][t] = pi_t V[t][m]: P - I = K diag(pi) with K = V diag(e) V'
    // symmetric, so only the 136 blocks (sb <= tb) of the 16 x 16 grid of
    // 4 x 4 blocks are contracted; each writes itself and its mirror
    // P[t][s] = pi_s K_st.
    if (tid >= 136) return;
    int sb = 0, rem = tid;
    while (rem >= 16 - sb) {
      rem -= 16 - sb;
      ++sb;
    }
    const int tb = sb + rem, s0 = 4 * sb, t0 = 4 * tb;
    DF kP[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) kP[i][j] = DF{0.f, 0.f};
    for (int m = 0; m < S; ++m) {
      const float4 sh = *reinterpret_cast<const float4*>(&sm.vt_h[m][s0]);
      const float4 sl = *reinterpret_cast<const float4*>(&sm.vt_l[m][s0]);
      const float4 th = *reinterpret_cast<const float4*>(&sm.vt_h[m][t0]);
      const float4 tl = *reinterpret_cast<const float4*>(&sm.vt_l[m][t0]);
      const DF em = sm.e[m];
      const DF v[4] = {{sh.x, sl.x}, {sh.y, sl.y}, {sh.z, sl.z}, {sh.w, sl.w}};
      const DF w[4] = {{th.x, tl.x}, {th.y, tl.y}, {th.z, tl.z}, {th.w, tl.w}};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const DF ve = df_mul(v[i], em);
#pragma unroll
        for (int j = 0; j < 4; ++j) df_fma(kP[i][j], ve, w[j]);
      }
    }
    float P[4][4], Pm[4][4];  // block (sb, tb) and its mirror (tb, sb)
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int s = s0 + i, t = t0 + j;
        const DF pt = {sm.pi_h[t], sm.pi_l[t]}, ps = {sm.pi_h[s], sm.pi_l[s]};
        P[i][j] = df_round(df_mul(kP[i][j], pt), s == t && s < S);
        Pm[j][i] = df_round(df_mul(kP[i][j], ps), s == t && s < S);
      }
    put_pblock(base, s0, t0, P);
    if (sb != tb) put_pblock(base, t0, s0, Pm);
    return;
  }
  const int s0 = 4 * (tid / 16), t0 = 4 * (tid % 16);
  DF acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = DF{0.f, 0.f};
  for (int m = 0; m < S; ++m) {
    const float4 vh = *reinterpret_cast<const float4*>(&sm.vt_h[m][s0]);
    const float4 vl = *reinterpret_cast<const float4*>(&sm.vt_l[m][s0]);
    const float4 ih = *reinterpret_cast<const float4*>(&sm.vi_h[m][t0]);
    const float4 il = *reinterpret_cast<const float4*>(&sm.vi_l[m][t0]);
    const DF em = sm.e[m];
    const DF v[4] = {{vh.x, vl.x}, {vh.y, vl.y}, {vh.z, vl.z}, {vh.w, vl.w}};
    const DF w[4] = {{ih.x, il.x}, {ih.y, il.y}, {ih.z, il.z}, {ih.w, il.w}};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const DF ve = df_mul(v[i], em);
#pragma unroll
      for (int j = 0; j < 4; ++j) df_fma(acc[i][j], ve, w[j]);
    }
  }
  float P[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int s = s0 + i, t = t0 + j;
      P[i][j] = df_round(acc[i][j], s == t && s < S);
    }
  put_pblock(base, s0, t0, P);
}

// ---------------------------------------------------------------------------
// Stored U rows and their exponents
// ---------------------------------------------------------------------------
// U slot of node x: internal nodes in slot x - N, tips with partial
// vectors in slot N - 1 + x; each slot is [c][r][64] floats.
__device__ __forceinline__ size_t u_slot(const LevelArgs<float>& a, int x) {
  return x >= a.n_tips ? (size_t)(x - a.n_tips) : (size_t)(a.n_tips - 1 + x);
}

__device__ __forceinline__ float* u_rows(const LevelArgs<float>& a, int x, int r) {
  return a.post + (u_slot(a, x) * a.n_patterns * a.n_cat + r) * 64;
}

// Rows c0 + coop_row(it) of U_x for a child x, in the cooperative layout
// (floats 8 j .. 8 j + 7, j = lane % 8), in two steps.  coop_child_u_issue
// loads the stored rows of a non-compact child with each row's exponent
// (0 for a tip), or the states of a compact tip; coop_child_u_finish then
// fills a compact tip's rows from its FP32 P' staged in shared memory: U_x
// is column y of P_x, i.e. row y of P'; a gap (y = S) gives the all-ones
// vector over the S states.  Rows past the last pattern are zero (y = -1).
struct UFetch {
  float4 v[8];
  int E[4], y[4];
};

__device__ __forceinline__ void coop_child_u_issue(UFetch& f, const LevelArgs<float>& a,
                                                   const TcChild& x, int r, int c0) {
  const int C = a.n_patterns;
  if (!x.compact) {
    coop_load(f.v, u_rows(a, x.b, r), (size_t)a.n_cat * 64, c0, C);
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int c = c0 + coop_row(it);
      f.y[it] = -1;
      f.E[it] = x.internal && c < C
                    ? a.escale[((size_t)(x.b - a.n_tips) * a.n_cat + r) * a.escale_stride + c]
                    : 0;
    }
    return;
  }
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int c = c0 + coop_row(it);
    f.y[it] = c < C ? (int)a.tip_states[(size_t)x.b * a.state_stride + c] : -1;
    f.E[it] = 0;
  }
}

__device__ __forceinline__ void coop_child_u_finish(UFetch& f, bool compact, const float* pt32,
                                                    int S) {
  if (!compact) return;
  const int j = threadIdx.x & 7;
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int yy = f.y[it];
    if (yy >= 0 && yy < S) {
      const float4* src = reinterpret_cast<const float4*>(pt32 + yy * 64 + 8 * j);
      f.v[2 * it] = src[0];
      f.v[2 * it + 1] = src[1];
    } else {
      const float g = yy < 0 ? 0.f : 1.f;  // past the last pattern, or a gap
      const int s = 8 * j;
      f.v[2 * it] = make_float4(s < S ? g : 0.f, s + 1 < S ? g : 0.f, s + 2 < S ? g : 0.f,
                                s + 3 < S ? g : 0.f);
      f.v[2 * it + 1] = make_float4(s + 4 < S ? g : 0.f, s + 5 < S ? g : 0.f,
                                    s + 6 < S ? g : 0.f, s + 7 < S ? g : 0.f);
    }
  }
}

__device__ __forceinline__ float4 mul4(float4 a, float4 b) {
  return make_float4(a.x * b.x, a.y * b.y, a.z * b.z, a.w * b.w);
}
__device__ __forceinline__ float dot4(float4 a, float4 b, float acc) {
  return fmaf(a.w, b.w, fmaf(a.z, b.z, fmaf(a.y, b.y, fmaf(a.x, b.x, acc))));
}
__device__ __forceinline__ float amax4(float4 a, float m) {
  return fmaxf(fmaxf(fmaxf(m, fabsf(a.x)), fmaxf(fabsf(a.y), fabsf(a.z))), fabsf(a.w));
}
// Sum / maximum over the 8 lanes that share a row in the cooperative layout.
__device__ __forceinline__ float row_sum8(float x) {
  x += __shfl_xor_sync(kFull, x, 1);
  x += __shfl_xor_sync(kFull, x, 2);
  return x + __shfl_xor_sync(kFull, x, 4);
}
__device__ __forceinline__ float row_max8(float x) {
  x = fmaxf(x, __shfl_xor_sync(kFull, x, 1));
  x = fmaxf(x, __shfl_xor_sync(kFull, x, 2));
  return fmaxf(x, __shfl_xor_sync(kFull, x, 4));
}

// Power-of-two exponent that brings a row maximum m into [1/2, 1) (0 for a
// zero row; never below -126, so that 2^-e stays finite); flags a NaN or
// infinite maximum.
__device__ __forceinline__ int rescale_exponent(float m, bool valid, int* err) {
  int e = 0;
  if (valid) {
    if (!isfinite(m)) atomicOr(err, ERR_ZERO_PARTIAL);
    else if (m > 0.f) (void)frexpf(m, &e);
    e = max(e, -126);
  }
  return e;
}

// ---------------------------------------------------------------------------
// Post-order level (Eq. 2), every level but the root's; with `tip_level`
// the level's nodes are tips with partial vectors, whose U = P p is formed
// from those vectors before the first level runs.
// ---------------------------------------------------------------------------
template <typename T>  // float only
__global__ void __launch_bounds__(kTcThreads, PHYLO_POST_U_BLOCKS) post_u_kernel(LevelArgs<T> a) {
  static_assert(std::is_same<T, float>::value, "tensor-core path is FP32");
  static_assert(kStageBytes <= kOp128, "staging fits in the operand buffer");
  static_assert(2 * kPt32Bytes <= kOp128, "staged lookup tables fit in the operand buffer");
  extern __shared__ unsigned char smraw[];
  unsigned char* base = align1024(smraw);
  unsigned char* A = base;            // p_k as three BF16 terms
  unsigned char* B = base + kOp128;   // P_k (rows = rows of P)
  float* stage = reinterpret_cast<float*>(A);  // U_k rows, after the MMAs
  // before the split, A holds the FP32 P' of the compact children (lookups)
  const float* pt32[2] = {reinterpret_cast<const float*>(A),
                          reinterpret_cast<const float*>(A + kPt32Bytes)};
  __shared__ uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid & (kTcRows - 1), h = tid / kTcRows;
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int4 d = a.level_desc[blockIdx.y];
  const int k = d.x, r = blockIdx.z;
  const int c0 = blockIdx.x * kTcRows;
  const bool tip = a.tip_level;
  const TcChild xs[2] = {tc_child(a.n_tips, d.y, d.w & kDescFlagCompact0),
                         tc_child(a.n_tips, d.z, d.w & kDescFlagCompact1)};
  // The descriptor (host-written) is read before the wait; so are the
  // matrix tiles when the launch before this one is not the matrix kernel.
  auto issue_operands = [&] {
    if (tid != 0) return;
    mbar_init_fenced(&bar_tma, 1);
    mbar_init_fenced(&bar_mma, 1);
    uint32_t bytes = kOp64;
    if (!tip)
      for (int x = 0; x < 2; ++x) bytes += xs[x].compact ? kPt32Bytes : 0;
    mbar_expect_tx(&bar_tma, bytes);
    bulk_g2s(B, unit_tiles(a, k, r) + kUnitP, kOp64, &bar_tma);
    if (!tip)
      for (int x = 0; x < 2; ++x)
        if (xs[x].compact)
          bulk_g2s(A + x * kPt32Bytes, unit_tiles(a, xs[x].b, r) + kUnitPt32, kPt32Bytes,
                   &bar_tma);
  };
  if (a.mats_ready) issue_operands();
  pdl_wait_and_release();  // before TMEM or any other global access
  if (!a.mats_ready) issue_operands();
  // every global load is issued before the first wait
  UFetch f0, f1;
  if (tip) {
    coop_load(f0.v, a.tip_partials + (size_t)k * C * 64, 64, c0, C);
  } else {
    coop_child_u_issue(f0, a, xs[0], r, c0);
    coop_child_u_issue(f1, a, xs[1], r, c0);
  }
  if (warp == 0) tc::alloc(&tmem_slot, 64);
  __syncthreads();  // barriers initialised, TMEM allocated
  tc::fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  uint32_t ptma = 0, pmma = 0;
  int pend_tma = -1, pend_mma = -1;
  bool ok = tc_block_wait(&bar_tma, ptma, pend_tma, a.err);
  if (ok) {
    if (!tip) {
      // p_k = U_i o U_j, each row rescaled into [1/2, 1)
      coop_child_u_finish(f0, xs[0].compact, pt32[0], S);
      coop_child_u_finish(f1, xs[1].compact, pt32[1], S);
#pragma unroll
      for (int it = 0; it < 4; ++it) {
        float4& v0 = f0.v[2 * it];
        float4& v1 = f0.v[2 * it + 1];
        v0 = mul4(v0, f1.v[2 * it]);
        v1 = mul4(v1, f1.v[2 * it + 1]);
        const float m = row_max8(amax4(v1, amax4(v0, 0.f)));
        const int c = c0 + coop_row(it);
        const int e = rescale_exponent(m, c < C, a.err);
        const float sc = ldexpf(1.f, -e);
        v0 = make_float4(v0.x * sc, v0.y * sc, v0.z * sc, v0.w * sc);
        v1 = make_float4(v1.x * sc, v1.y * sc, v1.z * sc, v1.w * sc);
        if (c < C && (lane & 7) == 0)
          a.escale[((size_t)(k - a.n_tips) * R + r) * a.escale_stride + c] =
              f0.E[it] + f1.E[it] + e;
      }
      __syncthreads();  // every lookup in A is done before the split overwrites it
    }
    coop_put(A, f0.v);
    tc::fence_smem_for_async();
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      uint32_t ta[3], tb[3];
      term_addrs(A, kTerm128, ta);
      term_addrs(B, kTerm64, tb);
      tc::mma_split_bf16x3<64>(tmem, ta, tb);
      tc::commit(&bar_mma);
    }
    ok = tc_block_wait(&bar_mma, pmma, pend_mma, a.err);
  }
  if (ok) {  // U_k = p_k P_k', stored as computed (exponent: escale of k)
    float u[32];
    tc::ld32(trow + 32 * h, u);
    stage_half(stage, row, h, u, 1.f);
    __syncthreads();
    coop_store(u_rows(a, k, r), (size_t)R * 64, c0, C, stage);
  }
  if (tid == 0) {  // bounded drain of whatever a timeout left in flight
    if (pend_tma >= 0) (void)mbar_wait(&bar_tma, (uint32_t)pend_tma);
    if (pend_mma >= 0) (void)mbar_wait(&bar_mma, (uint32_t)pend_mma);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, 64);
}

// ---------------------------------------------------------------------------
// Root (Eq. 3): L_c = sum_r w_r 2^(E_i + E_j) pi' (U_i o U_j), one thread
// per pattern, categories summed relative to the largest exponent; the
// tile's sum of W_c log L_c goes to lpart.
// ---------------------------------------------------------------------------
template <typename T>  // float only
__global__ void __launch_bounds__(kTcRows) root_u_kernel(LevelArgs<T> a) {
  static_assert(std::is_same<T, float>::value, "tensor-core path is FP32");
  pdl_wait_and_release();  // before any global access
  __shared__ double lred[kTcRows / 32];
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int4 d = a.level_desc[0];
  const TcChild xs[2] = {tc_child(a.n_tips, d.y, d.w & kDescFlagCompact0),
                         tc_child(a.n_tips, d.z, d.w & kDescFlagCompact1)};
  const int c = blockIdx.x * kTcRows + threadIdx.x, lane = threadIdx.x & 31;
  double term = 0.0;
  if (c < C) {
    int y[2] = {-1, -1};
    for (int x = 0; x < 2; ++x)
      if (xs[x].compact) y[x] = a.tip_states[(size_t)xs[x].b * a.state_stride + c];
    float lsum = 0.f;
    int lexp = INT_MIN / 2;
    for (int r = 0; r < R; ++r) {
      const float4* src[2];
      int E = 0;
      for (int x = 0; x < 2; ++x) {
        src[x] = nullptr;  // a gap: the all-ones vector
        if (!xs[x].compact) {
          src[x] = reinterpret_cast<const float4*>(u_rows(a, xs[x].b, r) + (size_t)c * R * 64);
          if (xs[x].internal)
            E += a.escale[((size_t)(xs[x].b - a.n_tips) * R + r) * a.escale_stride + c];
        } else if (y[x] < S) {
          src[x] = reinterpret_cast<const float4*>(
              reinterpret_cast<const float*>(unit_tiles(a, xs[x].b, r) + kUnitPt32) +
              y[x] * 64);
        }
      }
      float dot = 0.f;
#pragma unroll 4
      for (int q4 = 0; q4 < 16; ++q4) {
        const float4 ones = make_float4(1.f, 1.f, 1.f, 1.f);
        const float4 u0 = src[0] ? __ldg(src[0] + q4) : ones;
        const float4 u1 = src[1] ? __ldg(src[1] + q4) : ones;
        const int s = 4 * q4;
        const float4 pi4 = make_float4(s < S ? a.root_pit[s] : 0.f,
                                       s + 1 < S ? a.root_pit[s + 1] : 0.f,
                                       s + 2 < S ? a.root_pit[s + 2] : 0.f,
                                       s + 3 < S ? a.root_pit[s + 3] : 0.f);
        dot = dot4(mul4(u0, u1), pi4, dot);
      }
      if (dot != 0.f) {
        // L_c = sum_r w_r 2^E_r (pi' p_r): running sum relative to the largest E
        const float t = a.cat_wt[r] * dot;
        if (E > lexp) {
          lsum = lsum * pow2i(lexp - E) + t;
          lexp = E;
        } else {
          lsum += t * pow2i(E - lexp);
        }
      }
    }
    if (!(lsum > 0.f) || !isfinite(lsum)) atomicOr(a.err, ERR_ZERO_PARTIAL);
    term = (double)a.pattern_wt[c] * (log((double)lsum) + (double)lexp * 0.69314718055994530942);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) term += __shfl_down_sync(kFull, term, o);
  if (lane == 0) lred[threadIdx.x >> 5] = term;
  __syncthreads();
  if (threadIdx.x == 0) {
    double l = 0.0;
    for (int w = 0; w < kTcRows / 32; ++w) l += lred[w];
    a.lpart[blockIdx.x] = l;
  }
}

// ---------------------------------------------------------------------------
// Pre-order level (Eq. 4) with the per-category Eq. 8 terms: one CTA per
// (tile, node k, category r, child x); blockIdx.z = 2 r + x.
// ---------------------------------------------------------------------------
template <typename T>  // float only
__global__ void __launch_bounds__(kTcThreads, 2) pre_u_kernel(LevelArgs<T> a) {
  static_assert(std::is_same<T, float>::value, "tensor-core path is FP32");
  static_assert(kStageBytes <= kOp128 && kStageBytes <= 2 * kOp64, "staging fits");
  static_assert(kPt32Bytes <= kOp64, "a lookup table fits in the P' buffer");
  extern __shared__ unsigned char smraw[];
  unsigned char* base = align1024(smraw);
  unsigned char* A = base;                     // a_x as three BF16 terms
  unsigned char* Bp = base + kOp128;           // P_x' (rows = columns of P_x)
  unsigned char* Bq = base + kOp128 + kOp64;   // Q' (rows = columns of Q)
  float* stW = reinterpret_cast<float*>(A);    // W_x rows, after the MMAs
  float* stQ = reinterpret_cast<float*>(Bp);   // q_x rows, after the MMAs
  // lookup tables of compact children (FP32 P'): the sibling's in A until
  // the split, the child's own in Bp (unused by a tip child's MMA)
  const float* pt32x = reinterpret_cast<const float*>(Bp);
  const float* pt32y = reinterpret_cast<const float*>(A);
  __shared__ uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_slot;
  __shared__ int eexp[kTcRows];      // each row's rescale exponent of q_x
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, j = lane & 7;
  const int row = tid & (kTcRows - 1), h = tid / kTcRows;
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int4 d = a.level_desc[blockIdx.y];
  const int k = d.x, x = (int)(blockIdx.z & 1), r = (int)(blockIdx.z >> 1);
  const TcChild cx = tc_child(a.n_tips, x ? d.z : d.y,
                              d.w & (x ? kDescFlagCompact1 : kDescFlagCompact0));
  const TcChild cy = tc_child(a.n_tips, x ? d.y : d.z,
                              d.w & (x ? kDescFlagCompact0 : kDescFlagCompact1));
  const bool root = k == a.root;
  const size_t kslot = (size_t)(k - a.n_tips);
  const int c0 = blockIdx.x * kTcRows;
  const int estr = a.escale_stride;
  // The descriptor, Q' and the category constants (all written before the
  // matrix kernel ran) are read before the wait; so are the matrix tiles
  // when the launch before this one is not the matrix kernel.
  auto issue_operands = [&] {
    if (tid != 0) return;
    mbar_init_fenced(&bar_tma, 1);
    mbar_init_fenced(&bar_mma, 1);
    mbar_expect_tx(&bar_tma, kOp64 + (cx.internal ? kOp64 : 0) +
                                 (cx.compact ? kPt32Bytes : 0) + (cy.compact ? kPt32Bytes : 0));
    bulk_g2s(Bq, a.qt, kOp64, &bar_tma);
    if (cx.internal) bulk_g2s(Bp, unit_tiles(a, cx.b, r) + kUnitPt, kOp64, &bar_tma);
    if (cx.compact)
      bulk_g2s(Bp, unit_tiles(a, cx.b, r) + kUnitPt32, kPt32Bytes, &bar_tma);
    if (cy.compact)
      bulk_g2s(A, unit_tiles(a, cy.b, r) + kUnitPt32, kPt32Bytes, &bar_tma);
  };
  const double cw = a.cat_w[r], rate = a.rates[r];  // used in the epilogue
  const float wr = a.cat_wt[r];
  if (a.mats_ready) issue_operands();
  pdl_wait_and_release();  // before TMEM or any other global access
  if (!a.mats_ready) issue_operands();
  // every global load is issued before the first wait
  float4 q[8];
  int eq[4];
  if (!root) {
    coop_load(q, a.pre + (kslot * C * R + r) * 64, (size_t)R * 64, c0, C);
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int c = c0 + coop_row(it);
      eq[it] = c < C ? a.pre_escale[(kslot * R + r) * estr + c] : 0;
    }
  } else {  // q_root = pi
    const int s = 8 * j;
    const float4 p0 = make_float4(s < S ? a.root_pit[s] : 0.f, s + 1 < S ? a.root_pit[s + 1] : 0.f,
                                  s + 2 < S ? a.root_pit[s + 2] : 0.f,
                                  s + 3 < S ? a.root_pit[s + 3] : 0.f);
    const float4 p1 = make_float4(s + 4 < S ? a.root_pit[s + 4] : 0.f,
                                  s + 5 < S ? a.root_pit[s + 5] : 0.f,
                                  s + 6 < S ? a.root_pit[s + 6] : 0.f,
                                  s + 7 < S ? a.root_pit[s + 7] : 0.f);
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      q[2 * it] = p0;
      q[2 * it + 1] = p1;
      eq[it] = 0;
    }
  }
  UFetch fx, fy;
  coop_child_u_issue(fx, a, cx, r, c0);
  coop_child_u_issue(fy, a, cy, r, c0);
  if (warp == 0) tc::alloc(&tmem_slot, 128);
  __syncthreads();  // barriers initialised, TMEM allocated
  tc::fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  uint32_t ptma = 0, pmma = 0;
  int pend_tma = -1, pend_mma = -1;
  bool ok = tc_block_wait(&bar_tma, ptma, pend_tma, a.err);
  float den[4];
  if (ok) {
    coop_child_u_finish(fx, cx.compact, pt32x, S);
    coop_child_u_finish(fy, cy.compact, pt32y, S);
    // a_x = q_k o U_y (into q) and den = a_x . U_x per row
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      q[2 * it] = mul4(q[2 * it], fy.v[2 * it]);
      q[2 * it + 1] = mul4(q[2 * it + 1], fy.v[2 * it + 1]);
      den[it] = row_sum8(dot4(q[2 * it + 1], fx.v[2 * it + 1], dot4(q[2 * it], fx.v[2 * it], 0.f)));
    }
    __syncthreads();  // every lookup in A is done before the split overwrites it
    coop_put(A, q);
    tc::fence_smem_for_async();
    __syncthreads();
    if (tid == 0) {  // TMEM columns [q_x | W_x]
      tc::fence_after();
      uint32_t ta[3], tb[3];
      term_addrs(A, kTerm128, ta);
      term_addrs(Bq, kTerm64, tb);
      tc::mma_split_bf16x3<64>(tmem + 64, ta, tb);
      if (cx.internal) {
        term_addrs(Bp, kTerm64, tb);
        tc::mma_split_bf16x3<64>(tmem, ta, tb);
      }
      tc::commit(&bar_mma);
    }
    ok = tc_block_wait(&bar_mma, pmma, pend_mma, a.err);
  }
  if (ok) {
    // the second half of the threads stages W_x, the first half q_x (one
    // thread per row: the row maximum needs no exchange)
    if (h == 1) {
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        float w[32];
        tc::ld32(trow + 64 + 32 * hh, w);
#pragma unroll
        for (int i = 0; i < 32; i += 4)
          *reinterpret_cast<float4*>(stW + row * kStageLd + 32 * hh + i) =
              make_float4(w[i], w[i + 1], w[i + 2], w[i + 3]);
      }
    } else if (cx.internal) {  // q_x = a_x P_x, each row rescaled into [1/2, 1)
      float q0[32], q1[32];
      tc::ld32(trow, q0);
      tc::ld32(trow + 32, q1);
      float m = 0.f;
#pragma unroll
      for (int i = 0; i < 32; ++i) m = fmaxf(m, fmaxf(fabsf(q0[i]), fabsf(q1[i])));
      const int e = rescale_exponent(m, c0 + row < C, a.err);
      const float f = ldexpf(1.f, -e);
      stage_half(stQ, row, 0, q0, f);
      stage_half(stQ, row, 1, q1, f);
      eexp[row] = e;
    }
    __syncthreads();
    // num_x = W_x . U_x per row; the Eq. 8 terms of this category
    const float wg = (float)(cw * rate);
    float* rt = reinterpret_cast<float*>(a.rterm);
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int rr = coop_row(it), c = c0 + rr;
      const float4 w0 = *reinterpret_cast<const float4*>(stW + rr * kStageLd + 8 * j);
      const float4 w1 = *reinterpret_cast<const float4*>(stW + rr * kStageLd + 8 * j + 4);
      float num = row_sum8(dot4(w1, fx.v[2 * it + 1], dot4(w0, fx.v[2 * it], 0.f)));
      if (cx.compact && fx.y[it] >= S) num = 0.f;  // d/dt of the all-ones vector is 0
      if (c < C && j == 0) {
        float* t4 = rt + ((kslot * C + c) * R + r) * 4;
        t4[x] = wg * num;
        if (x == 0) {
          t4[2] = wr * den[it];
          t4[3] = __int_as_float(eq[it] + fx.E[it] + fy.E[it]);
        }
        if (cx.internal)  // q_x = P_x' (q_k o U_y): exponents of q_k and of U_y
          a.pre_escale[((size_t)(cx.b - a.n_tips) * R + r) * estr + c] =
              eexp[rr] + eq[it] + fy.E[it];
      }
    }
    if (cx.internal)
      coop_store(a.pre + ((size_t)(cx.b - a.n_tips) * C * R + r) * 64, (size_t)R * 64, c0, C,
                 stQ);
  }
  if (tid == 0) {  // bounded drain of whatever a timeout left in flight
    if (pend_tma >= 0) (void)mbar_wait(&bar_tma, (uint32_t)pend_tma);
    if (pend_mma >= 0) (void)mbar_wait(&bar_mma, (uint32_t)pend_mma);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, 128);
}

// ---------------------------------------------------------------------------
// Eq. 8 ratios and their per-tile sums (Eq. 7) for both children of every
// internal node, from the per-category terms of the pre-order kernels.
// ---------------------------------------------------------------------------
template <typename T>  // float only
__global__ void __launch_bounds__(kTcRows) ratio_tc_kernel(LevelArgs<T> a) {
  static_assert(std::is_same<T, float>::value, "tensor-core path is FP32");
  pdl_wait_and_release();  // before TMEM, smem or any global access
  __shared__ F2 red[kTcRows / 32][2];
  const int R = a.n_cat, C = a.n_patterns;
  const size_t slot = blockIdx.y;
  const int2 ch = a.children[a.n_tips + (int)slot];
  const int c = blockIdx.x * kTcRows + threadIdx.x;
  F2 gi = {0.f, 0.f}, gj = {0.f, 0.f};
  if (c < C) {
    const float4* src = reinterpret_cast<const float4*>(a.rterm) + (slot * C + c) * R;
    float Ni = 0.f, Nj = 0.f, Dn = 0.f;
    int g = INT_MIN / 2;
    for (int r = 0; r < R; ++r) {
      const float4 t = src[r];
      // a category whose terms all vanish carries an arbitrary exponent
      if (t.x == 0.f && t.y == 0.f && t.z == 0.f) continue;
      const int E = __float_as_int(t.w);
      if (E > g) {
        const float sc = pow2i(g - E);
        Ni = Ni * sc + t.x;
        Nj = Nj * sc + t.y;
        Dn = Dn * sc + t.z;
        g = E;
      } else {
        const float sc = pow2i(E - g);
        Ni += t.x * sc;
        Nj += t.y * sc;
        Dn += t.z * sc;
      }
    }
    if (!(Dn > 0.f) || !isfinite(Dn)) {
      atomicOr(a.err, ERR_BAD_RATIO);
    } else {
      const float W = a.pattern_wt[c];
      gi = Acc<float>::prod(W, Ni / Dn);
      gj = Acc<float>::prod(W, Nj / Dn);
    }
  }
  block_sum_acc<float, kTcRows>(gi, gj, red, 1);
  if (threadIdx.x == 0) {
    a.gpart[(size_t)ch.x * a.n_tiles + blockIdx.x] = Acc<float>::to_double(gi);
    a.gpart[(size_t)ch.y * a.n_tiles + blockIdx.x] = Acc<float>::to_double(gj);
  }
}

template <typename T = float>
inline cudaError_t launch_tc64(const LevelArgs<float>& a, bool post, cudaStream_t st) {
  if (post && a.root_level)
    return launch_pdl(root_u_kernel<float>, dim3(a.n_tiles), kTcRows, 0, st, a);
  if (post)
    return launch_pdl(post_u_kernel<float>, dim3(a.n_tiles, a.n_level, a.n_cat), kTcThreads,
                      kPostUSmem, st, a);
  return launch_pdl(pre_u_kernel<float>, dim3(a.n_tiles, a.n_level, 2 * a.n_cat), kTcThreads,
                    kPreUSmem, st, a);
}

template <typename T = float>
inline cudaError_t launch_ratio_tc64(const LevelArgs<float>& a, cudaStream_t st) {
  if (a.n_tiles <= 0 || a.n_tips < 2) return cudaSuccess;
  dim3 grid(a.n_tiles, a.n_tips - 1);
  return launch_pdl(ratio_tc_kernel<float>, grid, kTcRows, 0, st, a);
}

template <typename T = float>
inline cudaError_t launch_pmat_tc64(const PmatArgs& a, cudaStream_t st) {
  const int units = a.n_branches * a.n_cat;
  if (units <= 0) return cudaSuccess;
  // the reversible form has 136 blocks of (s, t) per unit: 5 warps
  pmat_tc_kernel<float><<<units, a.reversible ? 160 : kPmatTcThreads, kPmatTcSmem, st>>>(a);
  return cudaGetLastError();
}

template <typename T = float>
inline cudaError_t prepare_tc64() {
  cudaError_t e = cudaFuncSetAttribute(post_u_kernel<float>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kPostUSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pre_u_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPreUSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pmat_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPmatTcSmem);
  return e;
}

}  // namespace phylo
