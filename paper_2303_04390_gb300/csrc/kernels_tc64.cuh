// FP32 kernels for 21..64 states (codon models) on the tensor cores.
//
// Arithmetic of Eq. 2 (with Eq. 3 at the root) and Eq. 4 with the Eq. 8
// terms, per (node, tile of 128 patterns, category r):
//   post:  U_x = p_x P_x'            (x = the non-compact children)
//          p_k = U_i o U_j
//   pre:   [U_x | V_x] = p_x [P_x ; dP_x]'
//          a_i = q_k o U_j,  a_j = q_k o U_i
//          num_x = a_x . V_x,  den = a_i . U_i      (per pattern)
//          q_i = a_i P_i,  q_j = a_j P_j             (internal children)
// Every product with a partial tile is a 128 x N x 64 contraction issued as
// tcgen05.mma kind::f16 on BF16 operands with FP32 accumulation in TMEM.
// FP32 accuracy comes from splitting each operand into three BF16 terms
// and summing the six products of order up to 2^-16 (tc.cuh); BF16 MMAs
// run at eight times the TF32 rate on this GPU, so the six cost less
// tensor time than a three-pass TF32 split.  After each contraction one
// thread per pattern reads its accumulator row back from TMEM, so
// products, dot products and the rescale are thread-local.
//
// Matrices.  The transition-matrix kernel of this path writes, per (branch,
// r), the operand tiles the level kernels consume, already split and in the
// K-major 128-byte-swizzle layout of tc.cuh, so a level kernel stages them
// with 1-D bulk copies (cp.async.bulk) that overlap its partial loads:
//   [PdP term 0 | term 1 | term 2 | Pt term 0 | term 1 | term 2]
//   PdP: 128-row tile, rows 0..63 = rows of P, rows 64..127 = rows of dP
//   Pt:  64-row tile, row t = column t of P
// A compact tip reads its column of P or dP out of the staged tiles.
//
// Rescaling is per (node, pattern, category): each category's vector gets
// its own power of two, so categories are independent until Eqs. 3 and 8
// combine them.  Each CTA handles one category of one tile (grid z = r),
// except the root's post-order CTA, which loops over the categories and
// forms log L_c.  The pre-order CTAs write their per-category Eq. 8 terms
// (w_r num_i, w_r num_j, w_r den, exponent) and a final kernel forms the
// ratios, with sums over r taken relative to the largest exponent.
//   escale[node][r][c]:     cumulative post-order exponent of p_node,r,c
//   pre_escale[node][r][c]: cumulative pre-order exponent of q_node,r,c
// A tip child contributes exponent 0.
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
// Matrix tiles of one (branch, r) in the workspace.
constexpr uint32_t kUnitPdp = 0, kUnitPt = kOp128;
static_assert(kTcUnitBytes == kOp128 + kOp64, "matrix tile block size");

// Dynamic shared memory (+1024 for the alignment of the swizzled tiles):
//   post: A_i, A_j (48 KB each) | B_i, B_j (P, 24 KB each)
//   pre:  A_i, A_j (48 KB each; later Pt_i, Pt_j) | PdP_i, PdP_j (48 KB
//         each; later a_i, a_j as A operands)
constexpr size_t kTcPostSmem = 1024 + 2 * kOp128 + 2 * kOp64;
//   pipelined post: A_i, A_j | B for the current and the next item
constexpr size_t kTcPipePostSmem = 1024 + 2 * kOp128 + 4 * kOp64;
constexpr size_t kTcPreSmem = 1024 + 4 * kOp128;

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

// Write a cooperatively loaded tile into the staging (raw FP32).
__device__ __forceinline__ void coop_stage(float* st, const float4 (&v)[8]) {
  const int j = threadIdx.x & 7;
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    float* d = st + coop_row(it) * kStageLd + 8 * j;
    *reinterpret_cast<float4*>(d) = v[2 * it];
    *reinterpret_cast<float4*>(d + 4) = v[2 * it + 1];
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

// First row (pattern 0, category r) of a non-compact child's partials and
// the row stride, in floats.
__device__ __forceinline__ const float* child_base(const LevelArgs<float>& a, const TcChild& x,
                                                   int r, size_t* stride) {
  const int C = a.n_patterns;
  if (x.internal) {
    *stride = (size_t)a.n_cat * 64;
    return a.post + ((size_t)(x.b - a.n_tips) * C * a.n_cat + r) * 64;
  }
  *stride = 64;
  return a.tip_partials + (size_t)x.b * C * 64;
}

__device__ __forceinline__ const unsigned char* unit_tiles(const LevelArgs<float>& a, int b,
                                                           int r) {
  return reinterpret_cast<const unsigned char*>(a.P) +
         ((size_t)b * a.n_cat + r) * kTcUnitBytes;
}

// 32 accumulator columns of this thread's row, or for a compact tip the
// matching entries (states s0..s0+31) of its matrix column (rows row0 + s
// of a staged three-term operand with term stride `term`; a gap selects
// the all-ones vector).
__device__ __forceinline__ void child_cols(const TcChild& x, int y, int S, uint32_t taddr,
                                           const unsigned char* op, uint32_t term, int row0,
                                           int s0, float (&u)[32]) {
  if (!x.compact) {
    tc::ld32(taddr, u);
    return;
  }
#pragma unroll
  for (int i = 0; i < 32; ++i) {
    const int s = s0 + i;
    u[i] = y < S ? tc::get_split3(op, op + term, op + 2 * term, row0 + s, y)
                 : (s < S ? 1.f : 0.f);
  }
}

// ---------------------------------------------------------------------------
// Transition matrices (Eq. 1) in double-float arithmetic
// ---------------------------------------------------------------------------
// P - I = V diag(e^{lambda gamma t} - 1) Vinv and dP = V diag(gamma lambda
// e^{lambda gamma t}) Vinv.  The exponentials come from FP64; the two
// contractions run on the FP32 pipe with every value held as an unevaluated
// sum hi + lo of two floats (Dekker's double-float arithmetic: products
// split exactly with fmaf, sums with Knuth's TwoSum), about 48 significant
// bits, which keeps the small off-diagonal entries of short branches
// accurate to FP32 despite the cancellation in the sum over eigenvalues.
// The results are rounded once to FP32 and written as the split operand
// tiles.  V and Vinv arrive as double-float tables built on the host.
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

constexpr int kPmatTcThreads = 256;  // one 4 x 4 block of (s, t) per thread
struct PmatTcSmem {
  float vt_h[64][64], vt_l[64][64];  // V transposed: [m][s]
  float vi_h[64][64], vi_l[64][64];  // Vinv: [m][t]
  float pi_h[64], pi_l[64];          // root distribution (reversible form)
  DF e[64], d[64];
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
    double e = 0.0, de = 0.0;
    if (tid < S) {
      double t = a.t[b];
      if (!(t >= 0.0) || !isfinite(t)) {
        if (tid == 0 && r == 0) atomicOr(a.err, ERR_BAD_LENGTH);
        t = 0.0;
      }
      const double g = a.rates[r];
      const double x = a.lambda[tid] * g * t;
      e = expm1(x);
      de = g * a.lambda[tid] * exp(x);
    }
    sm.e[tid] = df_from(e);
    sm.d[tid] = df_from(de);
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
    DF kP[4][4], kD[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) kP[i][j] = kD[i][j] = DF{0.f, 0.f};
    for (int m = 0; m < S; ++m) {
      const float4 sh = *reinterpret_cast<const float4*>(&sm.vt_h[m][s0]);
      const float4 sl = *reinterpret_cast<const float4*>(&sm.vt_l[m][s0]);
      const float4 th = *reinterpret_cast<const float4*>(&sm.vt_h[m][t0]);
      const float4 tl = *reinterpret_cast<const float4*>(&sm.vt_l[m][t0]);
      const DF em = sm.e[m], dm = sm.d[m];
      const DF v[4] = {{sh.x, sl.x}, {sh.y, sl.y}, {sh.z, sl.z}, {sh.w, sl.w}};
      const DF w[4] = {{th.x, tl.x}, {th.y, tl.y}, {th.z, tl.z}, {th.w, tl.w}};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const DF ve = df_mul(v[i], em), vd = df_mul(v[i], dm);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          df_fma(kP[i][j], ve, w[j]);
          df_fma(kD[i][j], vd, w[j]);
        }
      }
    }
    float P[4][4], D[4][4], Pm[4][4], Dm[4][4];  // block (sb, tb) and its mirror
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int s = s0 + i, t = t0 + j;
        const DF pt = {sm.pi_h[t], sm.pi_l[t]}, ps = {sm.pi_h[s], sm.pi_l[s]};
        P[i][j] = df_round(df_mul(kP[i][j], pt), s == t && s < S);
        D[i][j] = df_round(df_mul(kD[i][j], pt), false);
        Pm[j][i] = df_round(df_mul(kP[i][j], ps), s == t && s < S);
        Dm[j][i] = df_round(df_mul(kD[i][j], ps), false);
      }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      put_split3_4(base + kUnitPdp, kTerm128, s0 + i, t0,
                   make_float4(P[i][0], P[i][1], P[i][2], P[i][3]));
      put_split3_4(base + kUnitPdp, kTerm128, 64 + s0 + i, t0,
                   make_float4(D[i][0], D[i][1], D[i][2], D[i][3]));
      put_split3_4(base + kUnitPt, kTerm64, t0 + i, s0,
                   make_float4(P[0][i], P[1][i], P[2][i], P[3][i]));
    }
    if (sb != tb) {
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        put_split3_4(base + kUnitPdp, kTerm128, t0 + j, s0,
                     make_float4(Pm[j][0], Pm[j][1], Pm[j][2], Pm[j][3]));
        put_split3_4(base + kUnitPdp, kTerm128, 64 + t0 + j, s0,
                     make_float4(Dm[j][0], Dm[j][1], Dm[j][2], Dm[j][3]));
        put_split3_4(base + kUnitPt, kTerm64, s0 + j, t0,
                     make_float4(Pm[0][j], Pm[1][j], Pm[2][j], Pm[3][j]));
      }
    }
    return;
  }
  const int s0 = 4 * (tid / 16), t0 = 4 * (tid % 16);
  DF accP[4][4], accD[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) accP[i][j] = accD[i][j] = DF{0.f, 0.f};
  for (int m = 0; m < S; ++m) {
    const float4 vh = *reinterpret_cast<const float4*>(&sm.vt_h[m][s0]);
    const float4 vl = *reinterpret_cast<const float4*>(&sm.vt_l[m][s0]);
    const float4 ih = *reinterpret_cast<const float4*>(&sm.vi_h[m][t0]);
    const float4 il = *reinterpret_cast<const float4*>(&sm.vi_l[m][t0]);
    const DF em = sm.e[m], dm = sm.d[m];
    const DF v[4] = {{vh.x, vl.x}, {vh.y, vl.y}, {vh.z, vl.z}, {vh.w, vl.w}};
    const DF w[4] = {{ih.x, il.x}, {ih.y, il.y}, {ih.z, il.z}, {ih.w, il.w}};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const DF ve = df_mul(v[i], em), vd = df_mul(v[i], dm);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        df_fma(accP[i][j], ve, w[j]);
        df_fma(accD[i][j], vd, w[j]);
      }
    }
  }
  float P[4][4], D[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int s = s0 + i, t = t0 + j;
      P[i][j] = df_round(accP[i][j], s == t && s < S);
      D[i][j] = df_round(accD[i][j], false);
    }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    put_split3_4(base + kUnitPdp, kTerm128, s0 + i, t0,
                 make_float4(P[i][0], P[i][1], P[i][2], P[i][3]));
    put_split3_4(base + kUnitPdp, kTerm128, 64 + s0 + i, t0,
                 make_float4(D[i][0], D[i][1], D[i][2], D[i][3]));
  }
#pragma unroll
  for (int j = 0; j < 4; ++j)
    put_split3_4(base + kUnitPt, kTerm64, t0 + j, s0,
                 make_float4(P[0][j], P[1][j], P[2][j], P[3][j]));
}

// ---------------------------------------------------------------------------
// Post-order level (Eq. 2; Eq. 3 at the root)
// ---------------------------------------------------------------------------
template <typename T>  // float only
__global__ void __launch_bounds__(kTcThreads) post_tc_kernel(LevelArgs<T> a) {
  static_assert(std::is_same<T, float>::value, "tensor-core path is FP32");
  pdl_wait_and_release();  // before TMEM, smem or any global access
  static_assert(kStageBytes <= kOp128, "staging fits in an operand buffer");
  extern __shared__ unsigned char smraw[];
  unsigned char* base = align1024(smraw);
  unsigned char* A[2] = {base, base + kOp128};
  unsigned char* B[2] = {base + 2 * kOp128, base + 2 * kOp128 + kOp64};
  float* stage = reinterpret_cast<float*>(A[0]);  // output rows, after the MMAs
  __shared__ uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_slot;
  __shared__ float xch[2][kTcRows];  // the two halves' partial row results
  __shared__ double lred[kTcRows / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int row = tid & (kTcRows - 1), h = tid / kTcRows;
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int4 d = a.level_desc[blockIdx.y];
  const int k = d.x;
  const TcChild xs[2] = {tc_child(a.n_tips, d.y, d.w & kDescFlagCompact0),
                         tc_child(a.n_tips, d.z, d.w & kDescFlagCompact1)};
  const bool any_mma = !xs[0].compact || !xs[1].compact;
  const int c0 = blockIdx.x * kTcRows, c = c0 + row;
  const bool valid = c < C;
  const int estr = a.escale_stride;
  const bool root = k == a.root;
  const int r_begin = root ? 0 : (int)blockIdx.z, r_end = root ? R : r_begin + 1;
  if (warp == 0) tc::alloc(&tmem_slot, 128);
  if (tid == 0) {
    mbar_init_fenced(&bar_tma, 1);
    mbar_init_fenced(&bar_mma, 1);
  }
  int y[2] = {0, 0};
  for (int x = 0; x < 2; ++x)
    if (xs[x].compact && valid) y[x] = a.tip_states[(size_t)xs[x].b * a.state_stride + c];
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  uint32_t ptma = 0, pmma = 0;
  int pend_tma = -1, pend_mma = -1;
  bool ok = true;
  // running log-likelihood sum of the root (value, exponent)
  float lsum = 0.f;
  int lexp = INT_MIN / 2;
  for (int r = r_begin; r < r_end && ok; ++r) {
    if (tid == 0) {
      mbar_expect_tx(&bar_tma, 2 * kOp64);
      for (int x = 0; x < 2; ++x) {
        const unsigned char* src = unit_tiles(a, xs[x].b, r) + kUnitPdp;
        // rows 0..63 (P) of each term of the 128-row PdP operand
        for (int t = 0; t < 3; ++t)
          bulk_g2s(B[x] + t * kTerm64, src + t * kTerm128, kTerm64, &bar_tma);
      }
    }
    // every global load of this category is issued before any is used
    int E = 0;
    if (valid)
      for (int x = 0; x < 2; ++x)
        if (xs[x].internal) E += a.escale[((size_t)(xs[x].b - a.n_tips) * R + r) * estr + c];
    {
      float4 v[2][8];
      for (int x = 0; x < 2; ++x)
        if (!xs[x].compact) {
          size_t stride;
          const float* src = child_base(a, xs[x], r, &stride);
          coop_load(v[x], src, stride, c0, C);
        }
      for (int x = 0; x < 2; ++x)
        if (!xs[x].compact) coop_put(A[x], v[x]);
    }
    tc::fence_smem_for_async();
    if (!(ok = tc_block_wait(&bar_tma, ptma, pend_tma, a.err))) break;
    if (any_mma) {
      if (tid == 0) {
        for (int x = 0; x < 2; ++x)
          if (!xs[x].compact) {
            uint32_t ta[3], tb[3];
            term_addrs(A[x], kTerm128, ta);
            term_addrs(B[x], kTerm64, tb);
            tc::mma_split_bf16x3<64>(tmem + 64 * x, ta, tb);
          }
        tc::commit(&bar_mma);
      }
      if (!(ok = tc_block_wait(&bar_mma, pmma, pend_mma, a.err))) break;
    }
    // epilogue: p = U_i o U_j on this half row, the row max, scale, store
    float p[32];
    float m = 0.f;
    {
      float uj[32];
      child_cols(xs[0], y[0], S, trow + 0 + 32 * h, B[0], kTerm64, 0, 32 * h, p);
      child_cols(xs[1], y[1], S, trow + 64 + 32 * h, B[1], kTerm64, 0, 32 * h, uj);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        p[i] *= uj[i];
        m = fmaxf(m, fabsf(p[i]));
      }
    }
    xch[h][row] = m;
    __syncthreads();
    m = fmaxf(m, xch[1 - h][row]);
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
    E += e;
    if (!root) {
      stage_half(stage, row, h, p, f);
      if (valid && h == 0) a.escale[((size_t)(k - a.n_tips) * R + r) * estr + c] = E;
      __syncthreads();
      coop_store(a.post + ((size_t)(k - a.n_tips) * C * R + r) * 64, (size_t)R * 64, c0, C,
                 stage);
    } else {
      float pi_dot = 0.f;
#pragma unroll
      for (int i = 0; i < 32; ++i)
        if (32 * h + i < S) pi_dot = fmaf(a.root_pit[32 * h + i], p[i] * f, pi_dot);
      __syncthreads();  // the max exchange above is read; reuse the buffer
      xch[h][row] = pi_dot;
      __syncthreads();
      pi_dot = xch[0][row] + xch[1][row];
      if (valid && pi_dot != 0.f) {
        // L_c = sum_r w_r 2^E_r (pi' p_r): running sum relative to the largest E
        const float term = a.cat_wt[r] * pi_dot;
        if (E > lexp) {
          lsum = lsum * pow2i(lexp - E) + term;
          lexp = E;
        } else {
          lsum += term * pow2i(E - lexp);
        }
      }
    }
    tc::fence_before();
    __syncthreads();  // TMEM, shared tiles and xch are reused next
    tc::fence_after();
  }
  if (ok && root) {
    double term = 0.0;
    if (valid && h == 0) {
      if (!(lsum > 0.f) || !isfinite(lsum)) atomicOr(a.err, ERR_ZERO_PARTIAL);
      term = (double)a.pattern_wt[c] *
             (log((double)lsum) + (double)lexp * 0.69314718055994530942);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) term += __shfl_down_sync(kFull, term, o);
    if (lane == 0 && h == 0) lred[warp] = term;
    __syncthreads();
    if (tid == 0) {
      double l = 0.0;
      for (int w = 0; w < kTcRows / 32; ++w) l += lred[w];
      a.lpart[blockIdx.x] = l;
    }
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
// Persistent, pipelined post-order levels.  One CTA per SM walks the
// level's items (node, 128-pattern tile, category) i = blockIdx.x,
// + gridDim.x, ...; while item i's contractions and epilogue run, the next
// item's partial rows are already loading into registers and its matrix
// tiles into the second shared buffer.  (The root level keeps
// post_tc_kernel above: one node, whose CTAs loop over the categories to
// form log L_c.)
// ---------------------------------------------------------------------------
struct TcItem {
  int k, c0, r;
  TcChild xs[2];
};

__device__ __forceinline__ TcItem tc_item(const LevelArgs<float>& a, int i) {
  TcItem it;
  it.r = i % a.n_cat;
  const int rest = i / a.n_cat;
  it.c0 = (rest % a.n_tiles) * kTcRows;
  const int4 d = a.level_desc[rest / a.n_tiles];
  it.k = d.x;
  it.xs[0] = tc_child(a.n_tips, d.y, d.w & kDescFlagCompact0);
  it.xs[1] = tc_child(a.n_tips, d.z, d.w & kDescFlagCompact1);
  return it;
}

// Bounded wait agreed by the whole block; the parity advances only on
// success, so after a timeout it still names the phase in flight.
__device__ __forceinline__ bool tc_wait_phase(uint64_t* bar, uint32_t& parity, int* err) {
  const bool ok = __syncthreads_and(mbar_wait(bar, parity));
  if (ok) parity ^= 1u;
  else if (threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
  tc::fence_after();
  return ok;
}

// What one thread loads ahead for an item: both children's rows (in the
// cooperative layout), its pattern's compact tip states and the children's
// post-order exponents.
struct TcPrefetch {
  float4 v[2][8];
  int y[2], ep[2];
};

__device__ __forceinline__ void tc_prefetch(const LevelArgs<float>& a, const TcItem& it, int row,
                                            TcPrefetch& pf) {
  const int C = a.n_patterns, c = it.c0 + row;
  const bool valid = c < C;
#pragma unroll
  for (int x = 0; x < 2; ++x) {
    pf.y[x] = 0;
    pf.ep[x] = 0;
    if (it.xs[x].compact) {
      if (valid) pf.y[x] = a.tip_states[(size_t)it.xs[x].b * a.state_stride + c];
    } else {
      size_t stride;
      const float* src = child_base(a, it.xs[x], it.r, &stride);
      coop_load(pf.v[x], src, stride, it.c0, C);
      if (it.xs[x].internal && valid)
        pf.ep[x] = a.escale[((size_t)(it.xs[x].b - a.n_tips) * a.n_cat + it.r) *
                                a.escale_stride + c];
    }
  }
}

// ---------------------------------------------------------------------------
// Post-order level (Eq. 2), every level but the root's
// ---------------------------------------------------------------------------
template <typename T>  // float only
__global__ void __launch_bounds__(kTcThreads) post_tc_pipe_kernel(LevelArgs<T> a) {
  static_assert(std::is_same<T, float>::value, "tensor-core path is FP32");
  pdl_wait_and_release();  // before TMEM, smem or any global access
  extern __shared__ unsigned char smraw[];
  unsigned char* base = align1024(smraw);
  unsigned char* A[2] = {base, base + kOp128};
  // B[buffer][child]: P_x of the current item, and of the next one
  unsigned char* B[2][2] = {{base + 2 * kOp128, base + 2 * kOp128 + kOp64},
                            {base + 2 * kOp128 + 2 * kOp64, base + 2 * kOp128 + 3 * kOp64}};
  float* stage = reinterpret_cast<float*>(A[0]);  // output rows, after the MMAs
  __shared__ uint64_t bar_tma[2], bar_mma;
  __shared__ uint32_t tmem_slot;
  __shared__ float xch[2][kTcRows];
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (kTcRows - 1), h = tid / kTcRows;
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int n_items = a.n_level * a.n_tiles * R;
  int i = blockIdx.x;
  if (i >= n_items) return;  // block-uniform, before any allocation
  if (warp == 0) tc::alloc(&tmem_slot, 128);
  if (tid == 0) {
    mbar_init_fenced(&bar_tma[0], 1);
    mbar_init_fenced(&bar_tma[1], 1);
    mbar_init_fenced(&bar_mma, 1);
  }
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  uint32_t ptma[2] = {0, 0}, pmma = 0;
  bool tpend[2] = {false, false}, mpend = false;
  auto issue_b = [&](const TcItem& it, int buf) {
    if (tid == 0) {
      mbar_expect_tx(&bar_tma[buf], 2 * kOp64);
      for (int x = 0; x < 2; ++x) {
        const unsigned char* src = unit_tiles(a, it.xs[x].b, it.r) + kUnitPdp;
        for (int t = 0; t < 3; ++t)  // rows 0..63 (P) of each term of the PdP operand
          bulk_g2s(B[buf][x] + t * kTerm64, src + t * kTerm128, kTerm64, &bar_tma[buf]);
      }
    }
    tpend[buf] = true;
  };
  TcItem it = tc_item(a, i);
  issue_b(it, 0);
  TcPrefetch pf;
  tc_prefetch(a, it, row, pf);
  int buf = 0;
  for (;;) {
    const TcItem cur = it;
    const int y0 = pf.y[0], y1 = pf.y[1];
    int E = pf.ep[0] + pf.ep[1];
    const int c = cur.c0 + row;
    const bool valid = c < C;
#pragma unroll
    for (int x = 0; x < 2; ++x)
      if (!cur.xs[x].compact) coop_put(A[x], pf.v[x]);
    tc::fence_smem_for_async();
    if (!tc_wait_phase(&bar_tma[buf], ptma[buf], a.err)) break;
    tpend[buf] = false;
    const bool any_mma = !cur.xs[0].compact || !cur.xs[1].compact;
    if (any_mma) {
      if (tid == 0) {
        for (int x = 0; x < 2; ++x)
          if (!cur.xs[x].compact)
            {
              uint32_t ta[3], tb[3];
              term_addrs(A[x], kTerm128, ta);
              term_addrs(B[buf][x], kTerm64, tb);
              tc::mma_split_bf16x3<64>(tmem + 64 * x, ta, tb);
            }
        tc::commit(&bar_mma);
      }
      mpend = true;
    }
    // the next item's matrices and rows load while this one computes
    const int inext = i + (int)gridDim.x;
    const bool more = inext < n_items;
    if (more) {
      it = tc_item(a, inext);
      issue_b(it, buf ^ 1);
      tc_prefetch(a, it, row, pf);
    }
    if (any_mma) {
      if (!tc_wait_phase(&bar_mma, pmma, a.err)) break;
      mpend = false;
    }
    // epilogue: p = U_i o U_j on this half row, the row max, scale, store
    float p[32];
    float m = 0.f;
    {
      float uj[32];
      child_cols(cur.xs[0], y0, S, trow + 0 + 32 * h, B[buf][0], kTerm64, 0, 32 * h, p);
      child_cols(cur.xs[1], y1, S, trow + 64 + 32 * h, B[buf][1], kTerm64, 0, 32 * h, uj);
#pragma unroll
      for (int q = 0; q < 32; ++q) {
        p[q] *= uj[q];
        m = fmaxf(m, fabsf(p[q]));
      }
    }
    xch[h][row] = m;
    __syncthreads();
    m = fmaxf(m, xch[1 - h][row]);
    // an all-zero vector is legitimate for one category (see post_tc_kernel)
    int e = 0;
    if (valid) {
      if (!isfinite(m)) atomicOr(a.err, ERR_ZERO_PARTIAL);
      else if (m > 0.f) (void)frexpf(m, &e);
      e = max(e, -126);  // 2^-e stays finite for a subnormal maximum
    }
    E += e;
    stage_half(stage, row, h, p, ldexpf(1.f, -e));
    if (valid && h == 0)
      a.escale[((size_t)(cur.k - a.n_tips) * R + cur.r) * a.escale_stride + c] = E;
    __syncthreads();
    coop_store(a.post + ((size_t)(cur.k - a.n_tips) * C * R + cur.r) * 64, (size_t)R * 64,
               cur.c0, C, stage);
    tc::fence_before();
    __syncthreads();  // TMEM, staging, B[buf] and xch are reused next
    tc::fence_after();
    if (!more) break;
    i = inext;
    buf ^= 1;
  }
  if (tid == 0) {  // bounded drain of whatever a timeout left in flight
    for (int b = 0; b < 2; ++b)
      if (tpend[b]) (void)mbar_wait(&bar_tma[b], ptma[b]);
    if (mpend) (void)mbar_wait(&bar_mma, pmma);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, 128);
}

// ---------------------------------------------------------------------------
// Pre-order level (Eq. 4) with the per-category Eq. 8 terms
// ---------------------------------------------------------------------------
template <typename T>  // float only
__global__ void __launch_bounds__(kTcThreads) pre_tc_kernel(LevelArgs<T> a) {
  static_assert(std::is_same<T, float>::value, "tensor-core path is FP32");
  pdl_wait_and_release();  // before TMEM, smem or any global access
  static_assert(kStageBytes + 0 <= kOp128 && 2 * kOp64 <= kOp128, "buffer reuse fits");
  extern __shared__ unsigned char smraw[];
  unsigned char* base = align1024(smraw);
  // A_x: the children's p tiles; after the first contractions A_0 holds Pt_i
  // and Pt_j and A_1 stages q_k; after the second, both stage the q_x rows
  unsigned char* A[2] = {base, base + kOp128};
  unsigned char* Tt[2] = {base, base + kOp64};
  // Cm_x: [P_x; dP_x] operand tiles; later a_x as an A operand
  unsigned char* Cm[2] = {base + 2 * kOp128, base + 3 * kOp128};
  __shared__ uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_slot;
  __shared__ float xch[2][3][kTcRows];  // the two halves' partial row results
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (kTcRows - 1), h = tid / kTcRows;
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int4 d = a.level_desc[blockIdx.y];
  const int k = d.x;
  const TcChild xs[2] = {tc_child(a.n_tips, d.y, d.w & kDescFlagCompact0),
                         tc_child(a.n_tips, d.z, d.w & kDescFlagCompact1)};
  const int c0 = blockIdx.x * kTcRows, c = c0 + row;
  const bool valid = c < C;
  const int estr = a.escale_stride;
  const bool root = k == a.root;
  const int r = blockIdx.z;
  const size_t kslot = (size_t)(k - a.n_tips);
  if (warp == 0) tc::alloc(&tmem_slot, 256);
  if (tid == 0) {
    mbar_init_fenced(&bar_tma, 1);
    mbar_init_fenced(&bar_mma, 1);
  }
  int y[2] = {0, 0};
  for (int x = 0; x < 2; ++x)
    if (xs[x].compact && valid) y[x] = a.tip_states[(size_t)xs[x].b * a.state_stride + c];
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);
  uint32_t ptma = 0, pmma = 0;
  int pend_tma = -1, pend_mma = -1;
  bool ok = true;
  if (tid == 0) {
    mbar_expect_tx(&bar_tma, 2 * kOp128);
    for (int x = 0; x < 2; ++x)
      bulk_g2s(Cm[x], unit_tiles(a, xs[x].b, r) + kUnitPdp, kOp128, &bar_tma);
  }
  // every global load is issued before any is used
  int E = 0, eq_k = 0, ep[2] = {0, 0};
  if (valid) {
    if (!root) eq_k = a.pre_escale[(kslot * R + r) * estr + c];
    for (int x = 0; x < 2; ++x)
      if (xs[x].internal) ep[x] = a.escale[((size_t)(xs[x].b - a.n_tips) * R + r) * estr + c];
    E = eq_k + ep[0] + ep[1];
  }
  float4 qv[8];
  if (!root) coop_load(qv, a.pre + (kslot * C * R + r) * 64, (size_t)R * 64, c0, C);
  {
    float4 v[2][8];
    for (int x = 0; x < 2; ++x)
      if (!xs[x].compact) {
        size_t stride;
        const float* src = child_base(a, xs[x], r, &stride);
        coop_load(v[x], src, stride, c0, C);
      }
    for (int x = 0; x < 2; ++x)
      if (!xs[x].compact) coop_put(A[x], v[x]);
  }
  tc::fence_smem_for_async();
  do {
    // ---- [U_x | V_x] = p_x [P_x ; dP_x]' ----
    if (!(ok = tc_block_wait(&bar_tma, ptma, pend_tma, a.err))) break;
    const bool any_mma = !xs[0].compact || !xs[1].compact;
    if (any_mma) {
      if (tid == 0) {
        for (int x = 0; x < 2; ++x)
          if (!xs[x].compact) {
            uint32_t ta[3], tb[3];
            term_addrs(A[x], kTerm128, ta);
            term_addrs(Cm[x], kTerm128, tb);
            tc::mma_split_bf16x3<128>(tmem + 128 * x, ta, tb);
          }
        tc::commit(&bar_mma);
      }
      if (!(ok = tc_block_wait(&bar_mma, pmma, pend_mma, a.err))) break;
    }
    // A is free: stage Pt of the internal children for q_x = a_x P_x, and
    // the rows of q_k
    const bool any_int = xs[0].internal || xs[1].internal;
    if (any_int && tid == 0) {
      mbar_expect_tx(&bar_tma, (xs[0].internal + xs[1].internal) * kOp64);
      for (int x = 0; x < 2; ++x)
        if (xs[x].internal)
          bulk_g2s(Tt[x], unit_tiles(a, xs[x].b, r) + kUnitPt, kOp64, &bar_tma);
    }
    float* qst = reinterpret_cast<float*>(A[1]);
    if (!root) coop_stage(qst, qv);
    __syncthreads();
    // ---- epilogue 1: a_i, a_j, the Eq. 8 terms; a_x staged as an A operand ----
    float ni = 0.f, nj = 0.f, dn = 0.f;
    {
      float q[32];
      if (!root) {
#pragma unroll
        for (int i = 0; i < 32; i += 4) {
          const float4 t4 = *reinterpret_cast<const float4*>(qst + row * kStageLd + 32 * h + i);
          q[i] = t4.x; q[i + 1] = t4.y; q[i + 2] = t4.z; q[i + 3] = t4.w;
        }
      } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) q[i] = 32 * h + i < S ? a.root_pit[32 * h + i] : 0.f;
      }
      float ai[32], aj[32];
      child_cols(xs[1], y[1], S, trow + 128 + 32 * h, Cm[1], kTerm128, 0, 32 * h, ai);
#pragma unroll
      for (int i = 0; i < 32; ++i) ai[i] *= q[i];  // a_i = q o U_j
      {
        float ui[32];
        child_cols(xs[0], y[0], S, trow + 0 + 32 * h, Cm[0], kTerm128, 0, 32 * h, ui);
#pragma unroll
        for (int i = 0; i < 32; ++i) {
          aj[i] = q[i] * ui[i];  // a_j = q o U_i
          dn = fmaf(ai[i], ui[i], dn);
        }
      }
      {
        float vv[32];
        if (!(xs[0].compact && y[0] >= S)) {  // a gap's d/dt of the all-ones vector is 0
          child_cols(xs[0], y[0], S, trow + 64 + 32 * h, Cm[0], kTerm128, 64, 32 * h, vv);
#pragma unroll
          for (int i = 0; i < 32; ++i) ni = fmaf(ai[i], vv[i], ni);
        }
        if (!(xs[1].compact && y[1] >= S)) {
          child_cols(xs[1], y[1], S, trow + 192 + 32 * h, Cm[1], kTerm128, 64, 32 * h, vv);
#pragma unroll
          for (int i = 0; i < 32; ++i) nj = fmaf(aj[i], vv[i], nj);
        }
      }
      // a_x becomes the A operand of q_x = a_x P_x (the PdP tile of an
      // internal child is no longer read: its U, V came from TMEM)
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        if (xs[0].internal) {
          const float x8[8] = {ai[8 * g], ai[8 * g + 1], ai[8 * g + 2], ai[8 * g + 3],
                               ai[8 * g + 4], ai[8 * g + 5], ai[8 * g + 6], ai[8 * g + 7]};
          tc::put_split3(Cm[0], Cm[0] + kTerm128, Cm[0] + 2 * kTerm128, row, 4 * h + g, x8);
        }
        if (xs[1].internal) {
          const float x8[8] = {aj[8 * g], aj[8 * g + 1], aj[8 * g + 2], aj[8 * g + 3],
                               aj[8 * g + 4], aj[8 * g + 5], aj[8 * g + 6], aj[8 * g + 7]};
          tc::put_split3(Cm[1], Cm[1] + kTerm128, Cm[1] + 2 * kTerm128, row, 4 * h + g, x8);
        }
      }
    }
    xch[h][0][row] = ni;
    xch[h][1][row] = nj;
    xch[h][2][row] = dn;
    tc::fence_smem_for_async();
    tc::fence_before();
    __syncthreads();
    if (valid && h == 0) {
      const float w = a.cat_wt[r];
      reinterpret_cast<float4*>(a.rterm)[(kslot * C + c) * R + r] =
          make_float4(w * (ni + xch[1][0][row]), w * (nj + xch[1][1][row]),
                      w * (dn + xch[1][2][row]), __int_as_float(E));
    }
    if (!any_int) break;
    // ---- q_x = a_x P_x for the internal children ----
    if (!(ok = tc_block_wait(&bar_tma, ptma, pend_tma, a.err))) break;
    if (tid == 0) {
      for (int x = 0; x < 2; ++x)
        if (xs[x].internal) {
          uint32_t ta[3], tb[3];
          term_addrs(Cm[x], kTerm128, ta);
          term_addrs(Tt[x], kTerm64, tb);
          tc::mma_split_bf16x3<64>(tmem + 64 * x, ta, tb);
        }
      tc::commit(&bar_mma);
    }
    if (!(ok = tc_block_wait(&bar_mma, pmma, pend_mma, a.err))) break;
    float qo[2][32];
    for (int x = 0; x < 2; ++x) {
      float m = 0.f;
      if (xs[x].internal) {
        tc::ld32(trow + 64 * x + 32 * h, qo[x]);
#pragma unroll
        for (int i = 0; i < 32; ++i) m = fmaxf(m, fabsf(qo[x][i]));
      }
      xch[h][x][row] = m;
    }
    __syncthreads();
    for (int x = 0; x < 2; ++x) {
      if (!xs[x].internal) continue;
      const float m = fmaxf(xch[0][x][row], xch[1][x][row]);
      int e = 0;
      if (valid) {
        if (!isfinite(m)) atomicOr(a.err, ERR_ZERO_PARTIAL);
        else if (m > 0.f) (void)frexpf(m, &e);
        e = max(e, -126);  // 2^-e stays finite for a subnormal maximum
      }
      stage_half(reinterpret_cast<float*>(A[1 - x]), row, h, qo[x], ldexpf(1.f, -e));
      // q_x = P_x' (q_k o U_sibling): exponents of q_k and of the sibling
      if (valid && h == 0)
        a.pre_escale[((size_t)(xs[x].b - a.n_tips) * R + r) * estr + c] = e + eq_k + ep[1 - x];
    }
    __syncthreads();
    for (int x = 0; x < 2; ++x)
      if (xs[x].internal)
        coop_store(a.pre + ((size_t)(xs[x].b - a.n_tips) * C * R + r) * 64, (size_t)R * 64,
                   c0, C, reinterpret_cast<const float*>(A[1 - x]));
  } while (false);
  if (tid == 0) {  // bounded drain of whatever a timeout left in flight
    if (pend_tma >= 0) (void)mbar_wait(&bar_tma, (uint32_t)pend_tma);
    if (pend_mma >= 0) (void)mbar_wait(&bar_mma, (uint32_t)pend_mma);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::dealloc(tmem, 256);
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

// Streaming multiprocessors of the current device (queried once per device).
inline int tc_sm_count() {
  static int count[64] = {0};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (!count[dev]) {
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    count[dev] = n > 0 ? n : 1;
  }
  return count[dev];
}

template <typename T = float>
inline cudaError_t launch_tc64(const LevelArgs<float>& a, bool post, cudaStream_t st) {
  if (post && a.root_level) {
    dim3 grid(a.n_tiles, a.n_level, 1);
    return launch_pdl(post_tc_kernel<float>, grid, kTcThreads, kTcPostSmem, st, a);
  }
  // post-order: persistent, one CTA per SM (shared memory admits no second),
  // never more CTAs than items
  const long items = (long)a.n_level * a.n_tiles * a.n_cat;
  const int grid = (int)(items < tc_sm_count() ? items : tc_sm_count());
  if (post)
    return launch_pdl(post_tc_pipe_kernel<float>, dim3(grid), kTcThreads, kTcPipePostSmem, st, a);
  // pre-order: one CTA per (tile, node, category); a persistent form of it
  // measured slower (its register pressure spills, and the next item's
  // [P; dP] tiles can only load once the current item's second MMA is done)
  dim3 grid3(a.n_tiles, a.n_level, a.n_cat);
  return launch_pdl(pre_tc_kernel<float>, grid3, kTcThreads, kTcPreSmem, st, a);
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
  // the reversible form has 136 blocks of (s, t) per unit: 5 warps, so that
  // three units share an SM
  pmat_tc_kernel<float><<<units, a.reversible ? 160 : kPmatTcThreads, kPmatTcSmem, st>>>(a);
  return cudaGetLastError();
}

template <typename T = float>
inline cudaError_t prepare_tc64() {
  cudaError_t e = cudaFuncSetAttribute(post_tc_kernel<float>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kTcPostSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(post_tc_pipe_kernel<float>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcPipePostSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pre_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTcPreSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pmat_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPmatTcSmem);
  return e;
}

}  // namespace phylo
