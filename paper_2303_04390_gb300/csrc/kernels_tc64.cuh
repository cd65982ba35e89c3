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
// tcgen05.mma kind::tf32 with FP32 accumulation in TMEM.  FP32 accuracy
// comes from splitting both operands into TF32 hi and remainder lo and
// summing Ahi Bhi + Ahi Blo + Alo Bhi (three passes).  After each
// contraction one thread per pattern reads its accumulator row back from
// TMEM, so products, dot products and the rescale are thread-local.
//
// Matrices.  The transition-matrix kernel of this path writes, per (branch,
// r), the operand tiles the level kernels consume, already split and in the
// K-major 128-byte-swizzle layout of tc.cuh, so a level kernel stages them
// with 1-D bulk copies (cp.async.bulk) that overlap its partial loads:
//   [PdP hi | PdP lo | Pt hi | Pt lo]
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
constexpr int kTcThreads = 128;           // one thread per pattern row
static_assert(kTcRows == kTcThreads, "one thread per accumulator lane");

constexpr uint32_t kTile128 = 128 * 256;  // 128 rows x 64 FP32
constexpr uint32_t kTile64 = 64 * 256;
// Matrix tiles of one (branch, r) in the workspace.
constexpr uint32_t kUnitPdpHi = 0, kUnitPdpLo = kTile128;
constexpr uint32_t kUnitPtHi = 2 * kTile128, kUnitPtLo = 2 * kTile128 + kTile64;
static_assert(kTcUnitBytes == 2 * kTile128 + 2 * kTile64, "matrix tile block size");

// Dynamic shared memory (+1024 for the alignment of the swizzled tiles):
//   post: A_i, A_j (hi+lo, 64 KB each) | B_i, B_j (P hi+lo, 32 KB each)
//   pre:  A (64 KB; later Pt_i, Pt_j) | PdP_i, PdP_j (hi+lo, 64 KB each)
constexpr size_t kTcPostSmem = 1024 + 4 * kTile128 + 4 * kTile64;
constexpr size_t kTcPreSmem = 1024 + 2 * kTile128 + 4 * kTile128;

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

// Load this thread's row of a partial tile (64 FP32) into registers.
__device__ __forceinline__ void load_row(float4 (&v)[16], const float* __restrict__ src,
                                         bool valid) {
#pragma unroll
  for (int j = 0; j < 16; ++j)
    v[j] = valid ? __ldg(reinterpret_cast<const float4*>(src) + j)
                 : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Split a register row into the hi/lo A tiles (row `row`).
__device__ __forceinline__ void put_row(unsigned char* hi, unsigned char* lo, int row,
                                        const float4 (&v)[16]) {
#pragma unroll
  for (int j = 0; j < 16; ++j) tc::put_split4(hi, lo, row, j, kTcRows, v[j]);
}

struct TcChild {
  int b;
  bool compact;  // tip with a compact state
  bool internal;
};

__device__ __forceinline__ TcChild tc_child(int n_tips, int b, bool compact) {
  return TcChild{b, compact, b >= n_tips};
}

__device__ __forceinline__ const float* child_row(const LevelArgs<float>& a, const TcChild& x,
                                                  int c, int r) {
  const int C = a.n_patterns;
  if (x.internal)
    return a.post + (((size_t)(x.b - a.n_tips) * C + c) * a.n_cat + r) * 64;
  return a.tip_partials + ((size_t)x.b * C + c) * 64;
}

__device__ __forceinline__ const unsigned char* unit_tiles(const LevelArgs<float>& a, int b,
                                                           int r) {
  return reinterpret_cast<const unsigned char*>(a.P) +
         ((size_t)b * a.n_cat + r) * kTcUnitBytes;
}

// 16 accumulator columns of this thread's row, or for a compact tip the
// matching entries of its matrix column (rows row0 + s of a staged tile
// with `rows` rows; a gap selects the all-ones vector).
__device__ __forceinline__ void child_chunk(const TcChild& x, int y, int S, uint32_t taddr,
                                            const unsigned char* hi, const unsigned char* lo,
                                            int rows, int row0, int s0, float (&u)[16]) {
  if (!x.compact) {
    tc::ld16(taddr, u);
    return;
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) {
    const int s = s0 + i;
    u[i] = y < S ? tc::get_split(hi, lo, row0 + s, y, rows) : (s < S ? 1.f : 0.f);
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
// The results are rounded to FP32 and written as the split operand tiles.
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

constexpr int kPmatTcThreads = 256;  // one 4 x 4 block of (s, t) per thread
struct PmatTcSmem {
  float vt_h[64][64], vt_l[64][64];  // V transposed: [m][s]
  float vi_h[64][64], vi_l[64][64];  // Vinv: [m][t]
  DF e[64], d[64];
};
constexpr size_t kPmatTcSmem = sizeof(PmatTcSmem);

template <typename T>  // float only
__global__ void __launch_bounds__(kPmatTcThreads) pmat_tc_kernel(PmatArgs a) {
  static_assert(std::is_same<T, float>::value, "tensor-core path is FP32");
  extern __shared__ __align__(16) unsigned char smraw[];
  PmatTcSmem& sm = *reinterpret_cast<PmatTcSmem*>(smraw);
  const int S = a.n_states, R = a.n_cat;
  const int unit = blockIdx.x, b = unit / R, r = unit % R;
  const int tid = threadIdx.x;
  for (int i = tid; i < 64 * 64; i += kPmatTcThreads) {
    const int m = i / 64, s = i % 64;
    const bool in = m < S && s < S;
    const DF v = df_from(in ? a.V[s * S + m] : 0.0);
    const DF w = df_from(in ? a.Vinv[m * S + s] : 0.0);
    sm.vt_h[m][s] = v.h;
    sm.vt_l[m][s] = v.l;
    sm.vi_h[m][s] = w.h;
    sm.vi_l[m][s] = w.l;
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
  __syncthreads();
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
  // Round to FP32 (adding the identity in FP64) and write the split tiles.
  unsigned char* base = static_cast<unsigned char*>(a.P) + (size_t)unit * kTcUnitBytes;
  float P[4][4], D[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int s = s0 + i, t = t0 + j;
      const double one = (s == t && s < S) ? 1.0 : 0.0;
      P[i][j] = (float)(((double)accP[i][j].h + (double)accP[i][j].l) + one);
      D[i][j] = (float)((double)accD[i][j].h + (double)accD[i][j].l);
    }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int s = s0 + i;
    tc::put_split4(base + kUnitPdpHi, base + kUnitPdpLo, s, t0 / 4, 128,
                   make_float4(P[i][0], P[i][1], P[i][2], P[i][3]));
    tc::put_split4(base + kUnitPdpHi, base + kUnitPdpLo, 64 + s, t0 / 4, 128,
                   make_float4(D[i][0], D[i][1], D[i][2], D[i][3]));
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int t = t0 + j;
    tc::put_split4(base + kUnitPtHi, base + kUnitPtLo, t, s0 / 4, 64,
                   make_float4(P[0][j], P[1][j], P[2][j], P[3][j]));
  }
}

// ---------------------------------------------------------------------------
// Post-order level (Eq. 2; Eq. 3 at the root)
// ---------------------------------------------------------------------------
template <typename T>  // float only
__global__ void __launch_bounds__(kTcThreads) post_tc_kernel(LevelArgs<T> a) {
  static_assert(std::is_same<T, float>::value, "tensor-core path is FP32");
  extern __shared__ unsigned char smraw[];
  unsigned char* base = align1024(smraw);
  unsigned char* A_hi[2] = {base, base + 2 * kTile128};
  unsigned char* A_lo[2] = {base + kTile128, base + 3 * kTile128};
  unsigned char* B_hi[2] = {base + 4 * kTile128, base + 4 * kTile128 + 2 * kTile64};
  unsigned char* B_lo[2] = {B_hi[0] + kTile64, B_hi[1] + kTile64};
  __shared__ uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_slot;
  __shared__ double lred[kTcThreads / 32];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int4 d = a.level_desc[blockIdx.y];
  const int k = d.x;
  const TcChild xs[2] = {tc_child(a.n_tips, d.y, d.w & kDescFlagCompact0),
                         tc_child(a.n_tips, d.z, d.w & kDescFlagCompact1)};
  const bool any_mma = !xs[0].compact || !xs[1].compact;
  const int c0 = blockIdx.x * kTcRows, c = c0 + tid;
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
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  uint32_t ptma = 0, pmma = 0;
  int pend_tma = -1, pend_mma = -1;
  bool ok = true;
  // running log-likelihood sum of the root (value, exponent)
  float lsum = 0.f;
  int lexp = INT_MIN / 2;
  for (int r = r_begin; r < r_end && ok; ++r) {
    if (tid == 0) {
      mbar_expect_tx(&bar_tma, 4 * kTile64);
      for (int x = 0; x < 2; ++x) {
        const unsigned char* src = unit_tiles(a, xs[x].b, r);
        // rows 0..63 (P) of each K-atom of the 128-row PdP tile
        bulk_g2s(B_hi[x], src + kUnitPdpHi, kTile64 / 2, &bar_tma);
        bulk_g2s(B_hi[x] + kTile64 / 2, src + kUnitPdpHi + kTile128 / 2, kTile64 / 2, &bar_tma);
        bulk_g2s(B_lo[x], src + kUnitPdpLo, kTile64 / 2, &bar_tma);
        bulk_g2s(B_lo[x] + kTile64 / 2, src + kUnitPdpLo + kTile128 / 2, kTile64 / 2, &bar_tma);
      }
    }
    for (int x = 0; x < 2; ++x) {
      if (xs[x].compact) continue;
      float4 v[16];
      load_row(v, child_row(a, xs[x], valid ? c : c0, r), valid);
      put_row(A_hi[x], A_lo[x], tid, v);
    }
    tc::fence_smem_for_async();
    if (!(ok = tc_block_wait(&bar_tma, ptma, pend_tma, a.err))) break;
    if (any_mma) {
      if (tid == 0) {
        for (int x = 0; x < 2; ++x)
          if (!xs[x].compact)
            tc::mma_split3<64>(tmem + 64 * x, smem_addr(A_hi[x]), smem_addr(A_lo[x]),
                               smem_addr(B_hi[x]), smem_addr(B_lo[x]));
        tc::commit(&bar_mma);
      }
      if (!(ok = tc_block_wait(&bar_mma, pmma, pend_mma, a.err))) break;
    }
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
    if (!root) {
      if (valid) {
        float* out = a.post + (((size_t)(k - a.n_tips) * C + c) * R + r) * 64;
#pragma unroll
        for (int i = 0; i < 64; i += 4)
          *reinterpret_cast<float4*>(out + i) =
              make_float4(p[i] * f, p[i + 1] * f, p[i + 2] * f, p[i + 3] * f);
        a.escale[((size_t)(k - a.n_tips) * R + r) * estr + c] = E;
      }
    } else {
      float pi_dot = 0.f;
#pragma unroll
      for (int i = 0; i < 64; ++i)
        if (i < S) pi_dot = fmaf(a.root_pit[i], p[i] * f, pi_dot);
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
    __syncthreads();  // TMEM and shared tiles are reused by the next category
    tc::fence_after();
  }
  if (ok && root) {
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
  if (tid == 0) {  // bounded drain of whatever a timeout left in flight
    if (pend_tma >= 0) (void)mbar_wait(&bar_tma, (uint32_t)pend_tma);
    if (pend_mma >= 0) (void)mbar_wait(&bar_mma, (uint32_t)pend_mma);
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
  extern __shared__ unsigned char smraw[];
  unsigned char* base = align1024(smraw);
  // A: the children's p tiles in turn; then Pt_i (hi, lo) and Pt_j (hi, lo)
  unsigned char* A_hi = base;
  unsigned char* A_lo = base + kTile128;
  unsigned char* T_hi[2] = {base, base + 2 * kTile64};
  unsigned char* T_lo[2] = {base + kTile64, base + 3 * kTile64};
  // PdP_x: [P_x; dP_x] operand tiles; later a_x as an A operand
  unsigned char* C_hi[2] = {base + 2 * kTile128, base + 4 * kTile128};
  unsigned char* C_lo[2] = {base + 3 * kTile128, base + 5 * kTile128};
  __shared__ uint64_t bar_tma, bar_mma;
  __shared__ uint32_t tmem_slot;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int4 d = a.level_desc[blockIdx.y];
  const int k = d.x;
  const TcChild xs[2] = {tc_child(a.n_tips, d.y, d.w & kDescFlagCompact0),
                         tc_child(a.n_tips, d.z, d.w & kDescFlagCompact1)};
  const int c0 = blockIdx.x * kTcRows, c = c0 + tid;
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
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  uint32_t ptma = 0, pmma = 0;
  int pend_tma = -1, pend_mma = -1;
  bool ok = true;
  if (tid == 0) {
    mbar_expect_tx(&bar_tma, 4 * kTile128);
    for (int x = 0; x < 2; ++x) {
      const unsigned char* src = unit_tiles(a, xs[x].b, r);
      bulk_g2s(C_hi[x], src + kUnitPdpHi, kTile128, &bar_tma);
      bulk_g2s(C_lo[x], src + kUnitPdpLo, kTile128, &bar_tma);
    }
  }
  // the non-compact children in order; the second one's row is prefetched
  // into registers while the first one's contraction runs
  int order[2] = {0, 1}, n_mma = 0;
  for (int x = 0; x < 2; ++x)
    if (!xs[x].compact) order[n_mma++] = x;
  float4 v[16];
  if (n_mma > 0) {
    load_row(v, child_row(a, xs[order[0]], valid ? c : c0, r), valid);
    put_row(A_hi, A_lo, tid, v);
  }
  if (n_mma > 1) load_row(v, child_row(a, xs[order[1]], valid ? c : c0, r), valid);
  tc::fence_smem_for_async();
  do {
    // ---- [U_x | V_x] = p_x [P_x ; dP_x]' ----
    if (!(ok = tc_block_wait(&bar_tma, ptma, pend_tma, a.err))) break;
    for (int i = 0; i < n_mma && ok; ++i) {
      if (i == 1) {
        put_row(A_hi, A_lo, tid, v);
        tc::fence_smem_for_async();
        __syncthreads();
      }
      if (tid == 0) {
        const int x = order[i];
        tc::mma_split3<128>(tmem + 128 * x, smem_addr(A_hi), smem_addr(A_lo),
                            smem_addr(C_hi[x]), smem_addr(C_lo[x]));
        tc::commit(&bar_mma);
      }
      ok = tc_block_wait(&bar_mma, pmma, pend_mma, a.err);
    }
    if (!ok) break;
    // A is free: stage Pt of the internal children for q_x = a_x P_x
    const bool any_int = xs[0].internal || xs[1].internal;
    if (any_int && tid == 0) {
      mbar_expect_tx(&bar_tma, (xs[0].internal + xs[1].internal) * 2 * kTile64);
      for (int x = 0; x < 2; ++x) {
        if (!xs[x].internal) continue;
        const unsigned char* src = unit_tiles(a, xs[x].b, r);
        bulk_g2s(T_hi[x], src + kUnitPtHi, kTile64, &bar_tma);
        bulk_g2s(T_lo[x], src + kUnitPtLo, kTile64, &bar_tma);
      }
    }
    // exponent of this category's products at node k
    int E = 0;
    if (valid) {
      if (!root) E += a.pre_escale[(kslot * R + r) * estr + c];
      for (int x = 0; x < 2; ++x)
        if (xs[x].internal) E += a.escale[((size_t)(xs[x].b - a.n_tips) * R + r) * estr + c];
    }
    // ---- epilogue 1: a_i, a_j, the Eq. 8 terms; a_x staged as an A operand ----
    const float* qrow = (!root && valid) ? a.pre + ((kslot * C + c) * R + r) * 64 : nullptr;
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
        float4 qv = make_float4(0.f, 0.f, 0.f, 0.f);
        if (qrow) {
          qv = __ldg(reinterpret_cast<const float4*>(qrow + s0 + i));
        } else if (root && valid) {
          qv.x = s0 + i < S ? a.root_pit[s0 + i] : 0.f;
          qv.y = s0 + i + 1 < S ? a.root_pit[s0 + i + 1] : 0.f;
          qv.z = s0 + i + 2 < S ? a.root_pit[s0 + i + 2] : 0.f;
          qv.w = s0 + i + 3 < S ? a.root_pit[s0 + i + 3] : 0.f;
        }
        q[i] = qv.x; q[i + 1] = qv.y; q[i + 2] = qv.z; q[i + 3] = qv.w;
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
      // a_x becomes the A operand of q_x = a_x P_x (the PdP tile of an
      // internal child is no longer read: its U, V came from TMEM)
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
    if (valid) {
      const float w = a.cat_wt[r];
      reinterpret_cast<float4*>(a.rterm)[(kslot * C + c) * R + r] =
          make_float4(w * ni, w * nj, w * dn, __int_as_float(E));
    }
    if (!any_int) break;
    // ---- q_x = a_x P_x for the internal children ----
    tc::fence_smem_for_async();
    tc::fence_before();
    if (!(ok = tc_block_wait(&bar_tma, ptma, pend_tma, a.err))) break;
    if (tid == 0) {
      for (int x = 0; x < 2; ++x)
        if (xs[x].internal)
          tc::mma_split3<64>(tmem + 64 * x, smem_addr(C_hi[x]), smem_addr(C_lo[x]),
                             smem_addr(T_hi[x]), smem_addr(T_lo[x]));
      tc::commit(&bar_mma);
    }
    if (!(ok = tc_block_wait(&bar_mma, pmma, pend_mma, a.err))) break;
    for (int x = 0; x < 2; ++x) {
      if (!xs[x].internal) continue;
      float qv[64];
      float m = 0.f;
#pragma unroll
      for (int s0 = 0; s0 < 64; s0 += 16) {
        float w16[16];
        tc::ld16(trow + 64 * x + s0, w16);
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          qv[s0 + i] = w16[i];
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
              make_float4(qv[i] * f, qv[i + 1] * f, qv[i + 2] * f, qv[i + 3] * f);
        // q_x = P_x' (q_k o U_sibling): exponents of q_k and of the sibling
        const int sib = 1 - x;
        int eq = e + (root ? 0 : a.pre_escale[(kslot * R + r) * estr + c]);
        if (xs[sib].internal) eq += a.escale[((size_t)(xs[sib].b - a.n_tips) * R + r) * estr + c];
        a.pre_escale[(slot * R + r) * estr + c] = eq;
      }
    }
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
__global__ void __launch_bounds__(kTcThreads) ratio_tc_kernel(LevelArgs<T> a) {
  static_assert(std::is_same<T, float>::value, "tensor-core path is FP32");
  __shared__ F2 red[kTcThreads / 32][2];
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
  block_sum_acc<float, kTcThreads>(gi, gj, red, 1);
  if (threadIdx.x == 0) {
    a.gpart[(size_t)ch.x * a.n_tiles + blockIdx.x] = Acc<float>::to_double(gi);
    a.gpart[(size_t)ch.y * a.n_tiles + blockIdx.x] = Acc<float>::to_double(gj);
  }
}

template <typename T = float>
inline cudaError_t launch_tc64(const LevelArgs<float>& a, bool post, cudaStream_t st) {
  if (post) {
    dim3 grid(a.n_tiles, a.n_level, a.root_level ? 1 : a.n_cat);
    post_tc_kernel<float><<<grid, kTcThreads, kTcPostSmem, st>>>(a);
  } else {
    dim3 grid(a.n_tiles, a.n_level, a.n_cat);
    pre_tc_kernel<float><<<grid, kTcThreads, kTcPreSmem, st>>>(a);
  }
  return cudaGetLastError();
}

template <typename T = float>
inline cudaError_t launch_ratio_tc64(const LevelArgs<float>& a, cudaStream_t st) {
  if (a.n_tiles <= 0 || a.n_tips < 2) return cudaSuccess;
  dim3 grid(a.n_tiles, a.n_tips - 1);
  ratio_tc_kernel<float><<<grid, kTcThreads, 0, st>>>(a);
  return cudaGetLastError();
}

template <typename T = float>
inline cudaError_t launch_pmat_tc64(const PmatArgs& a, cudaStream_t st) {
  const int units = a.n_branches * a.n_cat;
  if (units <= 0) return cudaSuccess;
  pmat_tc_kernel<float><<<units, kPmatTcThreads, kPmatTcSmem, st>>>(a);
  return cudaGetLastError();
}

template <typename T = float>
inline cudaError_t prepare_tc64() {
  cudaError_t e = cudaFuncSetAttribute(post_tc_kernel<float>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kTcPostSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pre_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTcPreSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pmat_tc_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kPmatTcSmem);
  return e;
}

}  // namespace phylo
