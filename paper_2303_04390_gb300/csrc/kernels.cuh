// Level-batched kernels for the post-order pass (Eq. 2, with Eq. 3 at the
// root), the pre-order pass (Eq. 4) with the fused per-branch gradient ratio
// (Eq. 8) and its cross-pattern reduction (Eq. 7), and the transition-matrix
// builder (Eq. 1) of arXiv 2303.04390.
//
// Layout.  Partials are pattern-major, [slot][c][r][SP] with SP the padded
// state count, so one pattern tile of every category is one contiguous
// block of memory.  Matrices are [branch][r][SP][SP] with row = parent
// state; padded rows and columns are zero, so padded partial entries stay 0.
//
// Rescaling (not in the paper): after every product the vector of (node, c)
// is divided by 2^e, e = exponent of its max over all r and s, so one power
// of two is shared by every category and state.  Post-order exponents are
// accumulated per (node, c) and enter log P(Y) at the root; pre-order
// exponents cancel in the gradient ratio and are dropped.
//
// Gradient.  For parent k with children i, j:
//   a_i = q_k o (P_j p_j),  num_i = a_i' (dP_i p_i),  den = a_i' (P_i p_i)
// which equals Eq. 8's p_i' Q' q_i / p_i' q_i with q_i = P_i' a_i, because
// dP_i = gamma_r Q P_i and P_i commutes with Q.  g_{i,c} = sum_r w_r num /
// sum_r w_r den; sum_c W_c g_{i,c} is reduced per tile in FP64.
#pragma once

#include <cstdint>
#include <type_traits>

#include "phylo_internal.h"
#include "tma.cuh"

namespace phylo {

constexpr unsigned kFull = 0xffffffffu;

template <typename T> struct Vec;
template <> struct Vec<float> { using type = float4; static constexpr int n = 4; };
template <> struct Vec<double> { using type = double2; static constexpr int n = 2; };

// Per-r matrix stride in shared memory: SP*SP plus 16 bytes, so that the up
// to 8 categories read by one warp fall in different banks.
template <typename T, int SP>
struct MatStride { static constexpr int v = SP * SP + 16 / (int)sizeof(T); };

template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

// Load / store a partial vector of SP values as SP/n vector chunks; chunk i
// sits i * cs vector-widths after the first (cs = 1: contiguous).
template <typename T, int SP>
__device__ __forceinline__ void load_vec(const T* __restrict__ src, T (&v)[SP],
                                         bool active, int cs = 1) {
  using V = typename Vec<T>::type;
  constexpr int n = Vec<T>::n;
  static_assert(SP % n == 0, "padded states must fill whole vectors");
  if (active) {
    const V* s = reinterpret_cast<const V*>(src);
#pragma unroll
    for (int i = 0; i < SP / n; ++i) {
      V x = __ldg(s + (size_t)i * cs);
      if constexpr (n == 4) {
        v[4 * i] = x.x; v[4 * i + 1] = x.y; v[4 * i + 2] = x.z; v[4 * i + 3] = x.w;
      } else {
        v[2 * i] = x.x; v[2 * i + 1] = x.y;
      }
    }
  } else {
#pragma unroll
    for (int s = 0; s < SP; ++s) v[s] = T(0);
  }
}

template <typename T, int SP>
__device__ __forceinline__ void store_vec(T* dst, const T (&v)[SP], int cs = 1) {
  using V = typename Vec<T>::type;
  constexpr int n = Vec<T>::n;
  V* d = reinterpret_cast<V*>(dst);
#pragma unroll
  for (int i = 0; i < SP / n; ++i) {
    V x;
    if constexpr (n == 4) {
      x.x = v[4 * i]; x.y = v[4 * i + 1]; x.z = v[4 * i + 2]; x.w = v[4 * i + 3];
    } else {
      x.x = v[2 * i]; x.y = v[2 * i + 1];
    }
    d[(size_t)i * cs] = x;
  }
}

// out = M v  (out[s] = sum_t M[s][t] v[t]); M row-major SP x SP in smem.
template <typename T, int SP>
__device__ __forceinline__ void matvec(const T* __restrict__ M,
                                       const T (&v)[SP], T (&out)[SP]) {
#pragma unroll
  for (int s = 0; s < SP; ++s) {
    T acc = T(0);
#pragma unroll
    for (int t = 0; t < SP; ++t) acc = fma(M[s * SP + t], v[t], acc);
    out[s] = acc;
  }
}

// out = M' v  (out[t] = sum_s M[s][t] v[s]).
template <typename T, int SP>
__device__ __forceinline__ void matvec_t(const T* __restrict__ M,
                                         const T (&v)[SP], T (&out)[SP]) {
#pragma unroll
  for (int t = 0; t < SP; ++t) out[t] = T(0);
#pragma unroll
  for (int s = 0; s < SP; ++s) {
#pragma unroll
    for (int t = 0; t < SP; ++t) out[t] = fma(M[s * SP + t], v[s], out[t]);
  }
}

// FP32 with 20 padded states reads its matrices in the transposed layout
// (uses_tr_layout) and forms every product on the packed FP32 FMA.
template <typename T, int SP>
constexpr bool kTrSmall = std::is_same<T, float>::value && SP == 20;

// Where the register kernels keep the partial vector of (slot, pattern c,
// category r).  FP32 with 20 padded states: tile-blocked by the kernels'
// block, [slot][tile][chunk][kSmallThreads][4] with tile = c / (threads /
// RP) and lane (c % (threads / RP)) RP + r, so a warp's access to one
// 16-byte chunk is 512 contiguous bytes (uses_p20_tiles); chunk stride
// kSmallThreads float4.  Otherwise pattern-major [slot][c][r][SP].
template <typename T, int SP, int RP>
struct SmallVec {
  static constexpr bool tiled = kTrSmall<T, SP>;
  static constexpr int cs = tiled ? kSmallThreads : 1;  // chunk stride (vectors)
  __device__ static size_t offset(size_t slot, int c, int r, int R, int C, int n_tiles) {
    if constexpr (tiled) {
      constexpr int CT = kSmallThreads / RP;
      const size_t tile = slot * n_tiles + c / CT;
      return tile * (size_t)(kSmallThreads * SP) + (size_t)((c % CT) * RP + r) * 4;
    } else {
      return ((slot * C + c) * R + r) * SP;
    }
  }
};

// out[j] = sum_i y[i] X[i][j], two outputs per packed FMA, i in order (the
// same operations as matvec / matvec_t): X = M' gives M v, X = M gives M' a.
template <int SP>
__device__ __forceinline__ void rowcomb2(const float* __restrict__ X, const float (&y)[SP],
                                         float (&out)[SP]) {
  float2 acc[SP / 2];
#pragma unroll
  for (int p = 0; p < SP / 2; ++p) acc[p] = make_float2(0.f, 0.f);
#pragma unroll
  for (int i = 0; i < SP; ++i) {
    const float2 yi = make_float2(y[i], y[i]);
    const float2* row = reinterpret_cast<const float2*>(X + i * SP);
#pragma unroll
    for (int p = 0; p < SP / 2; ++p) acc[p] = __ffma2_rn(row[p], yi, acc[p]);
  }
#pragma unroll
  for (int p = 0; p < SP / 2; ++p) {
    out[2 * p] = acc[p].x;
    out[2 * p + 1] = acc[p].y;
  }
}

// Max |v| over this lane's states, then over the RP lanes of one pattern.
template <typename T, int SP, int RP>
__device__ __forceinline__ T pattern_max(const T (&v)[SP], bool active) {
  T m = T(0);
#pragma unroll
  for (int s = 0; s < SP; ++s) m = tmax(m, fabs(v[s]));
  if (!active) m = T(0);
#pragma unroll
  for (int o = 1; o < RP; o <<= 1) m = tmax(m, __shfl_xor_sync(kFull, m, o));
  return m;
}

// Power-of-two rescale of the pattern's vector: returns the exponent e with
// max * 2^-e in [0.5, 1).  A zero or non-finite max raises ERR_ZERO_PARTIAL.
template <typename T, int SP>
__device__ __forceinline__ int rescale(T (&v)[SP], T m, bool valid_pattern,
                                       int* err) {
  int e = 0;
  if (valid_pattern) {
    if (!(m > T(0)) || !isfinite(m)) {
      atomicOr(err, ERR_ZERO_PARTIAL);
    } else {
      (void)frexp(m, &e);
    }
  }
  const T f = ldexp(T(1), -e);
#pragma unroll
  for (int s = 0; s < SP; ++s) v[s] *= f;
  return e;
}

template <int RP, typename X>
__device__ __forceinline__ X sum_over_lanes(X x) {
#pragma unroll
  for (int o = 1; o < RP; o <<= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

// Cross-pattern accumulator.  FP64 path: double.  FP32 path: an unevaluated
// pair hi + lo of floats kept exact with error-free transformations
// (Knuth's TwoSum, and TwoProd via fma), i.e. ~48-bit sums without FP64
// arithmetic, whose throughput on this part is a small fraction of FP32's.
// The pair is converted to FP64 once per tile; tiles are summed in FP64.
struct F2 {
  float hi, lo;
};

__device__ __forceinline__ F2 two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}

__device__ __forceinline__ F2 f2_add(F2 x, F2 y) {
  F2 s = two_sum(x.hi, y.hi);
  const float lo = s.lo + (x.lo + y.lo);
  const float hi = s.hi + lo;
  return {hi, lo - (hi - s.hi)};
}

template <typename T> struct Acc;
template <> struct Acc<double> {
  using type = double;
  __device__ static double zero() { return 0.0; }
  __device__ static double prod(double w, double g) { return w * g; }
  __device__ static double add(double a, double b) { return a + b; }
  __device__ static double shfl_down(double a, int o) {
    return __shfl_down_sync(kFull, a, o);
  }
  __device__ static double to_double(double a) { return a; }
};
template <> struct Acc<float> {
  using type = F2;
  __device__ static F2 zero() { return {0.f, 0.f}; }
  __device__ static F2 prod(float w, float g) {
    const float p = __fmul_rn(w, g);  // never fused into a later add
    return {p, fmaf(w, g, -p)};
  }
  __device__ static F2 add(F2 a, F2 b) { return f2_add(a, b); }
  __device__ static F2 shfl_down(F2 a, int o) {
    return {__shfl_down_sync(kFull, a.hi, o), __shfl_down_sync(kFull, a.lo, o)};
  }
  __device__ static double to_double(F2 a) { return (double)a.hi + (double)a.lo; }
};

// Block-wide sum of two accumulators; the result is valid in thread 0.
// Lanes below `first` never hold values, so the first shuffle distance is
// `first` (a power of two).
template <typename T, int NT>
__device__ __forceinline__ void block_sum_acc(typename Acc<T>::type& a,
                                              typename Acc<T>::type& b,
                                              typename Acc<T>::type (*sm)[2],
                                              int first) {
  using A = Acc<T>;
  for (int o = 16; o >= first; o >>= 1) {
    a = A::add(a, A::shfl_down(a, o));
    b = A::add(b, A::shfl_down(b, o));
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sm[w][0] = a; sm[w][1] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = sm[0][0]; b = sm[0][1];
#pragma unroll
    for (int i = 1; i < NT / 32; ++i) { a = A::add(a, sm[i][0]); b = A::add(b, sm[i][1]); }
  }
}

// Block-wide sum of one or two doubles (fixed order: deterministic).
template <int NT>
__device__ __forceinline__ void block_sum2(double& a, double& b,
                                           double (*sm)[2]) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(kFull, a, o);
    b += __shfl_down_sync(kFull, b, o);
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { sm[w][0] = a; sm[w][1] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    a = 0.0; b = 0.0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) { a += sm[i][0]; b += sm[i][1]; }
  }
}

// ---------------------------------------------------------------------------
// Eq. 1: P^(r)(t_b) = V diag(e^{lambda gamma_r t_b}) Vinv and
//        dP/dt       = V diag(gamma_r lambda e^{lambda gamma_r t_b}) Vinv,
// for every (branch, category) in one launch, computed and stored in FP64
// with zero padding (the FP64 path; the FP32 paths build their matrices in
// double-float arithmetic).  P is formed as I + V diag(expm1(.)) Vinv: the
// direct form cancels catastrophically in the off-diagonal entries of short
// branches (relative error ~ u |V||Vinv| / (gamma t |Q|)), and at t = 0 it
// gives P = I exactly.
// ---------------------------------------------------------------------------
template <typename T, int SP>
__global__ void __launch_bounds__(256) pmat_kernel(PmatArgs a) {
  constexpr int UPB = (256 / (SP * SP)) > 0 ? 256 / (SP * SP) : 1;
  __shared__ double she[UPB][SP];
  __shared__ double shd[UPB][SP];
  const int S = a.n_states, R = a.n_cat;
  const int n_units = a.n_branches * R;
  const int unit0 = blockIdx.x * UPB;
  for (int i = threadIdx.x; i < UPB * SP; i += blockDim.x) {
    const int u = i / SP, m = i % SP, unit = unit0 + u;
    double e = 0.0, de = 0.0;
    if (unit < n_units && m < S) {
      const int b = unit / R, r = unit % R;
      double t = a.t[b];
      if (!(t >= 0.0) || !isfinite(t)) {
        if (m == 0 && r == 0) atomicOr(a.err, ERR_BAD_LENGTH);
        t = 0.0;
      }
      const double g = a.rates[r];
      const double x = a.lambda[m] * g * t;
      e = expm1(x);                    // e^x - 1: no cancellation for small t
      de = g * a.lambda[m] * exp(x);
    }
    she[u][m] = e;
    shd[u][m] = de;
  }
  __syncthreads();
  T* P = static_cast<T*>(a.P);
  T* dP = static_cast<T*>(a.dP);
  for (int idx = threadIdx.x; idx < UPB * SP * SP; idx += blockDim.x) {
    const int u = idx / (SP * SP), e = idx % (SP * SP);
    const int unit = unit0 + u;
    if (unit >= n_units) continue;
    const int s = e / SP, t = e % SP;
    double acc = 0.0, dacc = 0.0;
    if (s < S && t < S) {
      for (int m = 0; m < S; ++m) {
        const double vv = a.V[s * S + m] * a.Vinv[m * S + t];
        acc = fma(vv, she[u][m], acc);
        dacc = fma(vv, shd[u][m], dacc);
      }
      if (s == t) acc += 1.0;  // P = I + V diag(e^x - 1) Vinv
    }
    P[(size_t)unit * SP * SP + e] = (T)acc;
    dP[(size_t)unit * SP * SP + e] = (T)dacc;
  }
}

// ---------------------------------------------------------------------------
// Register kernels (SP <= 20): one thread per (pattern, category) for NPT
// nodes of the level; the RP lanes of a pattern are adjacent so the shared
// rescale is a shuffle.  Every input of the block's NPT nodes is requested
// before any is used (more bytes in flight per warp), and the NPT x 2
// children's matrix blocks are staged in shared memory by 1-D bulk copies
// (cp.async.bulk) that complete on one mbarrier.
// ---------------------------------------------------------------------------

// One child's inputs for this thread's (pattern, category), loaded ahead.
template <typename T, int SP>
struct ChildIn {
  T v[SP];  // partial vector (internal child or tip with partials)
  int y;    // compact tip state, or -1
  int e;    // the child's cumulative exponent (internal child)
};

template <typename T, int SP, int RP>
__device__ __forceinline__ void load_child(const LevelArgs<T>& a, int b,
                                           bool compact, int c, int r,
                                           bool active, bool want_e,
                                           ChildIn<T, SP>& in) {
  const int C = a.n_patterns;
  in.e = 0;
  if (compact) {
    in.y = active ? (int)a.tip_states[(size_t)b * a.state_stride + c] : 0;
    return;
  }
  in.y = -1;
  if (b < a.n_tips) {
    load_vec<T, SP>(a.tip_partials + ((size_t)b * C + c) * SP, in.v, active);
  } else {
    const size_t slot = (size_t)(b - a.n_tips);
    using SV = SmallVec<T, SP, RP>;
    load_vec<T, SP>(a.post + SV::offset(slot, c, r, a.n_cat, C, a.n_tiles), in.v, active,
                    SV::cs);
    if (want_e && active) in.e = a.escale[slot * a.escale_stride + c];
  }
}

// u = M v (a compact state picks column y of M; the gap code gives the
// all-ones vector), and with WITH_D also w = dM v (0 for a gap).
template <typename T, int SP, bool WITH_D>
__device__ __forceinline__ void child_apply(const ChildIn<T, SP>& in, int S,
                                            const T* __restrict__ M,
                                            const T* __restrict__ dM,
                                            T (&u)[SP], T (&w)[SP]) {
  if (in.y >= 0) {
    if (in.y < S) {
#pragma unroll
      for (int s = 0; s < SP; ++s) u[s] = M[s * SP + in.y];
      if constexpr (WITH_D) {
#pragma unroll
        for (int s = 0; s < SP; ++s) w[s] = dM[s * SP + in.y];
      }
    } else {
#pragma unroll
      for (int s = 0; s < SP; ++s) u[s] = s < S ? T(1) : T(0);
      if constexpr (WITH_D) {
#pragma unroll
        for (int s = 0; s < SP; ++s) w[s] = T(0);
      }
    }
    return;
  }
  matvec<T, SP>(M, in.v, u);
  if constexpr (WITH_D) matvec<T, SP>(dM, in.v, w);
}

// Thread 0: copy the matrix blocks of the listed branches into shared
// slots [slot][r] of stride MS (16-byte aligned), one bulk copy per (branch,
// category), all completing on `bar`.  A branch holds `kinds` matrices of
// every category ([b][kind][r][SP][SP]); `kind` selects one.
template <typename T, int SP, int RP>
__device__ __forceinline__ void issue_mats(const T* __restrict__ base,
                                           const int* branches, int n_br,
                                           int R, T* dst, uint64_t* bar,
                                           int kinds = 1, int kind = 0) {
  constexpr int MS = MatStride<T, SP>::v;
  constexpr uint32_t bytes = SP * SP * sizeof(T);
  for (int i = 0; i < n_br; ++i)
    for (int q = 0; q < R; ++q)
      bulk_g2s(dst + ((size_t)i * RP + q) * MS,
               base + (((size_t)branches[i] * kinds + kind) * R + q) * SP * SP, bytes, bar);
}

// Matrix slots per node of the pre-order register kernels: P_i, P_j, dP_i,
// dP_j.
template <typename T, int SP>
constexpr int kPreSlots = 4;

constexpr int kDescCompactX = kDescFlagCompact0, kDescCompactY = kDescFlagCompact1;

// Post-order level (Eq. 2): p_k = (P_i p_i) o (P_j p_j), rescaled; at the
// root also log P(Y_c) (Eq. 3) weighted by W_c and summed per tile.
template <typename T, int SP, int RP, int NPT>
__global__ void __launch_bounds__(kSmallThreads)
post_small_kernel(LevelArgs<T> a) {
  constexpr int NT = kSmallThreads, CT = NT / RP;
  constexpr int MS = MatStride<T, SP>::v;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* mats = reinterpret_cast<T*>(smraw);  // [NPT][2][RP][MS]
  __shared__ uint64_t bar;
  __shared__ double red[NT / 32][2];
  const int g0 = blockIdx.y * NPT;
  const int nn = min(NPT, a.n_level - g0);
  const int R = a.n_cat, C = a.n_patterns;
  const int c = blockIdx.x * CT + threadIdx.x / RP;
  const int r = threadIdx.x % RP;
  const bool valid_c = c < C;
  const bool active = valid_c && r < R;
  const int rr = r < R ? r : 0;
  if (threadIdx.x == 0) mbar_init_fenced(&bar, 1);
  __syncthreads();
  pdl_wait_and_release();
  int4 d[NPT];
#pragma unroll
  for (int u = 0; u < NPT; ++u)
    d[u] = u < nn ? a.level_desc[g0 + u] : make_int4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    int br[2 * NPT];
    for (int u = 0; u < nn; ++u) { br[2 * u] = d[u].y; br[2 * u + 1] = d[u].z; }
    mbar_expect_tx(&bar, (uint32_t)(2 * nn * R * SP * SP * sizeof(T)));
    issue_mats<T, SP, RP>(a.P, br, 2 * nn, R, mats, &bar);
  }
  ChildIn<T, SP> in[NPT][2];
#pragma unroll
  for (int u = 0; u < NPT; ++u) {
    if (u < nn) {
      load_child<T, SP, RP>(a, d[u].y, d[u].w & kDescCompactX, c, r, active, true, in[u][0]);
      load_child<T, SP, RP>(a, d[u].z, d[u].w & kDescCompactY, c, r, active, true, in[u][1]);
    }
  }
  if (!__syncthreads_and(mbar_wait(&bar, 0))) {
    if (threadIdx.x == 0) atomicOr(a.err, ERR_TIMEOUT);
    return;
  }
#pragma unroll
  for (int u = 0; u < NPT; ++u) {
    if (u >= nn) break;
    const int k = d[u].x;
    T ui[SP], uj[SP], dummy[SP];
    child_apply<T, SP, false>(in[u][0], a.n_states, mats + ((2 * u) * RP + rr) * MS,
                              nullptr, ui, dummy);
    child_apply<T, SP, false>(in[u][1], a.n_states, mats + ((2 * u + 1) * RP + rr) * MS,
                              nullptr, uj, dummy);
#pragma unroll
    for (int s = 0; s < SP; ++s) ui[s] *= uj[s];
    const T m = pattern_max<T, SP, RP>(ui, active);
    const int e = rescale<T, SP>(ui, m, valid_c, a.err) + in[u][0].e + in[u][1].e;
    if (k != a.root) {
      const size_t slot = (size_t)(k - a.n_tips);
      if (active) {
        using SV = SmallVec<T, SP, RP>;
        store_vec<T, SP>(a.post + SV::offset(slot, c, r, R, C, a.n_tiles), ui, SV::cs);
        if (r == 0) a.escale[slot * a.escale_stride + c] = e;
      }
      continue;
    }
    // Root: L_c = sum_r w_r pi' p_root (Eq. 3), with the exponents restored.
    double lr = 0.0;
    if (active) {
#pragma unroll
      for (int s = 0; s < SP; ++s)
        if (s < a.n_states) lr += a.root_pi[s] * (double)ui[s];
      lr *= a.cat_w[r];
    }
    lr = sum_over_lanes<RP>(lr);
    double term = 0.0, unused = 0.0;
    if (valid_c && r == 0) {
      if (!(lr > 0.0) || !isfinite(lr)) atomicOr(a.err, ERR_ZERO_PARTIAL);
      term = a.pattern_w[c] * (log(lr) + (double)e * 0.69314718055994530942);
    }
    block_sum2<NT>(term, unused, red);
    if (threadIdx.x == 0) a.lpart[blockIdx.x] = term;
  }
}

// Pre-order level (Eq. 4) with the fused gradient (Eq. 8): for parent k,
//   q_i = P_i' (q_k o P_j p_j),  q_j = P_j' (q_k o P_i p_i)
// stored (rescaled) for internal children; the ratio for branches i and j
// is reduced over the tile's patterns with weights W_c (Eq. 7).
template <typename T, int SP, int RP, int NPT>
__global__ void __launch_bounds__(kSmallThreads)
pre_small_kernel(LevelArgs<T> a) {
  constexpr int NT = kSmallThreads, CT = NT / RP;
  constexpr int MS = MatStride<T, SP>::v;
  extern __shared__ __align__(16) unsigned char smraw[];
  constexpr int NS = kPreSlots<T, SP>;
  T* mats = reinterpret_cast<T*>(smraw);  // [NPT][NS][RP][MS]
  __shared__ uint64_t bar;
  __shared__ typename Acc<T>::type red[NT / 32][2];
  const int g0 = blockIdx.y * NPT;
  const int nn = min(NPT, a.n_level - g0);
  const int R = a.n_cat, C = a.n_patterns;
  const int c = blockIdx.x * CT + threadIdx.x / RP;
  const int r = threadIdx.x % RP;
  const bool valid_c = c < C;
  const bool active = valid_c && r < R;
  const int rr = r < R ? r : 0;
  if (threadIdx.x == 0) mbar_init_fenced(&bar, 1);
  __syncthreads();
  pdl_wait_and_release();
  int4 d[NPT];
#pragma unroll
  for (int u = 0; u < NPT; ++u)
    d[u] = u < nn ? a.level_desc[g0 + u] : make_int4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    int br[2 * NPT];
    mbar_expect_tx(&bar, (uint32_t)(NS * nn * R * SP * SP * sizeof(T)));
    for (int u = 0; u < nn; ++u) {
      br[0] = d[u].y;
      br[1] = d[u].z;
      T* slots = mats + (size_t)(NS * u) * RP * MS;
      issue_mats<T, SP, RP>(a.P, br, 2, R, slots, &bar);
      issue_mats<T, SP, RP>(a.dP, br, 2, R, slots + (size_t)2 * RP * MS, &bar);
    }
  }
  T q[NPT][SP];
  ChildIn<T, SP> in[NPT][2];
#pragma unroll
  for (int u = 0; u < NPT; ++u) {
    if (u < nn) {
      const int k = d[u].x;
      if (k == a.root) {
#pragma unroll
        for (int s = 0; s < SP; ++s)
          q[u][s] = (active && s < a.n_states) ? (T)a.root_pi[s] : T(0);
      } else {
        using SV = SmallVec<T, SP, RP>;
        load_vec<T, SP>(a.pre + SV::offset(k - a.n_tips, c, r, R, C, a.n_tiles), q[u], active,
                        SV::cs);
      }
      load_child<T, SP, RP>(a, d[u].y, d[u].w & kDescCompactX, c, r, active, false, in[u][0]);
      load_child<T, SP, RP>(a, d[u].z, d[u].w & kDescCompactY, c, r, active, false, in[u][1]);
    }
  }
  if (!__syncthreads_and(mbar_wait(&bar, 0))) {
    if (threadIdx.x == 0) atomicOr(a.err, ERR_TIMEOUT);
    return;
  }
  using A = Acc<T>;
  const T w = active ? a.cat_wt[r] : T(0);
#pragma unroll
  for (int u = 0; u < NPT; ++u) {
    if (u >= nn) break;
    const int bi = d[u].y, bj = d[u].z;
    const T* Pi = mats + ((NS * u) * RP + rr) * MS;
    const T* Pj = mats + ((NS * u + 1) * RP + rr) * MS;
    const T* Di = mats + ((NS * u + 2) * RP + rr) * MS;
    const T* Dj = mats + ((NS * u + 3) * RP + rr) * MS;
    T ui[SP], vi[SP], uj[SP], vj[SP];
    child_apply<T, SP, true>(in[u][0], a.n_states, Pi, Di, ui, vi);
    child_apply<T, SP, true>(in[u][1], a.n_states, Pj, Dj, uj, vj);
    // Per-category numerators and the shared denominator.
    T num_i = T(0), num_j = T(0), den = T(0);
#pragma unroll
    for (int s = 0; s < SP; ++s) {
      const T qi = q[u][s] * uj[s];  // a_i
      const T qj = q[u][s] * ui[s];  // a_j
      num_i = fma(qi, vi[s], num_i);
      num_j = fma(qj, vj[s], num_j);
      den = fma(qi, ui[s], den);
    }
    // sum over categories (Eq. 8) in T, then the ratio in T
    const T Ni = sum_over_lanes<RP>(w * num_i);
    const T Nj = sum_over_lanes<RP>(w * num_j);
    const T D = sum_over_lanes<RP>(w * den);
    typename A::type gi = A::zero(), gj = A::zero();
    if (valid_c && r == 0) {
      if (!(D > T(0)) || !isfinite(D)) {
        atomicOr(a.err, ERR_BAD_RATIO);
      } else {
        const T W = a.pattern_wt[c];
        gi = A::prod(W, Ni / D);
        gj = A::prod(W, Nj / D);
      }
    }
    // Children's pre-order partials (internal children only).
    if (bi >= a.n_tips) {
      T av[SP], out[SP];
#pragma unroll
      for (int s = 0; s < SP; ++s) av[s] = q[u][s] * uj[s];
      matvec_t<T, SP>(Pi, av, out);
      const T m = pattern_max<T, SP, RP>(out, active);
      rescale<T, SP>(out, m, valid_c, a.err);
      if (active) {
        using SV = SmallVec<T, SP, RP>;
        store_vec<T, SP>(a.pre + SV::offset(bi - a.n_tips, c, r, R, C, a.n_tiles), out, SV::cs);
      }
    }
    if (bj >= a.n_tips) {
      T av[SP], out[SP];
#pragma unroll
      for (int s = 0; s < SP; ++s) av[s] = q[u][s] * ui[s];
      matvec_t<T, SP>(Pj, av, out);
      const T m = pattern_max<T, SP, RP>(out, active);
      rescale<T, SP>(out, m, valid_c, a.err);
      if (active) {
        using SV = SmallVec<T, SP, RP>;
        store_vec<T, SP>(a.pre + SV::offset(bj - a.n_tips, c, r, R, C, a.n_tiles), out, SV::cs);
      }
    }
    block_sum_acc<T, NT>(gi, gj, red, RP);
    if (threadIdx.x == 0) {
      if constexpr (std::is_same<T, float>::value) {
        // the pair as stored (the reduction converts to FP64)
        float2* gp = reinterpret_cast<float2*>(a.gpart);
        gp[(size_t)bi * a.n_tiles + blockIdx.x] = make_float2(gi.hi, gi.lo);
        gp[(size_t)bj * a.n_tiles + blockIdx.x] = make_float2(gj.hi, gj.lo);
      } else {
        a.gpart[(size_t)bi * a.n_tiles + blockIdx.x] = A::to_double(gi);
        a.gpart[(size_t)bj * a.n_tiles + blockIdx.x] = A::to_double(gj);
      }
    }
    __syncthreads();  // red[] is reused by the next node
  }
}

// ---------------------------------------------------------------------------
// FP32 with 20 padded states (amino-acid models): the post-order pass stores,
// for every non-root node x with stored partials, U_x = P_x p_x -- the
// factor x contributes to its parent in Eq. 2 -- instead of p_x, and a
// node's p is formed from its children's U when its own step runs:
//   post:  p_k = U_i o U_j (rescaled);  U_k = P_k p_k stored   (Eq. 2)
//   root:  log sum_r w_r pi' p_root                             (Eq. 3)
//   pre:   a_i = q_k o U_j,  a_j = q_k o U_i,  den = a_i . U_i
//          num_x = gamma_r (a_x' Q) U_x  (a tip: a_x' dP_x e_y)  (Eq. 8)
//          q_x = P_x' a_x for internal children                 (Eq. 4)
// Eq. 8's numerator q_x' Q p_x (times gamma_r) equals a_x' P_x Q p_x =
// (a_x' Q)(P_x p_x) because P_x = exp(gamma_r t_x Q) commutes with Q, so an
// internal child costs two products in the pre-order step (Q' a and P' a)
// instead of three (P p, dP p, P' a).  U costs the post-order pass the bytes
// that storing p did.  Layouts as in the register kernels above (tile-blocked
// vectors; matrices [P' | dP' | P] per branch); tips with partial vectors
// keep their U in slots N - 1 + x of the post region, formed by a first
// launch over those tips (`tip_level`).
// ---------------------------------------------------------------------------
constexpr int kU20 = 20;

// U slot of node x: internal nodes x - N, tips with partials N - 1 + x.
__device__ __forceinline__ size_t u20_slot(const LevelArgs<float>& a, int x) {
  return x >= a.n_tips ? (size_t)(x - a.n_tips) : (size_t)(a.n_tips - 1 + x);
}

// A child's U row for this thread's (pattern, category): stored (internal
// child or tip with partials, with the child's exponent) or, for a compact
// tip, its state (resolved by u20_resolve from the staged P').
template <int RP>
__device__ __forceinline__ void load_u20(const LevelArgs<float>& a, int b, bool compact, int c,
                                         int r, bool active, bool want_e,
                                         ChildIn<float, kU20>& in) {
  using SV = SmallVec<float, kU20, RP>;
  in.e = 0;
  if (compact) {
    in.y = active ? (int)a.tip_states[(size_t)b * a.state_stride + c] : 0;
    return;
  }
  in.y = -1;
  load_vec<float, kU20>(
      a.post + SV::offset(u20_slot(a, b), c, r, a.n_cat, a.n_patterns, a.n_tiles), in.v,
      active, SV::cs);
  if (want_e && active && b >= a.n_tips)
    in.e = a.escale[(size_t)(b - a.n_tips) * a.escale_stride + c];
}

// U of a child: the loaded row, or column y of P (row y of P' = Pt); a gap
// selects the all-ones vector.
__device__ __forceinline__ void u20_resolve(const ChildIn<float, kU20>& in, int S,
                                            const float* __restrict__ Pt, float (&u)[kU20]) {
  if (in.y < 0) {
#pragma unroll
    for (int s = 0; s < kU20; ++s) u[s] = in.v[s];
  } else if (in.y < S) {
#pragma unroll
    for (int s = 0; s < kU20; ++s) u[s] = Pt[in.y * kU20 + s];
  } else {
#pragma unroll
    for (int s = 0; s < kU20; ++s) u[s] = s < S ? 1.f : 0.f;
  }
}

// Resident blocks of the U-form kernels' register bound.
#ifndef PHYLO_U20_POST_BLOCKS
#define PHYLO_U20_POST_BLOCKS 4
#endif
#ifndef PHYLO_U20_PRE_BLOCKS
#define PHYLO_U20_PRE_BLOCKS 4
#endif

// Post-order staging (thread 0): only what a lookup or U_k reads, P' of
// compact-tip children (a stored child's U is already P p) and of the node
// unless it is the root.
template <int RP, int NPT>
__device__ __forceinline__ void post_u20_stage(const LevelArgs<float>& a, const int4 (&d)[NPT],
                                               int nn, bool tip, float* mats, uint64_t* bar) {
  constexpr int SP = kU20, MS = MatStride<float, SP>::v;
  if (threadIdx.x != 0) return;
  uint32_t nmat = 0;
  for (int u = 0; u < nn; ++u)
    nmat += (!tip && (d[u].w & kDescCompactX)) + (!tip && (d[u].w & kDescCompactY)) +
            (d[u].x != a.root);
  mbar_expect_tx(bar, nmat * (uint32_t)(a.n_cat * SP * SP * sizeof(float)));
  for (int u = 0; u < nn; ++u) {
    float* slots = mats + (size_t)(3 * u) * RP * MS;
    const int br[3] = {d[u].y, d[u].z, d[u].x};
    const bool need[3] = {!tip && (d[u].w & kDescCompactX), !tip && (d[u].w & kDescCompactY),
                          d[u].x != a.root};
    for (int x = 0; x < 3; ++x)
      if (need[x])
        issue_mats<float, SP, RP>(a.P, br + x, 1, a.n_cat, slots + (size_t)x * RP * MS, bar,
                                  kP4MatKinds, 0);
  }
}

// Post-order level: per node of the block, slots [P'_child0 | P'_child1 |
// P'_node] (every category); on the tip level, P'_tip alone.
template <int RP, int NPT>
__global__ void __launch_bounds__(kSmallThreads, PHYLO_U20_POST_BLOCKS)
post_u20_kernel(LevelArgs<float> a) {
  constexpr int SP = kU20, NT = kSmallThreads, CT = NT / RP;
  constexpr int MS = MatStride<float, SP>::v;
  using SV = SmallVec<float, SP, RP>;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* mats = reinterpret_cast<float*>(smraw);  // [NPT][3][RP][MS]
  __shared__ uint64_t bar;
  __shared__ double red[NT / 32][2];
  const int g0 = blockIdx.y * NPT;
  const int nn = min(NPT, a.n_level - g0);
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int c = blockIdx.x * CT + threadIdx.x / RP;
  const int r = threadIdx.x % RP;
  const bool valid_c = c < C;
  const bool active = valid_c && r < R;
  const int rr = r < R ? r : 0;
  const bool tip = a.tip_level;
  if (threadIdx.x == 0) mbar_init_fenced(&bar, 1);
  __syncthreads();
  int4 d[NPT];  // host-written: readable before the wait
#pragma unroll
  for (int u = 0; u < NPT; ++u)
    d[u] = u < nn ? a.level_desc[g0 + u] : make_int4(0, 0, 0, 0);
  if (a.mats_ready) post_u20_stage<RP, NPT>(a, d, nn, tip, mats, &bar);
  pdl_wait_and_release();
  if (!a.mats_ready) post_u20_stage<RP, NPT>(a, d, nn, tip, mats, &bar);
  ChildIn<float, SP> in[NPT][2];
#pragma unroll
  for (int u = 0; u < NPT; ++u) {
    if (u >= nn) continue;
    if (tip) {  // the tip's partial vector
      in[u][0].y = -1;
      in[u][0].e = 0;
      load_vec<float, SP>(a.tip_partials + ((size_t)d[u].x * C + c) * SP, in[u][0].v, active);
    } else {
      load_u20<RP>(a, d[u].y, d[u].w & kDescCompactX, c, r, active, true, in[u][0]);
      load_u20<RP>(a, d[u].z, d[u].w & kDescCompactY, c, r, active, true, in[u][1]);
    }
  }
  if (!__syncthreads_and(mbar_wait(&bar, 0))) {
    if (threadIdx.x == 0) atomicOr(a.err, ERR_TIMEOUT);
    return;
  }
#pragma unroll
  for (int u = 0; u < NPT; ++u) {
    if (u >= nn) break;
    const int k = d[u].x;
    const float* Ptk = mats + ((3 * u + 2) * RP + rr) * MS;
    float p[SP], uk[SP];
    int e = 0;
    if (tip) {
#pragma unroll
      for (int s = 0; s < SP; ++s) p[s] = in[u][0].v[s];
    } else {
      float uj[SP];
      u20_resolve(in[u][0], S, mats + ((3 * u) * RP + rr) * MS, p);
      u20_resolve(in[u][1], S, mats + ((3 * u + 1) * RP + rr) * MS, uj);
#pragma unroll
      for (int s = 0; s < SP; ++s) p[s] *= uj[s];
      const float m = pattern_max<float, SP, RP>(p, active);
      e = rescale<float, SP>(p, m, valid_c, a.err) + in[u][0].e + in[u][1].e;
    }
    if (k != a.root) {
      rowcomb2<SP>(Ptk, p, uk);  // U_k = P_k p_k
      if (active) {
        store_vec<float, SP>(a.post + SV::offset(u20_slot(a, k), c, r, R, C, a.n_tiles), uk,
                             SV::cs);
        if (!tip && r == 0) a.escale[(size_t)(k - a.n_tips) * a.escale_stride + c] = e;
      }
      continue;
    }
    // Root: L_c = sum_r w_r pi' p_root (Eq. 3), with the exponents restored.
    double lr = 0.0;
    if (active) {
#pragma unroll
      for (int s = 0; s < SP; ++s)
        if (s < S) lr += a.root_pi[s] * (double)p[s];
      lr *= a.cat_w[r];
    }
    lr = sum_over_lanes<RP>(lr);
    double term = 0.0, unused = 0.0;
    if (valid_c && r == 0) {
      if (!(lr > 0.0) || !isfinite(lr)) atomicOr(a.err, ERR_ZERO_PARTIAL);
      term = a.pattern_w[c] * (log(lr) + (double)e * 0.69314718055994530942);
    }
    block_sum2<NT>(term, unused, red);
    if (threadIdx.x == 0) a.lpart[blockIdx.x] = term;
  }
}

// Pre-order staging (thread 0): Q (host-written) and only what the node's
// children read, P' and dP' of a compact tip (its U and numerator are
// lookups) and P of an internal child (q_x = P' a_x); a tip with partials
// needs neither.
template <int RP, int NPT>
__device__ __forceinline__ void pre_u20_stage(const LevelArgs<float>& a, const int4 (&d)[NPT],
                                              int nn, float* mats, float* Qm, uint64_t* bar) {
  constexpr int SP = kU20, MS = MatStride<float, SP>::v, NS = 6;
  if (threadIdx.x != 0) return;
  const int fl[2] = {kDescCompactX, kDescCompactY};
  uint32_t nmat = 0;
  for (int u = 0; u < nn; ++u) {
    const int br[2] = {d[u].y, d[u].z};
    for (int x = 0; x < 2; ++x) nmat += (d[u].w & fl[x]) ? 2 : (br[x] >= a.n_tips);
  }
  mbar_expect_tx(bar, (uint32_t)((nmat * a.n_cat + 1) * SP * SP * sizeof(float)));
  bulk_g2s(Qm, a.qmat, (uint32_t)(SP * SP * sizeof(float)), bar);
  for (int u = 0; u < nn; ++u) {
    const int br[2] = {d[u].y, d[u].z};
    float* slots = mats + (size_t)(NS * u) * RP * MS;
    for (int x = 0; x < 2; ++x)
      for (int kind = 0; kind < kP4MatKinds; ++kind)
        if ((d[u].w & fl[x]) ? kind < 2 : (kind == 2 && br[x] >= a.n_tips))
          issue_mats<float, SP, RP>(a.P, br + x, 1, a.n_cat,
                                    slots + (size_t)(2 * kind + x) * RP * MS, bar, kP4MatKinds,
                                    kind);
  }
}

// Pre-order level with the fused gradient: slots per node [P'_i | P'_j |
// dP'_i | dP'_j | P_i | P_j] (every category), then Q (one matrix).
template <int RP, int NPT>
__global__ void __launch_bounds__(kSmallThreads, PHYLO_U20_PRE_BLOCKS)
pre_u20_kernel(LevelArgs<float> a) {
  constexpr int SP = kU20, NT = kSmallThreads, CT = NT / RP;
  constexpr int MS = MatStride<float, SP>::v;
  constexpr int NS = 6;
  using SV = SmallVec<float, SP, RP>;
  extern __shared__ __align__(16) unsigned char smraw[];
  float* mats = reinterpret_cast<float*>(smraw);  // [NPT][NS][RP][MS]
  float* Qm = mats + (size_t)NPT * NS * RP * MS;  // Q, row-major SP x SP
  __shared__ uint64_t bar;
  __shared__ F2 red[NT / 32][2];
  const int g0 = blockIdx.y * NPT;
  const int nn = min(NPT, a.n_level - g0);
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int c = blockIdx.x * CT + threadIdx.x / RP;
  const int r = threadIdx.x % RP;
  const bool valid_c = c < C;
  const bool active = valid_c && r < R;
  const int rr = r < R ? r : 0;
  if (threadIdx.x == 0) mbar_init_fenced(&bar, 1);
  __syncthreads();
  int4 d[NPT];  // host-written: readable before the wait
#pragma unroll
  for (int u = 0; u < NPT; ++u)
    d[u] = u < nn ? a.level_desc[g0 + u] : make_int4(0, 0, 0, 0);
  if (a.mats_ready) pre_u20_stage<RP, NPT>(a, d, nn, mats, Qm, &bar);
  pdl_wait_and_release();
  if (!a.mats_ready) pre_u20_stage<RP, NPT>(a, d, nn, mats, Qm, &bar);
  float q[NPT][SP];
  ChildIn<float, SP> in[NPT][2];
#pragma unroll
  for (int u = 0; u < NPT; ++u) {
    if (u >= nn) continue;
    const int k = d[u].x;
    if (k == a.root) {
#pragma unroll
      for (int s = 0; s < SP; ++s) q[u][s] = (active && s < S) ? a.root_pit[s] : 0.f;
    } else {
      load_vec<float, SP>(a.pre + SV::offset(k - a.n_tips, c, r, R, C, a.n_tiles), q[u], active,
                          SV::cs);
    }
    load_u20<RP>(a, d[u].y, d[u].w & kDescCompactX, c, r, active, false, in[u][0]);
    load_u20<RP>(a, d[u].z, d[u].w & kDescCompactY, c, r, active, false, in[u][1]);
  }
  const float w = active ? a.cat_wt[r] : 0.f;
  const float gam = active ? (float)a.rates[r] : 0.f;
  if (!__syncthreads_and(mbar_wait(&bar, 0))) {
    if (threadIdx.x == 0) atomicOr(a.err, ERR_TIMEOUT);
    return;
  }
  using A = Acc<float>;
#pragma unroll
  for (int u = 0; u < NPT; ++u) {
    if (u >= nn) break;
    const int b[2] = {d[u].y, d[u].z};
    float ux[2][SP];
    u20_resolve(in[u][0], S, mats + ((NS * u) * RP + rr) * MS, ux[0]);
    u20_resolve(in[u][1], S, mats + ((NS * u + 1) * RP + rr) * MS, ux[1]);
    float den = 0.f;
#pragma unroll
    for (int s = 0; s < SP; ++s) den = fmaf(q[u][s] * ux[1][s], ux[0][s], den);
    float num[2];
    typename A::type g[2];
    // Both children stored: a_0' Q and a_1' Q in one pass over Q's rows (the
    // same operations in the same order as one rowcomb2 per child).
    const bool both_q = in[u][0].y < 0 && in[u][1].y < 0;
    if (both_q) {
      float2 w0[SP / 2], w1[SP / 2];
#pragma unroll
      for (int p = 0; p < SP / 2; ++p) w0[p] = w1[p] = make_float2(0.f, 0.f);
#pragma unroll
      for (int i = 0; i < SP; ++i) {
        const float2 a0 = make_float2(q[u][i] * ux[1][i], q[u][i] * ux[1][i]);
        const float2 a1 = make_float2(q[u][i] * ux[0][i], q[u][i] * ux[0][i]);
        const float2* row = reinterpret_cast<const float2*>(Qm + i * SP);
#pragma unroll
        for (int p = 0; p < SP / 2; ++p) {
          const float2 qr = row[p];
          w0[p] = __ffma2_rn(qr, a0, w0[p]);
          w1[p] = __ffma2_rn(qr, a1, w1[p]);
        }
      }
      float n0 = 0.f, n1 = 0.f;
#pragma unroll
      for (int p = 0; p < SP / 2; ++p) {
        n0 = fmaf(w0[p].x, ux[0][2 * p], n0);
        n0 = fmaf(w0[p].y, ux[0][2 * p + 1], n0);
        n1 = fmaf(w1[p].x, ux[1][2 * p], n1);
        n1 = fmaf(w1[p].y, ux[1][2 * p + 1], n1);
      }
      num[0] = n0 * gam;
      num[1] = n1 * gam;
    }
#pragma unroll
    for (int x = 0; x < 2; ++x) {
      float av[SP];  // a_x = q_k o U_y
#pragma unroll
      for (int s = 0; s < SP; ++s) av[s] = q[u][s] * ux[1 - x][s];
      const int y = in[u][x].y;
      float nx = 0.f;
      if (both_q) {
        nx = num[x];
      } else if (y >= 0) {  // compact tip: a_x' dP_x e_y, from row y of dP' (0 for a gap)
        if (y < S) {
          const float* Dt = mats + ((NS * u + 2 + x) * RP + rr) * MS;
#pragma unroll
          for (int s = 0; s < SP; ++s) nx = fmaf(av[s], Dt[y * SP + s], nx);
        }
      } else {       // gamma_r (a_x' Q) U_x
        float wq[SP];
        rowcomb2<SP>(Qm, av, wq);
#pragma unroll
        for (int s = 0; s < SP; ++s) nx = fmaf(wq[s], ux[x][s], nx);
        nx *= gam;
      }
      num[x] = nx;
      if (b[x] >= a.n_tips) {  // q_x = P_x' a_x, rescaled (only ratios use it)
        float out[SP];
        rowcomb2<SP>(mats + ((NS * u + 4 + x) * RP + rr) * MS, av, out);
        const float m = pattern_max<float, SP, RP>(out, active);
        rescale<float, SP>(out, m, valid_c, a.err);
        if (active)
          store_vec<float, SP>(a.pre + SV::offset(b[x] - a.n_tips, c, r, R, C, a.n_tiles), out,
                               SV::cs);
      }
    }
    // sum over categories (Eq. 8) in FP32, then the ratio
    const float Ni = sum_over_lanes<RP>(w * num[0]);
    const float Nj = sum_over_lanes<RP>(w * num[1]);
    const float D = sum_over_lanes<RP>(w * den);
    g[0] = A::zero();
    g[1] = A::zero();
    if (valid_c && r == 0) {
      if (!(D > 0.f) || !isfinite(D)) {
        atomicOr(a.err, ERR_BAD_RATIO);
      } else {
        const float W = a.pattern_wt[c];
        g[0] = A::prod(W, Ni / D);
        g[1] = A::prod(W, Nj / D);
      }
    }
    block_sum_acc<float, NT>(g[0], g[1], red, RP);
    if (threadIdx.x == 0) {  // the pair as stored (the reduction converts to FP64)
      float2* gp = reinterpret_cast<float2*>(a.gpart);
      gp[(size_t)b[0] * a.n_tiles + blockIdx.x] = make_float2(g[0].hi, g[0].lo);
      gp[(size_t)b[1] * a.n_tiles + blockIdx.x] = make_float2(g[1].hi, g[1].lo);
    }
    __syncthreads();  // red[] is reused by the next node
  }
}

template <int RP, int NPT>
constexpr size_t u20_smem(bool post) {
  return ((size_t)NPT * (post ? 3 : 6) * RP + (post ? 0 : 1)) * MatStride<float, kU20>::v *
         sizeof(float);
}

// ---------------------------------------------------------------------------
// Shared-memory kernels for SP = 64 (S in 21..64): one thread per (pattern
// group, state s); each thread owns CPG patterns of its group; categories
// are processed one at a time with that category's matrices staged in a
// padded (stride SP+1, bank-conflict-free both ways) shared layout.
// ---------------------------------------------------------------------------
template <typename T> struct WideCfg;
template <> struct WideCfg<float> { static constexpr int CT = kWidePatternsF32; };
template <> struct WideCfg<double> { static constexpr int CT = kWidePatternsF64; };

constexpr int kWideSP = 64;
constexpr int kWideLD = kWideSP + 1;

template <typename T>
__device__ __forceinline__ void stage_mat_padded(const T* __restrict__ src,
                                                 T* dst) {
  for (int idx = threadIdx.x; idx < kWideSP * kWideSP; idx += blockDim.x) {
    const int s = idx / kWideSP, t = idx % kWideSP;
    dst[s * kWideLD + t] = src[idx];
  }
}

// Stage child vectors for category r into vin[CT][SP]; tips with compact
// states store their state in ystate[CT] instead.
template <typename T>
__device__ __forceinline__ void stage_child_vec(const LevelArgs<T>& a, int b,
                                                int c0, int r, T* vin,
                                                int* ystate) {
  constexpr int CT = WideCfg<T>::CT;
  const int C = a.n_patterns, R = a.n_cat;
  const bool compact =
      b < a.n_tips && !(a.tip_has_partials && a.tip_has_partials[b]);
  if (compact) {
    for (int j = threadIdx.x; j < CT; j += blockDim.x) {
      const int c = c0 + j;
      ystate[j] = c < C ? (int)a.tip_states[(size_t)b * a.state_stride + c] : 0;
    }
    return;
  }
  for (int idx = threadIdx.x; idx < CT * kWideSP; idx += blockDim.x) {
    const int j = idx / kWideSP, s = idx % kWideSP, c = c0 + j;
    T v = T(0);
    if (c < C) {
      if (b < a.n_tips)
        v = a.tip_partials[((size_t)b * C + c) * kWideSP + s];
      else
        v = a.post[(((size_t)(b - a.n_tips) * C + c) * R + r) * kWideSP + s];
    }
    vin[j * kWideSP + s] = v;
  }
  if (threadIdx.x < CT) ystate[threadIdx.x] = -1;
}

// u = M v for state s of pattern j (M padded in smem).
template <typename T>
__device__ __forceinline__ T wide_up(const T* M, const T* vin, const int* ys,
                                     int j, int s, int S) {
  const int y = ys[j];
  if (y >= 0) {
    if (y < S) return M[s * kWideLD + y];
    return s < S ? T(1) : T(0);
  }
  const T* v = vin + j * kWideSP;
  T acc = T(0);
#pragma unroll 16
  for (int t = 0; t < kWideSP; ++t) acc = fma(M[s * kWideLD + t], v[t], acc);
  return acc;
}

template <typename T>
__device__ __forceinline__ T wide_up_gap_d(const int* ys, int j, int S,
                                           T dval) {
  // derivative of a gap tip's all-ones vector is exactly 0
  const int y = ys[j];
  return (y >= S) ? T(0) : dval;
}

template <typename T>
struct WideSmemPost {
  T mat[2][kWideSP * kWideLD];
  T vin[2][WideCfg<T>::CT * kWideSP];
  T pk[8][WideCfg<T>::CT * kWideSP];
  int ys[2][WideCfg<T>::CT];
  T redm[WideCfg<T>::CT][kWideThreads / 32];
  double redl[kWideThreads / 32][2];
};

template <typename T>
__global__ void __launch_bounds__(kWideThreads) post_wide_kernel(LevelArgs<T> a) {
  pdl_wait_and_release();
  constexpr int CT = WideCfg<T>::CT;
  constexpr int NT = kWideThreads;
  constexpr int GROUPS = NT / kWideSP;  // 4
  constexpr int CPG = CT / GROUPS;      // patterns per thread
  extern __shared__ __align__(16) unsigned char smraw[];
  WideSmemPost<T>& sm = *reinterpret_cast<WideSmemPost<T>*>(smraw);
  const int k = a.level_nodes[blockIdx.y];
  const int2 ch = a.children[k];
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int c0 = blockIdx.x * CT;
  const int g = threadIdx.x / kWideSP, s = threadIdx.x % kWideSP;
  int eacc[CPG];
#pragma unroll
  for (int jj = 0; jj < CPG; ++jj) eacc[jj] = 0;
  for (int r = 0; r < R; ++r) {
    __syncthreads();
    stage_mat_padded<T>(a.P + ((size_t)ch.x * R + r) * kWideSP * kWideSP,
                        sm.mat[0]);
    stage_mat_padded<T>(a.P + ((size_t)ch.y * R + r) * kWideSP * kWideSP,
                        sm.mat[1]);
    stage_child_vec<T>(a, ch.x, c0, r, sm.vin[0], sm.ys[0]);
    stage_child_vec<T>(a, ch.y, c0, r, sm.vin[1], sm.ys[1]);
    __syncthreads();
#pragma unroll
    for (int jj = 0; jj < CPG; ++jj) {
      const int j = g * CPG + jj;
      const T ui = wide_up<T>(sm.mat[0], sm.vin[0], sm.ys[0], j, s, S);
      const T uj = wide_up<T>(sm.mat[1], sm.vin[1], sm.ys[1], j, s, S);
      sm.pk[r][j * kWideSP + s] = ui * uj;
    }
  }
  __syncthreads();
  // exponents of the children (internal ones)
  for (int jj = 0; jj < CPG; ++jj) {
    const int j = g * CPG + jj, c = c0 + j;
    int e = 0;
    if (c < C) {
      if (ch.x >= a.n_tips) e += a.escale[(size_t)(ch.x - a.n_tips) * a.escale_stride + c];
      if (ch.y >= a.n_tips) e += a.escale[(size_t)(ch.y - a.n_tips) * a.escale_stride + c];
    }
    eacc[jj] = e;
  }
  // max over (r, s) per pattern: 64 threads of the group = 2 warps
  const int warp = threadIdx.x >> 5;
#pragma unroll
  for (int jj = 0; jj < CPG; ++jj) {
    const int j = g * CPG + jj;
    T m = T(0);
    for (int r = 0; r < R; ++r) m = tmax(m, fabs(sm.pk[r][j * kWideSP + s]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = tmax(m, __shfl_xor_sync(kFull, m, o));
    if ((threadIdx.x & 31) == 0) sm.redm[j][warp] = m;
  }
  __syncthreads();
  double lterm = 0.0;
#pragma unroll
  for (int jj = 0; jj < CPG; ++jj) {
    const int j = g * CPG + jj, c = c0 + j;
    const T m = tmax(sm.redm[j][2 * g], sm.redm[j][2 * g + 1]);
    int e = 0;
    if (c < C) {
      if (!(m > T(0)) || !isfinite(m)) atomicOr(a.err, ERR_ZERO_PARTIAL);
      else (void)frexp(m, &e);
    }
    const T f = ldexp(T(1), -e);
    const int etot = e + eacc[jj];
    if (k != a.root) {
      if (c < C) {
        const size_t slot = (size_t)(k - a.n_tips);
        for (int r = 0; r < R; ++r)
          a.post[((slot * C + c) * R + r) * kWideSP + s] =
              sm.pk[r][j * kWideSP + s] * f;
        if (s == 0) a.escale[slot * a.escale_stride + c] = etot;
      }
    } else {
      // root: sum_r w_r pi' p over the group's 64 threads
      double lr = 0.0;
      if (c < C && s < S)
        for (int r = 0; r < R; ++r)
          lr += a.cat_w[r] * a.root_pi[s] *
                (double)(sm.pk[r][j * kWideSP + s] * f);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) lr += __shfl_xor_sync(kFull, lr, o);
      // combine the group's two warps through shared memory
      __syncthreads();
      if ((threadIdx.x & 31) == 0) sm.redl[warp][0] = lr;
      __syncthreads();
      if (s == 0 && c < C) {
        const double L = sm.redl[2 * g][0] + sm.redl[2 * g + 1][0];
        if (!(L > 0.0) || !isfinite(L)) atomicOr(a.err, ERR_ZERO_PARTIAL);
        lterm += a.pattern_w[c] * (log(L) + (double)etot * 0.69314718055994530942);
      }
    }
  }
  if (k == a.root) {
    __syncthreads();
    double unused = 0.0;
    block_sum2<NT>(lterm, unused, sm.redl);
    if (threadIdx.x == 0) a.lpart[blockIdx.x] = lterm;
  }
}

template <typename T>
struct WideSmemPre {
  T mat[4][kWideSP * kWideLD];   // P_i, P_j, dP_i, dP_j for one r
  T vin[2][WideCfg<T>::CT * kWideSP];
  T qk[WideCfg<T>::CT * kWideSP];
  T av[2][WideCfg<T>::CT * kWideSP];
  int ys[2][WideCfg<T>::CT];
  T redm[2][WideCfg<T>::CT][kWideThreads / 32];
  typename Acc<T>::type red[kWideThreads / 32][2];
  T redg[3][WideCfg<T>::CT][kWideThreads / 32];
};

template <typename T>
__global__ void __launch_bounds__(kWideThreads) pre_wide_kernel(LevelArgs<T> a) {
  pdl_wait_and_release();
  constexpr int CT = WideCfg<T>::CT;
  constexpr int NT = kWideThreads;
  constexpr int GROUPS = NT / kWideSP;
  constexpr int CPG = CT / GROUPS;
  extern __shared__ __align__(16) unsigned char smraw[];
  WideSmemPre<T>& sm = *reinterpret_cast<WideSmemPre<T>*>(smraw);
  T* qout = reinterpret_cast<T*>(smraw + sizeof(WideSmemPre<T>));  // [2][R][CT][SP]
  const int k = a.level_nodes[blockIdx.y];
  const int2 ch = a.children[k];
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int c0 = blockIdx.x * CT;
  const int g = threadIdx.x / kWideSP, s = threadIdx.x % kWideSP;
  const bool int_i = ch.x >= a.n_tips, int_j = ch.y >= a.n_tips;
  T ni[CPG], nj[CPG], dd[CPG];
#pragma unroll
  for (int jj = 0; jj < CPG; ++jj) { ni[jj] = T(0); nj[jj] = T(0); dd[jj] = T(0); }
  for (int r = 0; r < R; ++r) {
    __syncthreads();
    stage_mat_padded<T>(a.P + ((size_t)ch.x * R + r) * kWideSP * kWideSP, sm.mat[0]);
    stage_mat_padded<T>(a.P + ((size_t)ch.y * R + r) * kWideSP * kWideSP, sm.mat[1]);
    stage_mat_padded<T>(a.dP + ((size_t)ch.x * R + r) * kWideSP * kWideSP, sm.mat[2]);
    stage_mat_padded<T>(a.dP + ((size_t)ch.y * R + r) * kWideSP * kWideSP, sm.mat[3]);
    stage_child_vec<T>(a, ch.x, c0, r, sm.vin[0], sm.ys[0]);
    stage_child_vec<T>(a, ch.y, c0, r, sm.vin[1], sm.ys[1]);
    for (int idx = threadIdx.x; idx < CT * kWideSP; idx += NT) {
      const int j = idx / kWideSP, ss = idx % kWideSP, c = c0 + j;
      T v = T(0);
      if (c < C) {
        if (k == a.root) v = ss < S ? (T)a.root_pi[ss] : T(0);
        else v = a.pre[(((size_t)(k - a.n_tips) * C + c) * R + r) * kWideSP + ss];
      }
      sm.qk[idx] = v;
    }
    __syncthreads();
    const T wr = a.cat_wt[r];
#pragma unroll
    for (int jj = 0; jj < CPG; ++jj) {
      const int j = g * CPG + jj;
      const T ui = wide_up<T>(sm.mat[0], sm.vin[0], sm.ys[0], j, s, S);
      const T uj = wide_up<T>(sm.mat[1], sm.vin[1], sm.ys[1], j, s, S);
      const T vi = wide_up_gap_d<T>(sm.ys[0], j, S,
                                   wide_up<T>(sm.mat[2], sm.vin[0], sm.ys[0], j, s, S));
      const T vj = wide_up_gap_d<T>(sm.ys[1], j, S,
                                   wide_up<T>(sm.mat[3], sm.vin[1], sm.ys[1], j, s, S));
      const T q = sm.qk[j * kWideSP + s];
      const T ai = q * uj, aj = q * ui;
      ni[jj] = fma(wr, ai * vi, ni[jj]);
      nj[jj] = fma(wr, aj * vj, nj[jj]);
      dd[jj] = fma(wr, ai * ui, dd[jj]);
      sm.av[0][j * kWideSP + s] = ai;
      sm.av[1][j * kWideSP + s] = aj;
    }
    __syncthreads();
    // q_child[t = s] = sum_s' P[s'][t] a[s'] for this r (unscaled)
#pragma unroll
    for (int jj = 0; jj < CPG; ++jj) {
      const int j = g * CPG + jj;
      for (int x = 0; x < 2; ++x) {
        if (!(x == 0 ? int_i : int_j)) continue;
        const T* M = sm.mat[x];
        const T* av = sm.av[x] + j * kWideSP;
        T acc = T(0);
#pragma unroll 16
        for (int sp = 0; sp < kWideSP; ++sp) acc = fma(M[sp * kWideLD + s], av[sp], acc);
        qout[((x * R + r) * CT + j) * kWideSP + s] = acc;
      }
    }
  }
  // Gradient ratio per pattern: reduce ni, nj, dd over the group's 64 states.
  const int warp = threadIdx.x >> 5;
#pragma unroll
  for (int jj = 0; jj < CPG; ++jj) {
    const int j = g * CPG + jj;
    T x0 = ni[jj], x1 = nj[jj], x2 = dd[jj];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      x0 += __shfl_xor_sync(kFull, x0, o);
      x1 += __shfl_xor_sync(kFull, x1, o);
      x2 += __shfl_xor_sync(kFull, x2, o);
    }
    if ((threadIdx.x & 31) == 0) {
      sm.redg[0][j][warp] = x0; sm.redg[1][j][warp] = x1; sm.redg[2][j][warp] = x2;
    }
  }
  // Max of each child's unscaled q over (r, s) per pattern.
  __syncthreads();
#pragma unroll
  for (int jj = 0; jj < CPG; ++jj) {
    const int j = g * CPG + jj;
    for (int x = 0; x < 2; ++x) {
      T m = T(0);
      if (x == 0 ? int_i : int_j)
        for (int r = 0; r < R; ++r)
          m = tmax(m, fabs(qout[((x * R + r) * CT + j) * kWideSP + s]));
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = tmax(m, __shfl_xor_sync(kFull, m, o));
      if ((threadIdx.x & 31) == 0) sm.redm[x][j][warp] = m;
    }
  }
  __syncthreads();
  using A = Acc<T>;
  typename A::type gi = A::zero(), gj = A::zero();
#pragma unroll
  for (int jj = 0; jj < CPG; ++jj) {
    const int j = g * CPG + jj, c = c0 + j;
    if (c >= C) continue;
    if (s == 0) {
      const T Ni = sm.redg[0][j][2 * g] + sm.redg[0][j][2 * g + 1];
      const T Nj = sm.redg[1][j][2 * g] + sm.redg[1][j][2 * g + 1];
      const T D = sm.redg[2][j][2 * g] + sm.redg[2][j][2 * g + 1];
      if (!(D > T(0)) || !isfinite(D)) {
        atomicOr(a.err, ERR_BAD_RATIO);
      } else {
        gi = A::add(gi, A::prod(a.pattern_wt[c], Ni / D));
        gj = A::add(gj, A::prod(a.pattern_wt[c], Nj / D));
      }
    }
    for (int x = 0; x < 2; ++x) {
      const int b = x == 0 ? ch.x : ch.y;
      if (b < a.n_tips) continue;
      const T m = tmax(sm.redm[x][j][2 * g], sm.redm[x][j][2 * g + 1]);
      int e = 0;
      if (!(m > T(0)) || !isfinite(m)) atomicOr(a.err, ERR_ZERO_PARTIAL);
      else (void)frexp(m, &e);
      const T f = ldexp(T(1), -e);
      const size_t slot = (size_t)(b - a.n_tips);
      for (int r = 0; r < R; ++r)
        a.pre[((slot * C + c) * R + r) * kWideSP + s] =
            qout[((x * R + r) * CT + j) * kWideSP + s] * f;
    }
  }
  __syncthreads();
  block_sum_acc<T, NT>(gi, gj, sm.red, 1);
  if (threadIdx.x == 0) {
    a.gpart[(size_t)ch.x * a.n_tiles + blockIdx.x] = A::to_double(gi);
    a.gpart[(size_t)ch.y * a.n_tiles + blockIdx.x] = A::to_double(gj);
  }
}

template <typename T>
inline size_t wide_post_smem() { return sizeof(WideSmemPost<T>); }
template <typename T>
inline size_t wide_pre_smem(int R) {
  return sizeof(WideSmemPre<T>) +
         (size_t)2 * R * WideCfg<T>::CT * kWideSP * sizeof(T);
}

}  // namespace phylo

#include "kernels_p4.cuh"
#include "kernels_tc64.cuh"
#include "kernels_big.cuh"
#include "kernels_tcb.cuh"

namespace phylo {

// ---------------------------------------------------------------------------
// Instantiation of the launchers for one element type.
// ---------------------------------------------------------------------------
// Nodes per block of the register kernels: more inputs in flight per warp,
// bounded by registers (the inputs of all NPT nodes are held at once).
template <typename T, int SP>
struct SmallNpt {
  static constexpr int post = (SP == 4) ? 4 : 2;
  static constexpr int pre = (SP == 4) ? (sizeof(T) == 4 ? 4 : 2) : 1;
};

template <typename T, int SP, int RP, int NPT>
constexpr size_t small_smem(bool post) {
  return (size_t)NPT * (post ? 2 : kPreSlots<T, SP>) * RP * MatStride<T, SP>::v * sizeof(T);
}

template <typename T, int SP, int RP>
cudaError_t launch_small(const LevelArgs<T>& a, bool post, cudaStream_t st) {
  constexpr int NPo = SmallNpt<T, SP>::post, NPr = SmallNpt<T, SP>::pre;
  if constexpr (kTrSmall<T, SP>) {  // FP32, 20 padded states: the U form
    if (post) {
      dim3 grid(a.n_tiles, (a.n_level + NPo - 1) / NPo);
      return launch_pdl(post_u20_kernel<RP, NPo>, grid, kSmallThreads, u20_smem<RP, NPo>(true),
                        st, a);
    }
    dim3 grid(a.n_tiles, (a.n_level + NPr - 1) / NPr);
    return launch_pdl(pre_u20_kernel<RP, NPr>, grid, kSmallThreads, u20_smem<RP, NPr>(false), st,
                      a);
  }
  if (post) {
    dim3 grid(a.n_tiles, (a.n_level + NPo - 1) / NPo);
    return launch_pdl(post_small_kernel<T, SP, RP, NPo>, grid, kSmallThreads,
                      small_smem<T, SP, RP, NPo>(true), st, a);
  }
  dim3 grid(a.n_tiles, (a.n_level + NPr - 1) / NPr);
  return launch_pdl(pre_small_kernel<T, SP, RP, NPr>, grid, kSmallThreads,
                    small_smem<T, SP, RP, NPr>(false), st, a);
}

template <typename T, int SP, int RP>
cudaError_t prepare_small() {
  constexpr int NPo = SmallNpt<T, SP>::post, NPr = SmallNpt<T, SP>::pre;
  if constexpr (kTrSmall<T, SP>) {
    cudaError_t e = cudaFuncSetAttribute(post_u20_kernel<RP, NPo>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)u20_smem<RP, NPo>(true));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(pre_u20_kernel<RP, NPr>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)u20_smem<RP, NPr>(false));
  }
  cudaError_t e = cudaFuncSetAttribute(
      post_small_kernel<T, SP, RP, NPo>, cudaFuncAttributeMaxDynamicSharedMemorySize,
      (int)small_smem<T, SP, RP, NPo>(true));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(pre_small_kernel<T, SP, RP, NPr>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)small_smem<T, SP, RP, NPr>(false));
}

template <typename T, int SP>
cudaError_t prepare_small_rp(int RP) {
  switch (RP) {
    case 1: return prepare_small<T, SP, 1>();
    case 2: return prepare_small<T, SP, 2>();
    case 4: return prepare_small<T, SP, 4>();
    case 8: return prepare_small<T, SP, 8>();
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int SP>
cudaError_t launch_small_rp(const LevelArgs<T>& a, int RP, bool post,
                            cudaStream_t st) {
  switch (RP) {
    case 1: return launch_small<T, SP, 1>(a, post, st);
    case 2: return launch_small<T, SP, 2>(a, post, st);
    case 4: return launch_small<T, SP, 4>(a, post, st);
    case 8: return launch_small<T, SP, 8>(a, post, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t launch_level_impl(const LevelArgs<T>& a, int SP, int RP, bool post,
                              cudaStream_t st) {
  if (a.n_tiles <= 0 || a.n_level <= 0) return cudaSuccess;
  switch (SP) {
    case 4:
      if constexpr (std::is_same<T, float>::value) return launch_p4_rp(a, RP, post, st);
      else return launch_small_rp<T, 4>(a, RP, post, st);
    case 20: return launch_small_rp<T, 20>(a, RP, post, st);
    case 64:
      if constexpr (std::is_same<T, float>::value) {
        return launch_tc64(a, post, st);
      } else {
        dim3 grid(a.n_tiles, a.n_level);
        if (post)
          return launch_pdl(post_wide_kernel<T>, grid, kWideThreads, wide_post_smem<T>(), st, a);
        return launch_pdl(pre_wide_kernel<T>, grid, kWideThreads, wide_pre_smem<T>(a.n_cat), st,
                          a);
      }
    case 128:
      if constexpr (std::is_same<T, float>::value) return launch_tcb(a, post, st);
      else return launch_big<T, 128>(a, post, st);
    case 256: return launch_big<T, 256>(a, post, st);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T>
cudaError_t prepare_impl(int SP, int RP) {
  if (SP == 4) return prepare_small_rp<T, 4>(RP);
  if (SP == 20) return prepare_small_rp<T, 20>(RP);
  if (SP == 64) {
    if constexpr (std::is_same<T, float>::value) {
      return prepare_tc64();
    } else {
      cudaError_t e = cudaFuncSetAttribute(
          post_wide_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
          (int)wide_post_smem<T>());
      if (e != cudaSuccess) return e;
      return cudaFuncSetAttribute(pre_wide_kernel<T>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)wide_pre_smem<T>(8));
    }
  }
  if (SP == 128) {
    if constexpr (std::is_same<T, float>::value) return prepare_tcb();
    else return prepare_big<T, 128>();
  }
  if (SP == 256) return prepare_big<T, 256>();
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_pmat_impl(const PmatArgs& a, int SP, cudaStream_t st) {
  const int units = a.n_branches * a.n_cat;
  if (units <= 0) return cudaSuccess;
  switch (SP) {
    case 4:
      if constexpr (std::is_same<T, float>::value) {
        return launch_pmat_df_small<4>(a, st);
      } else {
        constexpr int UPB = 256 / 16;
        pmat_kernel<T, 4><<<(units + UPB - 1) / UPB, 256, 0, st>>>(a);
      }
      break;
    case 20:
      if constexpr (std::is_same<T, float>::value) return launch_pmat_df_small<20>(a, st);
      else pmat_kernel<T, 20><<<units, 256, 0, st>>>(a);
      break;
    case 64:
      if constexpr (std::is_same<T, float>::value) return launch_pmat_tc64(a, st);
      else pmat_kernel<T, 64><<<units, 256, 0, st>>>(a);
      break;
    case 128:
      if constexpr (std::is_same<T, float>::value) return launch_pmat_tcb(a, st);
      else pmat_kernel<T, 128><<<units, 256, 0, st>>>(a);
      break;
    case 256:
      if constexpr (std::is_same<T, float>::value) return launch_pmat_big<256>(a, st);
      else pmat_kernel<T, 256><<<units, 256, 0, st>>>(a);
      break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_pre_finish_impl(const LevelArgs<T>& a, int SP, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (SP == 64 || SP == 128) return launch_ratio_tc64(a, st);
  }
  return cudaSuccess;
}

}  // namespace phylo

#define PHYLO_INSTANTIATE(T)                                                  \
  namespace phylo {                                                           \
  template <>                                                                 \
  cudaError_t launch_pmat<T>(const PmatArgs& a, int SP, cudaStream_t st) {    \
    return launch_pmat_impl<T>(a, SP, st);                                    \
  }                                                                           \
  template <>                                                                 \
  cudaError_t launch_post_level<T>(const LevelArgs<T>& a, int SP, int RP,     \
                                   cudaStream_t st) {                         \
    return launch_level_impl<T>(a, SP, RP, true, st);                         \
  }                                                                           \
  template <>                                                                 \
  cudaError_t launch_pre_level<T>(const LevelArgs<T>& a, int SP, int RP,      \
                                  cudaStream_t st) {                          \
    return launch_level_impl<T>(a, SP, RP, false, st);                        \
  }                                                                           \
  template <>                                                                 \
  cudaError_t launch_pre_finish<T>(const LevelArgs<T>& a, int SP,             \
                                   cudaStream_t st) {                         \
    return launch_pre_finish_impl<T>(a, SP, st);                              \
  }                                                                           \
  template <>                                                                 \
  cudaError_t prepare_kernels<T>(int SP, int RP) {                            \
    return prepare_impl<T>(SP, RP);                                           \
  }                                                                           \
  }
