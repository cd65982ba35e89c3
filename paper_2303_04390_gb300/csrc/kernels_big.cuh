// Level kernels for 65..256 states (S_pad 128 or 256), FP64 and FP32, on the
// CUDA cores: Eq. 2 (with Eq. 3 at the root) and Eq. 4 with the Eq. 8 ratio
// fused, as in the other level kernels, for state spaces whose transition
// matrices do not fit in shared memory -- the paper's 122-state
// Markov-modulated codon model (Results) and 256-state models (Discussion).
//
// A block takes a tile of CT patterns of one node and loops over the rate
// categories.  Thread (g, s) owns states s, s + TPG, ... (SPT of them, TPG =
// S_pad / SPT) of the patterns g*CPG .. g*CPG + CPG - 1 (G = 256 / TPG
// groups).  A matrix-vector product streams the matrix through shared
// memory in chunks, copied in by per-thread asynchronous copies into two
// buffers so that the next chunk is in flight while one is used:
//   u = M v   (Eq. 2, and P p, dP p of Eq. 8): chunks of KC columns; each
//             thread reads its SPT rows of the chunk, the patterns' vector
//             chunks are staged beside it and read as broadcasts;
//   q = M' a  (Eq. 4): chunks of KC rows; each thread reads its SPT columns,
//             a is read from shared memory as a broadcast.
// Rescaling follows the other kernels: one power of two per (node, pattern)
// shared by every category and state; the unscaled values are stored first
// and scaled in place once the block knows the pattern's maximum (each
// thread rescales only what it wrote).
#pragma once

namespace phylo {

constexpr int kBigThreads = 256;
// Two resident blocks for S_pad = 128 (registers capped at 128), one for
// 256.  Measured on the 122-state workload (FP32), post- + pre-order ms per
// evaluation: 16-pattern tiles, 32-column chunks staged through registers,
// one block per SM: 5.8 + 11.8; 8-pattern tiles, 64-column chunks, two
// blocks: 3.4 + 7.9; asynchronous copies into two 32-column buffers:
// 2.8 + 6.9; two states per thread with 16-pattern tiles: 2.2 + 5.4.
template <int SP> constexpr int kBigMinBlocks = SP == 128 ? 2 : 1;

// CT: patterns per block; KC: matrix columns (rows) per chunk; ST: chunk
// buffers; SPT: states per thread (each matrix read then feeds SPT rows).
template <typename T> struct BigCfg;
template <> struct BigCfg<float> {
  static constexpr int CT = kBigPatternsF32, KC = 32, ST = 2, SPT = kBigStatesPerThread;
};
template <> struct BigCfg<double> {
  static constexpr int CT = kBigPatternsF64, KC = 16, ST = 2, SPT = 1;
};

// Shared-memory plan of one block (element counts of T).
template <typename T, int SP>
struct BigPlan {
  static constexpr int CT = BigCfg<T>::CT, KC = BigCfg<T>::KC, ST = BigCfg<T>::ST;
  static constexpr int SPT = BigCfg<T>::SPT, TPG = SP / SPT;
  static constexpr int G = kBigThreads / TPG, CPG = CT / G;
  static constexpr int KP = KC + 16 / (int)sizeof(T);  // padded rows: no bank conflicts
  static constexpr int WPG = TPG / 32;                  // warps per group
  static constexpr size_t stage = 2 * (size_t)SP * KP;  // one buffer: row-chunks of M, dM
  static constexpr size_t mat = ST * stage;
  static constexpr size_t vec = (size_t)ST * CT * KC;   // the patterns' vector chunks
  static constexpr size_t uw = 2 * (size_t)CT * SP;     // U, W (pre-order)
  static constexpr size_t red = (size_t)CT * WPG;       // per-pattern partial sums
  static size_t bytes(bool pre) { return (mat + vec + (pre ? uw : 0) + red) * sizeof(T); }
  static_assert((size_t)KC * SP <= stage, "column chunk fits in a row-chunk buffer");
  static_assert(SP % KC == 0 && KC % 4 == 0, "whole chunks");
  static_assert(CT % G == 0 && TPG % 32 == 0 && CPG >= 1, "tile shape");
};

template <typename T> struct BigVec;
template <> struct BigVec<float> { using type = float4; static constexpr int n = 4; };
template <> struct BigVec<double> { using type = double2; static constexpr int n = 2; };

__device__ __forceinline__ float big_dot(float4 a, float4 b, float acc) {
  acc = fmaf(a.x, b.x, acc);
  acc = fmaf(a.y, b.y, acc);
  acc = fmaf(a.z, b.z, acc);
  return fmaf(a.w, b.w, acc);
}
__device__ __forceinline__ double big_dot(double2 a, double2 b, double acc) {
  acc = fma(a.x, b.x, acc);
  return fma(a.y, b.y, acc);
}
__device__ __forceinline__ float big_el(float4 v, int i) {
  return i == 0 ? v.x : i == 1 ? v.y : i == 2 ? v.z : v.w;
}
__device__ __forceinline__ double big_el(double2 v, int i) { return i == 0 ? v.x : v.y; }

// One child's vectors for category r: where they come from.
template <typename T>
struct BigChild {
  int b;            // node
  bool compact;     // tip with compact states (column lookups)
  const T* src;     // else: pattern c0's vector; pattern j at src + j * stride
  size_t stride;
};

template <typename T>
__device__ __forceinline__ BigChild<T> big_child(const LevelArgs<T>& a, int b, int c0, int r,
                                                 int SP) {
  BigChild<T> x;
  x.b = b;
  x.compact = b < a.n_tips && !(a.tip_has_partials && a.tip_has_partials[b]);
  if (b < a.n_tips) {
    x.src = a.tip_partials + (size_t)b * a.n_patterns * SP + (size_t)c0 * SP;
    x.stride = SP;
  } else {
    x.src = a.post + (((size_t)(b - a.n_tips) * a.n_patterns + c0) * a.n_cat + r) * SP;
    x.stride = (size_t)a.n_cat * SP;
  }
  return x;
}

// u[i][jj] = (M v_j)[s + i*TPG] and, with dM, w[i][jj] = (dM v_j)[...] for
// the thread's patterns j = g*CPG + jj.  M, dM: global [SP][SP] (padded
// rows/columns 0).  Every thread of the block calls this (it synchronises).
template <typename T, int SP, bool WITH_D>
__device__ __forceinline__ void big_row_mv(
    const LevelArgs<T>& a, const BigChild<T>& x, const T* __restrict__ M,
    const T* __restrict__ dM, int c0, int nvalid, T* smat, T* svec, int g, int s,
    T (&u)[BigPlan<T, SP>::SPT][BigPlan<T, SP>::CPG],
    T (&w)[BigPlan<T, SP>::SPT][BigPlan<T, SP>::CPG]) {
  using PL = BigPlan<T, SP>;
  constexpr int CPG = PL::CPG, KC = PL::KC, KP = PL::KP, CT = PL::CT, SPT = PL::SPT,
                TPG = PL::TPG;
  using V = typename BigVec<T>::type;
  constexpr int VN = BigVec<T>::n;
#pragma unroll
  for (int i = 0; i < SPT; ++i)
#pragma unroll
    for (int jj = 0; jj < CPG; ++jj) { u[i][jj] = T(0); w[i][jj] = T(0); }
  if (x.compact) {  // a column of M (gap: all ones, derivative 0)
    const int S = a.n_states;
#pragma unroll
    for (int jj = 0; jj < CPG; ++jj) {
      const int j = g * CPG + jj;
      if (j >= nvalid) continue;
      const int y = a.tip_states[(size_t)x.b * a.state_stride + c0 + j];
#pragma unroll
      for (int i = 0; i < SPT; ++i) {
        const int si = s + i * TPG;
        if (y < S) {
          u[i][jj] = M[(size_t)si * SP + y];
          if (WITH_D) w[i][jj] = dM[(size_t)si * SP + y];
        } else {
          u[i][jj] = si < S ? T(1) : T(0);
        }
      }
    }
    return;
  }
  constexpr int ST = PL::ST, NCH = SP / KC;
  // chunk k -> buffer b: per-thread asynchronous copies, one commit group
  auto issue = [&](int k, int b) {
    const int t0 = k * KC;
    T* sM = smat + (size_t)b * PL::stage;
    T* sD = sM + (size_t)SP * KP;
    for (int i = threadIdx.x; i < SP * (KC / VN); i += kBigThreads) {
      const int row = i / (KC / VN), cv = i % (KC / VN);
      cp_async16(sM + (size_t)row * KP + cv * VN, M + (size_t)row * SP + t0 + cv * VN);
      if (WITH_D) cp_async16(sD + (size_t)row * KP + cv * VN, dM + (size_t)row * SP + t0 + cv * VN);
    }
    T* sv = svec + (size_t)b * CT * KC;
    for (int i = threadIdx.x; i < CT * (KC / VN); i += kBigThreads) {
      const int j = i / (KC / VN), cv = i % (KC / VN);
      if (j < nvalid) cp_async16(sv + j * KC + cv * VN, x.src + (size_t)j * x.stride + t0 + cv * VN);
      else *reinterpret_cast<V*>(sv + j * KC + cv * VN) = V{};
    }
    cp_async_commit();
  };
  __syncthreads();  // the buffers' previous readers are done
  issue(0, 0);
  for (int k = 0; k < NCH; ++k) {
    if (ST > 1 && k + 1 < NCH) {
      issue(k + 1, (k + 1) % ST);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();  // every thread's copies of chunk k have landed
    const int b = ST > 1 ? k % ST : 0;
    const T* sM = smat + (size_t)b * PL::stage;
    const T* sD = sM + (size_t)SP * KP;
    const T* sv = svec + (size_t)b * CT * KC;
#pragma unroll 2
    for (int tt = 0; tt < KC; tt += VN) {
      V m[SPT], d[SPT];
#pragma unroll
      for (int i = 0; i < SPT; ++i) {
        m[i] = *reinterpret_cast<const V*>(sM + (size_t)(s + i * TPG) * KP + tt);
        d[i] = V{};
        if (WITH_D) d[i] = *reinterpret_cast<const V*>(sD + (size_t)(s + i * TPG) * KP + tt);
      }
#pragma unroll
      for (int jj = 0; jj < CPG; ++jj) {
        const V v = *reinterpret_cast<const V*>(sv + (g * CPG + jj) * KC + tt);
#pragma unroll
        for (int i = 0; i < SPT; ++i) {
          u[i][jj] = big_dot(m[i], v, u[i][jj]);
          if (WITH_D) w[i][jj] = big_dot(d[i], v, w[i][jj]);
        }
      }
    }
    __syncthreads();  // chunk k's buffer may be refilled
    if (ST == 1 && k + 1 < NCH) issue(k + 1, 0);
  }
}

// q[i][jj] = (M' a_j)[s + i*TPG], a_j = A[j][*] in shared memory.  Every
// thread of the block calls this (it synchronises).
template <typename T, int SP>
__device__ __forceinline__ void big_col_mv(const T* __restrict__ M, const T* A, T* smat, int g,
                                           int s,
                                           T (&q)[BigPlan<T, SP>::SPT][BigPlan<T, SP>::CPG]) {
  using PL = BigPlan<T, SP>;
  constexpr int CPG = PL::CPG, KC = PL::KC, SPT = PL::SPT, TPG = PL::TPG;
  using V = typename BigVec<T>::type;
  constexpr int VN = BigVec<T>::n;
  constexpr int ST = PL::ST, NCH = SP / KC;
#pragma unroll
  for (int i = 0; i < SPT; ++i)
#pragma unroll
    for (int jj = 0; jj < CPG; ++jj) q[i][jj] = T(0);
  auto issue = [&](int k, int b) {
    T* sb = smat + (size_t)b * PL::stage;
    for (int i = threadIdx.x; i < KC * (SP / VN); i += kBigThreads) {
      const int row = i / (SP / VN), cv = i % (SP / VN);
      cp_async16(sb + (size_t)row * SP + cv * VN, M + (size_t)(k * KC + row) * SP + cv * VN);
    }
    cp_async_commit();
  };
  __syncthreads();
  issue(0, 0);
  for (int k = 0; k < NCH; ++k) {
    if (ST > 1 && k + 1 < NCH) {
      issue(k + 1, (k + 1) % ST);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const T* sb = smat + (size_t)(ST > 1 ? k % ST : 0) * PL::stage;
    const int s0 = k * KC;
#pragma unroll 2
    for (int ss = 0; ss < KC; ss += VN) {
      T m[VN][SPT];
#pragma unroll
      for (int e = 0; e < VN; ++e)
#pragma unroll
        for (int i = 0; i < SPT; ++i) m[e][i] = sb[(size_t)(ss + e) * SP + s + i * TPG];
#pragma unroll
      for (int jj = 0; jj < CPG; ++jj) {
        const V av = *reinterpret_cast<const V*>(A + (size_t)(g * CPG + jj) * SP + s0 + ss);
#pragma unroll
        for (int e = 0; e < VN; ++e)
#pragma unroll
          for (int i = 0; i < SPT; ++i) q[i][jj] = fma(m[e][i], big_el(av, e), q[i][jj]);
      }
    }
    __syncthreads();
    if (ST == 1 && k + 1 < NCH) issue(k + 1, 0);
  }
}

// x[jj] summed (or maximised) over the TPG threads of the group, in a fixed
// order; every thread of the group receives the result.
template <typename T, int SP, bool MAX>
__device__ __forceinline__ void big_group_reduce(T (&x)[BigPlan<T, SP>::CPG], T* red, int g,
                                                 int s) {
  using PL = BigPlan<T, SP>;
  constexpr int CPG = PL::CPG, WPG = PL::WPG;
  const int lane = threadIdx.x & 31, wig = s >> 5;
#pragma unroll
  for (int jj = 0; jj < CPG; ++jj) {
    T v = x[jj];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const T y = __shfl_xor_sync(kFull, v, o);
      v = MAX ? tmax(v, y) : v + y;
    }
    if (lane == 0) red[(g * CPG + jj) * WPG + wig] = v;
  }
  __syncthreads();
#pragma unroll
  for (int jj = 0; jj < CPG; ++jj) {
    T v = red[(g * CPG + jj) * WPG];
    for (int i = 1; i < WPG; ++i) {
      const T y = red[(g * CPG + jj) * WPG + i];
      v = MAX ? tmax(v, y) : v + y;
    }
    x[jj] = v;
  }
  __syncthreads();
}

template <typename T, int SP>
__global__ void __launch_bounds__(kBigThreads, kBigMinBlocks<SP>) post_big_kernel(LevelArgs<T> a) {
  pdl_wait_and_release();
  using PL = BigPlan<T, SP>;
  constexpr int CT = PL::CT, CPG = PL::CPG, SPT = PL::SPT, TPG = PL::TPG;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* smat = reinterpret_cast<T*>(smraw);
  T* svec = smat + PL::mat;
  T* red = svec + PL::vec;
  __shared__ double lred[PL::G];
  const int k = a.level_nodes[blockIdx.y];
  const int2 ch = a.children[k];
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int c0 = blockIdx.x * CT, nvalid = min(CT, C - c0);
  const int s = threadIdx.x % TPG, g = threadIdx.x / TPG;
  const size_t msz = (size_t)SP * SP;
  T mx[CPG], lsum[CPG], pis[SPT];
#pragma unroll
  for (int jj = 0; jj < CPG; ++jj) { mx[jj] = T(0); lsum[jj] = T(0); }
#pragma unroll
  for (int i = 0; i < SPT; ++i) pis[i] = s + i * TPG < S ? (T)a.root_pi[s + i * TPG] : T(0);
  for (int r = 0; r < R; ++r) {
    T ui[SPT][CPG], uj[SPT][CPG], dummy[SPT][CPG];
    const BigChild<T> xi = big_child(a, ch.x, c0, r, SP), xj = big_child(a, ch.y, c0, r, SP);
    big_row_mv<T, SP, false>(a, xi, a.P + ((size_t)ch.x * R + r) * msz, nullptr, c0, nvalid,
                             smat, svec, g, s, ui, dummy);
    big_row_mv<T, SP, false>(a, xj, a.P + ((size_t)ch.y * R + r) * msz, nullptr, c0, nvalid,
                             smat, svec, g, s, uj, dummy);
    const T wr = a.cat_wt[r];
#pragma unroll
    for (int jj = 0; jj < CPG; ++jj) {
      const int j = g * CPG + jj;
#pragma unroll
      for (int i = 0; i < SPT; ++i) {
        const T p = ui[i][jj] * uj[i][jj];
        mx[jj] = tmax(mx[jj], fabs(p));
        if (k == a.root) lsum[jj] = fma(wr * pis[i], p, lsum[jj]);
        else if (j < nvalid)
          a.post[(((size_t)(k - a.n_tips) * C + c0 + j) * R + r) * SP + s + i * TPG] = p;
      }
    }
  }
  big_group_reduce<T, SP, true>(mx, red, g, s);
  if (k == a.root) big_group_reduce<T, SP, false>(lsum, red, g, s);
  double lterm = 0.0;
#pragma unroll
  for (int jj = 0; jj < CPG; ++jj) {
    const int j = g * CPG + jj, c = c0 + j;
    if (j >= nvalid) continue;
    int e = 0;
    if (!(mx[jj] > T(0)) || !isfinite(mx[jj])) {
      if (s == 0) atomicOr(a.err, ERR_ZERO_PARTIAL);
    } else {
      (void)frexp(mx[jj], &e);
    }
    const T f = ldexp(T(1), -e);
    int ec = e;
    if (ch.x >= a.n_tips) ec += a.escale[(size_t)(ch.x - a.n_tips) * a.escale_stride + c];
    if (ch.y >= a.n_tips) ec += a.escale[(size_t)(ch.y - a.n_tips) * a.escale_stride + c];
    if (k != a.root) {
      T* out = a.post + (((size_t)(k - a.n_tips) * C + c) * R) * SP + s;
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int i = 0; i < SPT; ++i) out[(size_t)r * SP + i * TPG] *= f;
      if (s == 0) a.escale[(size_t)(k - a.n_tips) * a.escale_stride + c] = ec;
    } else if (s == 0) {
      // Eq. 3: L_c = sum_r w_r pi' p_root,r (scaled by f), exponents restored
      const double L = (double)(lsum[jj] * f);
      if (!(L > 0.0) || !isfinite(L)) atomicOr(a.err, ERR_ZERO_PARTIAL);
      lterm += a.pattern_w[c] * (log(L) + (double)ec * 0.69314718055994530942);
    }
  }
  if (k == a.root) {
    if (s == 0) lred[g] = lterm;
    __syncthreads();
    if (threadIdx.x == 0) {
      double l = 0.0;
      for (int i = 0; i < PL::G; ++i) l += lred[i];
      a.lpart[blockIdx.x] = l;
    }
  }
}

template <typename T, int SP>
__global__ void __launch_bounds__(kBigThreads, kBigMinBlocks<SP>) pre_big_kernel(LevelArgs<T> a) {
  pdl_wait_and_release();
  using PL = BigPlan<T, SP>;
  constexpr int CT = PL::CT, CPG = PL::CPG, SPT = PL::SPT, TPG = PL::TPG;
  using A = Acc<T>;
  extern __shared__ __align__(16) unsigned char smraw[];
  T* smat = reinterpret_cast<T*>(smraw);
  T* svec = smat + PL::mat;
  T* U = svec + PL::vec;            // [CT][SP]: u_i, then a_i
  T* W = U + (size_t)CT * SP;       // [CT][SP]: w_i, then a_j
  T* red = W + (size_t)CT * SP;
  __shared__ typename A::type gred[PL::G][2];
  const int k = a.level_nodes[blockIdx.y];
  const int2 ch = a.children[k];
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int c0 = blockIdx.x * CT, nvalid = min(CT, C - c0);
  const int s = threadIdx.x % TPG, g = threadIdx.x / TPG;
  const size_t msz = (size_t)SP * SP;
  const bool int_i = ch.x >= a.n_tips, int_j = ch.y >= a.n_tips;
  T ni[CPG], nj[CPG], dd[CPG], mi[CPG], mj[CPG];
#pragma unroll
  for (int jj = 0; jj < CPG; ++jj) { ni[jj] = nj[jj] = dd[jj] = mi[jj] = mj[jj] = T(0); }
  for (int r = 0; r < R; ++r) {
    const size_t mi_off = ((size_t)ch.x * R + r) * msz, mj_off = ((size_t)ch.y * R + r) * msz;
    T u[SPT][CPG], w[SPT][CPG];
    const BigChild<T> xi = big_child(a, ch.x, c0, r, SP), xj = big_child(a, ch.y, c0, r, SP);
    big_row_mv<T, SP, true>(a, xi, a.P + mi_off, a.dP + mi_off, c0, nvalid, smat, svec, g, s, u, w);
#pragma unroll
    for (int jj = 0; jj < CPG; ++jj)
#pragma unroll
      for (int i = 0; i < SPT; ++i) {
        U[(size_t)(g * CPG + jj) * SP + s + i * TPG] = u[i][jj];
        W[(size_t)(g * CPG + jj) * SP + s + i * TPG] = w[i][jj];
      }
    big_row_mv<T, SP, true>(a, xj, a.P + mj_off, a.dP + mj_off, c0, nvalid, smat, svec, g, s, u, w);
    const T wr = a.cat_wt[r];
#pragma unroll
    for (int jj = 0; jj < CPG; ++jj) {
      const int j = g * CPG + jj;
#pragma unroll
      for (int i = 0; i < SPT; ++i) {
        const int si = s + i * TPG;
        T q = T(0);
        if (k == a.root) q = si < S ? (T)a.root_pi[si] : T(0);
        else if (j < nvalid) q = a.pre[(((size_t)(k - a.n_tips) * C + c0 + j) * R + r) * SP + si];
        const size_t o = (size_t)j * SP + si;
        const T ui = U[o], wi = W[o];
        const T ai = q * u[i][jj], aj = q * ui;  // a_i = q o P_j p_j, a_j = q o P_i p_i
        ni[jj] = fma(wr, ai * wi, ni[jj]);
        nj[jj] = fma(wr, aj * w[i][jj], nj[jj]);
        dd[jj] = fma(wr, ai * ui, dd[jj]);
        U[o] = ai;
        W[o] = aj;
      }
    }
    // Eq. 4 for internal children: q_x = P_x' a_x (unscaled for now)
    for (int x = 0; x < 2; ++x) {
      if (!(x == 0 ? int_i : int_j)) continue;
      T q[SPT][CPG];
      big_col_mv<T, SP>(a.P + (x == 0 ? mi_off : mj_off), x == 0 ? U : W, smat, g, s, q);
      const int b = x == 0 ? ch.x : ch.y;
#pragma unroll
      for (int jj = 0; jj < CPG; ++jj) {
        const int j = g * CPG + jj;
#pragma unroll
        for (int i = 0; i < SPT; ++i) {
          if (x == 0) mi[jj] = tmax(mi[jj], fabs(q[i][jj]));
          else mj[jj] = tmax(mj[jj], fabs(q[i][jj]));
          if (j < nvalid)
            a.pre[(((size_t)(b - a.n_tips) * C + c0 + j) * R + r) * SP + s + i * TPG] = q[i][jj];
        }
      }
    }
    __syncthreads();  // U and W are rewritten by the next category
  }
  big_group_reduce<T, SP, false>(ni, red, g, s);
  big_group_reduce<T, SP, false>(nj, red, g, s);
  big_group_reduce<T, SP, false>(dd, red, g, s);
  if (int_i) big_group_reduce<T, SP, true>(mi, red, g, s);
  if (int_j) big_group_reduce<T, SP, true>(mj, red, g, s);
  typename A::type gi = A::zero(), gj = A::zero();
#pragma unroll
  for (int jj = 0; jj < CPG; ++jj) {
    const int j = g * CPG + jj, c = c0 + j;
    if (j >= nvalid) continue;
    if (s == 0) {
      if (!(dd[jj] > T(0)) || !isfinite(dd[jj])) {
        atomicOr(a.err, ERR_BAD_RATIO);
      } else {
        gi = A::add(gi, A::prod(a.pattern_wt[c], ni[jj] / dd[jj]));
        gj = A::add(gj, A::prod(a.pattern_wt[c], nj[jj] / dd[jj]));
      }
    }
    for (int x = 0; x < 2; ++x) {
      if (!(x == 0 ? int_i : int_j)) continue;
      const T m = x == 0 ? mi[jj] : mj[jj];
      int e = 0;
      if (!(m > T(0)) || !isfinite(m)) {
        if (s == 0) atomicOr(a.err, ERR_ZERO_PARTIAL);
      } else {
        (void)frexp(m, &e);
      }
      const T f = ldexp(T(1), -e);
      const int b = x == 0 ? ch.x : ch.y;
      T* out = a.pre + (((size_t)(b - a.n_tips) * C + c) * R) * SP + s;
      for (int r = 0; r < R; ++r)
#pragma unroll
        for (int i = 0; i < SPT; ++i) out[(size_t)r * SP + i * TPG] *= f;
    }
  }
  if (s == 0) { gred[g][0] = gi; gred[g][1] = gj; }
  __syncthreads();
  if (threadIdx.x == 0) {
    gi = gred[0][0];
    gj = gred[0][1];
    for (int i = 1; i < PL::G; ++i) {
      gi = A::add(gi, gred[i][0]);
      gj = A::add(gj, gred[i][1]);
    }
    a.gpart[(size_t)ch.x * a.n_tiles + blockIdx.x] = A::to_double(gi);
    a.gpart[(size_t)ch.y * a.n_tiles + blockIdx.x] = A::to_double(gj);
  }
}

template <typename T, int SP>
cudaError_t launch_big(const LevelArgs<T>& a, bool post, cudaStream_t st) {
  dim3 grid(a.n_tiles, a.n_level);
  using PL = BigPlan<T, SP>;
  if (post) return launch_pdl(post_big_kernel<T, SP>, grid, kBigThreads, PL::bytes(false), st, a);
  return launch_pdl(pre_big_kernel<T, SP>, grid, kBigThreads, PL::bytes(true), st, a);
}

template <typename T, int SP>
cudaError_t prepare_big() {
  using PL = BigPlan<T, SP>;
  cudaError_t e = cudaFuncSetAttribute(post_big_kernel<T, SP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)PL::bytes(false));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(pre_big_kernel<T, SP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)PL::bytes(true));
}

}  // namespace phylo

namespace phylo {

// ---------------------------------------------------------------------------
// Transition matrices for S_pad 128 and 256 on the FP32 path (Eq. 1):
// P - I = V diag(e^{lambda gamma t} - 1) Vinv and dP = V diag(gamma lambda
// e^{lambda gamma t}) Vinv in the double-float arithmetic of the 64-state
// build (kernels_tc64.cuh: Dekker products, Knuth sums, ~48 bits), so that
// the small entries of short branches keep FP32 accuracy through the
// cancellation in the sum over eigenvalues.  A CTA computes one 64 x 64
// tile of P and dP of one (branch, category), streaming the double-float
// eigenvector tables through shared memory kPmatBigChunk eigenvalues at a
// time; each thread owns a 4 x 4 block.  With S_pad 128 (the tensor-core
// path, whose pre-order step needs no dP) only P is built, written as the
// split P and P' operand blocks.  For the symmetric decomposition
// of a reversible model (Vinv[m][t] = pi_t V[t][m]) P - I = K diag(pi) with
// K = V diag(e) V' symmetric: only the tiles on and above the diagonal are
// contracted, and an off-diagonal tile also writes its mirror.
// ---------------------------------------------------------------------------
constexpr int kPmatBigChunk = 32;

template <int SP>
__global__ void __launch_bounds__(256) pmat_big_df_kernel(PmatArgs a) {
  constexpr int T = SP / 64;
  constexpr bool kD = SP != 128;  // dP wanted (the S_pad 256 CUDA-core path)
  __shared__ __align__(16) float sv_h[kPmatBigChunk][64], sv_l[kPmatBigChunk][64];
  __shared__ __align__(16) float sw_h[kPmatBigChunk][64], sw_l[kPmatBigChunk][64];
  __shared__ DF se[SP], sd[SP];
  const int S = a.n_states, R = a.n_cat, tid = threadIdx.x;
  const bool rev = a.reversible != 0;
  const int nt = rev ? T * (T + 1) / 2 : T * T;
  const int unit = blockIdx.x / nt, tile = blockIdx.x % nt;
  int sb, tb;
  if (rev) {  // tile -> (sb, tb), sb <= tb, row by row
    sb = 0;
    int rem = tile;
    while (rem >= T - sb) {
      rem -= T - sb;
      ++sb;
    }
    tb = sb + rem;
  } else {
    sb = tile / T;
    tb = tile % T;
  }
  const int b = unit / R, r = unit % R;
  for (int i = tid; i < SP; i += 256) {
    double e = 0.0, de = 0.0;
    if (i < S) {
      double t = a.t[b];
      if (!(t >= 0.0) || !isfinite(t)) {
        if (i == 0 && r == 0 && tile == 0) atomicOr(a.err, ERR_BAD_LENGTH);
        t = 0.0;
      }
      const double g = a.rates[r];
      const double x = a.lambda[i] * g * t;
      e = expm1(x);
      de = g * a.lambda[i] * exp(x);
    }
    se[i] = df_from(e);
    sd[i] = df_from(de);
  }
  const size_t sq = (size_t)SP * SP;
  const float* vt_h = a.vsplit;           // V' : [m][s]
  const float* vt_l = a.vsplit + sq;
  const float* w_h = rev ? vt_h : a.vsplit + 2 * sq;  // Vinv [m][t], or V' again
  const float* w_l = rev ? vt_l : a.vsplit + 3 * sq;
  const int ls = 4 * (tid / 16), lt = 4 * (tid % 16);  // the thread's block in the tile
  DF accP[4][4], accD[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) accP[i][j] = accD[i][j] = DF{0.f, 0.f};
  for (int m0 = 0; m0 < S; m0 += kPmatBigChunk) {
    __syncthreads();  // exponentials staged / previous chunk read
    for (int i = tid; i < kPmatBigChunk * 16; i += 256) {
      const int row = i / 16, c4 = 4 * (i % 16);
      const size_t gs = (size_t)(m0 + row) * SP + 64 * sb + c4;
      const size_t gt = (size_t)(m0 + row) * SP + 64 * tb + c4;
      *reinterpret_cast<float4*>(&sv_h[row][c4]) = *reinterpret_cast<const float4*>(vt_h + gs);
      *reinterpret_cast<float4*>(&sv_l[row][c4]) = *reinterpret_cast<const float4*>(vt_l + gs);
      *reinterpret_cast<float4*>(&sw_h[row][c4]) = *reinterpret_cast<const float4*>(w_h + gt);
      *reinterpret_cast<float4*>(&sw_l[row][c4]) = *reinterpret_cast<const float4*>(w_l + gt);
    }
    __syncthreads();
    const int mend = min(kPmatBigChunk, S - m0);
    for (int mm = 0; mm < mend; ++mm) {
      const float4 vh = *reinterpret_cast<const float4*>(&sv_h[mm][ls]);
      const float4 vl = *reinterpret_cast<const float4*>(&sv_l[mm][ls]);
      const float4 wh = *reinterpret_cast<const float4*>(&sw_h[mm][lt]);
      const float4 wl = *reinterpret_cast<const float4*>(&sw_l[mm][lt]);
      const DF em = se[m0 + mm], dm = sd[m0 + mm];
      const DF v[4] = {{vh.x, vl.x}, {vh.y, vl.y}, {vh.z, vl.z}, {vh.w, vl.w}};
      const DF w[4] = {{wh.x, wl.x}, {wh.y, wl.y}, {wh.z, wl.z}, {wh.w, wl.w}};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const DF ve = df_mul(v[i], em);
#pragma unroll
        for (int j = 0; j < 4; ++j) df_fma(accP[i][j], ve, w[j]);
        if constexpr (kD) {
          const DF vd = df_mul(v[i], dm);
#pragma unroll
          for (int j = 0; j < 4; ++j) df_fma(accD[i][j], vd, w[j]);
        }
      }
    }
  }
  const int s0 = 64 * sb + ls, t0 = 64 * tb + lt;
  const float* pi_h = a.vsplit + 4 * sq;
  const float* pi_l = pi_h + SP;
  if constexpr (SP == 128) {
    // the tensor-core path's operand blocks instead of P: entry (s, t) goes
    // to row s % 64, column t % 64 of block P (sb, tb), and to row t % 64,
    // column s % 64 of block P' (tb, sb); the mirror entries (t, s) of a
    // reversible model to the transposed places
    unsigned char* U = static_cast<unsigned char*>(a.tiles) + (size_t)unit * kTcbUnitBytes;
    float p[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int s = s0 + i, t = t0 + j;
        DF kp = accP[i][j];
        if (rev) kp = df_mul(kp, DF{pi_h[t], pi_l[t]});
        p[i][j] = df_round(kp, s == t && s < S);
      }
#pragma unroll
    for (int i = 0; i < 4; ++i)
      put_split3_4(U + tcb_block(0, sb, tb), kTerm64, ls + i, lt,
                   make_float4(p[i][0], p[i][1], p[i][2], p[i][3]));
#pragma unroll
    for (int j = 0; j < 4; ++j)
      put_split3_4(U + tcb_block(1, tb, sb), kTerm64, lt + j, ls,
                   make_float4(p[0][j], p[1][j], p[2][j], p[3][j]));
    if (rev && sb != tb) {  // mirror: P[t][s] = delta + K_st pi_s
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
          p[i][j] = df_round(df_mul(accP[i][j], DF{pi_h[s0 + i], pi_l[s0 + i]}), false);
#pragma unroll
      for (int j = 0; j < 4; ++j)
        put_split3_4(U + tcb_block(0, tb, sb), kTerm64, lt + j, ls,
                     make_float4(p[0][j], p[1][j], p[2][j], p[3][j]));
#pragma unroll
      for (int i = 0; i < 4; ++i)
        put_split3_4(U + tcb_block(1, sb, tb), kTerm64, ls + i, lt,
                     make_float4(p[i][0], p[i][1], p[i][2], p[i][3]));
    }
    return;
  }
  float* P = static_cast<float*>(a.P) + (size_t)unit * sq;
  float* D = static_cast<float*>(a.dP) + (size_t)unit * sq;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int s = s0 + i;
    float p[4], d[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int t = t0 + j;
      DF kp = accP[i][j], kd = accD[i][j];
      if (rev) {
        const DF pt = {pi_h[t], pi_l[t]};
        kp = df_mul(kp, pt);
        kd = df_mul(kd, pt);
      }
      p[j] = df_round(kp, s == t && s < S);
      d[j] = df_round(kd, false);
    }
    *reinterpret_cast<float4*>(P + (size_t)s * SP + t0) = make_float4(p[0], p[1], p[2], p[3]);
    *reinterpret_cast<float4*>(D + (size_t)s * SP + t0) = make_float4(d[0], d[1], d[2], d[3]);
  }
  if (rev && sb != tb) {  // mirror tile: P[t][s] = delta + K_st pi_s
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int t = t0 + j;
      float p[4], d[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int s = s0 + i;
        const DF ps = {pi_h[s], pi_l[s]};
        p[i] = df_round(df_mul(accP[i][j], ps), false);
        d[i] = df_round(df_mul(accD[i][j], ps), false);
      }
      *reinterpret_cast<float4*>(P + (size_t)t * SP + s0) = make_float4(p[0], p[1], p[2], p[3]);
      *reinterpret_cast<float4*>(D + (size_t)t * SP + s0) = make_float4(d[0], d[1], d[2], d[3]);
    }
  }
}

template <int SP>
cudaError_t launch_pmat_big(const PmatArgs& a, cudaStream_t st) {
  constexpr int T = SP / 64;
  const int nt = a.reversible ? T * (T + 1) / 2 : T * T;
  const long long blocks = (long long)a.n_branches * a.n_cat * nt;
  if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
  pmat_big_df_kernel<SP><<<(unsigned)blocks, 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace phylo

namespace phylo {

// ---------------------------------------------------------------------------
// Transition matrices for 4 and 20 padded states on the FP32 path (Eq. 1),
// in the same double-float arithmetic, written in the transposed layout
// those kernels read ([P' | dP' | P] per branch).  A block takes UPB
// (branch, category) units; each thread owns entries (s, t) of a unit.
// ---------------------------------------------------------------------------
template <int SP>
__global__ void __launch_bounds__(256) pmat_df_small_kernel(PmatArgs a) {
  constexpr int SQ = SP * SP;
  constexpr int UPB = (256 / SQ) > 0 ? 256 / SQ : 1;
  __shared__ float vt_h[SQ], vt_l[SQ], vi_h[SQ], vi_l[SQ];  // V' [m][s], Vinv [m][t]
  __shared__ DF se[UPB][SP], sd[UPB][SP];
  const int S = a.n_states, R = a.n_cat, n_units = a.n_branches * R;
  const int unit0 = blockIdx.x * UPB;
  for (int i = threadIdx.x; i < SQ; i += blockDim.x) {
    vt_h[i] = a.vsplit[i];
    vt_l[i] = a.vsplit[SQ + i];
    vi_h[i] = a.vsplit[2 * SQ + i];
    vi_l[i] = a.vsplit[3 * SQ + i];
  }
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
      e = expm1(x);
      de = g * a.lambda[m] * exp(x);
    }
    se[u][m] = df_from(e);
    sd[u][m] = df_from(de);
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < UPB * SQ; idx += blockDim.x) {
    const int u = idx / SQ, e = idx % SQ, unit = unit0 + u;
    if (unit >= n_units) continue;
    const int s = e / SP, t = e % SP;
    DF ap = {0.f, 0.f}, ad = {0.f, 0.f};
    if (s < S && t < S) {
      for (int m = 0; m < S; ++m) {
        const DF v = {vt_h[m * SP + s], vt_l[m * SP + s]};
        const DF w = {vi_h[m * SP + t], vi_l[m * SP + t]};
        df_fma(ap, df_mul(v, se[u][m]), w);
        df_fma(ad, df_mul(v, sd[u][m]), w);
      }
    }
    const float p = df_round(ap, s == t && s < S), dp = df_round(ad, false);
    const int b = unit / R, r = unit % R;
    float* base = static_cast<float*>(a.P) + (size_t)b * kP4MatKinds * R * SQ;
    base[(size_t)r * SQ + t * SP + s] = p;
    base[(size_t)(R + r) * SQ + t * SP + s] = dp;
    base[(size_t)(2 * R + r) * SQ + e] = p;
  }
}

template <int SP>
cudaError_t launch_pmat_df_small(const PmatArgs& a, cudaStream_t st) {
  constexpr int UPB = (256 / (SP * SP)) > 0 ? 256 / (SP * SP) : 1;
  const long long units = (long long)a.n_branches * a.n_cat;
  pmat_df_small_kernel<SP><<<(unsigned)((units + UPB - 1) / UPB), 256, 0, st>>>(a);
  return cudaGetLastError();
}

}  // namespace phylo
