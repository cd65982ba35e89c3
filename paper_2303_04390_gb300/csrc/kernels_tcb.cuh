// FP32 kernels for 65..128 states (S_pad = 128: the paper's 122-state
// Markov-modulated codon model) on the tensor cores, K- and N-tiled.
//
// Arithmetic as on the 64-state tensor-core path (kernels_tc64.cuh), per
// (node, tile of 128 patterns, category r):
//   post:    U_x = p_x P_x'                       (both children)
//            p_k = U_i o U_j, rescaled
//   pre (A): [U_x | V_x] = p_x [P_x ; dP_x]'      (both children)
//            a_i = q_k o U_j,  a_j = q_k o U_i
//            num_x = a_x . V_x,  den = a_i . U_i   -> per-category Eq. 8 terms
//            a_x written into the q slot of each internal child
//   pre (B): q_x = a_x P_x, rescaled in place     (internal children)
// With 128 padded states every operand is cut into 64 x 64 blocks: a
// contraction D[128 x 128] = A[128 x 128] B[128 x 128]' is, for each of the
// two 64-column blocks of D, two MMA groups of K = 64 accumulated in TMEM.
// Each group is the BF16 x3 split of tc.cuh (six products per FP32
// product), so results carry FP32 accuracy.  Partial tiles are split into
// their three BF16 terms in shared memory (the A operand, one 64-column
// K-block at a time); the matrix kernel writes the matrix blocks pre-split
// (tcb_block) and they are bulk-copied (cp.async.bulk).  A and B buffers
// are double-buffered, so one round's loads and splits overlap the previous
// round's MMAs.  A compact tip child enters the MMA as its one-hot (or, for
// a gap, all-ones) rows, so every child takes the same path.
//
// TMEM: post 256 columns [U_i | U_j]; pre (A) 512 [U_i | V_i | U_j | V_j];
// pre (B) 128 [q_x].  One CTA per SM (192 KB of shared memory).
//
// Rescaling, exponents and the Eq. 8 terms follow the 64-state path
// (per-category exponents; ratio_tc_kernel combines the categories); the
// root's post-order CTAs store p_root and root_tcb_kernel forms log L_c.
// Every wait is bounded; on expiry the kernel raises ERR_TIMEOUT, drains
// (bounded) the copies and MMAs it issued, frees its TMEM and returns.
#pragma once

namespace phylo {

constexpr int kTcbSP = 128;                  // padded states of this path
constexpr int kTcbNB = kTcbSP / 64;          // 64-blocks per dimension
constexpr uint32_t kTcbBlock = 3 * kTerm64;  // one 64 x 64 three-term block
static_assert(kTcbUnitBytes == 3 * kTcbNB * kTcbNB * kTcbBlock, "tile block size");
// Shared memory: A ring 2 x 48 KB, B ring 2 x 48 KB (+1024 for alignment).
constexpr size_t kTcbSmem = 1024 + 2 * (size_t)kOp128 + 4 * (size_t)kTcbBlock;
constexpr int kTcbLd = kTcbSP + 4;           // output staging row stride (floats)
static_assert((size_t)kTcRows * kTcbLd * 4 <= 2 * (size_t)kOp128, "staging fits in A");
static_assert(2 * (size_t)kTcRows * kTcbLd * 4 <= 2 * (size_t)kOp128 + 4 * (size_t)kTcbBlock,
              "two staging buffers fit in A and B");

// First row (pattern 0, category r) of a non-compact child's partials on
// this path and the row stride, in floats.
__device__ __forceinline__ const float* tcb_child_base(const LevelArgs<float>& a,
                                                       const TcChild& x, int r, size_t* stride) {
  const int C = a.n_patterns;
  if (x.internal) {
    *stride = (size_t)a.n_cat * kTcbSP;
    return a.post + ((size_t)(x.b - a.n_tips) * C * a.n_cat + r) * kTcbSP;
  }
  *stride = kTcbSP;
  return a.tip_partials + (size_t)x.b * C * kTcbSP;
}

__device__ __forceinline__ const unsigned char* tcb_unit(const LevelArgs<float>& a, int b,
                                                         int r) {
  return a.tc_tiles + ((size_t)b * a.n_cat + r) * kTcbUnitBytes;
}

// The loads of one A fill (K-block kb, states 64 kb .. 64 kb + 63, of a
// child's rows), issued a round ahead of their use: the partial rows, or for
// a compact tip its states (the fill then writes one-hot rows, all ones up
// to S for a gap, zero rows past the last pattern).
struct TcbFill {
  float4 v[8];
  int y[4];
};

__device__ __forceinline__ void tcb_load_fill(TcbFill& f, const LevelArgs<float>& a,
                                              const TcChild& x, const float* src, size_t stride,
                                              int kb, int c0) {
  const int C = a.n_patterns;
  if (!x.compact) {
    coop_load(f.v, src + 64 * kb, stride, c0, C);
    return;
  }
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int c = c0 + coop_row(it);
    f.y[it] = c < C ? (int)a.tip_states[(size_t)x.b * a.state_stride + c] : -1;
  }
}

__device__ __forceinline__ void tcb_put_fill(unsigned char* A, const TcbFill& f,
                                             const TcChild& x, int kb, int S) {
  if (!x.compact) {
    coop_put(A, f.v);
    return;
  }
  const int j = threadIdx.x & 7;
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int y = f.y[it];
    float v8[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int kk = 64 * kb + 8 * j + i;
      v8[i] = y < 0 ? 0.f : y < S ? (kk == y ? 1.f : 0.f) : (kk < S ? 1.f : 0.f);
    }
    tc::put_split3(A, A + kTerm128, A + 2 * kTerm128, coop_row(it), j, v8);
  }
}

// D (+)= A B' for the two 64-column blocks jn of one K-block (the MMAs of
// one round): B holds the two blocks (jn = 0, 1) back to back.
__device__ __forceinline__ void tcb_mma_round(uint32_t d_tmem, const unsigned char* A,
                                              const unsigned char* B, bool accumulate) {
  uint32_t ta[3];
  term_addrs(A, kTerm128, ta);
#pragma unroll
  for (int jn = 0; jn < kTcbNB; ++jn) {
    uint32_t tb[3];
    term_addrs(B + jn * kTcbBlock, kTerm64, tb);
    tc::mma_split_bf16x3_acc<64>(d_tmem + 64 * jn, ta, tb, accumulate);
  }
}

// Coalesced store of staged 128-float rows (a quarter warp writes one
// 128-byte quarter row per instruction).
__device__ __forceinline__ void tcb_store_rows(float* __restrict__ base, size_t stride, int c0,
                                               int C, const float* st) {
  const int jj = threadIdx.x & 7;
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int row = coop_row(it), c = c0 + row;
    if (c < C) {
      float* dst = base + (size_t)c * stride;
#pragma unroll
      for (int q = 0; q < 4; ++q)
        *reinterpret_cast<float4*>(dst + 32 * q + 4 * jj) =
            *reinterpret_cast<const float4*>(st + row * kTcbLd + 32 * q + 4 * jj);
    }
  }
}

// Bookkeeping of the asynchronous phases a CTA has issued and waited on,
// so that a timeout can drain what is still in flight.  Barriers: 0, 1 =
// bulk copies into B buffer 0, 1; 2, 3 = MMA commits of rounds using B
// buffer 0, 1.  Scalars (not arrays), so that they stay in registers.
struct TcbPhases {
  uint32_t i0 = 0, i1 = 0, i2 = 0, i3 = 0;  // issued
  uint32_t w0 = 0, w1 = 0, w2 = 0, w3 = 0;  // waited
  __device__ uint32_t waited(int k) const { return k == 0 ? w0 : k == 1 ? w1 : k == 2 ? w2 : w3; }
  __device__ void wait_done(int k) {
    w0 += k == 0; w1 += k == 1; w2 += k == 2; w3 += k == 3;
  }
  __device__ void issue(int k) {
    i0 += k == 0; i1 += k == 1; i2 += k == 2; i3 += k == 3;
  }
};

__device__ __forceinline__ bool tcb_wait(uint64_t* bars, TcbPhases& ph, int k, int* err) {
  const bool mine = mbar_wait(&bars[k], ph.waited(k) & 1);
  const bool ok = __syncthreads_and(mine);
  if (ok) ph.wait_done(k);
  else if (threadIdx.x == 0) atomicOr(err, ERR_TIMEOUT);
  tc::fence_after();
  return ok;
}

__device__ __forceinline__ void tcb_drain(uint64_t* bars, const TcbPhases& ph) {
  if (threadIdx.x != 0) return;
  const uint32_t iss[4] = {ph.i0, ph.i1, ph.i2, ph.i3};
  const uint32_t wai[4] = {ph.w0, ph.w1, ph.w2, ph.w3};
#pragma unroll
  for (int k = 0; k < 4; ++k)
    for (uint32_t p = wai[k]; p < iss[k]; ++p) (void)mbar_wait(&bars[k], p & 1);
}

// Common prologue: barriers, TMEM, the block's row and half.
#define TCB_PROLOGUE(COLS)                                                   \
  extern __shared__ unsigned char smraw[];                                   \
  unsigned char* base = align1024(smraw);                                    \
  unsigned char* const A0 = base;                                           \
  unsigned char* const B0 = base + 2 * kOp128;                               \
  __shared__ uint64_t bars[4]; /* tma 0, tma 1, mma 0, mma 1 */              \
  __shared__ uint32_t tmem_slot;                                             \
  const int tid = threadIdx.x, warp = tid >> 5;                              \
  const int row = tid & (kTcRows - 1), h = tid / kTcRows;                    \
  if (warp == 0) tc::alloc(&tmem_slot, COLS);                                \
  if (tid == 0)                                                              \
    for (int i = 0; i < 4; ++i) mbar_init_fenced(&bars[i], 1);               \
  __syncthreads();                                                           \
  tc::fence_after();                                                         \
  const uint32_t tmem = tmem_slot;                                           \
  const uint32_t trow = tmem + ((uint32_t)((warp & 3) * 32) << 16);          \
  TcbPhases ph;

#define TCB_EPILOGUE(COLS)                                                   \
  tcb_drain(bars, ph);                                                       \
  tc::fence_before();                                                        \
  __syncthreads();                                                           \
  if (warp == 0) tc::dealloc(tmem, COLS);

// The rounds of a K- and N-tiled contraction.  Round i multiplies A buffer
// ab (a K-block of a child's rows, written by fill `fill` if >= 0) by the two
// matrix blocks at bsrc (blocks jn = 0, 1 of one kind and K-block, staged
// in B buffer i & 1) into d_tmem.  The rounds are pipelined: while round i's
// MMAs run, round i + 1's blocks are copied in and its A fill is written,
// and the loads of the fill after that are in flight.  Rounds and fills come
// from generator functions of their index (nothing indexed at run time lives
// in local memory); fills are written in index order.
struct TcbNext {
  TcChild x;
  const float* src;
  size_t stride;
  int kb;
};

struct TcbRound {
  const unsigned char* bsrc;
  int fill;  // the fill written before this round, or -1 (A buffer ab holds it)
  int ab;
  uint32_t d_tmem;
  bool accumulate;
};

// A buffers at A0 + ab kOp128, B buffers at B0 + b 2 kTcbBlock.
__device__ __forceinline__ unsigned char* tcb_a(unsigned char* A0, int ab) {
  return A0 + (size_t)ab * kOp128;
}
__device__ __forceinline__ unsigned char* tcb_b(unsigned char* B0, int b) {
  return B0 + (size_t)b * 2 * kTcbBlock;
}

__device__ __forceinline__ void tcb_issue_b(unsigned char* B0, uint64_t* bars, TcbPhases& ph,
                                            int i, const unsigned char* bsrc) {
  if (threadIdx.x == 0) {
    const int b = i & 1;
    mbar_expect_tx(&bars[b], 2 * kTcbBlock);
    ph.issue(b);
    bulk_g2s(tcb_b(B0, b), bsrc, 2 * kTcbBlock, &bars[b]);
  }
}

// Runs n rounds; false on a timeout (ERR_TIMEOUT raised).  On success every
// MMA has completed and the accumulators can be read.
template <class RoundOf, class FillOf>
__device__ __forceinline__ bool tcb_pipeline(unsigned char* A0, unsigned char* B0, uint64_t* bars,
                                             TcbPhases& ph, int n, int n_fills, RoundOf round_of,
                                             FillOf fill_of, const LevelArgs<float>& a, int c0) {
  const int S = a.n_states;
  TcbFill f;
  if (n_fills > 0) {
    const TcbNext q = fill_of(0);
    tcb_load_fill(f, a, q.x, q.src, q.stride, q.kb, c0);
  }
  TcbRound cur = round_of(0);
  tcb_issue_b(B0, bars, ph, 0, cur.bsrc);
  if (cur.fill >= 0) {
    tcb_put_fill(tcb_a(A0, cur.ab), f, fill_of(cur.fill).x, fill_of(cur.fill).kb, S);
    tc::fence_smem_for_async();
    if (cur.fill + 1 < n_fills) {
      const TcbNext q = fill_of(cur.fill + 1);
      tcb_load_fill(f, a, q.x, q.src, q.stride, q.kb, c0);
    }
  }
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    if (!tcb_wait(bars, ph, i & 1, a.err)) return false;  // round i's blocks (and A)
    if (threadIdx.x == 0) {
      tcb_mma_round(cur.d_tmem, tcb_a(A0, cur.ab), tcb_b(B0, i & 1), cur.accumulate);
      tc::commit(&bars[2 + (i & 1)]);
      ph.issue(2 + (i & 1));
    }
    if (i + 1 < n) {
      // round i - 1 done: its B buffer, and the A buffer the next fill
      // writes, are free
      if (i >= 1 && !tcb_wait(bars, ph, 2 + ((i - 1) & 1), a.err)) return false;
      cur = round_of(i + 1);
      tcb_issue_b(B0, bars, ph, i + 1, cur.bsrc);
      if (cur.fill >= 0) {
        const TcbNext q = fill_of(cur.fill);
        tcb_put_fill(tcb_a(A0, cur.ab), f, q.x, q.kb, S);
        tc::fence_smem_for_async();
        if (cur.fill + 1 < n_fills) {
          const TcbNext q2 = fill_of(cur.fill + 1);
          tcb_load_fill(f, a, q2.x, q2.src, q2.stride, q2.kb, c0);
        }
      }
    }
  }
  for (int i = n >= 2 ? n - 2 : 0; i < n; ++i)
    if (!tcb_wait(bars, ph, 2 + (i & 1), a.err)) return false;
  return true;
}

// ---------------------------------------------------------------------------
// Post-order level (Eq. 2); the root's p is stored like any other and
// root_tcb_kernel forms Eq. 3.
// ---------------------------------------------------------------------------
template <typename T>  // float only
__global__ void __launch_bounds__(kTcThreads) post_tcb_kernel(LevelArgs<T> a) {
  pdl_wait_and_release();  // before TMEM, smem or any global access
  TCB_PROLOGUE(256)
  __shared__ float xch[2][kTcRows];
  const int R = a.n_cat, C = a.n_patterns;
  const int4 d = a.level_desc[blockIdx.y];
  const int k = d.x;
  const TcChild xs[2] = {tc_child(a.n_tips, d.y, d.w & kDescFlagCompact0),
                         tc_child(a.n_tips, d.z, d.w & kDescFlagCompact1)};
  const int c0 = blockIdx.x * kTcRows, c = c0 + row;
  const bool valid = c < C;
  const int r = blockIdx.z, estr = a.escale_stride;
  int E = 0;
  if (valid)
    for (int x = 0; x < 2; ++x)
      if (xs[x].internal) E += a.escale[((size_t)(xs[x].b - a.n_tips) * R + r) * estr + c];
  const int2 xb2 = make_int2(xs[0].b, xs[1].b);
  size_t st0 = 0, st1 = 0;
  const float* src0 = xs[0].compact ? nullptr : tcb_child_base(a, xs[0], r, &st0);
  const float* src1 = xs[1].compact ? nullptr : tcb_child_base(a, xs[1], r, &st1);
  // fill i = round i = (child x, K-block kb): U_x (+)= p_x[:, kb] P_x[:, kb]'
  const TcChild x0 = xs[0], x1 = xs[1];
  auto fill_of = [=](int i) {
    const int x = i / kTcbNB;
    return TcbNext{x ? x1 : x0, x ? src1 : src0, x ? st1 : st0, i % kTcbNB};
  };
  auto round_of = [=, &a](int i) {
    const int x = i / kTcbNB, kb = i % kTcbNB;
    return TcbRound{tcb_unit(a, x ? xb2.y : xb2.x, r) + tcb_block(0, 0, kb), i, i & 1,
                    tmem + 128u * x, kb > 0};
  };
  const bool ok = tcb_pipeline(A0, B0, bars, ph, 2 * kTcbNB, 2 * kTcbNB, round_of, fill_of, a, c0);
  if (ok) {
    // epilogue: p = U_i o U_j on this half row, the row max, scale, store
    float p[64];
    float m = 0.f;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float ui[32], uj[32];
      tc::ld32(trow + 0 + 64 * h + 32 * q, ui);
      tc::ld32(trow + 128 + 64 * h + 32 * q, uj);
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        p[32 * q + i] = ui[i] * uj[i];
        m = fmaxf(m, fabsf(p[32 * q + i]));
      }
    }
    xch[h][row] = m;
    __syncthreads();
    m = fmaxf(m, xch[1 - h][row]);
    // an all-zero vector is legitimate for one category; the root's
    // log-likelihood kernel flags a pattern whose categories all vanish
    int e = 0;
    if (valid) {
      if (!isfinite(m)) atomicOr(a.err, ERR_ZERO_PARTIAL);
      else if (m > 0.f) (void)frexpf(m, &e);
      e = max(e, -126);  // 2^-e stays finite for a subnormal maximum
    }
    const float f = ldexpf(1.f, -e);
    float* st = reinterpret_cast<float*>(base);  // A is free: every MMA is done
#pragma unroll
    for (int i = 0; i < 64; i += 4)
      *reinterpret_cast<float4*>(st + row * kTcbLd + 64 * h + i) =
          make_float4(p[i] * f, p[i + 1] * f, p[i + 2] * f, p[i + 3] * f);
    const size_t kslot = (size_t)(k - a.n_tips);
    if (valid && h == 0) a.escale[(kslot * R + r) * estr + c] = E + e;
    __syncthreads();
    tcb_store_rows(a.post + (kslot * C * R + r) * kTcbSP, (size_t)R * kTcbSP, c0, C, st);
  }
  TCB_EPILOGUE(256)
}

// ---------------------------------------------------------------------------
// Eq. 3 at the root: L_c = sum_r w_r 2^{E_r} pi' p_root,r,c, the sum over r
// taken relative to the largest exponent; W_c log L_c summed per tile.
// ---------------------------------------------------------------------------
template <typename T>  // float only
__global__ void __launch_bounds__(kTcRows) root_tcb_kernel(LevelArgs<T> a) {
  pdl_wait_and_release();
  __shared__ double lred[kTcRows / 32];
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int c = blockIdx.x * kTcRows + threadIdx.x;
  const size_t rslot = (size_t)(a.root - a.n_tips);
  double term = 0.0;
  if (c < C) {
    float lsum = 0.f;
    int lexp = INT_MIN / 2;
    for (int r = 0; r < R; ++r) {
      const float4* p = reinterpret_cast<const float4*>(
          a.post + ((rslot * C + c) * R + r) * kTcbSP);
      float pd = 0.f;
      for (int s4 = 0; s4 < (S + 3) / 4; ++s4) {
        const float4 v = p[s4];
        const int s = 4 * s4;
        pd = fmaf(a.root_pit[s], v.x, pd);
        if (s + 1 < S) pd = fmaf(a.root_pit[s + 1], v.y, pd);
        if (s + 2 < S) pd = fmaf(a.root_pit[s + 2], v.z, pd);
        if (s + 3 < S) pd = fmaf(a.root_pit[s + 3], v.w, pd);
      }
      if (pd == 0.f) continue;
      const int E = a.escale[(rslot * R + r) * a.escale_stride + c];
      const float t = a.cat_wt[r] * pd;
      if (E > lexp) {
        lsum = lsum * pow2i(lexp - E) + t;
        lexp = E;
      } else {
        lsum += t * pow2i(E - lexp);
      }
    }
    if (!(lsum > 0.f) || !isfinite(lsum)) atomicOr(a.err, ERR_ZERO_PARTIAL);
    else term = (double)a.pattern_wt[c] * (log((double)lsum) + (double)lexp * 0.69314718055994530942);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) term += __shfl_down_sync(kFull, term, o);
  if ((threadIdx.x & 31) == 0) lred[threadIdx.x >> 5] = term;
  __syncthreads();
  if (threadIdx.x == 0) {
    double l = 0.0;
    for (int w = 0; w < kTcRows / 32; ++w) l += lred[w];
    a.lpart[blockIdx.x] = l;
  }
}

// ---------------------------------------------------------------------------
// Pre-order level, part A: [U_x | V_x], the Eq. 8 terms, a_x
// ---------------------------------------------------------------------------
template <typename T>  // float only
__global__ void __launch_bounds__(kTcThreads) pre_tcb_a_kernel(LevelArgs<T> a) {
  pdl_wait_and_release();
  TCB_PROLOGUE(512)
  __shared__ float xch[2][3][kTcRows];
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int4 d = a.level_desc[blockIdx.y];
  const int k = d.x;
  const TcChild xs[2] = {tc_child(a.n_tips, d.y, d.w & kDescFlagCompact0),
                         tc_child(a.n_tips, d.z, d.w & kDescFlagCompact1)};
  const int c0 = blockIdx.x * kTcRows, c = c0 + row;
  const bool valid = c < C;
  const int r = blockIdx.z, estr = a.escale_stride;
  const bool root = k == a.root;
  const size_t kslot = (size_t)(k - a.n_tips);
  int eq_k = 0, ep[2] = {0, 0};
  bool gap[2] = {false, false};
  if (valid) {
    if (!root) eq_k = a.pre_escale[(kslot * R + r) * estr + c];
    for (int x = 0; x < 2; ++x) {
      if (xs[x].internal) ep[x] = a.escale[((size_t)(xs[x].b - a.n_tips) * R + r) * estr + c];
      if (xs[x].compact) gap[x] = (int)a.tip_states[(size_t)xs[x].b * a.state_stride + c] >= S;
    }
  }
  // the rows of q_k this thread's epilogue reads, loaded before the MMAs
  float qv[64];
  if (!root && valid) {
    const float4* q4 = reinterpret_cast<const float4*>(a.pre + ((kslot * C + c) * R + r) * kTcbSP +
                                                       64 * h);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float4 t4 = q4[i];
      qv[4 * i] = t4.x; qv[4 * i + 1] = t4.y; qv[4 * i + 2] = t4.z; qv[4 * i + 3] = t4.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < 64; ++i)
      qv[i] = root && 64 * h + i < S ? a.root_pit[64 * h + i] : 0.f;
  }
  const int2 xb2 = make_int2(xs[0].b, xs[1].b);
  size_t st0 = 0, st1 = 0;
  const float* src0 = xs[0].compact ? nullptr : tcb_child_base(a, xs[0], r, &st0);
  const float* src1 = xs[1].compact ? nullptr : tcb_child_base(a, xs[1], r, &st1);
  // fill (child x, K-block kb) serves rounds 2 fill and 2 fill + 1
  const TcChild x0 = xs[0], x1 = xs[1];
  auto fill_of = [=](int fi) {
    const int x = fi / kTcbNB;
    return TcbNext{x ? x1 : x0, x ? src1 : src0, x ? st1 : st0, fi % kTcbNB};
  };
  // rounds i = (child x, K-block kb, kind m in {P, dP}):
  // [U_x | V_x] (+)= p_x[:, kb] [P_x ; dP_x][:, kb]'
  auto round_of = [=, &a](int i) {
    const int x = i / (2 * kTcbNB), kb = (i / 2) % kTcbNB, m = i & 1, fi = i / 2;
    return TcbRound{tcb_unit(a, x ? xb2.y : xb2.x, r) + tcb_block(m, 0, kb), m == 0 ? fi : -1,
                    fi & 1, tmem + 256u * x + 128u * m, kb > 0};
  };
  const bool ok = tcb_pipeline(A0, B0, bars, ph, 4 * kTcbNB, 2 * kTcbNB, round_of, fill_of, a, c0);
  if (ok) {
    // epilogue: per 16 columns of this half row
    float ni = 0.f, nj = 0.f, dn = 0.f;
    // a_i and a_j staged for coalesced stores (A and B are free: every MMA
    // is done)
    float* st[2] = {reinterpret_cast<float*>(base),
                    reinterpret_cast<float*>(base) + kTcRows * kTcbLd};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int s0 = 64 * h + 16 * q;
      float ui[16], vi[16], uj[16], vj[16];
      tc::ld16(trow + 0 + s0, ui);
      tc::ld16(trow + 128 + s0, vi);
      tc::ld16(trow + 256 + s0, uj);
      tc::ld16(trow + 384 + s0, vj);
      float ai[16], aj[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        ai[i] = qv[16 * q + i] * uj[i];  // a_i = q o U_j
        aj[i] = qv[16 * q + i] * ui[i];  // a_j = q o U_i
        dn = fmaf(ai[i], ui[i], dn);
        // a gap's d/dt of the all-ones vector is 0
        if (!gap[0]) ni = fmaf(ai[i], vi[i], ni);
        if (!gap[1]) nj = fmaf(aj[i], vj[i], nj);
      }
#pragma unroll
      for (int i = 0; i < 16; i += 4) {
        *reinterpret_cast<float4*>(st[0] + row * kTcbLd + s0 + i) =
            make_float4(ai[i], ai[i + 1], ai[i + 2], ai[i + 3]);
        *reinterpret_cast<float4*>(st[1] + row * kTcbLd + s0 + i) =
            make_float4(aj[i], aj[i + 1], aj[i + 2], aj[i + 3]);
      }
    }
    xch[h][0][row] = ni;
    xch[h][1][row] = nj;
    xch[h][2][row] = dn;
    __syncthreads();
    if (valid && h == 0) {
      const float w = a.cat_wt[r];
      reinterpret_cast<float4*>(a.rterm)[(kslot * C + c) * R + r] =
          make_float4(w * (ni + xch[1][0][row]), w * (nj + xch[1][1][row]),
                      w * (dn + xch[1][2][row]), __int_as_float(eq_k + ep[0] + ep[1]));
      // q_x = P_x' (q_k o U_sibling): exponents of q_k and of the sibling;
      // part B adds the rescale of q_x
      for (int x = 0; x < 2; ++x)
        if (xs[x].internal)
          a.pre_escale[((size_t)(xs[x].b - a.n_tips) * R + r) * estr + c] = eq_k + ep[1 - x];
    }
    for (int x = 0; x < 2; ++x)  // (the barrier above also orders the staging)
      if (xs[x].internal)
        tcb_store_rows(a.pre + ((size_t)(xs[x].b - a.n_tips) * C * R + r) * kTcbSP,
                       (size_t)R * kTcbSP, c0, C, st[x]);
  }
  TCB_EPILOGUE(512)
}

// ---------------------------------------------------------------------------
// Pre-order level, part B: q_x = a_x P_x for the internal children, in
// place of a_x, rescaled.  blockIdx.y = 2 (level node) + child.
// ---------------------------------------------------------------------------
template <typename T>  // float only
__global__ void __launch_bounds__(kTcThreads) pre_tcb_b_kernel(LevelArgs<T> a) {
  pdl_wait_and_release();
  const int4 d = a.level_desc[blockIdx.y >> 1];
  const int xb = (blockIdx.y & 1) ? d.z : d.y;
  if (xb < a.n_tips) return;  // a tip child has no q (the whole block leaves)
  TCB_PROLOGUE(128)
  __shared__ float xch[2][kTcRows];
  const int R = a.n_cat, C = a.n_patterns;
  const TcChild x = tc_child(a.n_tips, xb, false);
  const int c0 = blockIdx.x * kTcRows, c = c0 + row;
  const bool valid = c < C;
  const int r = blockIdx.z, estr = a.escale_stride;
  const size_t xslot = (size_t)(xb - a.n_tips);
  const size_t stride = (size_t)R * kTcbSP;
  float* arow = a.pre + (xslot * C * R + r) * kTcbSP;  // a_x rows in, q_x rows out
  auto fill_of = [=](int kb) { return TcbNext{x, arow, stride, kb}; };
  auto round_of = [=, &a](int kb) {  // q_x (+)= a_x[:, kb] P'_x[:, kb]'
    return TcbRound{tcb_unit(a, xb, r) + tcb_block(2, 0, kb), kb, kb, tmem, kb > 0};
  };
  const bool ok = tcb_pipeline(A0, B0, bars, ph, kTcbNB, kTcbNB, round_of, fill_of, a, c0);
  if (ok) {
    float q[64];
    float m = 0.f;
    tc::ld32(trow + 64 * h, *reinterpret_cast<float(*)[32]>(q));
    tc::ld32(trow + 64 * h + 32, *reinterpret_cast<float(*)[32]>(q + 32));
#pragma unroll
    for (int i = 0; i < 64; ++i) m = fmaxf(m, fabsf(q[i]));
    xch[h][row] = m;
    __syncthreads();
    m = fmaxf(m, xch[1 - h][row]);
    int e = 0;
    if (valid) {
      if (!isfinite(m)) atomicOr(a.err, ERR_ZERO_PARTIAL);
      else if (m > 0.f) (void)frexpf(m, &e);
      e = max(e, -126);
    }
    const float f = ldexpf(1.f, -e);
    float* st = reinterpret_cast<float*>(base);  // A is free: every MMA is done
#pragma unroll
    for (int i = 0; i < 64; i += 4)
      *reinterpret_cast<float4*>(st + row * kTcbLd + 64 * h + i) =
          make_float4(q[i] * f, q[i + 1] * f, q[i + 2] * f, q[i + 3] * f);
    if (valid && h == 0) a.pre_escale[(xslot * R + r) * estr + c] += e;
    __syncthreads();
    tcb_store_rows(arow, stride, c0, C, st);
  }
  TCB_EPILOGUE(128)
}

#undef TCB_PROLOGUE
#undef TCB_EPILOGUE

inline cudaError_t launch_tcb(const LevelArgs<float>& a, bool post, cudaStream_t st) {
  if (post) {
    dim3 grid(a.n_tiles, a.n_level, a.n_cat);
    cudaError_t e = launch_pdl(post_tcb_kernel<float>, grid, kTcThreads, kTcbSmem, st, a);
    if (e == cudaSuccess && a.root_level)
      e = launch_pdl(root_tcb_kernel<float>, dim3(a.n_tiles), kTcRows, 0, st, a);
    return e;
  }
  dim3 ga(a.n_tiles, a.n_level, a.n_cat);
  cudaError_t e = launch_pdl(pre_tcb_a_kernel<float>, ga, kTcThreads, kTcbSmem, st, a);
  if (e != cudaSuccess) return e;
  dim3 gb(a.n_tiles, 2 * a.n_level, a.n_cat);
  return launch_pdl(pre_tcb_b_kernel<float>, gb, kTcThreads, kTcbSmem, st, a);
}

inline cudaError_t launch_pmat_tcb(const PmatArgs& a, cudaStream_t st) {
  return launch_pmat_big<kTcbSP>(a, st);  // (writes the operand blocks: a.tiles is set)
}

inline cudaError_t prepare_tcb() {
  cudaError_t e = cudaFuncSetAttribute(post_tcb_kernel<float>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kTcbSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pre_tcb_a_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTcbSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pre_tcb_b_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTcbSmem);
  return e;
}

}  // namespace phylo
