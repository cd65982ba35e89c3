// FP32 kernels for 65..128 states (S_pad = 128: the paper's 122-state
// Markov-modulated codon model) on the tensor cores, K- and N-tiled.
//
// Arithmetic as on the 64-state tensor-core path (kernels_tc64.cuh, the U
// form: the post-order pass stores U_x = P_x p_x of every node), per
// (node k, tile of 128 patterns, category r):
//   post:  p_k = U_i o U_j (rescaled),  U_k = p_k P_k'            (Eq. 2)
//   root:  L_c = sum_r w_r pi' (U_i o U_j)                          (Eq. 3)
//   pre, per child x with sibling y (Eq. 4 with the Eq. 8 terms):
//          a_x = q_k o U_y,  den = a_x . U_x,
//          [q_x | W_x] = a_x [P_x | Q],  num_x = gamma_r W_x . U_x
// With 128 padded states every operand is cut into 64 x 64 blocks: a
// contraction D[128 x 128] = A[128 x 128] B[128 x 128]' is, for each of the
// two 64-column blocks of D, two MMA groups of K = 64 accumulated in TMEM.
// Each group is the BF16 x3 split of tc.cuh (six products per FP32
// product), so results carry FP32 accuracy.  The A operand (p_k or a_x, both
// K-blocks) is formed in registers and split into its three BF16 terms in
// shared memory before the first MMA; the matrix blocks (P and P' written
// pre-split by the matrix kernel, tcb_block; Q' from the host) are
// bulk-copied (cp.async.bulk) through two B buffers, one round's copy
// overlapping the previous round's MMAs.  A compact tip child's U is its
// column of P, read from the split P' blocks.
//
// TMEM: post 128 columns [U_k]; pre 256 [q_x | W_x].  One CTA per SM
// (192 KB of shared memory).
//
// Rescaling, exponents and the Eq. 8 terms follow the 64-state path
// (per-category exponents; ratio_tc_kernel combines the categories).
// Every wait is bounded; on expiry the kernel raises ERR_TIMEOUT, drains
// (bounded) the copies and MMAs it issued, frees its TMEM and returns.
#pragma once

namespace phylo {

constexpr int kTcbSP = 128;                  // padded states of this path
constexpr int kTcbNB = kTcbSP / 64;          // 64-blocks per dimension
constexpr uint32_t kTcbBlock = 3 * kTerm64;  // one 64 x 64 three-term block
static_assert(kTcbUnitBytes == 2 * kTcbNB * kTcbNB * kTcbBlock, "tile block size");
// Shared memory: A 2 x 48 KB (both K-blocks), B ring 2 x 48 KB (+1024 for alignment).
constexpr size_t kTcbSmem = 1024 + 2 * (size_t)kOp128 + 4 * (size_t)kTcbBlock;
constexpr int kTcbLd = kTcbSP + 4;           // output staging row stride (floats)
static_assert((size_t)kTcRows * kTcbLd * 4 <= 2 * (size_t)kOp128, "staging fits in A");

__device__ __forceinline__ const unsigned char* tcb_unit(const LevelArgs<float>& a, int b,
                                                         int r) {
  return a.tc_tiles + ((size_t)b * a.n_cat + r) * kTcbUnitBytes;
}

// Stored U rows of node x (pattern 0, category r); row stride R * 128 floats.
__device__ __forceinline__ const float* tcb_u_rows(const LevelArgs<float>& a, int x, int r) {
  return a.post + (u_slot(a, x) * a.n_patterns * a.n_cat + r) * kTcbSP;
}

// Entries 64 kb + 8 j .. 64 kb + 8 j + 7 of column y of P_x for branch b (row
// y of P', read from the split P' blocks: the three BF16 terms summed); a
// gap (y = S) gives ones up to S, y < 0 (past the last pattern) zeros.
__device__ __forceinline__ void tcb_col8(const LevelArgs<float>& a, int b, int r, int y, int kb,
                                         int j, float4& lo, float4& hi) {
  const int S = a.n_states;
  if (y < 0 || y >= S) {
    const float g = y < 0 ? 0.f : 1.f;
    const int s = 64 * kb + 8 * j;
    lo = make_float4(s < S ? g : 0.f, s + 1 < S ? g : 0.f, s + 2 < S ? g : 0.f,
                     s + 3 < S ? g : 0.f);
    hi = make_float4(s + 4 < S ? g : 0.f, s + 5 < S ? g : 0.f, s + 6 < S ? g : 0.f,
                     s + 7 < S ? g : 0.f);
    return;
  }
  const unsigned char* blk = tcb_unit(a, b, r) + tcb_block(1, y >> 6, kb);
  const uint32_t off = tc::b16_chunk(y & 63, j);
  const uint4 t0 = __ldg(reinterpret_cast<const uint4*>(blk + off));
  const uint4 t1 = __ldg(reinterpret_cast<const uint4*>(blk + kTerm64 + off));
  const uint4 t2 = __ldg(reinterpret_cast<const uint4*>(blk + 2 * kTerm64 + off));
  const uint32_t w0[4] = {t0.x, t0.y, t0.z, t0.w}, w1[4] = {t1.x, t1.y, t1.z, t1.w},
                 w2[4] = {t2.x, t2.y, t2.z, t2.w};
  float v[8];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    // element 2 i in the low half of word i, 2 i + 1 in the high half
    v[2 * i] = (__uint_as_float(w0[i] << 16) + __uint_as_float(w1[i] << 16)) +
               __uint_as_float(w2[i] << 16);
    v[2 * i + 1] = (__uint_as_float(w0[i] & 0xffff0000u) + __uint_as_float(w1[i] & 0xffff0000u)) +
                   __uint_as_float(w2[i] & 0xffff0000u);
  }
  lo = make_float4(v[0], v[1], v[2], v[3]);
  hi = make_float4(v[4], v[5], v[6], v[7]);
}

// Both K-blocks of a child's U rows in the cooperative layout (v[kb], rows
// c0 + coop_row(it)), each row's stored exponent in E[it] (0 for a tip),
// a compact tip's state in y[it] (-1 otherwise).
__device__ __forceinline__ void tcb_child_rows(float4 (&v)[2][8], int (&E)[4], int (&y)[4],
                                               const LevelArgs<float>& a, const TcChild& x,
                                               int r, int c0) {
  const int C = a.n_patterns, j = threadIdx.x & 7;
  if (!x.compact) {
    const float* base = tcb_u_rows(a, x.b, r);
#pragma unroll
    for (int kb = 0; kb < kTcbNB; ++kb)
      coop_load(v[kb], base + 64 * kb, (size_t)a.n_cat * kTcbSP, c0, C);
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int c = c0 + coop_row(it);
      y[it] = -1;
      E[it] = x.internal && c < C
                  ? a.escale[((size_t)(x.b - a.n_tips) * a.n_cat + r) * a.escale_stride + c]
                  : 0;
    }
    return;
  }
#pragma unroll
  for (int it = 0; it < 4; ++it) {
    const int c = c0 + coop_row(it);
    y[it] = c < C ? (int)a.tip_states[(size_t)x.b * a.state_stride + c] : -1;
    E[it] = 0;
  }
#pragma unroll
  for (int kb = 0; kb < kTcbNB; ++kb)
#pragma unroll
    for (int it = 0; it < 4; ++it) tcb_col8(a, x.b, r, y[it], kb, j, v[kb][2 * it], v[kb][2 * it + 1]);
}

// This thread's half row (states 64 h .. 64 h + 63) of a child's U, for
// pattern c: stored, or for a compact tip (state y) its column of P.
__device__ __forceinline__ void tcb_child_half(float (&u)[64], const LevelArgs<float>& a,
                                               const TcChild& x, int r, int c, int h, int y) {
  if (c >= a.n_patterns) {
#pragma unroll
    for (int i = 0; i < 64; ++i) u[i] = 0.f;
    return;
  }
  if (!x.compact) {
    const float4* src = reinterpret_cast<const float4*>(tcb_u_rows(a, x.b, r) +
                                                        (size_t)c * a.n_cat * kTcbSP + 64 * h);
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const float4 f = __ldg(src + i);
      u[4 * i] = f.x;
      u[4 * i + 1] = f.y;
      u[4 * i + 2] = f.z;
      u[4 * i + 3] = f.w;
    }
    return;
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    float4 lo, hi;
    tcb_col8(a, x.b, r, y, h, j, lo, hi);
    u[8 * j] = lo.x;
    u[8 * j + 1] = lo.y;
    u[8 * j + 2] = lo.z;
    u[8 * j + 3] = lo.w;
    u[8 * j + 4] = hi.x;
    u[8 * j + 5] = hi.y;
    u[8 * j + 6] = hi.z;
    u[8 * j + 7] = hi.w;
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

// One round of a contraction: the two matrix blocks at bsrc (blocks jn = 0,
// 1 of one K-block) times A buffer ab (that K-block of the A operand) into
// d_tmem.
struct TcbRound {
  const unsigned char* bsrc;
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

// Runs rounds 0 .. n-1 (round_of(i) generates round i) on A operands already
// staged; the caller has issued the block copies of rounds 0 and 1 (those
// that exist).  While round i's MMAs run, round i + 1's blocks are in flight
// and round i + 2's copy starts once round i's MMAs have freed its buffer.
// False on a timeout (ERR_TIMEOUT raised); on success every MMA is done.
template <class RoundOf>
__device__ __forceinline__ bool tcb_rounds(unsigned char* A0, unsigned char* B0, uint64_t* bars,
                                           TcbPhases& ph, int n, RoundOf round_of, int* err) {
#pragma unroll 1
  for (int i = 0; i < n; ++i) {
    const TcbRound cur = round_of(i);
    if (!tcb_wait(bars, ph, i & 1, err)) return false;  // round i's blocks (and the A operand)
    if (threadIdx.x == 0) {
      tcb_mma_round(cur.d_tmem, tcb_a(A0, cur.ab), tcb_b(B0, i & 1), cur.accumulate);
      tc::commit(&bars[2 + (i & 1)]);
      ph.issue(2 + (i & 1));
    }
    if (i + 2 < n) {  // round i's MMAs free its B buffer for round i + 2
      if (!tcb_wait(bars, ph, 2 + (i & 1), err)) return false;
      tcb_issue_b(B0, bars, ph, i + 2, round_of(i + 2).bsrc);
    }
  }
  for (int i = n >= 2 ? n - 2 : 0; i < n; ++i)
    if (!tcb_wait(bars, ph, 2 + (i & 1), err)) return false;
  return true;
}

// ---------------------------------------------------------------------------
// Post-order level (Eq. 2), every level but the root's; with `tip_level`
// the level's nodes are tips with partial vectors, whose U = P p is formed
// from those vectors before the first level runs.
// ---------------------------------------------------------------------------
template <typename T>  // float only
__global__ void __launch_bounds__(kTcThreads) post_tcb_kernel(LevelArgs<T> a) {
  static_assert(std::is_same<T, float>::value, "tensor-core path is FP32");
  pdl_wait_and_release();  // before TMEM, smem or any global access
  TCB_PROLOGUE(128)
  const int R = a.n_cat, C = a.n_patterns;
  const int4 d = a.level_desc[blockIdx.y];
  const int k = d.x, r = blockIdx.z, lane = tid & 31;
  const int c0 = blockIdx.x * kTcRows;
  const bool tip = a.tip_level;
  // round kb: U_k (+)= p_k[:, kb] P_k[:, kb]'; both rounds' blocks copied now
  auto round_of = [=, &a](int kb) {
    return TcbRound{tcb_unit(a, k, r) + tcb_block(0, 0, kb), kb, tmem, kb > 0};
  };
  tcb_issue_b(B0, bars, ph, 0, round_of(0).bsrc);
  tcb_issue_b(B0, bars, ph, 1, round_of(1).bsrc);
  float4 v[2][8];
  if (tip) {
#pragma unroll
    for (int kb = 0; kb < kTcbNB; ++kb)
      coop_load(v[kb], a.tip_partials + (size_t)k * C * kTcbSP + 64 * kb, kTcbSP, c0, C);
  } else {
    // p_k = U_i o U_j, each row rescaled into [1/2, 1)
    const TcChild x0 = tc_child(a.n_tips, d.y, d.w & kDescFlagCompact0);
    const TcChild x1 = tc_child(a.n_tips, d.z, d.w & kDescFlagCompact1);
    float4 u[2][8];
    int E0[4], E1[4], y[4];
    tcb_child_rows(v, E0, y, a, x0, r, c0);
    tcb_child_rows(u, E1, y, a, x1, r, c0);
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      float m = 0.f;
#pragma unroll
      for (int kb = 0; kb < kTcbNB; ++kb) {
        v[kb][2 * it] = mul4(v[kb][2 * it], u[kb][2 * it]);
        v[kb][2 * it + 1] = mul4(v[kb][2 * it + 1], u[kb][2 * it + 1]);
        m = amax4(v[kb][2 * it + 1], amax4(v[kb][2 * it], m));
      }
      m = row_max8(m);
      const int c = c0 + coop_row(it);
      const int e = rescale_exponent(m, c < C, a.err);
      const float sc = ldexpf(1.f, -e);
#pragma unroll
      for (int kb = 0; kb < kTcbNB; ++kb)
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          float4& w = v[kb][2 * it + q];
          w = make_float4(w.x * sc, w.y * sc, w.z * sc, w.w * sc);
        }
      if (c < C && (lane & 7) == 0)
        a.escale[((size_t)(k - a.n_tips) * R + r) * a.escale_stride + c] = E0[it] + E1[it] + e;
    }
  }
#pragma unroll
  for (int kb = 0; kb < kTcbNB; ++kb) coop_put(tcb_a(A0, kb), v[kb]);
  tc::fence_smem_for_async();
  const bool ok = tcb_rounds(A0, B0, bars, ph, kTcbNB, round_of, a.err);
  if (ok) {  // U_k, stored as computed (exponent: escale of k)
    float* st = reinterpret_cast<float*>(base);  // A is free: every MMA is done
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      float w[32];
      tc::ld32(trow + 64 * h + 32 * q, w);
#pragma unroll
      for (int i = 0; i < 32; i += 4)
        *reinterpret_cast<float4*>(st + row * kTcbLd + 64 * h + 32 * q + i) =
            make_float4(w[i], w[i + 1], w[i + 2], w[i + 3]);
    }
    __syncthreads();
    tcb_store_rows(a.post + (u_slot(a, k) * C * R + r) * kTcbSP, (size_t)R * kTcbSP, c0, C, st);
  }
  TCB_EPILOGUE(128)
}

// ---------------------------------------------------------------------------
// Eq. 3 at the root: L_c = sum_r w_r 2^(E_i + E_j) pi' (U_i o U_j), the sum
// over r taken relative to the largest exponent; W_c log L_c summed per tile.
// ---------------------------------------------------------------------------
template <typename T>  // float only
__global__ void __launch_bounds__(kTcRows) root_tcb_kernel(LevelArgs<T> a) {
  static_assert(std::is_same<T, float>::value, "tensor-core path is FP32");
  pdl_wait_and_release();
  __shared__ double lred[kTcRows / 32];
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int4 d = a.level_desc[0];
  const TcChild xs[2] = {tc_child(a.n_tips, d.y, d.w & kDescFlagCompact0),
                         tc_child(a.n_tips, d.z, d.w & kDescFlagCompact1)};
  const int c = blockIdx.x * kTcRows + threadIdx.x;
  double term = 0.0;
  if (c < C) {
    int y[2] = {-1, -1};
    for (int x = 0; x < 2; ++x)
      if (xs[x].compact) y[x] = a.tip_states[(size_t)xs[x].b * a.state_stride + c];
    float lsum = 0.f;
    int lexp = INT_MIN / 2;
    for (int r = 0; r < R; ++r) {
      int E = 0;
      for (int x = 0; x < 2; ++x)
        if (xs[x].internal)
          E += a.escale[((size_t)(xs[x].b - a.n_tips) * R + r) * a.escale_stride + c];
      float dot = 0.f;
      for (int kb = 0; kb < kTcbNB; ++kb)
        for (int j = 0; j < 8; ++j) {
          float4 u[2][2];
          for (int x = 0; x < 2; ++x) {
            if (xs[x].compact) {
              tcb_col8(a, xs[x].b, r, y[x], kb, j, u[x][0], u[x][1]);
            } else {
              const float4* src = reinterpret_cast<const float4*>(
                  tcb_u_rows(a, xs[x].b, r) + (size_t)c * R * kTcbSP + 64 * kb + 8 * j);
              u[x][0] = __ldg(src);
              u[x][1] = __ldg(src + 1);
            }
          }
          const int s = 64 * kb + 8 * j;
          for (int q = 0; q < 2; ++q) {
            const float4 p4 = mul4(u[0][q], u[1][q]);
            const float pe[4] = {p4.x, p4.y, p4.z, p4.w};
            for (int i = 0; i < 4; ++i)
              if (s + 4 * q + i < S) dot = fmaf(a.root_pit[s + 4 * q + i], pe[i], dot);
          }
        }
      if (dot != 0.f) {
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
// Pre-order level (Eq. 4) with the per-category Eq. 8 terms: one CTA per
// (tile, node k, category r, child x); blockIdx.z = 2 r + x.
// ---------------------------------------------------------------------------
template <typename T>  // float only
__global__ void __launch_bounds__(kTcThreads) pre_tcb_kernel(LevelArgs<T> a) {
  static_assert(std::is_same<T, float>::value, "tensor-core path is FP32");
  pdl_wait_and_release();
  TCB_PROLOGUE(256)
  __shared__ float xn[2][kTcRows], xm[2][kTcRows];  // the halves' num and q maximum
  const int R = a.n_cat, C = a.n_patterns, S = a.n_states;
  const int4 d = a.level_desc[blockIdx.y];
  const int k = d.x, x = (int)(blockIdx.z & 1), r = (int)(blockIdx.z >> 1);
  const int lane = tid & 31, j = lane & 7;
  const TcChild cx = tc_child(a.n_tips, x ? d.z : d.y,
                              d.w & (x ? kDescFlagCompact1 : kDescFlagCompact0));
  const TcChild cy = tc_child(a.n_tips, x ? d.y : d.z,
                              d.w & (x ? kDescFlagCompact0 : kDescFlagCompact1));
  const bool root = k == a.root;
  const size_t kslot = (size_t)(k - a.n_tips);
  const int c0 = blockIdx.x * kTcRows, c = c0 + row;
  const int estr = a.escale_stride;
  // rounds: W_x = a_x Q (K-blocks 0, 1), then for an internal child
  // q_x = a_x P_x (K-blocks 0, 1); TMEM columns [q_x | W_x]
  const int n_rounds = cx.internal ? 2 * kTcbNB : kTcbNB;
  auto round_of = [=, &a](int i) {
    const int kb = i % kTcbNB;
    if (i < kTcbNB) return TcbRound{a.qt + tcb_block(0, 0, kb), kb, tmem + 128u, kb > 0};
    return TcbRound{tcb_unit(a, cx.b, r) + tcb_block(1, 0, kb), kb, tmem, kb > 0};
  };
  tcb_issue_b(B0, bars, ph, 0, round_of(0).bsrc);
  tcb_issue_b(B0, bars, ph, 1, round_of(1).bsrc);
  // row-layout values of this thread's row for the epilogue
  int eq_row = 0, ey_row = 0, yx_row = -1;
  if (c < C) {
    if (!root) eq_row = a.pre_escale[(kslot * R + r) * estr + c];
    if (cy.internal) ey_row = a.escale[((size_t)(cy.b - a.n_tips) * R + r) * estr + c];
    if (cx.compact) yx_row = a.tip_states[(size_t)cx.b * a.state_stride + c];
  }
  // a_x = q_k o U_y in the cooperative layout, split into A
  float4 q[2][8];
  int eq[4];
  if (!root) {
#pragma unroll
    for (int kb = 0; kb < kTcbNB; ++kb)
      coop_load(q[kb], a.pre + (kslot * C * R + r) * kTcbSP + 64 * kb, (size_t)R * kTcbSP, c0, C);
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int cc = c0 + coop_row(it);
      eq[it] = cc < C ? a.pre_escale[(kslot * R + r) * estr + cc] : 0;
    }
  } else {  // q_root = pi
#pragma unroll
    for (int kb = 0; kb < kTcbNB; ++kb) {
      const int s = 64 * kb + 8 * j;
      const float4 p0 = make_float4(s < S ? a.root_pit[s] : 0.f, s + 1 < S ? a.root_pit[s + 1] : 0.f,
                                    s + 2 < S ? a.root_pit[s + 2] : 0.f,
                                    s + 3 < S ? a.root_pit[s + 3] : 0.f);
      const float4 p1 = make_float4(s + 4 < S ? a.root_pit[s + 4] : 0.f,
                                    s + 5 < S ? a.root_pit[s + 5] : 0.f,
                                    s + 6 < S ? a.root_pit[s + 6] : 0.f,
                                    s + 7 < S ? a.root_pit[s + 7] : 0.f);
#pragma unroll
      for (int it = 0; it < 4; ++it) {
        q[kb][2 * it] = p0;
        q[kb][2 * it + 1] = p1;
      }
    }
#pragma unroll
    for (int it = 0; it < 4; ++it) eq[it] = 0;
  }
  int Ey[4], Ex[4], yy[4], yxc[4];
  {
    float4 uy[2][8];
    tcb_child_rows(uy, Ey, yy, a, cy, r, c0);
#pragma unroll
    for (int kb = 0; kb < kTcbNB; ++kb)
#pragma unroll
      for (int i = 0; i < 8; ++i) q[kb][i] = mul4(q[kb][i], uy[kb][i]);
  }
#pragma unroll
  for (int kb = 0; kb < kTcbNB; ++kb) coop_put(tcb_a(A0, kb), q[kb]);
  tc::fence_smem_for_async();
  // den = a_x . U_x per row (U_x loads in flight during the MMAs)
  float den[4];
  {
    float4 ux[2][8];
    tcb_child_rows(ux, Ex, yxc, a, cx, r, c0);
    const bool ok0 = tcb_rounds(A0, B0, bars, ph, n_rounds, round_of, a.err);
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      float s = 0.f;
#pragma unroll
      for (int kb = 0; kb < kTcbNB; ++kb)
        s = dot4(q[kb][2 * it + 1], ux[kb][2 * it + 1], dot4(q[kb][2 * it], ux[kb][2 * it], s));
      den[it] = row_sum8(s);
    }
    if (!ok0) {
      TCB_EPILOGUE(256)
      return;
    }
  }
  // epilogue (row layout, thread (row, h) owns states 64 h .. 64 h + 63)
  float num = 0.f, m = 0.f;
  {
    float u[64];
    tcb_child_half(u, a, cx, r, c, h, yx_row);
#pragma unroll
    for (int qq = 0; qq < 2; ++qq) {
      float w[32];
      tc::ld32(trow + 128 + 64 * h + 32 * qq, w);
#pragma unroll
      for (int i = 0; i < 32; ++i) num = fmaf(w[i], u[32 * qq + i], num);
    }
  }
  float qo[64];
  if (cx.internal) {
    tc::ld32(trow + 64 * h, *reinterpret_cast<float(*)[32]>(qo));
    tc::ld32(trow + 64 * h + 32, *reinterpret_cast<float(*)[32]>(qo + 32));
#pragma unroll
    for (int i = 0; i < 64; ++i) m = fmaxf(m, fabsf(qo[i]));
  }
  xn[h][row] = num;
  xm[h][row] = m;
  __syncthreads();
  num += xn[1 - h][row];
  m = fmaxf(m, xm[1 - h][row]);
  if (cx.compact && yx_row >= S) num = 0.f;  // d/dt of the all-ones vector is 0
  float* rt = reinterpret_cast<float*>(a.rterm);
  if (c < C && h == 0) {
    rt[((kslot * C + c) * R + r) * 4 + x] = (float)(a.cat_w[r] * a.rates[r]) * num;
  }
  if (x == 0) {  // den and the exponent of the Eq. 8 terms, from the cooperative layout
#pragma unroll
    for (int it = 0; it < 4; ++it) {
      const int cc = c0 + coop_row(it);
      if (cc < C && j == 0) {
        float* t4 = rt + ((kslot * C + cc) * R + r) * 4;
        t4[2] = a.cat_wt[r] * den[it];
        t4[3] = __int_as_float(eq[it] + Ex[it] + Ey[it]);
      }
    }
  }
  if (cx.internal) {  // q_x = a_x P_x, the row rescaled into [1/2, 1)
    const int e = rescale_exponent(m, c < C, a.err);
    const float f = ldexpf(1.f, -e);
    float* st = reinterpret_cast<float*>(base);  // A is free: every MMA is done
#pragma unroll
    for (int i = 0; i < 64; i += 4)
      *reinterpret_cast<float4*>(st + row * kTcbLd + 64 * h + i) =
          make_float4(qo[i] * f, qo[i + 1] * f, qo[i + 2] * f, qo[i + 3] * f);
    if (c < C && h == 0)  // q_x = P_x' (q_k o U_y): exponents of q_k and of U_y
      a.pre_escale[((size_t)(cx.b - a.n_tips) * R + r) * estr + c] = e + eq_row + ey_row;
    __syncthreads();
    tcb_store_rows(a.pre + ((size_t)(cx.b - a.n_tips) * C * R + r) * kTcbSP, (size_t)R * kTcbSP,
                   c0, C, st);
  }
  TCB_EPILOGUE(256)
}

#undef TCB_PROLOGUE
#undef TCB_EPILOGUE

inline cudaError_t launch_tcb(const LevelArgs<float>& a, bool post, cudaStream_t st) {
  if (post) {
    if (a.root_level) return launch_pdl(root_tcb_kernel<float>, dim3(a.n_tiles), kTcRows, 0, st, a);
    dim3 grid(a.n_tiles, a.n_level, a.n_cat);
    return launch_pdl(post_tcb_kernel<float>, grid, kTcThreads, kTcbSmem, st, a);
  }
  dim3 grid(a.n_tiles, a.n_level, 2 * a.n_cat);
  return launch_pdl(pre_tcb_kernel<float>, grid, kTcThreads, kTcbSmem, st, a);
}

inline cudaError_t launch_pmat_tcb(const PmatArgs& a, cudaStream_t st) {
  return launch_pmat_big<kTcbSP>(a, st);  // (writes the operand blocks: a.tiles is set)
}

inline cudaError_t prepare_tcb() {
  cudaError_t e = cudaFuncSetAttribute(post_tcb_kernel<float>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kTcbSmem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pre_tcb_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTcbSmem);
  return e;
}

}  // namespace phylo
