// Internal declarations shared by the host API (phylo_api.cu) and the kernel
// translation units (kernels_fp32.cu, kernels_fp64.cu).  Not installed.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cstring>

#include <cuda_runtime.h>

namespace phylo {

// Flags of a level-node descriptor: child 0 / child 1 is a tip with a
// compact state; child 0 / child 1 is a cherry fused into this node (FP32,
// 4 states: kernels_p4.cuh).
constexpr int kDescFlagCompact0 = 1, kDescFlagCompact1 = 2;
constexpr int kDescFlagCherry0 = 4, kDescFlagCherry1 = 8;

// Device-side numeric flags (bit mask in the workspace's error word).
enum : int {
  ERR_ZERO_PARTIAL = 1,  // a partial vector was all zero / NaN for a pattern
  ERR_BAD_LENGTH = 2,    // a branch length was negative or not finite
  ERR_BAD_RATIO = 4,     // a gradient denominator was zero or not finite
  ERR_TIMEOUT = 8        // a bounded wait on an asynchronous copy expired
};

__host__ __device__ inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

// Padded state count used by the kernels for a model with S states.
inline int padded_states(int S) {
  if (S <= 4) return 4;
  if (S <= 20) return 20;
  if (S <= 64) return 64;
  if (S <= 128) return 128;
  return 256;
}

// Lanes per pattern in the register kernels (next power of two >= R).
inline int lanes_per_pattern(int R) {
  int rp = 1;
  while (rp < R) rp <<= 1;
  return rp;
}

// Threads per block of the register kernels (one thread per (pattern, r)).
constexpr int kSmallThreads = 128;
// Patterns per block of the shared-memory kernels for S_pad = 64.
constexpr int kWideThreads = 256;
constexpr int kWidePatternsF32 = 16;
constexpr int kWidePatternsF64 = 8;
// Patterns per block of the kernels for S_pad = 128 and 256 (kernels_big.cuh).
constexpr int kBigPatternsF32 = 16;
constexpr int kBigPatternsF64 = 8;
#ifndef PHYLO_BIG_SPT
#define PHYLO_BIG_SPT 2
#endif
constexpr int kBigStatesPerThread = PHYLO_BIG_SPT;  // FP32: states per thread
constexpr int kMaxStates = 256;

// FP32 4-state path (kernels_p4.cuh): one thread per pattern; patterns come
// in tiles of 32 (one warp), the unit of the partials' layout and of the
// per-tile sums.  Partials are tile-blocked, [slot][tile][r][32][4] floats,
// so a warp's access to one category is 512 contiguous bytes.
constexpr int kP4TilePatterns = 32;
__host__ __device__ inline size_t p4_index(size_t slot, int c, int r, int R, int n_tiles) {
  return ((slot * n_tiles + (size_t)(c >> 5)) * R + r) * 32 + (c & 31);
}
// Whether a path stores its partials tile-blocked (FP32, 4 padded states).
inline bool uses_p4_tiles(int SP, bool fp64) { return SP == 4 && !fp64; }
// Tip-state rows are padded to 16 bytes (row starts aligned for bulk copies).
inline int tip_state_stride(int C) { return round_up(C, 16); }
// The FP32 kernels for 4 and 20 padded states read their matrices in the
// orientations the products use, built that way by the matrix kernel: per
// branch, [P' of every category][dP' of every category][P of every
// category] (SP x SP floats each; P' rows are the columns of P).  The dP
// region is then empty.
inline bool uses_tr_layout(int SP, bool fp64) { return (SP == 4 || SP == 20) && !fp64; }
constexpr int kP4MatKinds = 3;

// FP32 with 21..64 states runs on the tensor cores (kernels_tc64.cuh):
// 128-pattern tiles and one rescale exponent per (node, category, pattern).
inline bool uses_tensor_cores(int SP, bool fp64) { return SP == 64 && !fp64; }
constexpr int kTcTilePatterns = 128;
// Matrix operand tiles of one (branch, category) on that path: P and P' as
// three-term BF16 splits, then P' in FP32 (kernels_tc64.cuh gives the
// layout); Q' as one more three-term 64 x 64 operand per model.
constexpr size_t kTcUnitBytes = 65536;
constexpr size_t kTcQtBytes = 3 * 64 * 128;

// Round-to-nearest-even BF16 of a finite float, and back (host side).
inline uint16_t host_bf16(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
inline float host_bf16_value(uint16_t b) {
  const uint32_t u = (uint32_t)b << 16;
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}

// Bytes of the Q' operand for SP = 64 or 128 padded states: (SP / 64)^2
// blocks of 64 x 64 three-term BF16 values.
inline size_t qt_bytes(int SP) { return (size_t)(SP / 64) * (SP / 64) * kTcQtBytes; }

// Q' as the three-term BF16 operand of the tensor-core pre-order step (the
// Eq. 8 numerator through dP = gamma Q P): row s holds column s of
// Q = V diag(lambda) Vinv (FP64, rounded once to FP32), each FP32 value
// split as x = t0 + t1 + t2 with t_i the round-to-nearest BF16 of the
// remainder, cut into 64 x 64 blocks (block (jn, jk) holds rows 64 jn ..,
// columns 64 jk ..; blocks of one K-block jk adjacent, jn fastest) stored
// in the K-major 128-byte-swizzle layout the MMAs read (element (row, k) of
// a term at row * 128 + (((k / 8) ^ (row % 8)) * 16) + (k % 8) * 2, terms
// 8 KB apart).  Rows and columns past S are zero.  out: qt_bytes(SP).
inline void build_qt_tile(int S, int SP, const double* V, const double* Vinv,
                          const double* lambda, unsigned char* out) {
  std::memset(out, 0, qt_bytes(SP));
  const size_t term = 64 * 128;
  const int NB = SP / 64;
  for (int s = 0; s < S; ++s)
    for (int t = 0; t < S; ++t) {
      double q = 0.0;  // Q[t][s]
      for (int m = 0; m < S; ++m) q += V[t * S + m] * lambda[m] * Vinv[m * S + s];
      float rem = (float)q;
      const int n = s & 63, k = t & 63;
      const size_t blk = ((size_t)(t >> 6) * NB + (s >> 6)) * kTcQtBytes;
      const size_t off = blk + (size_t)n * 128 + ((size_t)((k >> 3) ^ (n & 7)) << 4) + (k & 7) * 2;
      for (int i = 0; i < 3; ++i) {
        const uint16_t b = host_bf16(rem);
        std::memcpy(out + i * term + off, &b, 2);
        rem = rem - host_bf16_value(b);
      }
    }
}

// FP32 paths whose post-order pass stores U = P p per node instead of p
// (20 padded states, kernels.cuh; 21..64 and 65..128 states, kernels_tc64.cuh
// and kernels_tcb.cuh): tips
// with partial vectors keep their U in extra slots of the post region, and
// the pre-order step forms Eq. 8's numerator through Q.
inline bool uses_u_form(int SP, bool fp64) {
  return (SP == 20 || SP == 64 || SP == 128) && !fp64;
}

// Q = V diag(lambda) Vinv in FP64, rounded once to FP32, row-major SP x SP
// with zero padding (the pre-order step of the 4- and 20-state U form).
inline void build_q_matrix(int S, int SP, const double* V, const double* Vinv,
                           const double* lambda, float* out) {
  for (int i = 0; i < SP * SP; ++i) out[i] = 0.f;
  for (int t = 0; t < S; ++t)
    for (int s = 0; s < S; ++s) {
      double q = 0.0;
      for (int m = 0; m < S; ++m) q += V[t * S + m] * lambda[m] * Vinv[m * S + s];
      out[t * SP + s] = (float)q;
    }
}

// FP32 with 65..128 states runs on the tensor cores too (kernels_tcb.cuh):
// 128-pattern tiles, per-category exponents, and the matrices written by
// the matrix kernel directly as 64 x 64 BF16 operand blocks (kind P, P'
// x 2 x 2 blocks of 24 KB per (branch, category)).
inline bool uses_tc_big(int SP, bool fp64) { return SP == 128 && !fp64; }
constexpr size_t kTcbUnitBytes = 2 * 2 * 2 * (3 * 64 * 128);
// Offset of block (kind, jn, jk) in a (branch, category) unit: kind 0 = P,
// 1 = P' (its rows are the columns of P); block row n, column k
// holds M[64 jn + n][64 jk + k] as three BF16 terms of 8 KB each, in the
// K-major 128-byte-swizzle layout of tc.cuh.  The blocks of one K-block jk
// are adjacent (jn fastest), so one bulk copy stages a contraction round.
__host__ __device__ constexpr size_t tcb_block(int kind, int jn, int jk) {
  return (((size_t)kind * 2 + jk) * 2 + jn) * (3 * 64 * 128);
}
// Paths with per-category exponents and Eq. 8 terms combined by the ratio
// kernel (both tensor-core paths).
inline bool uses_tc_terms(int SP, bool fp64) {
  return uses_tensor_cores(SP, fp64) || uses_tc_big(SP, fp64);
}

// The eigenvectors as double-float pairs for the tensor-core path's matrix
// kernel: out = [V' hi][V' lo][Vinv hi][Vinv lo] (each 64 x 64 floats, V'
// the transpose of V, zero outside S x S) then [pi hi][pi lo] (64 each).
// Returns whether the decomposition is the symmetric one of a reversible
// model, Vinv[m][t] = pi_t V[t][m] (then P(t) = I + V diag(e) V' diag(pi)
// and P_st pi_s = P_ts pi_t, which the kernel exploits).
// The same tables for S_pad = 128 and 256 (FP32 matrix build of
// kernels_big.cuh): each SP x SP, then pi, SP each.
inline size_t eigen_split_floats(int SP) { return 4 * (size_t)SP * SP + 2 * (size_t)SP; }
constexpr size_t kEigenSplitFloats = 4 * 64 * 64 + 2 * 64;
inline bool build_eigen_split(int S, int SP, const double* V, const double* Vinv,
                              const double* pi, float* out) {
  const size_t sq = (size_t)SP * SP;
  for (size_t i = 0; i < eigen_split_floats(SP); ++i) out[i] = 0.f;
  double vmax = 0.0;
  for (int i = 0; i < S * S; ++i) vmax = Vinv[i] > vmax ? Vinv[i] : (-Vinv[i] > vmax ? -Vinv[i] : vmax);
  bool reversible = true;
  for (int m = 0; m < S; ++m)
    for (int s = 0; s < S; ++s) {
      const double v = V[s * S + m], w = Vinv[m * S + s];
      const float vh = (float)v, wh = (float)w;
      out[0 * sq + (size_t)m * SP + s] = vh;
      out[1 * sq + (size_t)m * SP + s] = (float)(v - (double)vh);
      out[2 * sq + (size_t)m * SP + s] = wh;
      out[3 * sq + (size_t)m * SP + s] = (float)(w - (double)wh);
      const double dev = w - pi[s] * v;
      if (!(dev <= 1e-10 * vmax && -dev <= 1e-10 * vmax)) reversible = false;
    }
  for (int s = 0; s < S; ++s) {
    const float ph = (float)pi[s];
    out[4 * sq + s] = ph;
    out[4 * sq + SP + s] = (float)(pi[s] - (double)ph);
  }
  return reversible;
}
// FP32 paths build their matrices from the double-float tables.
inline bool uses_eigen_split(int SP, bool fp64) { return !fp64; }

// Exponent planes per node: R on the tensor-core path, else 1 (one
// exponent per (node, pattern) shared by all categories).
inline int escale_planes(int SP, int R, bool fp64) {
  return uses_tc_terms(SP, fp64) ? R : 1;
}

// Patterns of one tile (the unit of the per-tile gradient sums).
inline int patterns_per_tile(int SP, int R, bool fp64) {
  if (SP == 4 && !fp64) return kP4TilePatterns;
  if (uses_tc_terms(SP, fp64)) return kTcTilePatterns;
  if (SP <= 20) return kSmallThreads / lanes_per_pattern(R);
  if (SP >= 128) return fp64 ? kBigPatternsF64 : kBigPatternsF32;
  return fp64 ? kWidePatternsF64 : kWidePatternsF32;
}

// Partial-vector elements stored per node.  Tile-blocked paths pad the
// patterns to whole tiles: FP32 with 4 padded states ([tile][r][32][4]),
// FP32 with 20 padded states ([tile][chunk][kSmallThreads][4], every lane of
// the RP-wide category slots present); the others store [C][R][SP].
inline size_t partial_elems_per_node(int SP, bool fp64, int C, int R, int n_tiles) {
  if (uses_p4_tiles(SP, fp64)) return (size_t)n_tiles * kP4TilePatterns * R * SP;
  if (SP == 20 && !fp64) return (size_t)n_tiles * kSmallThreads * SP;
  return (size_t)C * R * SP;
}

// Arguments of the post- and pre-order level kernels.  All arrays live in
// the caller's workspace.  Partials are pattern-major: [slot][c][r][SP],
// slot = node - n_tips for internal nodes.
template <typename T>
struct LevelArgs {
  const int2* children;        // [2N-1]; (-1,-1) for tips
  const int* level_nodes;      // internal nodes of this level
  const int4* level_desc;      // per level node: {k, child 0, child 1, flags}
  int n_level;                 // number of nodes in the level
  int root_level;              // 1 if the level is the root alone
  int level_cherry;            // 1 if a node of the level has a fused cherry child
  int n_tips, n_patterns, n_states, n_cat, root;
  const T* P;                  // [2N-2][R][SP][SP], row = parent state
                               // (tensor-core path: [2N-2][R] operand tiles;
                               // FP32 4 states: [2N-2][P' | dP' | P][R][16])
  const T* dP;                 // same layout: dP/dt = gamma_r Q P (null on
                               // the tensor-core and FP32 4-state paths,
                               // whose P region holds dP)
  T* post;                     // [N-1][C][R][SP] post-order partials (FP32,
                               // 20 and 64 padded states: U = P p of every
                               // internal node, then of every tip with partials)
  T* pre;                      // [N-1][C][R][SP] pre-order partials
  int* escale;                 // [N-1][planes][escale_stride] cumulative
                               // post-order exponents (planes: escale_planes)
  int* pre_escale;             // [N-1][R][escale_stride] cumulative pre-order
                               // exponents (tensor-core path only, else null)
  const uint8_t* tip_states;   // [N][state_stride]; value S = gap
  int state_stride;            // C rounded up to 16 (16-byte rows)
  int escale_stride;           // C rounded up to 4 (16-byte rows)
  const T* tip_partials;       // [N][C][SP] or nullptr
  const int* tip_has_partials; // [N] or nullptr
  const double* pattern_w;     // [C]
  const double* root_pi;       // [S]
  const double* cat_w;         // [R]
  const T* pattern_wt;         // [C] the same weights in T
  const T* cat_wt;             // [R] the same weights in T
  const T* root_pit;           // [S] the root distribution in T
  void* rterm;                 // tensor-core path: [N-1][C][R] float4 Eq. 8
                               // terms of each category (else null)
  double* gpart;               // [2N-2][n_tiles] per-tile gradient sums
  double* lpart;               // [n_tiles] per-tile log-likelihood sums
  int n_tiles;
  int* err;                    // numeric flags
  const unsigned char* tc_tiles;  // 65..128 states, FP32: the pre-split matrix
                                  // blocks [2N-2][R][kTcbUnitBytes] (else null)
  const unsigned char* qt;     // 21..64 states, FP32: Q' operand (kTcQtBytes)
  const float* qmat;           // 4 and 20 padded states, FP32: Q row-major [SP][SP]
  const double* rates;         // [R] category rates gamma_r
  int tip_level;               // U-form paths: the level's nodes are tips with
                               // partials (their U = P p, before level 1)
  int mats_ready;              // 1 if P was complete before the previous launch
                               // began (every launch but the first after the
                               // matrix kernel): the level may read P and its
                               // descriptors before griddepcontrol.wait
};

struct PmatArgs {
  const float* vsplit;   // tensor-core path: build_eigen_split's table
  int reversible;        // tensor-core path: the table's decomposition is symmetric
  const double* V;       // [S][S]
  const double* Vinv;    // [S][S]
  const double* lambda;  // [S]
  const double* rates;   // [R]
  const double* t;       // [n_branches]
  int n_branches, n_states, n_cat;
  void* P;               // [n_branches][R][SP][SP] of T
  void* dP;
  void* tiles;           // 65..128 states, FP32: the matrices written as pre-split
                         // operand blocks instead of P and dP (else null)
  int* err;
};

struct ReduceArgs {
  const double* gpart;   // [n_branches][n_tiles]; with gpart_pairs each entry
                         // holds a float pair {hi, lo} (value hi + lo)
  const double* lpart;   // [n_tiles]
  int n_tiles, n_branches;
  int gpart_pairs;       // FP32 with 4 or 20 padded states: tile sums as float
                         // pairs (no FP64 in those level kernels)
  double* out;           // [1 + n_branches]
};

// Launch with programmatic stream serialisation: the kernel may begin
// launching while its predecessor drains; every kernel launched this way
// starts with pdl_wait_and_release() (tma.cuh) before it touches memory
// that other kernels write.  PHYLO_PDL=0 at build time turns it off.
#ifndef PHYLO_PDL
#define PHYLO_PDL 1
#endif
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = PHYLO_PDL;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

// Launchers (kernels_fp32.cu / kernels_fp64.cu).  SP = padded states.
template <typename T>
cudaError_t launch_pmat(const PmatArgs& a, int SP, cudaStream_t st);
template <typename T>
cudaError_t launch_post_level(const LevelArgs<T>& a, int SP, int RP,
                              cudaStream_t st);
template <typename T>
cudaError_t launch_pre_level(const LevelArgs<T>& a, int SP, int RP,
                             cudaStream_t st);
// Work after the last pre-order level (the tensor-core path's Eq. 8
// ratios); a no-op elsewhere.
template <typename T>
cudaError_t launch_pre_finish(const LevelArgs<T>& a, int SP, cudaStream_t st);
template <typename T>
cudaError_t prepare_kernels(int SP, int RP);
cudaError_t launch_reduce(const ReduceArgs& a, cudaStream_t st);

// Chain-rule epilogues on the gradient g [2N-2] (kernels_fp64.cu).
cudaError_t launch_grad_rate_time(const double* g, int n_br, const double* rates,
                                  const double* times, double* d_rates, double* d_times,
                                  cudaStream_t st);
cudaError_t launch_grad_heights(const double* g, const int2* children, int n_tips,
                                const double* rates, double* d_heights, cudaStream_t st);
cudaError_t launch_grad_branch_sum(const double* g, const int* branches, const double* weights,
                                   int n, double* out, cudaStream_t st);

}  // namespace phylo
