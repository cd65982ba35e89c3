// phylo_evaluate_noalloc: one FP32 evaluation of log P(Y) and its gradient
// for a small problem, with every intermediate buffer (transition matrices,
// post- and pre-order partials, exponents, per-tile sums) placed in one
// statically sized device array instead of a caller workspace.
//
// Who needs it: callers that must not allocate device memory at all --
// runtimes whose GPU memory is owned by their own pool and that forbid side
// allocations, and fixed-footprint samplers or embedded services that must
// not grow their memory use after start-up.  They pass their inputs and
// receive the results; nothing is allocated per call.
//
// The array below is part of the library image: every GPU that loads the
// library keeps kNoAllocScratchBytes reserved until the process exits.
// Host code may only use its name to look its device address up with
// cudaGetSymbolAddress (done once per device, on the first call on that
// device, with that device current); the name itself is a host-side
// stand-in, not a device address, so it is never passed to a kernel.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "../../include/phylo_api.h"
#include "phylo_internal.h"

using namespace phylo;

namespace {

constexpr size_t kNoAllocScratchBytes = 32u << 20;  // 32 MiB
constexpr int kMaxNoAllocTips = 512;
constexpr int kMaxDevices = 64;
constexpr size_t kAlignNA = 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mutex;
void* g_scratch_ptr[kMaxDevices] = {};
thread_local char* t_err_buf = nullptr;  // the caller's message buffer
thread_local size_t t_err_cap = 0;

int na_fail(int code, const char* fmt, ...) {
  if (t_err_buf && t_err_cap) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(t_err_buf, t_err_cap, fmt, ap);
    va_end(ap);
  }
  return code;
}

struct NaRegion {
  size_t off = 0, bytes = 0;
};

struct NaLayout {
  int SP = 0, RP = 0, n_tiles = 0;
  NaRegion children, post_nodes, pre_nodes, post_desc, pre_desc, P, dP, post, pre, escale,
      pre_escale, rterm;
  NaRegion tip_states, pattern_w, V, Vinv, lambda, pi, rates, cat_w, t, vsplit, qt, qmat;
  NaRegion gpart, lpart, out, pattern_wt, cat_wt, pi_t;
  size_t total = 0;
};

void na_add(NaLayout& L, NaRegion& r, size_t bytes) {
  r.off = (L.total + kAlignNA - 1) / kAlignNA * kAlignNA;
  r.bytes = bytes;
  L.total = r.off + bytes;
}

// Sizes here are bounded (N <= 512, S <= 64, R <= 8, C checked against the
// scratch size), so no product below can overflow a size_t.
void na_layout(int N, int C, int S, int R, NaLayout* Lp) {
  NaLayout L;
  L.SP = padded_states(S);
  L.RP = lanes_per_pattern(R);
  const int ct = patterns_per_tile(L.SP, R, false);
  L.n_tiles = (C + ct - 1) / ct;
  const size_t n_nodes = 2 * (size_t)N - 1, n_br = 2 * (size_t)N - 2, n_int = (size_t)N - 1;
  const bool tc = uses_tensor_cores(L.SP, false);
  const bool p4 = uses_tr_layout(L.SP, false);
  const size_t mat = n_br * R * (tc ? kTcUnitBytes
                                    : L.SP * L.SP * sizeof(float) * (p4 ? kP4MatKinds : 1));
  const size_t part =
      n_int * partial_elems_per_node(L.SP, false, C, R, L.n_tiles) * sizeof(float);
  na_add(L, L.children, n_nodes * sizeof(int2));
  na_add(L, L.post_nodes, n_int * sizeof(int));
  na_add(L, L.pre_nodes, n_int * sizeof(int));
  na_add(L, L.post_desc, n_int * sizeof(int4));
  na_add(L, L.pre_desc, n_int * sizeof(int4));
  na_add(L, L.P, mat);
  na_add(L, L.dP, tc || p4 ? 0 : mat);  // else the P region holds dP
  na_add(L, L.post, part);
  na_add(L, L.pre, part);
  const size_t eplane = n_int * (size_t)round_up(C, 4) * sizeof(int);
  na_add(L, L.escale, eplane * escale_planes(L.SP, R, false));
  if (tc) {
    na_add(L, L.pre_escale, eplane * R);
    na_add(L, L.rterm, n_int * (size_t)C * R * 16);
    na_add(L, L.qt, kTcQtBytes);
  }
  if (L.SP == 4 || L.SP == 20) na_add(L, L.qmat, (size_t)L.SP * L.SP * sizeof(float));
  na_add(L, L.tip_states, (size_t)N * tip_state_stride(C));
  na_add(L, L.pattern_w, (size_t)C * 8);
  na_add(L, L.V, (size_t)S * S * 8);
  na_add(L, L.Vinv, (size_t)S * S * 8);
  na_add(L, L.vsplit, eigen_split_floats(L.SP) * sizeof(float));  // FP32: always
  na_add(L, L.lambda, (size_t)S * 8);
  na_add(L, L.pi, (size_t)S * 8);
  na_add(L, L.rates, (size_t)R * 8);
  na_add(L, L.cat_w, (size_t)R * 8);
  na_add(L, L.t, n_br * 8);
  na_add(L, L.gpart, n_br * (size_t)L.n_tiles * 8);
  na_add(L, L.lpart, (size_t)L.n_tiles * 8);
  na_add(L, L.out, n_nodes * 8 + 8);
  na_add(L, L.pattern_wt, (size_t)C * sizeof(float));
  na_add(L, L.cat_wt, (size_t)R * sizeof(float));
  na_add(L, L.pi_t, (size_t)S * sizeof(float));
  *Lp = L;
}

// Device address of the scratch array on the current device, looked up on
// the first call on that device.
int scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return na_fail(PHYLO_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return na_fail(PHYLO_EINVAL, "device %d out of range", dev);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return na_fail(PHYLO_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
    for (int sp : {4, 20, 64})
      for (int rp : {1, 2, 4, 8})
        if (e == cudaSuccess) e = prepare_kernels<float>(sp, rp);
    if (e != cudaSuccess)
      return na_fail(PHYLO_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return PHYLO_OK;
}

__global__ void to_float_kernel(const double* __restrict__ src, float* dst, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)src[i];
}

cudaError_t launch_to_float(const double* src, float* dst, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  to_float_kernel<<<(n + 255) / 256, 256, 0, st>>>(src, dst, n);
  return cudaGetLastError();
}

#define NA_TRY(call, what)                                                      \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess)                                                      \
      return na_fail(PHYLO_ECUDA, "%s: %s", what, cudaGetErrorString(e_));      \
  } while (0)

}  // namespace

extern "C" {

int phylo_evaluate_noalloc(int N, int C, int S, int R, const int32_t* parent,
                           const uint8_t* tip_states, const double* pattern_weights,
                           const double* V, const double* Vinv, const double* lambda,
                           const double* root_freqs, const double* rates,
                           const double* cat_weights, const double* branch_lengths,
                           double* log_likelihood, double* gradient, void* stream,
                           char* error_message, size_t error_capacity) {
  t_err_buf = error_message;
  t_err_cap = error_capacity;
  if (error_message && error_capacity) error_message[0] = '\0';
  // ---- sizes (host only, before any CUDA call) ----
  if (N < 2 || N > kMaxNoAllocTips)
    return na_fail(PHYLO_EINVAL, "n_tips must be in [2, %d] for the no-allocation entry point",
                   kMaxNoAllocTips);
  if (C < 0 || C > (1 << 24)) return na_fail(PHYLO_EINVAL, "n_patterns out of range");
  if (S < 2 || S > 64) return na_fail(PHYLO_EINVAL, "n_states must be in [2, 64]");
  if (R < 1 || R > 8) return na_fail(PHYLO_EINVAL, "n_categories must be in [1, 8]");
  NaLayout L;
  na_layout(N, C, S, R, &L);
  if (L.total > kNoAllocScratchBytes)
    return na_fail(PHYLO_EINVAL,
                   "problem needs %zu bytes of scratch; the no-allocation entry point "
                   "has %zu (use phylo_create with a workspace)",
                   L.total, kNoAllocScratchBytes);
  if (!parent || !pattern_weights || !V || !Vinv || !lambda || !root_freqs || !rates ||
      !cat_weights || !branch_lengths || !log_likelihood || (!tip_states && C))
    return na_fail(PHYLO_EINVAL, "NULL argument");
  // ---- inputs (host only) ----
  const int n = 2 * N - 1, root = n - 1;
  if (parent[root] != -1) return na_fail(PHYLO_EINVAL, "parent[%d] (the root) must be -1", root);
  int2 ch[2 * kMaxNoAllocTips - 1];
  for (int v = 0; v < n; ++v) ch[v] = make_int2(-1, -1);
  for (int v = 0; v < root; ++v) {
    const int p = parent[v];
    if (p < N || p > root) return na_fail(PHYLO_EINVAL, "parent[%d] = %d is not internal", v, p);
    if (ch[p].x < 0) ch[p].x = v;
    else if (ch[p].y < 0) ch[p].y = v;
    else return na_fail(PHYLO_EINVAL, "node %d has more than two children", p);
  }
  for (int v = N; v < n; ++v)
    if (ch[v].y < 0) return na_fail(PHYLO_EINVAL, "node %d has fewer than two children", v);
  int depth[2 * kMaxNoAllocTips - 1], height[2 * kMaxNoAllocTips - 1];
  for (int v = 0; v < n; ++v) { depth[v] = -1; height[v] = 0; }
  depth[root] = 0;
  int max_depth = 0;
  for (int v = 0; v < n; ++v) {  // walk up to a node of known depth
    int u = v, steps = 0;
    while (depth[u] < 0) {
      u = parent[u];
      if (++steps > n) return na_fail(PHYLO_EINVAL, "the parent array has a cycle");
    }
    int d = depth[u] + steps;
    for (u = v; depth[u] < 0; u = parent[u]) depth[u] = d--;
    if (depth[v] > max_depth) max_depth = depth[v];
  }
  for (int d = max_depth; d >= 0; --d)  // heights, deepest nodes first
    for (int v = N; v < n; ++v)
      if (depth[v] == d) {
        const int a = height[ch[v].x], b = height[ch[v].y];
        height[v] = 1 + (a > b ? a : b);
      }
  int post_nodes[kMaxNoAllocTips], post_off[kMaxNoAllocTips + 1];
  int pre_nodes[kMaxNoAllocTips], pre_off[kMaxNoAllocTips + 1];
  int n_post = 0, n_pre = 0, k = 0;
  post_off[0] = 0;
  for (int h = 1; h <= height[root]; ++h) {
    for (int v = N; v < n; ++v)
      if (height[v] == h) post_nodes[k++] = v;
    post_off[++n_post] = k;
  }
  k = 0;
  pre_off[0] = 0;
  for (int d = 0; d <= max_depth; ++d) {
    const int before = k;
    for (int v = N; v < n; ++v)
      if (depth[v] == d) pre_nodes[k++] = v;
    if (k > before) pre_off[++n_pre] = k;
  }
  for (size_t i = 0; i < (size_t)N * C; ++i)
    if (tip_states[i] > S) return na_fail(PHYLO_EINVAL, "tip state %d > n_states", (int)tip_states[i]);
  for (int c = 0; c < C; ++c)
    if (!(pattern_weights[c] >= 0.0) || !std::isfinite(pattern_weights[c]))
      return na_fail(PHYLO_EINVAL, "pattern weight %d must be finite and >= 0", c);
  double wsum = 0.0;
  for (int r = 0; r < R; ++r) {
    if (!(rates[r] >= 0.0) || !std::isfinite(rates[r]) || !(cat_weights[r] >= 0.0) ||
        !std::isfinite(cat_weights[r]))
      return na_fail(PHYLO_EINVAL, "category %d: rate and weight must be finite and >= 0", r);
    wsum += cat_weights[r];
  }
  if (std::fabs(wsum - 1.0) > 1e-10) return na_fail(PHYLO_EINVAL, "category weights must sum to 1");
  for (int b = 0; b < 2 * N - 2; ++b)
    if (!(branch_lengths[b] >= 0.0) || !std::isfinite(branch_lengths[b]))
      return na_fail(PHYLO_EINVAL, "branch length %d must be finite and >= 0", b);
  for (int i = 0; i < S; ++i)
    for (int j = 0; j < S; ++j) {
      double acc = 0.0;
      for (int m = 0; m < S; ++m) acc += V[i * S + m] * Vinv[m * S + j];
      if (!std::isfinite(acc) || std::fabs(acc - (i == j ? 1.0 : 0.0)) > 1e-8)
        return na_fail(PHYLO_EINVAL, "V * Vinv differs from I at (%d,%d)", i, j);
    }

  // ---- device work: one call at a time per process ----
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  void* base = nullptr;
  int rc = scratch_for_current_device(&base);
  if (rc) return rc;
  char* ws = static_cast<char*>(base);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // Declared after the lock, so it runs before the lock is released: once
  // work is queued on the stream, every return path (the error returns of
  // NA_TRY included) waits for that work, so no queued copy or kernel still
  // touches the shared array when the next call takes the lock.
  struct DrainOnExit {
    cudaStream_t st;
    ~DrainOnExit() { (void)cudaStreamSynchronize(st); }
  } drain{st};
  auto up = [&](const NaRegion& r, const void* src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(ws + r.off, src, bytes, cudaMemcpyHostToDevice, st)
                 : cudaSuccess;
  };
  NA_TRY(up(L.children, ch, n * sizeof(int2)), "upload tree");
  NA_TRY(up(L.post_nodes, post_nodes, (size_t)post_off[n_post] * sizeof(int)), "upload schedule");
  NA_TRY(up(L.pre_nodes, pre_nodes, (size_t)pre_off[n_pre] * sizeof(int)), "upload schedule");
  {  // level-node descriptors {k, child 0, child 1, flags}; every tip is compact
    int4 desc[kMaxNoAllocTips];
    for (int pass = 0; pass < 2; ++pass) {
      const int* nodes = pass == 0 ? post_nodes : pre_nodes;
      const int count = pass == 0 ? post_off[n_post] : pre_off[n_pre];
      for (int i = 0; i < count; ++i) {
        const int2 c2 = ch[nodes[i]];
        desc[i] = make_int4(nodes[i], c2.x, c2.y,
                            (c2.x < N ? kDescFlagCompact0 : 0) | (c2.y < N ? kDescFlagCompact1 : 0));
      }
      NA_TRY(up(pass == 0 ? L.post_desc : L.pre_desc, desc, (size_t)count * sizeof(int4)),
             "upload descriptors");
      // the host array is reused: finish this copy first
      NA_TRY(cudaStreamSynchronize(st), "cudaStreamSynchronize");
    }
  }
  if (C)
    NA_TRY(cudaMemcpy2DAsync(ws + L.tip_states.off, tip_state_stride(C), tip_states, C, C, N,
                             cudaMemcpyHostToDevice, st),
           "upload tip states");
  NA_TRY(up(L.pattern_w, pattern_weights, (size_t)C * 8), "upload weights");
  NA_TRY(up(L.V, V, (size_t)S * S * 8), "upload V");
  NA_TRY(up(L.Vinv, Vinv, (size_t)S * S * 8), "upload Vinv");
  // static storage, not an allocation; the copy completes before this call
  // returns (the stream is synchronised below)
  static thread_local float vsplit[kEigenSplitFloats];
  bool reversible = false;
  if (L.vsplit.bytes) {
    reversible = build_eigen_split(S, L.SP, V, Vinv, root_freqs, vsplit);
    NA_TRY(up(L.vsplit, vsplit, eigen_split_floats(L.SP) * sizeof(float)), "upload V split");
  }
  static thread_local float qmat[20 * 20];
  if (L.qmat.bytes) {
    build_q_matrix(S, L.SP, V, Vinv, lambda, qmat);
    NA_TRY(up(L.qmat, qmat, L.qmat.bytes), "upload Q");
  }
  static thread_local unsigned char qt[kTcQtBytes];
  if (L.qt.bytes) {
    build_qt_tile(S, L.SP, V, Vinv, lambda, qt);
    NA_TRY(up(L.qt, qt, kTcQtBytes), "upload Q operand");
  }
  NA_TRY(up(L.lambda, lambda, (size_t)S * 8), "upload lambda");
  NA_TRY(up(L.pi, root_freqs, (size_t)S * 8), "upload pi");
  NA_TRY(up(L.rates, rates, (size_t)R * 8), "upload rates");
  NA_TRY(up(L.cat_w, cat_weights, (size_t)R * 8), "upload weights");
  NA_TRY(up(L.t, branch_lengths, (2 * (size_t)N - 2) * 8), "upload branch lengths");
  // FP32 copies of the weights, converted on the GPU (no host buffer)
  NA_TRY(launch_to_float(reinterpret_cast<const double*>(ws + L.pattern_w.off),
                         reinterpret_cast<float*>(ws + L.pattern_wt.off), C, st),
         "convert weights");
  NA_TRY(launch_to_float(reinterpret_cast<const double*>(ws + L.cat_w.off),
                         reinterpret_cast<float*>(ws + L.cat_wt.off), R, st),
         "convert weights");
  NA_TRY(launch_to_float(reinterpret_cast<const double*>(ws + L.pi.off),
                         reinterpret_cast<float*>(ws + L.pi_t.off), S, st),
         "convert pi");
  // The scratch keeps the previous call's contents: the flag word is the
  // only location read before this call writes it.
  int* flag = reinterpret_cast<int*>(ws + L.out.off + (2 * (size_t)N - 1) * 8);
  NA_TRY(cudaMemsetAsync(flag, 0, sizeof(int), st), "clear flags");

  PmatArgs pa{};
  pa.vsplit = L.vsplit.bytes ? reinterpret_cast<const float*>(ws + L.vsplit.off) : nullptr;
  pa.reversible = reversible;
  pa.V = reinterpret_cast<const double*>(ws + L.V.off);
  pa.Vinv = reinterpret_cast<const double*>(ws + L.Vinv.off);
  pa.lambda = reinterpret_cast<const double*>(ws + L.lambda.off);
  pa.rates = reinterpret_cast<const double*>(ws + L.rates.off);
  pa.t = reinterpret_cast<const double*>(ws + L.t.off);
  pa.n_branches = 2 * N - 2;
  pa.n_states = S;
  pa.n_cat = R;
  pa.P = ws + L.P.off;
  pa.dP = ws + L.dP.off;
  pa.err = flag;
  NA_TRY(launch_pmat<float>(pa, L.SP, st), "matrix build");
  LevelArgs<float> a{};
  a.children = reinterpret_cast<const int2*>(ws + L.children.off);
  a.n_tips = N;
  a.n_patterns = C;
  a.n_states = S;
  a.n_cat = R;
  a.root = root;
  a.P = reinterpret_cast<const float*>(ws + L.P.off);
  a.dP = L.dP.bytes ? reinterpret_cast<const float*>(ws + L.dP.off) : nullptr;
  a.post = reinterpret_cast<float*>(ws + L.post.off);
  a.pre = reinterpret_cast<float*>(ws + L.pre.off);
  a.escale = reinterpret_cast<int*>(ws + L.escale.off);
  a.pre_escale = L.pre_escale.bytes ? reinterpret_cast<int*>(ws + L.pre_escale.off) : nullptr;
  a.rterm = L.rterm.bytes ? static_cast<void*>(ws + L.rterm.off) : nullptr;
  a.tip_states = reinterpret_cast<const uint8_t*>(ws + L.tip_states.off);
  a.state_stride = tip_state_stride(C);
  a.escale_stride = round_up(C, 4);
  a.tip_partials = nullptr;
  a.tip_has_partials = nullptr;
  a.pattern_w = reinterpret_cast<const double*>(ws + L.pattern_w.off);
  a.root_pi = reinterpret_cast<const double*>(ws + L.pi.off);
  a.cat_w = reinterpret_cast<const double*>(ws + L.cat_w.off);
  a.pattern_wt = reinterpret_cast<const float*>(ws + L.pattern_wt.off);
  a.cat_wt = reinterpret_cast<const float*>(ws + L.cat_wt.off);
  a.root_pit = reinterpret_cast<const float*>(ws + L.pi_t.off);
  a.gpart = reinterpret_cast<double*>(ws + L.gpart.off);
  a.lpart = reinterpret_cast<double*>(ws + L.lpart.off);
  a.n_tiles = L.n_tiles;
  a.err = flag;
  a.qt = L.qt.bytes ? reinterpret_cast<const unsigned char*>(ws + L.qt.off) : nullptr;
  a.qmat = L.qmat.bytes ? reinterpret_cast<const float*>(ws + L.qmat.off) : nullptr;
  a.rates = reinterpret_cast<const double*>(ws + L.rates.off);
  a.tip_level = 0;
  const int* dpost = reinterpret_cast<const int*>(ws + L.post_nodes.off);
  const int* dpre = reinterpret_cast<const int*>(ws + L.pre_nodes.off);
  const int4* dpostd = reinterpret_cast<const int4*>(ws + L.post_desc.off);
  const int4* dpred = reinterpret_cast<const int4*>(ws + L.pre_desc.off);
  for (int l = 0; l < n_post; ++l) {
    a.level_nodes = dpost + post_off[l];
    a.level_desc = dpostd + post_off[l];
    a.n_level = post_off[l + 1] - post_off[l];
    a.root_level = l + 1 == n_post;  // the last post level is the root alone
    NA_TRY(launch_post_level<float>(a, L.SP, L.RP, st), "post-order level");
  }
  a.root_level = 0;
  for (int l = 0; l < n_pre; ++l) {
    a.level_nodes = dpre + pre_off[l];
    a.level_desc = dpred + pre_off[l];
    a.n_level = pre_off[l + 1] - pre_off[l];
    NA_TRY(launch_pre_level<float>(a, L.SP, L.RP, st), "pre-order level");
  }
  if (C > 0) NA_TRY(launch_pre_finish<float>(a, L.SP, st), "gradient ratios");
  ReduceArgs ra{};
  ra.gpart = a.gpart;
  ra.lpart = a.lpart;
  ra.gpart_pairs = L.SP == 4 || L.SP == 20;  // FP32 4- and 20-state kernels
  ra.n_tiles = L.n_tiles;
  ra.n_branches = 2 * N - 2;
  ra.out = reinterpret_cast<double*>(ws + L.out.off);
  NA_TRY(launch_reduce(ra, st), "reduction");
  double host_out[2 * kMaxNoAllocTips];  // [logL, grad..., flag word]
  NA_TRY(cudaMemcpyAsync(host_out, ws + L.out.off, (2 * (size_t)N - 1) * 8 + 8,
                         cudaMemcpyDeviceToHost, st),
         "download results");
  NA_TRY(cudaStreamSynchronize(st), "cudaStreamSynchronize");
  int flags;
  std::memcpy(&flags, host_out + 2 * N - 1, sizeof(int));
  if (flags)
    return na_fail(PHYLO_ENUMERIC, "device flagged a zero partial, a bad length or a zero ratio");
  *log_likelihood = host_out[0];
  if (gradient) std::memcpy(gradient, host_out + 1, (2 * (size_t)N - 2) * 8);
  return PHYLO_OK;
}

}  // extern "C"
