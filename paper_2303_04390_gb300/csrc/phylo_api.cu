// Host side of libphylograd: input validation, the level schedule, the
// workspace layout, the host FP64 eigendecomposition and the CUDA-graph
// launch of one evaluation.  The C ABI is declared in include/phylo_api.h.
//
// One evaluation (arXiv 2303.04390, Eqs. 1-8) is the fixed launch sequence
//   memset(flags) -> pmat (Eq. 1, every branch and category)
//   -> post-order levels 1..H (Eq. 2; Eq. 3 at the root)
//   -> pre-order levels 0..D (Eq. 4 with the Eq. 8 ratio fused)
//   -> final FP64 reduction over pattern tiles (Eq. 7)
// captured once per tree into a CUDA graph and replayed on the caller's
// stream.  The paper instead launches one kernel per node (post-order and
// pre-order) plus separate gradient and site-reduction kernels.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/phylo_api.h"
#include "phylo_internal.h"
#include "tma.cuh"

using namespace phylo;

namespace {

constexpr size_t kAlign = 256;

struct Region {
  size_t off = 0, bytes = 0;
};

// Workspace layout of one context (all offsets 256-byte aligned).
struct Layout {
  int SP = 0, RP = 0, n_tiles = 0;
  size_t elem = 0;
  Region children, post_nodes, pre_nodes, post_desc, pre_desc;
  Region P, dP, post, pre, escale, pre_escale, rterm;
  Region tip_states, tip_partials, tip_has;
  Region pattern_w, V, Vinv, lambda, pi, rates, cat_w, t;
  Region vsplit;  // tensor-core path: eigenvectors as double-float tables
  Region tc_tiles;  // 65..128 states, FP32: pre-split matrix blocks
  Region qt;        // 21..128 states, FP32: Q' as a tensor-core operand
  Region qmat;      // 4 and 20 padded states, FP32: Q row-major
  Region tip_desc;  // U-form paths with tip partials: descriptors of the tips
                    // whose U = P p the first post-order launch forms
  Region pattern_wt, cat_wt, pi_t;  // weights and pi in the path's type
  Region gpart, lpart, out;  // out = [logL, grad...] followed by the flag word
  Region chain_a, chain_b, chain_out, chain_idx;  // chain-rule epilogue staging
  size_t total = 0;
};

bool mul_ok(size_t a, size_t b, size_t* out) {
  return !__builtin_mul_overflow(a, b, out);
}

bool add_region(Layout& L, Region& r, size_t bytes) {
  size_t off = (L.total + kAlign - 1) / kAlign * kAlign;
  if (off < L.total) return false;
  r.off = off;
  r.bytes = bytes;
  if (__builtin_add_overflow(off, bytes, &L.total)) return false;
  return true;
}

// Returns an error message or nullptr.
const char* compute_layout(int N, int C, int S, int R, int prec, int flags,
                           Layout* Lp) {
  if (N < 2 || N > 65536) return "n_tips must be in [2, 65536]";
  if (C < 0) return "n_patterns must be >= 0";
  if (S < 2 || S > kMaxStates) return "n_states must be in [2, 256]";
  if (R < 1 || R > 8) return "n_categories must be in [1, 8]";
  if (prec != PHYLO_FP64 && prec != PHYLO_FP32) return "unknown precision";
  if (flags & ~(PHYLO_FLAG_TIP_PARTIALS | PHYLO_FLAG_NO_GRAPH)) return "unknown flags";
  Layout L;
  L.SP = padded_states(S);
  L.RP = lanes_per_pattern(R);
  L.elem = prec == PHYLO_FP64 ? 8 : 4;
  const int ct = patterns_per_tile(L.SP, R, prec == PHYLO_FP64);
  L.n_tiles = (C + ct - 1) / ct;
  const size_t n_nodes = 2 * (size_t)N - 1, n_br = 2 * (size_t)N - 2;
  const size_t n_int = (size_t)N - 1;
  size_t mat, part, tmp, tmp2;
  const bool tc = uses_tensor_cores(L.SP, prec == PHYLO_FP64);
  const bool p4 = uses_tr_layout(L.SP, prec == PHYLO_FP64);
  const size_t unit = tc ? kTcUnitBytes
                         : (size_t)L.SP * L.SP * L.elem * (p4 ? kP4MatKinds : 1);
  if (!mul_ok(n_br * R, unit, &mat)) return "size overflow";
  if (C > (1 << 30)) return "n_patterns too large";
  const size_t per_node = partial_elems_per_node(L.SP, prec == PHYLO_FP64, C, R, L.n_tiles);
  if (!mul_ok(n_int, per_node, &tmp) || !mul_ok(tmp, L.elem, &part)) return "size overflow";
  bool ok = true;
  ok &= add_region(L, L.children, n_nodes * sizeof(int2));
  ok &= add_region(L, L.post_nodes, n_int * sizeof(int));
  ok &= add_region(L, L.pre_nodes, n_int * sizeof(int));
  ok &= add_region(L, L.post_desc, n_int * sizeof(int4));
  ok &= add_region(L, L.pre_desc, n_int * sizeof(int4));
  ok &= add_region(L, L.P, mat);
  ok &= add_region(L, L.dP, tc || p4 ? 0 : mat);  // else the P region holds dP
  if (uses_tc_big(L.SP, prec == PHYLO_FP64)) {
    // the matrix kernel writes the operand blocks instead of P and dP
    L.P.bytes = L.dP.bytes = 0;
    L.total = L.P.off;
    if (!mul_ok(n_br * R, kTcbUnitBytes, &tmp)) return "size overflow";
    ok &= add_region(L, L.tc_tiles, tmp);
  }
  const bool uform = uses_u_form(L.SP, prec == PHYLO_FP64);
  if (uform && (flags & PHYLO_FLAG_TIP_PARTIALS)) {
    // the post region holds U = P p of every internal node, then of every tip
    if (!mul_ok(n_int + N, per_node, &tmp) || !mul_ok(tmp, L.elem, &tmp2))
      return "size overflow";
    ok &= add_region(L, L.post, tmp2);
    ok &= add_region(L, L.tip_desc, (size_t)N * sizeof(int4));
  } else {
    ok &= add_region(L, L.post, part);
  }
  ok &= add_region(L, L.pre, part);
  if (tc || uses_tc_big(L.SP, prec == PHYLO_FP64)) ok &= add_region(L, L.qt, qt_bytes(L.SP));
  if (prec == PHYLO_FP32 && (L.SP == 4 || L.SP == 20))  // the U form's Q (FP32, row-major)
    ok &= add_region(L, L.qmat, (size_t)L.SP * L.SP * sizeof(float));
  if (C > (1 << 30)) return "n_patterns too large";
  const int planes = escale_planes(L.SP, R, prec == PHYLO_FP64);
  if (!mul_ok(n_int * planes, (size_t)round_up(C, 4) * sizeof(int), &tmp))
    return "size overflow";
  ok &= add_region(L, L.escale, tmp);
  if (uses_tc_terms(L.SP, prec == PHYLO_FP64)) {
    ok &= add_region(L, L.pre_escale, tmp);
    if (!mul_ok(n_int * C, (size_t)R * 16, &tmp)) return "size overflow";
    ok &= add_region(L, L.rterm, tmp);
  }
  if (!mul_ok((size_t)N, (size_t)tip_state_stride(C), &tmp)) return "size overflow";
  ok &= add_region(L, L.tip_states, tmp);
  if (!mul_ok((size_t)N, (size_t)C, &tmp)) return "size overflow";
  if (flags & PHYLO_FLAG_TIP_PARTIALS) {
    if (!mul_ok(tmp, (size_t)L.SP * L.elem, &tmp2)) return "size overflow";
    ok &= add_region(L, L.tip_partials, tmp2);
    ok &= add_region(L, L.tip_has, (size_t)N * sizeof(int));
  }
  ok &= add_region(L, L.pattern_w, (size_t)C * 8);
  ok &= add_region(L, L.V, (size_t)S * S * 8);
  ok &= add_region(L, L.Vinv, (size_t)S * S * 8);
  if (uses_eigen_split(L.SP, prec == PHYLO_FP64))
    ok &= add_region(L, L.vsplit, eigen_split_floats(L.SP) * sizeof(float));
  ok &= add_region(L, L.lambda, (size_t)S * 8);
  ok &= add_region(L, L.pi, (size_t)S * 8);
  ok &= add_region(L, L.rates, (size_t)R * 8);
  ok &= add_region(L, L.cat_w, (size_t)R * 8);
  ok &= add_region(L, L.pattern_wt, (size_t)C * L.elem);
  ok &= add_region(L, L.cat_wt, (size_t)R * L.elem);
  ok &= add_region(L, L.pi_t, (size_t)S * L.elem);
  ok &= add_region(L, L.t, n_br * 8);
  if (!mul_ok(n_br, (size_t)L.n_tiles * 8, &tmp)) return "size overflow";
  ok &= add_region(L, L.gpart, tmp);
  ok &= add_region(L, L.lpart, (size_t)L.n_tiles * 8);
  ok &= add_region(L, L.out, n_nodes * 8 + 8);
  ok &= add_region(L, L.chain_a, n_nodes * 8);
  ok &= add_region(L, L.chain_b, n_nodes * 8);
  ok &= add_region(L, L.chain_out, 2 * n_nodes * 8);
  ok &= add_region(L, L.chain_idx, n_br * sizeof(int));
  if (!ok) return "size overflow";
  *Lp = L;
  return nullptr;
}

thread_local std::string g_create_error;

}  // namespace

struct phylo_ctx {
  int N = 0, C = 0, S = 0, R = 0, precision = 0, flags = 0;
  Layout L;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraphExec_t phase_exec[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaGraphExec_t fwd_exec = nullptr;  // matrices + post-order + logL reduction
  cudaGraphExec_t bwd_exec = nullptr;  // pre-order + gradient reduction
  bool forward_valid = false;          // post-order partials match the inputs
  uint64_t partials_gen = 0;           // bumped by every launch that rewrites them
  bool have_grad = false;              // out holds the gradient of an evaluation
  bool eig_reversible = false;         // V, Vinv are the symmetric decomposition
  bool graph_dirty = true;
  bool phase_dirty = true;
  bool prepared = false;
  // schedule (host copies)
  std::vector<int2> children;
  std::vector<int> post_nodes, post_off;  // level l: [post_off[l], post_off[l+1])
  std::vector<int> pre_nodes, pre_off;
  std::vector<char> post_cherry, pre_cherry;  // per level: a node has a fused cherry child
  std::vector<int> height, depth;             // per node
  std::vector<char> cherry;                   // per node: fused into its parent
  std::vector<int> tip_has;
  bool have_tree = false, have_states = false, have_weights = false,
       have_eigen = false, have_cats = false, have_t = false;
  double* host_out = nullptr;  // pinned [2N-1] + flag word
  std::string err;

  template <typename T>
  T* dev(const Region& r) const {
    return reinterpret_cast<T*>(ws + r.off);
  }
};

namespace {

int fail(phylo_ctx* ctx, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (ctx) ctx->err = buf; else g_create_error = buf;
  return code;
}

int cuda_fail(phylo_ctx* ctx, cudaError_t e, const char* what) {
  return fail(ctx, PHYLO_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e),
              cudaGetErrorString(e));
}

// NVTX range with an integer payload (a level index); visible to profilers
// for direct launches and for graph launches (the range spans the launch).
struct NvtxRange {
  NvtxRange(const char* name, int payload = -1) {
    nvtxEventAttributes_t a{};
    a.version = NVTX_VERSION;
    a.size = NVTX_EVENT_ATTRIB_STRUCT_SIZE;
    a.messageType = NVTX_MESSAGE_TYPE_ASCII;
    a.message.ascii = name;
    if (payload >= 0) {
      a.payloadType = NVTX_PAYLOAD_TYPE_INT32;
      a.payload.iValue = payload;
    }
    nvtxRangePushEx(&a);
  }
  ~NvtxRange() { nvtxRangePop(); }
};

#define CUDA_TRY(ctx, call, what)                       \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
  } while (0)

void invalidate_graph(phylo_ctx* ctx) {
  if (ctx->gexec) {
    cudaGraphExecDestroy(ctx->gexec);
    ctx->gexec = nullptr;
  }
  for (auto& g : ctx->phase_exec) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
  }
  if (ctx->fwd_exec) cudaGraphExecDestroy(ctx->fwd_exec);
  if (ctx->bwd_exec) cudaGraphExecDestroy(ctx->bwd_exec);
  ctx->fwd_exec = ctx->bwd_exec = nullptr;
  ctx->graph_dirty = true;
  ctx->phase_dirty = true;
  ctx->forward_valid = false;
}

template <typename T>
LevelArgs<T> level_args(const phylo_ctx* ctx) {
  LevelArgs<T> a{};
  a.children = ctx->dev<int2>(ctx->L.children);
  a.n_tips = ctx->N;
  a.n_patterns = ctx->C;
  a.n_states = ctx->S;
  a.n_cat = ctx->R;
  a.root = 2 * ctx->N - 2;
  a.P = ctx->dev<T>(ctx->L.P);
  a.dP = ctx->L.dP.bytes ? ctx->dev<T>(ctx->L.dP) : nullptr;
  a.post = ctx->dev<T>(ctx->L.post);
  a.pre = ctx->dev<T>(ctx->L.pre);
  a.escale = ctx->dev<int>(ctx->L.escale);
  a.pre_escale = ctx->L.pre_escale.bytes ? ctx->dev<int>(ctx->L.pre_escale) : nullptr;
  a.rterm = ctx->L.rterm.bytes ? ctx->dev<void>(ctx->L.rterm) : nullptr;
  a.tip_states = ctx->dev<uint8_t>(ctx->L.tip_states);
  a.state_stride = tip_state_stride(ctx->C);
  a.escale_stride = round_up(ctx->C, 4);
  bool any_partials = false;
  for (int v : ctx->tip_has) any_partials |= v != 0;
  a.tip_partials = any_partials ? ctx->dev<T>(ctx->L.tip_partials) : nullptr;
  a.tip_has_partials = any_partials ? ctx->dev<int>(ctx->L.tip_has) : nullptr;
  a.pattern_w = ctx->dev<double>(ctx->L.pattern_w);
  a.root_pi = ctx->dev<double>(ctx->L.pi);
  a.cat_w = ctx->dev<double>(ctx->L.cat_w);
  a.pattern_wt = ctx->dev<T>(ctx->L.pattern_wt);
  a.cat_wt = ctx->dev<T>(ctx->L.cat_wt);
  a.root_pit = ctx->dev<T>(ctx->L.pi_t);
  a.gpart = ctx->dev<double>(ctx->L.gpart);
  a.lpart = ctx->dev<double>(ctx->L.lpart);
  a.n_tiles = ctx->L.n_tiles;
  a.err = reinterpret_cast<int*>(ctx->dev<double>(ctx->L.out) + 2 * ctx->N - 1);
  a.tc_tiles = ctx->L.tc_tiles.bytes ? ctx->dev<unsigned char>(ctx->L.tc_tiles) : nullptr;
  a.qt = ctx->L.qt.bytes ? ctx->dev<unsigned char>(ctx->L.qt) : nullptr;
  a.qmat = ctx->L.qmat.bytes ? ctx->dev<float>(ctx->L.qmat) : nullptr;
  a.rates = ctx->dev<double>(ctx->L.rates);
  a.tip_level = 0;
  return a;
}

// Whether the post-order phase starts with a launch over the tips with
// partial vectors (the U-form paths form those tips' U first).
bool has_tip_level(const phylo_ctx* ctx) {
  if (!ctx->L.tip_desc.bytes) return false;
  for (int v : ctx->tip_has)
    if (v) return true;
  return false;
}

int* flag_word(const phylo_ctx* ctx) {
  return reinterpret_cast<int*>(ctx->dev<double>(ctx->L.out) + 2 * ctx->N - 1);
}

// Phases of one evaluation: 0 = flag reset + matrices (Eq. 1), 1 = post-order
// levels (Eqs. 2-3), 2 = pre-order levels with the gradient (Eqs. 4, 8),
// 3 = final reduction (Eq. 7).  Phase 4 (not part of an evaluation) is the
// log-likelihood reduction alone, which ends the forward pass.
constexpr int kPhases = 4;
constexpr int kPhaseLogLOnly = 4;

template <typename T>
cudaError_t enqueue_phase(phylo_ctx* ctx, int phase, cudaStream_t st) {
  cudaError_t e = cudaSuccess;
  if (phase == 0) {
    NvtxRange range("phylo matrices (Eq. 1)");
    e = cudaMemsetAsync(flag_word(ctx), 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    PmatArgs pa{};
    pa.vsplit = ctx->L.vsplit.bytes ? ctx->dev<float>(ctx->L.vsplit) : nullptr;
    pa.reversible = ctx->eig_reversible;
    pa.V = ctx->dev<double>(ctx->L.V);
    pa.Vinv = ctx->dev<double>(ctx->L.Vinv);
    pa.lambda = ctx->dev<double>(ctx->L.lambda);
    pa.rates = ctx->dev<double>(ctx->L.rates);
    pa.t = ctx->dev<double>(ctx->L.t);
    pa.n_branches = 2 * ctx->N - 2;
    pa.n_states = ctx->S;
    pa.n_cat = ctx->R;
    pa.P = ctx->dev<T>(ctx->L.P);
    pa.dP = ctx->dev<T>(ctx->L.dP);
    pa.tiles = ctx->L.tc_tiles.bytes ? ctx->dev<void>(ctx->L.tc_tiles) : nullptr;
    pa.err = flag_word(ctx);
    return launch_pmat<T>(pa, ctx->L.SP, st);
  }
  if (phase == 1 || phase == 2) {
    LevelArgs<T> a = level_args<T>(ctx);
    const bool post = phase == 1;
    const int* nodes = ctx->dev<int>(post ? ctx->L.post_nodes : ctx->L.pre_nodes);
    const int4* desc = ctx->dev<int4>(post ? ctx->L.post_desc : ctx->L.pre_desc);
    const std::vector<int>& off = post ? ctx->post_off : ctx->pre_off;
    if (post && ctx->L.tip_desc.bytes && a.tip_partials) {
      // U-form paths: U = P p of the tips with partials, before level 1
      NvtxRange range("phylo post-order tips with partials (Eq. 2)");
      LevelArgs<T> at = a;
      at.level_desc = ctx->dev<int4>(ctx->L.tip_desc);
      at.level_nodes = nullptr;
      at.n_level = 0;
      for (int v : ctx->tip_has) at.n_level += v != 0;
      at.root_level = 0;
      at.level_cherry = 0;
      at.tip_level = 1;
      at.mats_ready = 0;  // directly after the matrix kernel
      e = launch_post_level<T>(at, ctx->L.SP, ctx->L.RP, st);
      if (e != cudaSuccess) return e;
    }
    // P may be staged before the wait on the previous launch unless that
    // launch is the matrix kernel itself (the first post-order launch).
    bool after_pmat = post && !(ctx->L.tip_desc.bytes && a.tip_partials);
    for (size_t l = 0; l + 1 < off.size(); ++l) {
      NvtxRange range(post ? "phylo post-order level (Eq. 2)"
                           : "phylo pre-order level (Eqs. 4, 8)", (int)l);
      a.mats_ready = after_pmat ? 0 : 1;
      after_pmat = false;
      a.level_nodes = nodes + off[l];
      a.level_desc = desc + off[l];
      a.n_level = off[l + 1] - off[l];
      a.root_level = post && l + 2 == off.size();  // the last post level is the root
      a.level_cherry = (post ? ctx->post_cherry : ctx->pre_cherry)[l];
      e = post ? launch_post_level<T>(a, ctx->L.SP, ctx->L.RP, st)
               : launch_pre_level<T>(a, ctx->L.SP, ctx->L.RP, st);
      if (e != cudaSuccess) return e;
    }
    if (!post && ctx->C > 0) return launch_pre_finish<T>(a, ctx->L.SP, st);
    return cudaSuccess;
  }
  NvtxRange range("phylo reduction (Eq. 7)");
  ReduceArgs ra{};
  ra.gpart = ctx->dev<double>(ctx->L.gpart);
  ra.lpart = ctx->dev<double>(ctx->L.lpart);
  ra.n_tiles = ctx->L.n_tiles;
  ra.n_branches = phase == kPhaseLogLOnly ? 0 : 2 * ctx->N - 2;
  ra.gpart_pairs = ctx->precision == PHYLO_FP32 && (ctx->L.SP == 4 || ctx->L.SP == 20);
  ra.out = ctx->dev<double>(ctx->L.out);
  return launch_reduce(ra, st);
}

cudaError_t enqueue_phases(phylo_ctx* ctx, int first, int last, cudaStream_t st) {
  for (int ph = first; ph <= last; ++ph) {
    if (ph == kPhases) continue;  // (no phase between the reduction forms)
    cudaError_t e = ctx->precision == PHYLO_FP64 ? enqueue_phase<double>(ctx, ph, st)
                                                 : enqueue_phase<float>(ctx, ph, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int ensure_cuda_objects(phylo_ctx* ctx) {
  if (!ctx->prepared) {
    cudaError_t e = ctx->precision == PHYLO_FP64
                        ? prepare_kernels<double>(ctx->L.SP, ctx->L.RP)
                        : prepare_kernels<float>(ctx->L.SP, ctx->L.RP);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel attributes");
    ctx->prepared = true;
  }
  return PHYLO_OK;
}

// The private stream that CUDA graphs are captured on (created on first
// capture; a context that never captures never creates it).
int ensure_capture_stream(phylo_ctx* ctx) {
  if (!ctx->cap_stream)
    CUDA_TRY(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking),
             "cudaStreamCreate");
  return PHYLO_OK;
}

// Pinned staging for results read back to the host (first host read-back).
int ensure_host_out(phylo_ctx* ctx) {
  if (!ctx->host_out) {
    void* p = nullptr;
    CUDA_TRY(ctx, cudaHostAlloc(&p, (2 * (size_t)ctx->N - 1) * 8 + 8, cudaHostAllocDefault),
             "cudaHostAlloc");
    ctx->host_out = static_cast<double*>(p);
  }
  return PHYLO_OK;
}

// Capture phases [first, last] into an executable graph.
int capture(phylo_ctx* ctx, int first, int last, cudaGraphExec_t* exec) {
  int rc = ensure_capture_stream(ctx);
  if (rc) return rc;
  CUDA_TRY(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal),
           "cudaStreamBeginCapture");
  cudaError_t le = enqueue_phases(ctx, first, last, ctx->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t ce = cudaStreamEndCapture(ctx->cap_stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(ctx, le, "kernel launch during capture");
  }
  if (ce != cudaSuccess) return cuda_fail(ctx, ce, "cudaStreamEndCapture");
  cudaError_t ie = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    *exec = nullptr;
    return cuda_fail(ctx, ie, "cudaGraphInstantiate");
  }
  return PHYLO_OK;
}

template <typename T>
int upload(phylo_ctx* ctx, const Region& r, const T* host, size_t count,
           const char* what);

// Level-node descriptors {k, child 0, child 1, flags} for both passes; the
// flags depend on which tips carry partial vectors.
// Level lists: post-order by height, pre-order by depth, one launch per
// non-empty level.  On the FP32 4-state path a cherry (a non-root node
// whose children are both tips with compact states) is fused into its
// parent's post-order launch (kernels_p4.cuh) and gets no post-order level
// entry of its own.
int build_schedule(phylo_ctx* ctx) {
  const int N = ctx->N, n = 2 * N - 1, root = n - 1;
  const bool fuse = ctx->precision == PHYLO_FP32 && ctx->L.SP == 4;
  const std::vector<int2>& ch = ctx->children;
  ctx->cherry.assign(n, 0);
  if (fuse)
    for (int v = N; v < root; ++v)
      ctx->cherry[v] = ch[v].x < N && ch[v].y < N && !ctx->tip_has[ch[v].x] &&
                       !ctx->tip_has[ch[v].y];
  auto has_cherry_child = [&](int v) {
    return (ch[v].x >= N && ctx->cherry[ch[v].x]) || (ch[v].y >= N && ctx->cherry[ch[v].y]);
  };
  int H = 0, D = 0;
  for (int v = N; v < n; ++v) {
    H = ctx->height[v] > H ? ctx->height[v] : H;
    D = ctx->depth[v] > D ? ctx->depth[v] : D;
  }
  std::vector<std::vector<int>> by_height(H + 1), by_depth(D + 1);
  for (int v = N; v < n; ++v) {
    if (!ctx->cherry[v]) by_height[ctx->height[v]].push_back(v);
    by_depth[ctx->depth[v]].push_back(v);
  }
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<int>& nodes = pass == 0 ? ctx->post_nodes : ctx->pre_nodes;
    std::vector<int>& off = pass == 0 ? ctx->post_off : ctx->pre_off;
    std::vector<char>& flag = pass == 0 ? ctx->post_cherry : ctx->pre_cherry;
    const std::vector<std::vector<int>>& lv = pass == 0 ? by_height : by_depth;
    nodes.clear();
    off.assign(1, 0);
    flag.clear();
    for (const std::vector<int>& level : lv) {
      if (level.empty()) continue;
      char any = 0;
      for (int v : level) {
        nodes.push_back(v);
        any |= has_cherry_child(v);
      }
      off.push_back((int)nodes.size());
      flag.push_back(any);
    }
  }
  int rc = upload(ctx, ctx->L.post_nodes, ctx->post_nodes.data(), ctx->post_nodes.size(),
                  "upload schedule");
  if (rc) return rc;
  rc = upload(ctx, ctx->L.pre_nodes, ctx->pre_nodes.data(), ctx->pre_nodes.size(),
              "upload schedule");
  if (rc) return rc;
  // the pageable uploads above must complete before the host vectors change
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  return PHYLO_OK;
}

int upload_descriptors(phylo_ctx* ctx) {
  if (ctx->L.tip_desc.bytes) {
    std::vector<int4> tips;
    for (int x = 0; x < ctx->N; ++x)
      if (ctx->tip_has[x]) tips.push_back(make_int4(x, -1, -1, 0));
    if (!tips.empty()) {
      int rc = upload(ctx, ctx->L.tip_desc, tips.data(), tips.size(), "upload tip descriptors");
      if (rc) return rc;
      CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    }
  }
  for (int pass = 0; pass < 2; ++pass) {
    const std::vector<int>& nodes = pass == 0 ? ctx->post_nodes : ctx->pre_nodes;
    std::vector<int4> desc(nodes.size());
    for (size_t i = 0; i < nodes.size(); ++i) {
      const int k = nodes[i];
      const int2 ch = ctx->children[k];
      int flags = 0;
      if (ch.x < ctx->N && !ctx->tip_has[ch.x]) flags |= kDescFlagCompact0;
      if (ch.y < ctx->N && !ctx->tip_has[ch.y]) flags |= kDescFlagCompact1;
      if (ch.x >= ctx->N && ctx->cherry[ch.x]) flags |= kDescFlagCherry0;
      if (ch.y >= ctx->N && ctx->cherry[ch.y]) flags |= kDescFlagCherry1;
      desc[i] = make_int4(k, ch.x, ch.y, flags);
    }
    if (!desc.empty()) {
      int rc = upload(ctx, pass == 0 ? ctx->L.post_desc : ctx->L.pre_desc, desc.data(),
                      desc.size(), "upload level descriptors");
      if (rc) return rc;
      CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    }
  }
  return PHYLO_OK;
}

// Run phases [first, last] on the context's stream: replayed from a cached
// graph, or launched directly when the context was created with
// PHYLO_FLAG_NO_GRAPH (one-shot contexts, where capture would cost more
// than it saves).
int run_phases(phylo_ctx* ctx, int first, int last, cudaGraphExec_t* cache) {
  int rc = ensure_cuda_objects(ctx);
  if (rc) return rc;
  if (ctx->graph_dirty || ctx->phase_dirty) {
    rc = upload_descriptors(ctx);
    if (rc) return rc;
  }
  if (ctx->flags & PHYLO_FLAG_NO_GRAPH) {
    cudaError_t e = enqueue_phases(ctx, first, last, ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "kernel launch");
    ctx->graph_dirty = ctx->phase_dirty = false;
    return PHYLO_OK;
  }
  if (!*cache) {
    rc = capture(ctx, first, last, cache);
    if (rc) return rc;
  }
  CUDA_TRY(ctx, cudaGraphLaunch(*cache, ctx->stream), "cudaGraphLaunch");
  return PHYLO_OK;
}

int build_graph(phylo_ctx* ctx) {
  int rc = ensure_cuda_objects(ctx);
  if (rc) return rc;
  rc = upload_descriptors(ctx);
  if (rc) return rc;
  invalidate_graph(ctx);
  rc = capture(ctx, 0, kPhases - 1, &ctx->gexec);
  if (rc) return rc;
  ctx->graph_dirty = false;
  return PHYLO_OK;
}

int build_phase_graphs(phylo_ctx* ctx) {
  int rc = ensure_cuda_objects(ctx);
  if (rc) return rc;
  rc = upload_descriptors(ctx);
  if (rc) return rc;
  for (int ph = 0; ph < kPhases; ++ph) {
    if (ctx->phase_exec[ph]) cudaGraphExecDestroy(ctx->phase_exec[ph]);
    ctx->phase_exec[ph] = nullptr;
  }
  for (int ph = 0; ph < kPhases; ++ph) {
    rc = capture(ctx, ph, ph, &ctx->phase_exec[ph]);
    if (rc) return rc;
  }
  ctx->phase_dirty = false;
  return PHYLO_OK;
}

int check_ready(phylo_ctx* ctx) {
  if (!ctx) return PHYLO_EINVAL;
  const char* missing = !ctx->have_tree      ? "tree"
                        : !ctx->have_states  ? "tip states"
                        : !ctx->have_weights ? "pattern weights"
                        : !ctx->have_eigen   ? "eigen-decomposition"
                        : !ctx->have_cats    ? "categories"
                        : !ctx->have_t       ? "branch lengths"
                                             : nullptr;
  if (missing) return fail(ctx, PHYLO_ESTATE, "%s not set", missing);
  return PHYLO_OK;
}

int launch_eval(phylo_ctx* ctx) {
  int rc = check_ready(ctx);
  if (rc) return rc;
  NvtxRange range("phylo evaluate");
  ++ctx->partials_gen;
  if (ctx->flags & PHYLO_FLAG_NO_GRAPH) {
    rc = run_phases(ctx, 0, kPhases - 1, nullptr);
    if (rc) return rc;
    ctx->forward_valid = true;
    ctx->have_grad = true;
    return PHYLO_OK;
  }
  if (ctx->graph_dirty || !ctx->gexec) {
    rc = build_graph(ctx);
    if (rc) return rc;
  }
  CUDA_TRY(ctx, cudaGraphLaunch(ctx->gexec, ctx->stream), "cudaGraphLaunch");
  ctx->forward_valid = true;
  ctx->have_grad = true;
  return PHYLO_OK;
}

int read_flags(phylo_ctx* ctx, int flags) {
  if (flags == 0) return PHYLO_OK;
  if (flags & ERR_TIMEOUT)
    return fail(ctx, PHYLO_ETIMEOUT, "device flagged: a bounded wait on an asynchronous copy expired");
  return fail(ctx, PHYLO_ENUMERIC,
              "device flagged:%s%s%s", (flags & ERR_ZERO_PARTIAL) ? " zero-or-nonfinite-partial" : "",
              (flags & ERR_BAD_LENGTH) ? " bad-branch-length" : "",
              (flags & ERR_BAD_RATIO) ? " zero-gradient-denominator" : "");
}

// Cyclic Jacobi eigen-decomposition of a symmetric matrix A (n x n, row
// major, overwritten): eigenvalues in w, eigenvectors as columns of U.
bool jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& U,
                  std::vector<double>& w) {
  U.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) U[(size_t)i * n + i] = 1.0;
  double fro = 0.0;
  for (double x : A) fro += x * x;
  fro = std::sqrt(fro);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += A[(size_t)p * n + q] * A[(size_t)p * n + q];
    if (std::sqrt(off) <= 1e-17 * fro || off == 0.0) {
      w.resize(n);
      for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
      return true;
    }
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double app = A[(size_t)p * n + p], aqq = A[(size_t)q * n + q];
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {  // A <- A J
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {  // A <- J' A
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {  // U <- U J
          const double ukp = U[(size_t)k * n + p], ukq = U[(size_t)k * n + q];
          U[(size_t)k * n + p] = c * ukp - s * ukq;
          U[(size_t)k * n + q] = s * ukp + c * ukq;
        }
      }
    }
  }
  return false;
}

template <typename T>
int upload(phylo_ctx* ctx, const Region& r, const T* host, size_t count,
           const char* what) {
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ws + r.off, host, count * sizeof(T),
                                cudaMemcpyHostToDevice, ctx->stream),
           what);
  return PHYLO_OK;
}

// Upload FP64 host values into a region of the path's element type
// (synchronous: the converted copy is a local buffer).
int upload_typed(phylo_ctx* ctx, const Region& r, const double* host, size_t count,
                 const char* what) {
  if (!count) return PHYLO_OK;
  if (ctx->precision == PHYLO_FP64) {
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ws + r.off, host, count * 8, cudaMemcpyHostToDevice,
                                  ctx->stream), what);
  } else {
    std::vector<float> buf(host, host + count);
    CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ws + r.off, buf.data(), count * 4,
                                  cudaMemcpyHostToDevice, ctx->stream), what);
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  }
  return PHYLO_OK;
}

// Self-test of the bounded waits: one CTA waits on an mbarrier that expects
// one arrival which never comes (nothing is armed on it: no copy, no MMA),
// with the same primitive and the same timeout report (ERR_TIMEOUT in the
// flag word) as the level kernels, then returns.
__device__ int g_selftest_flag;

__global__ void selftest_wait_kernel(int* flag, unsigned rounds) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) mbar_init_fenced(&bar, 1);
  __syncthreads();
  if (!__syncthreads_and(mbar_wait(&bar, 0, rounds)) && threadIdx.x == 0)
    atomicOr(flag, ERR_TIMEOUT);
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

int phylo_workspace_bytes(int n_tips, int n_patterns, int n_states,
                          int n_categories, int precision, int flags,
                          size_t* bytes) {
  if (!bytes) return fail(nullptr, PHYLO_EINVAL, "bytes is NULL");
  Layout L;
  const char* msg = compute_layout(n_tips, n_patterns, n_states, n_categories,
                                   precision, flags, &L);
  if (msg) return fail(nullptr, PHYLO_EINVAL, "%s", msg);
  *bytes = L.total;
  return PHYLO_OK;
}

int phylo_create(phylo_ctx** out, int n_tips, int n_patterns, int n_states,
                 int n_categories, int precision, int flags, void* workspace,
                 size_t workspace_bytes, void* stream) {
  if (!out) return fail(nullptr, PHYLO_EINVAL, "ctx is NULL");
  *out = nullptr;
  Layout L;
  const char* msg = compute_layout(n_tips, n_patterns, n_states, n_categories,
                                   precision, flags, &L);
  if (msg) return fail(nullptr, PHYLO_EINVAL, "%s", msg);
  if (!workspace) return fail(nullptr, PHYLO_EINVAL, "workspace is NULL");
  if (reinterpret_cast<uintptr_t>(workspace) % kAlign)
    return fail(nullptr, PHYLO_EINVAL, "workspace must be 256-byte aligned");
  if (workspace_bytes < L.total)
    return fail(nullptr, PHYLO_ENOMEM, "workspace has %zu bytes, needs %zu",
                workspace_bytes, L.total);
  phylo_ctx* ctx = new (std::nothrow) phylo_ctx();
  if (!ctx) return fail(nullptr, PHYLO_ENOMEM, "host allocation failed");
  ctx->N = n_tips;
  ctx->C = n_patterns;
  ctx->S = n_states;
  ctx->R = n_categories;
  ctx->precision = precision;
  ctx->flags = flags;
  ctx->L = L;
  ctx->ws = static_cast<char*>(workspace);
  ctx->ws_bytes = workspace_bytes;
  ctx->stream = static_cast<cudaStream_t>(stream);
  ctx->tip_has.assign(n_tips, 0);
  *out = ctx;
  return PHYLO_OK;
}

int phylo_set_tree(phylo_ctx* ctx, const int32_t* parent) {
  if (!ctx) return PHYLO_EINVAL;
  if (!parent) return fail(ctx, PHYLO_EINVAL, "parent is NULL");
  const int N = ctx->N, n = 2 * N - 1, root = n - 1;
  if (parent[root] != -1)
    return fail(ctx, PHYLO_EINVAL, "parent[%d] (the root) must be -1", root);
  std::vector<int2> ch(n, make_int2(-1, -1));
  for (int v = 0; v < root; ++v) {
    const int p = parent[v];
    if (p < N || p > root)
      return fail(ctx, PHYLO_EINVAL, "parent[%d] = %d is not an internal node", v, p);
    if (ch[p].x < 0) ch[p].x = v;
    else if (ch[p].y < 0) ch[p].y = v;
    else return fail(ctx, PHYLO_EINVAL, "node %d has more than two children", p);
  }
  for (int v = N; v < n; ++v)
    if (ch[v].y < 0)
      return fail(ctx, PHYLO_EINVAL, "internal node %d has fewer than two children", v);
  // depth by walking up (bounded: a cycle never reaches the root)
  std::vector<int> depth(n, -1), height(n, 0);
  depth[root] = 0;
  std::vector<int> path;
  for (int v = 0; v < n; ++v) {
    path.clear();
    int u = v;
    while (depth[u] < 0) {
      path.push_back(u);
      if ((int)path.size() > n)
        return fail(ctx, PHYLO_EINVAL, "the parent array has a cycle");
      u = parent[u];
    }
    int d = depth[u];
    for (size_t i = path.size(); i-- > 0;) depth[path[i]] = ++d;
  }
  // heights: process nodes by decreasing depth
  int max_depth = 0;
  for (int v = 0; v < n; ++v) max_depth = depth[v] > max_depth ? depth[v] : max_depth;
  std::vector<std::vector<int>> by_depth(max_depth + 1);
  for (int v = 0; v < n; ++v) by_depth[depth[v]].push_back(v);
  for (int d = max_depth; d >= 0; --d)
    for (int v : by_depth[d])
      if (v >= N) {
        const int a = height[ch[v].x], b = height[ch[v].y];
        height[v] = 1 + (a > b ? a : b);
      }
  ctx->children = ch;
  ctx->height = height;
  ctx->depth = depth;
  int rc = upload(ctx, ctx->L.children, ch.data(), ch.size(), "upload tree");
  if (rc) return rc;
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  if ((rc = build_schedule(ctx))) return rc;
  invalidate_graph(ctx);
  ctx->have_tree = true;
  ctx->have_grad = false;  // branch numbering may have changed
  return PHYLO_OK;
}

int phylo_set_tip_states(phylo_ctx* ctx, const uint8_t* states) {
  if (!ctx) return PHYLO_EINVAL;
  const size_t n = (size_t)ctx->N * ctx->C;
  if (!states && n) return fail(ctx, PHYLO_EINVAL, "states is NULL");
  for (size_t i = 0; i < n; ++i)
    if (states[i] > ctx->S)
      return fail(ctx, PHYLO_EINVAL, "tip %zu pattern %zu: state %d > n_states %d",
                  i / (ctx->C ? ctx->C : 1), i % (ctx->C ? ctx->C : 1),
                  (int)states[i], ctx->S);
  if (n) {  // rows padded to 16 bytes for the bulk copies
    CUDA_TRY(ctx, cudaMemcpy2DAsync(ctx->ws + ctx->L.tip_states.off, tip_state_stride(ctx->C),
                                    states, ctx->C, ctx->C, ctx->N, cudaMemcpyHostToDevice,
                                    ctx->stream),
             "upload tip states");
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  }
  ctx->have_states = true;
  return PHYLO_OK;
}

int phylo_set_tip_partials(phylo_ctx* ctx, int tip, const double* partials) {
  if (!ctx) return PHYLO_EINVAL;
  if (!(ctx->flags & PHYLO_FLAG_TIP_PARTIALS))
    return fail(ctx, PHYLO_EINVAL, "context created without PHYLO_FLAG_TIP_PARTIALS");
  if (tip < 0 || tip >= ctx->N) return fail(ctx, PHYLO_EINVAL, "tip %d out of range", tip);
  const int C = ctx->C, S = ctx->S, SP = ctx->L.SP;
  if (!partials && C) return fail(ctx, PHYLO_EINVAL, "partials is NULL");
  for (int c = 0; c < C; ++c) {
    double mx = 0.0;
    for (int s = 0; s < S; ++s) {
      const double x = partials[(size_t)c * S + s];
      if (!(x >= 0.0) || !std::isfinite(x))
        return fail(ctx, PHYLO_EINVAL, "tip %d pattern %d: partial must be finite and >= 0", tip, c);
      mx = x > mx ? x : mx;
    }
    if (mx == 0.0) return fail(ctx, PHYLO_EINVAL, "tip %d pattern %d: all-zero partial", tip, c);
  }
  const size_t count = (size_t)C * SP;
  const size_t off = ctx->L.tip_partials.off + (size_t)tip * count * ctx->L.elem;
  if (count) {
    if (ctx->precision == PHYLO_FP64) {
      std::vector<double> buf(count, 0.0);
      for (int c = 0; c < C; ++c)
        for (int s = 0; s < S; ++s) buf[(size_t)c * SP + s] = partials[(size_t)c * S + s];
      CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ws + off, buf.data(), count * 8,
                                    cudaMemcpyHostToDevice, ctx->stream), "upload tip partials");
      CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    } else {
      std::vector<float> buf(count, 0.0f);
      for (int c = 0; c < C; ++c)
        for (int s = 0; s < S; ++s) buf[(size_t)c * SP + s] = (float)partials[(size_t)c * S + s];
      CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ws + off, buf.data(), count * 4,
                                    cudaMemcpyHostToDevice, ctx->stream), "upload tip partials");
      CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
    }
  }
  const bool was = ctx->tip_has[tip] != 0;
  ctx->tip_has[tip] = 1;
  int rc = upload(ctx, ctx->L.tip_has, ctx->tip_has.data(), ctx->tip_has.size(),
                  "upload tip flags");
  if (rc) return rc;
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  if (!was) {  // kernels now take the partials path; a cherry above it is no longer fused
    invalidate_graph(ctx);
    if (ctx->have_tree && (rc = build_schedule(ctx))) return rc;
  }
  return PHYLO_OK;
}

int phylo_set_pattern_weights(phylo_ctx* ctx, const double* w) {
  if (!ctx) return PHYLO_EINVAL;
  if (!w && ctx->C) return fail(ctx, PHYLO_EINVAL, "weights is NULL");
  for (int c = 0; c < ctx->C; ++c)
    if (!(w[c] >= 0.0) || !std::isfinite(w[c]))
      return fail(ctx, PHYLO_EINVAL, "pattern weight %d must be finite and >= 0", c);
  if (ctx->C) {
    int rc = upload(ctx, ctx->L.pattern_w, w, ctx->C, "upload pattern weights");
    if (rc) return rc;
    rc = upload_typed(ctx, ctx->L.pattern_wt, w, ctx->C, "upload pattern weights");
    if (rc) return rc;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  }
  ctx->have_weights = true;
  return PHYLO_OK;
}

int phylo_set_eigen(phylo_ctx* ctx, const double* V, const double* Vinv,
                    const double* lambda, const double* pi) {
  if (!ctx) return PHYLO_EINVAL;
  if (!V || !Vinv || !lambda || !pi) return fail(ctx, PHYLO_EINVAL, "NULL argument");
  const int S = ctx->S;
  double psum = 0.0;
  for (int s = 0; s < S; ++s) {
    if (!(pi[s] >= 0.0) || !std::isfinite(pi[s]))
      return fail(ctx, PHYLO_EINVAL, "root frequency %d must be finite and >= 0", s);
    if (!std::isfinite(lambda[s]) || lambda[s] > 1e-8)
      return fail(ctx, PHYLO_EINVAL, "eigenvalue %d must be finite and <= 0", s);
    psum += pi[s];
  }
  if (std::fabs(psum - 1.0) > 1e-10)
    return fail(ctx, PHYLO_EINVAL, "root frequencies sum to %.17g, not 1", psum);
  for (int i = 0; i < S; ++i)
    for (int j = 0; j < S; ++j) {
      double acc = 0.0;
      for (int m = 0; m < S; ++m) acc += V[i * S + m] * Vinv[m * S + j];
      const double want = i == j ? 1.0 : 0.0;
      if (!std::isfinite(acc) || std::fabs(acc - want) > 1e-8)
        return fail(ctx, PHYLO_EINVAL, "V * Vinv differs from I at (%d,%d)", i, j);
    }
  int rc;
  if ((rc = upload(ctx, ctx->L.V, V, (size_t)S * S, "upload V"))) return rc;
  if ((rc = upload(ctx, ctx->L.Vinv, Vinv, (size_t)S * S, "upload Vinv"))) return rc;
  if (ctx->L.vsplit.bytes) {
    std::vector<float> split(eigen_split_floats(ctx->L.SP));
    ctx->eig_reversible = build_eigen_split(S, ctx->L.SP, V, Vinv, pi, split.data());
    if ((rc = upload(ctx, ctx->L.vsplit, split.data(), split.size(), "upload V split"))) return rc;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  }
  if (ctx->L.qmat.bytes) {
    std::vector<float> qm((size_t)ctx->L.SP * ctx->L.SP);
    build_q_matrix(S, ctx->L.SP, V, Vinv, lambda, qm.data());
    if ((rc = upload(ctx, ctx->L.qmat, qm.data(), qm.size(), "upload Q"))) return rc;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  }
  if (ctx->L.qt.bytes) {
    std::vector<unsigned char> qt(qt_bytes(ctx->L.SP));
    build_qt_tile(S, ctx->L.SP, V, Vinv, lambda, qt.data());
    if ((rc = upload(ctx, ctx->L.qt, qt.data(), qt.size(), "upload Q operand"))) return rc;
    CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  }
  if ((rc = upload(ctx, ctx->L.lambda, lambda, (size_t)S, "upload lambda"))) return rc;
  if ((rc = upload(ctx, ctx->L.pi, pi, (size_t)S, "upload pi"))) return rc;
  if ((rc = upload_typed(ctx, ctx->L.pi_t, pi, (size_t)S, "upload pi"))) return rc;
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  ctx->have_eigen = true;
  return PHYLO_OK;
}

int phylo_eigen_reversible(int S, const double* Q, const double* pi, double* V,
                           double* Vinv, double* lambda) {
  if (S < 2 || S > kMaxStates) return fail(nullptr, PHYLO_EINVAL, "n_states must be in [2, 256]");
  if (!Q || !pi || !V || !Vinv || !lambda) return fail(nullptr, PHYLO_EINVAL, "NULL argument");
  double qmax = 0.0, psum = 0.0;
  for (int i = 0; i < S; ++i) {
    if (!(pi[i] > 0.0) || !std::isfinite(pi[i]))
      return fail(nullptr, PHYLO_EINVAL, "pi[%d] must be finite and > 0", i);
    psum += pi[i];
    for (int j = 0; j < S; ++j) {
      const double q = Q[i * S + j];
      if (!std::isfinite(q)) return fail(nullptr, PHYLO_EINVAL, "Q[%d][%d] not finite", i, j);
      if (i != j && q < 0.0) return fail(nullptr, PHYLO_EINVAL, "Q[%d][%d] < 0", i, j);
      qmax = std::fabs(q) > qmax ? std::fabs(q) : qmax;
    }
  }
  if (std::fabs(psum - 1.0) > 1e-10) return fail(nullptr, PHYLO_EINVAL, "pi does not sum to 1");
  for (int i = 0; i < S; ++i) {
    double row = 0.0;
    for (int j = 0; j < S; ++j) row += Q[i * S + j];
    if (std::fabs(row) > 1e-10 * (qmax > 1.0 ? qmax : 1.0))
      return fail(nullptr, PHYLO_EINVAL, "row %d of Q does not sum to 0", i);
    for (int j = 0; j < S; ++j) {
      const double a = pi[i] * Q[i * S + j], b = pi[j] * Q[j * S + i];
      if (std::fabs(a - b) > 1e-10 * (std::fabs(a) + std::fabs(b) + 1e-300))
        if (std::fabs(a - b) > 1e-14)
          return fail(nullptr, PHYLO_EINVAL, "Q is not reversible w.r.t. pi at (%d,%d)", i, j);
    }
  }
  // B = D^1/2 Q D^-1/2 is symmetric; B = U diag(w) U'.
  std::vector<double> B((size_t)S * S), U, w;
  for (int i = 0; i < S; ++i)
    for (int j = 0; j < S; ++j) {
      const double bij = std::sqrt(pi[i]) * Q[i * S + j] / std::sqrt(pi[j]);
      const double bji = std::sqrt(pi[j]) * Q[j * S + i] / std::sqrt(pi[i]);
      B[(size_t)i * S + j] = 0.5 * (bij + bji);
    }
  if (!jacobi_eigen(S, B, U, w)) return fail(nullptr, PHYLO_EINVAL, "Jacobi did not converge");
  // A generator has the eigenvalue 0 (rows sum to 0): make it exact, so
  // that P(t) tends to the stationary rows for long branches.
  int zero = 0;
  for (int i = 1; i < S; ++i)
    if (std::fabs(w[i]) < std::fabs(w[zero])) zero = i;
  w[zero] = 0.0;
  for (int i = 0; i < S; ++i) {
    lambda[i] = w[i] > 0.0 ? 0.0 : w[i];
    for (int m = 0; m < S; ++m) {
      V[i * S + m] = U[(size_t)i * S + m] / std::sqrt(pi[i]);
      Vinv[m * S + i] = U[(size_t)i * S + m] * std::sqrt(pi[i]);
    }
  }
  return PHYLO_OK;
}

int phylo_set_rate_matrix(phylo_ctx* ctx, const double* Q, const double* pi) {
  if (!ctx) return PHYLO_EINVAL;
  const int S = ctx->S;
  std::vector<double> V((size_t)S * S), Vi((size_t)S * S), lam(S);
  if (phylo_eigen_reversible(S, Q, pi, V.data(), Vi.data(), lam.data()) != PHYLO_OK)
    return fail(ctx, PHYLO_EINVAL, "%s", g_create_error.c_str());
  return phylo_set_eigen(ctx, V.data(), Vi.data(), lam.data(), pi);
}

int phylo_set_categories(phylo_ctx* ctx, const double* rates, const double* weights) {
  if (!ctx) return PHYLO_EINVAL;
  if (!rates || !weights) return fail(ctx, PHYLO_EINVAL, "NULL argument");
  double wsum = 0.0;
  for (int r = 0; r < ctx->R; ++r) {
    if (!(rates[r] >= 0.0) || !std::isfinite(rates[r]))
      return fail(ctx, PHYLO_EINVAL, "category rate %d must be finite and >= 0", r);
    if (!(weights[r] >= 0.0) || !std::isfinite(weights[r]))
      return fail(ctx, PHYLO_EINVAL, "category weight %d must be finite and >= 0", r);
    wsum += weights[r];
  }
  if (std::fabs(wsum - 1.0) > 1e-10)
    return fail(ctx, PHYLO_EINVAL, "category weights sum to %.17g, not 1", wsum);
  int rc;
  if ((rc = upload(ctx, ctx->L.rates, rates, (size_t)ctx->R, "upload rates"))) return rc;
  if ((rc = upload(ctx, ctx->L.cat_w, weights, (size_t)ctx->R, "upload weights"))) return rc;
  if ((rc = upload_typed(ctx, ctx->L.cat_wt, weights, (size_t)ctx->R, "upload weights"))) return rc;
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  ctx->have_cats = true;
  return PHYLO_OK;
}

int phylo_set_branch_lengths(phylo_ctx* ctx, const double* t, int on_device) {
  if (!ctx) return PHYLO_EINVAL;
  const size_t nb = 2 * (size_t)ctx->N - 2;
  if (!t) return fail(ctx, PHYLO_EINVAL, "t is NULL");
  if (!on_device) {
    for (size_t b = 0; b < nb; ++b)
      if (!(t[b] >= 0.0) || !std::isfinite(t[b]))
        return fail(ctx, PHYLO_EINVAL, "branch length %zu must be finite and >= 0", b);
  }
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->ws + ctx->L.t.off, t, nb * 8,
                                on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                ctx->stream),
           "upload branch lengths");
  ctx->have_t = true;
  ctx->forward_valid = false;
  return PHYLO_OK;
}

int phylo_evaluate(phylo_ctx* ctx, double* logL, double* grad) {
  if (!ctx) return PHYLO_EINVAL;
  if (!logL) return fail(ctx, PHYLO_EINVAL, "log_likelihood is NULL");
  int rc = launch_eval(ctx);
  if (rc) return rc;
  rc = ensure_host_out(ctx);
  if (rc) return rc;
  const size_t n = 2 * (size_t)ctx->N - 1;
  CUDA_TRY(ctx, cudaMemcpyAsync(ctx->host_out, ctx->dev<double>(ctx->L.out), n * 8 + 8,
                                cudaMemcpyDeviceToHost, ctx->stream),
           "download results");
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  int flags;
  std::memcpy(&flags, ctx->host_out + n, sizeof(int));
  rc = read_flags(ctx, flags);
  if (rc) return rc;
  *logL = ctx->host_out[0];
  if (grad) std::memcpy(grad, ctx->host_out + 1, (n - 1) * 8);
  return PHYLO_OK;
}

int phylo_evaluate_device(phylo_ctx* ctx, double* out) {
  if (!ctx) return PHYLO_EINVAL;
  if (!out) return fail(ctx, PHYLO_EINVAL, "out is NULL");
  int rc = launch_eval(ctx);
  if (rc) return rc;
  const size_t n = 2 * (size_t)ctx->N - 1;
  if (out != ctx->dev<double>(ctx->L.out))
    CUDA_TRY(ctx, cudaMemcpyAsync(out, ctx->dev<double>(ctx->L.out), n * 8,
                                  cudaMemcpyDeviceToDevice, ctx->stream),
             "copy results");
  return PHYLO_OK;
}

int phylo_evaluate_device_timed(phylo_ctx* ctx, double* out, void* const* events) {
  if (!ctx) return PHYLO_EINVAL;
  if (!out || !events) return fail(ctx, PHYLO_EINVAL, "NULL argument");
  for (int i = 0; i <= kPhases; ++i)
    if (!events[i]) return fail(ctx, PHYLO_EINVAL, "event %d is NULL", i);
  int rc = check_ready(ctx);
  if (rc) return rc;
  if (ctx->phase_dirty || !ctx->phase_exec[0]) {
    rc = build_phase_graphs(ctx);
    if (rc) return rc;
  }
  ++ctx->partials_gen;
  ctx->forward_valid = true;
  ctx->have_grad = true;
  for (int ph = 0; ph < kPhases; ++ph) {
    CUDA_TRY(ctx, cudaEventRecord(static_cast<cudaEvent_t>(events[ph]), ctx->stream),
             "cudaEventRecord");
    CUDA_TRY(ctx, cudaGraphLaunch(ctx->phase_exec[ph], ctx->stream), "cudaGraphLaunch");
  }
  CUDA_TRY(ctx, cudaEventRecord(static_cast<cudaEvent_t>(events[kPhases]), ctx->stream),
           "cudaEventRecord");
  const size_t n = 2 * (size_t)ctx->N - 1;
  if (out != ctx->dev<double>(ctx->L.out))
    CUDA_TRY(ctx, cudaMemcpyAsync(out, ctx->dev<double>(ctx->L.out), n * 8,
                                  cudaMemcpyDeviceToDevice, ctx->stream),
             "copy results");
  return PHYLO_OK;
}

int phylo_forward_device(phylo_ctx* ctx, double* out, uint64_t* generation) {
  if (!ctx) return PHYLO_EINVAL;
  if (!out) return fail(ctx, PHYLO_EINVAL, "out is NULL");
  int rc = check_ready(ctx);
  if (rc) return rc;
  NvtxRange range("phylo forward");
  ++ctx->partials_gen;
  ctx->forward_valid = false;
  // matrices and post-order levels, then the log-likelihood alone
  if (ctx->flags & PHYLO_FLAG_NO_GRAPH) {
    rc = run_phases(ctx, 0, 1, nullptr);
    if (!rc) rc = run_phases(ctx, kPhaseLogLOnly, kPhaseLogLOnly, nullptr);
  } else {
    if (ctx->graph_dirty || ctx->phase_dirty) {
      invalidate_graph(ctx);
      rc = upload_descriptors(ctx);
      if (rc) return rc;
      ctx->graph_dirty = ctx->phase_dirty = false;
    }
    rc = run_phases(ctx, 0, kPhaseLogLOnly, &ctx->fwd_exec);
  }
  if (rc) return rc;
  ctx->forward_valid = true;
  if (generation) *generation = ctx->partials_gen;
  if (out != ctx->dev<double>(ctx->L.out))
    CUDA_TRY(ctx, cudaMemcpyAsync(out, ctx->dev<double>(ctx->L.out), 8,
                                  cudaMemcpyDeviceToDevice, ctx->stream),
             "copy log-likelihood");
  return PHYLO_OK;
}

int phylo_backward_device(phylo_ctx* ctx, double* out, uint64_t generation) {
  if (!ctx) return PHYLO_EINVAL;
  if (!out) return fail(ctx, PHYLO_EINVAL, "out is NULL");
  if (!ctx->forward_valid)
    return fail(ctx, PHYLO_ESTATE, "backward needs a forward pass on the current inputs");
  if (generation != ctx->partials_gen)
    return fail(ctx, PHYLO_ESTATE,
                "backward of forward %llu, but the partials now belong to a later "
                "pass (%llu): run that forward again",
                (unsigned long long)generation, (unsigned long long)ctx->partials_gen);
  NvtxRange range("phylo backward");
  int rc;
  if (ctx->flags & PHYLO_FLAG_NO_GRAPH) rc = run_phases(ctx, 2, 3, nullptr);
  else rc = run_phases(ctx, 2, 3, &ctx->bwd_exec);
  if (rc) return rc;
  ctx->have_grad = true;
  if (out != ctx->dev<double>(ctx->L.out) + 1)
    CUDA_TRY(ctx, cudaMemcpyAsync(out, ctx->dev<double>(ctx->L.out) + 1,
                                  (2 * (size_t)ctx->N - 2) * 8, cudaMemcpyDeviceToDevice,
                                  ctx->stream),
             "copy gradient");
  return PHYLO_OK;
}

// ---- chain-rule epilogues ------------------------------------------------

int gradient_ready(phylo_ctx* ctx) {
  if (!ctx->have_grad)
    return fail(ctx, PHYLO_ESTATE, "no gradient on this context: evaluate first");
  return PHYLO_OK;
}

int phylo_gradient_rate_time(phylo_ctx* ctx, const double* rates, const double* times,
                             double* d_rates, double* d_times, int on_device) {
  if (!ctx) return PHYLO_EINVAL;
  if (!rates || !times) return fail(ctx, PHYLO_EINVAL, "rates and times must not be NULL");
  int rc = gradient_ready(ctx);
  if (rc) return rc;
  const int nb = 2 * ctx->N - 2;
  const double* g = ctx->dev<double>(ctx->L.out) + 1;
  if (on_device) {
    CUDA_TRY(ctx, launch_grad_rate_time(g, nb, rates, times, d_rates, d_times, ctx->stream),
             "chain-rule kernel");
    return PHYLO_OK;
  }
  for (int i = 0; i < nb; ++i)
    if (!std::isfinite(rates[i]) || !std::isfinite(times[i]))
      return fail(ctx, PHYLO_EINVAL, "branch %d: rate and time must be finite", i);
  if ((rc = upload(ctx, ctx->L.chain_a, rates, nb, "upload rates"))) return rc;
  if ((rc = upload(ctx, ctx->L.chain_b, times, nb, "upload times"))) return rc;
  double* out = ctx->dev<double>(ctx->L.chain_out);
  CUDA_TRY(ctx, launch_grad_rate_time(g, nb, ctx->dev<double>(ctx->L.chain_a),
                                      ctx->dev<double>(ctx->L.chain_b), out, out + nb,
                                      ctx->stream),
           "chain-rule kernel");
  if (d_rates)
    CUDA_TRY(ctx, cudaMemcpyAsync(d_rates, out, nb * 8, cudaMemcpyDeviceToHost, ctx->stream),
             "download");
  if (d_times)
    CUDA_TRY(ctx, cudaMemcpyAsync(d_times, out + nb, nb * 8, cudaMemcpyDeviceToHost,
                                  ctx->stream),
             "download");
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  return PHYLO_OK;
}

int phylo_gradient_heights(phylo_ctx* ctx, const double* rates, double* d_heights,
                           int on_device) {
  if (!ctx) return PHYLO_EINVAL;
  if (!d_heights) return fail(ctx, PHYLO_EINVAL, "d_heights is NULL");
  int rc = gradient_ready(ctx);
  if (rc) return rc;
  const int nb = 2 * ctx->N - 2, n_nodes = 2 * ctx->N - 1;
  const double* g = ctx->dev<double>(ctx->L.out) + 1;
  const int2* children = ctx->dev<int2>(ctx->L.children);
  if (on_device) {
    CUDA_TRY(ctx, launch_grad_heights(g, children, ctx->N, rates, d_heights, ctx->stream),
             "chain-rule kernel");
    return PHYLO_OK;
  }
  const double* rd = nullptr;
  if (rates) {
    for (int i = 0; i < nb; ++i)
      if (!std::isfinite(rates[i]))
        return fail(ctx, PHYLO_EINVAL, "branch %d: rate must be finite", i);
    if ((rc = upload(ctx, ctx->L.chain_a, rates, nb, "upload rates"))) return rc;
    rd = ctx->dev<double>(ctx->L.chain_a);
  }
  double* out = ctx->dev<double>(ctx->L.chain_out);
  CUDA_TRY(ctx, launch_grad_heights(g, children, ctx->N, rd, out, ctx->stream),
           "chain-rule kernel");
  CUDA_TRY(ctx, cudaMemcpyAsync(d_heights, out, n_nodes * 8, cudaMemcpyDeviceToHost,
                                ctx->stream),
           "download");
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  return PHYLO_OK;
}

int phylo_gradient_branch_sum(phylo_ctx* ctx, const int32_t* branches, const double* weights,
                              int n, double* out, int on_device) {
  if (!ctx) return PHYLO_EINVAL;
  const int nb = 2 * ctx->N - 2;
  if (!out) return fail(ctx, PHYLO_EINVAL, "out is NULL");
  if (n < 0 || n > nb) return fail(ctx, PHYLO_EINVAL, "n = %d must be in [0, %d]", n, nb);
  if (n > 0 && !branches) return fail(ctx, PHYLO_EINVAL, "branches is NULL");
  int rc = gradient_ready(ctx);
  if (rc) return rc;
  const double* g = ctx->dev<double>(ctx->L.out) + 1;
  if (on_device) {
    CUDA_TRY(ctx, launch_grad_branch_sum(g, reinterpret_cast<const int*>(branches), weights, n,
                                         out, ctx->stream),
             "chain-rule kernel");
    return PHYLO_OK;
  }
  for (int j = 0; j < n; ++j) {
    if (branches[j] < 0 || branches[j] >= nb)
      return fail(ctx, PHYLO_EINVAL, "branches[%d] = %d is not a branch", j, branches[j]);
    if (weights && !std::isfinite(weights[j]))
      return fail(ctx, PHYLO_EINVAL, "weights[%d] must be finite", j);
  }
  const double* wd = nullptr;
  if (n > 0) {
    if ((rc = upload(ctx, ctx->L.chain_idx, branches, n, "upload branches"))) return rc;
    if (weights) {
      if ((rc = upload(ctx, ctx->L.chain_b, weights, n, "upload weights"))) return rc;
      wd = ctx->dev<double>(ctx->L.chain_b);
    }
  }
  double* dout = ctx->dev<double>(ctx->L.chain_out);
  CUDA_TRY(ctx, launch_grad_branch_sum(g, ctx->dev<int>(ctx->L.chain_idx), wd, n, dout,
                                       ctx->stream),
           "chain-rule kernel");
  CUDA_TRY(ctx, cudaMemcpyAsync(out, dout, 8, cudaMemcpyDeviceToHost, ctx->stream), "download");
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  return PHYLO_OK;
}

int phylo_check(phylo_ctx* ctx) {
  if (!ctx) return PHYLO_EINVAL;
  int flags = 0;
  CUDA_TRY(ctx, cudaMemcpyAsync(&flags, flag_word(ctx), sizeof(int),
                                cudaMemcpyDeviceToHost, ctx->stream),
           "read flags");
  CUDA_TRY(ctx, cudaStreamSynchronize(ctx->stream), "cudaStreamSynchronize");
  return read_flags(ctx, flags);
}

int phylo_launches_per_evaluation(const phylo_ctx* ctx) {
  if (!ctx || !ctx->have_tree) return 0;
  int n = 2;  // pmat + final reduction
  if (ctx->C > 0) {
    const bool fp64 = ctx->precision == PHYLO_FP64;
    n += (int)(ctx->post_off.size() - 1) + (int)(ctx->pre_off.size() - 1);
    if (uses_tc_terms(ctx->L.SP, fp64)) ++n;  // Eq. 8 ratios
    if (has_tip_level(ctx)) ++n;                // U of the tips with partials
  }
  return n;
}

int phylo_level_counts(const phylo_ctx* ctx, int* n_post_levels,
                       int* n_pre_levels) {
  if (!ctx || !n_post_levels || !n_pre_levels) return PHYLO_EINVAL;
  *n_post_levels = ctx->have_tree ? (int)ctx->post_off.size() - 1 : 0;
  *n_pre_levels = ctx->have_tree ? (int)ctx->pre_off.size() - 1 : 0;
  if (ctx->have_tree && ctx->C > 0 && has_tip_level(ctx)) ++*n_post_levels;
  return PHYLO_OK;
}

int phylo_selftest_bounded_wait(int rounds, void* stream) {
  if (rounds < 1 || rounds > 1024)
    return fail(nullptr, PHYLO_EINVAL, "rounds must be in [1, 1024]");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  int* flag = nullptr;
  cudaError_t e = cudaGetSymbolAddress(reinterpret_cast<void**>(&flag), g_selftest_flag);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress");
  if ((e = cudaMemsetAsync(flag, 0, sizeof(int), st)) != cudaSuccess)
    return cuda_fail(nullptr, e, "cudaMemsetAsync");
  selftest_wait_kernel<<<1, 32, 0, st>>>(flag, (unsigned)rounds);
  if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(nullptr, e, "launch");
  int flags = 0;
  if ((e = cudaMemcpyAsync(&flags, flag, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess)
    return cuda_fail(nullptr, e, "read flag");
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess)
    return cuda_fail(nullptr, e, "cudaStreamSynchronize");
  if (flags & ERR_TIMEOUT)
    return fail(nullptr, PHYLO_ETIMEOUT, "device flagged: a bounded wait expired (self-test)");
  return read_flags(nullptr, flags);
}

const char* phylo_last_error(const phylo_ctx* ctx) {
  return ctx ? ctx->err.c_str() : g_create_error.c_str();
}

int phylo_destroy(phylo_ctx* ctx) {
  if (!ctx) return PHYLO_OK;
  invalidate_graph(ctx);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->host_out) cudaFreeHost(ctx->host_out);
  delete ctx;
  return PHYLO_OK;
}

}  // extern "C"
