/*
 * phylo_api.h -- C ABI of libphylograd: the phylogenetic log-likelihood and
 * its gradient with respect to all 2N-2 branch lengths on one GPU
 * (arXiv 2303.04390, "Many-core algorithms for high-dimensional gradients on
 * phylogenetic trees").
 *
 * Problem statement (paper, Methods): an alignment of C unique site
 * patterns with integer weights W_c over N taxa; a rooted binary tree with
 * tips 0..N-1, internal nodes N..2N-2 and the root 2N-2; branch i is the
 * branch above node i (length t_i); a reversible CTMC with generator Q and
 * root distribution pi; R rate categories with rates gamma_r and weights
 * w_r.  P^(r)(t) = exp(gamma_r t Q) (Eq. 1), entry (s,u) = Pr(child u |
 * parent s).  The library returns
 *     log P(Y) = sum_c W_c log sum_r w_r pi' p_root,r,c          (Eq. 3)
 *     d log P(Y) / d t_i  for every i < 2N-2                      (Eqs. 7, 8)
 * via post-order partials (Eq. 2), pre-order partials (Eq. 4) and the
 * per-branch ratio of Eq. 8, with per-node power-of-two rescaling.
 *
 * Conventions for every call:
 *  - Return value: PHYLO_OK (0) or a negative phylo_status.  After an error
 *    phylo_last_error(ctx) describes it.  Nothing aborts or exits.
 *  - Host pointers are read during the call and not kept; the caller keeps
 *    ownership.  Device pointers are noted as such.
 *  - The library allocates no device memory.  The caller provides one
 *    device workspace of phylo_workspace_bytes() bytes at phylo_create and
 *    keeps it alive until phylo_destroy.
 *  - All device work is ordered on the stream given to phylo_create
 *    (NULL = the legacy default stream).
 *  - Matrices are row-major FP64.  Sizes: N tips, C patterns, S states
 *    (2 <= S <= 256; S <= 64 for phylo_evaluate_noalloc), R categories
 *    (1 <= R <= 8).  Kernels by padded state count S_pad: 4 and 20 (CUDA
 *    cores), 64 and 128 (FP32: tensor cores), 256 and the FP64 path above 64
 *    (CUDA cores, matrices streamed through shared memory).
 */
#ifndef PHYLO_API_H
#define PHYLO_API_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct phylo_ctx phylo_ctx; /* opaque; host-side state only */

enum phylo_status {
  PHYLO_OK = 0,
  PHYLO_EINVAL = -1,   /* an argument or input failed validation          */
  PHYLO_ENOMEM = -2,   /* workspace too small or host allocation failed    */
  PHYLO_ECUDA = -3,    /* a CUDA runtime call failed (message has details) */
  PHYLO_ESTATE = -4,   /* a required input has not been set yet            */
  PHYLO_ENUMERIC = -5, /* the device flagged a zero/NaN partial or a bad t */
  PHYLO_ETIMEOUT = -6  /* a bounded device-side wait expired (results void) */
};

enum phylo_precision {
  PHYLO_FP64 = 0, /* partials, matrices and arithmetic in FP64 (baseline) */
  PHYLO_FP32 = 1  /* FP32 partials and arithmetic, FP64 reductions        */
};

enum phylo_flags {
  PHYLO_FLAG_TIP_PARTIALS = 1, /* reserve storage so tips may carry partials */
  PHYLO_FLAG_NO_GRAPH = 2      /* launch kernels directly, no CUDA graph
                                  (one-shot contexts: capture would cost
                                  more than it saves) */
};

/* Bytes of device workspace a context of this shape needs.  Host only.
 * Returns PHYLO_EINVAL for out-of-range sizes or size_t overflow. */
int phylo_workspace_bytes(int n_tips, int n_patterns, int n_states,
                          int n_categories, int precision, int flags,
                          size_t* bytes);

/* Create a context over a caller-owned device workspace (device pointer,
 * 256-byte aligned, at least phylo_workspace_bytes()).  `stream` is a
 * cudaStream_t (NULL = legacy default stream).  Host only: no CUDA call is
 * made until the first input is uploaded.  n_patterns may be 0 (then
 * log P(Y) = 0 and the gradient is 0). */
int phylo_create(phylo_ctx** ctx, int n_tips, int n_patterns, int n_states,
                 int n_categories, int precision, int flags,
                 void* workspace, size_t workspace_bytes, void* stream);

/* Tree topology (paper, Methods).  parent: host int32 [2N-1];
 * parent[2N-2] = -1 (the root); every other entry names an internal node
 * in [N, 2N-2]; each internal node has exactly two children; tips
 * 0..N-1 have none.  Builds the level schedule (nodes grouped by height
 * for the post-order pass and by depth for the pre-order pass). */
int phylo_set_tree(phylo_ctx* ctx, const int32_t* parent);

/* Compact tip data (Methods, gradient subsection: an observed tip is
 * stored as one integer per pattern).  states: host uint8 [N][C], values in
 * [0, S]; S marks a gap or unknown character (an all-ones partial).  With
 * S = 256 every byte value is a state (no gap code): gaps then go through
 * phylo_set_tip_partials. */
int phylo_set_tip_states(phylo_ctx* ctx, const uint8_t* states);

/* Partial likelihood vector for one tip (ambiguity codes, sequencing
 * error): host FP64 [C][S], finite, >= 0, not all zero for any c.
 * Requires PHYLO_FLAG_TIP_PARTIALS.  Overrides the tip's states. */
int phylo_set_tip_partials(phylo_ctx* ctx, int tip, const double* partials);

/* Pattern weights W_c (paper, Methods: unique columns reweighted).
 * host FP64 [C], finite and >= 0. */
int phylo_set_pattern_weights(phylo_ctx* ctx, const double* weights);

/* Eigen-decomposition Q = V diag(lambda) Vinv and root distribution pi,
 * used for P(t) = V diag(e^{lambda gamma t}) Vinv (Eq. 1).  Host FP64:
 * V, Vinv [S][S], lambda [S], pi [S] (>= 0, sums to 1).  V*Vinv must be
 * the identity within 1e-8. */
int phylo_set_eigen(phylo_ctx* ctx, const double* V, const double* Vinv,
                    const double* lambda, const double* root_freqs);

/* Convenience: a reversible generator Q (host FP64 [S][S], rows summing to
 * 0, pi_i Q_ij = pi_j Q_ji) with stationary pi (> 0) is decomposed on the
 * host in FP64 (Jacobi on the symmetrised matrix) and passed to
 * phylo_set_eigen.  pi is also the root distribution. */
int phylo_set_rate_matrix(phylo_ctx* ctx, const double* Q, const double* pi);

/* Host-only utility behind phylo_set_rate_matrix: writes V, Vinv [S][S]
 * and lambda [S] for a reversible Q with stationary pi (> 0). */
int phylo_eigen_reversible(int n_states, const double* Q, const double* pi,
                           double* V, double* Vinv, double* lambda);

/* Rate categories (paper, Methods; Yang 1994): rates gamma_r >= 0 and
 * weights w_r >= 0 summing to 1 (within 1e-10).  Host FP64 [R] each. */
int phylo_set_categories(phylo_ctx* ctx, const double* rates,
                         const double* weights);

/* Branch lengths t_i for i < 2N-2 (FP64 [2N-2]).  on_device = 0: host
 * pointer (validated: finite, >= 0); on_device = 1: device pointer, copied
 * on the stream (validated on the device; a bad value makes the next
 * evaluation return PHYLO_ENUMERIC). */
int phylo_set_branch_lengths(phylo_ctx* ctx, const double* t, int on_device);

/* One evaluation: P and dP/dt for all branches and categories, the
 * post-order pass with log P(Y), the pre-order pass with the gradient, and
 * the cross-pattern FP64 reductions.  Writes log P(Y) to *log_likelihood
 * and d log P(Y)/d t_i to gradient[i] (host FP64 [2N-2], or NULL for
 * log P(Y) only).  Synchronises the stream. */
int phylo_evaluate(phylo_ctx* ctx, double* log_likelihood, double* gradient);

/* Same evaluation, asynchronous: writes [log P(Y), grad_0 .. grad_{2N-3}]
 * (FP64, 2N-1 values) to the device pointer `out` on the stream and
 * returns without synchronising.  Device-side numeric flags are reported
 * by the next phylo_check / phylo_evaluate. */
int phylo_evaluate_device(phylo_ctx* ctx, double* out);

/* Same as phylo_evaluate_device, split into its four phases with a
 * caller-created cudaEvent_t recorded on the stream at each boundary:
 * events[0] before the matrix build (Eq. 1), events[1] before the
 * post-order pass (Eqs. 2-3), events[2] before the pre-order pass with the
 * gradient (Eqs. 4, 8), events[3] before the final reduction (Eq. 7) and
 * events[4] after it.  `events` is a host array of 5 cudaEvent_t; the
 * caller owns them.  The phases run as four graph launches instead of one,
 * so per-phase device times can be read with cudaEventElapsedTime. */
int phylo_evaluate_device_timed(phylo_ctx* ctx, double* out,
                                void* const* events);

/* The evaluation split at its natural seam, for reverse-mode use (the
 * pre-order pass of Eq. 4 with the Eq. 8 ratio is the backward of the
 * post-order pass of Eqs. 2-3): forward runs the matrix build, the
 * post-order pass and the log-likelihood reduction and writes log P(Y)
 * (1 FP64 value) to the device pointer `out`; backward runs the pre-order
 * pass with the fused gradient and the gradient reduction and writes
 * d log P(Y)/d t (2N-2 FP64 values) to the device pointer `out`.  Both are
 * asynchronous on the stream.
 *
 * Every pass that rewrites the context's post-order partials (a forward,
 * any evaluation) gets a new generation number; forward returns its own in
 * *generation (may be NULL).  Backward takes the generation of the forward
 * it differentiates and returns PHYLO_ESTATE, without launching anything,
 * unless that forward is still the latest such pass and the branch
 * lengths have not changed since: two forwards before one backward cannot
 * silently return the second forward's gradient for the first. */
int phylo_forward_device(phylo_ctx* ctx, double* out, uint64_t* generation);
int phylo_backward_device(phylo_ctx* ctx, double* out, uint64_t generation);

/* Chain-rule epilogues on the gradient of the most recent evaluation on
 * this context (phylo_evaluate, phylo_evaluate_device or
 * phylo_backward_device; PHYLO_ESTATE before the first), for the branch
 * parameterisations the paper names (Methods: a branch length is the
 * difference of the parent's and child's node heights in time units times
 * a possibly branch-specific rate; for a strict clock the branch
 * derivatives are further reduced over a set of branches).  g_i denotes
 * d log P(Y)/d t_i, branch i being the branch above node i.
 *
 * With on_device = 0 every pointer is host memory and the call
 * synchronises the stream; with on_device = 1 every pointer is device
 * memory and the call is asynchronous on the stream (the inputs are read
 * by the kernels, so they must stay valid until the stream reaches them).
 * Inputs are validated on the host only in the host form. */

/* t_i = rate_i x time_i (2N-2 of each):
 *   d_rates[i] = time_i g_i,  d_times[i] = rate_i g_i.
 * Either output may be NULL. */
int phylo_gradient_rate_time(phylo_ctx* ctx, const double* rates, const double* times,
                             double* d_rates, double* d_times, int on_device);

/* t_i = rate_i (h_parent(i) - h_i) for node heights h (2N-1 values, tips
 * included): d_heights[k] = -rate_k g_k (k not the root)
 *                          + sum over children c of k of rate_c g_c.
 * rates may be NULL (all 1). */
int phylo_gradient_heights(phylo_ctx* ctx, const double* rates, double* d_heights,
                           int on_device);

/* *out = sum_j weights[j] g_{branches[j]} over n entries (n <= 2N-2;
 * branches[j] in [0, 2N-2); weights may be NULL for all 1).  A strict
 * clock t_i = rate x time_i gives d/d rate = this sum with weights time_i
 * over all branches.  One FP64 value; the sum runs in a fixed order. */
int phylo_gradient_branch_sum(phylo_ctx* ctx, const int32_t* branches, const double* weights,
                              int n, double* out, int on_device);

/* Synchronise the stream and report device-side numeric flags raised since
 * the last check (PHYLO_ENUMERIC) or PHYLO_OK. */
int phylo_check(phylo_ctx* ctx);

/* Number of kernel launches one evaluation makes (the level schedule's
 * length plus the matrix build and the final reduction); 0 before the
 * tree is set. */
int phylo_launches_per_evaluation(const phylo_ctx* ctx);

/* Length of the level schedule: the number of post-order launches (tree
 * height, less the heights left empty by fused cherries on the FP32
 * 4-state path; plus one for Eq. 3 at the root on the FP32 path for 65-128
 * states) and of pre-order launches (distinct depths of internal nodes;
 * twice that on the FP32 path for 65-128 states, which runs two kernels per
 * level).  Both 0 before the tree is set. */
int phylo_level_counts(const phylo_ctx* ctx, int* n_post_levels,
                       int* n_pre_levels);

/* Self-test of the bounded device waits (no counterpart in the paper; the
 * kernels' asynchronous copies and MMAs complete on mbarriers, and every
 * wait gives up after a bounded number of try_wait rounds, raising a flag
 * that the host reports as PHYLO_ETIMEOUT).  Launches one CTA on `stream`
 * (a cudaStream_t, NULL = legacy default) that waits, with the same
 * primitive and limit logic, on an mbarrier nothing is armed on, giving up
 * after `rounds` rounds (1..1024), and synchronises the stream.  Returns
 * PHYLO_ETIMEOUT when the wait expired and was reported (the expected
 * result), PHYLO_OK if the flag stayed clear, PHYLO_EINVAL for a bad
 * `rounds`, PHYLO_ECUDA on a CUDA error.  Nothing is left in flight, so the
 * CUDA context stays usable.  Uses a static device word, not the heap. */
int phylo_selftest_bounded_wait(int rounds, void* stream);

/* Message for the last error on ctx (or for the last failed phylo_create
 * when ctx is NULL).  Valid until the next call on ctx. */
const char* phylo_last_error(const phylo_ctx* ctx);

/* No-allocation evaluation (the paper has no counterpart).  It exists for
 * callers that cannot allocate device memory: runtimes that own all of the
 * GPU's memory through their own pools and forbid side allocations, and
 * fixed-footprint samplers or embedded services that must not grow their
 * memory use after start-up.  cudaMalloc is either unavailable to them or
 * would break their memory accounting.
 *
 * One FP32 evaluation of log P(Y) and its gradient, as phylo_evaluate,
 * from host inputs to host outputs, without a context or a workspace.  All
 * intermediate buffers live in one static device array of 32 MiB inside
 * the library, reserved on every GPU that loads the library until the
 * process exits.  Limits: 2 <= n_tips <= 512, 2 <= n_states <= 64,
 * 1 <= n_categories <= 8, and the problem's buffers must fit in 32 MiB
 * (e.g. 64 tips x 4,000 patterns x 4 states x 4 categories); larger
 * problems return PHYLO_EINVAL with a message naming the bytes needed,
 * before any CUDA call.  Arguments as in phylo_set_tree /
 * phylo_set_tip_states / phylo_set_pattern_weights / phylo_set_eigen /
 * phylo_set_categories / phylo_set_branch_lengths (all host pointers,
 * validated first); gradient may be NULL; error_message (may be NULL)
 * receives up to error_capacity bytes of text on failure.
 *
 * The first call on a device, with that device current, looks the array's
 * device address up (cudaGetSymbolAddress) and sets kernel attributes for
 * that device.  Calls allocate no device or pinned memory and call no
 * allocating library routine.  Every call on a device shares the same
 * array and finds it holding the previous call's contents (the call clears
 * the one word it reads before writing).  Calls are synchronous: the stream
 * is synchronised before returning, on error paths too once device work has
 * been queued.  Calls are serialised within a process; device work that
 * overlaps a call while touching the same array (kernels launched by
 * another thread of this process from a copy of the array's address) races
 * with it. */
int phylo_evaluate_noalloc(int n_tips, int n_patterns, int n_states,
                           int n_categories, const int32_t* parent,
                           const uint8_t* tip_states,
                           const double* pattern_weights, const double* V,
                           const double* Vinv, const double* lambda,
                           const double* root_freqs, const double* rates,
                           const double* category_weights,
                           const double* branch_lengths,
                           double* log_likelihood, double* gradient,
                           void* stream, char* error_message,
                           size_t error_capacity);

/* Release the host-side state and any CUDA objects (graph, streams) of the
 * context.  The caller frees the workspace afterwards. */
int phylo_destroy(phylo_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* PHYLO_API_H */
