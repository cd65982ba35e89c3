// FP64 instantiation of the level kernels and the matrix builder, plus the
// final cross-tile reduction shared by both precisions.
#include "kernels.cuh"

PHYLO_INSTANTIATE(double)

namespace phylo {

// Final reduction (Eq. 7 across pattern tiles, and Eq. 3's sum): one warp
// per output, lane-strided sums then a fixed shuffle tree, so the result is
// deterministic.  Output 0 is log P(Y); output 1 + b is the gradient of
// branch b.
__global__ void __launch_bounds__(256) reduce_kernel(ReduceArgs a) {
  pdl_wait_and_release();
  const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (warp > a.n_branches) return;  // warp-uniform
  const double* src = warp < a.n_branches
                          ? a.gpart + (size_t)warp * a.n_tiles
                          : a.lpart;
  if (a.gpart_pairs && warp < a.n_branches) {
    // float-pair tile sums: summed as pairs (error-free transformations,
    // ~48 bits), converted to FP64 once
    const float2* s2 = reinterpret_cast<const float2*>(src);
    F2 acc = {0.f, 0.f};
    for (int i = lane; i < a.n_tiles; i += 32) {
      const float2 p = s2[i];
      acc = f2_add(acc, F2{p.x, p.y});
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
      acc = f2_add(acc, F2{__shfl_xor_sync(kFull, acc.hi, o), __shfl_xor_sync(kFull, acc.lo, o)});
    if (lane == 0) a.out[1 + warp] = (double)acc.hi + (double)acc.lo;
    return;
  }
  double acc = 0.0;
  for (int i = lane; i < a.n_tiles; i += 32) acc += src[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
  if (lane == 0) a.out[warp < a.n_branches ? 1 + warp : 0] = acc;
}

cudaError_t launch_reduce(const ReduceArgs& a, cudaStream_t st) {
  const int warps = a.n_branches + 1;
  const int blocks = (warps * 32 + 255) / 256;
  return launch_pdl(reduce_kernel, dim3(blocks), dim3(256), 0, st, a);
}

// ---------------------------------------------------------------------------
// Chain-rule epilogues (branch parameterisations of the paper's Methods):
// FP64, a few thousand values, one pass each.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) grad_rate_time_kernel(const double* g, int n_br,
                                                             const double* rates,
                                                             const double* times,
                                                             double* d_rates, double* d_times) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n_br) return;
  if (d_rates) d_rates[i] = times[i] * g[i];
  if (d_times) d_times[i] = rates[i] * g[i];
}

// d log P / d h_k = -rate_k g_k + sum_{c child of k} rate_c g_c; the root
// (node 2N-2) has no branch of its own.
__global__ void __launch_bounds__(256) grad_heights_kernel(const double* g,
                                                           const int2* children, int n_tips,
                                                           const double* rates,
                                                           double* d_heights) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_nodes = 2 * n_tips - 1, root = n_nodes - 1;
  if (k >= n_nodes) return;
  double acc = 0.0;
  if (k != root) acc = -(rates ? rates[k] : 1.0) * g[k];
  if (k >= n_tips) {
    const int2 ch = children[k];
    acc += (rates ? rates[ch.x] : 1.0) * g[ch.x];
    acc += (rates ? rates[ch.y] : 1.0) * g[ch.y];
  }
  d_heights[k] = acc;
}

// One block; thread t sums entries t, t + 256, ... then a fixed-order tree.
__global__ void __launch_bounds__(256) grad_branch_sum_kernel(const double* g,
                                                              const int* branches,
                                                              const double* weights, int n,
                                                              double* out) {
  __shared__ double red[256];
  double acc = 0.0;
  for (int j = threadIdx.x; j < n; j += 256) acc += (weights ? weights[j] : 1.0) * g[branches[j]];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0];
}

cudaError_t launch_grad_rate_time(const double* g, int n_br, const double* rates,
                                  const double* times, double* d_rates, double* d_times,
                                  cudaStream_t st) {
  if (n_br <= 0) return cudaSuccess;
  grad_rate_time_kernel<<<(n_br + 255) / 256, 256, 0, st>>>(g, n_br, rates, times, d_rates,
                                                            d_times);
  return cudaGetLastError();
}

cudaError_t launch_grad_heights(const double* g, const int2* children, int n_tips,
                                const double* rates, double* d_heights, cudaStream_t st) {
  const int n_nodes = 2 * n_tips - 1;
  grad_heights_kernel<<<(n_nodes + 255) / 256, 256, 0, st>>>(g, children, n_tips, rates,
                                                             d_heights);
  return cudaGetLastError();
}

cudaError_t launch_grad_branch_sum(const double* g, const int* branches, const double* weights,
                                   int n, double* out, cudaStream_t st) {
  grad_branch_sum_kernel<<<1, 256, 0, st>>>(g, branches, weights, n, out);
  return cudaGetLastError();
}

}  // namespace phylo
