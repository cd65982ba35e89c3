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

}  // namespace phylo
