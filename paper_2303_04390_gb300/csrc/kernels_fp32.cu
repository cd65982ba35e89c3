// FP32 instantiation of the level kernels and the matrix builder.
#include "kernels.cuh"

PHYLO_INSTANTIATE(float)
