// fused_s.cu -- fused batched Jacobi SVD kernels for scalar type float.
#include "fused_launch.cuh"

BSVD_DEFINE_FUSED(float, s)
