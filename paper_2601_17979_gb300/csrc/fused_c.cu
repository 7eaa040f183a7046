// fused_c.cu -- fused batched Jacobi SVD kernels for scalar type float2.
#include "fused_launch.cuh"

BSVD_DEFINE_FUSED(float2, c)
