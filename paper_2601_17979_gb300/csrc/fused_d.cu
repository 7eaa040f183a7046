// fused_d.cu -- fused batched Jacobi SVD kernels for scalar type double.
#include "fused_launch.cuh"

BSVD_DEFINE_FUSED(double, d)
