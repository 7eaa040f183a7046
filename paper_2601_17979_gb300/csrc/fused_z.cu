// fused_z.cu -- fused batched Jacobi SVD kernels for scalar type double2.
#include "fused_launch.cuh"

BSVD_DEFINE_FUSED(double2, z)
