// blocked_z.cu -- multi-kernel batched Jacobi SVD for scalar type double2.
#include "blocked_launch.cuh"

BSVD_DEFINE_BLOCKED(double2, z)
