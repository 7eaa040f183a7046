// blocked_d.cu -- multi-kernel batched Jacobi SVD for scalar type double.
#include "blocked_launch.cuh"

BSVD_DEFINE_BLOCKED(double, d)
