// blocked_s.cu -- multi-kernel batched Jacobi SVD for scalar type float.
#include "blocked_launch.cuh"

BSVD_DEFINE_BLOCKED(float, s)
