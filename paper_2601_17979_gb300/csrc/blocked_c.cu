// blocked_c.cu -- multi-kernel batched Jacobi SVD for scalar type float2.
#include "blocked_launch.cuh"

BSVD_DEFINE_BLOCKED(float2, c)
