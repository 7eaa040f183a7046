// internal.h -- declarations shared by the C-ABI layer and the per-type
// kernel translation units.  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace bsvd {

struct FusedArgs;

#define BSVD_DECLARE_FUSED(TAG)                                                          \
    size_t fused_plan_##TAG(int nb, int M, int N, bool needVs, FusedArgs& a, int& nt);  \
    cudaError_t fused_launch_##TAG(int nb, const FusedArgs& a, int grid, size_t smem,   \
                                   cudaStream_t st);

BSVD_DECLARE_FUSED(s)
BSVD_DECLARE_FUSED(d)
BSVD_DECLARE_FUSED(c)
BSVD_DECLARE_FUSED(z)

#undef BSVD_DECLARE_FUSED

}  // namespace bsvd
