// internal.h -- declarations shared by the C-ABI layer and the per-type
// kernel translation units.  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

namespace bsvd {

struct FusedArgs;
struct BlockedArgs;

// Bytes of workspace the multi-kernel path needs for `count` matrices of one
// shape (defined in bsvd_api.cu from the same layout as blocked_launch.cuh).
size_t blocked_bytes(int nb, int M, int N, int count, bool two_stage, size_t elt);

#define BSVD_DECLARE_FUSED(TAG)                                                          \
    size_t fused_plan_##TAG(int nb, int M, int N, bool needVs, FusedArgs& a, int& nt);  \
    cudaError_t fused_launch_##TAG(int nb, const FusedArgs& a, int grid, size_t smem,   \
                                   cudaStream_t st);

#define BSVD_DECLARE_BLOCKED(TAG)                                                               \
    cudaError_t blocked_run_##TAG(int nb, const BlockedArgs& a, void* work, cudaStream_t st,   \
                                  bool two_stage, bool host_sync);

BSVD_DECLARE_BLOCKED(s)
BSVD_DECLARE_BLOCKED(d)
BSVD_DECLARE_BLOCKED(c)
BSVD_DECLARE_BLOCKED(z)

#undef BSVD_DECLARE_BLOCKED

BSVD_DECLARE_FUSED(s)
BSVD_DECLARE_FUSED(d)
BSVD_DECLARE_FUSED(c)
BSVD_DECLARE_FUSED(z)

#undef BSVD_DECLARE_FUSED

}  // namespace bsvd
