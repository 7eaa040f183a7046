// internal.h -- declarations shared by the C-ABI layer and the per-type
// kernel translation units.  Not part of the public interface.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "bsvd.h"

namespace bsvd {

struct FusedArgs;
struct BlockedArgs;
struct BlkVarPlan;
struct PersistArgs;

// Buffers of the mixed-precision path (strided batches; per matrix, in the
// working orientation M = max(m, n) rows, N = min(m, n) columns).
struct MixedArgs {
    int m, n, M, N, trans;
    const void* A; long long sA; int lda;   // the caller's FP64 / complex128 A (strided), or
    const void* const* Ap; const int* ldap; // pointer arrays by matrix id, with
    const int* index;                       // the ids of this launch's matrices
    void* A32;                              // M x N, ld M: FP32 copy of 2^-ex A (or A^H)
    void* V32;                              // N x N, ld N: V of the FP32 solve
    void* V64; void* Vtmp; void* E;         // N x N, ld N, FP64: restored V and scratch
    void* Ahat;                             // M x N, ld M, FP64: A V
};

// Buffers of the QR pre-processing path (strided batches; working
// orientation M = max(m, n) rows, N = min(m, n) columns).
struct QrArgs {
    int m, n, M, N, trans;
    const void* A; long long sA; int lda;   // the caller's A
    void* W;                                // M x N, ld M: reflectors below the diagonal
    void* tau;                              // N scalars per matrix
    void* R;                                // N x N, ld N: the triangular factor
    int* ex;                                // the power-of-two scaling of each matrix
    void* Uhat;                             // N x N, ld N: left vectors of R
    void* Y; long long sY; int ldy;         // Q [Uhat; 0]: the caller's U (V when m < n), or null
    void* S; long long sS;                  // singular values, rescaled by 2^ex
};

cudaError_t qr_factor_s(const QrArgs& a, int batch, cudaStream_t st);
cudaError_t qr_factor_d(const QrArgs& a, int batch, cudaStream_t st);
cudaError_t qr_factor_c(const QrArgs& a, int batch, cudaStream_t st);
cudaError_t qr_factor_z(const QrArgs& a, int batch, cudaStream_t st);
cudaError_t qr_apply_s(const QrArgs& a, int batch, cudaStream_t st);
cudaError_t qr_apply_d(const QrArgs& a, int batch, cudaStream_t st);
cudaError_t qr_apply_c(const QrArgs& a, int batch, cudaStream_t st);
cudaError_t qr_apply_z(const QrArgs& a, int batch, cudaStream_t st);

cudaError_t mixed_prepare_d(const MixedArgs& a, int batch, cudaStream_t st);
cudaError_t mixed_prepare_z(const MixedArgs& a, int batch, cudaStream_t st);
cudaError_t mixed_restore_d(const MixedArgs& a, int batch, cudaStream_t st);
cudaError_t mixed_restore_z(const MixedArgs& a, int batch, cudaStream_t st);

// Bytes of workspace the multi-kernel path needs for `count` matrices of one
// shape (defined in bsvd_api.cu from the same layout as blocked_launch.cuh).
size_t blocked_bytes(int nb, int M, int N, int count, bool two_stage, size_t elt);

// The persistent launch of a pointer-array batch (as bsvd_?gesvj_batched with
// path PERSISTENT) that also raises d_done[i] once matrix i's outputs are
// written (d_done zeroed by the caller, typically host-mapped memory) and
// starts no further matrix once *d_abort is nonzero (d_abort may be null).
bsvd_status persistent_with_flags(bsvd_handle h, char t, bool wantU, bool wantV, int batch, const int* m,
                                  const int* n, const void* const* dA, const int* lda, void* const* dS,
                                  void* const* dU, const int* ldu, void* const* dV, const int* ldv,
                                  int* d_info, int* d_sweeps, int* d_done, const int* d_abort,
                                  void* d_work, size_t work_bytes, const bsvd_opts* opts, cudaStream_t s);

#define BSVD_DECLARE_FUSED(TAG)                                                          \
    size_t fused_plan_##TAG(int nb, int M, int N, bool needVs, FusedArgs& a, int& nt);  \
    cudaError_t fused_launch_##TAG(int nb, const FusedArgs& a, int grid, size_t smem,   \
                                   cudaStream_t st);                                    \
    cudaError_t persist_launch_##TAG(int nb, bool onchip, size_t wv, const PersistArgs& p, int grid, \
                                     int maxN, cudaStream_t st);                        \
    long long persist_slot_##TAG(int nb, int m, int n);                                 \
    size_t persist_smem_##TAG(int nb, size_t wv, int maxN);

#define BSVD_DECLARE_BLOCKED(TAG)                                                               \
    cudaError_t blocked_run_##TAG(int nb, const BlockedArgs& a, void* work, cudaStream_t st,   \
                                  bool two_stage, bool host_sync, cudaStream_t capture);       \
    cudaError_t blocked_run_var_##TAG(int nb, const BlockedArgs& a, const BlkVarPlan& var,      \
                                      void* work, cudaStream_t st, cudaStream_t capture);

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
