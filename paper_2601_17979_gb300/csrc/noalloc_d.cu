// noalloc_d.cu -- a double-precision batched SVD entry point that allocates
// nothing on the device.
//
// Some callers cannot call cudaMalloc: code running inside a host framework
// that owns the whole device-memory budget (an inference server or a plugin
// whose memory is reserved up front), code on a latency path where
// cudaMalloc's implicit device synchronisation is not acceptable, or callers
// that simply have no allocator at hand to size and pass a workspace.  For
// them this file keeps the multi-kernel path's workspace in a fixed
// file-scope __device__ array, which every GPU that loads the library holds
// until the process exits, and forwards to bsvd_dgesvj_strided with it.
#include <cuda_runtime.h>

#include <cstring>

#include "bsvd.h"

namespace {

// Capacity of the static scratch.  A 128x64 FP64 matrix needs about 165 KB
// on the multi-kernel path, so this holds batches of up to 203 such
// matrices; larger batches are rejected with BSVD_ERR_WORKSPACE.
constexpr size_t kStaticScratchBytes = size_t(32) << 20;   // 32 MiB

}  // namespace

static __device__ __align__(256) unsigned char g_bsvd_static_scratch[kStaticScratchBytes];

// The array's name in host code is only a host-side stand-in: its device
// address is looked up with the calling thread's device current.  It is
// looked up on every call, not cached: after cudaDeviceReset, or in another
// context, the module is loaded again and the address may change, and a
// cached pointer would then point at memory this call does not own.  The
// lookup may load the module on a device's first call, so that first call
// should come before any stream capture.
static bsvd_status static_scratch(void** ptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_bsvd_static_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return BSVD_ERR_CUDA;
    }
    *ptr = p;
    return BSVD_OK;
}

extern "C" bsvd_status bsvd_dgesvj_strided_noalloc(
    bsvd_handle handle, bsvd_job jobu, bsvd_job jobv, int batch, int m, int n, const double* dA,
    int lda, long long strideA, double* dS, long long strideS, double* dU, int ldu,
    long long strideU, double* dV, int ldv, long long strideV, int* d_info, int* d_sweeps,
    const bsvd_opts* opts, void* stream) {
    // Always the multi-kernel path (the one that needs scratch): the paper's
    // baseline when PLAIN is asked for, Designs 2-4 otherwise.
    bsvd_opts o;
    if (opts) o = *opts;
    else std::memset(&o, 0, sizeof o);
    if (o.path != BSVD_PATH_PLAIN) o.path = BSVD_PATH_BLOCKED;
    o.flags |= 8;   // no CUDA graph: instantiating one may allocate device memory
    void* scratch = nullptr;
    if (batch > 0 && m > 0 && n > 0) {
        const bsvd_status st = static_scratch(&scratch);
        if (st != BSVD_OK) return st;
    }
    // Every call shares the array.  The multi-kernel path initialises all the
    // workspace it reads (status words, flags, W, V, Gram and rotation blocks)
    // before reading it, so stale contents of an earlier call never matter;
    // calls that overlap on the GPU (other streams, other host threads) race
    // on the array and must be serialised by the caller.
    return bsvd_dgesvj_strided(handle, jobu, jobv, batch, m, n, dA, lda, strideA, dS, strideS, dU,
                               ldu, strideU, dV, ldv, strideV, d_info, d_sweeps, scratch,
                               scratch ? kStaticScratchBytes : 0, &o, stream);
}
