// launch_util.cuh -- host helpers shared by the launch code.
#pragma once

#include <cuda_runtime.h>

#include <atomic>

namespace bsvd {

// Lets kernel K take as much dynamic shared memory as the device allows (the
// opt-in limit less K's static shared memory), once per device.  Every caller
// sets the same maximum, so launches from several host threads cannot race: a
// per-call value set by one thread between another thread's set and launch
// could fall below that launch's need and make it fail.  The launch's own
// size still decides the occupancy.
template <auto K>
cudaError_t allow_dynamic_smem() {
    static std::atomic<unsigned long long> done{0};      // one bit per device (< 64)
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = dev < 64 ? 1ull << dev : 0ull;
    if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
    cudaFuncAttributes fa;
    if ((e = cudaFuncGetAttributes(&fa, K)) != cudaSuccess) return e;
    int optin = 0;
    if ((e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev)) != cudaSuccess) return e;
    e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
    if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_release);
    return e;
}

}  // namespace bsvd
