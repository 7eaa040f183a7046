// fused_launch.cuh -- shared-memory planning and launch of the fused kernel,
// instantiated once per scalar type by fused_{s,d,c,z}.cu.
#pragma once

#include <algorithm>
#include <type_traits>

#include "gesvj_fused.cuh"
#include "internal.h"
#include "launch_util.cuh"

namespace bsvd {

// Thread organisation per block width: NG groups of GT threads, one group
// per block pair of a round-robin round.
template <int NB> struct FusedCfg;
template <> struct FusedCfg<4>  { static constexpr int NG = 2, GT = 32; };
template <> struct FusedCfg<8>  { static constexpr int NG = 2, GT = 64; };
template <> struct FusedCfg<16> { static constexpr int NG = 2, GT = 128; };

// A matrix of at most 2nb columns has a single block pair per round, so one
// of two groups would idle: FP64 and complex then run one group of all the
// threads (same per-entry arithmetic; FP32's register tiles would sum in
// another order, so FP32 keeps the two-group shape).
template <class T>
__host__ __device__ inline bool fused_single_group(const FusedArgs& a) {
    return !std::is_same<T, float>::value && a.l == 2;
}

inline size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <class T, int NB>
size_t fused_plan_nb(int M, int N, bool needVs, FusedArgs& a, int& nthreads) {
    using C = FusedCfg<NB>;
    using R = Real<T>;
    fused_dims<T, NB>(M, N, a);    // (M, N): the working orientation
    const int ng = fused_single_group<T>(a) ? 1 : C::NG;
    size_t off = 0;
    a.offW = 0;
    off = align16((size_t)a.ldw * a.Np * sizeof(T));
    a.offV = (int)off;
    if (needVs) off = align16(off + (size_t)a.ldvs * a.Np * sizeof(T));
    a.offG = (int)off;
    a.groupBytes = fused_group_bytes<T, NB>();
    off += (size_t)ng * a.groupBytes;
    a.offMisc = (int)off;
    const int NT = C::NG * C::GT, NW = NT / 32;
    off += kMaxSweeps * 4 + 16 + 2 * sizeof(T);
    off += (size_t)((NW + 3) & ~3) * sizeof(R) + (size_t)((N + 3) & ~3) * sizeof(R) + (size_t)N * 4;
    nthreads = NT;
    return align16(off);
}

template <class T>
size_t fused_plan(int nb, int M, int N, bool needVs, FusedArgs& a, int& nthreads) {
    switch (nb) {
        case 4: return fused_plan_nb<T, 4>(M, N, needVs, a, nthreads);
        case 8: return fused_plan_nb<T, 8>(M, N, needVs, a, nthreads);
        case 16: return fused_plan_nb<T, 16>(M, N, needVs, a, nthreads);
        default: return 0;
    }
}

// Shared memory of a persistent launch: the working arrays of the segment's
// largest matrix when on chip (wv bytes, 0 for global slots), the groups'
// Gram/rotation scratch and the per-matrix flags sized for the largest N.
template <class T, int NB>
size_t persist_smem_nb(int maxN, size_t wv, FusedArgs& a, int& nthreads) {
    using C = FusedCfg<NB>;
    using R = Real<T>;
    a.offW = a.offV = 0;
    a.offG = (int)align16(wv);
    a.groupBytes = fused_group_bytes<T, NB>();
    size_t off = a.offG + (size_t)C::NG * a.groupBytes;
    a.offMisc = (int)off;
    const int NT = C::NG * C::GT, NW = NT / 32;
    off += kMaxSweeps * 4 + 16 + 2 * sizeof(T);
    off += (size_t)((NW + 3) & ~3) * sizeof(R) + (size_t)((maxN + 3) & ~3) * sizeof(R) + (size_t)maxN * 4;
    nthreads = NT;
    return align16(off);
}

// On chip the grid follows the kernel's occupancy at this shared-memory size
// (small block widths run 64 or 128 threads per CTA and fit many CTAs per
// SM); `grid` is then the cap (the segment's matrix count).  Global-slot
// launches use `grid` as planned: the workspace holds that many slots.
template <class T, int NB, bool OnChip>
cudaError_t persist_launch_nb(const PersistArgs& p, int grid, size_t smem, cudaStream_t st) {
    using C = FusedCfg<NB>;
    constexpr auto k = gesvj_persistent_kernel<T, NB, C::NG, C::GT, OnChip>;
    cudaError_t e = allow_dynamic_smem<k>();
    if (e != cudaSuccess) return e;
    if (OnChip) {
        int dev = 0, sms = 0, occ = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess ||
            (e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess ||
            (e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k, C::NG * C::GT, smem)) != cudaSuccess)
            return e;
        grid = std::max(1, std::min(grid, sms * std::max(occ, 1)));
    }
    k<<<grid, C::NG * C::GT, smem, st>>>(p);
    return cudaGetLastError();
}

// Slot elements for matrix (m, n) with block width NB.
template <class T, int NB>
long long persist_slot_nb(int m, int n) {
    FusedArgs a;
    fused_dims<T, NB>(m, n, a);
    return fused_slot_elems<T>(a);
}

template <class T>
size_t persist_smem(int nb, size_t wv, int maxN) {
    FusedArgs a;
    int nt = 0;
    switch (nb) {
        case 4: return persist_smem_nb<T, 4>(maxN, wv, a, nt);
        case 8: return persist_smem_nb<T, 8>(maxN, wv, a, nt);
        case 16: return persist_smem_nb<T, 16>(maxN, wv, a, nt);
        default: return 0;
    }
}

template <class T, bool OnChip>
cudaError_t persist_launch_on(int nb, PersistArgs p, int grid, size_t wv, int maxN, cudaStream_t st) {
    int nt = 0;
    switch (nb) {
        case 4: { size_t sm = persist_smem_nb<T, 4>(maxN, wv, p.base, nt); return persist_launch_nb<T, 4, OnChip>(p, grid, sm, st); }
        case 8: { size_t sm = persist_smem_nb<T, 8>(maxN, wv, p.base, nt); return persist_launch_nb<T, 8, OnChip>(p, grid, sm, st); }
        case 16: { size_t sm = persist_smem_nb<T, 16>(maxN, wv, p.base, nt); return persist_launch_nb<T, 16, OnChip>(p, grid, sm, st); }
        default: return cudaErrorInvalidValue;
    }
}

template <class T>
cudaError_t persist_launch(int nb, bool onchip, size_t wv, PersistArgs p, int grid, int maxN, cudaStream_t st) {
    return onchip ? persist_launch_on<T, true>(nb, p, grid, wv, maxN, st)
                  : persist_launch_on<T, false>(nb, p, grid, 0, maxN, st);
}

template <class T>
long long persist_slot(int nb, int m, int n) {
    switch (nb) {
        case 4: return persist_slot_nb<T, 4>(m, n);
        case 8: return persist_slot_nb<T, 8>(m, n);
        case 16: return persist_slot_nb<T, 16>(m, n);
        default: return -1;
    }
}

// Bytes of W and V of matrix (m, n) on chip (the on-chip kernel's layout:
// V after W at a 16-byte boundary), or 0 for an unsupported block width.
template <class T>
size_t persist_onchip_bytes(int nb, int m, int n) {
    const long long e = persist_slot<T>(nb, m, n);
    return e < 0 ? 0 : (size_t)e * sizeof(T);
}

template <class T, int NB>
cudaError_t fused_launch_nb(const FusedArgs& a, int grid, size_t smem, cudaStream_t st) {
    using C = FusedCfg<NB>;
    if constexpr (!std::is_same<T, float>::value) {
        if (fused_single_group<T>(a)) {
            constexpr auto k1 = gesvj_fused_kernel<T, NB, 1, C::NG * C::GT>;
            cudaError_t e = allow_dynamic_smem<k1>();
            if (e != cudaSuccess) return e;
            k1<<<grid, C::NG * C::GT, smem, st>>>(a);
            return cudaGetLastError();
        }
    }
    constexpr auto k = gesvj_fused_kernel<T, NB, C::NG, C::GT>;
    cudaError_t e = allow_dynamic_smem<k>();
    if (e != cudaSuccess) return e;
    k<<<grid, C::NG * C::GT, smem, st>>>(a);
    return cudaGetLastError();
}

template <class T>
cudaError_t fused_launch(int nb, const FusedArgs& a, int grid, size_t smem, cudaStream_t st) {
    switch (nb) {
        case 4: return fused_launch_nb<T, 4>(a, grid, smem, st);
        case 8: return fused_launch_nb<T, 8>(a, grid, smem, st);
        case 16: return fused_launch_nb<T, 16>(a, grid, smem, st);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace bsvd

// One TU per type defines these with FUSED_TYPE / FUSED_TAG.
#define BSVD_DEFINE_FUSED(TYPE, TAG)                                                           \
    size_t bsvd::fused_plan_##TAG(int nb, int M, int N, bool needVs, FusedArgs& a, int& nt) { \
        return fused_plan<TYPE>(nb, M, N, needVs, a, nt);                                    \
    }                                                                                        \
    cudaError_t bsvd::persist_launch_##TAG(int nb, bool onchip, size_t wv, const PersistArgs& p, int grid, \
                                           int maxN, cudaStream_t st) {                      \
        return persist_launch<TYPE>(nb, onchip, wv, p, grid, maxN, st);                      \
    }                                                                                        \
    long long bsvd::persist_slot_##TAG(int nb, int m, int n) { return persist_slot<TYPE>(nb, m, n); } \
    size_t bsvd::persist_smem_##TAG(int nb, size_t wv, int maxN) { return persist_smem<TYPE>(nb, wv, maxN); } \
    cudaError_t bsvd::fused_launch_##TAG(int nb, const FusedArgs& a, int grid, size_t smem,  \
                                         cudaStream_t st) {                                  \
        return fused_launch<TYPE>(nb, a, grid, smem, st);                                    \
    }
