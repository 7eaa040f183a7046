// mixed.cu -- kernels of the mixed-precision path for FP64 output.
//
// FP64 results from mostly-FP32 work: the FP32 solver runs on an FP32 copy
// of A until its own convergence test passes, giving V32; this file's
// kernels then restore an orthonormal V in FP64 (two Newton-Schulz steps
// V <- V - V (V^H V - I) / 2 from the widened V32) and form A_hat = A V in
// FP64; FP64 polish sweeps on A_hat, starting from that V, win the accuracy
// back (the FP64 test decides convergence).  On a GB300, whose FP64 rate is
// about 1/64 of its FP32 rate, the polish needs a few FP64 sweeps instead of
// the full count.
#include <cuda_runtime.h>

#include "internal.h"
#include "jacobi_common.cuh"

namespace bsvd {

__device__ __forceinline__ float narrow_s(double x) { return __double2float_rn(x); }
__device__ __forceinline__ float2 narrow_s(double2 x) { return make_float2(__double2float_rn(x.x), __double2float_rn(x.y)); }
__device__ __forceinline__ double widen_s(float x) { return (double)x; }
__device__ __forceinline__ double2 widen_s(float2 x) { return make_double2((double)x.x, (double)x.y); }

constexpr int kMxThreads = 256;

// A32 (M x N, ld M) = fl32(2^-ex A) or fl32(2^-ex A^H) when m < n, ex the
// exponent of max |a_ij| (exact scaling: FP32's range holds the result).
template <class T64, class T32>
__global__ void __launch_bounds__(kMxThreads) mx_convert(const MixedArgs a) {
    using R = Real<T64>;
    constexpr int NT = kMxThreads, NW = NT / 32;
    __shared__ R red[NW];
    __shared__ int ex_s;
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T64* A = static_cast<const T64*>(a.A) + (long long)b * a.sA;
    R mx = 0;
    for (int e = tid; e < a.m * a.n; e += NT) {
        const T64 x = A[(e % a.m) + (long long)(e / a.m) * a.lda];
        if (finite_s(x)) mx = fmax(mx, maxabs(x));
    }
    mx = warp_max(mx);
    if (lane == 0) red[warp] = mx;
    __syncthreads();
    if (tid == 0) {
        R m2 = 0;
        for (int w = 0; w < NW; ++w) m2 = fmax(m2, red[w]);
        ex_s = m2 > 0 ? ilogb_r(m2) : 0;
    }
    __syncthreads();
    const int ex = ex_s;
    T32* A32 = static_cast<T32*>(a.A32) + (long long)b * a.M * a.N;
    for (int e = tid; e < a.m * a.n; e += NT) {
        const int i = e % a.m, j = e / a.m;
        const T64 x = scalb_s(A[i + (long long)j * a.lda], -ex);
        if (a.trans) A32[j + (long long)i * a.M] = narrow_s(conj_s(x));
        else         A32[i + (long long)j * a.M] = narrow_s(x);
    }
}

// V (N x N) = two Newton-Schulz steps from widen(V32); A_hat (M x N, ld M) =
// A' V in FP64, A' = A or A^H.  One CTA per matrix on L2-resident buffers.
template <class T64, class T32>
__global__ void __launch_bounds__(kMxThreads) mx_restore(const MixedArgs a) {
    using R = Real<T64>;
    constexpr int NT = kMxThreads;
    const int b = blockIdx.x, tid = threadIdx.x;
    const int M = a.M, N = a.N;
    const long long nn = (long long)N * N;
    const T32* V32 = static_cast<const T32*>(a.V32) + b * nn;
    T64* Va = static_cast<T64*>(a.V64) + b * nn;
    T64* Vb = static_cast<T64*>(a.Vtmp) + b * nn;
    T64* E = static_cast<T64*>(a.E) + b * nn;
    for (int e = tid; e < N * N; e += NT) Va[e] = widen_s(V32[e]);
    __syncthreads();
    for (int it = 0; it < 2; ++it) {
        for (int e = tid; e < N * (N + 1) / 2; e += NT) {
            int ca, cb;
            tri_index(e, ca, cb);
            T64 acc = make_s<T64>(0);
            for (int i = 0; i < N; ++i) acc = cfma(Va[i + (long long)ca * N], Va[i + (long long)cb * N], acc);
            if (ca == cb) acc = make_s<T64>(re(acc) - R(1));
            E[ca + (long long)cb * N] = acc;
            E[cb + (long long)ca * N] = conj_s(acc);
        }
        __syncthreads();
        for (int e = tid; e < N * N; e += NT) {
            const int i = e % N, k = e / N;
            T64 acc = make_s<T64>(0);
            for (int j = 0; j < N; ++j) acc = fma_s(Va[i + (long long)j * N], E[j + (long long)k * N], acc);
            Vb[i + (long long)k * N] = sub(Va[i + (long long)k * N], scale(acc, R(0.5)));
        }
        __syncthreads();
        T64* t = Va; Va = Vb; Vb = t;     // two steps: the result is back in the V64 buffer
    }
    const T64* A = static_cast<const T64*>(a.A) + (long long)b * a.sA;
    T64* Ah = static_cast<T64*>(a.Ahat) + (long long)b * M * N;
    for (int e = tid; e < M * N; e += NT) {
        const int i = e % M, k = e / M;
        T64 acc = make_s<T64>(0);
        for (int j = 0; j < N; ++j) {
            const T64 aij = a.trans ? conj_s(A[j + (long long)i * a.lda]) : A[i + (long long)j * a.lda];
            acc = fma_s(aij, Va[j + (long long)k * N], acc);
        }
        Ah[i + (long long)k * M] = acc;
    }
}

template <class T64, class T32>
cudaError_t mixed_prepare(const MixedArgs& a, int batch, cudaStream_t st) {
    mx_convert<T64, T32><<<batch, kMxThreads, 0, st>>>(a);
    return cudaGetLastError();
}

template <class T64, class T32>
cudaError_t mixed_restore(const MixedArgs& a, int batch, cudaStream_t st) {
    mx_restore<T64, T32><<<batch, kMxThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t mixed_prepare_d(const MixedArgs& a, int batch, cudaStream_t st) { return mixed_prepare<double, float>(a, batch, st); }
cudaError_t mixed_prepare_z(const MixedArgs& a, int batch, cudaStream_t st) { return mixed_prepare<double2, float2>(a, batch, st); }
cudaError_t mixed_restore_d(const MixedArgs& a, int batch, cudaStream_t st) { return mixed_restore<double, float>(a, batch, st); }
cudaError_t mixed_restore_z(const MixedArgs& a, int batch, cudaStream_t st) { return mixed_restore<double2, float2>(a, batch, st); }

}  // namespace bsvd
