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

#include <algorithm>

#include "internal.h"
#include "jacobi_common.cuh"

namespace bsvd {

__device__ __forceinline__ float narrow_s(double x) { return __double2float_rn(x); }
__device__ __forceinline__ float2 narrow_s(double2 x) { return make_float2(__double2float_rn(x.x), __double2float_rn(x.y)); }
__device__ __forceinline__ double widen_s(float x) { return (double)x; }
__device__ __forceinline__ double2 widen_s(float2 x) { return make_double2((double)x.x, (double)x.y); }

constexpr int kMxThreads = 256;

// Matrix b of the launch: the caller's strided batch, or by id through the
// pointer array.
template <class T64>
__device__ __forceinline__ const T64* mixed_a(const MixedArgs& a, int b) {
    return a.Ap ? static_cast<const T64*>(a.Ap[a.index[b]]) : static_cast<const T64*>(a.A) + (long long)b * a.sA;
}

// A32 (M x N, ld M) = fl32(2^-ex A) or fl32(2^-ex A^H) when m < n, ex the
// exponent of max |a_ij| (exact scaling: FP32's range holds the result).
template <class T64, class T32>
__global__ void __launch_bounds__(kMxThreads) mx_convert(const MixedArgs a) {
    using R = Real<T64>;
    constexpr int NT = kMxThreads, NW = NT / 32;
    __shared__ R red[NW];
    __shared__ int ex_s;
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const T64* A = mixed_a<T64>(a, b);
    const int lda = a.Ap ? a.ldap[a.index[b]] : a.lda;
    R mx = 0;
    for (int e = tid; e < a.m * a.n; e += NT) {
        const T64 x = A[(e % a.m) + (long long)(e / a.m) * lda];
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
        const T64 x = scalb_s(A[i + (long long)j * lda], -ex);
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
    const T64* A = mixed_a<T64>(a, b);
    const int lda = a.Ap ? a.ldap[a.index[b]] : a.lda;
    T64* Ah = static_cast<T64*>(a.Ahat) + (long long)b * M * N;
    for (int e = tid; e < M * N; e += NT) {
        const int i = e % M, k = e / M;
        T64 acc = make_s<T64>(0);
        for (int j = 0; j < N; ++j) {
            const T64 aij = a.trans ? conj_s(A[j + (long long)i * lda]) : A[i + (long long)j * lda];
            acc = fma_s(aij, Va[j + (long long)k * N], acc);
        }
        Ah[i + (long long)k * M] = acc;
    }
}

// ---- the restoration tiled over the whole GPU (N >= kMxTiledN) ---------------
// For large N one CTA per matrix leaves most SMs idle for O(N^3) work, so the
// same steps run as 64 x 64 output tiles over (matrix, tile, tile) grids:
// widen, E = V^H V - I, V <- V - V E / 2 (twice), A_hat = A' V.  Each output
// keeps one accumulator summed over the contraction index in increasing
// order with the same multiply-adds as mx_restore, so the results are the
// single-CTA kernel's bits.
constexpr int kMxBT = 64, kMxKC = 16, kMxTiledN = 128;

template <class T64, class T32>
__global__ void __launch_bounds__(kMxThreads) mx_widen(const MixedArgs a) {
    const long long nn = (long long)a.N * a.N;
    const T32* V32 = static_cast<const T32*>(a.V32) + blockIdx.x * nn;
    T64* Va = static_cast<T64*>(a.V64) + blockIdx.x * nn;
    for (long long e = blockIdx.y * (long long)kMxThreads + threadIdx.x; e < nn; e += (long long)gridDim.y * kMxThreads)
        Va[e] = widen_s(V32[e]);
}

// acc[u][v] += sum over the chunk of X(r0 + tr + 16u, k) Y(k, c0 + tc + 16v),
// X and Y staged as Xs[k][row], Ys[k][col]; conj_x: X entries conjugated.
template <class T, bool ConjX>
__device__ __forceinline__ void mx_mac(T (&acc)[4][4], const T (*Xs)[kMxBT + 1], const T (*Ys)[kMxBT + 1], int tr,
                                       int tc, int kc) {
    for (int k = 0; k < kc; ++k) {
        T x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = Xs[k][tr + 16 * u];
#pragma unroll
        for (int v = 0; v < 4; ++v) y[v] = Ys[k][tc + 16 * v];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = ConjX ? cfma(x[u], y[v], acc[u][v]) : fma_s(x[u], y[v], acc[u][v]);
    }
}

// E (N x N) = V^H V - I for V = V64 (it = 0, 2: the buffer holding the
// current iterate), upper tiles computed and mirrored.
template <class T64>
__global__ void __launch_bounds__(kMxThreads) mx_gram_tiled(const MixedArgs a, int cur) {
    using R = Real<T64>;
    const int b = blockIdx.x, ta = blockIdx.y, tb = blockIdx.z, tid = threadIdx.x, tr = tid & 15, tc = tid >> 4;
    if (ta > tb) return;
    const int N = a.N, r0 = ta * kMxBT, c0 = tb * kMxBT;
    const long long nn = (long long)N * N;
    const T64* V = static_cast<const T64*>(cur ? a.Vtmp : a.V64) + b * nn;
    T64* E = static_cast<T64*>(a.E) + b * nn;
    __shared__ T64 Xs[kMxKC][kMxBT + 1], Ys[kMxKC][kMxBT + 1];
    const T64 zero = make_s<T64>(0);
    T64 acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = zero;
    for (int i0 = 0; i0 < N; i0 += kMxKC) {
        for (int e = tid; e < kMxKC * kMxBT; e += kMxThreads) {
            const int kk = e % kMxKC, cc = e / kMxKC, i = i0 + kk;
            Xs[kk][cc] = (i < N && r0 + cc < N) ? V[i + (long long)(r0 + cc) * N] : zero;
            Ys[kk][cc] = (i < N && c0 + cc < N) ? V[i + (long long)(c0 + cc) * N] : zero;
        }
        __syncthreads();
        mx_mac<T64, true>(acc, Xs, Ys, tr, tc, min(kMxKC, N - i0));
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = r0 + tr + 16 * u, c = c0 + tc + 16 * v;
            if (r >= N || c >= N || r > c) continue;
            T64 x = acc[u][v];
            if (r == c) x = make_s<T64>(re(x) - R(1));
            E[r + (long long)c * N] = x;
            E[c + (long long)r * N] = conj_s(x);
        }
}

// Vnext = Vcur - Vcur E / 2 (cur = 0: V64 -> Vtmp; 1: Vtmp -> V64)
template <class T64>
__global__ void __launch_bounds__(kMxThreads) mx_ns_tiled(const MixedArgs a, int cur) {
    using R = Real<T64>;
    const int b = blockIdx.x, ti = blockIdx.y, tk = blockIdx.z, tid = threadIdx.x, tr = tid & 15, tc = tid >> 4;
    const int N = a.N, r0 = ti * kMxBT, c0 = tk * kMxBT;
    const long long nn = (long long)N * N;
    const T64* V = static_cast<const T64*>(cur ? a.Vtmp : a.V64) + b * nn;
    T64* Vn = static_cast<T64*>(cur ? a.V64 : a.Vtmp) + b * nn;
    const T64* E = static_cast<const T64*>(a.E) + b * nn;
    __shared__ T64 Xs[kMxKC][kMxBT + 1], Ys[kMxKC][kMxBT + 1];
    const T64 zero = make_s<T64>(0);
    T64 acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = zero;
    for (int j0 = 0; j0 < N; j0 += kMxKC) {
        for (int e = tid; e < kMxKC * kMxBT; e += kMxThreads) {
            const int kk = e / kMxBT, cc = e % kMxBT, j = j0 + kk;
            Xs[kk][cc] = (j < N && r0 + cc < N) ? V[(r0 + cc) + (long long)j * N] : zero;
            Ys[kk][cc] = (j < N && c0 + cc < N) ? E[j + (long long)(c0 + cc) * N] : zero;
        }
        __syncthreads();
        mx_mac<T64, false>(acc, Xs, Ys, tr, tc, min(kMxKC, N - j0));
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = r0 + tr + 16 * u, k = c0 + tc + 16 * v;
            if (i >= N || k >= N) continue;
            Vn[i + (long long)k * N] = sub(V[i + (long long)k * N], scale(acc[u][v], R(0.5)));
        }
}

// A_hat (M x N) = A' V64, A' = A or A^H
template <class T64>
__global__ void __launch_bounds__(kMxThreads) mx_ahat_tiled(const MixedArgs a) {
    const int b = blockIdx.x, ti = blockIdx.y, tk = blockIdx.z, tid = threadIdx.x, tr = tid & 15, tc = tid >> 4;
    const int M = a.M, N = a.N, r0 = ti * kMxBT, c0 = tk * kMxBT;
    const long long nn = (long long)N * N;
    const T64* A = mixed_a<T64>(a, b);
    const int lda = a.Ap ? a.ldap[a.index[b]] : a.lda;
    const T64* V = static_cast<const T64*>(a.V64) + b * nn;
    T64* Ah = static_cast<T64*>(a.Ahat) + (long long)b * M * N;
    __shared__ T64 Xs[kMxKC][kMxBT + 1], Ys[kMxKC][kMxBT + 1];
    const T64 zero = make_s<T64>(0);
    T64 acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = zero;
    for (int j0 = 0; j0 < N; j0 += kMxKC) {
        for (int e = tid; e < kMxKC * kMxBT; e += kMxThreads) {
            const int kk = e / kMxBT, cc = e % kMxBT, j = j0 + kk, i = r0 + cc;
            T64 x = zero;
            if (j < N && i < M) x = a.trans ? conj_s(A[j + (long long)i * lda]) : A[i + (long long)j * lda];
            Xs[kk][cc] = x;
            Ys[kk][cc] = (j < N && c0 + cc < N) ? V[j + (long long)(c0 + cc) * N] : zero;
        }
        __syncthreads();
        mx_mac<T64, false>(acc, Xs, Ys, tr, tc, min(kMxKC, N - j0));
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int i = r0 + tr + 16 * u, k = c0 + tc + 16 * v;
            if (i < M && k < N) Ah[i + (long long)k * M] = acc[u][v];
        }
}

template <class T64, class T32>
cudaError_t mixed_restore_tiled(const MixedArgs& a, int batch, cudaStream_t st) {
    const int tn = (a.N + kMxBT - 1) / kMxBT, tm = (a.M + kMxBT - 1) / kMxBT;
    const long long nn = (long long)a.N * a.N;
    const int wblocks = (int)std::min<long long>((nn + kMxThreads - 1) / kMxThreads, 1024);
    mx_widen<T64, T32><<<dim3(batch, wblocks), kMxThreads, 0, st>>>(a);
    for (int it = 0; it < 2; ++it) {      // two Newton-Schulz steps: V64 -> Vtmp -> V64
        mx_gram_tiled<T64><<<dim3(batch, tn, tn), kMxThreads, 0, st>>>(a, it);
        mx_ns_tiled<T64><<<dim3(batch, tn, tn), kMxThreads, 0, st>>>(a, it);
    }
    mx_ahat_tiled<T64><<<dim3(batch, tm, tn), kMxThreads, 0, st>>>(a);
    return cudaGetLastError();
}

template <class T64, class T32>
cudaError_t mixed_prepare(const MixedArgs& a, int batch, cudaStream_t st) {
    mx_convert<T64, T32><<<batch, kMxThreads, 0, st>>>(a);
    return cudaGetLastError();
}

template <class T64, class T32>
cudaError_t mixed_restore(const MixedArgs& a, int batch, cudaStream_t st) {
    if (a.N >= kMxTiledN) return mixed_restore_tiled<T64, T32>(a, batch, st);
    mx_restore<T64, T32><<<batch, kMxThreads, 0, st>>>(a);
    return cudaGetLastError();
}

cudaError_t mixed_prepare_d(const MixedArgs& a, int batch, cudaStream_t st) { return mixed_prepare<double, float>(a, batch, st); }
cudaError_t mixed_prepare_z(const MixedArgs& a, int batch, cudaStream_t st) { return mixed_prepare<double2, float2>(a, batch, st); }
cudaError_t mixed_restore_d(const MixedArgs& a, int batch, cudaStream_t st) { return mixed_restore<double, float>(a, batch, st); }
cudaError_t mixed_restore_z(const MixedArgs& a, int batch, cudaStream_t st) { return mixed_restore<double2, float2>(a, batch, st); }

}  // namespace bsvd
