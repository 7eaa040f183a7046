// qr.cu -- QR pre-processing of tall matrices (Sec. "Pre-processing the SVD
// using a QR Factorization"): A = Q [R; 0] by Householder reflections (the
// non-pivoted factorization the paper uses), the SVD of the N x N factor R by
// the regular paths, then U = Q [U_R; 0].
//
// One CTA per matrix on L2-resident buffers.  For column j the CTA forms the
// reflector H_j = I - tau_j v_j v_j^H (v_j(j) = 1, beta_j real, the LAPACK
// larfg convention) and applies H_j^H to the trailing columns in passes of
// kQrChunk columns: one sweep over the rows accumulates v^H W for the whole
// chunk, one block reduction, one sweep applies the rank-1 update.  Q is
// never formed; qr_apply applies H_{N-1}, ..., H_0 to [U_R; 0] in turn.
// Where the matrix fits (at most 2,048 rows and the kQrSmemMax bytes below),
// the factorization works on a copy in shared memory and the application
// keeps Y there, staging each reflector through a double buffer that is
// filled while the previous reflector is applied; otherwise both work on
// L2-resident global buffers.
#include <cuda_runtime.h>

#include "internal.h"
#include "jacobi_common.cuh"
#include "launch_util.cuh"

namespace bsvd {

constexpr int kQrThreads = 256;
constexpr int kQrChunk = 16;
constexpr int kQrSmemMax = 200 * 1024;
constexpr int kQrRowsPerThread = 8;                        // the shared-memory variants: M <= 2,048

__device__ __forceinline__ float im_s(float) { return 0.f; }
__device__ __forceinline__ double im_s(double) { return 0.0; }
__device__ __forceinline__ float im_s(float2 x) { return x.y; }
__device__ __forceinline__ double im_s(double2 x) { return x.y; }

__device__ __forceinline__ float recip_s(float x) { return 1.f / x; }
__device__ __forceinline__ double recip_s(double x) { return 1.0 / x; }
__device__ __forceinline__ float2 recip_s(float2 x) {
    const float d = abs2(x);
    return make_float2(x.x / d, -x.y / d);
}
__device__ __forceinline__ double2 recip_s(double2 x) {
    const double d = abs2(x);
    return make_double2(x.x / d, -x.y / d);
}

template <class T> __device__ __forceinline__ T make_c(Real<T> r, Real<T> i);
template <> __device__ __forceinline__ float make_c<float>(float r, float) { return r; }
template <> __device__ __forceinline__ double make_c<double>(double r, double) { return r; }
template <> __device__ __forceinline__ float2 make_c<float2>(float r, float i) { return make_float2(r, i); }
template <> __device__ __forceinline__ double2 make_c<double2>(double r, double i) { return make_double2(r, i); }

__device__ __forceinline__ bool is_zero(float x) { return x == 0.f; }
__device__ __forceinline__ bool is_zero(double x) { return x == 0.0; }
__device__ __forceinline__ bool is_zero(float2 x) { return x.x == 0.f && x.y == 0.f; }
__device__ __forceinline__ bool is_zero(double2 x) { return x.x == 0.0 && x.y == 0.0; }

// Sums CH values per thread over the CTA (fixed order: lanes, then warps);
// the totals land in out[0..CH).  Ends with a barrier.
template <class T, int CH>
__device__ __forceinline__ void block_sum(T (&v)[CH], T* red, T* out) {
    constexpr int NW = kQrThreads / 32;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int c = 0; c < CH; ++c) v[c] = warp_sum_s(v[c]);
    if (lane == 0)
#pragma unroll
        for (int c = 0; c < CH; ++c) red[warp * CH + c] = v[c];
    __syncthreads();
    if (threadIdx.x < CH) {
        T acc = red[threadIdx.x];
        for (int w = 1; w < NW; ++w) acc = add(acc, red[w * CH + threadIdx.x]);
        out[threadIdx.x] = acc;
    }
    __syncthreads();
}

template <class R>
__device__ __forceinline__ R block_sum_r(R v, R* red) {
    constexpr int NW = kQrThreads / 32;
    v = warp_sum(v);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    R t = red[0];
    for (int w = 1; w < NW; ++w) t += red[w];
    __syncthreads();
    return t;
}

// X(j:M, k0:k0+nk) -= f v (v^H X(j:M, k0:k0+nk)), v(j) = 1 and v(i > j) =
// v[i]; f is conj(tau) for H^H and tau for H.
template <class T>
__device__ __forceinline__ void apply_reflector(const T* v_col, int M, int j, T f, T* X, int ldx, int k0, int nk,
                                                T* red, T* sh) {
    constexpr int NT = kQrThreads, CH = kQrChunk;
    T acc[CH];
#pragma unroll
    for (int c = 0; c < CH; ++c) acc[c] = make_s<T>(0);
    for (int i = j + threadIdx.x; i < M; i += NT) {
        const T v = i == j ? make_s<T>(1) : v_col[i];
#pragma unroll
        for (int c = 0; c < CH; ++c)
            if (c < nk) acc[c] = cfma(v, X[i + (long long)(k0 + c) * ldx], acc[c]);
    }
    block_sum<T, CH>(acc, red, sh);
    for (int i = j + threadIdx.x; i < M; i += NT) {
        const T v = i == j ? make_s<T>(1) : v_col[i];
        const T fv = mul(f, v);
#pragma unroll
        for (int c = 0; c < CH; ++c)
            if (c < nk) {
                T* p = &X[i + (long long)(k0 + c) * ldx];
                *p = sub(*p, mul(fv, sh[c]));
            }
    }
    __syncthreads();
}

// W = 2^-ex A' (A' = A, or A^H when m < n; ex the exponent of max |a_ij|,
// an exact scaling), then the Householder QR of W: reflectors below the
// diagonal of W, tau, and R (N x N, ld N, zeros below the diagonal).
template <class T, bool SM>
__global__ void __launch_bounds__(kQrThreads) qr_factor(const QrArgs a) {
    using R = Real<T>;
    constexpr int NT = kQrThreads, NW = NT / 32, CH = kQrChunk;
    extern __shared__ __align__(16) unsigned char qr_smem[];
    __shared__ T red[NW * CH];
    __shared__ T sh[CH];
    __shared__ R redr[NW];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int M = a.M, N = a.N;
    const T* A = static_cast<const T*>(a.A) + (long long)b * a.sA;
    T* const Wg = static_cast<T*>(a.W) + (long long)b * M * N;
    T* const W = SM ? reinterpret_cast<T*>(qr_smem) : Wg;
    T* tau = static_cast<T*>(a.tau) + (long long)b * N;
    T* Rm = static_cast<T*>(a.R) + (long long)b * N * N;

    R mx = 0;
    for (int e = tid; e < M * N; e += NT) {
        const int i = e % M, j = e / M;
        const T x = a.trans ? A[j + (long long)i * a.lda] : A[i + (long long)j * a.lda];
        if (finite_s(x)) mx = fmax(mx, maxabs(x));
    }
    mx = warp_max(mx);
    if ((tid & 31) == 0) redr[tid >> 5] = mx;
    __syncthreads();
    R m2 = redr[0];
    for (int w = 1; w < NW; ++w) m2 = fmax(m2, redr[w]);
    const int ex = m2 > 0 ? ilogb_r(m2) : 0;
    __syncthreads();
    for (int e = tid; e < M * N; e += NT) {
        const int i = e % M, j = e / M;
        const T x = a.trans ? conj_s(A[j + (long long)i * a.lda]) : A[i + (long long)j * a.lda];
        W[i + (long long)j * M] = scalb_s(x, -ex);
    }
    __syncthreads();

    for (int j = 0; j < N; ++j) {
        T* col = W + (long long)j * M;
        const T alpha = col[j];
        R ss = 0;
        for (int i = j + 1 + tid; i < M; i += NT) ss += abs2(col[i]);
        ss = block_sum_r(ss, redr);
        // every thread derives the same reflector from the same values
        T tj = make_s<T>(0), scal = make_s<T>(0);
        R beta = re(alpha);
        if (ss != 0 || im_s(alpha) != 0) {
            beta = -copysign(hypot(abs_s(alpha), sqrt_r(ss)), re(alpha));
            tj = make_c<T>((beta - re(alpha)) / beta, -im_s(alpha) / beta);
            scal = recip_s(sub(alpha, make_s<T>(beta)));
        }
        if (!is_zero(tj))
            for (int i = j + 1 + tid; i < M; i += NT) col[i] = mul(scal, col[i]);
        __syncthreads();
        if (tid == 0) {
            tau[j] = tj;
            col[j] = make_s<T>(beta);
        }
        if (!is_zero(tj))
            for (int k0 = j + 1; k0 < N; k0 += CH)
                apply_reflector(col, M, j, conj_s(tj), W, M, k0, min(CH, N - k0), red, sh);
        __syncthreads();
    }
    for (int e = tid; e < N * N; e += NT) {
        const int i = e % N, k = e / N;
        Rm[i + (long long)k * N] = i <= k ? W[i + (long long)k * M] : make_s<T>(0);
    }
    if (SM)   // the reflectors, for qr_apply
        for (int e = tid; e < M * N; e += NT) Wg[e] = W[e];
    if (tid == 0) a.ex[b] = ex;
}

// S <- 2^ex S; Y = Q [U_R; 0] (M x N, ld ldy) when Y is wanted.  SM: Y is
// built in shared memory (ld M) and written out at the end; each reflector is
// staged in a shared buffer, the next one read into registers meanwhile.
template <class T, bool SM>
__global__ void __launch_bounds__(kQrThreads) qr_apply(const QrArgs a) {
    using R = Real<T>;
    constexpr int NT = kQrThreads, NW = NT / 32, CH = kQrChunk, RPT = kQrRowsPerThread;
    extern __shared__ __align__(16) unsigned char qr_smem[];
    __shared__ T red[NW * CH];
    __shared__ T sh[CH];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int M = a.M, N = a.N;
    const int ex = a.ex[b];
    R* S = static_cast<R*>(a.S) + (long long)b * a.sS;
    for (int k = tid; k < N; k += NT) S[k] = scalb_s(S[k], ex);
    if (!a.Y) return;
    const T* W = static_cast<const T*>(a.W) + (long long)b * M * N;
    const T* tau = static_cast<const T*>(a.tau) + (long long)b * N;
    const T* Uh = static_cast<const T*>(a.Uhat) + (long long)b * N * N;
    T* const Yg = static_cast<T*>(a.Y) + (long long)b * a.sY;
    T* const Y = SM ? reinterpret_cast<T*>(qr_smem) : Yg;
    const int ldy = SM ? M : a.ldy;
    T* const vbuf = reinterpret_cast<T*>(qr_smem) + (long long)M * N;    // [2][M], SM only
    for (int e = tid; e < M * N; e += NT) {
        const int i = e % M, k = e / M;
        Y[i + (long long)k * ldy] = i < N ? Uh[i + (long long)k * N] : make_s<T>(0);
    }
    T nxt[RPT];
    if (SM) {   // the last reflector into its buffer (buffer j & 1 holds reflector j)
        T* v0 = vbuf + (long long)((N - 1) & 1) * M;
#pragma unroll
        for (int t = 0; t < RPT; ++t) {
            const int i = N - 1 + tid + t * NT;
            if (i < M) v0[i] = W[i + (long long)(N - 1) * M];
        }
    }
    __syncthreads();
    for (int j = N - 1; j >= 0; --j) {
        const T tj = tau[j];
        if (SM && j > 0)   // reflector j-1 on its way while j is applied
#pragma unroll
            for (int t = 0; t < RPT; ++t) {
                const int i = j - 1 + tid + t * NT;
                if (i < M) nxt[t] = W[i + (long long)(j - 1) * M];
            }
        const T* v = SM ? vbuf + (long long)(j & 1) * M : W + (long long)j * M;
        if (!is_zero(tj))
            for (int k0 = 0; k0 < N; k0 += CH) apply_reflector(v, M, j, tj, Y, ldy, k0, min(CH, N - k0), red, sh);
        if (SM && j > 0) {
            T* vn = vbuf + (long long)((j - 1) & 1) * M;
#pragma unroll
            for (int t = 0; t < RPT; ++t) {
                const int i = j - 1 + tid + t * NT;
                if (i < M) vn[i] = nxt[t];
            }
            __syncthreads();
        }
    }
    if (SM) {
        __syncthreads();
        for (int e = tid; e < M * N; e += NT) {
            const int i = e % M, k = e / M;
            Yg[i + (long long)k * a.ldy] = Y[e];
        }
    }
}

template <class T>
size_t qr_factor_smem(int M, int N) {
    const size_t b = (size_t)M * N * sizeof(T);
    return (M <= kQrThreads * kQrRowsPerThread && b <= (size_t)kQrSmemMax) ? b : 0;
}

template <class T>
size_t qr_apply_smem(int M, int N) {
    const size_t b = ((size_t)M * N + 2 * (size_t)M) * sizeof(T);
    return (M <= kQrThreads * kQrRowsPerThread && b <= (size_t)kQrSmemMax) ? b : 0;
}

template <class T>
cudaError_t qr_factor_t(const QrArgs& a, int batch, cudaStream_t st) {
    const size_t sm = qr_factor_smem<T>(a.M, a.N);
    if (sm) {
        const cudaError_t e = allow_dynamic_smem<qr_factor<T, true>>();
        if (e != cudaSuccess) return e;
        qr_factor<T, true><<<batch, kQrThreads, sm, st>>>(a);
    } else {
        qr_factor<T, false><<<batch, kQrThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

template <class T>
cudaError_t qr_apply_t(const QrArgs& a, int batch, cudaStream_t st) {
    const size_t sm = a.Y ? qr_apply_smem<T>(a.M, a.N) : 0;
    if (sm) {
        const cudaError_t e = allow_dynamic_smem<qr_apply<T, true>>();
        if (e != cudaSuccess) return e;
        qr_apply<T, true><<<batch, kQrThreads, sm, st>>>(a);
    } else {
        qr_apply<T, false><<<batch, kQrThreads, 0, st>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t qr_factor_s(const QrArgs& a, int batch, cudaStream_t st) { return qr_factor_t<float>(a, batch, st); }
cudaError_t qr_factor_d(const QrArgs& a, int batch, cudaStream_t st) { return qr_factor_t<double>(a, batch, st); }
cudaError_t qr_factor_c(const QrArgs& a, int batch, cudaStream_t st) { return qr_factor_t<float2>(a, batch, st); }
cudaError_t qr_factor_z(const QrArgs& a, int batch, cudaStream_t st) { return qr_factor_t<double2>(a, batch, st); }
cudaError_t qr_apply_s(const QrArgs& a, int batch, cudaStream_t st) { return qr_apply_t<float>(a, batch, st); }
cudaError_t qr_apply_d(const QrArgs& a, int batch, cudaStream_t st) { return qr_apply_t<double>(a, batch, st); }
cudaError_t qr_apply_c(const QrArgs& a, int batch, cudaStream_t st) { return qr_apply_t<float2>(a, batch, st); }
cudaError_t qr_apply_z(const QrArgs& a, int batch, cudaStream_t st) { return qr_apply_t<double2>(a, batch, st); }

}  // namespace bsvd
