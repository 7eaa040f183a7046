// gesvj_blocked.cuh -- the multi-kernel blocked one-sided Jacobi SVD.
//
// The structure of Sec. 4: per round of the round-robin ordering, one launch
// per stage over all (block pair, matrix) items, with the working matrix W,
// V, the Gram blocks G and the eigenvector blocks J in a global-memory
// workspace.  Options select the paper's design ladder:
//   baseline (Sec. 4)  inner eigensolver run to convergence, two-stage
//                      vector update through a temporary, no masks, the
//                      batch converges when every matrix has (host check
//                      once per sweep);
//   Design-2 (Sec. 5)  one inner sweep;
//   Design-3 (Sec. 6)  fused vector update (Alg. 4): one read, one write;
//   Design-4 (Sec. 7)  masks: converged matrices and pairs whose J = I skip
//                      the eigensolver and the update.
// The same kernels serve any matrix too large for the on-chip fused path.
#pragma once

#include <type_traits>

#include "blocked_layout.h"
#include "jacobi_common.cuh"
#include "tc_c64.cuh"
#include "tc_f32.cuh"

namespace bsvd {

enum : int { kBlkThreads = 256, kUpdRows = 128, kGramChunk = 64 };

__device__ __forceinline__ int blk_mid(const BlockedArgs& a, int b) { return a.index ? a.index[b] : b; }

// working shape of matrix b and its offsets in the workspace regions: the
// per-matrix record of a variable-shape batch, else the batch's one shape
__device__ __forceinline__ BlkShape blk_shape(const BlockedArgs& a, int b) {
    if (a.shapes) return a.shapes[b];
    BlkShape s;
    s.M = a.M; s.N = a.N; s.trans = a.trans; s.m = a.m; s.n = a.n; s.l = a.l; s.L = a.L; s.Np = a.Np;
    s.oW = b * a.sW; s.oV = b * a.sVw; s.oG = b * a.sG; s.oJ = b * a.sJ; s.oT = b * a.sT;
    return s;
}

// block pair q of round r of matrix b, or false when the matrix has no such
// pair (a phantom block, or a round or pair beyond a smaller matrix's count)
__device__ __forceinline__ bool blk_pair(const BlkShape& s, int r, int q, int& bi, int& bj) {
    if (r >= s.L - 1 || q >= s.L / 2) return false;
    rr_pair(s.L, r, q, bi, bj);
    return bj < s.l;
}

// skip this matrix? (bad input always; converged ones only with masks)
__device__ __forceinline__ bool blk_skip(const BlockedArgs& a, int b) {
    const int st = a.state[4 * b];
    return st < 0 || (a.masks && st == 0);
}

// ---- load: W = A * 2^-ex (or A^H), padded; V = I; status -------------------
// ---- S2, real FP32: register tiles --------------------------------------------
// The full 2nb x 2nb Gram block of the pair in 4 x 4 register tiles (float4
// reads of row-chunks staged in shared memory, column stride KP = KC + 4: 16-
// byte aligned, KP/4 odd), each tile's rows split over KS lanes and summed
// with shuffles at the end; upper tiles written and mirrored.  Twice the
// flops of the three blocks the generic kernel forms, an eighth of its
// shared-memory reads per FMA.  Needs KS = 256 / (2nb/4)^2 <= 32: nb >= 8.
template <int NB>
__global__ void __launch_bounds__(kBlkThreads) blk_gram_f32(const BlockedArgs a, int r) {
    constexpr int TWO = 2 * NB, NT = kBlkThreads, TT = TWO / 4, NTILE = TT * TT, KS = NT / NTILE;
    static_assert(NT % NTILE == 0 && KS >= 1 && KS <= 32 && (KS & (KS - 1)) == 0, "tile split");
    constexpr int KC = kGramChunk, KP = KC + 4;
    __shared__ __align__(16) float P[KP * TWO];
    const int b = blockIdx.x, q = blockIdx.y, tid = threadIdx.x;
    if (blk_skip(a, b)) return;
    const BlkShape sh = blk_shape(a, b);
    int bi, bj;
    if (!blk_pair(sh, r, q, bi, bj)) return;
    const float* W = static_cast<const float*>(a.W) + sh.oW;
    const int M = sh.M;
    const int tile = tid / KS, ks = tid % KS, ti = tile / TT, tj = tile % TT;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    for (int k0 = 0; k0 < M; k0 += KC) {
        const int kc = min(KC, M - k0);
        for (int e = tid; e < KC * TWO; e += NT) {
            const int kk = e % KC, c = e / KC;
            const int col = c < NB ? bi * NB + c : bj * NB + (c - NB);
            P[kk + c * KP] = kk < kc ? W[k0 + kk + (long long)col * M] : 0.f;   // zero tail: adds nothing
        }
        __syncthreads();
        const int chunks = (kc + 3) >> 2;
        for (int ch = ks; ch < chunks; ch += KS) {
            float4 av[4], bv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                av[u] = *reinterpret_cast<const float4*>(P + 4 * ch + (4 * ti + u) * KP);
                bv[u] = *reinterpret_cast<const float4*>(P + 4 * ch + (4 * tj + u) * KP);
            }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    float t = acc[i][j];
                    t = fmaf(av[i].x, bv[j].x, t);
                    t = fmaf(av[i].y, bv[j].y, t);
                    t = fmaf(av[i].z, bv[j].z, t);
                    t = fmaf(av[i].w, bv[j].w, t);
                    acc[i][j] = t;
                }
        }
        __syncthreads();
    }
#pragma unroll
    for (int o = 1; o < KS; o <<= 1)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += __shfl_xor_sync(0xffffffffu, acc[i][j], o);
    float* G = static_cast<float*>(a.G) + sh.oG + (long long)q * TWO * TWO;
    if (ks == 0 && ti <= tj) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int rr = 4 * ti + i, cc = 4 * tj + j;
                if (ti == tj && rr > cc) continue;             // diagonal tile: upper part, mirrored
                G[rr + cc * TWO] = acc[i][j];
                G[cc + rr * TWO] = acc[i][j];
            }
    }
}

// ---- S2, real FP32 on the tensor cores (nb = 8, 16) -------------------------------
// The same 64-row chunks staged in shared memory; the 16 x 16 blocks of the
// Gram block formed by split-TF32 mma tiles (tc_f32.cuh).  The eight warps
// split each chunk's eight k-steps: nb = 16 has four blocks, two warps a
// block; nb = 8 one block, all eight warps.  The warps' partial blocks are
// summed in warp order (a fixed order: the bits do not depend on timing),
// and the upper entries written and mirrored.
template <int NB>
__global__ void __launch_bounds__(kBlkThreads) blk_gram_f32_tc(const BlockedArgs a, int r) {
    constexpr int TWO = 2 * NB, NT = kBlkThreads, NW = NT / 32, NBLK = TWO / 16, NB2 = NBLK * NBLK;
    constexpr int WPB = NW / NB2;                       // warps per block
    static_assert(NW % NB2 == 0, "warps per Gram block");
    constexpr int KC = kGramChunk, KP = KC + 4;
    __shared__ __align__(16) float P[2][KP * TWO];     // two chunks: the next loads during this one
    __shared__ float red[NW * 32 * 8];
    const int b = blockIdx.x, q = blockIdx.y, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (blk_skip(a, b)) return;
    const BlkShape sh = blk_shape(a, b);
    int bi, bj;
    if (!blk_pair(sh, r, q, bi, bj)) return;
    const float* W = static_cast<const float*>(a.W) + sh.oW;
    const int M = sh.M;
    const int blk = warp % NB2, sub = warp / NB2, bm = blk / NBLK, bn = blk % NBLK;
    float acc[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[j][i] = 0.f;
    auto stage = [&](int buf, int k0) {        // zero tail: adds nothing
        const int kc = min(KC, M - k0);
        for (int e = tid; e < KC * TWO; e += NT) {
            const int kk = e % KC, c = e / KC;
            const int col = c < NB ? bi * NB + c : bj * NB + (c - NB);
            cp_async<4>(&P[buf][kk + c * KP], W + k0 + (kk < kc ? kk : 0) + (long long)col * M, kk < kc ? 4 : 0);
        }
        cp_async_commit();
    };
    stage(0, 0);
    for (int k0 = 0, it = 0; k0 < M; k0 += KC, ++it) {
        const int kc = min(KC, M - k0);
        if (k0 + KC < M) {
            stage((it + 1) & 1, k0 + KC);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();
        if (bm <= bn)                           // blocks below the diagonal are mirrors
            gram_block_acc<NB>(P[it & 1], KP, kc, 0, NB, bm, bn, sub, WPB, lane, acc);
        __syncthreads();                        // before this buffer is refilled
    }
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) red[(warp * 32 + lane) * 8 + 4 * j + i] = acc[j][i];
    __syncthreads();
    if (sub != 0) return;
    float* G = static_cast<float*>(a.G) + sh.oG + (long long)q * TWO * TWO;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float x = red[(blk * 32 + lane) * 8 + 4 * j + i];
            for (int s2 = 1; s2 < WPB; ++s2) x += red[((blk + s2 * NB2) * 32 + lane) * 8 + 4 * j + i];
            const int rr = 16 * bm + g + 8 * (i >> 1), cc = 16 * bn + 8 * j + 2 * t + (i & 1);
            if (rr > cc) continue;                          // lower entries: the mirror of an upper one
            G[rr + cc * TWO] = x;
            G[cc + rr * TWO] = x;
        }
}

// ---- S2, complex64 on the tensor cores (nb = 8, 16) ------------------------------
// As blk_gram_f32_tc with the panel's real and imaginary parts staged as two
// planes; each 16 x 16 block of G = P^H P is Re = Pr^T Pr + Pi^T Pi and
// Im = Pr^T Pi - Pi^T Pr (tc_c64.cuh), the warps' partial blocks summed in
// warp order, the upper entries written and mirrored (conjugate), the
// diagonal real.
template <int NB>
__global__ void __launch_bounds__(kBlkThreads) blk_gram_c64_tc(const BlockedArgs a, int r) {
    constexpr int TWO = 2 * NB, NT = kBlkThreads, NW = NT / 32, NBLK = TWO / 16, NB2 = NBLK * NBLK;
    constexpr int WPB = NW / NB2;
    static_assert(NW % NB2 == 0, "warps per Gram block");
    constexpr int KC = kGramChunk, KP = KC + 4;
    __shared__ __align__(16) float2 P[KP * TWO];
    __shared__ float red[NW * 32 * 16];
    const int b = blockIdx.x, q = blockIdx.y, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    if (blk_skip(a, b)) return;
    const BlkShape sh = blk_shape(a, b);
    int bi, bj;
    if (!blk_pair(sh, r, q, bi, bj)) return;
    const float2* W = static_cast<const float2*>(a.W) + sh.oW;
    const int M = sh.M;
    const int blk = warp % NB2, sub = warp / NB2, bm = blk / NBLK, bn = blk % NBLK;
    float re[2][4], im[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) re[j][i] = im[j][i] = 0.f;
    for (int k0 = 0; k0 < M; k0 += KC) {
        const int kc = min(KC, M - k0);
        for (int e = tid; e < KC * TWO; e += NT) {
            const int kk = e % KC, c = e / KC;
            const int col = c < NB ? bi * NB + c : bj * NB + (c - NB);
            P[kk + c * KP] = kk < kc ? W[k0 + kk + (long long)col * M] : make_float2(0.f, 0.f);
        }
        __syncthreads();
        if (bm <= bn)                           // blocks below the diagonal are mirrors
            gram_c64_block_acc<NB>(P, KP, kc, 0, NB, bm, bn, sub, WPB, lane, re, im);
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            red[(warp * 32 + lane) * 16 + 4 * j + i] = re[j][i];
            red[(warp * 32 + lane) * 16 + 8 + 4 * j + i] = im[j][i];
        }
    __syncthreads();
    if (sub != 0) return;
    float2* G = static_cast<float2*>(a.G) + sh.oG + (long long)q * TWO * TWO;
    const int g = lane >> 2, t = lane & 3;
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            float xr = red[(blk * 32 + lane) * 16 + 4 * j + i], xi = red[(blk * 32 + lane) * 16 + 8 + 4 * j + i];
            for (int s2 = 1; s2 < WPB; ++s2) {
                xr += red[((blk + s2 * NB2) * 32 + lane) * 16 + 4 * j + i];
                xi += red[((blk + s2 * NB2) * 32 + lane) * 16 + 8 + 4 * j + i];
            }
            const int rr = 16 * bm + g + 8 * (i >> 1), cc = 16 * bn + 8 * j + 2 * t + (i & 1);
            if (rr > cc) continue;                          // lower entries: the mirror of an upper one
            if (rr == cc) xi = 0.f;                         // Hermitian: a real diagonal
            G[rr + cc * TWO] = make_float2(xr, xi);
            G[cc + rr * TWO] = make_float2(xr, -xi);
        }
}

template <class T>
__global__ void __launch_bounds__(kBlkThreads) blk_load(const BlockedArgs a) {
    using R = Real<T>;
    constexpr int NT = kBlkThreads, NW = NT / 32;
    __shared__ R red[NW];
    __shared__ int bad_s, ex_s;
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int mid = blk_mid(a, b);
    const BlkShape sh = blk_shape(a, b);
    const int sid = a.in_local ? b : mid;                     // position of strided inputs
    const T* A = a.Ap ? static_cast<const T*>(a.Ap[mid]) : static_cast<const T*>(a.A) + (long long)sid * a.sA;
    const int lda = a.ldap ? a.ldap[mid] : a.lda;
    R mx = 0;
    int nonfin = 0;
    for (int e = tid; e < sh.m * sh.n; e += NT) {
        const T x = A[(e % sh.m) + (long long)(e / sh.m) * lda];
        if (!finite_s(x)) nonfin = 1; else mx = fmax(mx, maxabs(x));
    }
    mx = warp_max(mx);
    const bool wbad = __any_sync(0xffffffffu, nonfin);
    if (lane == 0) red[warp] = wbad ? R(-1) : mx;
    __syncthreads();
    if (tid == 0) {
        R m2 = 0;
        int bd = 0;
        for (int w = 0; w < NW; ++w) { bd |= red[w] < 0; m2 = fmax(m2, red[w]); }
        bad_s = bd;
        ex_s = (m2 > 0) ? ilogb_r(m2) : 0;
        a.state[4 * b + 0] = bd ? -1 : 1;
        a.state[4 * b + 1] = 0;
        a.state[4 * b + 2] = 0;
        a.state[4 * b + 3] = ex_s;
    }
    __syncthreads();
    if (bad_s) return;
    const int ex = ex_s;
    T* W = static_cast<T*>(a.W) + sh.oW;
    T* V = static_cast<T*>(a.Vw) + sh.oV;
    const int M = sh.M, N = sh.N;
    for (int e = tid; e < sh.m * sh.n; e += NT) {
        const int i = e % sh.m, j = e / sh.m;
        const T x = scalb_s(A[i + (long long)j * lda], -ex);
        if (sh.trans) W[j + (long long)i * M] = conj_s(x);
        else          W[i + (long long)j * M] = x;
    }
    for (int e = tid; e < M * (sh.Np - N); e += NT) W[(e % M) + (long long)(N + e / M) * M] = make_s<T>(0);
    const T* V0 = a.V0 ? static_cast<const T*>(a.V0) + (long long)sid * a.sV0 : nullptr;
    for (int e = tid; e < N * sh.Np; e += NT) {
        const int i = e % N, j = e / N;
        V[i + (long long)j * N] = (V0 && j < N) ? V0[i + (long long)j * a.ldv0] : make_s<T>(i == j && !V0 ? 1 : 0);
    }
}

// ---- S2: G = [A_i A_j]^H [A_i A_j] as three nb x nb products -----------------
// (A_i^H A_i, A_j^H A_i, A_j^H A_j; Sec. 4.2) accumulated over chunks of rows
// staged in shared memory.  grid (count, L/2).
template <class T, int NB>
__global__ void __launch_bounds__(kBlkThreads) blk_gram(const BlockedArgs a, int r) {
    constexpr int TWO = 2 * NB, NT = kBlkThreads;
    // rows per staged chunk: kGramChunk, fewer when the 2nb-wide tile would pass 32 KB
    constexpr int KC = (kGramChunk * TWO * (int)sizeof(T) <= 32768) ? kGramChunk
                                                                   : 32768 / (TWO * (int)sizeof(T));
    constexpr int NE = 3 * NB * NB, PER = (NE + NT - 1) / NT;
    // column stride KC + 1: the threads of a warp read one row of several
    // columns, which a stride of a multiple of 32 words would put in one bank
    constexpr int KP = KC + 1;
    __shared__ T P[KP * TWO];
    const int b = blockIdx.x, q = blockIdx.y, tid = threadIdx.x;
    if (blk_skip(a, b)) return;
    const BlkShape sh = blk_shape(a, b);
    int bi, bj;
    if (!blk_pair(sh, r, q, bi, bj)) return;
    const T* W = static_cast<const T*>(a.W) + sh.oW;
    const int M = sh.M;
    // two partial sums per entry, rows [0, M/2) and [M/2, M), added at the end
    // (the same summation as the on-chip kernel)
    T lo[PER], hi[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) { lo[u] = make_s<T>(0); hi[u] = make_s<T>(0); }
    const int mh = M / 2;
    for (int k0 = 0; k0 < M; k0 += KC) {
        const int kc = min(KC, M - k0);
        for (int e = tid; e < KC * TWO; e += NT) {
            const int kk = e % KC, c = e / KC;
            const int col = c < NB ? bi * NB + c : bj * NB + (c - NB);
            P[kk + c * KP] = kk < kc ? W[k0 + kk + (long long)col * M] : make_s<T>(0);
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int e = tid + u * NT;
            if (e < NE) {
                const int blk = e / (NB * NB), w = e % (NB * NB), ra = w % NB, cb = w / NB;
                const int row = (blk == 0) ? ra : NB + ra;      // (i,i), (j,i), (j,j)
                const int col = (blk == 2) ? NB + cb : cb;
                const int split = min(max(mh - k0, 0), kc);    // rows of this chunk below M/2
                T s0 = lo[u], s1 = hi[u];
                for (int kk = 0; kk < split; ++kk) s0 = cfma(P[kk + row * KP], P[kk + col * KP], s0);
                for (int kk = split; kk < kc; ++kk) s1 = cfma(P[kk + row * KP], P[kk + col * KP], s1);
                lo[u] = s0;
                hi[u] = s1;
            }
        }
        __syncthreads();
    }
    T acc[PER];
#pragma unroll
    for (int u = 0; u < PER; ++u) acc[u] = add(lo[u], hi[u]);
    T* G = static_cast<T*>(a.G) + sh.oG + (long long)q * TWO * TWO;
#pragma unroll
    for (int u = 0; u < PER; ++u) {
        const int e = tid + u * NT;
        if (e < NE) {
            const int blk = e / (NB * NB), w = e % (NB * NB), ra = w % NB, cb = w / NB;
            const int row = (blk == 0) ? ra : NB + ra;
            const int col = (blk == 2) ? NB + cb : cb;
            G[row + col * TWO] = acc[u];
            if (blk == 1) G[col + row * TWO] = conj_s(acc[u]);
        }
    }
}

// ---- S3: the Hermitian eigensolver on each Gram block --------------------------
// grid (count, L/2), GT threads.  J to global; flags the pair and the matrix.
template <class T, int NB, int GT>
__global__ void __launch_bounds__(GT) blk_heevj(const BlockedArgs a, int r) {
    constexpr int TWO = 2 * NB, LDG = TWO + 1;
    extern __shared__ __align__(16) unsigned char smem[];
    const int b = blockIdx.x, q = blockIdx.y, tid = threadIdx.x;
    int* pf = a.pairflag + (long long)b * (a.L / 2) + q;
    if (blk_skip(a, b)) { if (tid == 0) *pf = 0; return; }
    const BlkShape sh = blk_shape(a, b);
    int bi, bj;
    if (!blk_pair(sh, r, q, bi, bj)) { if (tid == 0) *pf = 0; return; }
    T* G = reinterpret_cast<T*>(smem);
    T* J = G + TWO * LDG;
    const InnerTables<T, NB> tb(J + TWO * LDG);
    const T* Gg = static_cast<const T*>(a.G) + sh.oG + (long long)q * TWO * TWO;
    for (int e = tid; e < TWO * TWO; e += GT) {       // upper triangle, mirrored
        const int i = e % TWO, j = e / TWO;
        if (i > j) continue;
        T g = Gg[i + j * TWO];
        if (i == j) g = make_s<T>(re(g));
        G[i + j * LDG] = g;
        G[j + i * LDG] = conj_s(g);
    }
    __syncthreads();
    const int seen = inner_jacobi<T, NB, GT>(G, J, tb, (Real<T>)a.tol, a.inner_sweeps, tid, 1, NoBackground(),
                                             nullptr, (a.flags & 256) != 0);
    T* Jg = static_cast<T*>(a.J) + sh.oJ + (long long)q * TWO * TWO;
    for (int e = tid; e < TWO * TWO; e += GT) Jg[(e % TWO) + (e / TWO) * TWO] = J[(e % TWO) + (e / TWO) * LDG];
    if (tid == 0) {
        *pf = seen > 0;
        if (seen > 0) a.state[4 * b + 1] = 1;
    }
}

// panel row helpers: row `row` of [W; V] (rows 0..M-1 of W, then N of V)
template <class T>
__device__ __forceinline__ T* blk_row(const BlockedArgs& a, const BlkShape& sh, int row, long long& ld) {
    if (row < sh.M) { ld = sh.M; return static_cast<T*>(a.W) + sh.oW + row; }
    ld = sh.N;
    return static_cast<T*>(a.Vw) + sh.oV + (row - sh.M);
}

// ---- S4/S5 fused (Design-3, Alg. 4): [P_i P_j] <- [P_i P_j] J, one read and one
// write per element.  grid (count, L/2, row blocks), kUpdRows threads.
// Row blocks z, z + gridDim.z, ...: the launcher caps gridDim.z once the
// batch has enough block pairs to fill the GPU, so that masked (converged)
// matrices and pairs cost fewer empty CTAs per launch.
template <class T, int NB>
__global__ void __launch_bounds__(kUpdRows) blk_update_fused(const BlockedArgs a, int r) {
    constexpr int TWO = 2 * NB;
    extern __shared__ __align__(16) unsigned char smem_js[];
    T* Js = reinterpret_cast<T*>(smem_js);
    const int b = blockIdx.x, q = blockIdx.y, tid = threadIdx.x;
    if (blk_skip(a, b)) return;
    if (a.masks && !a.pairflag[(long long)b * (a.L / 2) + q]) return;
    const BlkShape sh = blk_shape(a, b);
    int bi, bj;
    if (!blk_pair(sh, r, q, bi, bj)) return;
    const int rows = sh.M + sh.N;
    if (blockIdx.z * kUpdRows >= rows) return;
    const T* Jg = static_cast<const T*>(a.J) + sh.oJ + (long long)q * TWO * TWO;
    if constexpr (std::is_same<T, float>::value && (NB == 8 || NB == 16))
      if (!(a.flags & 128)) {
        // real FP32: 16-row tiles of W, then of V, on the tensor cores
        // (split TF32, tc_f32.cuh); a CTA's four warps take the tiles of its
        // row blocks, eight tiles a block
        uint4* Jf = reinterpret_cast<uint4*>(smem_js);
        j_fragments<NB, kUpdRows, TWO>(Jg, Jf, tid);
        __syncthreads();
        const int tw = (sh.M + 15) / 16, tt = tw + (sh.N + 15) / 16, warp = tid >> 5, lane = tid & 31;
        float* Wm = static_cast<float*>(a.W) + sh.oW;
        float* Vm = static_cast<float*>(a.Vw) + sh.oV;
        for (int base = blockIdx.z * (kUpdRows / 16); base < tt; base += gridDim.z * (kUpdRows / 16))
            for (int tile = base + warp; tile < min(tt, base + kUpdRows / 16); tile += kUpdRows / 32) {
                if (tile < tw) update_rows_mma<NB>(Wm, sh.M, sh.M, 16 * tile, bi * NB, bj * NB, Jf, lane);
                else           update_rows_mma<NB>(Vm, sh.N, sh.N, 16 * (tile - tw), bi * NB, bj * NB, Jf, lane);
            }
        return;
    }
    if constexpr (std::is_same<T, float2>::value && (NB == 8 || NB == 16))
      if (!(a.flags & 128)) {
        // complex64 on the tensor cores: 16-row tiles of W, then of V, as
        // real split-TF32 products of the parts (tc_c64.cuh)
        uint4* Jf = reinterpret_cast<uint4*>(smem_js);
        jc_fragments<NB, kUpdRows, TWO>(Jg, Jf, tid);
        __syncthreads();
        const int tw = (sh.M + 15) / 16, tt = tw + (sh.N + 15) / 16, warp = tid >> 5, lane = tid & 31;
        float2* Wm = static_cast<float2*>(a.W) + sh.oW;
        float2* Vm = static_cast<float2*>(a.Vw) + sh.oV;
        for (int base = blockIdx.z * (kUpdRows / 16); base < tt; base += gridDim.z * (kUpdRows / 16))
            for (int tile = base + warp; tile < min(tt, base + kUpdRows / 16); tile += kUpdRows / 32) {
                if (tile < tw) update_rows_c64_mma<NB>(Wm, sh.M, sh.M, 16 * tile, bi * NB, bj * NB, Jf, lane);
                else           update_rows_c64_mma<NB>(Vm, sh.N, sh.N, 16 * (tile - tw), bi * NB, bj * NB, Jf, lane);
            }
        return;
      }
    if constexpr (std::is_same<T, float2>::value && NB <= 16) {
        // complex64: 4 rows x 2nb/4 columns per thread.  The four lanes of a
        // quad share 4 rows (rs, rs + 32, ...) and take columns cg, cg + 4,
        // ...; J is kept with column stride 2nb + 1 so the quad's reads hit
        // different banks.  A quarter of a J read per multiply-add instead of
        // one; each output still sums k in order, the bits of the generic
        // branch below.
        constexpr int LDJ = TWO + 1, CJ = TWO / 4, RS = kUpdRows / 4;
        for (int e = tid; e < TWO * TWO; e += kUpdRows) Js[(e % TWO) + (e / TWO) * LDJ] = Jg[e];
        __syncthreads();
        const int cg = tid & 3, rs = tid >> 2;
        for (int base = blockIdx.z * kUpdRows; base < rows; base += gridDim.z * kUpdRows) {
            T* X[4];
            long long ldx[4];
            bool ok[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int row = base + rs + RS * i;
                ok[i] = row < rows;
                ldx[i] = 0;
                X[i] = ok[i] ? blk_row<T>(a, sh, row, ldx[i]) : nullptr;
            }
            T acc[4][CJ];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < CJ; ++j) acc[i][j] = make_s<T>(0);
#pragma unroll 4
            for (int k = 0; k < TWO; ++k) {
                const long long ck = k < NB ? bi * NB + k : bj * NB + k - NB;
                T xk[4], jk[CJ];
#pragma unroll
                for (int i = 0; i < 4; ++i) xk[i] = ok[i] ? X[i][ck * ldx[i]] : make_s<T>(0);
#pragma unroll
                for (int j = 0; j < CJ; ++j) jk[j] = Js[k + (cg + 4 * j) * LDJ];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < CJ; ++j) acc[i][j] = fma_s(xk[i], jk[j], acc[i][j]);
            }
            __syncwarp();   // the quad has read its rows before any of it writes them
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (ok[i]) {
#pragma unroll
                    for (int j = 0; j < CJ; ++j) {
                        const int c = cg + 4 * j;
                        X[i][(long long)(c < NB ? bi * NB + c : bj * NB + c - NB) * ldx[i]] = acc[i][j];
                    }
                }
        }
        return;
    }
    for (int e = tid; e < TWO * TWO; e += kUpdRows) Js[e] = Jg[e];
    __syncthreads();
    for (int row = blockIdx.z * kUpdRows + tid; row < rows; row += gridDim.z * kUpdRows) {
        long long ld;
        T* X = blk_row<T>(a, sh, row, ld);
        T x[TWO];
#pragma unroll
        for (int k = 0; k < TWO; ++k) x[k] = X[(long long)(k < NB ? bi * NB + k : bj * NB + k - NB) * ld];
#pragma unroll
        for (int c = 0; c < TWO; ++c) {
            T acc = make_s<T>(0);
#pragma unroll
            for (int k = 0; k < TWO; ++k) acc = fma_s(x[k], Js[k + c * TWO], acc);
            X[(long long)(c < NB ? bi * NB + c : bj * NB + c - NB) * ld] = acc;
        }
    }
}

// ---- S4/S5 baseline, stage 1 (Sec. 4.4): T_i = P_i J11, T_j = P_i J12 -------------
template <class T, int NB>
__global__ void __launch_bounds__(kUpdRows) blk_update_stage1(const BlockedArgs a, int r) {
    constexpr int TWO = 2 * NB;
    extern __shared__ __align__(16) unsigned char smem_js[];
    T* Js = reinterpret_cast<T*>(smem_js);
    const int b = blockIdx.x, q = blockIdx.y, tid = threadIdx.x;
    if (blk_skip(a, b)) return;
    if (a.masks && !a.pairflag[(long long)b * (a.L / 2) + q]) return;
    const BlkShape sh = blk_shape(a, b);
    int bi, bj;
    if (!blk_pair(sh, r, q, bi, bj)) return;
    if (blockIdx.z * kUpdRows >= sh.M + sh.N) return;
    const T* Jg = static_cast<const T*>(a.J) + sh.oJ + (long long)q * TWO * TWO;
    for (int e = tid; e < TWO * TWO; e += kUpdRows) Js[e] = Jg[e];
    __syncthreads();
    const int row = blockIdx.z * kUpdRows + tid, rows = sh.M + sh.N;
    if (row >= rows) return;
    long long ld;
    const T* X = blk_row<T>(a, sh, row, ld);
    T* Tt = static_cast<T*>(a.T) + sh.oT + (long long)q * rows * TWO + row;
    T x[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) x[k] = X[(long long)(bi * NB + k) * ld];
#pragma unroll
    for (int c = 0; c < TWO; ++c) {
        T acc = make_s<T>(0);
#pragma unroll
        for (int k = 0; k < NB; ++k) acc = fma_s(x[k], Js[k + c * TWO], acc);
        Tt[(long long)c * rows] = acc;
    }
}

// ---- stage 2: P_i = T_i + P_j J21, P_j = T_j + P_j J22 ------------------------------
template <class T, int NB>
__global__ void __launch_bounds__(kUpdRows) blk_update_stage2(const BlockedArgs a, int r) {
    constexpr int TWO = 2 * NB;
    extern __shared__ __align__(16) unsigned char smem_js[];
    T* Js = reinterpret_cast<T*>(smem_js);
    const int b = blockIdx.x, q = blockIdx.y, tid = threadIdx.x;
    if (blk_skip(a, b)) return;
    if (a.masks && !a.pairflag[(long long)b * (a.L / 2) + q]) return;
    const BlkShape sh = blk_shape(a, b);
    int bi, bj;
    if (!blk_pair(sh, r, q, bi, bj)) return;
    if (blockIdx.z * kUpdRows >= sh.M + sh.N) return;
    const T* Jg = static_cast<const T*>(a.J) + sh.oJ + (long long)q * TWO * TWO;
    for (int e = tid; e < TWO * TWO; e += kUpdRows) Js[e] = Jg[e];
    __syncthreads();
    const int row = blockIdx.z * kUpdRows + tid, rows = sh.M + sh.N;
    if (row >= rows) return;
    long long ld;
    T* X = blk_row<T>(a, sh, row, ld);
    const T* Tt = static_cast<const T*>(a.T) + sh.oT + (long long)q * rows * TWO + row;
    T x[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) x[k] = X[(long long)(bj * NB + k) * ld];
#pragma unroll
    for (int c = 0; c < TWO; ++c) {
        T acc = Tt[(long long)c * rows];
#pragma unroll
        for (int k = 0; k < NB; ++k) acc = fma_s(x[k], Js[NB + k + c * TWO], acc);
        X[(long long)(c < NB ? bi * NB + c : bj * NB + c - NB) * ld] = acc;
    }
}

// ---- a6: end of a sweep: count it, retire converged matrices ----------------------
static __global__ void blk_converge(const BlockedArgs a) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= a.count) return;
    int* s = a.state + 4 * b;
    if (s[0] == 1) {
        s[2] += 1;
        if (!s[1]) s[0] = 0;               // a sweep without rotation: converged
    }
    s[1] = 0;
    if (s[0] == 1) atomicOr(a.any_active, 1);
}

// ---- a7: finalise -------------------------------------------------------------
// rank of each column of a finished matrix, kept in the finalisation scratch
// after x (M) and E (N x N)
template <class T>
__device__ __forceinline__ int* fin_rank(const BlockedArgs& a, const BlkShape& sh) {
    return reinterpret_cast<int*>(static_cast<T*>(a.T) + sh.oT + sh.M + (long long)sh.N * sh.N);
}

template <class T>
__global__ void __launch_bounds__(kBlkThreads) blk_finalize(const BlockedArgs a) {
    using R = Real<T>;
    constexpr int NT = kBlkThreads;
    extern __shared__ __align__(16) unsigned char smem[];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int mid = blk_mid(a, b);
    const BlkShape sh = blk_shape(a, b);
    const int N = sh.N, M = sh.M;
    R* red = reinterpret_cast<R*>(smem);                 // [NT/32]
    int* iscr = reinterpret_cast<int*>(red + NT / 32);   // [4]
    T* bcast = reinterpret_cast<T*>(iscr + 4);           // [2]
    R* sig = reinterpret_cast<R*>(bcast + 2);            // [N]
    int* rank = reinterpret_cast<int*>(sig + N);         // [N]
    R* Sout = a.Sp ? static_cast<R*>(a.Sp[mid]) : static_cast<R*>(a.S) + (long long)mid * a.sS;
    T* Uout = nullptr;
    T* Vout = nullptr;
    long long ldu = 1, ldv = 1;
    if (a.wantU) {
        Uout = a.Up ? static_cast<T*>(a.Up[mid]) : static_cast<T*>(a.U) + (long long)mid * a.sU;
        ldu = a.ldup ? a.ldup[mid] : a.ldu;
    }
    if (a.wantV) {
        Vout = a.Vp ? static_cast<T*>(a.Vp[mid]) : static_cast<T*>(a.V) + (long long)mid * a.sV;
        ldv = a.ldvp ? a.ldvp[mid] : a.ldv;
    }
    const int status = a.state[4 * b], sw = a.state[4 * b + 2], ex = a.state[4 * b + 3];
    if (status < 0) {
        for (int e = tid; e < N; e += NT) Sout[e] = nan_s<R>();
        if (Uout) for (int e = tid; e < sh.m * N; e += NT) Uout[(e % sh.m) + (long long)(e / sh.m) * ldu] = nan_s<T>();
        if (Vout) for (int e = tid; e < sh.n * N; e += NT) Vout[(e % sh.n) + (long long)(e / sh.n) * ldv] = nan_s<T>();
        if (tid == 0) {
            a.info[mid] = -1;
            if (a.sweeps) a.sweeps[mid] = 0;
        }
        return;
    }
    const T* W = static_cast<const T*>(a.W) + sh.oW;
    const T* V = static_cast<const T*>(a.Vw) + sh.oV;
    T* scratch = static_cast<T*>(a.T) + sh.oT;           // x (M), E (N x N), rank (N)
    const bool wantWout = sh.trans ? a.wantV : a.wantU;
    T* Y = sh.trans ? Vout : Uout;
    const FinalScratch<T> fs{sig, rank, red, iscr, bcast};
    // Sigma and U here; V (and its Newton-Schulz step) in the tiled kernels
    // below, which read the columns' ranks from the workspace
    finalize_outputs<T, NT>(W, M, V, N, M, N, ex, scratch, scratch + M, N,
                            false, Sout, Y, sh.trans ? ldv : ldu, wantWout, nullptr, 1, false, fs);
    int* grank = fin_rank<T>(a, sh);
    for (int k = tid; k < N; k += NT) grank[k] = rank[k];
    if (tid == 0) {
        a.info[mid] = status == 0 ? 0 : sw;
        if (a.sweeps) a.sweeps[mid] = sw;
    }
}

// ---- Newton-Schulz step of V over the whole GPU ------------------------------
// The correction of the end of Alg. 2 costs 1.5 N^3 multiply-adds per matrix,
// more than the rest of the finalisation together once N is in the hundreds,
// so it runs as two tiled products over (matrix, 64 x 64 output tile) CTAs:
//   blk_fin_gram: E = V^H V - I (upper tiles, mirrored);
//   blk_fin_z:    Z[:, rank_k] = v_k - (V E)_k / 2 (a plain copy without the step).
// Each output keeps one accumulator over the contraction index in increasing
// order: the rounding sequence of the on-chip finalisation.
enum : int { kFinBT = 64, kFinKC = 16, kFinThreads = 256 };

template <class T, bool ConjA>
__device__ __forceinline__ void fin_mac(T (&acc)[4][4], const T (*As)[kFinBT + 1], const T (*Bs)[kFinBT + 1],
                                        int tr, int tc, int kmax) {
    auto step = [&](int kk) {
        T x[4], y[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) { x[u] = As[kk][tr + 16 * u]; y[u] = Bs[kk][tc + 16 * u]; }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = ConjA ? cfma(x[u], y[v], acc[u][v]) : fma_s(x[u], y[v], acc[u][v]);
    };
    if (kmax == kFinKC) {
#pragma unroll
        for (int kk = 0; kk < kFinKC; ++kk) step(kk);
    } else {
        for (int kk = 0; kk < kmax; ++kk) step(kk);
    }
}

__device__ __forceinline__ bool fin_skip(const BlockedArgs& a, const BlkShape& sh, int b) {
    return a.state[4 * b] < 0 || !(sh.trans ? a.wantU : a.wantV);
}

template <class T>
__global__ void __launch_bounds__(kFinThreads) blk_fin_gram(const BlockedArgs a) {
    using R = Real<T>;
    const int b = blockIdx.x, ta = blockIdx.y, tb = blockIdx.z, tid = threadIdx.x;
    if (ta > tb) return;
    const BlkShape sh = blk_shape(a, b);
    const int N = sh.N, r0 = ta * kFinBT, c0 = tb * kFinBT, tr = tid & 15, tc = tid >> 4;
    if (c0 >= N || fin_skip(a, sh, b)) return;
    __shared__ T As[kFinKC][kFinBT + 1], Bs[kFinKC][kFinBT + 1];
    const T* V = static_cast<const T*>(a.Vw) + sh.oV;                    // N x N, ld N
    T* E = static_cast<T*>(a.T) + sh.oT + sh.M;                           // N x N, ld N
    const T zero = make_s<T>(0);
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = zero;
    for (int i0 = 0; i0 < N; i0 += kFinKC) {
        for (int e = tid; e < kFinKC * kFinBT; e += kFinThreads) {
            const int kk = e % kFinKC, cc = e / kFinKC, i = i0 + kk;
            As[kk][cc] = (i < N && r0 + cc < N) ? V[i + (long long)(r0 + cc) * N] : zero;
            Bs[kk][cc] = (i < N && c0 + cc < N) ? V[i + (long long)(c0 + cc) * N] : zero;
        }
        __syncthreads();
        fin_mac<T, true>(acc, As, Bs, tr, tc, min(kFinKC, N - i0));
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            const int r = r0 + tr + 16 * u, c = c0 + tc + 16 * v;
            if (r >= N || c >= N || r > c) continue;
            T x = acc[u][v];
            if (r == c) x = make_s<T>(re(x) - R(1));
            E[r + (long long)c * N] = x;
            E[c + (long long)r * N] = conj_s(x);
        }
}

template <class T>
__global__ void __launch_bounds__(kFinThreads) blk_fin_z(const BlockedArgs a) {
    using R = Real<T>;
    const int b = blockIdx.x, ti = blockIdx.y, tk = blockIdx.z, tid = threadIdx.x;
    const BlkShape sh = blk_shape(a, b);
    const int N = sh.N, r0 = ti * kFinBT, c0 = tk * kFinBT, tr = tid & 15, tc = tid >> 4;
    if (r0 >= N || c0 >= N || fin_skip(a, sh, b)) return;
    __shared__ T As[kFinKC][kFinBT + 1], Bs[kFinKC][kFinBT + 1];
    const bool correct = !(a.flags & 1);
    const T* V = static_cast<const T*>(a.Vw) + sh.oV;
    const T* E = static_cast<const T*>(a.T) + sh.oT + sh.M;
    const int* rank = fin_rank<T>(a, sh);
    const int mid = blk_mid(a, b);
    T* Z;
    long long ldz;
    if (sh.trans) {
        Z = a.Up ? static_cast<T*>(a.Up[mid]) : static_cast<T*>(a.U) + (long long)mid * a.sU;
        ldz = a.ldup ? a.ldup[mid] : a.ldu;
    } else {
        Z = a.Vp ? static_cast<T*>(a.Vp[mid]) : static_cast<T*>(a.V) + (long long)mid * a.sV;
        ldz = a.ldvp ? a.ldvp[mid] : a.ldv;
    }
    const T zero = make_s<T>(0);
    T acc[4][4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = zero;
    if (correct) {
        for (int j0 = 0; j0 < N; j0 += kFinKC) {
            for (int e = tid; e < kFinKC * kFinBT; e += kFinThreads) {
                const int rr = e % kFinBT, ka = e / kFinBT;
                As[ka][rr] = (j0 + ka < N && r0 + rr < N) ? V[(r0 + rr) + (long long)(j0 + ka) * N] : zero;
                const int kb = e % kFinKC, cc = e / kFinKC;
                Bs[kb][cc] = (j0 + kb < N && c0 + cc < N) ? E[(j0 + kb) + (long long)(c0 + cc) * N] : zero;
            }
            __syncthreads();
            fin_mac<T, false>(acc, As, Bs, tr, tc, min(kFinKC, N - j0));
            __syncthreads();
        }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
        const int k = c0 + tc + 16 * v;
        if (k >= N) continue;
        T* zc = Z + (long long)rank[k] * ldz;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = r0 + tr + 16 * u;
            if (i >= N) continue;
            T z = V[i + (long long)k * N];
            if (correct) z = sub(z, scale(acc[u][v], R(0.5)));
            zc[i] = z;
        }
    }
}

}  // namespace bsvd
