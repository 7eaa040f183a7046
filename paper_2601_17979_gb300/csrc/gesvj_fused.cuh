// gesvj_fused.cuh -- the fused batched one-sided Jacobi SVD kernel.
//
// One CTA solves one matrix with the whole working matrix W (m x n, A scaled)
// and V (n x n) resident in shared memory, so A is read from HBM once and
// U, Sigma, V are written once (the single-kernel path of Sec. 7.1, here for
// the blocked method).  Per outer sweep the CTA walks the round-robin block
// ordering (Sec. 4.1): l-1 rounds of l/2 disjoint block pairs; thread groups
// take the pairs of a round concurrently.  Per pair (i, j):
//   S2  G = [W_i W_j]^H [W_i W_j]             (Eq. block-gram), upper triangle
//   S3  one sweep of Alg. 1 on G (Design-2, Sec. 5): 2nb-1 parallel steps of
//       nb disjoint rotations, Eq. (sin-cos), accumulated into J
//   S4/S5  [W_i W_j] <- [W_i W_j] J, [V_i V_j] <- [V_i V_j] J, each element
//       read and written once (Design-3, Alg. 4); skipped when no rotation
//       fired (the pair-level mask of Design-4, Sec. 6)
// A matrix is converged after a sweep in which no rotation fired.  Then
// sigma_k = ||w_k||_2, a stable descending sort, U = W Sigma^-1 (Alg. 2), and
// one Newton-Schulz step V <- V - V (V^H V - I) / 2 that restores the
// orthogonality V loses over many J products.
#pragma once

#include <type_traits>

#include "fused_f32.cuh"
#include "jacobi_common.cuh"
#include "tc_f32.cuh"

namespace bsvd {

constexpr int kMaxSweeps = 128;   // per-sweep flags kept in shared memory

// Kernel arguments (type-erased pointers; layout computed on the host).
struct FusedArgs {
    int M, N;              // working shape, M >= N (A^H when the caller's m < n)
    int trans;             // 1: W = A^H
    int m, n;              // caller's shape
    int l, L, Np;          // l >= 2 real blocks, L = l + (l odd), Np = l * nb columns
    int ldw, ldvs, lde;    // shared-memory leading dimensions
    int offW, offV, offG, offMisc, groupBytes;
    // strided addressing (p* == nullptr) or pointer arrays
    const void* A; long long sA; int lda; const void* const* Ap; const int* ldap;
    const void* V0; long long sV0; int ldv0;   // initial V (N x N, by matrix id) or nullptr for I
    void* S; long long sS; void* const* Sp;
    void* U; long long sU; int ldu; void* const* Up; const int* ldup;
    void* V; long long sV; int ldv; void* const* Vp; const int* ldvp;
    const int* index;      // matrix ids of this launch, or nullptr for 0..grid-1
    int in_local;          // 1: strided A and V0 by launch position, outputs by matrix id
    int* info; int* sweeps;
    double tol;
    int max_sweeps, inner_sweeps, flags;
    int wantU, wantV;
};

// bsvd_opts.flags bits read by the kernels: 0 no Newton-Schulz step on V;
// 7 real FP32 Gram and update on the FMA pipes (register tiles) instead of
// the tensor cores; 8 single-precision rotations and pair test in FP64.
enum : int { kFlagNoVCorrection = 1, kFlagF32Ffma = 128, kFlagWideAngles = 256 };

// Shared-memory bytes of one thread group's scratch (G, J, rotation table).
// Working shape and leading dimensions of one matrix: M >= N (A^H when
// m < n), l >= 2 blocks of NB columns (padded), and for FP32 16-byte aligned
// columns (an odd multiple of 4 floats) for the float4 tiles, for the other
// types an odd leading dimension (different columns in different banks).
template <class T, int NB>
__host__ __device__ inline void fused_dims(int m, int n, FusedArgs& a) {
    a.m = m;
    a.n = n;
    a.trans = m < n;
    a.M = m < n ? n : m;
    a.N = m < n ? m : n;
    const int M = a.M, N = a.N;
    const int l = N > 2 * NB ? (N + NB - 1) / NB : 2;
    a.l = l;
    a.L = l + (l & 1);
    a.Np = l * NB;
    if (std::is_same<T, float>::value) {
        a.ldw = (M + 3) & ~3;
        if (a.ldw % 8 == 0) a.ldw += 4;
        a.ldvs = (N + 3) & ~3;
        if (a.ldvs % 8 == 0) a.ldvs += 4;
    } else {
        a.ldw = M | 1;
        a.ldvs = N | 1;
    }
    a.lde = ((long long)(N | 1) * N <= (long long)a.ldw * a.Np) ? (N | 1) : N;
}

// Elements of the W + V working arrays of one matrix (V after W at a 16-byte
// boundary), for a global-memory slot.
template <class T>
__host__ __device__ inline long long fused_slot_elems(const FusedArgs& a) {
    const long long per16 = 16 / (long long)sizeof(T) > 0 ? 16 / (long long)sizeof(T) : 1;
    const long long w = ((long long)a.ldw * a.Np + per16 - 1) / per16 * per16;
    return w + (long long)a.ldvs * a.Np;
}

// FP32 adds J as split-TF32 fragments for the tensor-core update (nb >= 8:
// 8 (2nb)^2 bytes) or J^T for the FFMA-tiled update (nb = 4), 16-byte
// aligned; the other types a second J (the previous pair's, for the
// deferred V update).
template <class T, int NB>
__host__ __device__ constexpr int fused_group_bytes() {
    return ((2 * (2 * NB) * (2 * NB + 1) * (int)sizeof(T) + InnerTables<T, NB>::bytes() + 15) & ~15) +
           (std::is_same<T, float>::value ? (NB >= 8 ? 8 * (2 * NB) * (2 * NB) : (2 * NB) * (2 * NB) * 4)
                                          : (((2 * NB) * (2 * NB + 1) * (int)sizeof(T) + 15) & ~15));
}

// The V update of a block pair, [V_i V_j] <- [V_i V_j] J, run by whole warps
// at a time: a warp takes 32 / 2nb rows, lane c of a row computing output
// column c (summed over k in order, like the on-chip A update) and writing
// it after the warp has read the row.  Used to defer a pair's V update into
// the next pair step's inner sweep, where the FP64 pipe has room.
template <class T, int NB>
struct DeferredV {
    T* V;
    int ldv, rows;
    const T* J;        // the pair's J (ld 2nb + 1), or nullptr: nothing pending
    int bi, bj;
    __device__ __forceinline__ int tasks() const { return (rows + 32 / (2 * NB) - 1) / (32 / (2 * NB)); }
    __device__ __forceinline__ void operator()(int wt) const {
        constexpr int TWO = 2 * NB, LDG = TWO + 1, RPW = 32 / TWO;
        if (!J || wt >= tasks()) return;                      // uniform over the warp
        const int lane = threadIdx.x & 31, r = wt * RPW + lane / TWO, c = lane % TWO;
        T acc = make_s<T>(0);
        if (r < rows) {
#pragma unroll
            for (int k = 0; k < TWO; ++k) {
                const int ck = k < NB ? bi * NB + k : bj * NB + k - NB;
                acc = fma_s(V[r + (long long)ck * ldv], J[k + c * LDG], acc);
            }
        }
        __syncwarp();
        if (r < rows) V[r + (long long)(c < NB ? bi * NB + c : bj * NB + c - NB) * ldv] = acc;
    }
};

// Real FP32 keeps two CTAs per SM (its shared memory allows them).
template <class T>
constexpr int fused_min_blocks() { return std::is_same<T, float>::value ? 2 : 1; }

// The whole solve of matrix `mid` by one CTA: load, sweeps, finalise.  W
// (ldw x Np) and Vs (ldvs x Np) are the working arrays -- shared memory for
// the on-chip kernel, a global-memory slot for the persistent one; the Gram
// blocks, rotation tables and flags are always in shared memory at the
// offsets of `a`.  All threads of the CTA call it and return together.
template <class T, int NB, int NG, int GT, bool OnChip>
__device__ __forceinline__ void fused_solve(const FusedArgs& a, const int mid, const int lid, T* const W,
                                            T* const Vs, unsigned char* const smem) {
    using R = Real<T>;
    constexpr int TWO = 2 * NB, LDG = TWO + 1, NT = NG * GT, NW = NT / 32;

    const int tid = threadIdx.x, g = tid / GT, gt = tid % GT, lane = tid & 31, warp = tid >> 5;
    const int M = a.M, N = a.N, ldw = a.ldw, ldvs = a.ldvs;
    const bool needVs = a.trans ? a.wantU : a.wantV;   // V is part of the output
    const bool wantWout = a.trans ? a.wantV : a.wantU; // W / sigma is part of the output

    unsigned char* gb = smem + a.offG + g * a.groupBytes;
    T* G = reinterpret_cast<T*>(gb);
    T* const J0 = G + TWO * LDG;
    const InnerTables<T, NB> tb(J0 + TWO * LDG);
    // after the tables, 16-byte aligned: J^T for the FP32 tiled update, or
    // the second J buffer of the other types
    unsigned char* const gb_tail = gb + ((2 * TWO * LDG * (int)sizeof(T) + InnerTables<T, NB>::bytes() + 15) & ~15);
    float* Jt = reinterpret_cast<float*>(gb_tail);
    T* const J1 = reinterpret_cast<T*>(gb_tail);
    T* J = J0;
    int* swflag = reinterpret_cast<int*>(smem + a.offMisc);   // [kMaxSweeps] per-sweep "rotated"
    int* iscr = swflag + kMaxSweeps;                           // [4]: 0 bad input, 1 pivot row
    T* bcast = reinterpret_cast<T*>(iscr + 4);                 // [2] broadcast slot
    R* red = reinterpret_cast<R*>(bcast + 2);                  // [NW, padded to 4]
    R* sig = red + ((NW + 3) & ~3);                            // [N, padded to 4]
    int* rank = reinterpret_cast<int*>(sig + ((N + 3) & ~3));  // [N]

    // ---- load W = A (or A^H) and find max |a| and non-finite entries ----------
    const int sid = a.in_local ? lid : mid;                    // position of strided inputs
    const T* A = a.Ap ? static_cast<const T*>(a.Ap[mid]) : static_cast<const T*>(a.A) + (long long)sid * a.sA;
    const int lda = a.ldap ? a.ldap[mid] : a.lda;
    for (int e = tid; e < kMaxSweeps; e += NT) swflag[e] = 0;
    R mx = 0;
    int nonfin = 0;
    for (int e = tid; e < a.m * a.n; e += NT) {
        const int i = e % a.m, j = e / a.m;                   // coalesced along A's rows
        const T x = A[i + (long long)j * lda];
        if (!finite_s(x)) nonfin = 1; else mx = fmax(mx, maxabs(x));
        if (a.trans) W[j + i * ldw] = conj_s(x);
        else         W[i + j * ldw] = x;
    }
    for (int e = tid; e < M * (a.Np - N); e += NT) W[(e % M) + (N + e / M) * ldw] = make_s<T>(0);
    if (ldw > M)   // rows M..ldw-1 (read, never used, by the FP32 tiles)
        for (int e = tid; e < (ldw - M) * a.Np; e += NT) W[M + e % (ldw - M) + (e / (ldw - M)) * ldw] = make_s<T>(0);
    if (needVs && ldvs > N)
        for (int e = tid; e < (ldvs - N) * a.Np; e += NT) Vs[N + e % (ldvs - N) + (e / (ldvs - N)) * ldvs] = make_s<T>(0);
    if (needVs) {
        const T* V0 = a.V0 ? static_cast<const T*>(a.V0) + (long long)sid * a.sV0 : nullptr;
        for (int e = tid; e < N * a.Np; e += NT) {
            const int i = e % N, j = e / N;
            Vs[i + j * ldvs] = (V0 && j < N) ? V0[i + (long long)j * a.ldv0] : make_s<T>(i == j && !V0 ? 1 : 0);
        }
    }
    mx = warp_max(mx);
    const bool wbad = __any_sync(0xffffffffu, nonfin);
    if (lane == 0) red[warp] = wbad ? R(-1) : mx;             // -1 marks a non-finite entry
    __syncthreads();
    if (tid == 0) {
        R m2 = 0;
        int b = 0;
        for (int w = 0; w < NW; ++w) { b |= red[w] < 0; m2 = fmax(m2, red[w]); }
        red[0] = m2;
        iscr[0] = b;
    }
    __syncthreads();
    const bool bad = iscr[0] != 0;
    const R amax = red[0];
    const int ex = (amax > 0) ? ilogb_r(amax) : 0;             // W = A * 2^-ex, exact

    // S and the output pointers
    R* Sout = a.Sp ? static_cast<R*>(a.Sp[mid]) : static_cast<R*>(a.S) + (long long)mid * a.sS;
    T* Uout = nullptr;
    T* Vout = nullptr;
    int ldu = 1, ldv = 1;
    if (a.wantU) {
        Uout = a.Up ? static_cast<T*>(a.Up[mid]) : static_cast<T*>(a.U) + (long long)mid * a.sU;
        ldu = a.ldup ? a.ldup[mid] : a.ldu;
    }
    if (a.wantV) {
        Vout = a.Vp ? static_cast<T*>(a.Vp[mid]) : static_cast<T*>(a.V) + (long long)mid * a.sV;
        ldv = a.ldvp ? a.ldvp[mid] : a.ldv;
    }
    const int k_out = N;   // min(m, n)

    if (bad) {
        for (int e = tid; e < k_out; e += NT) Sout[e] = nan_s<R>();
        if (Uout) for (int e = tid; e < a.m * k_out; e += NT) Uout[(e % a.m) + (long long)(e / a.m) * ldu] = nan_s<T>();
        if (Vout) for (int e = tid; e < a.n * k_out; e += NT) Vout[(e % a.n) + (long long)(e / a.n) * ldv] = nan_s<T>();
        if (tid == 0) {
            a.info[mid] = -1;
            if (a.sweeps) a.sweeps[mid] = 0;
        }
        return;
    }
    if (ex != 0)
        for (int e = tid; e < M * N; e += NT) {
            T* p = &W[(e % M) + (e / M) * ldw];
            *p = scalb_s(*p, -ex);
        }
    __syncthreads();

    // ---- sweeps -----------------------------------------------------------------
    const R tol = (R)a.tol;
    int sw = 0;
    bool converged = false;
    // FP64 and complex on chip: a pair's V update is deferred to the group's
    // next pair step and run by the J-update warps during its inner sweep
    // (same arithmetic; the V blocks are read by nothing else in between).
    // Not with V in global memory: a warp reads one row of V, which in
    // global memory would touch a separate cache line per element.
    constexpr bool kDefer = OnChip && !std::is_same<T, float>::value;
    DeferredV<T, NB> dv{Vs, ldvs, N, nullptr, 0, 0};
    while (sw < a.max_sweeps) {
        for (int r = 0; r < a.L - 1; ++r) {
            for (int q0 = 0; q0 < a.L / 2; q0 += NG) {
              const int q = q0 + g;
              bool stepped = false;                            // ran an inner sweep this time
              if (q < a.L / 2) do {
                int bi, bj;
                rr_pair(a.L, r, q, bi, bj);
                if (bj >= a.l) break;                          // phantom block
                auto col = [&](int c) { return c < NB ? bi * NB + c : bj * NB + (c - NB); };

                // S2: G = P^H P, upper triangle, mirrored to keep G Hermitian.
                // Lanes l and l+16 of a warp sum the same entry over the two
                // halves of the rows [0, M/2) and [M/2, M); one shuffle adds them.
                // FP32: split-TF32 tensor-core tiles (tc_f32.cuh), or
                // FFMA register tiles for nb = 4 (fused_f32.cuh).
                if constexpr (std::is_same<T, float>::value) {
                    if (NB >= 8 && !(a.flags & kFlagF32Ffma)) gram_f32_mma<NB < 8 ? 8 : NB, GT>(W, ldw, M, bi * NB, bj * NB, G, gt);
                    else gram_f32_tiled<NB, GT>(W, ldw, M, bi * NB, bj * NB, G, gt);
                } else if constexpr (!OnChip) {
                    // W in global memory: 2 x 2 tiles of upper entries per lane
                    // pair, four independent sums (half the loads per FMA of
                    // one entry at a time); each entry still sums k in order
                    // over its half of the rows, so the bits are those of the
                    // branch below
                    constexpr int TH = TWO / 2, NTL = TH * (TH + 1) / 2, NWG = GT / 32;
                    const int wg = gt >> 5, kh = (gt >> 4) & 1, el = gt & 15;
                    const int kb = kh ? M / 2 : 0, ke = kh ? M : M / 2;
                    for (int t0 = wg * 16; t0 < NTL; t0 += NWG * 16) {
                        const int t = t0 + el;
                        int ti = 0, tj = 0;
                        T acc[2][2];
#pragma unroll
                        for (int u = 0; u < 2; ++u)
#pragma unroll
                            for (int v = 0; v < 2; ++v) acc[u][v] = make_s<T>(0);
                        if (t < NTL) {
                            tri_index(t, ti, tj);
                            const T* x0 = W + col(2 * ti) * ldw;
                            const T* x1 = W + col(2 * ti + 1) * ldw;
                            const T* y0 = W + col(2 * tj) * ldw;
                            const T* y1 = W + col(2 * tj + 1) * ldw;
#pragma unroll 4
                            for (int k = kb; k < ke; ++k) {
                                const T a0 = x0[k], a1 = x1[k], b0 = y0[k], b1 = y1[k];
                                acc[0][0] = cfma(a0, b0, acc[0][0]);
                                acc[0][1] = cfma(a0, b1, acc[0][1]);
                                acc[1][0] = cfma(a1, b0, acc[1][0]);
                                acc[1][1] = cfma(a1, b1, acc[1][1]);
                            }
                        }
#pragma unroll
                        for (int u = 0; u < 2; ++u)
#pragma unroll
                            for (int v = 0; v < 2; ++v) acc[u][v] = add(acc[u][v], shfl_xor_s(acc[u][v], 16));
                        if (kh == 0 && t < NTL) {
#pragma unroll
                            for (int u = 0; u < 2; ++u)
#pragma unroll
                                for (int v = 0; v < 2; ++v) {
                                    const int ca = 2 * ti + u, cb = 2 * tj + v;
                                    if (ca > cb) continue;             // lower entry of a diagonal tile
                                    T x = acc[u][v];
                                    if (ca == cb) x = make_s<T>(re(x));
                                    G[ca + cb * LDG] = x;
                                    G[cb + ca * LDG] = conj_s(x);
                                }
                        }
                    }
                } else {
                    constexpr int NUP = TWO * (TWO + 1) / 2, NWG = GT / 32;
                    const int wg = gt >> 5, kh = (gt >> 4) & 1, el = gt & 15;
                    const int kb = kh ? M / 2 : 0, ke = kh ? M : M / 2;
                    for (int e0 = wg * 16; e0 < NUP; e0 += NWG * 16) {
                        const int e = e0 + el;
                        int ca = 0, cb = 0;
                        T acc = make_s<T>(0);
                        if (e < NUP) {
                            tri_index(e, ca, cb);
                            const T* x = W + col(ca) * ldw;
                            const T* y = W + col(cb) * ldw;
                            for (int k = kb; k < ke; ++k) acc = cfma(x[k], y[k], acc);
                        }
                        acc = add(acc, shfl_xor_s(acc, 16));
                        if (kh == 0 && e < NUP) {
                            if (ca == cb) acc = make_s<T>(re(acc));
                            G[ca + cb * LDG] = acc;
                            G[cb + ca * LDG] = conj_s(acc);
                        }
                    }
                }
                group_sync(g, GT);

                // S3: inner Jacobi sweeps on G (round-robin over the 2nb indices)
                int seen;
                stepped = true;
                if constexpr (kDefer) {
                    int ns = 0;
                    seen = inner_jacobi<T, NB, GT>(G, J, tb, tol, a.inner_sweeps, gt, g + 1, dv, &ns,
                                                   (a.flags & kFlagWideAngles) != 0);
                    if (dv.J) {   // the deferred V rows the background warps did not reach
                        for (int wt = ns * inner_background_warps<GT>() + (gt >> 5); wt < dv.tasks(); wt += GT / 32)
                            dv(wt);
                        dv.J = nullptr;
                    }
                    group_sync(g, GT);
                } else {
                    seen = inner_jacobi<T, NB, GT>(G, J, tb, tol, a.inner_sweeps, gt, g + 1, NoBackground(), nullptr,
                                                   (a.flags & kFlagWideAngles) != 0);
                }
                if (seen == 0) break;                       // J = I: pair masked (Design-4)
                if (gt == 0) swflag[sw] = 1;

                // S4/S5: [W_i W_j] <- [W_i W_j] J and [V_i V_j] <- [V_i V_j] J.
                // A warp takes 16 rows at a time; lanes l and l+16 both read row
                // l and write the first and the second nb outputs of it, so the
                // M + n rows spread evenly over the group.  FP32: register tiles.
                if constexpr (std::is_same<T, float>::value) {
                    if (NB >= 8 && !(a.flags & kFlagF32Ffma)) {
                        constexpr int NBT = NB < 8 ? 8 : NB;       // (nb = 4 never takes this branch)
                        uint4* Jf = reinterpret_cast<uint4*>(gb_tail);
                        j_fragments<NBT, GT>(J, Jf, gt);
                        group_sync(g, GT);
                        update_f32_mma<NBT, GT>(W, ldw, M, Vs, ldvs, needVs ? N : 0, bi * NB, bj * NB, Jf, gt);
                    } else {
                        for (int e = gt; e < TWO * TWO; e += GT) Jt[(e / TWO) + (e % TWO) * TWO] = J[(e % TWO) + (e / TWO) * LDG];
                        group_sync(g, GT);
                        update_f32_tiled<NB, GT, 2>(W, ldw, ldw, Vs, ldvs, needVs ? ldvs : 0, bi * NB, bj * NB, Jt, gt, g + 1);
                    }
                } else if constexpr (std::is_same<T, float2>::value) {
                    // complex64: 4 rows x 2nb/8 columns per lane (columns
                    // cg, cg + 8, ...: conflict-free J reads with its padded
                    // stride), a 16-row slab per warp; each output still sums
                    // k in order, the bits of the generic branch below.  The
                    // generic mapping (one row, nb columns per lane) reads J
                    // once per multiply-add, two-way bank-conflicted, and is
                    // bound by shared-memory wavefronts in single precision.
                    constexpr int CJ = TWO / 8, NWG = GT / 32;
                    const int rows = M + (needVs && !kDefer ? N : 0);
                    const int wg = gt >> 5, cg = gt & 7, rs = (gt >> 3) & 3;
                    for (int r0 = wg * 16; r0 < rows; r0 += NWG * 16) {
                        T* X[4];
                        int ldx[4];
                        bool ok[4];
#pragma unroll
                        for (int i = 0; i < 4; ++i) {
                            const int r = r0 + rs + 4 * i;
                            ok[i] = r < rows;
                            X[i] = r < M ? W + r : Vs + (r - M);
                            ldx[i] = r < M ? ldw : ldvs;
                        }
                        T acc[4][CJ];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < CJ; ++j) acc[i][j] = make_s<T>(0);
#pragma unroll 4
                        for (int k = 0; k < TWO; ++k) {
                            const int ck = col(k);
                            T xk[4], jk[CJ];
#pragma unroll
                            for (int i = 0; i < 4; ++i) xk[i] = ok[i] ? X[i][ck * ldx[i]] : make_s<T>(0);
#pragma unroll
                            for (int j = 0; j < CJ; ++j) jk[j] = J[k + (cg + 8 * j) * LDG];
#pragma unroll
                            for (int i = 0; i < 4; ++i)
#pragma unroll
                                for (int j = 0; j < CJ; ++j) acc[i][j] = fma_s(xk[i], jk[j], acc[i][j]);
                        }
                        __syncwarp();
#pragma unroll
                        for (int i = 0; i < 4; ++i)
                            if (ok[i]) {
#pragma unroll
                                for (int j = 0; j < CJ; ++j) X[i][col(cg + 8 * j) * ldx[i]] = acc[i][j];
                            }
                    }
                    if (kDefer && needVs) {   // this pair's V update, run during the next pair step
                        dv.J = J; dv.bi = bi; dv.bj = bj;
                        J = (J == J0) ? J1 : J0;
                    }
                } else {
                    const int rows = M + (needVs && !kDefer ? N : 0);   // on chip V is deferred (DeferredV)
                    const int wg = gt >> 5, half = (gt >> 4) & 1, rl = gt & 15;
                    constexpr int NWG = GT / 32;
                    for (int r0 = wg * 16; r0 < rows; r0 += NWG * 16) {
                        const int i = r0 + rl;
                        const bool ok = i < rows;
                        T* X = W;
                        int ld = ldw, row = i;
                        if (i >= M) { X = Vs; ld = ldvs; row = i - M; }
                        // nb accumulators, each summed over k in order (the
                        // multi-kernel path's order); x is read one k at a time
                        T acc[NB];
#pragma unroll
                        for (int c = 0; c < NB; ++c) acc[c] = make_s<T>(0);
                        if (ok) {
#pragma unroll
                            for (int k = 0; k < TWO; ++k) {
                                const T xk = X[row + col(k) * ld];
#pragma unroll
                                for (int c = 0; c < NB; ++c) acc[c] = fma_s(xk, J[k + (half * NB + c) * LDG], acc[c]);
                            }
                        }
                        __syncwarp();
                        if (ok) {
#pragma unroll
                            for (int c = 0; c < NB; ++c) X[row + col(half * NB + c) * ld] = acc[c];
                        }
                    }
                    if (kDefer && needVs) {   // this pair's V update, run during the next pair step
                        dv.J = J; dv.bi = bi; dv.bj = bj;
                        J = (J == J0) ? J1 : J0;
                    }
                }
                group_sync(g, GT);
              } while (0);
              if (kDefer && !stepped && dv.J) {   // no pair step (phantom or none): apply the pending V update now
                  for (int wt = gt >> 5; wt < dv.tasks(); wt += GT / 32) dv(wt);
                  dv.J = nullptr;
                  group_sync(g, GT);
              }
              // FP64 / complex with several pairs per group in a round: the V
              // updates still deferred from the previous round finish during
              // each group's first pair step; a barrier after it keeps them
              // apart from the deferred updates of this round's pairs
              if (kDefer && q0 == 0 && a.L / 2 > NG) __syncthreads();
            }
            __syncthreads();
        }
        const int fired = swflag[sw];
        ++sw;
        if (!fired) { converged = true; break; }
    }
    if constexpr (kDefer) {   // the last pending V update
        if (dv.J)
            for (int wt = gt >> 5; wt < dv.tasks(); wt += GT / 32) dv(wt);
        __syncthreads();
    }

    // ---- finalise (Alg. 2): sigma, sort, U = W Sigma^-1, V correction --------
    {
        T* Y = a.trans ? Vout : Uout;
        T* Z = a.trans ? Uout : Vout;
        const long long ldy = a.trans ? ldv : ldu, ldz = a.trans ? ldu : ldv;
        const FinalScratch<T> fs{sig, rank, red, iscr, bcast};
        // W's space is free once Y is written: it holds the completion vector and V^H V - I
        finalize_outputs<T, NT>(W, ldw, Vs, ldvs, M, N, ex, W, W, a.lde,
                                !(a.flags & kFlagNoVCorrection), Sout, Y, ldy, wantWout, Z, ldz,
                                needVs, fs);
    }
    if (tid == 0) {
        a.info[mid] = converged ? 0 : sw;
        if (a.sweeps) a.sweeps[mid] = sw;
    }
}

// Resident CTAs the register allocation must allow: the type's count for
// 256-thread CTAs, scaled up for smaller CTAs (nb = 4, 8: 64 and 128
// threads) so that small matrices keep as many threads per SM.
template <int Base, int NT>
constexpr int min_blocks_for() { return Base * (256 / NT > 1 ? 256 / NT : 1); }

template <class T, int NB, int NG, int GT>
__global__ void __launch_bounds__(NG * GT, (min_blocks_for<fused_min_blocks<T>(), NG * GT>()))
gesvj_fused_kernel(const FusedArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int mid = a.index ? a.index[blockIdx.x] : (int)blockIdx.x;
    fused_solve<T, NB, NG, GT, true>(a, mid, (int)blockIdx.x, reinterpret_cast<T*>(smem + a.offW),
                                     reinterpret_cast<T*>(smem + a.offV), smem);
}

// Pointer-array batches of any shapes in persistent launches: each CTA
// takes the next matrix from a work queue (ids in `order`, largest first),
// lays it out in its working arrays and solves it with the same per-matrix
// code as the on-chip kernel.  A launch serves one segment of a batch: one
// block width, and either working arrays in shared memory (OnChip: W and V
// of the segment's largest matrix fit there; the layout of the on-chip
// kernel) or in the CTA's own global-memory slot.  With `done` given, the
// CTA raises done[id] once matrix id's outputs are written, so a host that
// polls the flags can hand each result out before the launch ends; with
// `abort` given, a CTA that finds it set takes no further matrix (those not
// started keep their done flag at zero).
struct PersistArgs {
    FusedArgs base;            // outputs, options, jobs and shared-memory offsets
    const int* mm;             // m of each matrix (by id)
    const int* nn;             // n of each matrix (by id)
    const int* order;          // queue of ids
    int count;                 // queue length
    int* head;                 // queue head, zero at launch
    void* ws;                  // gridDim.x slots of slot_elems elements (global-slot launches)
    long long slot_elems;
    int* done;                 // per-id completion flags (host-mapped memory) or nullptr
    const int* abort;          // nonzero: take no further matrix (host-mapped) or nullptr
};

// Release store at system scope: every write this CTA made before the barrier
// that precedes it (each writer fenced at system scope) is visible to the host
// before the flag is.
__device__ __forceinline__ void store_release_sys(int* p, int v) {
    asm volatile("st.release.sys.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Two CTAs per SM for every type but complex128: with W in global memory the
// kernel is latency-bound, and a second CTA's groups hide more of it than
// the registers the cap (128) takes away.
template <class T>
constexpr int persist_min_blocks() {
    return std::is_same<T, double2>::value ? 1 : 2;
}

// On-chip launches keep the on-chip kernel's occupancy (two CTAs per SM for
// real FP32, else one).
template <class T, bool OnChip>
constexpr int persist_blocks() { return OnChip ? fused_min_blocks<T>() : persist_min_blocks<T>(); }

template <class T, int NB, int NG, int GT, bool OnChip>
__global__ void __launch_bounds__(NG * GT, (min_blocks_for<persist_blocks<T, OnChip>(), NG * GT>()))
gesvj_persistent_kernel(const PersistArgs p) {
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ int s_mid;
    T* const slot = OnChip ? reinterpret_cast<T*>(smem) : static_cast<T*>(p.ws) + (long long)blockIdx.x * p.slot_elems;
    for (;;) {
        if (threadIdx.x == 0) {
            if (p.abort && *reinterpret_cast<const volatile int*>(p.abort)) {
                s_mid = -1;
            } else {
                const int k = atomicAdd(p.head, 1);
                s_mid = k < p.count ? p.order[k] : -1;
            }
        }
        __syncthreads();
        const int mid = s_mid;
        __syncthreads();                                   // all have read s_mid
        if (mid < 0) break;
        FusedArgs a = p.base;
        fused_dims<T, NB>(p.mm[mid], p.nn[mid], a);
        const long long per16 = 16 / (long long)sizeof(T) > 0 ? 16 / (long long)sizeof(T) : 1;
        T* const W = slot;
        T* const Vs = slot + ((long long)a.ldw * a.Np + per16 - 1) / per16 * per16;
        fused_solve<T, NB, NG, GT, OnChip>(a, mid, mid, W, Vs, smem);
        if (p.done) __threadfence_system();                // this thread's outputs before the flag
        __syncthreads();                                   // shared scratch reused next
        if (p.done && threadIdx.x == 0) store_release_sys(p.done + mid, 1);
    }
}

}  // namespace bsvd
