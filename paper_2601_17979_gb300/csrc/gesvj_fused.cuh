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

#include "scalar.cuh"

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
    void* S; long long sS; void* const* Sp;
    void* U; long long sU; int ldu; void* const* Up; const int* ldup;
    void* V; long long sV; int ldv; void* const* Vp; const int* ldvp;
    const int* index;      // matrix ids of this launch, or nullptr for 0..grid-1
    int* info; int* sweeps;
    double tol;
    int max_sweeps, inner_sweeps, flags;
    int wantU, wantV;
};

enum : int { kFlagNoVCorrection = 1 };

// Round-robin ordering on L (even) players (Brent and Luk; Sec. 3, Sec. 4.1):
// top row 0,2,4,..., bottom row 1,3,5,...; player 0 stays, the other L-1 sit on
// the ring top[1..k-1], bottom[k-1..0] and advance one place per round.
__device__ __forceinline__ int rr_start(int L, int pos) {
    const int k = L >> 1;
    return pos < k - 1 ? 2 * (pos + 1) : 2 * (L - 2 - pos) + 1;
}
__device__ __forceinline__ void rr_pair(int L, int r, int q, int& i, int& j) {
    const int ring = L - 1;
    const int a = (q == 0) ? 0 : rr_start(L, ((q - 1 - r) % ring + ring) % ring);
    const int b = rr_start(L, ((L - 2 - q - r) % ring + ring) % ring);
    i = min(a, b);
    j = max(a, b);
}

// e -> (a, b), a <= b, for the column-major upper triangle
__device__ __forceinline__ void tri_index(int e, int& a, int& b) {
    int c = (int)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
    while (c * (c + 1) / 2 > e) --c;
    while ((c + 1) * (c + 2) / 2 <= e) ++c;
    b = c;
    a = e - c * (c + 1) / 2;
}

__device__ __forceinline__ void group_sync(int g, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(g + 1), "r"(nthreads) : "memory");
}

template <class R> __device__ __forceinline__ R warp_max(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
template <class R> __device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum_s(float v) { return warp_sum(v); }
__device__ __forceinline__ double warp_sum_s(double v) { return warp_sum(v); }
__device__ __forceinline__ float2 warp_sum_s(float2 v) { return make_float2(warp_sum(v.x), warp_sum(v.y)); }
__device__ __forceinline__ double2 warp_sum_s(double2 v) { return make_double2(warp_sum(v.x), warp_sum(v.y)); }

// Shared-memory bytes of one thread group's scratch (G, J, rotation table).
template <class T, int NB>
__host__ __device__ constexpr int fused_group_bytes() {
    return ((2 * (2 * NB) * (2 * NB + 1) * (int)sizeof(T) + NB * (3 * (int)sizeof(Real<T>) + (int)sizeof(T)) +
             NB * 3 * 4 + 16) + 15) & ~15;
}

template <class T, int NB, int NG, int GT>
__global__ void __launch_bounds__(NG * GT)
gesvj_fused_kernel(const FusedArgs a) {
    using R = Real<T>;
    constexpr int TWO = 2 * NB, LDG = TWO + 1, NT = NG * GT, NW = NT / 32;
    extern __shared__ __align__(16) unsigned char smem[];

    const int tid = threadIdx.x, g = tid / GT, gt = tid % GT, lane = tid & 31, warp = tid >> 5;
    const int mid = a.index ? a.index[blockIdx.x] : (int)blockIdx.x;
    const int M = a.M, N = a.N, ldw = a.ldw, ldvs = a.ldvs;
    const bool needVs = a.trans ? a.wantU : a.wantV;   // V is part of the output
    const bool wantWout = a.trans ? a.wantV : a.wantU; // W / sigma is part of the output

    T* W = reinterpret_cast<T*>(smem + a.offW);
    T* Vs = reinterpret_cast<T*>(smem + a.offV);
    unsigned char* gb = smem + a.offG + g * a.groupBytes;
    T* G = reinterpret_cast<T*>(gb);
    T* J = G + TWO * LDG;
    R* rc = reinterpret_cast<R*>(J + TWO * LDG);
    R* rs = rc + NB;
    R* rt = rs + NB;
    T* rph = reinterpret_cast<T*>(rt + NB);
    int* rp = reinterpret_cast<int*>(rph + NB);
    int* rq = rp + NB;
    int* rf = rq + NB;
    int* gflag = rf + NB;
    int* swflag = reinterpret_cast<int*>(smem + a.offMisc);   // [kMaxSweeps] per-sweep "rotated"
    int* iscr = swflag + kMaxSweeps;                           // [4]: 0 bad input, 1 pivot row
    T* bcast = reinterpret_cast<T*>(iscr + 4);                 // [2] broadcast slot
    R* red = reinterpret_cast<R*>(bcast + 2);                  // [NW, padded to 4]
    R* sig = red + ((NW + 3) & ~3);                            // [N, padded to 4]
    int* rank = reinterpret_cast<int*>(sig + ((N + 3) & ~3));  // [N]

    // ---- load W = A (or A^H) and find max |a| and non-finite entries ----------
    const T* A = a.Ap ? static_cast<const T*>(a.Ap[mid]) : static_cast<const T*>(a.A) + (long long)mid * a.sA;
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
    if (needVs)
        for (int e = tid; e < N * a.Np; e += NT) Vs[(e % N) + (e / N) * ldvs] = make_s<T>((e % N) == (e / N) ? 1 : 0);
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
    while (sw < a.max_sweeps) {
        for (int r = 0; r < a.L - 1; ++r) {
            for (int q = g; q < a.L / 2; q += NG) {
                int bi, bj;
                rr_pair(a.L, r, q, bi, bj);
                if (bj >= a.l) continue;                       // phantom block
                auto col = [&](int c) { return c < NB ? bi * NB + c : bj * NB + (c - NB); };

                // S2: G = P^H P, upper triangle, mirrored to keep G Hermitian
                constexpr int NUP = TWO * (TWO + 1) / 2;
                for (int e = gt; e < NUP; e += GT) {
                    int ca, cb;
                    tri_index(e, ca, cb);
                    const T* x = W + col(ca) * ldw;
                    const T* y = W + col(cb) * ldw;
                    T acc = make_s<T>(0);
                    for (int k = 0; k < M; ++k) acc = cfma(x[k], y[k], acc);
                    if (ca == cb) acc = make_s<T>(re(acc));
                    G[ca + cb * LDG] = acc;
                    G[cb + ca * LDG] = conj_s(acc);
                }
                for (int e = gt; e < TWO * TWO; e += GT)
                    J[(e % TWO) + (e / TWO) * LDG] = make_s<T>((e % TWO) == (e / TWO) ? 1 : 0);
                if (gt == 0) *gflag = 0;
                group_sync(g, GT);

                // S3: inner Jacobi sweeps on G (round-robin over the 2nb indices)
                int seen = 0;
                for (int isw = 0; isw < a.inner_sweeps; ++isw) {
                    for (int s = 0; s < TWO - 1; ++s) {
                        if (gt < NB) {
                            int p, q2;
                            rr_pair(TWO, s, gt, p, q2);
                            const R gpp = re(G[p + p * LDG]), gqq = re(G[q2 + q2 * LDG]);
                            const T gpq = G[p + q2 * LDG];
                            const R apq = abs_s(gpq);
                            const bool fire = gpp > 0 && gqq > 0 && apq > 0 &&
                                              apq >= tol * sqrt_r(gpp) * sqrt_r(gqq);
                            R c = 1, sn = 0, t = 0;
                            T ph = make_s<T>(1);
                            if (fire) {
                                const R tau = (gpp - gqq) / (2 * apq);
                                t = (tau >= 0 ? R(1) : R(-1)) / (fabs(tau) + hypot_r(R(1), tau));
                                c = R(1) / sqrt_r(R(1) + t * t);
                                sn = t * c;
                                ph = divr(gpq, apq);
                                atomicAdd(gflag, 1);
                            }
                            rc[gt] = c; rs[gt] = sn; rt[gt] = t; rph[gt] = ph;
                            rp[gt] = p; rq[gt] = q2; rf[gt] = fire;
                        }
                        group_sync(g, GT);
                        // G <- R^H G R on 2x2 blocks (q1 <= q2), mirrored
                        constexpr int NBLK = NB * (NB + 1) / 2;
                        for (int e = gt; e < NBLK; e += GT) {
                            int q1, qq;
                            tri_index(e, q1, qq);
                            const bool f1 = rf[q1], f2 = rf[qq];
                            if (!f1 && !f2) continue;
                            const int p1 = rp[q1], r1 = rq[q1], p2 = rp[qq], r2 = rq[qq];
                            if (q1 == qq) {
                                const R tt = rt[q1];
                                const R apq = abs_s(G[p1 + r1 * LDG]);
                                G[p1 + p1 * LDG] = make_s<T>(re(G[p1 + p1 * LDG]) + tt * apq);
                                G[r1 + r1 * LDG] = make_s<T>(re(G[r1 + r1 * LDG]) - tt * apq);
                                G[p1 + r1 * LDG] = make_s<T>(0);
                                G[r1 + p1 * LDG] = make_s<T>(0);
                                continue;
                            }
                            T b00 = G[p1 + p2 * LDG], b01 = G[p1 + r2 * LDG];
                            T b10 = G[r1 + p2 * LDG], b11 = G[r1 + r2 * LDG];
                            if (f2) {   // columns (p2, r2) times R2
                                const R c2 = rc[qq];
                                const T es = scale(rph[qq], rs[qq]), ces = conj_s(es);
                                const T n00 = add(scale(b00, c2), mul(b01, ces));
                                const T n01 = sub(scale(b01, c2), mul(b00, es));
                                const T n10 = add(scale(b10, c2), mul(b11, ces));
                                const T n11 = sub(scale(b11, c2), mul(b10, es));
                                b00 = n00; b01 = n01; b10 = n10; b11 = n11;
                            }
                            if (f1) {   // rows (p1, r1) times R1^H
                                const R c1 = rc[q1];
                                const T es = scale(rph[q1], rs[q1]), ces = conj_s(es);
                                const T n00 = add(scale(b00, c1), mul(es, b10));
                                const T n10 = sub(scale(b10, c1), mul(ces, b00));
                                const T n01 = add(scale(b01, c1), mul(es, b11));
                                const T n11 = sub(scale(b11, c1), mul(ces, b01));
                                b00 = n00; b01 = n01; b10 = n10; b11 = n11;
                            }
                            G[p1 + p2 * LDG] = b00; G[p1 + r2 * LDG] = b01;
                            G[r1 + p2 * LDG] = b10; G[r1 + r2 * LDG] = b11;
                            G[p2 + p1 * LDG] = conj_s(b00); G[r2 + p1 * LDG] = conj_s(b01);
                            G[p2 + r1 * LDG] = conj_s(b10); G[r2 + r1 * LDG] = conj_s(b11);
                        }
                        // J <- J R for every rotating slot
                        for (int e = gt; e < TWO * NB; e += GT) {
                            const int i = e % TWO, qs = e / TWO;
                            if (!rf[qs]) continue;
                            const int p = rp[qs], q2 = rq[qs];
                            const R c = rc[qs];
                            const T es = scale(rph[qs], rs[qs]), ces = conj_s(es);
                            const T x = J[i + p * LDG], y = J[i + q2 * LDG];
                            J[i + p * LDG] = add(scale(x, c), mul(y, ces));
                            J[i + q2 * LDG] = sub(scale(y, c), mul(x, es));
                        }
                        group_sync(g, GT);
                    }
                    const int now = *gflag;
                    group_sync(g, GT);   // all have read gflag before the next sweep bumps it
                    const bool quiet = (now == seen);
                    seen = now;
                    if (quiet) break;                          // inner solve converged
                }
                if (seen == 0) continue;                       // J = I: pair masked (Design-4)
                if (gt == 0) swflag[sw] = 1;

                // S4/S5: [W_i W_j] <- [W_i W_j] J and [V_i V_j] <- [V_i V_j] J
                const int rows = M + (needVs ? N : 0);
                for (int i = gt; i < rows; i += GT) {
                    T* X;
                    int ld, row;
                    if (i < M) { X = W; ld = ldw; row = i; }
                    else       { X = Vs; ld = ldvs; row = i - M; }
                    T x[TWO];
#pragma unroll
                    for (int k = 0; k < TWO; ++k) x[k] = X[row + col(k) * ld];
#pragma unroll
                    for (int c = 0; c < TWO; ++c) {
                        T acc = make_s<T>(0);
#pragma unroll
                        for (int k = 0; k < TWO; ++k) acc = fma_s(x[k], J[k + c * LDG], acc);
                        X[row + col(c) * ld] = acc;
                    }
                }
                group_sync(g, GT);
            }
            __syncthreads();
        }
        const int fired = swflag[sw];
        ++sw;
        if (!fired) { converged = true; break; }
    }

    // ---- finalise: sigma_k = ||w_k||, stable descending sort ------------------
    for (int k = warp; k < N; k += NW) {
        R m2 = 0;
        for (int i = lane; i < M; i += 32) m2 = fmax(m2, maxabs(W[i + k * ldw]));
        m2 = warp_max(m2);
        R ss = 0;
        const int e2 = (m2 > 0) ? ilogb_r(m2) : 0;             // exact power-of-two scaling
        for (int i = lane; i < M; i += 32) ss += abs2(scalb_s(W[i + k * ldw], -e2));
        ss = warp_sum(ss);
        if (lane == 0) sig[k] = (m2 > 0) ? scalb_r(sqrt_r(ss), e2) : R(0);
    }
    __syncthreads();
    for (int k = tid; k < N; k += NT) {
        const R sk = sig[k];
        int rk = 0;
        for (int j = 0; j < N; ++j) {
            const R sj = sig[j];
            rk += (sj > sk) || (sj == sk && j < k);
        }
        rank[k] = rk;
        Sout[rk] = scalb_r(sk, ex);
    }
    __syncthreads();

    // W-derived output: U (or V when working on A^H), column rank[k] = w_k / sigma_k
    T* Y = a.trans ? Vout : Uout;
    const int ldy = a.trans ? ldv : ldu;
    if (wantWout) {
        for (int e = tid; e < M * N; e += NT) {
            const int i = e % M, k = e / M;
            const R sk = sig[k];
            if (sk > 0) Y[i + (long long)rank[k] * ldy] = divr(W[i + k * ldw], sk);
        }
        __syncthreads();
        // Zero columns (sigma_k = 0) hold the last ranks.  Complete Y's
        // orthonormal basis: take the standard basis vector e_r with the
        // largest residual 1 - sum_q |Y[r,q]|^2, project it off Y[:, 0:p]
        // twice and normalise.  Rare; written for clarity, not speed.
        int nz = 0;
        for (int k = 0; k < N; ++k) nz += (sig[k] == R(0));
        T* x = W;                                              // W is free now
        for (int p = N - nz; p < N; ++p) {
            if (tid == 0) {
                R best = -1;
                int r0 = 0;
                for (int r = 0; r < M; ++r) {
                    R s2 = 0;
                    for (int q = 0; q < p; ++q) s2 += abs2(Y[r + (long long)q * ldy]);
                    if (R(1) - s2 > best) { best = R(1) - s2; r0 = r; }
                }
                iscr[1] = r0;
            }
            __syncthreads();
            const int r0 = iscr[1];
            for (int r = tid; r < M; r += NT) x[r] = make_s<T>(r == r0 ? 1 : 0);
            __syncthreads();
            for (int pass = 0; pass < 2; ++pass)
                for (int q = 0; q < p; ++q) {
                    if (warp == 0) {
                        T d = make_s<T>(0);
                        for (int r = lane; r < M; r += 32) d = cfma(Y[r + (long long)q * ldy], x[r], d);
                        d = warp_sum_s(d);
                        if (lane == 0) bcast[0] = d;
                    }
                    __syncthreads();
                    const T dd = bcast[0];
                    for (int r = tid; r < M; r += NT) x[r] = sub(x[r], mul(Y[r + (long long)q * ldy], dd));
                    __syncthreads();
                }
            if (warp == 0) {
                R ss = 0;
                for (int r = lane; r < M; r += 32) ss += abs2(x[r]);
                ss = warp_sum(ss);
                if (lane == 0) red[0] = sqrt_r(ss);
            }
            __syncthreads();
            const R nx = red[0];
            for (int r = tid; r < M; r += NT) Y[r + (long long)p * ldy] = divr(x[r], nx);
            __syncthreads();
        }
    }
    __syncthreads();

    // V-derived output (V, or U when working on A^H): one Newton-Schulz step
    // Z = V - V E / 2 with E = V^H V - I, columns permuted by rank.
    if (needVs) {
        T* Z = a.trans ? Uout : Vout;
        const int ldz = a.trans ? ldu : ldv;
        const bool correct = !(a.flags & kFlagNoVCorrection);
        T* E = W;   // W is free now
        const int lde = a.lde;
        if (correct) {
            for (int e = tid; e < N * (N + 1) / 2; e += NT) {
                int ca, cb;
                tri_index(e, ca, cb);
                T acc = make_s<T>(0);
                for (int i = 0; i < N; ++i) acc = cfma(Vs[i + ca * ldvs], Vs[i + cb * ldvs], acc);
                if (ca == cb) acc = make_s<T>(re(acc) - R(1));
                E[ca + cb * lde] = acc;
                E[cb + ca * lde] = conj_s(acc);
            }
            __syncthreads();
        }
        for (int e = tid; e < N * N; e += NT) {
            const int i = e % N, k = e / N;
            T z = Vs[i + k * ldvs];
            if (correct) {
                T acc = make_s<T>(0);
                for (int j = 0; j < N; ++j) acc = fma_s(Vs[i + j * ldvs], E[j + k * lde], acc);
                z = sub(z, scale(acc, R(0.5)));
            }
            Z[i + (long long)rank[k] * ldz] = z;
        }
    }
    if (tid == 0) {
        a.info[mid] = converged ? 0 : sw;
        if (a.sweeps) a.sweeps[mid] = sw;
    }
}

}  // namespace bsvd
