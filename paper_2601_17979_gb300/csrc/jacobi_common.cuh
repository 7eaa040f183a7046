// jacobi_common.cuh -- device building blocks shared by the fused and the
// multi-kernel Jacobi SVD paths: the round-robin ordering, barriers and warp
// reductions, and the inner Jacobi eigensolver on a 2nb x 2nb Gram block.
#pragma once

#include "scalar.cuh"

namespace bsvd {

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

// Named barrier `id` (1..15) over `nthreads` threads (a multiple of 32).
__device__ __forceinline__ void group_sync(int id_minus_1, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id_minus_1 + 1), "r"(nthreads) : "memory");
}
__device__ __forceinline__ void named_sync(int id, int nthreads) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(nthreads) : "memory");
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
__device__ __forceinline__ float shfl_xor_s(float v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ double shfl_xor_s(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ float2 shfl_xor_s(float2 v, int o) {
    return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ double2 shfl_xor_s(double2 v, int o) {
    return make_double2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}
__device__ __forceinline__ float warp_sum_s(float v) { return warp_sum(v); }
__device__ __forceinline__ double warp_sum_s(double v) { return warp_sum(v); }
__device__ __forceinline__ float2 warp_sum_s(float2 v) { return make_float2(warp_sum(v.x), warp_sum(v.y)); }
__device__ __forceinline__ double2 warp_sum_s(double2 v) { return make_double2(warp_sum(v.x), warp_sum(v.y)); }

// Rotation table of one inner step (nb disjoint rotations) plus a counter of
// fired rotations, laid out in shared memory right after J.
template <class T, int NB>
struct InnerTables {
    using R = Real<T>;
    R* c; R* s; R* t; T* ph; int* p; int* q; int* fired; int* count;
    __device__ explicit InnerTables(void* base) {
        c = static_cast<R*>(base);
        s = c + NB;
        t = s + NB;
        ph = reinterpret_cast<T*>(t + NB);
        p = reinterpret_cast<int*>(ph + NB);
        q = p + NB;
        fired = q + NB;
        count = fired + NB;
    }
    __host__ __device__ static constexpr int bytes() {
        return NB * (3 * (int)sizeof(R) + (int)sizeof(T)) + NB * 3 * 4 + 16;
    }
};

// Up to `sweeps` sweeps of Alg. 1 on the Hermitian G (2NB x 2NB, leading
// dimension 2NB+1, in shared memory), accumulating the rotations into J
// (set to I here).  One sweep is 2NB-1 parallel steps of the round-robin
// ordering on the 2NB indices; in each, NB threads test their pair
// (|g_pq| >= tol sqrt(g_pp) sqrt(g_qq), Alg. 1) and compute (c, s, e^{i phi})
// by Eq. (sin-cos) with sign(0) = +1; then G <- R^H G R is applied as 2x2
// block transforms (rows of one slot, columns of another; the diagonal
// block by the closed form g_pp += t|g_pq|, g_qq -= t|g_pq|, g_pq = 0) and
// J <- J R.  Sweeps stop early once one rotates nothing.
// Executed by GT threads (index gt) that share named barrier `bar`.  The
// caller must have finished writing G and synchronised.  Returns the number
// of rotations fired (0: G was diagonal to tol); uniform over the group.
template <class T, int NB, int GT>
__device__ int inner_jacobi(T* G, T* J, const InnerTables<T, NB>& tb, Real<T> tol, int sweeps,
                            int gt, int bar) {
    using R = Real<T>;
    constexpr int TWO = 2 * NB, LDG = TWO + 1;
    for (int e = gt; e < TWO * TWO; e += GT)
        J[(e % TWO) + (e / TWO) * LDG] = make_s<T>((e % TWO) == (e / TWO) ? 1 : 0);
    if (gt == 0) *tb.count = 0;
    named_sync(bar, GT);
    int seen = 0;
    for (int isw = 0; isw < sweeps; ++isw) {
        for (int st = 0; st < TWO - 1; ++st) {
            if (gt < NB) {
                int p, q;
                rr_pair(TWO, st, gt, p, q);
                const R gpp = re(G[p + p * LDG]), gqq = re(G[q + q * LDG]);
                const T gpq = G[p + q * LDG];
                const R apq = abs_s(gpq);
                const bool fire = gpp > 0 && gqq > 0 && apq > 0 && apq >= tol * sqrt_r(gpp) * sqrt_r(gqq);
                R c = 1, sn = 0, t = 0;
                T ph = make_s<T>(1);
                if (fire) {
                    // Eq. (sin-cos) with tau = x / y, x = g_pp - g_qq, y = 2 |g_pq|:
                    // t = sign(tau) / (|tau| + sqrt(1 + tau^2)) = sign(x) y / (|x| + hypot(x, y))
                    const R x = gpp - gqq, y = 2 * apq;
                    t = (x >= 0 ? y : -y) / (fabs(x) + hypot_r(x, y));
                    c = rsqrt_r(R(1) + t * t);
                    sn = t * c;
                    ph = phase_s(gpq, apq);
                    atomicAdd(tb.count, 1);
                }
                tb.c[gt] = c; tb.s[gt] = sn; tb.t[gt] = t; tb.ph[gt] = ph;
                tb.p[gt] = p; tb.q[gt] = q; tb.fired[gt] = fire;
            }
            named_sync(bar, GT);
            // G <- R^H G R on 2x2 blocks (slot q1 <= slot q2), mirrored
            constexpr int NBLK = NB * (NB + 1) / 2;
            for (int e = gt; e < NBLK; e += GT) {
                int q1, q2;
                tri_index(e, q1, q2);
                const bool f1 = tb.fired[q1], f2 = tb.fired[q2];
                if (!f1 && !f2) continue;
                const int p1 = tb.p[q1], r1 = tb.q[q1], p2 = tb.p[q2], r2 = tb.q[q2];
                if (q1 == q2) {
                    const R tt = tb.t[q1];
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
                    const R c2 = tb.c[q2];
                    const T es = scale(tb.ph[q2], tb.s[q2]), ces = conj_s(es);
                    const T n00 = add(scale(b00, c2), mul(b01, ces));
                    const T n01 = sub(scale(b01, c2), mul(b00, es));
                    const T n10 = add(scale(b10, c2), mul(b11, ces));
                    const T n11 = sub(scale(b11, c2), mul(b10, es));
                    b00 = n00; b01 = n01; b10 = n10; b11 = n11;
                }
                if (f1) {   // rows (p1, r1) times R1^H
                    const R c1 = tb.c[q1];
                    const T es = scale(tb.ph[q1], tb.s[q1]), ces = conj_s(es);
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
                if (!tb.fired[qs]) continue;
                const int p = tb.p[qs], q = tb.q[qs];
                const R c = tb.c[qs];
                const T es = scale(tb.ph[qs], tb.s[qs]), ces = conj_s(es);
                const T x = J[i + p * LDG], y = J[i + q * LDG];
                J[i + p * LDG] = add(scale(x, c), mul(y, ces));
                J[i + q * LDG] = sub(scale(y, c), mul(x, es));
            }
            named_sync(bar, GT);
        }
        const int now = *tb.count;
        named_sync(bar, GT);   // all have read the counter before the next sweep bumps it
        const bool quiet = (now == seen);
        seen = now;
        if (quiet) break;      // this sweep rotated nothing: the inner solve has converged
    }
    return seen;
}

// Shared-memory scratch of finalize_outputs: sig[N], rank[N], red[>= warps],
// iscr[>= 2], bcast[>= 1].
template <class T>
struct FinalScratch {
    Real<T>* sig; int* rank; Real<T>* red; int* iscr; T* bcast;
};

// The end of Alg. 2 for one matrix, by a whole CTA of NT threads.
//   sigma_k = ||w_k||_2 (exact power-of-two scaled sum of squares), a stable
//   descending sort (rank of each column), Sout[rank] = sigma * 2^ex;
//   Y[:, rank_k] = w_k / sigma_k (U, or V for a transposed problem) when
//   wantY, with zero columns completed to an orthonormal basis;
//   Z[:, rank_k] = v_k - (V (V^H V - I))_k / 2 (one Newton-Schulz step
//   towards the nearest orthonormal V) when wantZ; `correct` = false copies V.
// W (M x N, ldw) and V (N x N, ldvs) may live in shared or global memory.
// x (M elements) and E (N x N, lde) are scratch and may alias W: W is not
// read after Y is complete.
template <class T, int NT>
__device__ void finalize_outputs(const T* W, int ldw, const T* V, int ldvs, int M, int N, int ex,
                                 T* x, T* E, int lde, bool correct, Real<T>* Sout, T* Y,
                                 long long ldy, bool wantY, T* Z, long long ldz, bool wantZ,
                                 const FinalScratch<T>& fs) {
    using R = Real<T>;
    constexpr int NW = NT / 32;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    R* sig = fs.sig;
    int* rank = fs.rank;
    for (int k = warp; k < N; k += NW) {
        R m2 = 0;
        for (int i = lane; i < M; i += 32) m2 = fmax(m2, maxabs(W[i + (long long)k * ldw]));
        m2 = warp_max(m2);
        R ss = 0;
        const int e2 = (m2 > 0) ? ilogb_r(m2) : 0;             // exact power-of-two scaling
        for (int i = lane; i < M; i += 32) ss += abs2(scalb_s(W[i + (long long)k * ldw], -e2));
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
    if (wantY) {
        for (int e = tid; e < M * N; e += NT) {
            const int i = e % M, k = e / M;
            const R sk = sig[k];
            if (sk > 0) Y[i + (long long)rank[k] * ldy] = divr(W[i + (long long)k * ldw], sk);
        }
        __syncthreads();
        // Zero columns (sigma_k = 0) hold the last ranks.  Complete Y's
        // orthonormal basis: the standard basis vector e_r with the largest
        // residual 1 - sum_q |Y[r,q]|^2, projected off Y[:, 0:p] twice and
        // normalised.  Rare; written for clarity, not speed.
        int nz = 0;
        for (int k = 0; k < N; ++k) nz += (sig[k] == R(0));
        for (int p = N - nz; p < N; ++p) {
            if (tid == 0) {
                R best = -1;
                int r0 = 0;
                for (int r = 0; r < M; ++r) {
                    R s2 = 0;
                    for (int q = 0; q < p; ++q) s2 += abs2(Y[r + (long long)q * ldy]);
                    if (R(1) - s2 > best) { best = R(1) - s2; r0 = r; }
                }
                fs.iscr[1] = r0;
            }
            __syncthreads();
            const int r0 = fs.iscr[1];
            for (int r = tid; r < M; r += NT) x[r] = make_s<T>(r == r0 ? 1 : 0);
            __syncthreads();
            for (int pass = 0; pass < 2; ++pass)
                for (int q = 0; q < p; ++q) {
                    if (warp == 0) {
                        T d = make_s<T>(0);
                        for (int r = lane; r < M; r += 32) d = cfma(Y[r + (long long)q * ldy], x[r], d);
                        d = warp_sum_s(d);
                        if (lane == 0) fs.bcast[0] = d;
                    }
                    __syncthreads();
                    const T dd = fs.bcast[0];
                    for (int r = tid; r < M; r += NT) x[r] = sub(x[r], mul(Y[r + (long long)q * ldy], dd));
                    __syncthreads();
                }
            if (warp == 0) {
                R ss = 0;
                for (int r = lane; r < M; r += 32) ss += abs2(x[r]);
                ss = warp_sum(ss);
                if (lane == 0) fs.red[0] = sqrt_r(ss);
            }
            __syncthreads();
            const R nx = fs.red[0];
            for (int r = tid; r < M; r += NT) Y[r + (long long)p * ldy] = divr(x[r], nx);
            __syncthreads();
        }
    }
    __syncthreads();
    if (wantZ) {
        if (correct) {
            for (int e = tid; e < N * (N + 1) / 2; e += NT) {
                int ca, cb;
                tri_index(e, ca, cb);
                T acc = make_s<T>(0);
                for (int i = 0; i < N; ++i)
                    acc = cfma(V[i + (long long)ca * ldvs], V[i + (long long)cb * ldvs], acc);
                if (ca == cb) acc = make_s<T>(re(acc) - R(1));
                E[ca + (long long)cb * lde] = acc;
                E[cb + (long long)ca * lde] = conj_s(acc);
            }
            __syncthreads();
        }
        for (int e = tid; e < N * N; e += NT) {
            const int i = e % N, k = e / N;
            T z = V[i + (long long)k * ldvs];
            if (correct) {
                T acc = make_s<T>(0);
                for (int j = 0; j < N; ++j) acc = fma_s(V[i + (long long)j * ldvs], E[j + (long long)k * lde], acc);
                z = sub(z, scale(acc, R(0.5)));
            }
            Z[i + (long long)rank[k] * ldz] = z;
        }
    }
}

}  // namespace bsvd
