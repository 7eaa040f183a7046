// fused_f32.cuh -- register-tiled Gram and block-rotation steps of the fused
// kernel for real single precision.
//
// In FP32 the fused kernel is bound by instruction issue, not by the FMA pipe,
// so these versions trade flops for fewer instructions: 4x4 register tiles and
// float4 shared-memory loads along columns (column-major rows are contiguous).
// The Gram block is formed in full (twice the flops of its upper triangle) so
// that every thread has the same work; only upper tiles are written.
#pragma once

#include "jacobi_common.cuh"

namespace bsvd {

// G = P^H P for the panel P = [W_i W_j] (columns cbi.., cbj.. of W, M rows,
// leading dimension ldw, a multiple of 4 with 16-byte aligned columns).
// GT threads: tile (ti, tj) of 4x4 entries, the rows split over KS lanes in
// interleaved chunks of 4 and summed with shuffles.
template <int NB, int GT>
__device__ __forceinline__ void gram_f32_tiled(const float* W, int ldw, int M, int cbi, int cbj, float* G,
                                               int gt) {
    constexpr int TWO = 2 * NB, LDG = TWO + 1, TT = TWO / 4, NTILE = TT * TT, KS = GT / NTILE;
    static_assert(GT % NTILE == 0 && KS >= 1 && KS <= 32 && (KS & (KS - 1)) == 0, "tile split");
    const int tile = gt / KS, ks = gt % KS, ti = tile / TT, tj = tile % TT;
    const float* a[4];
    const float* b[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int ca = 4 * ti + q, cb = 4 * tj + q;
        a[q] = W + (long long)(ca < NB ? cbi + ca : cbj + ca - NB) * ldw;
        b[q] = W + (long long)(cb < NB ? cbi + cb : cbj + cb - NB) * ldw;
    }
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    const int chunks = M >> 2;
    for (int ch = ks; ch < chunks; ch += KS) {
        float4 av[4], bv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            av[q] = *reinterpret_cast<const float4*>(a[q] + 4 * ch);
            bv[q] = *reinterpret_cast<const float4*>(b[q] + 4 * ch);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float s = acc[i][j];
                s = fmaf(av[i].x, bv[j].x, s);
                s = fmaf(av[i].y, bv[j].y, s);
                s = fmaf(av[i].z, bv[j].z, s);
                s = fmaf(av[i].w, bv[j].w, s);
                acc[i][j] = s;
            }
    }
    if (ks == 0)
        for (int k = chunks * 4; k < M; ++k)
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i][k], b[j][k], acc[i][j]);
#pragma unroll
    for (int o = 1; o < KS; o <<= 1)
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] += __shfl_xor_sync(0xffffffffu, acc[i][j], o);
    if (ks == 0 && ti <= tj) {
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int r = 4 * ti + i, c = 4 * tj + j;
                if (ti == tj && r > c) continue;           // diagonal tile: upper part, mirrored
                G[r + c * LDG] = acc[i][j];
                G[c + r * LDG] = acc[i][j];
            }
    }
}

// [X_i X_j] <- [X_i X_j] J for the rows of W (rowsW, a multiple of 4) and of V
// (rowsV, a multiple of 4, or 0), J given transposed: Jt[c + k*2NB] = J(k, c).
// 4x4 output tiles (4 rows x 4 columns), all of a pass in registers, one
// barrier, then written back: a pass covers whole rows, so every read of a
// row precedes every write of it.
template <int NB, int GT, int TPP>
__device__ __forceinline__ void update_f32_tiled(float* W, int ldw, int rowsW, float* V, int ldv, int rowsV,
                                                 int cbi, int cbj, const float* Jt, int gt, int bar) {
    constexpr int TWO = 2 * NB, TC = TWO / 4;
    constexpr int RPP = GT * TPP / TC;                       // row groups per pass
    static_assert((GT * TPP) % TC == 0, "tiles per pass");
    const int RW = rowsW >> 2, RT = RW + (rowsV >> 2);
    for (int p0 = 0; p0 < RT; p0 += RPP) {
        const int npass = min(RPP, RT - p0) * TC;
        float acc[TPP][4][4];
#pragma unroll
        for (int u = 0; u < TPP; ++u) {
            const int t = u * GT + gt;
            if (t >= npass) continue;
            const int rg = p0 + t / TC, cg = t % TC;
            float* X;
            int ld, r;
            if (rg < RW) { X = W; ld = ldw; r = 4 * rg; }
            else         { X = V; ld = ldv; r = 4 * (rg - RW); }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[u][i][j] = 0.f;
#pragma unroll
            for (int k = 0; k < TWO; ++k) {
                const int ck = k < NB ? cbi + k : cbj + k - NB;
                const float4 x = *reinterpret_cast<const float4*>(X + r + (long long)ck * ld);
                const float4 jv = *reinterpret_cast<const float4*>(Jt + 4 * cg + k * TWO);
                const float xs[4] = {x.x, x.y, x.z, x.w};
                const float js[4] = {jv.x, jv.y, jv.z, jv.w};
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[u][i][j] = fmaf(xs[i], js[j], acc[u][i][j]);
            }
        }
        named_sync(bar, GT);
#pragma unroll
        for (int u = 0; u < TPP; ++u) {
            const int t = u * GT + gt;
            if (t >= npass) continue;
            const int rg = p0 + t / TC, cg = t % TC;
            float* X;
            int ld, r;
            if (rg < RW) { X = W; ld = ldw; r = 4 * rg; }
            else         { X = V; ld = ldv; r = 4 * (rg - RW); }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = 4 * cg + j;
                const int cc = c < NB ? cbi + c : cbj + c - NB;
                *reinterpret_cast<float4*>(X + r + (long long)cc * ld) =
                    make_float4(acc[u][0][j], acc[u][1][j], acc[u][2][j], acc[u][3][j]);
            }
        }
        named_sync(bar, GT);
    }
}

}  // namespace bsvd
