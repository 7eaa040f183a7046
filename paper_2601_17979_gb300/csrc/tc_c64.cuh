// tc_c64.cuh -- the complex64 Gram block and block rotation update on the
// tensor cores, as real split-TF32 products (tc_f32.cuh) of the real and
// imaginary parts.
//
// With P = Pr + i Pi and J = Jr + i Ji:
//   G = P^H P:  Re G = Pr^T Pr + Pi^T Pi,   Im G = Pr^T Pi - Pi^T Pr
//   P J:        Re = Pr Jr - Pi Ji,         Im = Pr Ji + Pi Jr
// Each real product is a split-TF32 mma.sync tile product (three TF32 MMAs,
// FP32 accumulate); the two terms of each real or imaginary part accumulate
// into one FP32 accumulator, in a fixed order, so results are reproducible
// and identical wherever these functions are used.  A negated operand is
// negated exactly (sign bit) in its split parts.
#pragma once

#include <cstdint>

#include "tc_f32.cuh"

namespace bsvd {

__device__ __forceinline__ uint32_t neg_tf32(uint32_t x) { return x ^ 0x80000000u; }

// The real and imaginary parts of four values of a 16-column block of the
// complex panel P (column-major, leading dimension ld, rows >= M read as
// zero), split in TF32 parts, in the layout of panel_block (tc_f32.cuh).
template <int NB>
__device__ __forceinline__ void panel_block_c(const float2* W, int ld, int M, int cbi, int cbj, int c0, int k0,
                                              int g, int t, uint32_t (&rh)[4], uint32_t (&rl)[4], uint32_t (&ih)[4],
                                              uint32_t (&il)[4]) {
    const int ca = c0 + g, cb = c0 + g + 8;
    const float2* xa = W + (long long)(ca < NB ? cbi + ca : cbj + ca - NB) * ld;
    const float2* xb = W + (long long)(cb < NB ? cbi + cb : cbj + cb - NB) * ld;
    const int r0 = k0 + t, r1 = k0 + t + 4;
    const float2 z = make_float2(0.f, 0.f);
    const float2 v[4] = {r0 < M ? xa[r0] : z, r0 < M ? xb[r0] : z, r1 < M ? xa[r1] : z, r1 < M ? xb[r1] : z};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        tf32_split(v[i].x, rh[i], rl[i]);
        tf32_split(v[i].y, ih[i], il[i]);
    }
}

// The 16 x 16 block (bm, bn) of G = P^H P accumulated over the k-steps
// ks0, ks0 + kstride, ... of rows [0, M): re and im parts, two 16 x 8 tiles
// each.
template <int NB>
__device__ __forceinline__ void gram_c64_block_acc(const float2* W, int ld, int M, int cbi, int cbj, int bm, int bn,
                                                   int ks0, int kstride, int lane, float (&re)[2][4],
                                                   float (&im)[2][4]) {
    const int g = lane >> 2, t = lane & 3;
    for (int ks = ks0; 8 * ks < M; ks += kstride) {
        uint32_t arh[4], arl[4], aih[4], ail[4], brh[4], brl[4], bih[4], bil[4];
        panel_block_c<NB>(W, ld, M, cbi, cbj, 16 * bm, 8 * ks, g, t, arh, arl, aih, ail);
        if (bn == bm) {
#pragma unroll
            for (int i = 0; i < 4; ++i) { brh[i] = arh[i]; brl[i] = arl[i]; bih[i] = aih[i]; bil[i] = ail[i]; }
        } else {
            panel_block_c<NB>(W, ld, M, cbi, cbj, 16 * bn, 8 * ks, g, t, brh, brl, bih, bil);
        }
#pragma unroll
        for (int j = 0; j < 2; ++j) {
            const int x = j, y = j + 2;      // B fragment of column tile j: values {x, y} of the block
            // Re += Pr^T Pr + Pi^T Pi
            mma_3xtf32(re[j], arh, arl, brh[x], brh[y], brl[x], brl[y]);
            mma_3xtf32(re[j], aih, ail, bih[x], bih[y], bil[x], bil[y]);
            // Im += Pr^T Pi - Pi^T Pr
            mma_3xtf32(im[j], arh, arl, bih[x], bih[y], bil[x], bil[y]);
            mma_3xtf32(im[j], aih, ail, neg_tf32(brh[x]), neg_tf32(brh[y]), neg_tf32(brl[x]), neg_tf32(brl[y]));
        }
    }
}

// Jr and Ji (2NB x 2NB, column stride LDJ) as split-TF32 B fragments in
// fragment order (j_fragments, tc_f32.cuh): Jf[0 .. F) for Jr, Jf[F .. 2F)
// for Ji, F = (2NB / 8)^2 * 32.
template <int NB, int GT, int LDJ>
__device__ __forceinline__ void jc_fragments(const float2* J, uint4* Jf, int gt) {
    constexpr int TWO = 2 * NB, KS = TWO / 8, NT = TWO / 8, F = KS * NT * 32;
    for (int e = gt; e < F; e += GT) {
        const int lane = e & 31, f = e >> 5, ks = f / NT, nt = f % NT, g = lane >> 2, t = lane & 3;
        const float2 j0 = J[(8 * ks + t) + (8 * nt + g) * LDJ], j1 = J[(8 * ks + t + 4) + (8 * nt + g) * LDJ];
        uint32_t h0, l0, h1, l1;
        tf32_split(j0.x, h0, l0);
        tf32_split(j1.x, h1, l1);
        Jf[e] = make_uint4(h0, h1, l0, l1);
        tf32_split(j0.y, h0, l0);
        tf32_split(j1.y, h1, l1);
        Jf[F + e] = make_uint4(h0, h1, l0, l1);
    }
}

template <int NB>
__host__ __device__ constexpr int jc_fragment_bytes() { return 2 * 8 * (2 * NB) * (2 * NB); }

// Rows [r0, r0 + 16) of the complex column-major X (rows valid below `rows`)
// times J on the tensor cores, in place.  One warp; all inputs are read
// before any output is written, and no other warp touches these rows.
template <int NB>
__device__ __forceinline__ void update_rows_c64_mma(float2* X, int ld, int rows, int r0, int cbi, int cbj,
                                                    const uint4* Jf, int lane) {
    constexpr int TWO = 2 * NB, KS = TWO / 8, NT = TWO / 8, F = KS * NT * 32;
    const int g = lane >> 2, t = lane & 3;
    auto col = [&](int c) { return (long long)(c < NB ? cbi + c : cbj + c - NB) * ld; };
    const int ra = r0 + g, rb = r0 + g + 8;
    float re[NT][4], im[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) re[j][i] = im[j][i] = 0.f;
    const float2 z = make_float2(0.f, 0.f);
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
        const long long c0 = col(8 * ks + t), c1 = col(8 * ks + t + 4);
        const float2 v[4] = {ra < rows ? X[ra + c0] : z, rb < rows ? X[rb + c0] : z,
                             ra < rows ? X[ra + c1] : z, rb < rows ? X[rb + c1] : z};
        uint32_t rh[4], rl[4], ih[4], il[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            tf32_split(v[i].x, rh[i], rl[i]);
            tf32_split(v[i].y, ih[i], il[i]);
        }
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const uint4 jr = Jf[(ks * NT + nt) * 32 + lane], ji = Jf[F + (ks * NT + nt) * 32 + lane];
            // Re += Xr Jr - Xi Ji;  Im += Xr Ji + Xi Jr
            mma_3xtf32(re[nt], rh, rl, jr.x, jr.y, jr.z, jr.w);
            mma_3xtf32(re[nt], ih, il, neg_tf32(ji.x), neg_tf32(ji.y), neg_tf32(ji.z), neg_tf32(ji.w));
            mma_3xtf32(im[nt], rh, rl, ji.x, ji.y, ji.z, ji.w);
            mma_3xtf32(im[nt], ih, il, jr.x, jr.y, jr.z, jr.w);
        }
    }
    __syncwarp();
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const long long c0 = col(8 * nt + 2 * t), c1 = col(8 * nt + 2 * t + 1);
        if (ra < rows) {
            X[ra + c0] = make_float2(re[nt][0], im[nt][0]);
            X[ra + c1] = make_float2(re[nt][1], im[nt][1]);
        }
        if (rb < rows) {
            X[rb + c0] = make_float2(re[nt][2], im[nt][2]);
            X[rb + c1] = make_float2(re[nt][3], im[nt][3]);
        }
    }
}

}  // namespace bsvd
