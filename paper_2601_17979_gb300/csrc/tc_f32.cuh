// tc_f32.cuh -- the Gram block and the block rotation update of real FP32
// on the tensor cores, in split TF32 ("3xTF32").
//
// A tensor-core TF32 product rounds each operand to a 10-bit significand,
// far coarser than the one-sided Jacobi test |g_pq| >= tol sqrt(g_pp g_qq)
// (tol = 30 u_32) can tolerate.  Every operand is therefore split into two
// TF32 parts, x = x_hi + x_lo with x_hi = rna_tf32(x) and x_lo =
// rna_tf32(x - x_hi), and a product is formed as x_lo y_hi + x_hi y_lo +
// x_hi y_hi, the small terms first, into one FP32 accumulator; the dropped
// x_lo y_lo term and the rounding of x_lo are below 2^-21 relative to
// |x y|, the accuracy of an FP32 product.  The products
// are mma.sync.m16n8k8 tiles (PTX ISA, warp-level MMA, .tf32):
//   A fragment (16 x 8, row major)  a0 (g, t)  a1 (g+8, t)  a2 (g, t+4)  a3 (g+8, t+4)
//   B fragment (8 x 8, column major) b0 (t, g)  b1 (t+4, g)
//   C fragment (16 x 8)             c0 (g, 2t) c1 (g, 2t+1) c2 (g+8, 2t) c3 (g+8, 2t+1)
// with g = lane / 4 and t = lane % 4.  Each warp's summation order is fixed
// by the tile loop, so results are reproducible run to run and identical in
// every kernel that calls these functions.
#pragma once

#include <cstdint>

#include "jacobi_common.cuh"

namespace bsvd {

// Global -> shared copies of 4 or 8 bytes that do not wait for the data, so
// that the next staged panel chunk loads while the tensor cores work on the
// current one; a source size of 0 writes zeros.
template <int BYTES>
__device__ __forceinline__ void cp_async(void* dst, const void* src, int src_bytes) {
    static_assert(BYTES == 4 || BYTES == 8, "4- or 8-byte copies");
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;\n" ::"r"(d), "l"(src), "n"(BYTES), "r"(src_bytes)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

__device__ __forceinline__ uint32_t tf32_rna(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return r;
}

// x = hi + lo, both TF32 bit patterns
__device__ __forceinline__ void tf32_split(float x, uint32_t& hi, uint32_t& lo) {
    hi = tf32_rna(x);
    lo = tf32_rna(x - __uint_as_float(hi));
}

// d += a b for one m16n8k8 TF32 tile
__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One split-TF32 tile product: d += a_lo b_hi + a_hi b_lo + a_hi b_hi.
__device__ __forceinline__ void mma_3xtf32(float (&d)[4], const uint32_t (&ah)[4], const uint32_t (&al)[4],
                                           uint32_t bh0, uint32_t bh1, uint32_t bl0, uint32_t bl1) {
    mma_tf32(d, al, bh0, bh1);
    mma_tf32(d, ah, bl0, bl1);
    mma_tf32(d, ah, bh0, bh1);
}

// Four values of a 16-column block of the panel P = [W_i W_j] at rows
// k0 + t and k0 + t + 4 (zero at rows >= M): v0 = P(k0+t, c0+g),
// v1 = P(k0+t, c0+g+8), v2 = P(k0+t+4, c0+g), v3 = P(k0+t+4, c0+g+8) --
// as the A fragment of P^T (rows of A = panel columns), and as two B
// fragments of P ({v0, v2} for columns c0..c0+7, {v1, v3} for c0+8..).
// W is column-major with leading dimension ldw; `col` maps a panel column
// to a column of W.
template <int NB>
__device__ __forceinline__ void panel_block(const float* W, int ldw, int M, int cbi, int cbj, int c0, int k0,
                                            int g, int t, uint32_t (&hi)[4], uint32_t (&lo)[4]) {
    const int ca = c0 + g, cb = c0 + g + 8;
    const float* xa = W + (long long)(ca < NB ? cbi + ca : cbj + ca - NB) * ldw;
    const float* xb = W + (long long)(cb < NB ? cbi + cb : cbj + cb - NB) * ldw;
    const int r0 = k0 + t, r1 = k0 + t + 4;
    const float v[4] = {r0 < M ? xa[r0] : 0.f, r0 < M ? xb[r0] : 0.f, r1 < M ? xa[r1] : 0.f,
                        r1 < M ? xb[r1] : 0.f};
#pragma unroll
    for (int i = 0; i < 4; ++i) tf32_split(v[i], hi[i], lo[i]);
}

// The 16 x 16 block (bm, bn) of P^T P accumulated over the k-steps
// ks0, ks0 + kstride, ... below `steps` of rows [0, M) of P (8 rows a step):
// the building block of a Gram block whose rows are split over warps.
template <int NB>
__device__ __forceinline__ void gram_block_acc(const float* W, int ldw, int M, int cbi, int cbj, int bm, int bn,
                                               int ks0, int kstride, int lane, float (&acc)[2][4]) {
    const int g = lane >> 2, t = lane & 3;
    for (int ks = ks0; 8 * ks < M; ks += kstride) {
        uint32_t ah[4], al[4], bh[4], bl[4];
        panel_block<NB>(W, ldw, M, cbi, cbj, 16 * bm, 8 * ks, g, t, ah, al);
        if (bn == bm) {
#pragma unroll
            for (int i = 0; i < 4; ++i) { bh[i] = ah[i]; bl[i] = al[i]; }
        } else {
            panel_block<NB>(W, ldw, M, cbi, cbj, 16 * bn, 8 * ks, g, t, bh, bl);
        }
        mma_3xtf32(acc[0], ah, al, bh[0], bh[2], bl[0], bl[2]);
        mma_3xtf32(acc[1], ah, al, bh[1], bh[3], bl[1], bl[3]);
    }
}

// S2 on the tensor cores: G = P^T P (2NB x 2NB, leading dimension 2NB+1)
// for the panel P = [W_i W_j] (M rows).  NB = 16: four warps, warp w forms
// the 16 x 16 block (w / 2, w % 2) of G over all M rows (the lower off-
// diagonal block is formed and dropped: every warp has the same work);
// NB = 8: one warp forms the whole 16 x 16 block.  Upper entries are
// written and mirrored, so G is exactly symmetric.  GT threads (a multiple
// of 32) call it; warps beyond the block count idle.
template <int NB, int GT>
__device__ __forceinline__ void gram_f32_mma(const float* W, int ldw, int M, int cbi, int cbj, float* G, int gt) {
    constexpr int TWO = 2 * NB, LDG = TWO + 1, NBLK = TWO / 16;
    static_assert(NB == 8 || NB == 16, "tensor-core Gram: nb = 8 or 16");
    const int warp = gt >> 5, lane = gt & 31, g = lane >> 2, t = lane & 3;
    if (warp >= NBLK * NBLK) return;
    const int bm = warp / NBLK, bn = warp % NBLK;
    if (bm > bn) return;          // a block below the diagonal: the mirror of one above it
    float acc[2][4];
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[j][i] = 0.f;
    gram_block_acc<NB>(W, ldw, M, cbi, cbj, bm, bn, 0, 1, lane, acc);
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = 16 * bm + g + 8 * (i >> 1), c = 16 * bn + 8 * j + 2 * t + (i & 1);
            if (r > c) continue;                               // lower entries: the mirror of an upper one
            const float x = acc[j][i];
            G[r + c * LDG] = x;
            G[c + r * LDG] = x;
        }
}

// J (2NB x 2NB, leading dimension 2NB+1) as split-TF32 B fragments of the
// update, in fragment order: Jf[(ks * NT + nt) * 32 + lane] = {hi(b0),
// hi(b1), lo(b0), lo(b1)} of k-step ks and column tile nt, so a lane reads
// its fragment with one 16-byte load.  GT threads; the caller synchronises
// before the fragments are read.
template <int NB, int GT, int LDJ = 2 * NB + 1>
__device__ __forceinline__ void j_fragments(const float* J, uint4* Jf, int gt) {
    constexpr int TWO = 2 * NB, KS = TWO / 8, NT = TWO / 8;
    for (int e = gt; e < KS * NT * 32; e += GT) {
        const int lane = e & 31, f = e >> 5, ks = f / NT, nt = f % NT, g = lane >> 2, t = lane & 3;
        uint32_t h0, l0, h1, l1;
        tf32_split(J[(8 * ks + t) + (8 * nt + g) * LDJ], h0, l0);
        tf32_split(J[(8 * ks + t + 4) + (8 * nt + g) * LDJ], h1, l1);
        Jf[e] = make_uint4(h0, h1, l0, l1);
    }
}

// Bytes of the fragment array of j_fragments.
template <int NB>
__host__ __device__ constexpr int j_fragment_bytes() { return 8 * (2 * NB) * (2 * NB); }

// Rows [r0, r0 + 16) of a column-major array X (rows valid below `rows`)
// times J on the tensor cores, written back in place: [X_i X_j] <- [X_i X_j] J
// for those rows.  One warp; it reads all 16 x 2NB inputs before it writes
// any output, and no other warp touches these rows.
template <int NB>
__device__ __forceinline__ void update_rows_mma(float* X, int ld, int rows, int r0, int cbi, int cbj,
                                                const uint4* Jf, int lane) {
    constexpr int TWO = 2 * NB, KS = TWO / 8, NT = TWO / 8;
    const int g = lane >> 2, t = lane & 3;
    auto col = [&](int c) { return (long long)(c < NB ? cbi + c : cbj + c - NB) * ld; };
    const int ra = r0 + g, rb = r0 + g + 8;
    float acc[NT][4];
#pragma unroll
    for (int j = 0; j < NT; ++j)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[j][i] = 0.f;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
        const long long c0 = col(8 * ks + t), c1 = col(8 * ks + t + 4);
        const float v[4] = {ra < rows ? X[ra + c0] : 0.f, rb < rows ? X[rb + c0] : 0.f,
                            ra < rows ? X[ra + c1] : 0.f, rb < rows ? X[rb + c1] : 0.f};
        uint32_t ah[4], al[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) tf32_split(v[i], ah[i], al[i]);
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
            const uint4 b = Jf[(ks * NT + nt) * 32 + lane];
            mma_3xtf32(acc[nt], ah, al, b.x, b.y, b.z, b.w);
        }
    }
    __syncwarp();
#pragma unroll
    for (int nt = 0; nt < NT; ++nt) {
        const long long c0 = col(8 * nt + 2 * t), c1 = col(8 * nt + 2 * t + 1);
        if (ra < rows) {
            X[ra + c0] = acc[nt][0];
            X[ra + c1] = acc[nt][1];
        }
        if (rb < rows) {
            X[rb + c0] = acc[nt][2];
            X[rb + c1] = acc[nt][3];
        }
    }
}

// S4/S5 on the tensor cores: [W_i W_j] <- [W_i W_j] J for rowsW rows of W
// and [V_i V_j] <- [V_i V_j] J for rowsV rows of V (0: V not kept), in
// 16-row tiles dealt round-robin to the GT / 32 warps of the group.
template <int NB, int GT>
__device__ __forceinline__ void update_f32_mma(float* W, int ldw, int rowsW, float* V, int ldv, int rowsV,
                                               int cbi, int cbj, const uint4* Jf, int gt) {
    constexpr int NWG = GT / 32;
    const int warp = gt >> 5, lane = gt & 31;
    const int tw = (rowsW + 15) / 16, tv = (rowsV + 15) / 16;
    for (int tile = warp; tile < tw + tv; tile += NWG) {
        if (tile < tw) update_rows_mma<NB>(W, ldw, rowsW, 16 * tile, cbi, cbj, Jf, lane);
        else           update_rows_mma<NB>(V, ldv, rowsV, 16 * (tile - tw), cbi, cbj, Jf, lane);
    }
}

}  // namespace bsvd
