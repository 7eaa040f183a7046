// gesvj_pairstep.cuh -- one kernel per round for single precision (real
// FP32 and complex64, nb = 8 or 16) on the multi-kernel path: a CTA takes
// one block pair of one matrix through S2-S5 (Gram block, inner Jacobi
// sweep, rotation of the pair's columns of W and V) with G, J and the
// rotation tables in shared memory.
//
// The three per-round kernels of gesvj_blocked.cuh (Gram, eigensolver,
// update) exchange G and J through global memory, read each pair's panel
// twice from DRAM once the batch's W and V exceed L2, and run as three
// launches whose CTAs are all in the same phase at once.  Here the phases of
// one pair follow each other inside a CTA: G and J never leave the SM, the
// update re-reads the panel the Gram has just brought into L2, and the CTAs
// resident on an SM overlap one pair's latency-bound inner sweep with
// another pair's tensor-core Gram or update.
//
// Each phase performs the operations of its separate kernel in the same
// order, so the results are the three kernels' bits: the Gram kernel's
// eight warps become eight virtual warps, two per warp here, each with its
// own accumulators over the same k-steps, and their partial blocks are
// summed in the same order; the inner solver's per-element arithmetic does
// not depend on the thread count; the update works on the same 16-row
// tiles.
#pragma once

#include <type_traits>

#include "gesvj_blocked.cuh"
#include "tc_c64.cuh"
#include "tc_f32.cuh"

namespace bsvd {

constexpr int kPairThreads = 128;
constexpr int kPairVirtualWarps = kBlkThreads / 32;    // the Gram kernel's warps

// Shared memory: two staged 64-row panel chunks and the virtual warps'
// partial blocks (S2), reused for J's split fragments (S4/S5); then G and J
// (leading dimension 2nb + 1) and the rotation tables.
template <class T, int NB>
struct PairLayout {
    static constexpr bool kCplx = std::is_same<T, float2>::value;
    static constexpr int TWO = 2 * NB, LDG = TWO + 1, KP = kGramChunk + 4;
    static constexpr int RW = kCplx ? 16 : 8;            // floats per lane in a partial block
    static constexpr int kChunk = (KP * TWO * (int)sizeof(T) + 15) & ~15;
    static constexpr int kStage = 2 * kChunk;
    static constexpr int kRed = kPairVirtualWarps * 32 * RW * (int)sizeof(float);
    static constexpr int kFrag = kCplx ? jc_fragment_bytes<NB>() : j_fragment_bytes<NB>();
    static constexpr int kRegionA = ((kStage + kRed > kFrag ? kStage + kRed : kFrag) + 15) & ~15;
    static constexpr int kBytes = kRegionA + 2 * TWO * LDG * (int)sizeof(T) + InnerTables<T, NB>::bytes();
};

// Resident CTAs per SM the register budget is written for: three for
// complex64 (166 registers), four for real FP32.
template <class T> constexpr int pair_min_blocks() { return std::is_same<T, float2>::value ? 3 : 4; }

template <class T, int NB>
__global__ void __launch_bounds__(kPairThreads, pair_min_blocks<T>()) blk_pairstep(const BlockedArgs a, int r) {
    static_assert(std::is_same<T, float>::value || std::is_same<T, float2>::value, "single precision");
    using L = PairLayout<T, NB>;
    constexpr bool kCplx = L::kCplx;
    constexpr int RW = L::RW;
    constexpr int TWO = 2 * NB, LDG = TWO + 1, NT = kPairThreads, NW = NT / 32, KC = kGramChunk, KP = L::KP;
    constexpr int VW = kPairVirtualWarps, H = VW / NW;           // virtual warps per warp
    constexpr int NBLK = TWO / 16, NB2 = NBLK * NBLK, WPB = VW / NB2;
    static_assert(VW % NB2 == 0 && NW % NB2 == 0, "a warp's virtual warps share one Gram block");
    extern __shared__ __align__(16) unsigned char smem[];
    T* P = reinterpret_cast<T*>(smem);
    float* red = reinterpret_cast<float*>(smem + L::kStage);
    uint4* Jf = reinterpret_cast<uint4*>(smem);
    T* G = reinterpret_cast<T*>(smem + L::kRegionA);
    T* J = G + TWO * LDG;
    const InnerTables<T, NB> tb(J + TWO * LDG);

    const int b = blockIdx.x, q = blockIdx.y, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    int* pf = a.pairflag + (long long)b * (a.L / 2) + q;
    if (blk_skip(a, b)) { if (tid == 0) *pf = 0; return; }
    const BlkShape sh = blk_shape(a, b);
    int bi, bj;
    if (!blk_pair(sh, r, q, bi, bj)) { if (tid == 0) *pf = 0; return; }
    T* Wm = static_cast<T*>(a.W) + sh.oW;
    T* Vm = static_cast<T*>(a.Vw) + sh.oV;
    const int M = sh.M;

    // ---- S2: G = P^H P on the tensor cores (as blk_gram_f32_tc / _c64_tc) ----
    {
        const int blk = warp % NB2, bm = blk / NBLK, bn = blk % NBLK;   // virtual warps warp + h NW
        float re[H][2][4], im[H][2][4];
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i) re[h][j][i] = im[h][j][i] = 0.f;
        // chunk k0 of the pair's columns into buffer `buf` (rows past M as zeros)
        auto stage = [&](int buf, int k0) {
            const int kc = min(KC, M - k0);
            T* Pb = P + buf * (L::kChunk / (int)sizeof(T));
            for (int e = tid; e < KC * TWO; e += NT) {
                const int kk = e % KC, c = e / KC;
                const int col = c < NB ? bi * NB + c : bj * NB + (c - NB);
                cp_async<(int)sizeof(T)>(Pb + kk + c * KP, Wm + k0 + (kk < kc ? kk : 0) + (long long)col * M,
                                         kk < kc ? (int)sizeof(T) : 0);
            }
            cp_async_commit();
        };
        stage(0, 0);
        for (int k0 = 0, it = 0; k0 < M; k0 += KC, ++it) {
            const int kc = min(KC, M - k0);
            if (k0 + KC < M) {                 // the next chunk loads during this one
                stage((it + 1) & 1, k0 + KC);
                cp_async_wait<1>();
            } else {
                cp_async_wait<0>();
            }
            __syncthreads();
            const T* Pc = P + (it & 1) * (L::kChunk / (int)sizeof(T));
#pragma unroll
            for (int h = 0; h < H; ++h) {
                if (bm > bn) break;            // blocks below the diagonal are mirrors
                if constexpr (kCplx)
                    gram_c64_block_acc<NB>(Pc, KP, kc, 0, NB, bm, bn, (warp + h * NW) / NB2, WPB, lane, re[h], im[h]);
                else
                    gram_block_acc<NB>(Pc, KP, kc, 0, NB, bm, bn, (warp + h * NW) / NB2, WPB, lane, re[h]);
            }
            __syncthreads();                   // before this buffer is refilled
        }
#pragma unroll
        for (int h = 0; h < H; ++h)
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    red[((warp + h * NW) * 32 + lane) * RW + 4 * j + i] = re[h][j][i];
                    if constexpr (kCplx) red[((warp + h * NW) * 32 + lane) * RW + 8 + 4 * j + i] = im[h][j][i];
                }
        __syncthreads();
        if (warp < NB2) {      // the virtual warps of sub-index 0, blocks 0 .. NB2-1
            const int g = lane >> 2, t = lane & 3;
#pragma unroll
            for (int j = 0; j < 2; ++j)
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    float xr = red[(blk * 32 + lane) * RW + 4 * j + i], xi = 0.f;
                    if constexpr (kCplx) xi = red[(blk * 32 + lane) * RW + 8 + 4 * j + i];
                    for (int s2 = 1; s2 < WPB; ++s2) {
                        xr += red[((blk + s2 * NB2) * 32 + lane) * RW + 4 * j + i];
                        if constexpr (kCplx) xi += red[((blk + s2 * NB2) * 32 + lane) * RW + 8 + 4 * j + i];
                    }
                    const int rr = 16 * bm + g + 8 * (i >> 1), cc = 16 * bn + 8 * j + 2 * t + (i & 1);
                    if (rr > cc) continue;                  // lower entries: the mirror of an upper one
                    if constexpr (kCplx) {
                        if (rr == cc) xi = 0.f;             // Hermitian: a real diagonal
                        G[rr + cc * LDG] = make_float2(xr, xi);
                        G[cc + rr * LDG] = make_float2(xr, -xi);
                    } else {
                        G[rr + cc * LDG] = xr;
                        G[cc + rr * LDG] = xr;
                    }
                }
        }
        __syncthreads();
    }

    // ---- S3: one sweep of the inner Jacobi solver (as blk_heevj) ------------
    const int seen = inner_jacobi<T, NB, NT>(G, J, tb, (float)a.tol, a.inner_sweeps, tid, 1, NoBackground(),
                                                  nullptr, (a.flags & 256) != 0);
    if (tid == 0) {
        *pf = seen > 0;
        if (seen > 0) a.state[4 * b + 1] = 1;
    }
    if (a.masks && seen == 0) return;                       // J = I: pair masked (Design-4)

    // ---- S4/S5: [W_i W_j] <- [W_i W_j] J, [V_i V_j] <- [V_i V_j] J ----------
    if constexpr (kCplx) jc_fragments<NB, NT, LDG>(J, Jf, tid);
    else                 j_fragments<NB, NT, LDG>(J, Jf, tid);
    __syncthreads();
    const int tw = (sh.M + 15) / 16, tt = tw + (sh.N + 15) / 16;
    for (int tile = warp; tile < tt; tile += NW) {
        if constexpr (kCplx) {
            if (tile < tw) update_rows_c64_mma<NB>(Wm, sh.M, sh.M, 16 * tile, bi * NB, bj * NB, Jf, lane);
            else           update_rows_c64_mma<NB>(Vm, sh.N, sh.N, 16 * (tile - tw), bi * NB, bj * NB, Jf, lane);
        } else {
            if (tile < tw) update_rows_mma<NB>(Wm, sh.M, sh.M, 16 * tile, bi * NB, bj * NB, Jf, lane);
            else           update_rows_mma<NB>(Vm, sh.N, sh.N, 16 * (tile - tw), bi * NB, bj * NB, Jf, lane);
        }
    }
}

}  // namespace bsvd
