// blocked_layout.h -- arguments and per-matrix workspace layout of the
// multi-kernel path (shared by the C-ABI layer and the kernel launcher).
#pragma once

#include <stddef.h>

#include <algorithm>
#include <vector>

namespace bsvd {

// One matrix of a variable-shape batch: its working shape and where its
// regions start in the workspace (elements from each region's base).
struct BlkShape {
    int M, N, trans, m, n, l, L, Np;
    long long oW, oV, oG, oJ, oT;
};

// Arguments of the multi-kernel path (type-erased pointers).
struct BlockedArgs {
    int M, N, trans, m, n;     // working shape (M >= N) and the caller's
    int l, L, Np;              // blocks (l >= 2), L = l + (l odd), Np = l * nb
    int count;                 // matrices in this launch group
    // workspace, per matrix: W (M x Np, ld M), Vw (N x Np, ld N), G and J
    // (L/2 blocks of 2nb x 2nb), T (L/2 x (M+N) x 2nb two-stage temporary,
    // also the finalisation scratch: >= M + N*N + N elements)
    void* W; void* Vw; void* G; void* J; void* T;
    long long sW, sVw, sG, sJ, sT;
    int* state;                // count x 4: status (1 active, 0 converged, -1 bad), rotated, sweeps, exponent
    int* pairflag;             // count x L/2: the pair rotated in this round
    int* any_active;           // one int: some matrix still active after a sweep
    // caller's arrays (as FusedArgs)
    const void* A; long long sA; int lda; const void* const* Ap; const int* ldap;
    const void* V0; long long sV0; int ldv0;   // initial V (N x N, by matrix id) or nullptr for I
    void* S; long long sS; void* const* Sp;
    void* U; long long sU; int ldu; void* const* Up; const int* ldup;
    void* V; long long sV; int ldv; void* const* Vp; const int* ldvp;
    const int* index;
    int in_local;              // 1: strided A and V0 by launch position, outputs by matrix id
    int* info; int* sweeps;
    double tol;
    int max_sweeps, inner_sweeps, flags;
    int masks;                 // Design-4
    int wantU, wantV;
    // variable-shape batch: per-matrix shapes and offsets (device, count
    // entries); the scalar shape fields above then hold the maxima
    const BlkShape* shapes;
};

inline size_t blk_align(size_t x) { return (x + 255) & ~size_t(255); }

// Per-matrix element counts of each workspace region.
struct BlkSizes {
    long long W, V, G, J, T;
    int l, L, Np;
};

inline BlkSizes blk_sizes(int nb, int M, int N, bool two_stage) {
    BlkSizes z;
    z.l = std::max(2, (N + nb - 1) / nb);
    z.L = z.l + (z.l & 1);
    z.Np = z.l * nb;
    const long long two = 2LL * nb, pairs = z.L / 2;
    z.W = (long long)M * z.Np;
    z.V = (long long)N * z.Np;
    z.G = pairs * two * two;
    z.J = z.G;
    const long long fin = (long long)M + (long long)N * N + N;       // finalisation: x, E, rank
    z.T = std::max(two_stage ? pairs * (M + N) * two : 0LL, fin);
    return z;
}

// A variable-shape batch (fused vector update, no two-stage temporary):
// per-matrix shapes and offsets, the maxima, and the workspace bytes.
struct BlkVarPlan {
    std::vector<BlkShape> shapes;
    int Mmax = 0, Nmax = 0, lmax = 2, Lmax = 2;
    long long W = 0, V = 0, G = 0, J = 0, T = 0;   // region sizes (elements)
    size_t bytes = 0;
};

inline void blk_var_plan(int nb, int count, const int* m, const int* n, size_t elt, BlkVarPlan& p) {
    p = BlkVarPlan();
    p.shapes.resize(count);
    for (int b = 0; b < count; ++b) {
        BlkShape& s = p.shapes[b];
        s.m = m[b]; s.n = n[b]; s.trans = m[b] < n[b];
        s.M = std::max(m[b], n[b]); s.N = std::min(m[b], n[b]);
        const BlkSizes z = blk_sizes(nb, s.M, s.N, false);
        s.l = z.l; s.L = z.L; s.Np = z.Np;
        s.oW = p.W; s.oV = p.V; s.oG = p.G; s.oJ = p.J; s.oT = p.T;
        p.W += z.W; p.V += z.V; p.G += z.G; p.J += z.J; p.T += z.T;
        p.Mmax = std::max(p.Mmax, s.M); p.Nmax = std::max(p.Nmax, s.N);
        p.lmax = std::max(p.lmax, s.l); p.Lmax = std::max(p.Lmax, s.L);
    }
    p.bytes = blk_align((size_t)count * 4 * sizeof(int)) + blk_align((size_t)count * (p.Lmax / 2) * sizeof(int)) +
              blk_align(sizeof(int)) + blk_align((size_t)count * sizeof(BlkShape)) +
              blk_align((size_t)(p.W + p.V + p.G + p.J + p.T) * elt);
}

inline size_t blk_bytes(int nb, int M, int N, int count, bool two_stage, size_t elt) {
    const BlkSizes z = blk_sizes(nb, M, N, two_stage);
    size_t b = blk_align((size_t)count * 4 * sizeof(int)) + blk_align((size_t)count * (z.L / 2) * sizeof(int)) +
               blk_align(sizeof(int));
    b += blk_align((size_t)count * (z.W + z.V + z.G + z.J + z.T) * elt);
    return b;
}

}  // namespace bsvd
