// jacobi_common.cuh -- device building blocks shared by the fused and the
// multi-kernel Jacobi SVD paths: the round-robin ordering, barriers and warp
// reductions, and the inner Jacobi eigensolver on a 2nb x 2nb Gram block.
#pragma once

#include <type_traits>

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

// One slot's pair over consecutive round-robin steps: the ring positions of
// its two players move back one place per step, so advancing costs two
// compares instead of rr_pair's modular arithmetic.  Starts at step 0.
struct RRSlot {
    int L, slot, pa, pb;
    __device__ __forceinline__ RRSlot(int L_, int slot_)
        : L(L_), slot(slot_), pa(slot_ == 0 ? 0 : slot_ - 1), pb(L_ - 2 - slot_) {}
    __device__ __forceinline__ void next() {
        pa = pa == 0 ? L - 2 : pa - 1;
        pb = pb == 0 ? L - 2 : pb - 1;
    }
    __device__ __forceinline__ void pair(int& i, int& j) const {
        const int a = slot == 0 ? 0 : rr_start(L, pa), b = rr_start(L, pb);
        i = min(a, b);
        j = max(a, b);
    }
};

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

// Rotation tables of the inner solver: two steps' worth (double-buffered, so
// the next step's rotations can be formed while the current step's are still
// being applied) of nb disjoint rotations, one 16-byte-aligned record per
// rotation -- c, t = tan(theta), e s with e = e^{i phi}, and the index pair
// with a fired flag packed in one word -- so a reader fetches a rotation with
// one or two vector loads; plus one fired-rotation counter per sweep parity.
// Laid out in shared memory right after J.
template <class T, int NB>
struct InnerTables {
    using R = Real<T>;
    struct alignas(16) Slot {
        R c, t;
        T es;
        int pqf;   // p | q << 8 | fired << 16
    };
    using Step = Slot*;
    static constexpr int kStepBytes = NB * (int)sizeof(Slot);
    char* base;
    int* count;   // [2]
    __device__ explicit InnerTables(void* b)
        : base(static_cast<char*>(b)), count(reinterpret_cast<int*>(static_cast<char*>(b) + 2 * kStepBytes)) {}
    // step k's records, by address arithmetic (an indexed array of pointers
    // would live in local memory and cost a load per use)
    __device__ __forceinline__ Slot* step(int k) const { return reinterpret_cast<Slot*>(base + k * kStepBytes); }
    __host__ __device__ static constexpr int bytes() { return 2 * kStepBytes + 16; }
};

// Below this, g_pp g_qq is not squared-compared (its square could underflow).
template <class R> constexpr R kJacobiProdMin = R(0);
template <> constexpr float kJacobiProdMin<float> = 1e-30f;
template <> constexpr double kJacobiProdMin<double> = 1e-280;

// Products that the compiler may not fuse into a neighbouring add, and the
// combinations c x + y e and c x - y e (c real) of the 2 x 2 rotations with
// every rounding fixed by explicit FMAs: the inner solver then gives the same
// bits in every kernel that inlines it, whatever the surrounding code.
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }

__device__ __forceinline__ float rot_add(float x, float c, float y, float e) { return fmaf(y, e, __fmul_rn(x, c)); }
__device__ __forceinline__ double rot_add(double x, double c, double y, double e) { return fma(y, e, __dmul_rn(x, c)); }
__device__ __forceinline__ float2 rot_add(float2 x, float c, float2 y, float2 e) {
    return make_float2(fmaf(y.x, e.x, fmaf(-y.y, e.y, __fmul_rn(x.x, c))),
                       fmaf(y.x, e.y, fmaf(y.y, e.x, __fmul_rn(x.y, c))));
}
__device__ __forceinline__ double2 rot_add(double2 x, double c, double2 y, double2 e) {
    return make_double2(fma(y.x, e.x, fma(-y.y, e.y, __dmul_rn(x.x, c))),
                        fma(y.x, e.y, fma(y.y, e.x, __dmul_rn(x.y, c))));
}
__device__ __forceinline__ float rot_sub(float x, float c, float y, float e) { return fmaf(-y, e, __fmul_rn(x, c)); }
__device__ __forceinline__ double rot_sub(double x, double c, double y, double e) { return fma(-y, e, __dmul_rn(x, c)); }
__device__ __forceinline__ float2 rot_sub(float2 x, float c, float2 y, float2 e) {
    return make_float2(fmaf(-y.x, e.x, fmaf(y.y, e.y, __fmul_rn(x.x, c))),
                       fmaf(-y.x, e.y, fmaf(-y.y, e.x, __fmul_rn(x.y, c))));
}
__device__ __forceinline__ double2 rot_sub(double2 x, double c, double2 y, double2 e) {
    return make_double2(fma(-y.x, e.x, fma(y.y, e.y, __dmul_rn(x.x, c))),
                        fma(-y.x, e.y, fma(-y.y, e.x, __dmul_rn(x.y, c))));
}

// t = sign(x) y / (|x| + hypot(x, y)), y > 0.  Within the range where
// x^2 + y^2 neither overflows nor underflows the hypotenuse is one square
// root of an FMA (hypot elsewhere); FP32 then divides with the fast division
// (a couple of ulp), FP64 with the IEEE one.  Any t close to the exact one
// gives an orthogonal rotation, since c = 1/sqrt(1 + t^2) and s = t c.
__device__ __forceinline__ float rotation_tan(float x, float y) {
    const float ax = fabsf(x), m = fmaxf(ax, y);
    const float h = (m > 1e-18f && m < 1e18f) ? sqrtf(fmaf(x, x, __fmul_rn(y, y))) : hypotf(x, y);
    const float yy = x >= 0.f ? y : -y;
    return (m > 1e-18f && m < 1e18f) ? __fdividef(yy, ax + h) : yy / (ax + h);
}
__device__ __forceinline__ double rotation_tan(double x, double y) {
    const double ax = fabs(x), m = fmax(ax, y);
    const double h = (m > 1e-150 && m < 1e150) ? sqrt(fma(x, x, __dmul_rn(y, y))) : hypot(x, y);
    return (x >= 0 ? y : -y) / (ax + h);
}

// |g_pq| for the pair test and the rotation: the same one-square-root form
// for complex entries in the safe range, hypot elsewhere.
__device__ __forceinline__ float abs_rot(float x) { return fabsf(x); }
__device__ __forceinline__ double abs_rot(double x) { return fabs(x); }
__device__ __forceinline__ float abs_rot(float2 z) {
    const float m = fmaxf(fabsf(z.x), fabsf(z.y));
    return (m > 1e-18f && m < 1e18f) ? sqrtf(fmaf(z.x, z.x, __fmul_rn(z.y, z.y))) : hypotf(z.x, z.y);
}
__device__ __forceinline__ double abs_rot(double2 z) {
    const double m = fmax(fabs(z.x), fabs(z.y));
    return (m > 1e-150 && m < 1e150) ? sqrt(fma(z.x, z.x, __dmul_rn(z.y, z.y))) : hypot(z.x, z.y);
}

// Bit patterns ordered like the values for non-negative reals (and below
// zero for negative ones): sign and range tests on the integer pipes, which
// the FP64 pipe does not share.
__device__ __forceinline__ int as_ord(float x) { return __float_as_int(x); }
__device__ __forceinline__ long long as_ord(double x) { return __double_as_longlong(x); }
template <class R> struct RotRange;
template <> struct RotRange<float> { static constexpr float lo = 1e-18f, hi = 1e18f; };
template <> struct RotRange<double> { static constexpr double lo = 1e-150, hi = 1e150; };

// Eq. (sin-cos) for x = g_pp - g_qq and y = 2|g_pq| > 0.  With h = hypot(x, y)
// and d = |x| + h:  t = sign(x) y / d,  c = 1/sqrt(1 + t^2) = d / sqrt(d^2 + y^2),
// and since d^2 + y^2 = 2 h d:  c = d r,  s = t c = sign(x) y r,  t = s (2 h r),
// with r = 1/sqrt(2 h d) and h = q/sqrt(q), q = x^2 + y^2 -- two reciprocal
// square roots and no division.  Used where q and 2 h d neither overflow nor
// underflow (max(|x|, y) in [lo, hi]); elsewhere t = sign(x) y / (|x| + h),
// c = 1/sqrt(1 + t^2), s = t c.  sign(0) = +1 (x = g_pp - g_qq is never -0).
template <class R>
__device__ __forceinline__ void rotation_cst(R x, R y, R& c, R& s, R& t) {
    const R ax = abs_s(x);
    const auto bm = as_ord(ax) > as_ord(y) ? as_ord(ax) : as_ord(y);
    if (bm > as_ord(RotRange<R>::lo) && bm < as_ord(RotRange<R>::hi)) {
        const R q = fma_s(x, x, rmul(y, y));
        const R h = rmul(q, rsqrt_r(q));
        const R d = ax + h, h2 = h + h;
        const R r = rsqrt_r(rmul(h2, d));
        const R sy = rmul(y, r);
        s = as_ord(x) >= 0 ? sy : -sy;
        c = rmul(d, r);
        t = rmul(s, rmul(h2, r));
    } else {
        t = rotation_tan(x, y);
        c = rsqrt_r(fma_s(t, t, R(1)));
        s = rmul(t, c);
    }
}

// e^{i phi} s for the rotation, phi the phase of g_pq (|g_pq| = a > 0):
// for real data the sign of g_pq applied to s.
__device__ __forceinline__ float phase_times(float g, float, float s) {
    return __int_as_float(__float_as_int(s) ^ (__float_as_int(g) & (int)0x80000000u));
}
__device__ __forceinline__ double phase_times(double g, double, double s) {
    return __longlong_as_double(__double_as_longlong(s) ^ (__double_as_longlong(g) & (long long)0x8000000000000000ull));
}
__device__ __forceinline__ float2 phase_times(float2 g, float a, float s) {
    const float k = s * (1.0f / a);
    return make_float2(g.x * k, g.y * k);
}
__device__ __forceinline__ double2 phase_times(double2 g, double a, double s) {
    const double k = s * (1.0 / a);
    return make_double2(g.x * k, g.y * k);
}

// FP64 counterparts of the single-precision types, for rotations computed in
// FP64 from FP32 Gram entries (the mixed-precision option).
template <class T> struct WideOf { using type = T; };
template <> struct WideOf<float> { using type = double; };
template <> struct WideOf<float2> { using type = double2; };
__device__ __forceinline__ double to_wide(float x) { return (double)x; }
__device__ __forceinline__ double2 to_wide(float2 x) { return make_double2((double)x.x, (double)x.y); }
__device__ __forceinline__ float to_narrow(double x) { return __double2float_rn(x); }
__device__ __forceinline__ float2 to_narrow(double2 x) { return make_float2(__double2float_rn(x.x), __double2float_rn(x.y)); }

// The pair's diagonal 2 x 2 block of G <- R^H G R by the closed form:
// g_pp += t |g_pq|, g_qq -= t |g_pq|, g_pq = g_qp = 0.  Applied by the lane
// that formed the rotation, as soon as it is formed: in the steps between,
// no other block transform and no other lane reads these four entries.
template <class T, int LDG>
__device__ __forceinline__ void diagonal_block(T* G, int p, int q, Real<T> gpp, Real<T> gqq, Real<T> apq,
                                               Real<T> t) {
    G[p + p * LDG] = make_s<T>(fma_s(t, apq, gpp));
    G[q + q * LDG] = make_s<T>(fma_s(-t, apq, gqq));
    G[p + q * LDG] = make_s<T>(0);
    G[q + p * LDG] = make_s<T>(0);
}

// The rotation of inner_rotation with the pair test and Eq. (sin-cos)
// evaluated in FP64 on the single-precision Gram entries (exactly widened),
// c, t and e s rounded once to the working precision at the end.
template <class T, int NB>
__device__ __forceinline__ int inner_rotation_wide(T* G, Real<T> tol, int p, int q, int slot,
                                                   typename InnerTables<T, NB>::Slot* out) {
    using R = Real<T>;
    using TW = typename WideOf<T>::type;
    using RW = Real<TW>;
    constexpr int LDG = 2 * NB + 1;
    const RW gpp = (RW)re(G[p + p * LDG]), gqq = (RW)re(G[q + q * LDG]);
    const TW gpq = to_wide(G[p + q * LDG]);
    const RW apq = abs_rot(gpq), tw = (RW)tol;
    // squares of widened single-precision values stay inside FP64's range
    const bool fire = gpp > 0 && gqq > 0 && apq > 0 && apq * apq >= (tw * tw) * (gpp * gqq);
    RW c = 1, t = 0;
    TW es = make_s<TW>(0);
    if (fire) {
        RW sn;
        rotation_cst(gpp - gqq, 2 * apq, c, sn, t);
        es = phase_times(gpq, apq, sn);
    }
    typename InnerTables<T, NB>::Slot rec;
    rec.c = (R)c; rec.t = (R)t; rec.es = to_narrow(es);
    rec.pqf = p | (q << 8) | ((fire ? 1 : 0) << 16);
    out[slot] = rec;
    // the closed form in the working precision, with the rounded t
    if (fire) diagonal_block<T, LDG>(G, p, q, (R)gpp, (R)gqq, abs_rot(G[p + q * LDG]), rec.t);
    return fire;
}

// One thread's rotation for slot `slot` (index pair p < q of the current
// round-robin step on the 2NB indices): test |g_pq| >= tol sqrt(g_pp)
// sqrt(g_qq) (Alg. 1) and form (c, s, e^{i phi}) by Eq. (sin-cos) with
// sign(0) = +1.  Returns fired.  `wide` (single precision only): test and
// rotation in FP64.
template <class T, int NB>
__device__ __forceinline__ int inner_rotation(T* G, Real<T> tol, int p, int q, int slot,
                                              typename InnerTables<T, NB>::Slot* out, bool wide = false) {
    using R = Real<T>;
    constexpr int TWO = 2 * NB, LDG = TWO + 1;
    if constexpr (!std::is_same<T, typename WideOf<T>::type>::value)
        if (wide) return inner_rotation_wide<T, NB>(G, tol, p, q, slot, out);
    const R gpp = re(G[p + p * LDG]), gqq = re(G[q + q * LDG]);
    const T gpq = G[p + q * LDG];
    const R apq = abs_rot(gpq);
    // |g_pq| >= tol sqrt(g_pp) sqrt(g_qq), compared in squares while the
    // product stays well inside the normal range; the sign and range tests
    // on the bit patterns (a NaN operand still fails the comparison)
    const R prod = rmul(gpp, gqq);
    const bool pos = (as_ord(gpp) > 0) & (as_ord(gqq) > 0) & (as_ord(apq) > 0);
    const bool fire = pos && (as_ord(prod) > as_ord(kJacobiProdMin<R>)
                                  ? rmul(apq, apq) >= rmul(rmul(tol, tol), prod)
                                  : apq >= rmul(rmul(tol, sqrt_r(gpp)), sqrt_r(gqq)));
    R c = 1, t = 0;
    T es = make_s<T>(0);
    if (fire) {
        // tau = x / y with x = g_pp - g_qq, y = 2 |g_pq|:
        // t = sign(tau) / (|tau| + sqrt(1 + tau^2)) = sign(x) y / (|x| + hypot(x, y))
        R sn;
        rotation_cst(gpp - gqq, 2 * apq, c, sn, t);
        es = phase_times(gpq, apq, sn);
    }
    typename InnerTables<T, NB>::Slot rec;
    rec.c = c; rec.t = t; rec.es = es;
    rec.pqf = p | (q << 8) | ((fire ? 1 : 0) << 16);
    out[slot] = rec;
    if (fire) diagonal_block<T, LDG>(G, p, q, gpp, gqq, apq, t);
    return fire;
}

// Up to `sweeps` sweeps of Alg. 1 on the Hermitian G (2NB x 2NB, leading
// dimension 2NB+1, in shared memory), accumulating the rotations into J
// (set to I here).  One sweep is 2NB-1 parallel steps of the round-robin
// ordering on the 2NB indices, each applying nb disjoint rotations:
// G <- R^H G R as 2x2 block transforms (rows of one slot, columns of another;
// the diagonal block by the closed form g_pp += t|g_pq|, g_qq -= t|g_pq|,
// g_pq = 0, applied by the lane that forms the rotation) and J <- J R.
// Pipelined: while the other warps apply step s to J, warp 0 already forms
// the rotations of step s+1 from the updated G.
// Sweeps stop early once one rotates nothing.  Executed by GT threads (index
// gt) sharing named barrier `bar`; the caller must have finished writing G and
// synchronised.  Returns the number of rotations fired (0: G was diagonal to
// tol); uniform over the group.
// Work the caller hands the J-update warps: called once per step by each of
// them, with a running per-warp task index (step * background warps + warp).
struct NoBackground {
    __device__ __forceinline__ void operator()(int) const {}
};
template <int GT>
__host__ __device__ constexpr int inner_background_warps() { return GT > 32 ? GT / 32 - 1 : 1; }

template <class T, int NB, int GT, class Bg = NoBackground>
__device__ int inner_jacobi(T* G, T* J, const InnerTables<T, NB>& tb, Real<T> tol, int sweeps,
                            int gt, int bar, const Bg& bg = Bg(), int* nsteps = nullptr, bool wide = false) {
    using R = Real<T>;
    constexpr int TWO = 2 * NB, LDG = TWO + 1, STEPS = TWO - 1;
    // The off-diagonal 2x2 blocks of G by slot pair (two rotations each);
    // the diagonal ones (the closed form) are applied by the lane of warp 0
    // that forms their rotation, right after forming it.
    constexpr int NOFF = NB * (NB - 1) / 2, NBU = (NOFF + GT - 1) / GT;
    // J-update workers: every warp but the first when there is more than one
    constexpr int JW0 = GT > 32 ? 32 : 0, JWN = GT - JW0;
    // Items of the first round go to the last NOFF threads (at most warp 0's
    // 32 threads left idle, so that warp 0 can find the next step's pairs
    // meanwhile); further rounds alternate in direction.  Blocks are
    // disjoint: the assignment does not change any result.
    constexpr int BASE = GT - NOFF < 0 ? 0 : (GT - NOFF < 32 ? GT - NOFF : 32);
    int bq1[NBU], bq2[NBU];
#pragma unroll
    for (int u = 0; u < NBU; ++u) {
        const int e = u * GT + ((u & 1) ? GT - 1 - gt : gt - BASE);
        if (e >= 0 && e < NOFF) {
            int a, c;
            tri_index(e, a, c);           // a <= c: the strict pair (a, c + 1)
            bq1[u] = a; bq2[u] = c + 1;
        } else {
            bq1[u] = -1; bq2[u] = -1;
        }
    }
    for (int e = gt; e < TWO * TWO; e += GT)
        J[(e % TWO) + (e / TWO) * LDG] = make_s<T>((e % TWO) == (e / TWO) ? 1 : 0);
    named_sync(bar, GT);
    // warp 0 forms the rotations, lane `slot` those of one slot, following
    // its pair through the steps (the next step's pair is found during the
    // block transforms, where warp 0 is not the last to finish); one ballot
    // counts the fired ones, summed per sweep in a register of thread 0 and
    // stored to tb.count[sweep parity] at the sweep's last step
    RRSlot rs(TWO, gt < NB ? gt : 0);
    int np = 0, nq = 0, fired_sweep = 0;
    if (gt < 32) {
        rs.pair(np, nq);
        const int f = gt < NB ? inner_rotation<T, NB>(G, tol, np, nq, gt, tb.step(0), wide) : 0;
        fired_sweep = __popc(__ballot_sync(0xffffffffu, f));
    }
    named_sync(bar, GT);
    int seen = 0;
    for (int isw = 0; isw < sweeps; ++isw) {
        for (int st = 0; st < STEPS; ++st) {
            const int gs = isw * STEPS + st;
            const auto cur = tb.step(gs & 1);
            // G <- R^H G R on 2x2 blocks (slot q1 <= slot q2), mirrored.  A
            // thread's blocks are disjoint: all loads first, then the math,
            // then the stores, so their latencies overlap.
            {
                int f1[NBU], f2[NBU], p1[NBU], r1[NBU], p2[NBU], r2[NBU];
                R c1[NBU], c2[NBU];
                T e1[NBU], e2[NBU], b00[NBU], b01[NBU], b10[NBU], b11[NBU];
#pragma unroll
                for (int u = 0; u < NBU; ++u) {
                    f1[u] = f2[u] = 0;
                    if (bq1[u] < 0) continue;
                    const auto s1 = cur[bq1[u]], s2 = cur[bq2[u]];
                    f1[u] = s1.pqf >> 16; f2[u] = s2.pqf >> 16;
                    p1[u] = s1.pqf & 255; r1[u] = (s1.pqf >> 8) & 255;
                    p2[u] = s2.pqf & 255; r2[u] = (s2.pqf >> 8) & 255;
                    c1[u] = s1.c; c2[u] = s2.c;
                    e1[u] = s1.es; e2[u] = s2.es;
                }
#pragma unroll
                for (int u = 0; u < NBU; ++u) {
                    if (!f1[u] && !f2[u]) continue;
                    b00[u] = G[p1[u] + p2[u] * LDG]; b01[u] = G[p1[u] + r2[u] * LDG];
                    b10[u] = G[r1[u] + p2[u] * LDG]; b11[u] = G[r1[u] + r2[u] * LDG];
                }
#pragma unroll
                for (int u = 0; u < NBU; ++u) {
                    if (!f1[u] && !f2[u]) continue;
                    if (f2[u]) {   // columns (p2, r2) times R2
                        const T es = e2[u], ces = conj_s(es);
                        const T n00 = rot_add(b00[u], c2[u], b01[u], ces);
                        const T n01 = rot_sub(b01[u], c2[u], b00[u], es);
                        const T n10 = rot_add(b10[u], c2[u], b11[u], ces);
                        const T n11 = rot_sub(b11[u], c2[u], b10[u], es);
                        b00[u] = n00; b01[u] = n01; b10[u] = n10; b11[u] = n11;
                    }
                    if (f1[u]) {   // rows (p1, r1) times R1^H
                        const T es = e1[u], ces = conj_s(es);
                        const T n00 = rot_add(b00[u], c1[u], b10[u], es);
                        const T n10 = rot_sub(b10[u], c1[u], b00[u], ces);
                        const T n01 = rot_add(b01[u], c1[u], b11[u], es);
                        const T n11 = rot_sub(b11[u], c1[u], b01[u], ces);
                        b00[u] = n00; b01[u] = n01; b10[u] = n10; b11[u] = n11;
                    }
                }
#pragma unroll
                for (int u = 0; u < NBU; ++u) {
                    if (!f1[u] && !f2[u]) continue;
                    G[p1[u] + p2[u] * LDG] = b00[u]; G[p1[u] + r2[u] * LDG] = b01[u];
                    G[r1[u] + p2[u] * LDG] = b10[u]; G[r1[u] + r2[u] * LDG] = b11[u];
                    G[p2[u] + p1[u] * LDG] = conj_s(b00[u]); G[r2[u] + p1[u] * LDG] = conj_s(b01[u]);
                    G[p2[u] + r1[u] * LDG] = conj_s(b10[u]); G[r2[u] + r1[u] * LDG] = conj_s(b11[u]);
                }
            }
            if (gt < 32) {
                rs.next();                    // step st + 1, or step 0 of the next sweep (2NB - 1 = 0 mod the ring)
                rs.pair(np, nq);
            }
            named_sync(bar, GT);
            // warp 0: the rotations of the next step (this sweep, or the first
            // step of the next one) from the updated G
            const bool last = (st + 1 == STEPS);
            auto form_next = [&]() {
                unsigned m = 0;
                if (!(last && isw + 1 == sweeps)) {
                    const int f = gt < NB ? inner_rotation<T, NB>(G, tol, np, nq, gt, tb.step((gs + 1) & 1), wide) : 0;
                    m = __ballot_sync(0xffffffffu, f);
                }
                if (gt == 0) {
                    if (last) {       // sweep isw complete; m starts sweep isw + 1
                        tb.count[isw & 1] = fired_sweep;
                        fired_sweep = __popc(m);
                    } else {
                        fired_sweep += __popc(m);
                    }
                }
            };
            // the other warps: J <- J R for every rotating slot of this step
            // (items are disjoint: all loads, then the math, then the stores)
            auto update_j = [&]() {
                constexpr int NJU = (TWO * NB + JWN - 1) / JWN;
                int fj[NJU], pj[NJU], qj[NJU], ij[NJU];
                R cj[NJU];
                T ej[NJU], xj[NJU], yj[NJU];
#pragma unroll
                for (int u = 0; u < NJU; ++u) {
                    const int e = gt - JW0 + u * JWN;
                    fj[u] = 0;
                    if (e >= TWO * NB) continue;
                    const auto sj = cur[e / TWO];
                    ij[u] = e % TWO;
                    fj[u] = sj.pqf >> 16; pj[u] = sj.pqf & 255; qj[u] = (sj.pqf >> 8) & 255;
                    cj[u] = sj.c; ej[u] = sj.es;
                }
#pragma unroll
                for (int u = 0; u < NJU; ++u)
                    if (fj[u]) { xj[u] = J[ij[u] + pj[u] * LDG]; yj[u] = J[ij[u] + qj[u] * LDG]; }
#pragma unroll
                for (int u = 0; u < NJU; ++u)
                    if (fj[u]) {
                        const T es = ej[u], ces = conj_s(es);
                        J[ij[u] + pj[u] * LDG] = rot_add(xj[u], cj[u], yj[u], ces);
                        J[ij[u] + qj[u] * LDG] = rot_sub(yj[u], cj[u], xj[u], es);
                    }
                bg(gs * inner_background_warps<GT>() + (gt - JW0) / 32);
            };
            if constexpr (JW0 == 0) {          // one warp: both, in turn
                form_next();
                update_j();
            } else if (gt < 32) {
                form_next();
            } else {
                update_j();
            }
            named_sync(bar, GT);
            if (nsteps) *nsteps = gs + 1;
        }
        // written by thread 0 before the last barrier; rewritten only at the
        // end of sweep isw + 2, after every thread has passed this point
        const int fired = tb.count[isw & 1];
        seen += fired;
        if (fired == 0) break;         // a sweep with no rotation: the inner solve has converged
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
