/*
 * oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow FP64 / complex128 CPU restatement of the one-sided Jacobi SVD
 * of "An Efficient Batch Solver for the Singular Value Decomposition on GPUs"
 * (Abdelfattah and Fasi).  It exists to check the CUDA path and shares no
 * code, header, table or helper with it.  Only the test suite, the smoke
 * check and the benchmark's CPU-baseline leg may load it.  FP32 inputs are
 * widened to FP64 (exactly) by the caller; all arithmetic here is FP64.
 *
 * Entry points (each cites the passage it restates):
 *   oracle_rr_pair           Brent-Luk round-robin ordering (Sec. 3; Sec. 4.1),
 *                            pinned by the worked example of Sec. 5.1.
 *   oracle_{d,z}heevj        Alg. 1, the Jacobi Hermitian eigensolver, rotation
 *                            by Eq. (sin-cos), round-robin order (Sec. 4.3).
 *   oracle_{d,z}gesvj        Alg. 2, unblocked one-sided Jacobi SVD, row-cyclic
 *                            pairs (Forsythe-Henrici, Sec. 3); sigma = column
 *                            norms, U = A / sigma, descending sort.
 *   oracle_{d,z}gesvj_blocked  the blocked method of Sec. 3 (Eq. block-gram,
 *                            right-sv) in the steps S1-S5 of Sec. 4, with a
 *                            fixed number of inner sweeps (1 = Design-2, Sec. 5).
 *   oracle_gesvj_blocked_rounds  the first k round-robin iterations of it only,
 *                            returning A^(k) (to check the states of Sec. 5.1).
 *   oracle_gesvj_batch       an OpenMP loop over independent matrices.
 *
 * Readings where the paper is silent or garbled:
 *   R1  Eq. (jacobi-rotation) prints -e^{-i phi} sin(theta) at (i,j), which is
 *       not unitary; the 2x2 form of Eq. (background-eigenproblem-jacobi) is
 *       used, J = [[c, -e^{i phi} s], [e^{-i phi} s, c]].
 *   R2  sign(0) = +1 in t_min, so equal diagonals rotate by pi/4.
 *   R3  sqrt(1 + tau^2) is evaluated as hypot(1, tau), which cannot overflow.
 *   R4  A pair with a zero diagonal (zero column) takes no rotation.
 *   R5  A column of norm exactly zero gets as left singular vector the standard
 *       basis vector with the largest residual off the columns of U already
 *       set, projected off them twice and normalised, so that U^H U = I.
 *   R6  m < n is solved on A^H (Sec. 6.2: A^H = V Sigma U^H).
 *   R7  The matrix is first scaled by an exact power of two taking its largest
 *       entry into [1, 2); sigma is scaled back at the end.  No rounding
 *       changes; squared column norms stay inside the exponent range.
 *   R8  info = 0 when converged; info = number of sweeps run when the last
 *       one still rotated (max_sweeps reached); info = -1 when an input entry
 *       is not finite (outputs are then NaN).
 *
 * Storage: column-major with leading dimensions (LAPACK); complex data is
 * interleaved (re, im) doubles, i.e. C99 double complex.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------------ */
/* Round-robin parallel ordering (Brent and Luk; Sec. 3, Sec. 4.1).          */
/* Players 0..l-1 (l even) sit in two rows, top T = [0,2,4,...] and bottom   */
/* B = [1,3,5,...]; slot q of a round pairs T[q] with B[q].  T[0] stays put;  */
/* the other l-1 players sit on the ring T[1..k-1], B[k-1..0] and move one    */
/* place along it per round.  For l = 4 the rounds are (0,1)(2,3),            */
/* (0,3)(1,2), (0,2)(1,3): the block-pair sequence of the worked example in  */
/* Sec. 5.1 (pairs (1,2),(3,4), then (1,4),(2,3) in 1-based numbering).       */
/* ------------------------------------------------------------------------ */
static int rr_initial(int l, int p0)
{
    int k = l / 2;
    if (p0 < k - 1) return 2 * (p0 + 1);           /* T[p0+1] */
    return 2 * (l - 2 - p0) + 1;                   /* B[l-2-p0] */
}

void oracle_rr_pair(int l, int r, int q, int* i, int* j)
{
    int ring = l - 1, a, b;
    if (q == 0) a = 0;
    else        a = rr_initial(l, (((q - 1) - r) % ring + ring) % ring);
    b = rr_initial(l, (((l - 2 - q) - r) % ring + ring) % ring);
    *i = a < b ? a : b;
    *j = a < b ? b : a;
}

/* ---- real instantiation ---- */
#define S_T double
#define F(name) name##_d
#define CONJ(x) (x)
#define ABSV(x) fabs(x)
#define ABS2(x) ((x) * (x))
#define REAL(x) (x)
#define LDEXP_S(x, e) ldexp((x), (e))
#define FINITE_S(x) isfinite(x)
#define NAN_S NAN
#define NPARTS 1
#define PART(x, h) (x)
#include "oracle_core.h"
#undef S_T
#undef F
#undef CONJ
#undef ABSV
#undef ABS2
#undef REAL
#undef LDEXP_S
#undef FINITE_S
#undef NAN_S
#undef NPARTS
#undef PART

/* ---- complex instantiation ---- */
typedef double complex zc;
static inline double zpart(zc x, int h) { return h ? cimag(x) : creal(x); }
#define S_T zc
#define F(name) name##_z
#define CONJ(x) conj(x)
#define ABSV(x) cabs(x)
#define ABS2(x) (creal(x) * creal(x) + cimag(x) * cimag(x))
#define REAL(x) creal(x)
#define LDEXP_S(x, e) CMPLX(ldexp(creal(x), (e)), ldexp(cimag(x), (e)))
#define FINITE_S(x) (isfinite(creal(x)) && isfinite(cimag(x)))
#define NAN_S CMPLX(NAN, NAN)
#define NPARTS 2
#define PART(x, h) zpart((x), (h))
#include "oracle_core.h"

/* ------------------------------------------------------------------------ */
/* Public entry points                                                       */
/* ------------------------------------------------------------------------ */
int oracle_dheevj(int n, double* G, int ldg, double* Z, int ldz, double tol,
                  int max_sweeps, int* converged)
{
    return heevj_core_d(n, G, ldg, Z, ldz, tol, max_sweeps, converged);
}

int oracle_zheevj(int n, double* G, int ldg, double* Z, int ldz, double tol,
                  int max_sweeps, int* converged)
{
    return heevj_core_z(n, (zc*)G, ldg, (zc*)Z, ldz, tol, max_sweeps, converged);
}

/* nb <= 0: Alg. 2 (unblocked); nb > 0: the blocked method. */
static int svd_any(char dtype, int m, int n, const void* A, int lda, int nb, int inner_sweeps,
                   double tol, int max_sweeps, double* S, void* U, int ldu, void* V, int ldv,
                   int* sweeps)
{
    if (dtype == 'z') {
        if (nb <= 0)
            return gesvj_z(m, n, (const zc*)A, lda, tol, max_sweeps, S, (zc*)U, ldu, (zc*)V, ldv, sweeps);
        return gesvj_blocked_z(m, n, (const zc*)A, lda, nb, inner_sweeps, tol, max_sweeps,
                               S, (zc*)U, ldu, (zc*)V, ldv, sweeps, -1, NULL, 0);
    }
    if (nb <= 0)
        return gesvj_d(m, n, (const double*)A, lda, tol, max_sweeps, S, (double*)U, ldu,
                       (double*)V, ldv, sweeps);
    return gesvj_blocked_d(m, n, (const double*)A, lda, nb, inner_sweeps, tol, max_sweeps,
                           S, (double*)U, ldu, (double*)V, ldv, sweeps, -1, NULL, 0);
}

int oracle_dgesvj(int m, int n, const double* A, int lda, double tol, int max_sweeps,
                  double* S, double* U, int ldu, double* V, int ldv, int* sweeps)
{
    return svd_any('d', m, n, A, lda, 0, 0, tol, max_sweeps, S, U, ldu, V, ldv, sweeps);
}

int oracle_zgesvj(int m, int n, const double* A, int lda, double tol, int max_sweeps,
                  double* S, double* U, int ldu, double* V, int ldv, int* sweeps)
{
    return svd_any('z', m, n, A, lda, 0, 0, tol, max_sweeps, S, U, ldu, V, ldv, sweeps);
}

int oracle_dgesvj_blocked(int m, int n, const double* A, int lda, int nb, int inner_sweeps,
                          double tol, int max_sweeps, double* S, double* U, int ldu,
                          double* V, int ldv, int* sweeps)
{
    return svd_any('d', m, n, A, lda, nb, inner_sweeps, tol, max_sweeps, S, U, ldu, V, ldv, sweeps);
}

int oracle_zgesvj_blocked(int m, int n, const double* A, int lda, int nb, int inner_sweeps,
                          double tol, int max_sweeps, double* S, double* U, int ldu,
                          double* V, int ldv, int* sweeps)
{
    return svd_any('z', m, n, A, lda, nb, inner_sweeps, tol, max_sweeps, S, U, ldu, V, ldv, sweeps);
}

/* The first `rounds` round-robin iterations of the blocked method only; the */
/* working matrix A^(k) (m >= n orientation, m x n) is written to W.         */
int oracle_gesvj_blocked_rounds(char dtype, int m, int n, const double* A, int lda, int nb,
                                int inner_sweeps, double tol, int rounds, double* W, int ldw)
{
    if (dtype == 'z')
        return gesvj_blocked_z(m, n, (const zc*)A, lda, nb, inner_sweeps, tol, 1 << 20, NULL,
                               NULL, 1, NULL, 1, NULL, rounds, (zc*)W, ldw);
    return gesvj_blocked_d(m, n, A, lda, nb, inner_sweeps, tol, 1 << 20, NULL, NULL, 1, NULL, 1,
                           NULL, rounds, W, ldw);
}

/* Independent matrices, one per OpenMP iteration.  Host pointer arrays of    */
/* length batch; U and V may be NULL; tol is per matrix.  nb <= 0 selects     */
/* Alg. 2.  Returns the number of threads used.                               */
int oracle_gesvj_batch(char dtype, int batch, const int* m, const int* n,
                       const void* const* A, const int* lda, int nb, int inner_sweeps,
                       const double* tol, int max_sweeps, double* const* S,
                       void* const* U, const int* ldu, void* const* V, const int* ldv,
                       int* sweeps, int* info, int nthreads)
{
    int used = 1;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#pragma omp parallel
    {
#pragma omp single
        used = omp_get_num_threads();
#pragma omp for schedule(dynamic, 1)
        for (int b = 0; b < batch; ++b)
            info[b] = svd_any(dtype, m[b], n[b], A[b], lda[b], nb, inner_sweeps, tol[b], max_sweeps,
                              S[b], U ? U[b] : NULL, ldu ? ldu[b] : 1, V ? V[b] : NULL,
                              ldv ? ldv[b] : 1, sweeps ? &sweeps[b] : NULL);
    }
#else
    (void)nthreads;
    for (int b = 0; b < batch; ++b)
        info[b] = svd_any(dtype, m[b], n[b], A[b], lda[b], nb, inner_sweeps, tol[b], max_sweeps,
                          S[b], U ? U[b] : NULL, ldu ? ldu[b] : 1, V ? V[b] : NULL,
                          ldv ? ldv[b] : 1, sweeps ? &sweeps[b] : NULL);
#endif
    return used;
}
