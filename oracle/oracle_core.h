/*
 * oracle_core.h -- TEST INFRASTRUCTURE ONLY; part of oracle.c.
 *
 * The body of the oracle, written once and included by oracle.c once per
 * scalar type (double, double complex).  The including file defines:
 *   S_T          scalar type
 *   F(name)      name with the type suffix (_d or _z)
 *   CONJ(x)      complex conjugate (identity for real)
 *   ABSV(x)      |x|
 *   ABS2(x)      |x|^2 as a real
 *   REAL(x)      real part
 *   LDEXP_S(x,e) x * 2^e, exactly, part by part
 *   FINITE_S(x)  every part finite
 *   NAN_S        a NaN of type S_T
 *   NPARTS, PART(x,h)  the real parts of x for the scaled norm
 * See oracle.c for the citations and the readings R1-R8.
 */

/* Eq. (sin-cos) for the 2x2 Hermitian block [[aii, aij], [conj(aij), ajj]]: */
/* phi = arg(aij), tau = (aii - ajj)/(2|aij|),                                 */
/* t = sign(tau)/(|tau| + sqrt(1 + tau^2)), c = 1/sqrt(1+t^2), s = t c.        */
/* *e = e^{i phi} = aij/|aij| (for real data: the sign of aij).                */
static void F(rotation)(double aii, double ajj, S_T aij, double* c, double* s, S_T* e)
{
    double g = ABSV(aij);
    if (g == 0.0) { *c = 1.0; *s = 0.0; *e = 1.0; return; }
    double tau = (aii - ajj) / (2.0 * g);
    double sg = tau >= 0.0 ? 1.0 : -1.0;                  /* R2 */
    double t = sg / (fabs(tau) + hypot(1.0, tau));        /* R3 */
    *c = 1.0 / sqrt(1.0 + t * t);
    *s = t * (*c);
    *e = aij / g;
}

/* Columns i, j of X (rows x ., leading dim ld) times                         */
/* J = [[c, -e s], [conj(e) s, c]] (R1): x_i' = c x_i + conj(e) s x_j,         */
/* x_j' = -e s x_i + c x_j.                                                    */
static void F(rotate_cols)(S_T* X, int rows, int ld, int i, int j, double c, double s, S_T e)
{
    S_T j11 = c, j12 = -e * s, j21 = CONJ(e) * s, j22 = c;
    for (int p = 0; p < rows; ++p) {
        S_T x = X[p + (size_t)i * ld], y = X[p + (size_t)j * ld];
        X[p + (size_t)i * ld] = x * j11 + y * j21;
        X[p + (size_t)j * ld] = x * j12 + y * j22;
    }
}

/* Rows i, j of X (cols ., leading dim ld) times J^H from the left:           */
/* x_i' = conj(j11) x_i + conj(j21) x_j, x_j' = conj(j12) x_i + conj(j22) x_j. */
static void F(rotate_rows)(S_T* X, int cols, int ld, int i, int j, double c, double s, S_T e)
{
    S_T j11 = c, j12 = -e * s, j21 = CONJ(e) * s, j22 = c;
    for (int p = 0; p < cols; ++p) {
        S_T x = X[i + (size_t)p * ld], y = X[j + (size_t)p * ld];
        X[i + (size_t)p * ld] = CONJ(j11) * x + CONJ(j21) * y;
        X[j + (size_t)p * ld] = CONJ(j12) * x + CONJ(j22) * y;
    }
}

/* Alg. 1 on the order-n Hermitian G with the round-robin ordering (Sec. 4.3): */
/* rotate (i,j) iff |g_ij| >= tol sqrt(g_ii) sqrt(g_jj); G <- J^H G J and      */
/* Z <- Z J from Z = I.  Returns the sweeps run; *converged = 1 iff the last   */
/* sweep rotated nothing.  The diagonal is taken as non-negative (Gram).       */
static int F(heevj_core)(int n, S_T* G, int ldg, S_T* Z, int ldz, double tol,
                         int max_sweeps, int* converged)
{
    int sweeps = 0, conv = 0;
    for (int c = 0; c < n; ++c)
        for (int r = 0; r < n; ++r) Z[r + (size_t)c * ldz] = (r == c) ? 1.0 : 0.0;
    if (n < 2) { *converged = 1; return 0; }
    int l = n + (n & 1);                          /* phantom index n if n odd */
    while (!conv && sweeps < max_sweeps) {
        conv = 1;
        sweeps++;
        for (int r = 0; r < l - 1; ++r) {
            for (int q = 0; q < l / 2; ++q) {
                int i, j;
                oracle_rr_pair(l, r, q, &i, &j);
                if (j >= n) continue;             /* phantom partner */
                double gii = REAL(G[i + (size_t)i * ldg]);
                double gjj = REAL(G[j + (size_t)j * ldg]);
                S_T gij = G[i + (size_t)j * ldg];
                if (gii <= 0.0 || gjj <= 0.0) continue;             /* R4 */
                if (!(ABSV(gij) >= tol * sqrt(gii) * sqrt(gjj))) continue;
                if (ABSV(gij) == 0.0) continue;
                conv = 0;
                double c, s;
                S_T e;
                F(rotation)(gii, gjj, gij, &c, &s, &e);
                F(rotate_cols)(G, n, ldg, i, j, c, s, e);           /* G J   */
                F(rotate_rows)(G, n, ldg, i, j, c, s, e);           /* J^H . */
                F(rotate_cols)(Z, n, ldz, i, j, c, s, e);           /* Z J   */
            }
        }
    }
    *converged = conv;
    return sweeps;
}

typedef struct {
    int m, n;        /* working shape, m >= n (R6) */
    int trans;       /* 1 if working on A^H */
    S_T* W;          /* m x n, ld m */
    S_T* V;          /* n x n, ld n */
    int ex;          /* R7: W = 2^-ex * A (or A^H) */
    int bad;         /* some input entry is not finite */
} F(work_t);

static void F(work_load)(F(work_t)* w, int m, int n, const S_T* A, int lda)
{
    w->trans = m < n;
    w->m = w->trans ? n : m;
    w->n = w->trans ? m : n;
    w->W = malloc(sizeof(S_T) * (size_t)w->m * w->n + 1);
    w->V = malloc(sizeof(S_T) * (size_t)w->n * w->n + 1);
    w->bad = 0;
    double amax = 0.0;
    for (int c = 0; c < n; ++c)
        for (int r = 0; r < m; ++r) {
            S_T a = A[r + (size_t)c * lda];
            if (!FINITE_S(a)) { w->bad = 1; continue; }
            for (int h = 0; h < NPARTS; ++h) amax = fmax(amax, fabs(PART(a, h)));
        }
    int ex = 0;
    if (amax > 0.0) { frexp(amax, &ex); ex -= 1; }   /* amax * 2^-ex in [1, 2) */
    w->ex = ex;
    for (int c = 0; c < n; ++c)
        for (int r = 0; r < m; ++r) {
            S_T x = LDEXP_S(A[r + (size_t)c * lda], -ex);
            if (w->trans) w->W[c + (size_t)r * w->m] = CONJ(x);
            else          w->W[r + (size_t)c * w->m] = x;
        }
    for (int c = 0; c < w->n; ++c)
        for (int r = 0; r < w->n; ++r) w->V[r + (size_t)c * w->n] = (r == c) ? 1.0 : 0.0;
}

/* LAPACK-style scaled 2-norm of a vector (no overflow, no underflow). */
static double F(vec_norm)(const S_T* x, int len)
{
    double scale = 0.0, ssq = 1.0;
    for (int p = 0; p < len; ++p)
        for (int h = 0; h < NPARTS; ++h) {
            double a = fabs(PART(x[p], h));
            if (a == 0.0) continue;
            if (scale < a) { ssq = 1.0 + ssq * (scale / a) * (scale / a); scale = a; }
            else           { ssq += (a / scale) * (a / scale); }
        }
    return scale * sqrt(ssq);
}

/* The end of Alg. 2: sigma_i = ||a_i||_2, U_i = a_i/sigma_i, stable sort of  */
/* sigma in descending order with U and V reordered alike; R5 for sigma = 0;  */
/* R6 swaps U and V back for A^H; R7 scales sigma back.                        */
static void F(finalize)(F(work_t)* w, double* Sg, S_T* U, int ldu, S_T* V, int ldv)
{
    int m = w->m, n = w->n;
    double* sig = malloc(sizeof(double) * (size_t)n + 1);
    int* perm = malloc(sizeof(int) * (size_t)n + 1);
    for (int k = 0; k < n; ++k) { sig[k] = F(vec_norm)(w->W + (size_t)k * m, m); perm[k] = k; }
    for (int a = 1; a < n; ++a) {                  /* stable insertion sort */
        int key = perm[a], b = a - 1;
        while (b >= 0 && sig[perm[b]] < sig[key]) { perm[b + 1] = perm[b]; --b; }
        perm[b + 1] = key;
    }
    S_T* Uw = malloc(sizeof(S_T) * (size_t)m * n + 1);
    S_T* Vw = malloc(sizeof(S_T) * (size_t)n * n + 1);
    S_T* x = malloc(sizeof(S_T) * (size_t)m + 1);
    for (int p = 0; p < n; ++p) {
        int k = perm[p];
        double sk = sig[k];
        for (int r = 0; r < n; ++r) Vw[r + (size_t)p * n] = w->V[r + (size_t)k * n];
        if (sk > 0.0) {
            for (int r = 0; r < m; ++r) Uw[r + (size_t)p * m] = w->W[r + (size_t)k * m] / sk;
            continue;
        }
        /* R5: the standard basis vector with the largest residual after one */
        /* projection off U(:, 0:p), projected twice more and normalised.     */
        int best = 0;
        double bestn = -1.0;
        for (int e = 0; e < m; ++e) {
            for (int r = 0; r < m; ++r) x[r] = (r == e) ? 1.0 : 0.0;
            for (int q = 0; q < p; ++q) {
                S_T d = CONJ(Uw[e + (size_t)q * m]);
                for (int r = 0; r < m; ++r) x[r] -= Uw[r + (size_t)q * m] * d;
            }
            double nx = F(vec_norm)(x, m);
            if (nx > bestn) { bestn = nx; best = e; }
        }
        for (int r = 0; r < m; ++r) x[r] = (r == best) ? 1.0 : 0.0;
        for (int pass = 0; pass < 2; ++pass)
            for (int q = 0; q < p; ++q) {
                S_T d = 0.0;
                for (int r = 0; r < m; ++r) d += CONJ(Uw[r + (size_t)q * m]) * x[r];
                for (int r = 0; r < m; ++r) x[r] -= Uw[r + (size_t)q * m] * d;
            }
        double nx = F(vec_norm)(x, m);
        for (int r = 0; r < m; ++r) Uw[r + (size_t)p * m] = x[r] / nx;
    }
    for (int p = 0; p < n; ++p) Sg[p] = ldexp(sig[perm[p]], w->ex);     /* R7 */
    /* R6: A^H = W = U_w Sigma V_w^H gives A = V_w Sigma U_w^H: the roles swap. */
    S_T* Uo = w->trans ? Vw : Uw;
    S_T* Vo = w->trans ? Uw : Vw;
    int urows = w->trans ? n : m, vrows = w->trans ? m : n;
    if (U) for (int p = 0; p < n; ++p) for (int r = 0; r < urows; ++r)
        U[r + (size_t)p * ldu] = Uo[r + (size_t)p * urows];
    if (V) for (int p = 0; p < n; ++p) for (int r = 0; r < vrows; ++r)
        V[r + (size_t)p * ldv] = Vo[r + (size_t)p * vrows];
    free(sig); free(perm); free(Uw); free(Vw); free(x);
}

static void F(fill_nan)(int m, int n, double* Sg, S_T* U, int ldu, S_T* V, int ldv)
{
    int k = m < n ? m : n;
    for (int p = 0; p < k; ++p) Sg[p] = NAN;
    if (U) for (int p = 0; p < k; ++p) for (int r = 0; r < m; ++r) U[r + (size_t)p * ldu] = NAN_S;
    if (V) for (int p = 0; p < k; ++p) for (int r = 0; r < n; ++r) V[r + (size_t)p * ldv] = NAN_S;
}

/* Alg. 2: unblocked one-sided Jacobi; pairs i < j in row-cyclic order. */
static int F(gesvj)(int m, int n, const S_T* A, int lda, double tol, int max_sweeps,
                    double* Sg, S_T* U, int ldu, S_T* V, int ldv, int* sweeps_out)
{
    if (sweeps_out) *sweeps_out = 0;
    if (m == 0 || n == 0) return 0;
    F(work_t) w;
    F(work_load)(&w, m, n, A, lda);
    if (w.bad) { F(fill_nan)(m, n, Sg, U, ldu, V, ldv); free(w.W); free(w.V); return -1; }
    int M = w.m, N = w.n, sweeps = 0, converged = 0;
    while (!converged && sweeps < max_sweeps) {
        converged = 1;
        sweeps++;
        for (int i = 0; i < N; ++i)
            for (int j = i + 1; j < N; ++j) {
                const S_T* wi = w.W + (size_t)i * M;
                const S_T* wj = w.W + (size_t)j * M;
                double gii = 0.0, gjj = 0.0;
                S_T gij = 0.0;
                for (int p = 0; p < M; ++p) {
                    gii += ABS2(wi[p]);
                    gjj += ABS2(wj[p]);
                    gij += CONJ(wi[p]) * wj[p];                  /* a_i^H a_j */
                }
                if (gii == 0.0 || gjj == 0.0) continue;          /* R4 */
                if (!(ABSV(gij) >= tol * sqrt(gii) * sqrt(gjj))) continue;
                if (ABSV(gij) == 0.0) continue;
                converged = 0;
                double c, s;
                S_T e;
                F(rotation)(gii, gjj, gij, &c, &s, &e);
                F(rotate_cols)(w.W, M, M, i, j, c, s, e);
                F(rotate_cols)(w.V, N, N, i, j, c, s, e);
            }
    }
    F(finalize)(&w, Sg, U, ldu, V, ldv);
    free(w.W); free(w.V);
    if (sweeps_out) *sweeps_out = sweeps;
    return converged ? 0 : sweeps;
}

/* One round r of the blocked method (Sec. 4, steps S1-S5): for each block  */
/* pair (i,j) of round r of the round-robin ordering on L blocks (blocks >= l */
/* are phantoms and skipped): P = [A_i A_j] (Eq. block-gram), G = P^H P,      */
/* inner_sweeps sweeps of Alg. 1 on G give J, then P <- P J and               */
/* [V_i V_j] <- [V_i V_j] J (Eq. right-sv).  W is M x np (ld M), Vp is np x np */
/* (ld np), np = l*nb.  Scratch P, Q, G, J.  Returns 1 if some inner rotation */
/* fired ("converged after exactly one inner sweep" is the negation).         */
static int F(blocked_round)(int M, int l, int L, int nb, int r, int inner_sweeps, double tol,
                            S_T* W, S_T* Vp, S_T* P, S_T* Q, S_T* G, S_T* J)
{
    int np = l * nb, two = 2 * nb, fired = 0;
    for (int q = 0; q < L / 2; ++q) {
        int bi, bj;
        oracle_rr_pair(L, r, q, &bi, &bj);
        if (bj >= l) continue;                                        /* phantom */
        for (int c = 0; c < two; ++c) {
            int src = (c < nb) ? bi * nb + c : bj * nb + (c - nb);
            memcpy(P + (size_t)c * M, W + (size_t)src * M, sizeof(S_T) * (size_t)M);
            if (Vp) memcpy(Q + (size_t)c * np, Vp + (size_t)src * np, sizeof(S_T) * (size_t)np);
        }
        for (int b = 0; b < two; ++b)                                 /* G = P^H P */
            for (int a = 0; a < two; ++a) {
                S_T acc = 0.0;
                for (int p = 0; p < M; ++p) acc += CONJ(P[p + (size_t)a * M]) * P[p + (size_t)b * M];
                G[a + (size_t)b * two] = acc;
            }
        int conv;
        int isw = F(heevj_core)(two, G, two, J, two, tol, inner_sweeps, &conv);
        if (!(conv && isw == 1)) fired = 1;
        for (int c = 0; c < two; ++c) {                               /* P J, Q J */
            int dst = (c < nb) ? bi * nb + c : bj * nb + (c - nb);
            for (int p = 0; p < M; ++p) {
                S_T acc = 0.0;
                for (int k = 0; k < two; ++k) acc += P[p + (size_t)k * M] * J[k + (size_t)c * two];
                W[p + (size_t)dst * M] = acc;
            }
            if (Vp)
                for (int p = 0; p < np; ++p) {
                    S_T acc = 0.0;
                    for (int k = 0; k < two; ++k) acc += Q[p + (size_t)k * np] * J[k + (size_t)c * two];
                    Vp[p + (size_t)dst * np] = acc;
                }
        }
    }
    return fired;
}

/* The blocked method (Sec. 3, Eq. block-gram and right-sv; Sec. 4 S1-S5).    */
/* n is padded with zero columns to l*nb (Sec. 3), with l >= 2 (a lone block  */
/* is paired with a zero block); l odd adds a phantom block whose pairs are   */
/* skipped.  Sweeps of l-1 (or l) rounds run until a sweep in which no inner  */
/* rotation fired.  If stop_after_rounds >= 0, only that many rounds run and  */
/* the working matrix (unscaled, m >= n orientation) is copied to Wout        */
/* instead of finalising -- the worked example of Sec. 5.1 is checked so.     */
static int F(gesvj_blocked)(int m, int n, const S_T* A, int lda, int nb, int inner_sweeps,
                            double tol, int max_sweeps, double* Sg, S_T* U, int ldu,
                            S_T* V, int ldv, int* sweeps_out, int stop_after_rounds,
                            S_T* Wout, int ldw)
{
    if (sweeps_out) *sweeps_out = 0;
    if (m == 0 || n == 0) return 0;
    F(work_t) w;
    F(work_load)(&w, m, n, A, lda);
    if (w.bad) { F(fill_nan)(m, n, Sg, U, ldu, V, ldv); free(w.W); free(w.V); return -1; }
    int M = w.m, N = w.n;
    int l = (N + nb - 1) / nb;
    if (l < 2) l = 2;
    int np = l * nb, L = l + (l & 1), two = 2 * nb;
    S_T* W = calloc((size_t)M * np + 1, sizeof(S_T));
    S_T* Vp = calloc((size_t)np * np + 1, sizeof(S_T));
    S_T* P = malloc(sizeof(S_T) * (size_t)M * two + 1);
    S_T* Q = malloc(sizeof(S_T) * (size_t)np * two + 1);
    S_T* G = malloc(sizeof(S_T) * (size_t)two * two + 1);
    S_T* J = malloc(sizeof(S_T) * (size_t)two * two + 1);
    for (int c = 0; c < N; ++c)
        for (int r = 0; r < M; ++r) W[r + (size_t)c * M] = w.W[r + (size_t)c * M];
    for (int c = 0; c < np; ++c) Vp[c + (size_t)c * np] = 1.0;
    int sweeps = 0, converged = 0, rounds = 0;
    while (!converged && sweeps < max_sweeps) {
        if (stop_after_rounds >= 0 && rounds >= stop_after_rounds) break;
        converged = 1;
        sweeps++;
        for (int r = 0; r < L - 1; ++r) {
            if (stop_after_rounds >= 0 && rounds >= stop_after_rounds) break;
            if (F(blocked_round)(M, l, L, nb, r, inner_sweeps, tol, W, Vp, P, Q, G, J)) converged = 0;
            rounds++;
        }
    }
    if (stop_after_rounds >= 0) {
        for (int c = 0; c < N; ++c)
            for (int r = 0; r < M; ++r) Wout[r + (size_t)c * ldw] = LDEXP_S(W[r + (size_t)c * M], w.ex);
    } else {
        for (int c = 0; c < N; ++c) {                                  /* trim */
            for (int r = 0; r < M; ++r) w.W[r + (size_t)c * M] = W[r + (size_t)c * M];
            for (int r = 0; r < N; ++r) w.V[r + (size_t)c * N] = Vp[r + (size_t)c * np];
        }
        F(finalize)(&w, Sg, U, ldu, V, ldv);
    }
    free(W); free(Vp); free(P); free(Q); free(G); free(J); free(w.W); free(w.V);
    if (sweeps_out) *sweeps_out = sweeps;
    return converged ? 0 : sweeps;
}
