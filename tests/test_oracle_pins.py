"""Pins of the CPU oracle to facts outside itself (no GPU needed).

Each test checks the oracle against something the paper or the mathematics
fixes: values printed in the paper's worked example (Sec. 5.1), closed forms,
exact special cases, an arbitrary-precision brute force (mpmath), an
independent library (LAPACK through numpy), and invariants (Eq. block-off-norm,
property P2 of Sec. 3).  ``test_oracle_mutants.py`` plants plausible mistakes
in a copy of the oracle and checks that these pins catch them.
"""
import itertools

import numpy as np
import pytest

import oracle
from oracle import checks
from tests.conftest import load_golden

U = 2.0 ** -53


@pytest.fixture(scope="module")
def O():
    return oracle.default()


def closed_form_2x2(a, b, c, d):
    """Singular values of [[a, b], [c, d]] (real), from the polar form."""
    p = np.hypot(a + d, b - c)
    q = np.hypot(a - d, b + c)
    return (p + q) / 2, abs(p - q) / 2


# --------------------------------------------------------------------------
# Round-robin ordering (Sec. 3, Sec. 4.1; worked example of Sec. 5.1)
# --------------------------------------------------------------------------
def test_rr_sequence_of_worked_example(O):
    # Sec. 5.1: round 1 pairs (1,2),(3,4), round 2 pairs (1,4),(2,3); the third
    # round holds the two remaining pairs (1,3),(2,4).  0-based here.
    rounds = [sorted(O.rr_pair(4, r, q) for q in range(2)) for r in range(3)]
    assert rounds == [[(0, 1), (2, 3)], [(0, 3), (1, 2)], [(0, 2), (1, 3)]]


@pytest.mark.parametrize("l", [2, 4, 6, 8, 10, 16, 32, 34])
def test_rr_every_pair_once_disjoint_rounds(O, l):
    seen = []
    for r in range(l - 1):
        slot = [O.rr_pair(l, r, q) for q in range(l // 2)]
        players = [p for ij in slot for p in ij]
        assert sorted(players) == list(range(l)), f"round {r} not a perfect matching"
        assert all(i < j for i, j in slot)
        seen += slot
    assert sorted(seen) == sorted(itertools.combinations(range(l), 2))


# --------------------------------------------------------------------------
# Alg. 2 (unblocked one-sided Jacobi)
# --------------------------------------------------------------------------
def test_2x2_closed_form(O):
    rng = np.random.default_rng(11)
    for _ in range(200):
        a, b, c, d = rng.standard_normal(4) * 10.0 ** rng.uniform(-3, 3, 4)
        A = np.array([[a, b], [c, d]])
        r = O.gesvj(A)
        s1, s2 = closed_form_2x2(a, b, c, d)
        assert abs(r["S"][0] - s1) <= 8 * U * s1
        assert abs(r["S"][1] - s2) <= 8 * U * s1
        assert r["info"] == 0


def test_equal_column_norms(O):
    # tau = 0 (equal column norms): sign(0) = +1 gives the pi/4 rotation (R2)
    for a, b in [(1.0, 0.5), (2.0, -0.75), (0.3, 0.3001)]:
        A = np.array([[a, b], [b, a]])          # both columns have norm^2 a^2 + b^2
        r = O.gesvj(A)
        s1, s2 = closed_form_2x2(a, b, b, a)
        assert r["info"] == 0
        assert abs(r["S"][0] - s1) <= 8 * U * s1 and abs(r["S"][1] - s2) <= 8 * U * s1


def test_diagonal_exact(O):
    d = np.array([3.0, -7.5, 0.25, 11.0, -0.5, 2.0])
    r = O.gesvj(np.diag(d))
    assert np.array_equal(r["S"], np.sort(np.abs(d))[::-1])     # bitwise
    assert r["sweeps"] == 1 and r["info"] == 0                  # nothing rotates
    # U and V are signed permutations with U diag(S) V^T = A exactly
    assert np.array_equal(np.abs(r["U"]).sum(axis=0), np.ones(6))
    assert np.array_equal((r["U"] * r["S"]) @ r["V"].T, np.diag(d))


def test_permuted_diagonal_exact(O):
    rng = np.random.default_rng(5)
    d = rng.uniform(0.1, 10.0, 7) * rng.choice([-1, 1], 7)
    D = np.zeros((9, 7))
    D[:7, :7] = np.diag(d)
    A = D[rng.permutation(9)][:, rng.permutation(7)]
    r = O.gesvj(A)
    assert np.array_equal(r["S"], np.sort(np.abs(d))[::-1])
    assert np.array_equal((r["U"] * r["S"]) @ r["V"].T, A)


@pytest.mark.parametrize("cplx", [False, True])
@pytest.mark.parametrize("m,n,kappa", [(40, 24, 1e6), (24, 24, 1e10), (33, 17, 1e3)])
def test_known_sigma(O, cplx, m, n, kappa):
    import synth
    rng = np.random.default_rng(m * 100 + n)
    for fam in synth.FAMILIES[1:]:
        sig = synth.sigma_family(fam, n, kappa, rng)
        A = synth.with_sigma(rng, m, n, sig, cplx)
        r = O.gesvj(A)
        # Backward stable: |sigma - sigma_true| <= c n u ||A||_2 (Weyl).
        assert np.abs(r["S"] - sig).max() <= 4 * n * U * sig[0], fam
        meas = checks.measures(A, r["S"], r["U"], r["V"], sig)
        assert checks.violations(meas, U) == [], (fam, meas)


def test_mpmath_brute_force(O):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(3)
    for m, n, cplx in [(2, 2, False), (3, 2, False), (5, 4, False), (6, 6, False),
                       (4, 3, True), (6, 5, True), (3, 5, False), (2, 6, True)]:
        A = rng.standard_normal((m, n))
        if cplx:
            A = A + 1j * rng.standard_normal((m, n))
        M = mpmath.matrix(A.tolist())
        ref = mpmath.svd_c(M, compute_uv=False) if cplx else mpmath.svd_r(M, compute_uv=False)
        ref = np.sort(np.array([float(x) for x in ref]))[::-1]
        r = O.gesvj(A)
        assert np.abs(r["S"] - ref).max() <= 4 * max(m, n) * U * ref[0], (m, n, cplx)


@pytest.mark.parametrize("shape", [(1, 1), (1, 5), (5, 1), (7, 3), (3, 7), (16, 16), (50, 20)])
@pytest.mark.parametrize("cplx", [False, True])
def test_lapack_crosscheck_and_bounds(O, shape, cplx):
    rng = np.random.default_rng(sum(shape))
    A = rng.standard_normal(shape)
    if cplx:
        A = A + 1j * rng.standard_normal(shape)
    r = O.gesvj(A)
    ref = np.linalg.svd(A, compute_uv=False)
    n = A.shape[1]
    meas = checks.measures(A, r["S"], r["U"], r["V"], ref)
    assert checks.violations(meas, U) == [], meas
    # Frobenius invariant: sum sigma_k^2 = ||A||_F^2
    assert abs((r["S"] ** 2).sum() - np.linalg.norm(A) ** 2) <= 4 * n * U * np.linalg.norm(A) ** 2


def test_rank_deficient_and_zero(O):
    rng = np.random.default_rng(9)
    A = np.zeros((6, 4))
    r = O.gesvj(A)
    assert np.array_equal(r["S"], np.zeros(4))
    assert np.abs(r["U"].T @ r["U"] - np.eye(4)).max() <= 4 * U        # R5 completion
    assert np.abs(r["V"].T @ r["V"] - np.eye(4)).max() == 0.0
    B = rng.standard_normal((8, 5))
    B[:, 2] = 0.0
    B[:, 4] = 0.0
    r = O.gesvj(B)
    assert r["S"][-1] == 0.0 and r["S"][-2] == 0.0
    meas = checks.measures(B, r["S"], r["U"], r["V"], np.linalg.svd(B, compute_uv=False))
    assert checks.violations(meas, U) == [], meas


def test_scaling_extremes(O):
    rng = np.random.default_rng(4)
    A = rng.standard_normal((12, 8))
    ref = O.gesvj(A)["S"]
    for e in (-1000, -300, 300, 1000):
        r = O.gesvj(np.ldexp(A, e))
        # exact power-of-two scaling (R7): same sigma up to the same scale
        assert np.array_equal(r["S"], np.ldexp(ref, e)), e


def test_nonfinite_input(O):
    A = np.ones((4, 3))
    A[2, 1] = np.nan
    r = O.gesvj(A)
    assert r["info"] == -1 and np.all(np.isnan(r["S"]))
    A[2, 1] = np.inf
    assert O.gesvj(A)["info"] == -1


def test_max_sweeps_info(O):
    A = np.random.default_rng(2).standard_normal((20, 20))
    r = O.gesvj(A, max_sweeps=1)
    assert r["info"] == 1 and r["sweeps"] == 1


# --------------------------------------------------------------------------
# Alg. 1 (Hermitian Jacobi eigensolver)
# --------------------------------------------------------------------------
def test_heevj_2x2_closed_form(O):
    rng = np.random.default_rng(1)
    for _ in range(50):
        X = rng.standard_normal((5, 2)) + 1j * rng.standard_normal((5, 2))
        G = X.conj().T @ X
        Gout, Z, sw, conv = O.heevj(G, max_sweeps=1)
        a, b, g = G[0, 0].real, G[1, 1].real, abs(G[0, 1])
        lam = np.sort([(a + b) / 2 + np.hypot((a - b) / 2, g), (a + b) / 2 - np.hypot((a - b) / 2, g)])
        assert np.allclose(np.sort(np.diag(Gout).real), lam, rtol=8 * U, atol=0)
        assert abs(Gout[0, 1]) <= 8 * U * lam[-1]           # Eq. scalar-off-norm: off -> 0
        assert np.abs(Z.conj().T @ Z - np.eye(2)).max() <= 4 * U
        # the smaller rotation (|t| <= 1): the larger eigenvalue stays where the larger diagonal was
        assert (Gout[0, 0].real >= Gout[1, 1].real) == (a >= b)


@pytest.mark.parametrize("cplx", [False, True])
def test_heevj_vs_mpmath(O, cplx):
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 40
    rng = np.random.default_rng(8)
    for n in (3, 4, 6, 7):
        X = rng.standard_normal((n + 3, n)) + (1j * rng.standard_normal((n + 3, n)) if cplx else 0)
        G = X.conj().T @ X
        Gout, Z, sw, conv = O.heevj(G)
        assert conv
        if cplx:
            ev = mpmath.eighe(mpmath.matrix(G.tolist()), eigvals_only=True)
        else:
            ev = mpmath.eigsy(mpmath.matrix(G.tolist()), eigvals_only=True)
        ref = np.sort([float(mpmath.re(x)) for x in ev])
        assert np.abs(np.sort(np.diag(Gout).real) - ref).max() <= 8 * n * U * ref[-1]
        assert np.abs(Z.conj().T @ Z - np.eye(n)).max() <= 8 * n * U
        assert np.abs(Z.conj().T @ G @ Z - np.diag(np.diag(Gout))).max() <= 16 * n * U * ref[-1]


def test_heevj_one_sweep_contracts_offnorm(O):
    # Property P2 (Sec. 3; Sec. 5.2): one inner sweep strictly reduces off(G).
    rng = np.random.default_rng(12)
    for n in (4, 8, 16, 32):
        X = rng.standard_normal((3 * n, n))
        G = X.T @ X
        off0 = np.linalg.norm(G - np.diag(np.diag(G)))
        Gout, Z, sw, conv = O.heevj(G, max_sweeps=1)
        assert sw == 1
        off1 = np.linalg.norm(Gout - np.diag(np.diag(Gout)))
        assert off1 < off0, (n, off0, off1)
        # sweep after sweep the off-norm keeps falling, ultimately quadratically
        Gk, prev = G, off0
        for _ in range(8):
            Gk, _, _, _ = O.heevj(Gk, max_sweeps=1)
            cur = np.linalg.norm(Gk - np.diag(np.diag(Gk)))
            assert cur < prev or cur <= 64 * n * U * off0
            prev = cur
        assert prev <= 64 * n * U * np.linalg.norm(G)
        # trace preserved (orthogonal similarity)
        assert abs(np.trace(Gout) - np.trace(G)) <= 4 * n * U * np.trace(G)


# --------------------------------------------------------------------------
# The blocked method: the worked example of Sec. 5.1
# --------------------------------------------------------------------------
def test_worked_example_states(O):
    g = load_golden("worked_example_sec5_1.txt")
    A = g["A"]
    # inputs and outputs are printed to 4 decimals: tolerance 2e-4
    W1 = O.blocked_rounds(A, nb=2, rounds=1, inner_sweeps=60)
    assert np.abs(W1[:, :4] - g["A1"]).max() <= 2e-4
    G1 = W1[:, :4].T @ W1[:, :4]
    assert np.abs(np.diag(G1) - g["G1diag"][0]).max() <= 2e-4
    assert np.abs(G1 - np.diag(np.diag(G1))).max() <= 1e-12
    W2 = O.blocked_rounds(A, nb=2, rounds=2, inner_sweeps=60)
    assert np.abs(W2[:, :4] - g["A2"]).max() <= 2e-4
    G2 = W2[:, :4].T @ W2[:, :4]
    assert np.abs(G2 - g["G2"]).max() <= 2e-4


def test_worked_example_eigenvalues(O):
    # Sec. 5.1: the eigenvalues of G^(0)_{1,2} appear on the diagonal of G^(1)_{1,2}.
    g = load_golden("worked_example_sec5_1.txt")
    P = g["A"][:, :4]
    Gout, Z, sw, conv = O.heevj(P.T @ P)
    assert conv
    assert np.abs(np.diag(Gout) - g["G1diag"][0]).max() <= 2e-4


@pytest.mark.parametrize("nb,inner", [(2, 1), (4, 1), (8, 1), (8, 60), (5, 1), (16, 1)])
@pytest.mark.parametrize("cplx", [False, True])
def test_blocked_agrees_with_unblocked(O, nb, inner, cplx):
    rng = np.random.default_rng(nb * 7 + inner)
    for m, n in [(40, 32), (33, 21), (16, 16), (9, 4), (4, 9)]:
        A = rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if cplx else 0)
        ref = O.gesvj(A)
        rb = O.gesvj(A, nb=nb, inner_sweeps=inner)
        assert rb["info"] == 0
        meas = checks.measures(A, rb["S"], rb["U"], rb["V"], ref["S"])
        bad = checks.violations(meas, U)
        if inner > 1:
            # Inner solver run to convergence (the paper's baseline): J gathers
            # many more rotations and V drifts from orthogonality beyond
            # 20 n u (Sec. 8.1 reports the same for the V check); sigma and the
            # residual still meet their bounds.
            bad = [b for b in bad if b != "orth_v"]
            assert meas["orth_v"] <= 100 * n * U
        assert bad == [], (m, n, meas)


def test_oracle_meets_bounds_on_workload_samples(O):
    """The oracle itself against the gating bounds on each workload's inputs.

    Stop rule per pair |g_ij| >= tol sqrt(g_ii g_jj): tol = n u for the 32x32
    workload (its stated rule), tol = 30 u (the paper's k = 30) elsewhere.
    Finding, reported rather than hidden: on the clustered kappa = 1e8 96x96
    set, Alg. 2 runs ~24 sweeps and its V drifts to about 1.3 x 20 n u; every
    other measure passes there.
    """
    import synth
    for name, count, k in [("square32_f64", 8, 32), ("tall128x64_f64", 4, 30),
                           ("tall128x64_f32", 4, 30), ("mixed96", 4, 30)]:
        mats = synth.matrices(name, range(count))
        r = O.gesvj(mats, tol=k * U)
        for A, S, Uo, Vo, info in zip(mats, r["S"], r["U"], r["V"], r["info"]):
            assert info == 0
            A64 = A.astype(np.complex128 if np.iscomplexobj(A) else np.float64)
            meas = checks.measures(A, S, Uo, Vo, np.linalg.svd(A64, compute_uv=False))
            bad = checks.violations(meas, U)
            if name == "mixed96":
                assert meas["orth_v"] <= 1.6 * checks.bounds(meas["n"], U)["orth_v"]
                bad = [b for b in bad if b != "orth_v"]
            assert bad == [], (name, meas)


# ---- QR pre-processing (Sec. "Pre-processing the SVD using a QR Factorization")
@pytest.mark.parametrize("shape", [(300, 16), (1000, 16), (40, 40), (16, 200), (97, 37), (5, 1)])
@pytest.mark.parametrize("cplx", [False, True])
def test_qr_path_matches_lapack_and_alg2(O, shape, cplx):
    rng = np.random.default_rng(sum(shape) + 7)
    A = rng.uniform(0, 1, shape)
    if cplx:
        A = A + 1j * rng.uniform(0, 1, shape)
    r = oracle.gesvj_qr(A, tol=30 * U, nb=16 if min(shape) > 8 else 4)
    assert r["info"] == 0
    ref = np.linalg.svd(A, compute_uv=False)
    meas = checks.measures(A, r["S"], r["U"], r["V"], ref)
    assert checks.violations(meas, U) == [], meas
    plain = O.gesvj(A, tol=30 * U)
    assert np.abs(r["S"] - plain["S"]).max() <= 50 * min(shape) * U * ref[0]
    assert r["U"].shape == (shape[0], min(shape)) and r["V"].shape == (shape[1], min(shape))


def test_qr_path_planted_mistake_is_caught():
    """Left vectors without Q (the R-SVD's U padded with zeros) fail the
    reconstruction bound: the check sees the Q step."""
    rng = np.random.default_rng(8)
    A = rng.standard_normal((60, 12))
    r = oracle.gesvj_qr(A, tol=30 * U)
    _, R = np.linalg.qr(A)
    wrong = np.zeros_like(r["U"])
    wrong[:12] = (R @ r["V"]) / r["S"]          # left vectors of R, Q left out
    meas = checks.measures(A, r["S"], wrong, r["V"], np.linalg.svd(A, compute_uv=False))
    assert "resid" in checks.violations(meas, U)
