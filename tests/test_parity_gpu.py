"""Parity of the CUDA path with the CPU oracle (needs a GB300).

Bounds (north-star), u = unit roundoff of the working precision, n = columns:
    max_k |sigma_k - sigma_oracle_k| / sigma_max <= 50 n u
    ||A - U S V^H||_F / ||A||_F <= 20 n u
    ||U^H U - I||_F, ||V^H V - I||_F <= 20 n u
U and V are never compared element-wise (sign/phase freedom, Sec. 1).
Every call goes through the C-ABI (ctypes binding).
"""
import numpy as np
import pytest
import torch

import __graft_entry__  # noqa: F401
import oracle
import paper_2601_17979_gb300 as bsvd
import synth
from oracle import checks

pytestmark = pytest.mark.gpu

TORCH = {np.float32: torch.float32, np.float64: torch.float64,
         np.complex64: torch.complex64, np.complex128: torch.complex128}


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available(), "GPU tests need CUDA"


def run_gpu(mats, **kw):
    A = torch.from_numpy(np.stack(mats)).cuda()
    r = bsvd.gesvj(A, **kw)
    torch.cuda.synchronize()
    return (r.S.cpu().numpy(), None if r.U is None else r.U.cpu().numpy(),
            None if r.V is None else r.V.cpu().numpy(), r.info.cpu().numpy(), r.sweeps.cpu().numpy())


def assert_parity(mats, S, U, V, info, ref_S, label=""):
    u = checks.unit_roundoff(mats[0].dtype)
    for i, A in enumerate(mats):
        assert info[i] == 0, f"{label} matrix {i}: info {info[i]}"
        meas = checks.measures(A, S[i], None if U is None else U[i], None if V is None else V[i], ref_S[i])
        bad = checks.violations(meas, u)
        assert not bad, f"{label} matrix {i}: {bad} {meas}"


def random_mats(rng, count, m, n, dtype):
    if np.issubdtype(dtype, np.complexfloating):
        return [(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))).astype(dtype) for _ in range(count)]
    return [rng.standard_normal((m, n)).astype(dtype) for _ in range(count)]


@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.complex128, np.complex64])
@pytest.mark.parametrize("m,n,nb", [(32, 32, 8), (40, 24, 8), (33, 19, 4), (24, 40, 8),
                                    (7, 3, 4), (3, 7, 4), (64, 64, 16), (100, 50, 16),
                                    (17, 17, 16), (1, 1, 4), (9, 1, 4), (1, 9, 4), (72, 72, 8)])
def test_random_shapes(dtype, m, n, nb):
    rng = np.random.default_rng(m * 1000 + n * 10 + nb)
    mats = random_mats(rng, 6, m, n, dtype)
    S, U, V, info, sw = run_gpu(mats, nb=nb)
    ref = oracle.gesvj(mats)
    assert_parity(mats, S, U, V, info, ref["S"], f"{dtype.__name__} {m}x{n} nb{nb}")


@pytest.mark.parametrize("name,count,k,nb", [("square32_f64", 64, 32, 8), ("tall128x64_f64", 24, 30, 16),
                                             ("tall128x64_f32", 24, 30, 16)])
def test_workload_samples(name, count, k, nb):
    mats = synth.matrices(name, range(count))
    u = checks.unit_roundoff(mats[0].dtype)
    S, U, V, info, sw = run_gpu(mats, nb=nb, tol=k * u)
    ref = oracle.gesvj(mats, tol=k * 2.0 ** -53)
    assert_parity(mats, S, U, V, info, ref["S"], name)


def test_mixed96_real_samples():
    mats = [synth.matrix("mixed96", i) for i in range(0, 16, 2)]   # the real half
    S, U, V, info, sw = run_gpu(mats, nb=16)
    ref = oracle.gesvj(mats, tol=30 * 2.0 ** -53)
    assert_parity(mats, S, U, V, info, ref["S"], "mixed96 real")


def test_full_size_tall128x64_sampled():
    """The full 10,000-matrix FP64 batch in the benchmark's launch
    configuration; sampled matrices checked against the oracle."""
    A = synth.uniform_batch("tall128x64_f64")
    At = torch.from_numpy(A).cuda()
    r = bsvd.gesvj(At, nb=16)
    torch.cuda.synchronize()
    info = r.info.cpu().numpy()
    assert (info == 0).all(), np.unique(info, return_counts=True)
    idx = np.random.default_rng(0).choice(len(A), 12, replace=False)
    mats = [A[i] for i in idx]
    ref = oracle.gesvj(mats, tol=30 * 2.0 ** -53)
    S, U, V = r.S.cpu().numpy()[idx], r.U.cpu().numpy()[idx], r.V.cpu().numpy()[idx]
    assert_parity(mats, S, U, V, info[idx], ref["S"], "full tall128x64")
    # every matrix: sigma sorted, Frobenius invariant sum sigma^2 = ||A||_F^2
    Sall = r.S.cpu().numpy()
    assert np.all(Sall[:, :-1] >= Sall[:, 1:])
    fro = np.linalg.norm(A, axis=(1, 2)) ** 2
    assert np.max(np.abs((Sall ** 2).sum(1) - fro) / fro) <= 20 * 64 * 2.0 ** -53


def test_jobs_none_and_sigma_only():
    rng = np.random.default_rng(1)
    mats = random_mats(rng, 4, 30, 20, np.float64)
    ref = oracle.gesvj(mats)
    for cu, cv in [(False, False), (True, False), (False, True)]:
        S, U, V, info, _ = run_gpu(mats, compute_u=cu, compute_v=cv, nb=8)
        assert (U is None) == (not cu) and (V is None) == (not cv)
        assert_parity(mats, S, U, V, info, ref["S"], f"jobs {cu}{cv}")
    # wide matrices exercise the A^H path with the roles of U and V swapped
    wide = [m.T.copy() for m in mats]
    for cu, cv in [(False, True), (True, False)]:
        S, U, V, info, _ = run_gpu(wide, compute_u=cu, compute_v=cv, nb=8)
        assert_parity(wide, S, U, V, info, ref["S"], f"wide jobs {cu}{cv}")


def test_diagonal_exact_and_zero():
    d = np.array([3.0, -7.5, 0.25, 11.0, -0.5, 2.0, 9.0, -1.0])
    mats = [np.diag(d), np.zeros((8, 8)), np.diag(d)[:, ::-1].copy()]
    S, U, V, info, sw = run_gpu(mats, nb=4)
    assert np.array_equal(S[0], np.sort(np.abs(d))[::-1])
    assert np.array_equal(S[2], np.sort(np.abs(d))[::-1])
    assert np.array_equal(S[1], np.zeros(8))
    for i in range(3):
        assert info[i] == 0
        meas = checks.measures(mats[i], S[i], U[i], V[i])
        assert checks.violations(meas, checks.U64) == [], (i, meas)


def test_rank_deficient():
    rng = np.random.default_rng(5)
    B = rng.standard_normal((20, 12))
    B[:, 3] = 0.0
    B[:, 7] = 0.0
    C = rng.standard_normal((20, 4)) @ rng.standard_normal((4, 12))    # rank 4
    mats = [B, C]
    S, U, V, info, sw = run_gpu(mats, nb=4)
    ref = oracle.gesvj(mats)
    assert_parity(mats, S, U, V, info, ref["S"], "rank deficient")


def test_nonfinite_and_max_sweeps():
    rng = np.random.default_rng(6)
    mats = random_mats(rng, 3, 16, 16, np.float64)
    mats[1][4, 5] = np.nan
    mats[2][0, 0] = np.inf
    S, U, V, info, sw = run_gpu(mats, nb=4)
    assert info[0] == 0 and info[1] == -1 and info[2] == -1
    assert np.isnan(S[1]).all() and np.isnan(U[2]).all()
    S, U, V, info, sw = run_gpu(mats[:1], nb=4, max_sweeps=1)
    assert info[0] == 1 and sw[0] == 1


def test_scaling_extremes():
    rng = np.random.default_rng(7)
    base = rng.standard_normal((24, 16))
    mats = [np.ldexp(base, e) for e in (-900, -300, 0, 300, 900)]
    S, U, V, info, sw = run_gpu(mats, nb=8)
    for i, e in enumerate((-900, -300, 0, 300, 900)):
        assert np.array_equal(S[i], np.ldexp(S[2], e))     # exact power-of-two scaling
        assert info[i] == 0


def test_pointer_array_mixed_shapes():
    rng = np.random.default_rng(8)
    shapes = [(32, 32), (40, 24), (24, 40), (64, 64), (40, 24), (5, 3), (0, 4), (17, 9)]
    for dtype in (np.float64, np.complex64):
        mats = [random_mats(rng, 1, m, n, dtype)[0] for m, n in shapes]
        T = [torch.from_numpy(x).cuda() for x in mats]
        r = bsvd.gesvj_batched(T, nb=8)
        info = r.info.cpu().numpy()
        nonempty = [i for i, (m, n) in enumerate(shapes) if min(m, n) > 0]
        ref = oracle.gesvj([mats[i] for i in nonempty])
        assert (info == 0).all()
        for j, i in enumerate(nonempty):
            meas = checks.measures(mats[i], r.S[i].cpu().numpy(), r.U[i].cpu().numpy(),
                                   r.V[i].cpu().numpy(), ref["S"][j])
            assert checks.violations(meas, checks.unit_roundoff(dtype)) == [], (i, meas)


def test_results_independent_of_batch_neighbours():
    """A matrix's result is bitwise the same alone and inside a batch."""
    mats = synth.matrices("tall128x64_f64", range(6))
    S_all, U_all, V_all, _, sw_all = run_gpu(mats, nb=16)
    S_one, U_one, V_one, _, sw_one = run_gpu(mats[3:4], nb=16)
    assert np.array_equal(S_all[3], S_one[0])
    assert np.array_equal(U_all[3], U_one[0]) and np.array_equal(V_all[3], V_one[0])


def test_blocked_oracle_sweep_counts_close():
    """Same algorithm on both sides: sweep counts of the blocked oracle (one
    inner sweep, same tolerance) and of the kernel agree within one sweep on
    most matrices (rounding differs, so exact equality is not required)."""
    mats = synth.matrices("square32_f64", range(32))
    tol = 32 * 2.0 ** -53
    _, _, _, info, sw = run_gpu(mats, nb=8, tol=tol)
    ref = oracle.gesvj(mats, nb=8, inner_sweeps=1, tol=tol)
    diff = np.abs(sw - ref["sweeps"])
    assert (diff <= 1).mean() >= 0.9, (sw, ref["sweeps"])


F32_VARIANTS = {"tensor_cores": 0, "ffma_tiles": bsvd.FLAG_F32_FFMA, "fp64_angles": bsvd.FLAG_WIDE_ANGLES,
                "ffma_fp64_angles": bsvd.FLAG_F32_FFMA | bsvd.FLAG_WIDE_ANGLES}


@pytest.mark.parametrize("variant", sorted(F32_VARIANTS))
@pytest.mark.parametrize("m,n,nb", [(128, 64, 16), (100, 72, 16), (72, 100, 16), (45, 37, 8), (130, 64, 16),
                                    (33, 19, 4)])
def test_fp32_gram_and_update_variants(variant, m, n, nb):
    """Real FP32 with the Gram blocks and rotation updates on the tensor cores
    (split TF32; the default for nb = 8, 16), on the FMA register tiles, and
    with the rotations and pair test in FP64: each meets the FP32 bounds
    against the FP64 oracle.  Shapes with ragged 16-row tiles included."""
    rng = np.random.default_rng(m * 31 + n + nb)
    mats = random_mats(rng, 6, m, n, np.float32)
    S, U, V, info, sw = run_gpu(mats, nb=nb, flags=F32_VARIANTS[variant])
    ref = oracle.gesvj(mats)
    assert_parity(mats, S, U, V, info, ref["S"], f"{variant} {m}x{n} nb{nb}")


@pytest.mark.parametrize("variant", ["tensor_cores", "ffma_tiles", "fp64_angles"])
def test_fp32_variants_tall128x64_workload(variant):
    mats = synth.matrices("tall128x64_f32", range(24))
    S, U, V, info, sw = run_gpu(mats, nb=16, tol=30 * 2.0 ** -24, flags=F32_VARIANTS[variant])
    ref = oracle.gesvj(mats, tol=30 * 2.0 ** -53)
    assert_parity(mats, S, U, V, info, ref["S"], variant)


def test_complex64_fp64_angles():
    rng = np.random.default_rng(77)
    mats = random_mats(rng, 4, 60, 44, np.complex64)
    S, U, V, info, sw = run_gpu(mats, nb=8, flags=bsvd.FLAG_WIDE_ANGLES)
    ref = oracle.gesvj(mats)
    assert_parity(mats, S, U, V, info, ref["S"], "c64 fp64 angles")
