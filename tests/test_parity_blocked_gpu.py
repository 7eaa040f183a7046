"""Parity of the multi-kernel paths (needs a GB300): the paper's baseline
(PLAIN: inner solver to convergence, two-stage update, no masks), the design
ladder of Sec. 5-7 (Design-2, -3, -4) and the BLOCKED path that serves
matrices too large for shared memory.  Bounds as in test_parity_gpu."""
import numpy as np
import pytest
import torch

import __graft_entry__  # noqa: F401
import oracle
import paper_2601_17979_gb300 as bsvd
import synth
from oracle import checks

pytestmark = pytest.mark.gpu

LADDER = {
    "baseline": dict(path="plain"),
    "design2": dict(path="plain", inner_sweeps=1),
    "design3": dict(path="blocked", flags=bsvd.FLAG_NO_MASKS),
    "design4": dict(path="blocked"),
}


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def run_gpu(mats, **kw):
    A = torch.from_numpy(np.stack(mats)).cuda()
    r = bsvd.gesvj(A, **kw)
    torch.cuda.synchronize()
    return (r.S.cpu().numpy(), None if r.U is None else r.U.cpu().numpy(),
            None if r.V is None else r.V.cpu().numpy(), r.info.cpu().numpy(), r.sweeps.cpu().numpy())


def check(mats, S, U, V, info, ref_S, label):
    u = checks.unit_roundoff(mats[0].dtype)
    for i, A in enumerate(mats):
        assert info[i] == 0, f"{label} {i}: info {info[i]}"
        meas = checks.measures(A, S[i], None if U is None else U[i], None if V is None else V[i], ref_S[i])
        bad = checks.violations(meas, u)
        assert not bad, f"{label} {i}: {bad} {meas}"


@pytest.mark.parametrize("variant", sorted(LADDER))
def test_design_ladder_tall128x64(variant):
    mats = synth.matrices("tall128x64_f64", range(12))
    S, U, V, info, sw = run_gpu(mats, nb=16, **LADDER[variant])
    ref = oracle.gesvj(mats, tol=30 * 2.0 ** -53)
    check(mats, S, U, V, info, ref["S"], variant)


@pytest.mark.parametrize("variant", sorted(LADDER))
def test_design_ladder_square32(variant):
    mats = synth.matrices("square32_f64", range(16))
    tol = 32 * 2.0 ** -53
    S, U, V, info, sw = run_gpu(mats, nb=8, tol=tol, **LADDER[variant])
    ref = oracle.gesvj(mats, tol=tol)
    check(mats, S, U, V, info, ref["S"], variant)


def test_blocked_equals_fused_bitwise_fp64():
    """Same algorithm, same summation order: Design-4 on the multi-kernel path
    gives the same bits as the on-chip kernel for real FP64 data (the inner
    solver's roundings are fixed by explicit FMAs, so inlining it into
    different kernels cannot change them)."""
    rng = np.random.default_rng(3)
    mats = [rng.standard_normal((80, 48)) for _ in range(5)]
    S1, U1, V1, i1, w1 = run_gpu(mats, nb=8, path="fused")
    S2, U2, V2, i2, w2 = run_gpu(mats, nb=8, path="blocked")
    assert np.array_equal(w1, w2)
    assert np.array_equal(S1, S2) and np.array_equal(U1, U2) and np.array_equal(V1, V2)


@pytest.mark.parametrize("m,n,flags", [(100, 72, 0), (72, 100, 0), (100, 72, bsvd.FLAG_NO_V_CORRECTION)])
def test_blocked_equals_fused_bitwise_fp64_tiled_finalisation(m, n, flags):
    """The multi-kernel path forms V's Newton-Schulz step in 64 x 64 output
    tiles; with k = 72 that is two tiles and a ragged tail per side, and the
    bits still match the on-chip finalisation (one accumulator per output,
    contraction index in increasing order).  m < n puts the step on U."""
    rng = np.random.default_rng(m * n + flags)
    mats = [rng.standard_normal((m, n)) for _ in range(4)]
    S1, U1, V1, i1, w1 = run_gpu(mats, nb=8, path="fused", flags=flags)
    S2, U2, V2, i2, w2 = run_gpu(mats, nb=8, path="blocked", flags=flags)
    assert (i1 == 0).all() and np.array_equal(w1, w2)
    assert np.array_equal(S1, S2) and np.array_equal(U1, U2) and np.array_equal(V1, V2)


def test_blocked_and_fused_agree_fp32():
    """FP32: the on-chip kernel sums its register-tiled Gram in another order,
    so the two paths agree to the bounds, not bitwise."""
    rng = np.random.default_rng(3)
    mats = [rng.standard_normal((80, 48)).astype(np.float32) for _ in range(5)]
    S1, U1, V1, i1, _ = run_gpu(mats, nb=8, path="fused")
    S2, U2, V2, i2, _ = run_gpu(mats, nb=8, path="blocked")
    ref = oracle.gesvj(mats)
    check(mats, S1, U1, V1, i1, ref["S"], "fused fp32")
    check(mats, S2, U2, V2, i2, ref["S"], "blocked fp32")
    assert np.abs(S1 - S2).max() <= 50 * 48 * 2.0 ** -24 * S1.max()


@pytest.mark.parametrize("dtype", [np.float64, np.float32, np.complex128, np.complex64])
@pytest.mark.parametrize("m,n,nb", [(200, 150, 16), (150, 260, 16), (257, 33, 8), (130, 130, 32),
                                    (64, 64, 32), (300, 5, 4), (140, 136, 16)])
def test_large_shapes_blocked(dtype, m, n, nb):
    rng = np.random.default_rng(m + n + nb)
    if np.issubdtype(dtype, np.complexfloating):
        mats = [(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))).astype(dtype) for _ in range(3)]
    else:
        mats = [rng.standard_normal((m, n)).astype(dtype) for _ in range(3)]
    S, U, V, info, sw = run_gpu(mats, nb=nb)             # AUTO: blocked when it does not fit
    ref = oracle.gesvj(mats)
    check(mats, S, U, V, info, ref["S"], f"{dtype.__name__} {m}x{n}")


def test_mixed96_complex_samples():
    """The complex half of the 96x96 clustered workload does not fit on chip."""
    mats = [synth.matrix("mixed96", i) for i in range(1, 12, 2)]
    assert mats[0].dtype == np.complex128
    S, U, V, info, sw = run_gpu(mats, nb=16)
    ref = oracle.gesvj(mats, tol=30 * 2.0 ** -53)
    check(mats, S, U, V, info, ref["S"], "mixed96 complex")


def test_uneven_pointer_array_sample():
    mats = synth.matrices("uneven", range(12))       # m in [8, 512], half complex64
    for cplx in (False, True):
        sub = [x for x in mats if np.iscomplexobj(x) == cplx]
        T = [torch.from_numpy(x).cuda() for x in sub]
        r = bsvd.gesvj_batched(T)
        info = r.info.cpu().numpy()
        ref = oracle.gesvj(sub)
        assert (info == 0).all(), info
        for i, A in enumerate(sub):
            meas = checks.measures(A, r.S[i].cpu().numpy(), r.U[i].cpu().numpy(), r.V[i].cpu().numpy(),
                                   ref["S"][i])
            assert checks.violations(meas, checks.U32) == [], (i, A.shape, meas)


def test_plain_nonfinite_and_jobs():
    rng = np.random.default_rng(4)
    mats = [rng.standard_normal((40, 30)) for _ in range(3)]
    mats[1][3, 3] = np.nan
    S, U, V, info, sw = run_gpu(mats, nb=8, path="plain")
    assert info[1] == -1 and np.isnan(S[1]).all()
    assert info[0] == 0 and info[2] == 0
    ref = oracle.gesvj([mats[0], mats[2]])
    check([mats[0], mats[2]], S[[0, 2]], U[[0, 2]], V[[0, 2]], info[[0, 2]], ref["S"], "plain")
    S2, U2, V2, info2, _ = run_gpu([mats[0]], nb=8, path="blocked", compute_u=False)
    assert U2 is None and info2[0] == 0
    check([mats[0]], S2, None, V2, info2, [ref["S"][0]], "blocked jobu=N")


def test_caller_workspace_too_small_is_reported():
    mats = [np.random.default_rng(5).standard_normal((300, 200))]
    A = torch.from_numpy(np.stack(mats)).cuda()
    work = torch.empty(64, dtype=torch.uint8, device="cuda")
    with pytest.raises(bsvd.BsvdError, match="WORKSPACE"):
        bsvd.gesvj(A, work=work)


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_host_convergence_check_gives_same_bits(dtype):
    """Flag bit 4 only stops launching sweeps after the batch converged."""
    rng = np.random.default_rng(21)
    mats = [rng.standard_normal((150, 100)).astype(dtype) for _ in range(6)]
    S1, U1, V1, i1, w1 = run_gpu(mats, nb=16, path="blocked")
    S2, U2, V2, i2, w2 = run_gpu(mats, nb=16, path="blocked", flags=bsvd.FLAG_SYNC_CHECK)
    assert (i1 == 0).all() and np.array_equal(w1, w2)
    assert np.array_equal(S1, S2) and np.array_equal(U1, U2) and np.array_equal(V1, V2)


@pytest.mark.parametrize("flags", [0, bsvd.FLAG_F32_FFMA, bsvd.FLAG_WIDE_ANGLES, bsvd.FLAG_THREE_KERNELS])
@pytest.mark.parametrize("m,n,nb", [(200, 150, 16), (257, 33, 8), (150, 260, 16)])
def test_blocked_fp32_tensor_core_and_ffma(flags, m, n, nb):
    """The multi-kernel FP32 Gram and update on the tensor cores (default),
    on the FMA tiles (flags bit 7), and with FP64 rotations (bit 8)."""
    rng = np.random.default_rng(m * 3 + n + nb + flags)
    mats = [rng.standard_normal((m, n)).astype(np.float32) for _ in range(3)]
    S, U, V, info, sw = run_gpu(mats, nb=nb, path="blocked", flags=flags)
    ref = oracle.gesvj(mats)
    check(mats, S, U, V, info, ref["S"], f"flags {flags} {m}x{n}")


@pytest.mark.parametrize("flags", [0, bsvd.FLAG_F32_FFMA, bsvd.FLAG_WIDE_ANGLES, bsvd.FLAG_THREE_KERNELS])
@pytest.mark.parametrize("m,n,nb", [(200, 150, 16), (257, 33, 8), (150, 260, 16), (130, 130, 16)])
def test_blocked_complex64_tensor_core_and_ffma(flags, m, n, nb):
    """The multi-kernel complex64 Gram and update as real split-TF32 products
    of the real and imaginary parts, in one pair-step kernel per round
    (default) or three kernels (bit 12), on the FMA pipes (flags bit 7), and
    with FP64 rotations (bit 8): bounds against the oracle."""
    rng = np.random.default_rng(m * 5 + n + nb + flags)
    mats = [(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))).astype(np.complex64) for _ in range(3)]
    S, U, V, info, sw = run_gpu(mats, nb=nb, path="blocked", flags=flags)
    ref = oracle.gesvj(mats)
    check(mats, S, U, V, info, ref["S"], f"c64 flags {flags} {m}x{n}")


@pytest.mark.parametrize("dtype", [np.complex64, np.float32])
@pytest.mark.parametrize("m,n,nb,extra", [(200, 150, 16, 0), (257, 33, 8, 0), (150, 260, 16, 0), (70, 200, 8, 0),
                                          (333, 97, 16, bsvd.FLAG_WIDE_ANGLES), (96, 96, 8, bsvd.FLAG_NO_MASKS),
                                          (40, 24, 8, 0), (24, 60, 16, 0)])
def test_pairstep_equals_three_kernels_bitwise(dtype, m, n, nb, extra):
    """The pair-step kernel performs each stage's operations in the order of
    the three per-round kernels (flags bit 12): the same bits; also with
    fewer rows than one staged 64-row chunk."""
    rng = np.random.default_rng(m + 7 * n + nb + extra)
    if dtype == np.complex64:
        mats = [(rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))).astype(dtype) for _ in range(4)]
    else:
        mats = [rng.standard_normal((m, n)).astype(dtype) for _ in range(4)]
    S1, U1, V1, i1, w1 = run_gpu(mats, nb=nb, path="blocked", flags=extra)
    S2, U2, V2, i2, w2 = run_gpu(mats, nb=nb, path="blocked", flags=extra | bsvd.FLAG_THREE_KERNELS)
    assert (i1 == 0).all() and (i2 == 0).all() and np.array_equal(w1, w2)
    assert np.array_equal(S1, S2) and np.array_equal(U1, U2) and np.array_equal(V1, V2)
