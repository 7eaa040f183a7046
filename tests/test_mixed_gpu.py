"""Mixed precision for FP64 output (needs a GB300): FP32 sweeps, FP64
restoration of V, FP64 polish.  Results must meet the FP64 bounds against
the FP64 oracle (u = 2^-53), exactly like the native FP64 path."""
import numpy as np
import pytest
import torch

import __graft_entry__  # noqa: F401
import oracle
import paper_2601_17979_gb300 as bsvd
import synth
from oracle import checks

pytestmark = pytest.mark.gpu
U = 2.0 ** -53


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def run(mats, **kw):
    A = torch.from_numpy(np.stack(mats)).cuda()
    r = bsvd.gesvj(A, **kw)
    torch.cuda.synchronize()
    return (r.S.cpu().numpy(), None if r.U is None else r.U.cpu().numpy(),
            None if r.V is None else r.V.cpu().numpy(), r.info.cpu().numpy(), r.sweeps.cpu().numpy())


def check(mats, S, Uo, Vo, info, ref_S, label):
    for i, A in enumerate(mats):
        assert info[i] == 0, (label, i, info[i])
        meas = checks.measures(A, S[i], None if Uo is None else Uo[i], None if Vo is None else Vo[i], ref_S[i])
        assert checks.violations(meas, U) == [], (label, i, meas)


def test_mixed_tall128x64_fewer_fp64_sweeps():
    mats = synth.matrices("tall128x64_f64", range(16))
    S, Uo, Vo, info, sw = run(mats, nb=16, prec="mixed")
    ref = oracle.gesvj(mats, tol=30 * U)
    check(mats, S, Uo, Vo, info, ref["S"], "mixed tall")
    _, _, _, _, sw_native = run(mats, nb=16)
    assert sw.max() <= 6 and sw.mean() < 0.4 * sw_native.mean(), (sw, sw_native)


@pytest.mark.parametrize("half", ["real", "complex"])
def test_mixed96_clustered(half):
    ids = range(0, 16, 2) if half == "real" else range(1, 16, 2)
    mats = [synth.matrix("mixed96", i) for i in ids]
    S, Uo, Vo, info, sw = run(mats, nb=16, prec="mixed")
    ref = oracle.gesvj(mats, tol=30 * U)
    check(mats, S, Uo, Vo, info, ref["S"], "mixed96 " + half)


@pytest.mark.parametrize("dtype", [np.float64, np.complex128])
@pytest.mark.parametrize("m,n", [(64, 48), (48, 64), (33, 33), (200, 40), (9, 3), (260, 140), (140, 260)])
def test_mixed_random_shapes(dtype, m, n):
    rng = np.random.default_rng(m * 7 + n)
    mats = [rng.standard_normal((m, n)) + (1j * rng.standard_normal((m, n)) if dtype == np.complex128 else 0)
            for _ in range(4)]
    mats = [x.astype(dtype) for x in mats]
    S, Uo, Vo, info, sw = run(mats, prec="mixed")
    ref = oracle.gesvj(mats)
    check(mats, S, Uo, Vo, info, ref["S"], f"{m}x{n}")


def test_mixed_jobs_and_nonfinite():
    rng = np.random.default_rng(2)
    mats = [rng.standard_normal((40, 24)) for _ in range(3)]
    ref = oracle.gesvj(mats)
    for cu, cv in [(True, False), (False, True), (False, False)]:
        S, Uo, Vo, info, _ = run(mats, prec="mixed", compute_u=cu, compute_v=cv)
        check(mats, S, Uo, Vo, info, ref["S"], f"jobs {cu}{cv}")
    bad = [m.copy() for m in mats]
    bad[1][0, 0] = np.inf
    S, Uo, Vo, info, _ = run(bad, prec="mixed")
    assert info[1] == -1 and info[0] == 0 and info[2] == 0


def test_mixed_rejected_for_single_precision():
    A = torch.zeros((2, 8, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(bsvd.BsvdError, match="INVALID"):
        bsvd.gesvj(A, prec="mixed")


@pytest.mark.parametrize("flags", [bsvd.FLAG_WIDE_ANGLES, bsvd.FLAG_F32_FFMA])
def test_mixed_variants_meet_fp64_bounds(flags):
    """Mixed precision with FP64 rotations in the FP32 sweeps (bit 8), and
    with the FP32 Gram and update on the FMA pipes (bit 7): FP64 bounds."""
    mats = synth.matrices("tall128x64_f64", range(12)) + [synth.matrix("mixed96", i) for i in (0, 2)]
    ref = oracle.gesvj(mats, tol=30 * U)
    for lo, hi in ((0, 12), (12, 14)):
        S, Uo, Vo, info, sw = run(mats[lo:hi], nb=16, prec="mixed", flags=flags)
        check(mats[lo:hi], S, Uo, Vo, info, ref["S"][lo:hi], f"flags {flags}")


@pytest.mark.parametrize("path", ["auto", "persistent"])
@pytest.mark.parametrize("dtype", [np.float64, np.complex128])
def test_mixed_pointer_array_mixed_shapes(path, dtype):
    """Mixed precision on a pointer-array batch of several shapes (grouped by
    shape, inputs and outputs through the pointer arrays, wide shapes solved
    as A^H): every result meets the FP64 bounds against the oracle, and each
    equals the strided mixed call on its own shape group bitwise."""
    rng = np.random.default_rng(61)
    shapes = [(64, 48), (48, 64), (64, 48), (130, 40), (33, 33), (0, 3), (64, 48), (40, 130)]
    cplx = dtype == np.complex128
    mats = [(rng.standard_normal(s) + (1j * rng.standard_normal(s) if cplx else 0)).astype(dtype) for s in shapes]
    T = [torch.from_numpy(np.asfortranarray(x)).cuda() for x in mats]
    r = bsvd.gesvj_batched(T, prec="mixed", path=path)
    torch.cuda.synchronize()
    info = r.info.cpu().numpy()
    assert (info == 0).all(), info
    for k, (A, s) in enumerate(zip(mats, shapes)):
        if min(s) == 0:
            continue
        ref = oracle.gesvj(A, tol=30 * U)
        check([A], [r.S[k].cpu().numpy()], [r.U[k].cpu().numpy()], [r.V[k].cpu().numpy()], [0], [ref["S"]],
              f"{path} {s}")
    same = [k for k, s in enumerate(shapes) if s == (64, 48)]
    Sg, Ug, Vg, ig, wg = run([mats[k] for k in same], prec="mixed")
    for j, k in enumerate(same):
        assert np.array_equal(r.S[k].cpu().numpy(), Sg[j]) and np.array_equal(r.U[k].cpu().numpy(), Ug[j])
        assert np.array_equal(r.V[k].cpu().numpy(), Vg[j]) and int(r.sweeps[k]) == wg[j]
