"""QR pre-processing (Sec. "Pre-processing the SVD using a QR
Factorization") on a GB300: A = Q [R; 0] by Householder QR, the SVD of R,
U = Q [U_R; 0].  Outputs against the oracle under the same bounds as every
other path."""
import numpy as np
import pytest
import torch

import __graft_entry__  # noqa: F401
import oracle
import paper_2601_17979_gb300 as bsvd
from oracle import checks

pytestmark = pytest.mark.gpu

DT = {"s": np.float32, "d": np.float64, "c": np.complex64, "z": np.complex128}


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def rand(rng, shape, t, count):
    out = []
    for _ in range(count):
        x = rng.uniform(0, 1, shape)
        if t in "cz":
            x = x + 1j * rng.uniform(0, 1, shape)
        out.append(x.astype(DT[t]))
    return out


def run(mats, **kw):
    A = torch.from_numpy(np.stack(mats)).cuda()
    r = bsvd.gesvj(A, flags=bsvd.FLAG_QR, **kw)
    torch.cuda.synchronize()
    return (r.S.cpu().numpy(), None if r.U is None else r.U.cpu().numpy(),
            None if r.V is None else r.V.cpu().numpy(), r.info.cpu().numpy())


def check(mats, S, U, V, info, label):
    ref = oracle.gesvj(mats)
    u = checks.unit_roundoff(mats[0].dtype)
    for i, A in enumerate(mats):
        assert info[i] == 0, (label, i, info[i])
        meas = checks.measures(A, S[i], None if U is None else U[i], None if V is None else V[i], ref["S"][i])
        bad = checks.violations(meas, u)
        assert not bad, f"{label} {i}: {bad} {meas}"


@pytest.mark.parametrize("t", list("sdcz"))
@pytest.mark.parametrize("shape", [(100, 16), (1000, 16), (2000, 16), (129, 40), (64, 64), (16, 300),
                                   (500, 5), (7, 1), (300, 37)])
def test_qr_path_parity(t, shape):
    rng = np.random.default_rng(ord(t) * 10007 + shape[0] * 31 + shape[1])
    mats = rand(rng, shape, t, 4)
    S, U, V, info = run(mats)
    check(mats, S, U, V, info, f"{t} {shape}")


@pytest.mark.parametrize("path", ["fused", "blocked"])
def test_qr_then_each_path_for_r(path):
    rng = np.random.default_rng(3)
    mats = rand(rng, (400, 48), "d", 3)
    S, U, V, info = run(mats, path=path, nb=16)
    check(mats, S, U, V, info, path)


def test_qr_jobs():
    rng = np.random.default_rng(4)
    mats = rand(rng, (250, 20), "d", 3)
    S1, U1, V1, i1 = run(mats, compute_u=False)
    assert U1 is None
    check(mats, S1, None, V1, i1, "jobu=N")
    S2, U2, V2, i2 = run(mats, compute_v=False)
    assert V2 is None
    check(mats, S2, U2, None, i2, "jobv=N")
    wide = [x.T.copy() for x in mats]
    S3, U3, V3, i3 = run(wide, compute_u=False)
    check(wide, S3, None, V3, i3, "wide jobu=N")


def test_qr_scaling_and_nonfinite():
    rng = np.random.default_rng(5)
    mats = rand(rng, (300, 12), "d", 3)
    mats[0] = mats[0] * 2.0 ** 1000        # squares would overflow without the exact scaling
    mats[1] = mats[1] * 2.0 ** -1000
    mats[2][5, 3] = np.inf
    S, U, V, info = run(mats)
    assert info[2] == -1 and np.isnan(S[2]).all()
    # measure on the problem scaled back by the same powers of two (exact)
    back = [mats[0] * 2.0 ** -1000, mats[1] * 2.0 ** 1000]
    Sb = np.stack([S[0] * 2.0 ** -1000, S[1] * 2.0 ** 1000])
    check(back, Sb, U[:2], V[:2], info[:2], "scaled")


def test_qr_agrees_with_unpreprocessed():
    rng = np.random.default_rng(6)
    mats = rand(rng, (600, 16), "d", 8)
    A = torch.from_numpy(np.stack(mats)).cuda()
    a = bsvd.gesvj(A)
    b = bsvd.gesvj(A, flags=bsvd.FLAG_QR)
    s0 = a.S.cpu().numpy()
    assert np.abs(s0 - b.S.cpu().numpy()).max() <= 50 * 16 * 2.0 ** -53 * s0.max()


def test_qr_not_with_mixed_or_pointer_arrays():
    A = torch.rand(2, 50, 10, dtype=torch.float64, device="cuda")
    with pytest.raises(bsvd.BsvdError, match="NOT_IMPLEMENTED"):
        bsvd.gesvj(A, flags=bsvd.FLAG_QR, prec="mixed")
    with pytest.raises(bsvd.BsvdError, match="NOT_IMPLEMENTED"):
        bsvd.gesvj_batched([A[0], A[1]], flags=bsvd.FLAG_QR)


def test_qr_workspace_too_small():
    A = torch.rand(3, 200, 16, dtype=torch.float64, device="cuda")
    work = torch.empty(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(bsvd.BsvdError, match="WORKSPACE"):
        bsvd.gesvj(A, flags=bsvd.FLAG_QR, work=work)
