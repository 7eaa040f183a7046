"""Uneven batches in one persistent launch (needs a GB300): CTAs take
matrices of any shape from a largest-first queue and solve each whole in a
global-memory slot.  Parity with the oracle, and agreement with the on-chip
kernel when both use the same block width."""
import numpy as np
import pytest
import torch

import __graft_entry__  # noqa: F401
import oracle
import paper_2601_17979_gb300 as bsvd
import synth
from oracle import checks

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()


def run_batched(mats, **kw):
    T = [torch.from_numpy(x).cuda() for x in mats]
    r = bsvd.gesvj_batched(T, **kw)
    return ([s.cpu().numpy() for s in r.S], None if r.U is None else [u.cpu().numpy() for u in r.U],
            None if r.V is None else [v.cpu().numpy() for v in r.V], r.info.cpu().numpy(), r.sweeps.cpu().numpy())


@pytest.mark.parametrize("cplx", [False, True])
def test_uneven_sample_one_launch(cplx):
    ids = [i for i in range(80) if (i % 2 == 1) == cplx][:24]
    mats = synth.matrices("uneven", ids)
    S, U, V, info, sw = run_batched(mats, path="persistent")
    ref = oracle.gesvj(mats)
    assert (info == 0).all(), info
    for i, A in enumerate(mats):
        meas = checks.measures(A, S[i], U[i], V[i], ref["S"][i])
        assert checks.violations(meas, checks.U32) == [], (i, A.shape, meas)


@pytest.mark.parametrize("dtype", [np.float64, np.complex128, np.float32])
def test_mixed_shapes_and_edges(dtype):
    rng = np.random.default_rng(21)
    shapes = [(40, 24), (24, 40), (1, 1), (7, 1), (1, 7), (0, 5), (5, 0), (130, 70), (64, 64), (33, 17), (3, 3)]
    mats = []
    for m, n in shapes:
        x = rng.standard_normal((m, n))
        if np.issubdtype(dtype, np.complexfloating):
            x = x + 1j * rng.standard_normal((m, n))
        mats.append(x.astype(dtype))
    mats[3][2, 0] = np.nan                                   # one non-finite matrix
    S, U, V, info, sw = run_batched(mats, path="persistent", nb=8)
    u = checks.unit_roundoff(dtype)
    for i, (A, (m, n)) in enumerate(zip(mats, shapes)):
        if min(m, n) == 0:
            assert info[i] == 0
            continue
        if i == 3:
            assert info[i] == -1 and np.isnan(S[i]).all()
            continue
        assert info[i] == 0
        meas = checks.measures(A, S[i], U[i], V[i], oracle.gesvj(A)["S"])
        assert checks.violations(meas, u) == [], (i, meas)


@pytest.mark.parametrize("flags", [0, bsvd.FLAG_NO_ONCHIP])
@pytest.mark.parametrize("dtype", [np.float32, np.float64, np.complex64, np.complex128])
def test_persistent_equals_on_chip_bitwise(dtype, flags):
    """Both kernels run the same per-matrix code (the layout of each matrix
    comes from its own shape, the rotations' roundings are fixed by explicit
    FMAs), so the persistent launch gives the on-chip kernel's bits, with W
    and V in shared memory (these shapes fit) or in global slots (bit 9)."""
    rng = np.random.default_rng(22)
    shapes = [(48, 32), (32, 48), (100, 64), (20, 20)]
    cplx = np.issubdtype(dtype, np.complexfloating)
    mats = [(rng.standard_normal(s) + (1j * rng.standard_normal(s) if cplx else 0)).astype(dtype) for s in shapes]
    S1, U1, V1, i1, w1 = run_batched(mats, path="persistent", nb=8, flags=flags)
    S2, U2, V2, i2, w2 = run_batched(mats, path="fused", nb=8)
    assert (i1 == 0).all() and (i2 == 0).all()
    assert np.array_equal(w1, w2)
    for k, A in enumerate(mats):
        assert np.array_equal(S1[k], S2[k]) and np.array_equal(U1[k], U2[k]) and np.array_equal(V1[k], V2[k]), k
    u = checks.unit_roundoff(dtype)
    ref = oracle.gesvj(mats)
    for k, A in enumerate(mats):
        meas = checks.measures(A, S1[k], U1[k], V1[k], ref["S"][k])
        assert checks.violations(meas, u) == [], (k, meas)


def test_persistent_jobs_none():
    mats = synth.matrices("uneven", range(0, 16, 2))
    S, U, V, info, sw = run_batched(mats, path="persistent", compute_u=False, compute_v=False)
    assert U is None and V is None and (info == 0).all()
    ref = oracle.gesvj(mats, want_u=False, want_v=False)
    for i in range(len(mats)):
        assert np.abs(S[i] - ref["S"][i]).max() <= 50 * min(mats[i].shape) * checks.U32 * ref["S"][i][0]


@pytest.mark.parametrize("dtype", [np.complex64, np.float32])
def test_split_large_bitwise(dtype):
    """Flags bit 6: complex64 matrices with min(m, n) >= 112 run as one
    variable-shape multi-kernel batch beside the persistent launch.  Each of
    them gets the bits of the multi-kernel path run on its shape alone (the
    kernels do the same per-matrix arithmetic; rounds and pairs a smaller
    matrix lacks are skipped), each of the rest the bits of the plain
    persistent launch.  FP32 batches ignore the flag."""
    rng = np.random.default_rng(31)
    shapes = [(300, 150), (40, 30), (128, 128), (140, 260), (64, 20), (513, 129), (90, 90), (0, 4), (200, 131),
              (120, 115), (111, 200)]
    cplx = np.issubdtype(dtype, np.complexfloating)
    mats = [(rng.uniform(-1, 1, s) + (1j * rng.uniform(-1, 1, s) if cplx else 0)).astype(dtype) for s in shapes]
    S, U, V, info, sw = run_batched(mats, path="persistent", flags=bsvd.FLAG_SPLIT_LARGE)
    Sp, Up, Vp, ip, wp = run_batched(mats, path="persistent")
    assert (info == 0).all() and (ip == 0).all()
    u = checks.unit_roundoff(dtype)
    for k, (A, (m, n)) in enumerate(zip(mats, shapes)):
        if min(m, n) == 0:
            continue
        if min(m, n) >= 112 and cplx:
            S1, U1, V1, i1, w1 = run_batched([A], path="blocked", nb=16)
        else:
            S1, U1, V1, i1, w1 = [Sp[k]], [Up[k]], [Vp[k]], [ip[k]], [wp[k]]
        assert sw[k] == w1[0], (k, sw[k], w1[0])
        assert np.array_equal(S[k], S1[0]) and np.array_equal(U[k], U1[0]) and np.array_equal(V[k], V1[0]), k
        meas = checks.measures(A, S[k], U[k], V[k], oracle.gesvj(A)["S"])
        assert checks.violations(meas, u) == [], (k, A.shape, meas)


@pytest.mark.parametrize("cplx", [True])
def test_split_large_uneven_sample_and_jobs(cplx):
    """The uneven workload's recipe with the split, parity with the oracle;
    then without U and V."""
    pool = [(i, synth.matrix("uneven", i)) for i in range(1 if cplx else 0, 160, 2)]
    big = [x for _, x in pool if min(x.shape) >= 112][:4]
    small = [x for _, x in pool if min(x.shape) < 112][:6]
    mats = big + small
    S, U, V, info, sw = run_batched(mats, path="persistent", flags=bsvd.FLAG_SPLIT_LARGE | bsvd.FLAG_SYNC_CHECK)
    ref = oracle.gesvj(mats)
    assert (info == 0).all(), info
    for i, A in enumerate(mats):
        meas = checks.measures(A, S[i], U[i], V[i], ref["S"][i])
        assert checks.violations(meas, checks.U32) == [], (i, A.shape, meas)
    S2, U2, V2, i2, _ = run_batched(mats, path="persistent", flags=bsvd.FLAG_SPLIT_LARGE, compute_u=False,
                                    compute_v=False)
    assert U2 is None and V2 is None and (i2 == 0).all()
    for i in range(len(mats)):
        assert np.abs(S2[i] - S[i]).max() <= 50 * min(mats[i].shape) * checks.U32 * S[i][0]


@pytest.mark.parametrize("dtype", [np.float32, np.complex64, np.float64])
def test_segments_per_shape_block_width(dtype):
    """A batch whose shapes take different block widths (4, 8, 16) and both
    homes of W and V (shared memory, global slot) runs as several persistent
    launches; each matrix gets the bits of the same matrix solved alone with
    its planned block width, and meets the bounds against the oracle."""
    rng = np.random.default_rng(41)
    shapes = [(8, 8), (30, 20), (9, 5), (100, 64), (420, 200), (64, 130), (25, 14), (260, 180)]
    cplx = np.issubdtype(dtype, np.complexfloating)
    mats = [(rng.uniform(-1, 1, s) + (1j * rng.uniform(-1, 1, s) if cplx else 0)).astype(dtype) for s in shapes]
    nb, where, launches = bsvd.persistent_plan(dtype, shapes)
    assert launches >= 3 and set(where.tolist()) == {0, 1}, (nb, where)
    S, U, V, info, sw = run_batched(mats, path="persistent")
    assert (info == 0).all(), info
    u = checks.unit_roundoff(dtype)
    for k, A in enumerate(mats):
        S1, U1, V1, i1, w1 = run_batched([A], path="persistent", nb=int(nb[k]))
        assert sw[k] == w1[0] and np.array_equal(S[k], S1[0]), k
        assert np.array_equal(U[k], U1[0]) and np.array_equal(V[k], V1[0]), k
        meas = checks.measures(A, S[k], U[k], V[k], oracle.gesvj(A)["S"])
        assert checks.violations(meas, u) == [], (k, A.shape, meas)


def test_autotune_batched_buckets_are_followed():
    """Per-bucket autotuning of a mixed-shape batch: every bucket gets a
    block width among 4, 8, 16 whose time is the smallest measured; the
    persistent plan then uses each bucket's width, and the batch still
    meets the bounds.  Run on its own host thread, whose library handle
    (and so its tuning table) no other test shares."""
    import threading
    out = {}

    def body():
        try:
            mats = synth.matrices("uneven", range(0, 120, 2))          # FP32 sample of the workload
            T = [torch.from_numpy(np.asfortranarray(x)).cuda() for x in mats]
            table = bsvd.autotune_batched(T, sample=8)
            nb, where, _ = bsvd.persistent_plan(np.float32, [x.shape for x in mats])
            r = bsvd.gesvj_batched(T, path="persistent")
            torch.cuda.synchronize()
            out.update(mats=mats, table=table, nb=nb, r=r)
        except Exception as e:                                     # reported by the main thread
            out["error"] = e

    th = threading.Thread(target=body)
    th.start()
    th.join()
    assert "error" not in out, out.get("error")
    table, mats, nb, r = out["table"], out["mats"], out["nb"], out["r"]
    assert table and all(b["nb"] in (4, 8, 16) for b in table)
    for b in table:
        done = {w: t for w, t in b["ms"].items() if t >= 0}
        assert b["ms"][b["nb"]] == min(done.values()), b
    chosen = {(b["M"], b["N"]): b["nb"] for b in table}

    def p2(x):
        p = 1
        while p < x:
            p *= 2
        return p
    for k, A in enumerate(mats):
        m, n = A.shape
        assert nb[k] == chosen[(p2(max(m, n)), p2(min(m, n)))], (A.shape, nb[k])
    info = r.info.cpu().numpy()
    assert (info == 0).all()
    ref = oracle.gesvj(mats)
    for k, A in enumerate(mats):
        meas = checks.measures(A, r.S[k].cpu().numpy(), r.U[k].cpu().numpy(), r.V[k].cpu().numpy(), ref["S"][k])
        assert checks.violations(meas, checks.U32) == [], (k, A.shape, meas)
