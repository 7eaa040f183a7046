"""The serving loop (needs a GB300): results of requests served through the
continuous-batching server meet the bounds, are the same bit for bit alone
and in a mix, complete before the rest of their batch, and stay within the
device-memory arena."""
import ctypes
import threading
import time

import numpy as np
import pytest
import torch

import __graft_entry__  # noqa: F401
import oracle
import paper_2601_17979_gb300 as bsvd
from oracle import checks

pytestmark = pytest.mark.gpu

MiB = 1 << 20
DT = {"s": np.float32, "d": np.float64, "c": np.complex64, "z": np.complex128}


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def rand(rng, m, n, t):
    x = rng.standard_normal((m, n))
    if t in "cz":
        x = x + 1j * rng.standard_normal((m, n))
    return x.astype(DT[t])


def pinned(x):
    """Column-major page-locked CPU tensor holding x."""
    return torch.from_numpy(np.ascontiguousarray(x.T)).pin_memory().t()


def check_result(A, r, label):
    ref = oracle.gesvj([A])
    u = checks.unit_roundoff(A.dtype)
    assert r.info == 0, f"{label}: info {r.info}"
    meas = checks.measures(A, r.S.numpy(), None if r.U is None else r.U.numpy(),
                           None if r.V is None else r.V.numpy(), ref["S"][0])
    bad = checks.violations(meas, u)
    assert not bad, f"{label}: {bad} {meas}"


def test_server_results_meet_bounds():
    rng = np.random.default_rng(11)
    cases = []
    for i in range(40):
        t = "sdcz"[i % 4]
        m = int(rng.integers(1, 120))
        n = int(rng.integers(1, 120))
        cases.append((rand(rng, m, n, t), t))
    cases.append((rand(rng, 150, 100, "d"), "d"))     # above big_k: the multi-kernel path
    cases.append((rand(rng, 90, 130, "c"), "c"))
    with bsvd.Server(256 * MiB, big_k=64) as srv:
        ids = [srv.submit(pinned(A)) for A, _ in cases]
        for (A, t), rid in zip(cases, ids):
            check_result(A, srv.fetch(rid), f"{t} {A.shape}")
        st = srv.stats()
        assert st["completed"] == len(cases) and st["failed"] == 0 and st["queued"] == 0
        assert st["arena_used"] == 0 and 0 < st["arena_peak"] <= 256 * MiB


def test_jobs_and_device_inputs():
    rng = np.random.default_rng(12)
    A = rand(rng, 70, 50, "d")
    with bsvd.Server(64 * MiB) as srv:
        r1 = srv.fetch(srv.submit(torch.from_numpy(A).cuda(), compute_u=False))
        r2 = srv.fetch(srv.submit(pinned(A), compute_v=False))
    assert r1.U is None and r2.V is None
    check_result(A, r1, "jobu=N")
    check_result(A, r2, "jobv=N")


def test_mix_invariance_bitwise():
    """Each probe's result alone equals its result inside a mixed stream."""
    rng = np.random.default_rng(13)
    probes = [rand(rng, 40, 30, "s"), rand(rng, 100, 64, "d"), rand(rng, 20, 20, "c"),
              rand(rng, 70, 90, "z"), rand(rng, 160, 90, "d")]      # the last above big_k
    alone = []
    with bsvd.Server(128 * MiB, big_k=80) as srv:
        for P in probes:
            alone.append(srv.fetch(srv.submit(pinned(P))))
    mix = []
    for i in range(240):
        t = "sdcz"[int(rng.integers(0, 4))]
        mix.append(rand(rng, int(rng.integers(8, 110)), int(rng.integers(8, 110)), t))
    mix.append(rand(rng, 160, 90, "d"))          # same shape as the big probe: batched with it
    with bsvd.Server(512 * MiB, big_k=80) as srv:
        srv.pause()
        ids = [srv.submit(pinned(A)) for A in mix[:120]]
        pid = [srv.submit(pinned(P)) for P in probes]
        ids += [srv.submit(pinned(A)) for A in mix[120:]]
        srv.pause(False)
        inmix = [srv.fetch(r) for r in pid]
        for r in ids:
            srv.fetch(r)
    for P, a, b in zip(probes, alone, inmix):
        assert a.info == b.info == 0
        assert torch.equal(a.S, b.S) and torch.equal(a.U, b.U) and torch.equal(a.V, b.V), P.shape


def test_requests_retire_before_their_batch_ends():
    """A small matrix in the same batch as a large one completes first."""
    rng = np.random.default_rng(14)
    big = rand(rng, 256, 256, "d")
    small = [rand(rng, 48, 48, "d") for _ in range(30)]
    with bsvd.Server(256 * MiB, max_inflight=1) as srv:
        srv.pause()
        bid = srv.submit(pinned(big))
        sid = [srv.submit(pinned(A)) for A in small]
        srv.pause(False)
        t_big = srv.wait(bid)[2]
        t_small = [srv.wait(r)[2] for r in sid]
        assert srv.stats()["batches"] == 1
        assert max(t_small) < t_big
        for A, r in zip(small[:3], sid[:3]):
            check_result(A, srv.fetch(r), "small")
        check_result(big, srv.fetch(bid), "big")


def test_memory_budget_admission():
    """A 2 MiB arena serves 60 requests (66 KB of outputs each) in several
    batches, never above budget; a request that cannot fit even alone fails
    with BSVD_ERR_WORKSPACE."""
    rng = np.random.default_rng(15)
    mats = [rand(rng, 64, 64, "d") for _ in range(60)]
    with bsvd.Server(2 * MiB) as srv:
        ids = [srv.submit(pinned(A)) for A in mats]
        for A, r in zip(mats, ids):
            res = srv.fetch(r)
            if r % 10 == 0:
                check_result(A, res, "budget")
        st = srv.stats()
        assert st["completed"] == 60 and st["arena_peak"] <= 2 * MiB and st["batches"] > 1
        huge = srv.submit(pinned(rand(rng, 1024, 1024, "d")))
        with pytest.raises(bsvd.BsvdError, match="WORKSPACE"):
            srv.wait(huge, timeout=30)
        srv.release(huge)


def test_rejects_pageable_input():
    L = bsvd.load()
    with bsvd.Server(16 * MiB) as srv:
        A = np.ones((8, 8), order="F")
        rid = ctypes.c_longlong()
        st = L.bsvd_server_submit(srv.srv, b"d", 8, 8, A.ctypes.data, 8, 1, 1, ctypes.byref(rid))
        assert st == -1
        assert srv.stats()["submitted"] == 0


def test_replay_and_collect():
    """A trace replayed at 4000 requests/s: every request completes, with
    t_done after its scheduled arrival."""
    rng = np.random.default_rng(16)
    N = 400
    mats = [pinned(rand(rng, int(rng.integers(16, 64)), int(rng.integers(16, 64)), "sdc"[i % 3]))
            for i in range(N)]
    t = np.cumsum(rng.exponential(1 / 4000, N))
    got = []
    with bsvd.Server(256 * MiB) as srv:
        done = threading.Event()

        def collector():
            while not done.is_set() or sum(len(g["id"]) for g in got) < N:
                got.append(srv.collect())
                time.sleep(0.002)
                if time.monotonic() > deadline:
                    break

        deadline = time.monotonic() + 60
        th = threading.Thread(target=collector)
        th.start()
        ids, t0 = srv.replay(t, mats)
        done.set()
        th.join()
        st = srv.stats()
    ids_done = np.concatenate([g["id"] for g in got])
    assert sorted(ids_done.tolist()) == sorted(ids.tolist())
    status = np.concatenate([g["status"] for g in got])
    info = np.concatenate([g["info"] for g in got])
    assert (status == 0).all() and (info == 0).all()
    ts = np.concatenate([g["t_submit"] for g in got])
    td = np.concatenate([g["t_done"] for g in got])
    assert (td > ts).all()
    assert np.allclose(np.sort(ts) - t0, t, atol=1e-6)
    assert st["completed"] == N and st["arena_used"] == 0


def test_destroy_with_queued_requests():
    rng = np.random.default_rng(17)
    A = pinned(rand(rng, 32, 32, "s"))
    srv = bsvd.Server(64 * MiB, max_inflight=1)
    srv.pause()
    for _ in range(500):
        srv.submit(A)
    st = srv.stats()
    assert st["queued"] == 500 and st["running"] == 0
    srv.pause(False)
    t = time.monotonic()
    srv.close()
    assert time.monotonic() - t < 30


def test_cancel_stops_queued_and_running_work():
    """Cancel: every request completes either with its result or as
    cancelled, and the server serves normally afterwards."""
    rng = np.random.default_rng(18)
    mats = [rand(rng, 128, 128, "d") for _ in range(400)]
    with bsvd.Server(1024 * MiB, max_inflight=1, max_batch=200) as srv:
        srv.pause()
        ids = [srv.submit(pinned(A)) for A in mats]
        srv.pause(False)
        time.sleep(0.01)
        srv.cancel()
        status = []
        for A, r in zip(mats, ids):
            try:
                res = srv.fetch(r)
                status.append(0)
                if len(status) < 3:
                    check_result(A, res, "before cancel")
            except bsvd.BsvdError as e:
                assert e.status == -7, e
                status.append(-7)
                srv.release(r)
        st = srv.stats()
        assert st["completed"] + st["cancelled"] == 400 and st["failed"] == 0
        assert status.count(-7) == st["cancelled"] > 0
        A = rand(rng, 50, 40, "d")
        check_result(A, srv.fetch(srv.submit(pinned(A))), "after cancel")


def test_concurrent_multi_kernel_batches():
    """Multi-kernel batches of distinct shapes launch from several host
    threads at once; every one completes within the bounds."""
    rng = np.random.default_rng(19)
    mats = [rand(rng, 70 + 9 * i, 66 + 7 * i, "sdc"[i % 3]) for i in range(12)]
    with bsvd.Server(1024 * MiB, big_k=64) as srv:
        srv.pause()
        ids = [srv.submit(pinned(A)) for A in mats]
        srv.pause(False)
        for A, r in zip(mats, ids):
            check_result(A, srv.fetch(r), f"{A.dtype} {A.shape}")
        assert srv.stats()["failed"] == 0


def test_fp64_mixed_precision_for_large_requests():
    """With fp64_prec = mixed the server solves FP64 and complex128 requests
    on the multi-kernel path (min(m, n) > big_k) by FP32 sweeps and FP64
    polish: the results meet the FP64 bounds; smaller FP64 requests and
    other types are unaffected."""
    rng = np.random.default_rng(71)
    cases = [(rand(rng, 70, 50, "d"), "d"), (rand(rng, 50, 70, "d"), "d"), (rand(rng, 66, 40, "z"), "z"),
             (rand(rng, 70, 50, "d"), "d"), (rand(rng, 30, 20, "d"), "d"), (rand(rng, 60, 45, "s"), "s")]
    with bsvd.Server(256 * MiB, big_k=32, fp64_prec="mixed") as srv:
        ids = [srv.submit(pinned(A)) for A, _ in cases]
        for (A, t), r in zip(cases, ids):
            check_result(A, srv.fetch(r), f"mixed server {t} {A.shape}")
