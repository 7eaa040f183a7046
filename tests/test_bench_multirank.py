"""The multi-GPU logic of bench.py on CPU: two gloo ranks (127.0.0.1).

The path shards by matrix (replicas solving disjoint slices of the seeded
workload, no collective on the data path); the only cross-rank step is the
scalar all-reduce of the step time (max) or of a throughput (sum)."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import __graft_entry__  # noqa: F401
import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                       # rank 1 is the slower one
        worst = bench.max_over_ranks(ms, dist, "cpu")
        total = bench.sum_over_ranks(100.0 * (rank + 1), dist, "cpu")
        idx = bench.shard(rank, 4)
        A64, A32 = bench.build_inputs(rank, 4)
        out.put((rank, worst, total, list(idx), float(A64.sum()), float(A32.astype(np.float64).sum())))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, w0, t0, i0, a0, b0), (_, w1, t1, i1, a1, b1) = res
    assert w0 == w1 == 15.0                          # max over ranks, seen by both
    assert t0 == t1 == 300.0                         # sum over ranks
    assert i0 == [0, 1, 2, 3] and i1 == [4, 5, 6, 7]   # disjoint shards
    assert a0 != a1 and b0 != b1                     # different matrices per rank
    # rank 1's matrices are the workload's matrices 4..7
    import synth
    ref = synth.uniform_batch("tall128x64_f64", 4, start=4)
    assert np.isclose(a1, ref.sum())


def test_single_rank_is_identity():
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.sum_over_ranks(2.0, None, "cpu") == 2.0
    assert list(bench.shard(0, 3)) == [0, 1, 2]


def test_uneven_launch_count():
    """The uneven step's launch claim: one persistent launch per segment of
    each type (from the plan), and for each split batch (the plan's
    where = 2) the multi-kernel batch's load, max-sweeps sweeps of
    k (L_max - 1) + 2 kernels (the device stops the loop; k = 1 for the
    pair step, 3 with flags bit 7 or 12) and three finalisation kernels."""
    from types import SimpleNamespace
    f32, c64 = np.dtype(np.float32), np.dtype(np.complex64)
    groups = {f32: [np.zeros((300, 200), np.float32), np.zeros((100, 90), np.float32)],
              c64: [np.zeros((40, 30), np.complex64), np.zeros((512, 300), np.complex64),
                    np.zeros((200, 130), np.complex64)]}
    res = {f32: SimpleNamespace(sweeps=torch.tensor([12, 8])),
           c64: SimpleNamespace(sweeps=torch.tensor([20, 13, 9]))}
    plans = {f32: (np.array([16, 16]), np.array([2, 0]), 1),
             c64: (np.array([8, 16, 16]), np.array([1, 2, 2]), 1)}
    # FP32 split: n = 200 -> l = 13 blocks, L = 14; 12 sweeps issued
    # complex64 split: n up to 300 -> l = 19 blocks, L = 20; 13 sweeps issued
    per_step = 2 + 1 + 12 * (1 * 13 + 2) + 3 + 1 + 13 * (1 * 19 + 2) + 3
    assert bench.uneven_launches(groups, res, plans, steps=1, flags=0) == per_step
    assert bench.uneven_launches(groups, res, plans, steps=3, flags=0) == 3 * per_step
    # flags bit 12: rounds as three kernels
    three = 2 + 1 + 12 * (3 * 13 + 2) + 3 + 1 + 13 * (3 * 19 + 2) + 3
    assert bench.uneven_launches(groups, res, plans, steps=1, flags=4096) == three
    res_small = {f32: SimpleNamespace(sweeps=torch.tensor([12])), c64: SimpleNamespace(sweeps=torch.tensor([20]))}
    plans_small = {f32: (np.array([16]), np.array([0]), 1), c64: (np.array([8]), np.array([1]), 1)}
    assert bench.uneven_launches({f32: groups[f32][:1], c64: groups[c64][:1]}, res_small, plans_small,
                                 steps=2, flags=0) == 4
