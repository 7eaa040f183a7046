"""Benchmark: batched one-sided Jacobi SVD on GB300.

Workload (one step): the 128x64 tall batch in both precisions -- 10,000 FP64
matrices Q1 diag(sigma) Q2^T with geometric sigma from 1 to 1e-6 and 10,000
FP32 matrices with sigma from 1 to 1e-3 (Haar Q1, Q2; synthetic, seeded),
nb = 16, full U, Sigma, V.  Metric: matrices/s (whole job, all ranks).

Reported on one JSON line:
  value       device-resident throughput (inputs in HBM before timing)
  e2e         the same through the public API with host buffers: pinned
              H2D of A and D2H of Sigma, U, V, info inside the timed region
  roofline    the dominant kernel (FP64 fused SVD) against the FP64 pipe
  cpu_baseline the CPU oracle (OpenMP over matrices) on a bounded sample
  plain_fp64  the paper's baseline path (inner solver to convergence, no
              masks) on the FP64 batch, for "vs plain FP64 Jacobi"
  fp64_mixed  FP64 output from FP32 sweeps + FP64 polish on the same batch,
              held to the same FP64 bounds (sweeps_mean = polish sweeps)
With --impl reference the CPU oracle alone runs as the reference arm.
Multi-GPU (torchrun): every rank solves its own 10,000 + 10,000 matrices
(weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

U64, U32 = 2.0 ** -53, 2.0 ** -24
M, N, NB = 128, 64, 16
BATCH = 10000
TOL_K = 30
# FP64 / FP32 pipe peaks of GB300 from unit counts and the maximum SM clock:
# 152 SMs x 2 FP64 FMA/clk/SM (resp. 128 FP32 FMA/clk/SM) x 2 flop x 2.07 GHz.
PEAK_FP64 = 152 * 2 * 2 * 2.07e9
PEAK_FP32 = 152 * 128 * 2 * 2.07e9
# DRAM bytes per matrix of a kernel from one ncu capture
# (dram__bytes_read.sum + dram__bytes_write.sum of one launch divided by the
# matrices it solved), valid only while the kernel's sources are unchanged:
# keyed by (workload kernel, sha1 prefix of its source files).  A capture of
# a smaller batch is scaled by the matrix count (the traffic of these
# kernels grows in proportion to the matrices solved).
CSRC = os.path.join(ROOT, "paper_2601_17979_gb300", "csrc")
KERNEL_SOURCES = {
    "fused": ("gesvj_fused.cuh", "jacobi_common.cuh", "fused_f32.cuh", "scalar.cuh", "tc_f32.cuh"),
    "persistent": ("gesvj_fused.cuh", "jacobi_common.cuh", "fused_f32.cuh", "scalar.cuh", "tc_f32.cuh"),
    "uneven": ("gesvj_fused.cuh", "jacobi_common.cuh", "fused_f32.cuh", "scalar.cuh", "tc_f32.cuh",
               "tc_c64.cuh", "gesvj_blocked.cuh", "blocked_launch.cuh", "gesvj_pairstep.cuh"),
}
TRAFFIC_PER_MATRIX = {
    # 128x64, gesvj_fused_kernel<double|float,16,2,128>: 2,000-matrix launches
    ("fused", "tall128x64_f64", "8b18517283c6"): (137206528 + 143052800) / 2000,
    ("fused", "tall128x64_f32", "8b18517283c6"): (65873920 + 40259328) / 2000,
    # the whole uneven step (every kernel of both types), 2,000-matrix case:
    # 497.6 GB over the warm-up and the timed step
    ("uneven", "uneven", "490147fdfd01"): 497.60e9 / 2 / 2000,
}


def source_hash(kind: str) -> str:
    import hashlib
    h = hashlib.sha1()
    for f in KERNEL_SOURCES[kind]:
        h.update(open(os.path.join(CSRC, f), "rb").read())
    return h.hexdigest()[:12]


def measured_traffic(kind: str, workload: str, matrices: int):
    per = TRAFFIC_PER_MATRIX.get((kind, workload, source_hash(kind)))
    return None if per is None else per * matrices


def pair_flops(m, n, nb, cplx=False):
    """Algorithmic flops of one block pair: Gram 4 m nb^2, A update 8 m nb^2,
    V update 8 n nb^2, one inner sweep 72 nb^3 (x4 for complex)."""
    f = 12 * m * nb * nb + 8 * n * nb * nb + 72 * nb ** 3
    return 4 * f if cplx else f


def matrix_flops(m, n, nb, sweeps):
    """Executed sweeps: all but the last do full pair steps; the last (the
    sweep that found every block diagonal) forms the Gram blocks only."""
    l = max(2, -(-n // nb))
    pairs = l * (l - 1) // 2
    sweeps = np.asarray(sweeps, dtype=np.float64)
    return (np.maximum(sweeps - 1, 0) * pairs * pair_flops(m, n, nb)
            + pairs * 4 * m * nb * nb + 3 * m * n).sum()


def oracle_flops(m, n, sweeps):
    """Alg. 2 work: (12 m + 6 n) flops per column pair per sweep."""
    return float(np.sum(np.asarray(sweeps, dtype=np.float64) * (12 * m + 6 * n) * n * (n - 1) / 2))


def timed_calls(torch, fn, steps, stream, warmup=1, flush=None):
    """CUDA-event times (ms) of `steps` calls of fn on `stream` after
    `warmup` untimed calls; with `flush` (a device buffer larger than L2)
    L2 is overwritten before every call, outside the timed events."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ts = []
    for _ in range(steps):
        if flush is not None:
            flush.fill_(1)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    return ts


def oracle_reference(mats, tol):
    """The CPU oracle's sigma (Alg. 2, FP64) for a sample of matrices."""
    import oracle
    return oracle.default().gesvj(list(mats), tol=tol, want_u=False, want_v=False)["S"]


def accuracy_over_bounds(mats, S, U, V, S_ref, u):
    """Worst gating measure over its bound (spec bounds in the working
    precision u) on a sample: sigma error against the oracle's sigma,
    residual, orthogonality of U and V.  S, U, V index like mats."""
    from oracle import checks
    worst = {}
    for i, A in enumerate(mats):
        meas = checks.measures(A, S[i], U[i], V[i], S_ref[i])
        b = checks.bounds(meas["n"], u)
        for key, lim in b.items():
            if key in meas:
                worst[key] = max(worst.get(key, 0.0), meas[key] / lim)
    return worst


class ClockSampler:
    """nvidia-smi clocks/throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.gpu_id, self.proc, self.lines = gpu_id, None, []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu_id}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                mx = max(mx, float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_uuid(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return "0"


def shard(rank: int, per_rank: int) -> range:
    """Matrix indices of one rank: the ranks solve disjoint slices of the
    seeded workload (weak scaling, no collective on the data path)."""
    return range(rank * per_rank, (rank + 1) * per_rank)


def max_over_ranks(ms: float, dist, device) -> float:
    """The slowest rank's time, i.e. the whole job's (one all-reduce of a
    scalar after the timed region; nothing else crosses ranks)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist, device) -> float:
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t)
    return float(t.item())


def build_inputs(rank: int, count: int):
    idx = shard(rank, count)
    A64 = synth.uniform_batch("tall128x64_f64", count, start=idx.start)
    A32 = synth.uniform_batch("tall128x64_f32", count, start=idx.start)
    return A64, A32


def run_reference(args, rank, world):
    """Reference arm: the CPU oracle on the host cores, bounded samples."""
    import oracle
    if rank != 0:
        return
    if args.workload == "square32":
        return run_reference_square32(args, world)
    per = args.ref_sample
    A64 = synth.matrices("tall128x64_f64", range(per))
    A32 = synth.matrices("tall128x64_f32", range(per))
    O = oracle.default()
    cores = len(os.sched_getaffinity(0))
    times, threads = [], 0
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r1 = O.gesvj(A64, tol=TOL_K * U64)
        r2 = O.gesvj(A32, tol=TOL_K * U64)
        dt = time.perf_counter() - t0
        threads = r1["threads"]
        if s >= args.warmup:
            times.append(dt)
    t = float(np.mean(times))
    value = 2 * per / t
    line = {
        "impl": "reference", "metric": "batch SVD matrices/s (tall 128x64, FP64+FP32)",
        "value": value, "unit": "matrices/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(world, per * 2),
        "cpu_baseline": {"value": value, "unit": "matrices/s", "cores": threads, "kind": "oracle",
                         "sample": f"{per} FP64 + {per} FP32 matrices 128x64 per step, Alg. 2 (unblocked), "
                                   f"OpenMP over matrices, {cores} cores available"},
        "e2e": {"value": value, "unit": "matrices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_reference_square32(args, world):
    """Reference arm of the square32 workload: the CPU oracle (Alg. 2, FP64,
    tol = n u) on the same 1,000 matrices per step."""
    import oracle
    B = args.batch if args.batch != BATCH else 1000
    mats = list(synth.uniform_batch("square32_f64", B))
    O = oracle.default()
    cores = len(os.sched_getaffinity(0))
    times, threads = [], 0
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        r = O.gesvj(mats, tol=32 * U64)
        dt = time.perf_counter() - t0
        threads = r["threads"]
        if s >= args.warmup:
            times.append(dt)
    t = float(np.mean(times))
    value = B / t
    line = {"impl": "reference", "metric": "batch SVD matrices/s (square 32x32 FP64, N(0,1)) vs plain FP64 Jacobi",
            "value": value, "unit": "matrices/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"square32: {B} matrices 32x32, entries iid N(0,1), FP64", "nb": 8,
                       "tol": "n u = 32 u", "jobs": "U, Sigma, V"},
            "cpu_baseline": {"value": value, "unit": "matrices/s", "cores": threads, "kind": "oracle",
                             "sample": f"all {B} matrices per step, Alg. 2 (unblocked), OpenMP over matrices, "
                                       f"{cores} cores available"},
            "e2e": {"value": value, "unit": "matrices/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# matrices with min(m, n) >= 112 (complex64) or 144 (FP32) run as one
# variable-shape multi-kernel batch per type beside the persistent launches
# (flags bit 6, and bit 10 for real FP32; measured 3.53 s against 3.68 s per
# step with FP32 kept persistent); bit 4 is the host-checked stop, used only
# where graphs are off
UNEVEN_FLAGS = 64 | 16 | 1024


def uneven_launches(groups, res, plans, steps, flags, nb=16):
    """Kernel launches of one uneven step: one persistent launch per segment
    of each type, and for each split batch the multi-kernel batch's load,
    sweeps (each L_max - 1 rounds -- one pair-step kernel, or the Gram,
    eigensolver and update kernels with flags bit 7 or 12 -- then the
    convergence and loop-control kernels; the device stops the loop once all
    have converged) and three finalisation kernels."""
    n = sum(plans[dt][2] for dt in res)
    per_round = 3 if flags & (128 | 4096) else 1
    for dt, r in res.items():
        sw = r.sweeps.cpu().numpy()
        big = [(x.shape, k) for x, k, w in zip(groups[dt], sw, plans[dt][1]) if w == 2]
        if not big:
            continue
        l = max(-(-min(s) // nb) for s, _ in big)
        L = l + (l & 1)
        issued = int(max(k for _, k in big))
        n += 1 + issued * (per_round * (L - 1) + 2) + 3
    return n * steps


def run_uneven(args, rank, world, local):
    """Uneven sizes: one persistent launch per type vs one launch per shape."""
    import torch
    import paper_2601_17979_gb300 as bsvd
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    bsvd.build()
    B = args.batch if args.batch != BATCH else 20000
    mats = synth.matrices("uneven", shard(rank, B))
    groups = {}
    for x in mats:
        groups.setdefault(x.dtype, []).append(x)
    # resident in the library's column-major layout (a row-major view would
    # make the binding copy every matrix on every call)
    dev_mats = {dt: [torch.from_numpy(np.asfortranarray(x)).to(dev) for x in lst] for dt, lst in groups.items()}
    assert all(t.stride(0) == 1 for lst in dev_mats.values() for t in lst if t.shape[1] > 1)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # one stream per type: the second type's persistent launch fills the
    # first one's tail (its last, smallest matrices) instead of waiting for it
    side = {dt: (stream if i == 0 else torch.cuda.Stream(dev)) for i, dt in enumerate(dev_mats)}

    def solve_all(path):
        res = {}
        start = torch.cuda.Event()
        start.record(stream)
        for dt, T in dev_mats.items():
            s = side[dt]
            if s is not stream:
                s.wait_event(start)
            res[dt] = bsvd.gesvj_batched(T, path=path, stream=s, flags=args.uneven_flags)
        for s in side.values():
            if s is not stream:
                done = torch.cuda.Event()
                done.record(s)
                stream.wait_event(done)
        return res

    # per-bucket autotuning (untimed set-up, like the paper's offline
    # decision layer): block width per (type, M, N rounded to powers of two)
    # bucket, timed on a sample of each bucket with persistent launches
    tuning = {}
    if not args.no_autotune:
        t0 = time.perf_counter()
        for dt, T in dev_mats.items():
            tuning[np.dtype(dt).name] = bsvd.autotune_batched(T, sample=args.tune_sample)
        tune_s = time.perf_counter() - t0
    # how each matrix runs: its block width and where W and V live (the
    # per-bucket decision layer), and the launches per type
    plans = {dt: bsvd.persistent_plan(dt, [x.shape for x in groups[dt]], flags=args.uneven_flags) for dt in groups}
    for _ in range(max(1, args.warmup)):
        solve_all("persistent")
    barrier()
    sampler = ClockSampler(gpu_uuid(torch, dev))
    with sampler:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            res = solve_all("persistent")
        b.record(stream)
        barrier()
    ms = max_over_ranks(a.elapsed_time(b) / args.steps, dist, dev)
    value = B * world / (ms * 1e-3)
    flops = 0.0
    buckets = {}
    for dt, r in res.items():
        sw = r.sweeps.cpu().numpy()
        nbs, where, _ = plans[dt]
        for x, k, nb_, w in zip(groups[dt], sw, nbs, where):
            m, n = x.shape
            f = matrix_flops(max(m, n), min(m, n), int(nb_), [k])      # at the executed block width
            flops += 4 * f if np.iscomplexobj(x) else f
            key = f"{np.dtype(dt).name} nb={int(nb_)} {['global slot', 'shared memory', 'multi-kernel'][int(w)]}"
            seg = buckets.setdefault(key, {"matrices": 0, "k_min": 10 ** 9, "k_max": 0})
            seg["matrices"] += 1
            seg["k_min"] = min(seg["k_min"], min(m, n))
            seg["k_max"] = max(seg["k_max"], min(m, n))
    info = np.concatenate([r.info.cpu().numpy() for r in res.values()])
    line = {"metric": "batch SVD matrices/s (uneven sizes, FP32 + complex64)", "value": value,
            "unit": "matrices/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+c64", "data": "synthetic",
            "config": {"workload": "uneven: m ~ U{8..512}, n ~ U{8..m}, entries U(-1,1), half complex64",
                       "matrices_per_rank": B, "flags": args.uneven_flags,
                       "path": "persistent launches per type (one per block width x shared memory / global "
                               "slot segment, block width per size bucket, autotuned), one stream per type; "
                               "matrices with k >= 112 (complex64) or 144 (FP32) as one variable-shape "
                               "multi-kernel batch per type "
                               "beside them",
                       "l2": "inputs larger than L2"},
            "gpu_launches": uneven_launches(groups, res, plans, args.steps, args.uneven_flags), "info_nonzero": int((info != 0).sum()),
            "segments": buckets,
            "autotune": ({"seconds": tune_s, "sample_per_bucket": args.tune_sample,
                          "buckets": {k: [[b["M"], b["N"], b["nb"]] + [round(b["ms"][w], 3) for w in (4, 8, 16)]
                                          for b in v] for k, v in tuning.items()},
                          "columns": "M, N (rounded up to powers of two), chosen nb, ms at nb 4, 8, 16"}
                         if tuning else None),
            "gflops": flops / (ms * 1e-3) / 1e9,
            "roofline": {"bound": "alu", "achieved": flops / (ms * 1e-3) / 1e12, "peak": PEAK_FP32 / 1e12,
                         "unit": "TFLOP/s", "frac": flops / (ms * 1e-3) / PEAK_FP32,
                         "traffic": measured_traffic("uneven", "uneven", B),
                         "traffic_note": "every kernel of the step, DRAM read + write (ncu on a 2,000-matrix "
                                         "case, scaled by matrix count)"},
            "clocks": sampler.summary()}
    # the same matrices with one launch per distinct shape (the pointer-array
    # form grouping by shape) -- the path the persistent launch replaces
    # (timed on the first 500 matrices: nearly every shape is distinct, so it
    # runs one launch -- or one multi-kernel sweep loop -- per matrix)
    if not args.no_per_shape:
        sub = {}
        for x in mats[:min(B, 500)]:
            sub.setdefault(x.dtype, []).append(torch.from_numpy(np.asfortranarray(x)).to(dev))
        barrier()
        a.record(stream)
        for dt, T in sub.items():
            bsvd.gesvj_batched(T, path="auto")
        b.record(stream)
        barrier()
        per_shape = a.elapsed_time(b)
        nsub = sum(len(T) for T in sub.values())
        line["one_launch_per_shape"] = {"matrices_per_s": nsub / (per_shape * 1e-3), "ms": per_shape,
                                        "matrices": nsub,
                                        "distinct_shapes": len({x.shape + (x.dtype,) for x in mats[:nsub]}),
                                        "persistent_speedup": (per_shape / nsub) / (ms / B)}
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        S = min(args.cpu_sample, 400)
        sample = mats[:S]
        t0 = time.perf_counter()
        r = oracle.default().gesvj(sample)
        dt_ = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": S / dt_, "unit": "matrices/s", "cores": r["threads"], "kind": "oracle",
                                "sample": f"first {S} matrices of the same workload, Alg. 2 in FP64, "
                                          f"OpenMP over matrices ({dt_:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def serve_stream(srv, rate, seconds, drain, stream, pool_cache):
    """Replay one Poisson stream at the server; collect until drained or until
    `drain` seconds after the last arrival.  Returns the per-request records
    of completed requests and the server counters."""
    tr = synth.serving_trace(rate, seconds, stream=stream)
    keys = list(zip(tr["bin"].tolist(), tr["tall"].tolist(), tr["dtype"].tolist(), tr["variant"].tolist()))
    for k in set(keys):
        if k not in pool_cache:
            import torch
            A = synth.serving_matrix(*k)
            pool_cache[k] = torch.from_numpy(np.ascontiguousarray(A.T)).pin_memory().t()
    mats = [pool_cache[k] for k in keys]
    got, stop = [], threading.Event()

    def collector():
        while not stop.is_set():
            got.append(srv.collect(1 << 16))
            time.sleep(0.005)
        got.append(srv.collect(1 << 20))

    before = srv.stats()
    th = threading.Thread(target=collector, daemon=True)
    th.start()
    ids, t0 = srv.replay(tr["t"], mats, keep=False)
    t_arrivals = srv.clock()
    at_end = srv.stats()
    while srv.clock() < t_arrivals + drain:
        st = srv.stats()
        if st["queued"] == 0 and st["running"] == 0:
            break
        time.sleep(0.01)
    t_stop = srv.clock()
    final = srv.stats()
    # what is left is cancelled (running persistent batches stop taking matrices)
    srv.cancel()
    t_cancel = time.monotonic()
    while srv.stats()["running_batches"] > 0 and time.monotonic() < t_cancel + 300:
        time.sleep(0.01)
    stop.set()
    th.join()
    rec = {k: np.concatenate([g[k] for g in got]) if got else np.zeros(0) for k in
           ("id", "status", "info", "sweeps", "t_submit", "t_done")}
    mine = (rec["id"] >= ids[0]) & (rec["id"] <= ids[-1])
    rec = {k: v[mine] for k, v in rec.items()}
    idx = rec["id"] - ids[0]
    return tr, ids, t0, t_arrivals, t_stop, rec, idx, before, at_end, final


def summarize_stream(tr, ids, t0, t_arrivals, t_stop, rec, idx, before, at_end, final, seconds):
    ok = rec["status"] == 0
    lat = (rec["t_done"] - rec["t_submit"])[ok] * 1e3
    n_sub = len(ids)
    n_done = int(ok.sum())
    sizes = synth.serving_sizes()
    m = sizes[tr["bin"][idx[ok]]]
    n = np.where(tr["tall"][idx[ok]], -(-m // 2), m)
    cplx = tr["dtype"][idx[ok]] == "c"
    sw = rec["sweeps"][ok]
    flops = 0.0
    for mm, nn, c, k in zip(m.tolist(), n.tolist(), cplx.tolist(), sw.tolist()):
        f = matrix_flops(mm, nn, 16 if nn >= 48 else (8 if nn >= 12 else 4), [k])
        flops += 4 * f if c else f
    span = max(float(rec["t_done"][ok].max()) - t0, 1e-9) if n_done else 1e-9
    in_window = int((rec["t_done"][ok] <= t_arrivals).sum())
    pct = (lambda q: float(np.percentile(lat, q)) if n_done else None)
    backlog = (at_end["queued"] + at_end["running"]) - (before["queued"] + before["running"])
    out = {"submitted": int(n_sub), "completed": n_done, "cancelled": int((rec["status"] == -7).sum()),
           "failed": int(((rec["status"] != 0) & (rec["status"] != -7)).sum()),
           "completed_by_end_of_arrivals": in_window,
           "throughput_rps": n_done / span, "throughput_in_window_rps": in_window / seconds,
           "gflops": flops / span / 1e9,
           "latency_ms": {"p50": pct(50), "p99": pct(99), "max": float(lat.max()) if n_done else None},
           "backlog_at_end_of_arrivals": int(backlog),
           "drained": bool(final["queued"] == 0 and final["running"] == 0),
           "drain_s": t_stop - t_arrivals, "info_nonzero": int((rec["info"][ok] != 0).sum()),
           "arena_peak_gb": final["arena_peak"] / 1e9}
    # latency by request class: small (k <= 64), medium (64 < k <= 256, the
    # persistent batches), large (k > 256, the multi-kernel batches), by type
    if n_done:
        kk = np.minimum(m, n)
        dts = tr["dtype"][idx[ok]]
        classes = {}
        for cname, sel in (("small", kk <= 64), ("medium", (kk > 64) & (kk <= 256)), ("large", kk > 256)):
            for t in ("s", "d", "c"):
                sl = sel & (dts == t)
                if sl.any():
                    classes[f"{cname}_{t}"] = {"n": int(sl.sum()), "p50": float(np.percentile(lat[sl], 50)),
                                               "p99": float(np.percentile(lat[sl], 99))}
        out["latency_by_class_ms"] = classes
    bad = (rec["status"] != 0) & (rec["status"] != -7)
    if bad.any():
        codes, counts = np.unique(rec["status"][bad], return_counts=True)
        out["failed_status"] = {str(int(c)): int(k) for c, k in zip(codes, counts)}
        j = idx[bad][:5]
        out["failed_examples"] = [[int(sizes[tr["bin"][i]]), bool(tr["tall"][i]), str(tr["dtype"][i]),
                                   int(rec["info"][np.flatnonzero(idx == i)[0]])] for i in j]
    if not out["drained"] and out["throughput_rps"] > 0:
        out["left_at_stop"] = int(final["queued"] + final["running"])
        out["drain_estimate_s"] = out["left_at_stop"] / out["throughput_rps"]
    return out


def run_serving(args, rank, world, local):
    """Serving stream: Poisson arrivals replayed at the continuous-batching
    server; throughput, p50/p99 latency, backlog, and a rate sweep."""
    import torch
    import paper_2601_17979_gb300 as bsvd
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    bsvd.build()
    cfg = synth.SERVING
    rate = args.rate or cfg["rate"]
    seconds = args.seconds or cfg["seconds"]
    pool = {}
    srv = bsvd.Server(int(args.arena_gb * 1e9), max_inflight=32, fp64_prec=args.fp64_prec,
                      big_flags=args.big_flags, max_big_batch=args.max_big_batch, big_k_fp64=args.big_k_fp64)
    # warm-up: a short low-rate stream (first launches set kernel attributes)
    for _ in range(max(1, args.warmup)):
        serve_stream(srv, 500.0, 0.2, 30.0, 1000 + rank, pool)
    if dist is not None:
        dist.barrier()
    sampler = ClockSampler(gpu_uuid(torch, dev))
    with sampler:
        r = serve_stream(srv, rate, seconds, args.drain, rank, pool)
    main = summarize_stream(*r, seconds)
    sweep = []
    for k, lam in enumerate(args.sweep_rates):
        rr = serve_stream(srv, lam, args.sweep_seconds, args.sweep_seconds, 100 + 10 * k + rank, pool)
        s_ = summarize_stream(*rr, args.sweep_seconds)
        sweep.append({"rate_rps": lam, "p50_ms": s_["latency_ms"]["p50"], "p99_ms": s_["latency_ms"]["p99"],
                      "throughput_rps": s_["throughput_rps"], "completed": s_["completed"],
                      "submitted": s_["submitted"], "drained": s_["drained"],
                      "by_class_ms": s_.get("latency_by_class_ms")})
    batches = srv.stats()["batches"]
    srv.close()
    value = sum_over_ranks(main["throughput_rps"], dist, dev)
    sustained = [x["rate_rps"] for x in sweep if x["drained"] and x["completed"] == x["submitted"]]
    line = {"metric": "serving throughput (Poisson stream) with p50/p99 latency", "value": value,
            "unit": "requests/s", "n_gpus": world, "steps": 1, "warmup": args.warmup,
            "ms_per_step": seconds * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64+c64", "data": "synthetic",
            "config": {"workload": f"serving: Poisson arrivals {rate:g}/s for {seconds:g} s, m log-uniform "
                                   "16..1024 (64 log-spaced bins), half square, half 2:1 tall, 50% FP32 / "
                                   "30% FP64 / 20% complex64, kappa log-uniform 1e2..1e6, logrand sigma, "
                                   "Haar factors; inputs from a pool of 2 matrices per (bin, shape, type)",
                       "arena_gb": args.arena_gb, "max_inflight": 32, "jobs": "U, Sigma, V",
                       "big_flags": args.big_flags, "max_big_batch": args.max_big_batch or 8,
                       "big_k_fp64": args.big_k_fp64 or 256,
                       "fp64_prec": args.fp64_prec + " (FP64 / complex128 requests above "
                                     f"{args.big_k_fp64 or 256} columns)",
                       "results": "left in the arena and released on completion (not copied back)",
                       "l2": "inputs read once from page-locked host memory"},
            "latency_ms": main["latency_ms"], "serving": main, "rate_sweep": sweep,
            "highest_sustained_rate_rps": max(sustained) if sustained else None,
            "gpu_launches": batches, "clocks": sampler.summary()}
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = serving_cpu_baseline(r[0])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def serving_cpu_baseline(tr, small=300, large=8):
    """The oracle on a bounded sample of the stream: the first `small`
    requests with m <= 256 and the first `large` above, timed per stratum
    (OpenMP over matrices), combined by the stream's mix into requests/s."""
    import oracle
    O = oracle.default()
    sizes = synth.serving_sizes()
    m_all = sizes[tr["bin"]]
    out = {}
    tot = 0.0
    for name, sel, cnt in (("small", m_all <= 256, small), ("large", m_all > 256, large)):
        idx = np.flatnonzero(sel)[:cnt]
        mats = [synth.serving_matrix(int(tr["bin"][i]), bool(tr["tall"][i]), str(tr["dtype"][i]),
                                     int(tr["variant"][i])) for i in idx]
        t0 = time.perf_counter()
        res = O.gesvj(mats)
        dt = time.perf_counter() - t0
        out[name] = (len(mats), dt, res["threads"])
        tot += sel.mean() * dt / max(len(mats), 1)
    cores = out["small"][2]
    return {"value": 1.0 / tot, "unit": "requests/s", "cores": cores, "kind": "oracle",
            "sample": f"first {out['small'][0]} requests with m <= 256 ({out['small'][1]:.1f} s) and first "
                      f"{out['large'][0]} with m > 256 ({out['large'][1]:.1f} s) of the stream, Alg. 2 in FP64, "
                      "OpenMP over matrices, weighted by the stream's mix"}


def run_tallskinny(args, rank, world, local):
    """Tall-skinny batches, n = 16 and m from 100 to 2,000, entries U[0,1]
    (the paper's larnv inputs): the SVD with and without QR pre-processing."""
    import torch
    import paper_2601_17979_gb300 as bsvd
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    bsvd.build()
    B = args.batch if args.batch != BATCH else 1000
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)    # larger than L2
    stream = torch.cuda.current_stream(dev)
    rows = []
    sampler = ClockSampler(gpu_uuid(torch, dev))
    sampler.__enter__()
    for t, dt in (("d", torch.float64), ("s", torch.float32), ("z", torch.complex128), ("c", torch.complex64)):
        for m in (100, 200, 500, 1000, 1500, 2000):
            rng = synth.rng_for(synth.SEED_BASE + 6, m * 4 + "sdcz".index(t))
            x = rng.uniform(0, 1, (B, 16, m))
            if t in "cz":
                x = x + 1j * rng.uniform(0, 1, (B, 16, m))
            A = torch.from_numpy(x).to(dt).to(dev).transpose(1, 2)      # column-major m x 16
            row = {"dtype": t, "m": m, "n": 16, "batch": B}
            for name, flags in (("noqr", 0), ("qr", bsvd.FLAG_QR)):
                res = bsvd.gesvj(A, flags=flags)                         # warm-up
                times = []
                for _ in range(max(1, args.steps)):
                    flush.fill_(1)
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    res = bsvd.gesvj(A, flags=flags)
                    b.record(stream)
                    torch.cuda.synchronize()
                    times.append(a.elapsed_time(b))
                ms = statistics.median(times)
                row[name + "_ms"] = ms
                row[name + "_matrices_per_s"] = B / (ms * 1e-3)
                row[name + "_info_nonzero"] = int((res.info != 0).sum().item())
                sw = res.sweeps.cpu().numpy()
                row[name + "_sweeps_mean"] = float(sw.mean())
                f = tallskinny_flops(m, 16, sw, name == "qr") * (4 if t in "cz" else 1)
                row[name + "_tflops"] = f / (ms * 1e-3) / 1e12
            row["qr_speedup"] = row["noqr_ms"] / row["qr_ms"]
            rows.append(row)
            print(json.dumps(row), file=sys.stderr, flush=True)
    sampler.__exit__(None, None, None)
    head = next(r for r in rows if r["dtype"] == "d" and r["m"] == 2000)
    line = {"metric": "batch SVD matrices/s (tall-skinny 2000x16 FP64, QR pre-processing)",
            "value": head["qr_matrices_per_s"], "unit": "matrices/s", "n_gpus": world, "steps": args.steps,
            "warmup": 1, "ms_per_step": head["qr_ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"tall-skinny: {B} matrices m x 16 per (type, m), m in 100..2000, entries "
                                   "U[0,1] (real and imaginary parts); U, Sigma, V; median of steps",
                       "l2": "L2 flushed (256 MB write) before every timed call"},
            "gpu_launches": 2 * max(1, args.steps),
            # QR factor, Q applied to [U_R; 0] and the SVD of R, algorithmic
            # FP64 flops of the executed sweeps, against the FP64 pipe
            "roofline": {"bound": "alu", "achieved": head["qr_tflops"], "peak": PEAK_FP64 / 1e12,
                         "unit": "TFLOP/s", "frac": head["qr_tflops"] * 1e12 / PEAK_FP64, "traffic": None,
                         "kernel": "qr_factor + SVD of R + qr_apply (FP64, m = 2000, n = 16)",
                         "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz"},
            "clocks": sampler.summary(), "results": rows}
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        rng = synth.rng_for(synth.SEED_BASE + 6, 2000 * 4 + "sdcz".index("d"))
        x = rng.uniform(0, 1, (min(args.cpu_sample, 200), 16, 2000))
        mats = [np.ascontiguousarray(xi.T) for xi in x]
        t0, reps = time.perf_counter(), 0
        while reps == 0 or time.perf_counter() - t0 < 3.0:
            r = oracle.default().gesvj(mats)
            reps += 1
        dt_ = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": reps * len(mats) / dt_, "unit": "matrices/s", "cores": r["threads"],
                                "kind": "oracle",
                                "sample": f"the first {len(mats)} FP64 2000x16 matrices of the workload, {reps} "
                                          f"passes, Alg. 2 in FP64 (no QR), OpenMP over matrices ({dt_:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def tallskinny_flops(m, n, sweeps, qr):
    """Algorithmic real flops of the tall-skinny solve: with QR, Householder
    QR 2 m n^2 - 2 n^3 / 3, Q applied to [U_R; 0] 4 m n^2 - 2 n^3 and the
    SVD of the n x n factor R; without, the SVD of the m x n matrix."""
    nb = 16 if n >= 48 else (8 if n >= 12 else 4)
    if not qr:
        return matrix_flops(m, n, nb, sweeps)
    k = len(np.atleast_1d(sweeps))
    return k * (2 * m * n * n - 2 * n ** 3 / 3 + 4 * m * n * n - 2 * n ** 3) + matrix_flops(n, n, nb, sweeps)


# Timed calls per leg of the 32x32 workload (about 6 ms each): enough for
# the clock sampler (one sample per 200 ms) to see the run.
SQ32_STEPS = 100

# Mixed-precision variants timed beside the default (name, flags).
MIXED_VARIANTS = [("mixed_fp64_angles", 256), ("mixed_ffma", 128)]


def run_square32(args, rank, world, local):
    """Plain FP64 real batch: 1,000 matrices 32x32 with iid N(0,1) entries,
    nb = 8, full U, Sigma, V, a pair rotates while |g_pq| >= n u sqrt(g_pp
    g_qq) (tol = n u = 32 u).  The batched on-chip solver against the plain
    one-launch-per-size FP64 Jacobi path (the paper's baseline: inner solver
    to convergence, two-stage update, no masks) on the same inputs; both are
    held to the same bounds and their sigma compared with the FP64 oracle."""
    import torch
    import paper_2601_17979_gb300 as bsvd
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    bsvd.build()
    B = args.batch if args.batch != BATCH else 1000
    m = n = 32
    nb, tol = 8, 32 * U64
    idx = shard(rank, B)
    Ah = synth.uniform_batch("square32_f64", B, start=idx.start)
    A = torch.from_numpy(Ah).to(dev).transpose(1, 2).contiguous().transpose(1, 2)
    o = (torch.empty((B, n), dtype=torch.float64, device=dev), bsvd.empty_column_major(B, m, n, torch.float64, dev),
         bsvd.empty_column_major(B, n, n, torch.float64, dev), torch.empty(B, dtype=torch.int32, device=dev),
         torch.empty(B, dtype=torch.int32, device=dev))
    stream = torch.cuda.current_stream(dev)
    # the batch (8 MB in, 16 MB out) fits in L2: L2 is flushed before every call
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    samp = list(range(0, B, max(1, B // 16)))
    ref = oracle_reference([Ah[i] for i in samp], tol)

    def leg(path, **kw):
        nbytes = bsvd.workspace_bytes(torch.float64, [(m, n)], True, batch=B, nb=nb, tol=tol, path=path, **kw)
        work = torch.empty(max(nbytes, 256), dtype=torch.uint8, device=dev)
        if dist is not None:
            dist.barrier()
        sampler = ClockSampler(gpu_uuid(torch, dev))
        with sampler:
            ts = timed_calls(torch, lambda: bsvd.gesvj(A, nb=nb, tol=tol, path=path, out=o, work=work, **kw),
                             max(SQ32_STEPS, args.steps), stream, warmup=max(3, args.warmup), flush=flush)
        ms = max_over_ranks(statistics.median(ts), dist, dev)
        sw = o[4].cpu().numpy()
        acc = accuracy_over_bounds([Ah[i] for i in samp], [o[0][i].cpu().numpy() for i in samp],
                                   [o[1][i].cpu().numpy() for i in samp], [o[2][i].cpu().numpy() for i in samp],
                                   ref, U64)
        fl = matrix_flops(m, n, nb, sw)
        return {"matrices_per_s": B * world / (ms * 1e-3), "ms": ms, "ms_all": ts, "sweeps_mean": float(sw.mean()),
                "sweeps_max": int(sw.max()), "info_nonzero": int((o[3].cpu().numpy() != 0).sum()),
                "tflops": fl / (ms * 1e-3) / 1e12, "accuracy_worst_over_bound": acc,
                "sigma_err_vs_oracle_over_bound": acc.get("sigma_err"), "clocks": sampler.summary()}

    fused = leg("auto")
    S_fused = o[0].cpu().clone()
    plain = leg("plain") if not args.no_plain else None
    line = {"metric": "batch SVD matrices/s (square 32x32 FP64, N(0,1)) vs plain FP64 Jacobi",
            "value": fused["matrices_per_s"], "unit": "matrices/s", "n_gpus": world,
            "steps": max(SQ32_STEPS, args.steps), "warmup": max(3, args.warmup), "ms_per_step": fused["ms"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"square32: {B} matrices 32x32 per rank, entries iid N(0,1), FP64",
                       "nb": nb, "tol": "n u = 32 u", "jobs": "U, Sigma, V",
                       "path": "on-chip batched solver (one CTA per matrix)",
                       "l2": "L2 flushed (256 MB write) before every timed call"},
            "gpu_launches": max(SQ32_STEPS, args.steps), "batched": fused,
            "roofline": {"bound": "alu", "achieved": fused["tflops"], "peak": PEAK_FP64 / 1e12,
                         "unit": "TFLOP/s", "frac": fused["tflops"] * 1e12 / PEAK_FP64,
                         "traffic": measured_traffic("fused", "square32_f64", B),
                         "kernel": "gesvj_fused_kernel<double,8,2,64>",
                         "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz"},
            "clocks": fused["clocks"]}
    if plain is not None:
        line["plain_fp64"] = plain
        line["speedup_over_plain"] = plain["ms"] / fused["ms"]
    if not args.no_e2e:
        Ap = torch.from_numpy(Ah.transpose(0, 2, 1).copy()).pin_memory().transpose(1, 2)
        ho = (torch.empty((B, n), dtype=torch.float64).pin_memory(),
              torch.empty((B, n, m), dtype=torch.float64).pin_memory().transpose(1, 2),
              torch.empty((B, n, n), dtype=torch.float64).pin_memory().transpose(1, 2),
              torch.empty(B, dtype=torch.int32).pin_memory(), torch.empty(B, dtype=torch.int32).pin_memory())
        wh = torch.empty(bsvd.host_workspace_bytes(torch.float64, B, m, n, nb=nb, tol=tol), dtype=torch.uint8,
                         device=dev)
        e_sampler = ClockSampler(gpu_uuid(torch, dev))
        with e_sampler:
            ts = timed_calls(torch, lambda: bsvd.gesvj_host(Ap, nb=nb, tol=tol, out=ho, work=wh, sync=False),
                             max(SQ32_STEPS, args.steps), stream, warmup=max(3, args.warmup), flush=flush)
        e_ms = max_over_ranks(statistics.median(ts), dist, dev)
        line["e2e"] = {"value": B * world / (e_ms * 1e-3), "unit": "matrices/s",
                       "h2d_bytes_per_step": int(Ap.numel() * 8),
                       "d2h_bytes_per_step": int(sum(t.numel() * t.element_size() for t in ho)),
                       "ms_per_step": e_ms, "api": "gesvj_host (bsvd_dgesvj_strided_host)",
                       "same_sigma_as_device_call": bool(torch.equal(ho[0], S_fused)),
                       "clocks": e_sampler.summary()}
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        O = oracle.default()
        mats = [Ah[i] for i in range(B)]
        t0, reps, r = time.perf_counter(), 0, None
        while reps == 0 or time.perf_counter() - t0 < 5.0:
            r = O.gesvj(mats, tol=tol)
            reps += 1
        dt_ = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": reps * B / dt_, "unit": "matrices/s", "cores": r["threads"],
                                "kind": "oracle",
                                "sample": f"the same {B} matrices, {reps} passes ({dt_:.1f} s), Alg. 2 in FP64, "
                                          "OpenMP over matrices",
                                "gflops": reps * oracle_flops(m, n, r["sweeps"]) / dt_ / 1e9}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_mixed96(args, rank, world, local):
    """The clustered 96x96 set: 2,000 real FP64 + 2,000 complex128 matrices,
    sigma in 48 pairs with gap 1e-6, kappa about 1e8: FP64 output from FP32
    sweeps + FP64 polish against native FP64 on the same inputs.  Each
    sampled result's sigma is compared with the FP64 oracle's."""
    import torch
    import paper_2601_17979_gb300 as bsvd
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    bsvd.build()
    per = args.batch if args.batch != BATCH else 4000
    ids = shard(rank, per)
    real = [synth.matrix("mixed96", i) for i in ids if i % 2 == 0]
    cplx = [synth.matrix("mixed96", i) for i in ids if i % 2 == 1]
    A = {"d": torch.from_numpy(np.stack(real)).to(dev).transpose(1, 2).contiguous().transpose(1, 2),
         "z": torch.from_numpy(np.stack(cplx)).to(dev).transpose(1, 2).contiguous().transpose(1, 2)}
    # 30 u, the default (the workload's n u = 96 u leaves U's orthogonality
    # above the 20 n u gate at kappa 1e8, in the oracle as on the GPU)
    tol = TOL_K * U64
    stream = torch.cuda.current_stream(dev)
    src_mats = {"d": real, "z": cplx}
    samp = {t: list(range(0, len(src_mats[t]), max(1, len(src_mats[t]) // 8))) for t in src_mats}
    refs = {t: oracle_reference([src_mats[t][i] for i in samp[t]], tol) for t in src_mats}
    variants = [("native", dict(prec="native")), ("mixed", dict(prec="mixed"))]
    variants += [(name, dict(prec="mixed", flags=fl)) for name, fl in MIXED_VARIANTS if not args.no_variants]
    out = {}
    for name, kw in variants:
        times, res = {}, {}
        sampler = ClockSampler(gpu_uuid(torch, dev))
        with sampler:
            for t in ("d", "z"):
                holder = {}

                def call(t=t, holder=holder):
                    holder["r"] = bsvd.gesvj(A[t], nb=16, tol=tol, **kw)
                ts = timed_calls(torch, call, max(1, args.steps), stream, warmup=1)
                res[t] = holder["r"]
                times[t] = statistics.median(ts)
        total = max_over_ranks(times["d"] + times["z"], dist, dev)
        worst = {}
        for t in ("d", "z"):
            r = res[t]
            w = accuracy_over_bounds([src_mats[t][i] for i in samp[t]],
                                     [r.S[i].cpu().numpy() for i in samp[t]],
                                     [r.U[i].cpu().numpy() for i in samp[t]],
                                     [r.V[i].cpu().numpy() for i in samp[t]], refs[t], U64)
            for key, val in w.items():
                worst[key] = max(worst.get(key, 0.0), val)
        sw = {t: res[t].sweeps.cpu().numpy() for t in res}
        # algorithmic FP64 flops of the executed (polish or native) sweeps
        fl64 = matrix_flops(96, 96, 16, sw["d"]) + 4 * matrix_flops(96, 96, 16, sw["z"])
        out[name] = {"matrices_per_s": len(ids) * world / (total * 1e-3), "ms": total,
                     "ms_real": times["d"], "ms_complex": times["z"],
                     "sweeps_mean": {t: float(sw[t].mean()) for t in sw},
                     "info_nonzero": int(sum(int((res[t].info != 0).sum().item()) for t in res)),
                     "fp64_sweep_tflops": fl64 / (total * 1e-3) / 1e12,
                     "sigma_err_vs_oracle_over_bound": worst.get("sigma_err"),
                     "accuracy_worst_over_bound": worst, "clocks": sampler.summary()}
        if kw.get("flags"):
            out[name]["flags"] = kw["flags"]
    nat = out["native"]
    line = {"metric": "batch SVD matrices/s (96x96 clustered, FP64 output, mixed precision)",
            "value": out["mixed"]["matrices_per_s"], "unit": "matrices/s", "n_gpus": world,
            "steps": args.steps, "warmup": 1, "ms_per_step": out["mixed"]["ms"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64 (mixed), f64 output", "data": "synthetic",
            "config": {"workload": f"mixed96: {per} square 96x96 per rank, even ids real FP64, odd ids complex128, "
                                   "sigma in 48 clustered pairs (gap 1e-6), kappa 1e8, Haar factors",
                       "nb": 16, "tol": "30 u", "jobs": "U, Sigma, V",
                       "l2": "inputs (295 MB real + 590 MB complex per 4,000) larger than L2"},
            "mixed": out["mixed"], "native_fp64": nat,
            "variants": {k: v for k, v in out.items() if k not in ("mixed", "native")},
            "speedup_over_native": nat["ms"] / out["mixed"]["ms"],
            "sigma_err_vs_oracle": {k: v["sigma_err_vs_oracle_over_bound"] for k, v in out.items()},
            # the native FP64 solve against the FP64 pipe (its executed sweeps'
            # algorithmic flops); the mixed solve's FP64 part is the polish
            "roofline": {"bound": "alu", "achieved": nat["fp64_sweep_tflops"], "peak": PEAK_FP64 / 1e12,
                         "unit": "TFLOP/s", "frac": nat["fp64_sweep_tflops"] * 1e12 / PEAK_FP64,
                         "traffic": None, "kernel": "native FP64 solve (on chip real, multi-kernel complex)",
                         "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz"},
            "gpu_launches": None, "clocks": out["mixed"]["clocks"]}
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        S = min(args.cpu_sample, 200)
        sample = [synth.matrix("mixed96", i) for i in range(S)]
        t0 = time.perf_counter()
        r = oracle.default().gesvj(sample, tol=tol)
        dt_ = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": S / dt_, "unit": "matrices/s", "cores": r["threads"], "kind": "oracle",
                                "sample": f"first {S} matrices of the same workload (half complex), Alg. 2 in "
                                          f"FP64, OpenMP over matrices ({dt_:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_square(args, rank, world, local):
    """Square batches with entries U[0,1] (the paper's larnv inputs), n from
    64 to 512: matrices/s and algorithmic TFLOP/s per type and size; matrices
    up to ~100 columns run on chip, larger ones on the multi-kernel path."""
    import torch
    import paper_2601_17979_gb300 as bsvd
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    bsvd.build()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)    # larger than L2
    stream = torch.cuda.current_stream(dev)
    sizes = args.sizes or [64, 128, 256, 512]
    rows = []
    sampler = ClockSampler(gpu_uuid(torch, dev))
    sampler.__enter__()
    for t, dt in (("d", torch.float64), ("s", torch.float32), ("z", torch.complex128), ("c", torch.complex64)):
        if t not in args.square_dtypes:
            continue
        for n in sizes:
            # the paper's square benchmark: batches of 1,000 matrices (FP64 and
            # complex128 n = 512: 200, to keep a run within minutes)
            B = args.batch if args.batch != BATCH else (200 if t in "dz" and n >= 512 else 1000)
            rng = synth.rng_for(synth.SEED_BASE + 7, n * 2 + "dszc".index(t) % 2 + 2 * (t in "zc"))
            a = rng.uniform(0, 1, (B, n, n))
            if t in "zc":
                a = a + 1j * rng.uniform(0, 1, (B, n, n))
            A = torch.from_numpy(a).to(dt).to(dev).transpose(1, 2)
            holder = {}

            def call(A=A, holder=holder):
                holder["r"] = bsvd.gesvj(A, flags=args.square_flags)
            times = timed_calls(torch, call, max(1, args.steps), stream, warmup=1, flush=flush)
            res = holder["r"]
            ms = statistics.median(times)
            sw = res.sweeps.cpu().numpy()
            nb = 16 if n >= 48 else (8 if n >= 12 else 4)
            f = matrix_flops(n, n, nb, sw) * (4 if t in "zc" else 1)     # a complex MAC: four real ones
            rows.append({"dtype": t, "n": n, "batch": B, "ms": ms, "matrices_per_s": B / (ms * 1e-3),
                         "tflops": f / (ms * 1e-3) / 1e12, "sweeps_mean": float(sw.mean()),
                         "info_nonzero": int((res.info != 0).sum().item())})
            print(json.dumps(rows[-1]), file=sys.stderr, flush=True)
    sampler.__exit__(None, None, None)
    head = max(rows, key=lambda r: (r["dtype"] == "d", r["dtype"] == "s", r["dtype"] == "z", r["n"]))
    peak_head = PEAK_FP64 if head["dtype"] in "dz" else PEAK_FP32
    tname = {"d": "FP64", "s": "FP32", "z": "complex128", "c": "complex64"}
    line = {"metric": f"batch SVD matrices/s (square {head['n']}x{head['n']} "
                      f"{tname[head['dtype']]}, U[0,1])",
            "value": head["matrices_per_s"], "unit": "matrices/s", "n_gpus": world, "steps": args.steps,
            "warmup": 1, "ms_per_step": head["ms"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"d": "f64", "s": "f32", "z": "c128", "c": "c64"}[head["dtype"]],
            "data": "synthetic",
            "config": {"workload": "square: n x n, entries U[0,1] (complex: U[0,1] + i U[0,1]), "
                                   f"types {args.square_dtypes}, U, Sigma, V; batches of 1,000 matrices "
                                   "(FP64 / complex128 n = 512: 200) unless --batch; median of steps",
                       "flags": args.square_flags,
                       "l2": "L2 flushed (256 MB write) before every timed call"},
            "roofline": {"bound": "alu", "achieved": head["tflops"], "peak": peak_head / 1e12,
                         "unit": "TFLOP/s", "frac": head["tflops"] * 1e12 / peak_head, "traffic": None,
                         "kernel": f"{head['dtype'].upper()} solve at n = {head['n']} (multi-kernel path above "
                                   "~100 columns)",
                         "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz"},
            "roofline_fp32": [{"dtype": r["dtype"], "n": r["n"], "achieved": r["tflops"], "peak": PEAK_FP32 / 1e12,
                               "frac": r["tflops"] * 1e12 / PEAK_FP32} for r in rows if r["dtype"] in "sc"],
            "clocks": sampler.summary(), "results": rows}
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        n0 = min(sizes)
        rng = synth.rng_for(synth.SEED_BASE + 7, n0 * 2)
        mats = [rng.uniform(0, 1, (n0, n0)) for _ in range(min(args.cpu_sample, 64))]
        t0, reps = time.perf_counter(), 0
        while reps == 0 or time.perf_counter() - t0 < 3.0:
            r = oracle.default().gesvj(mats)
            reps += 1
        dt_ = time.perf_counter() - t0
        line["cpu_baseline"] = {"value": reps * len(mats) / dt_, "unit": "matrices/s", "cores": r["threads"],
                                "kind": "oracle",
                                "sample": f"{len(mats)} FP64 {n0}x{n0} U[0,1] matrices of the workload's recipe, "
                                          f"{reps} passes, Alg. 2 in FP64, OpenMP over matrices ({dt_:.1f} s)"}
    if rank == 0:
        print(json.dumps(line), flush=True)


def config_dict(world, per_rank):
    return {"workload": "tall128x64: 10,000 FP64 (sigma geometric 1..1e-6) + 10,000 FP32 "
                        "(1..1e-3) matrices 128x64 = Q1 diag(sigma) Q2^T, Haar Q1, Q2",
            "m": M, "n": N, "nb": NB, "matrices_per_rank": per_rank, "tol": f"{TOL_K} u",
            "jobs": "U, Sigma, V", "l2": "inputs (983 MB per rank) larger than L2 (129 MB)",
            "parallelism": f"replicas x{world} (independent matrices per rank)"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--batch", type=int, default=BATCH, help="matrices per precision per rank")
    ap.add_argument("--cpu-sample", type=int, default=3000, help="oracle sample per precision")
    ap.add_argument("--ref-sample", type=int, default=512, help="reference arm: matrices per precision per step")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 baseline path")
    ap.add_argument("--ladder", action="store_true", help="also time Design-2/3/4 (multi-kernel)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision FP64 leg")
    ap.add_argument("--workload", default="tall128x64",
                    choices=["tall128x64", "square32", "uneven", "serving", "tallskinny", "mixed96", "square"],
                    help="tall128x64 (default); square32: 1,000 FP64 32x32 N(0,1), nb = 8, tol = n u, "
                         "batched against the plain path; uneven: 10,000 FP32 + 10,000 complex64 matrices, "
                         "m ~ U{8..512}, n ~ U{8..m}, one persistent launch per type; serving: a Poisson "
                         "stream of single-matrix requests at the continuous-batching server; tallskinny: "
                         "n = 16, m = 100..2000, with and without QR pre-processing; mixed96: the clustered "
                         "96x96 FP64/complex128 set, mixed precision against native FP64; square: n x n "
                         "U[0,1] batches, n = 64..512")
    ap.add_argument("--sizes", type=int, nargs="*", default=None, help="square: the sizes n")
    ap.add_argument("--square-flags", type=int, default=0, help="square: bsvd_opts.flags of every solve")
    ap.add_argument("--square-dtypes", default="dsc", help="square: types to run, of 'd', 's', 'z' and 'c'")
    ap.add_argument("--rate", type=float, default=0.0, help="serving: arrivals per second (default 50,000)")
    ap.add_argument("--seconds", type=float, default=0.0, help="serving: stream length (default 10 s)")
    ap.add_argument("--drain", type=float, default=10.0, help="serving: seconds to drain after arrivals")
    ap.add_argument("--arena-gb", type=float, default=40.0, help="serving: device-memory budget")
    ap.add_argument("--big-flags", type=int, default=0, help="serving: flags added to multi-kernel batches")
    ap.add_argument("--max-big-batch", type=int, default=0, help="serving: requests per multi-kernel batch")
    ap.add_argument("--big-k-fp64", type=int, default=128,
                    help="serving: columns above which FP64 requests take the multi-kernel path (0: big_k, 256)")
    ap.add_argument("--fp64-prec", default="mixed", choices=["native", "mixed"],
                    help="serving: precision path of large FP64 requests (FP64 accuracy either way)")
    ap.add_argument("--sweep-rates", type=float, nargs="*", default=[25, 50, 100, 200])
    ap.add_argument("--sweep-seconds", type=float, default=4.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-variants", action="store_true", help="mixed96: skip the optional mixed variants")
    ap.add_argument("--uneven-flags", type=int, default=UNEVEN_FLAGS,
                    help="uneven: bsvd_opts.flags of the persistent calls (default: split complex64 k >= 112, FP32 k >= 144)")
    ap.add_argument("--no-autotune", action="store_true", help="uneven: skip the per-bucket autotuning")
    ap.add_argument("--tune-sample", type=int, default=64, help="uneven: autotuning sample per bucket")
    ap.add_argument("--no-per-shape", action="store_true",
                    help="uneven: skip the one-launch-per-shape comparison (thousands of launches)")
    args = ap.parse_args()

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.workload == "square32":
        run_square32(args, rank, world, local)
        return
    if args.workload == "uneven":
        run_uneven(args, rank, world, local)
        return
    if args.workload == "serving":
        run_serving(args, rank, world, local)
        return
    if args.workload == "tallskinny":
        run_tallskinny(args, rank, world, local)
        return
    if args.workload == "mixed96":
        run_mixed96(args, rank, world, local)
        return
    if args.workload == "square":
        run_square(args, rank, world, local)
        return

    import torch
    import paper_2601_17979_gb300 as bsvd
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    bsvd.build()

    A64h, A32h = build_inputs(rank, args.batch)
    B = args.batch
    # column-major device inputs and preallocated outputs
    def to_dev(Ah, dt):
        return torch.from_numpy(Ah).to(dev).transpose(1, 2).contiguous().transpose(1, 2)
    A64 = to_dev(A64h, torch.float64)
    A32 = to_dev(A32h, torch.float32)

    def outputs(dt, rdt):
        return (torch.empty((B, N), dtype=rdt, device=dev), bsvd.empty_column_major(B, M, N, dt, dev),
                bsvd.empty_column_major(B, N, N, dt, dev), torch.empty(B, dtype=torch.int32, device=dev),
                torch.empty(B, dtype=torch.int32, device=dev))
    o64 = outputs(torch.float64, torch.float64)
    o32 = outputs(torch.float32, torch.float32)
    stream = torch.cuda.current_stream(dev)

    def step(ev=None):
        if ev is not None:
            ev[0].record(stream)
        bsvd.gesvj(A64, nb=NB, tol=TOL_K * U64, out=o64)
        if ev is not None:
            ev[1].record(stream)
        bsvd.gesvj(A32, nb=NB, tol=TOL_K * U32, out=o32)
        if ev is not None:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(gpu_uuid(torch, dev))
    barrier()
    with sampler:
        t_start = torch.cuda.Event(enable_timing=True)
        t_end = torch.cuda.Event(enable_timing=True)
        t_start.record(stream)
        for s in range(args.steps):
            step(evs[s])
        t_end.record(stream)
        barrier()
    total_ms = t_start.elapsed_time(t_end)
    k64 = [e[0].elapsed_time(e[1]) for e in evs]
    k32 = [e[1].elapsed_time(e[2]) for e in evs]
    ms_step = max_over_ranks(total_ms / args.steps, dist, dev)
    value = 2 * B * world / (ms_step * 1e-3)

    # results of the last step: convergence and a bounds check on a sample
    info64, sw64 = o64[3].cpu().numpy(), o64[4].cpu().numpy()
    info32, sw32 = o32[3].cpu().numpy(), o32[4].cpu().numpy()
    flops64 = matrix_flops(M, N, NB, sw64)
    flops32 = matrix_flops(M, N, NB, sw32)
    t64 = float(np.mean(k64)) * 1e-3
    t32 = float(np.mean(k32)) * 1e-3
    # sampled results against the FP64 oracle (sigma) and the residual and
    # orthogonality bounds, in each precision's own unit roundoff
    samp = list(range(0, B, max(1, B // 8)))
    ref64 = oracle_reference([A64h[i] for i in samp], TOL_K * U64)
    ref32 = oracle_reference([A32h[i] for i in samp], TOL_K * U64)

    def sampled(o):
        return ([o[0][i].cpu().numpy() for i in samp], [o[1][i].cpu().numpy() for i in samp],
                [o[2][i].cpu().numpy() for i in samp])
    worst = {"fp64": accuracy_over_bounds([A64h[i] for i in samp], *sampled(o64), ref64, U64),
             "fp32": accuracy_over_bounds([A32h[i] for i in samp], *sampled(o32), ref32, U32)}

    line = {
        "metric": "batch SVD matrices/s (tall 128x64, FP64+FP32)", "value": value, "unit": "matrices/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32",
        "data": "synthetic", "config": config_dict(world, 2 * B),
        "gpu_launches": 2 * args.steps,
        "fp64": {"matrices_per_s": B / t64, "kernel_ms": t64 * 1e3, "gflops": flops64 / t64 / 1e9,
                 "sweeps_mean": float(sw64.mean()), "sweeps_max": int(sw64.max()),
                 "info_nonzero": int((info64 != 0).sum())},
        "fp32": {"matrices_per_s": B / t32, "kernel_ms": t32 * 1e3, "gflops": flops32 / t32 / 1e9,
                 "sweeps_mean": float(sw32.mean()), "sweeps_max": int(sw32.max()),
                 "info_nonzero": int((info32 != 0).sum()),
                 "roofline": {"bound": "alu", "achieved": flops32 / t32 / 1e12, "peak": PEAK_FP32 / 1e12,
                              "unit": "TFLOP/s", "frac": flops32 / t32 / PEAK_FP32,
                              "traffic": measured_traffic("fused", "tall128x64_f32", B)}},
        "roofline": {"bound": "alu", "achieved": flops64 / t64 / 1e12, "peak": PEAK_FP64 / 1e12,
                     "unit": "TFLOP/s", "frac": flops64 / t64 / PEAK_FP64, "traffic": measured_traffic("fused", "tall128x64_f64", B),
                     "kernel": "gesvj_fused_kernel<double,16,2,128>",
                     "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz"},
        "accuracy_worst_over_bound": worst,
        "clocks": sampler.summary(),
    }

    # end to end through the public API with host buffers: the library's
    # host-buffer entry point, which copies chunks in and out on its own
    # streams while other chunks are solved (timed right after the device
    # step, under the same conditions)
    if not args.no_e2e:
        A64p = torch.from_numpy(A64h.transpose(0, 2, 1).copy()).pin_memory().transpose(1, 2)
        A32p = torch.from_numpy(A32h.transpose(0, 2, 1).copy()).pin_memory().transpose(1, 2)

        def host_outputs(dt, rdt):
            return (torch.empty((B, N), dtype=rdt).pin_memory(),
                    torch.empty((B, N, M), dtype=dt).pin_memory().transpose(1, 2),
                    torch.empty((B, N, N), dtype=dt).pin_memory().transpose(1, 2),
                    torch.empty(B, dtype=torch.int32).pin_memory(), torch.empty(B, dtype=torch.int32).pin_memory())
        h64 = host_outputs(torch.float64, torch.float64)
        h32 = host_outputs(torch.float32, torch.float32)
        h2d = A64p.numel() * 8 + A32p.numel() * 4
        d2h = sum(t.numel() * t.element_size() for o in (h64, h32) for t in o)
        w64 = torch.empty(bsvd.host_workspace_bytes(torch.float64, B, M, N, nb=NB), dtype=torch.uint8, device=dev)
        w32 = torch.empty(bsvd.host_workspace_bytes(torch.float32, B, M, N, nb=NB), dtype=torch.uint8, device=dev)

        def e2e_step():
            bsvd.gesvj_host(A64p, nb=NB, tol=TOL_K * U64, out=h64, work=w64, sync=False)
            bsvd.gesvj_host(A32p, nb=NB, tol=TOL_K * U32, out=h32, work=w32, sync=False)
        e2e_step()
        barrier()
        e_sampler = ClockSampler(gpu_uuid(torch, dev))
        with e_sampler:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(args.steps):
                e2e_step()
            b.record(stream)
            barrier()
        e_ms = max_over_ranks(a.elapsed_time(b) / args.steps, dist, dev)
        ok = bool(torch.equal(h64[0], o64[0].cpu()) and torch.equal(h32[0], o32[0].cpu()))
        line["e2e"] = {"value": 2 * B * world / (e_ms * 1e-3), "unit": "matrices/s",
                       "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                       "ms_per_step": e_ms, "api": "gesvj_host (bsvd_?gesvj_strided_host)",
                       "same_sigma_as_device_call": ok, "clocks": e_sampler.summary()}
        line["gpu_launches"] += 2 * args.steps * 4

    # The paper's baseline path on the same FP64 batch ("vs plain FP64 Jacobi"):
    # multi-kernel, inner eigensolver to convergence, two-stage update, no masks.
    variants = [("fp64_mixed", dict(prec="mixed"))] if not args.no_mixed else []
    if not args.no_mixed and not args.no_variants:
        # the FP32 sweeps with FP64 rotations and pair test (flags bit 8), and
        # with the Gram and update on the FMA pipes instead of the tensor cores
        variants += [("fp64_mixed_fp64_angles", dict(prec="mixed", flags=256)),
                     ("fp64_mixed_ffma", dict(prec="mixed", flags=128))]
    if not args.no_plain:
        variants.append(("plain_fp64", dict(path="plain")))
    if args.ladder:
        variants += [("design2_fp64", dict(path="plain", inner_sweeps=1)),
                     ("design3_fp64", dict(path="blocked", flags=bsvd.FLAG_NO_MASKS)),
                     ("design4_fp64", dict(path="blocked"))]
    for name, kw in variants:
        nbytes = bsvd.workspace_bytes(torch.float64, [(M, N)], True, batch=B, nb=NB, **kw)
        work = torch.empty(nbytes, dtype=torch.uint8, device=dev)
        barrier()
        v_sampler = ClockSampler(gpu_uuid(torch, dev))
        with v_sampler:
            ts = timed_calls(torch, lambda: bsvd.gesvj(A64, nb=NB, tol=TOL_K * U64, out=o64, work=work, **kw),
                             max(5, min(args.steps, 10)), stream, warmup=1)
        barrier()
        p_ms = statistics.median(ts)
        sw = o64[4].cpu().numpy()
        line[name] = {"matrices_per_s": B / (p_ms * 1e-3), "ms": p_ms, "ms_all": ts,
                      "native_fused_ms_over_this": (t64 * 1e3) / p_ms, "sweeps_mean": float(sw.mean()),
                      "info_nonzero": int((o64[3].cpu().numpy() != 0).sum()),
                      "accuracy_worst_over_bound": accuracy_over_bounds([A64h[i] for i in samp], *sampled(o64),
                                                                        ref64, U64),
                      "clocks": v_sampler.summary()}
        del work

    # the FP32 batch with the Gram and update on the FMA pipes (flags bit 7)
    # instead of the tensor cores, for comparison
    if not args.no_variants:
        barrier()
        f_sampler = ClockSampler(gpu_uuid(torch, dev))
        with f_sampler:
            ts = timed_calls(torch, lambda: bsvd.gesvj(A32, nb=NB, tol=TOL_K * U32, out=o32, flags=128),
                             max(5, min(args.steps, 10)), stream, warmup=1)
        f_ms = statistics.median(ts)
        sw = o32[4].cpu().numpy()
        line["fp32_ffma"] = {"matrices_per_s": B / (f_ms * 1e-3), "ms": f_ms, "sweeps_mean": float(sw.mean()),
                             "tensor_core_ms_over_this": t32 * 1e3 / f_ms,
                             "info_nonzero": int((o32[3].cpu().numpy() != 0).sum()),
                             "accuracy_worst_over_bound": accuracy_over_bounds(
                                 [A32h[i] for i in samp], *sampled(o32), ref32, U32),
                             "clocks": f_sampler.summary()}

    # CPU oracle baseline on a bounded sample (rank 0, N = 1 only)
    if rank == 0 and world == 1 and not args.no_cpu:
        import oracle
        S = min(args.cpu_sample, B)
        O = oracle.default()
        t0 = time.perf_counter()
        r1 = O.gesvj([A64h[i] for i in range(S)], tol=TOL_K * U64)
        r2 = O.gesvj([A32h[i] for i in range(S)], tol=TOL_K * U64)
        dt = time.perf_counter() - t0
        fl = oracle_flops(M, N, r1["sweeps"]) + oracle_flops(M, N, r2["sweeps"])
        line["cpu_baseline"] = {
            "value": 2 * S / dt, "unit": "matrices/s", "cores": r1["threads"], "kind": "oracle",
            "sample": f"first {S} FP64 + {S} FP32 matrices of the same workload, Alg. 2 in FP64, "
                      f"OpenMP over matrices ({dt:.1f} s)", "gflops": fl / dt / 1e9}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
