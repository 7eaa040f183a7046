"""Autotuner and CUDA-graph sweeps (needs a GB300)."""
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


def test_autotune_picks_a_converging_candidate_and_auto_follows_it():
    mats = synth.uniform_batch("tall128x64_f32", 256)
    A = torch.from_numpy(mats).cuda()
    best, times = bsvd.autotune(A)
    assert best["path"] in ("fused", "blocked") and best["nb"] in (4, 8, 16, 32)
    assert (best["path"], best["nb"]) in times
    assert times[(best["path"], best["nb"])] == min(times.values())
    assert len(times) >= 4
    # AUTO now follows the tuned choice: the workspace query reflects the path
    need = bsvd.workspace_bytes(torch.float32, [(128, 64)], True, batch=256)
    assert (need > 0) == (best["path"] == "blocked")
    r = bsvd.gesvj(A)
    torch.cuda.synchronize()
    ref = oracle.gesvj([mats[i] for i in range(8)], tol=30 * 2.0 ** -53)
    for i in range(8):
        meas = checks.measures(mats[i], r.S[i].cpu().numpy(), r.U[i].cpu().numpy(), r.V[i].cpu().numpy(),
                               ref["S"][i])
        assert checks.violations(meas, checks.U32) == [], meas


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32, torch.complex64])
def test_graph_replay_equals_direct_launches(dtype):
    rng = np.random.default_rng(9)
    x = rng.standard_normal((6, 150, 90))
    if dtype.is_complex:
        x = x + 1j * rng.standard_normal((6, 150, 90))
    A = torch.from_numpy(x).to(dtype).cuda()
    r1 = bsvd.gesvj(A, path="blocked", nb=16)
    r2 = bsvd.gesvj(A, path="blocked", nb=16, flags=bsvd.FLAG_NO_GRAPH)
    torch.cuda.synchronize()
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)
    assert (r1.info == 0).all()


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("max_sweeps", [1, 3])
def test_device_sweep_loop_stops_at_max_sweeps(dtype, max_sweeps):
    """The graph's device-side sweep loop runs at most max_sweeps sweeps: a
    batch that needs more ends with info = sweeps = max_sweeps, the same
    bits as issuing max_sweeps sweeps from the host (graphs off)."""
    rng = np.random.default_rng(31)
    A = torch.from_numpy(rng.standard_normal((5, 140, 100))).to(dtype).cuda()
    r1 = bsvd.gesvj(A, path="blocked", nb=16, max_sweeps=max_sweeps)
    r2 = bsvd.gesvj(A, path="blocked", nb=16, max_sweeps=max_sweeps, flags=bsvd.FLAG_NO_GRAPH)
    torch.cuda.synchronize()
    assert (r1.info == max_sweeps).all() and (r1.sweeps == max_sweeps).all()
    for a, b in zip(r1, r2):
        assert torch.equal(a, b)
