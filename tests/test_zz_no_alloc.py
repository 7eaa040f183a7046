"""The FP64 entry point that allocates nothing (needs a GB300).

bsvd_dgesvj_strided_noalloc serves callers that cannot allocate device
memory: it keeps the multi-kernel path's workspace in a static device array.
These tests call it through the C-ABI and check, on two calls in a row, that
it returns what the regular entry point returns with a caller-allocated
workspace, within the bounds the other parity tests use; and that a batch
beyond the array's capacity is refused cleanly.  This file is collected last
on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

import __graft_entry__  # noqa: F401
import paper_2601_17979_gb300 as bsvd
import synth
from oracle import checks
from paper_2601_17979_gb300 import binding

pytestmark = pytest.mark.gpu

U = 2.0 ** -53
M, N = 128, 64


@pytest.fixture(scope="module")
def lib():
    __graft_entry__.build()
    L = bsvd.load()
    P, I, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong
    L.bsvd_dgesvj_strided_noalloc.argtypes = [P, I, I, I, I, I, P, I, LL, P, LL, P, I, LL, P, I, LL,
                                              P, P, ctypes.POINTER(binding.Opts), P]
    return L


def outputs(B):
    dev = torch.device("cuda")
    return (torch.empty((B, N), dtype=torch.float64, device=dev),
            torch.empty((B, N, M), dtype=torch.float64, device=dev),     # U column-major
            torch.empty((B, N, N), dtype=torch.float64, device=dev),     # V column-major
            torch.full((B,), -7, dtype=torch.int32, device=dev),
            torch.full((B,), -7, dtype=torch.int32, device=dev))


def call_noalloc(L, At, out, opts):
    B = At.shape[0]
    S, U_, V, info, sw = out
    return L.bsvd_dgesvj_strided_noalloc(
        bsvd.handle(), 1, 1, B, M, N, At.data_ptr(), M, M * N, S.data_ptr(), N, U_.data_ptr(), M,
        M * N, V.data_ptr(), N, N * N, info.data_ptr(), sw.data_ptr(), ctypes.byref(opts),
        torch.cuda.current_stream().cuda_stream)


def call_regular(L, At, out, opts):
    B = At.shape[0]
    S, U_, V, info, sw = out
    nbytes = binding.workspace_bytes(torch.float64, [(M, N)], True, batch=B, path="blocked")
    work = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    st = L.bsvd_dgesvj_strided(
        bsvd.handle(), 1, 1, B, M, N, At.data_ptr(), M, M * N, S.data_ptr(), N, U_.data_ptr(), M,
        M * N, V.data_ptr(), N, N * N, info.data_ptr(), sw.data_ptr(), work.data_ptr(), nbytes,
        ctypes.byref(opts), torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    return st


def host(out):
    S, U_, V, info, sw = out
    return (S.cpu().numpy(), U_.transpose(1, 2).cpu().numpy(), V.transpose(1, 2).cpu().numpy(),
            info.cpu().numpy(), sw.cpu().numpy())


def test_noalloc_matches_regular_entry_point_twice(lib):
    opts = binding.make_opts(nb=16, path="blocked")
    for call, start in enumerate((0, 500)):          # two calls in a row, different inputs
        mats = synth.uniform_batch("tall128x64_f64", 48, start=start)
        At = torch.from_numpy(mats.transpose(0, 2, 1).copy()).cuda()    # column-major storage
        got, ref = outputs(48), outputs(48)
        assert call_noalloc(lib, At, got, opts) == 0
        torch.cuda.synchronize()
        assert call_regular(lib, At, ref, opts) == 0
        S1, U1, V1, i1, w1 = host(got)
        S2, U2, V2, i2, w2 = host(ref)
        assert (i1 == 0).all() and np.array_equal(i1, i2), (call, i1)
        for b in range(48):
            # sigma against the regular entry point, vectors through the bounds
            assert np.abs(S1[b] - S2[b]).max() <= 50 * N * U * S2[b].max(), (call, b)
            meas = checks.measures(mats[b], S1[b], U1[b], V1[b], S2[b])
            assert checks.violations(meas, U) == [], (call, b, meas)


def test_noalloc_stale_scratch_from_a_different_call(lib):
    """A first call leaves the array in another state (a larger batch stopped
    after one sweep, so its status words and pair flags are still set); the
    next, smaller call must start from scratch: converged, and sigma within
    50 n u of the FP64 oracle, residual and orthogonality within their bounds."""
    import oracle
    big = synth.uniform_batch("tall128x64_f64", 150, start=2000)
    Ab = torch.from_numpy(big.transpose(0, 2, 1).copy()).cuda()
    out = outputs(150)
    assert call_noalloc(lib, Ab, out, binding.make_opts(nb=16, max_sweeps=1, path="blocked")) == 0
    torch.cuda.synchronize()
    assert (out[3].cpu().numpy() == 1).all()        # not converged after 1 sweep: info = 1
    mats = synth.uniform_batch("tall128x64_f64", 24, start=3000)
    At = torch.from_numpy(mats.transpose(0, 2, 1).copy()).cuda()
    got = outputs(24)
    assert call_noalloc(lib, At, got, binding.make_opts(nb=16, path="blocked")) == 0
    torch.cuda.synchronize()
    S1, U1, V1, i1, w1 = host(got)
    assert (i1 == 0).all(), i1
    ref = oracle.gesvj(list(mats), tol=30 * U)
    for b in range(24):
        meas = checks.measures(mats[b], S1[b], U1[b], V1[b], ref["S"][b])
        assert checks.violations(meas, U) == [], (b, meas)


def test_noalloc_rejects_batches_beyond_capacity(lib):
    B = 204                                          # needs more than the 32 MiB array
    At = torch.zeros((B, N, M), dtype=torch.float64, device="cuda")
    out = outputs(B)
    st = call_noalloc(lib, At, out, binding.make_opts(nb=16))
    assert st == -2                                  # BSVD_ERR_WORKSPACE, nothing launched
    torch.cuda.synchronize()
    assert (out[3].cpu().numpy() == -7).all()
