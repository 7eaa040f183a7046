"""The host-buffer entry points (needs a GB300): a batch in host memory is cut
into chunks that are copied in, solved and copied out on overlapping streams.
Per-matrix arithmetic is that of the device call, so the results match it bit
for bit."""
import numpy as np
import pytest
import torch

import __graft_entry__  # noqa: F401
import paper_2601_17979_gb300 as bsvd

pytestmark = pytest.mark.gpu

DT = {"s": torch.float32, "d": torch.float64, "c": torch.complex64, "z": torch.complex128}


@pytest.fixture(scope="module", autouse=True)
def built():
    __graft_entry__.build()
    assert torch.cuda.is_available()


def rand(batch, m, n, t, seed):
    g = torch.Generator().manual_seed(seed)
    x = torch.randn(batch, m, n, generator=g, dtype=torch.float64)
    if t in "cz":
        x = torch.complex(x, torch.randn(batch, m, n, generator=g, dtype=torch.float64))
    return x.to(DT[t])


@pytest.mark.parametrize("t", list("sdcz"))
@pytest.mark.parametrize("batch,m,n", [(2000, 64, 32), (7, 40, 24), (1, 30, 50), (700, 20, 33)])
def test_host_pipeline_matches_device_call(t, batch, m, n):
    A = rand(batch, m, n, t, batch + m + n)
    dev = bsvd.gesvj(A.cuda())
    torch.cuda.synchronize()
    host = bsvd.gesvj_host(A)
    assert not host.S.is_cuda and host.S.is_pinned()
    assert torch.equal(host.info, dev.info.cpu()) and torch.equal(host.sweeps, dev.sweeps.cpu())
    assert torch.equal(host.S, dev.S.cpu())
    assert torch.equal(host.U, dev.U.cpu()) and torch.equal(host.V, dev.V.cpu())


def test_host_pipeline_jobs_and_strides():
    A = rand(1500, 50, 20, "d", 5)
    dev = bsvd.gesvj(A.cuda(), compute_u=False)
    r = bsvd.gesvj_host(A, compute_u=False)
    assert r.U is None and torch.equal(r.S, dev.S.cpu()) and torch.equal(r.V, dev.V.cpu())
    # a row-major, pageable input: the binding makes the page-locked column-major copy
    B = torch.randn(900, 24, 18, dtype=torch.float64)
    r2 = bsvd.gesvj_host(B)
    d2 = bsvd.gesvj(B.cuda())
    assert torch.equal(r2.S, d2.S.cpu()) and torch.equal(r2.U, d2.U.cpu())


def test_host_pipeline_workspace_too_small():
    A = rand(100, 30, 20, "d", 6)
    with pytest.raises(bsvd.BsvdError, match="WORKSPACE"):
        bsvd.gesvj_host(A, work=torch.empty(256, dtype=torch.uint8, device="cuda"))
