"""The C-ABI library loads, exports every declared symbol, and rejects bad
arguments on the host with the documented argument positions (no GPU needed:
argument checks run before any CUDA call)."""
import ctypes
import os
import re

import pytest

import __graft_entry__  # noqa: F401  (puts the repo root on sys.path)
import paper_2601_17979_gb300 as bsvd
from paper_2601_17979_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    bsvd.build()
    return bsvd.load()


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "bsvd.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bsvd_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(L):
    syms = declared_symbols()
    assert len(syms) >= 15
    missing = [s for s in syms if not hasattr(L, s)]
    assert missing == []
    assert sorted(binding.EXPORTS) == syms


def test_version_and_status_strings(L):
    assert L.bsvd_version() == 1
    for st in (0, -1, -2, -3, -4, -5, -6, -7):
        assert L.bsvd_status_string(st).startswith(b"BSVD_")


def call_strided(L, t="d", **kw):
    a = dict(jobu=1, jobv=1, batch=2, m=8, n=4, dA=16, lda=8, sA=32, dS=16, sS=4, dU=16, ldu=8,
             sU=32, dV=16, ldv=4, sV=16, info=16, sweeps=None, work=None, wbytes=0)
    a.update(kw)
    o = binding.make_opts(**kw.get("opts", {}))
    f = getattr(L, f"bsvd_{t}gesvj_strided")
    return f(bsvd.handle(), a["jobu"], a["jobv"], a["batch"], a["m"], a["n"], a["dA"], a["lda"],
             a["sA"], a["dS"], a["sS"], a["dU"], a["ldu"], a["sU"], a["dV"], a["ldv"], a["sV"],
             a["info"], a["sweeps"], a["work"], a["wbytes"], ctypes.byref(o), None)


@pytest.mark.parametrize("field,value,pos", [
    ("jobu", 7, 2), ("jobv", -1, 3), ("batch", -1, 4), ("m", -2, 5), ("n", -1, 6),
    ("dA", None, 7), ("lda", 7, 8), ("sA", 31, 9), ("dS", None, 10), ("sS", 3, 11),
    ("dU", None, 12), ("ldu", 7, 13), ("sU", 31, 14), ("dV", None, 15), ("ldv", 3, 16),
    ("sV", 15, 17), ("info", None, 18),
])
def test_strided_invalid_argument_positions(L, field, value, pos):
    st = call_strided(L, **{field: value})
    assert st == -1
    assert L.bsvd_last_arg(bsvd.handle()) == pos


def test_invalid_options(L):
    assert call_strided(L, opts=dict(nb=-1)) == -1
    assert L.bsvd_last_arg(bsvd.handle()) == 22
    # mixed precision exists for FP64 output only
    assert call_strided(L, t="s", opts=dict(prec="mixed")) == -1
    assert L.bsvd_last_arg(bsvd.handle()) == 22


def test_empty_batch_is_a_noop(L):
    assert call_strided(L, batch=0, dA=None, dS=None, dU=None, dV=None, info=None) == 0


def test_jobs_none_skip_vector_checks(L):
    # with jobu = jobv = NONE the U/V pointers and leading dimensions are ignored
    st = call_strided(L, jobu=0, jobv=0, dU=None, ldu=0, sU=0, dV=None, ldv=0, sV=0, batch=-3)
    assert st == -1 and L.bsvd_last_arg(bsvd.handle()) == 4


def test_workspace_query(L):
    h = bsvd.handle()
    n = ctypes.c_size_t(123)
    m_arr = (ctypes.c_int * 3)(4, 5, 6)
    o = binding.make_opts()
    assert L.bsvd_gesvj_workspace(h, b"d", 3, m_arr, m_arr, 1, 1, 1, ctypes.byref(o), ctypes.byref(n)) == 0
    assert n.value == 0
    assert L.bsvd_gesvj_workspace(h, b"z", 3, m_arr, m_arr, 0, 1, 1, ctypes.byref(o), ctypes.byref(n)) == 0
    assert n.value >= 4 * 3 * 4 and n.value % 256 == 0
    assert L.bsvd_gesvj_workspace(h, b"q", 3, m_arr, m_arr, 0, 1, 1, ctypes.byref(o), ctypes.byref(n)) == -1
    assert L.bsvd_last_arg(h) == 2
    # shapes that do not fit on chip, and the paper's baseline path, need workspace
    big = (ctypes.c_int * 1)(1000)
    assert L.bsvd_gesvj_workspace(h, b"d", 2, big, big, 1, 1, 1, ctypes.byref(o), ctypes.byref(n)) == 0
    assert n.value > 2 * 1000 * 1000 * 8
    m64 = (ctypes.c_int * 1)(64)
    plain = binding.make_opts(path="plain")
    assert L.bsvd_gesvj_workspace(h, b"d", 4, m64, m64, 1, 1, 1, ctypes.byref(plain), ctypes.byref(n)) == 0
    assert n.value > 4 * 3 * 64 * 64 * 8
    mixed = binding.make_opts(prec="mixed")
    assert L.bsvd_gesvj_workspace(h, b"d", 4, m64, m64, 1, 1, 1, ctypes.byref(mixed), ctypes.byref(n)) == 0
    assert n.value > 4 * (64 * 64 * (4 + 4 + 8 * 4))
    fused = binding.make_opts(path="fused")
    assert L.bsvd_gesvj_workspace(h, b"z", 1, big, big, 1, 1, 1, ctypes.byref(fused), ctypes.byref(n)) == -5


def test_batched_invalid_arguments(L):
    h = bsvd.handle()
    B = 2
    ms = (ctypes.c_int * B)(8, 6)
    ns = (ctypes.c_int * B)(4, 6)
    lda_bad = (ctypes.c_int * B)(8, 5)
    ld = (ctypes.c_int * B)(8, 6)
    o = binding.make_opts()
    f = L.bsvd_dgesvj_batched
    st = f(h, 1, 1, B, ms, ns, 16, lda_bad, 16, 16, ld, 16, ld, 16, None, 16, 4096, ctypes.byref(o), None)
    assert st == -1 and L.bsvd_last_arg(h) == 8
    # workspace too small
    st = f(h, 1, 1, B, ms, ns, 16, ld, 16, 16, ld, 16, ns, 16, None, 16, 8, ctypes.byref(o), None)
    assert st == -2


def test_missing_library_fails_loudly(monkeypatch, tmp_path):
    # the binding never falls back to another implementation
    monkeypatch.setattr(binding, "_lib", None)
    monkeypatch.setattr(binding._build, "LIB", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="not built"):
        binding.load()


def test_server_host_argument_checks(L):
    """Server calls reject bad arguments before touching the device."""
    srv = ctypes.c_void_p()
    big = 1 << 30
    assert L.bsvd_server_create(None, big, None, ctypes.byref(srv)) == -1           # no arena
    assert L.bsvd_server_create(0x100001, big, None, ctypes.byref(srv)) == -1       # misaligned
    assert L.bsvd_server_create(0x100000, 4096, None, ctypes.byref(srv)) == -1      # under 1 MiB
    o = binding.ServerOpts()
    o.max_inflight = 65
    assert L.bsvd_server_create(0x100000, big, ctypes.byref(o), ctypes.byref(srv)) == -1
    o.max_inflight, o.max_batch = 4, -1
    assert L.bsvd_server_create(0x100000, big, ctypes.byref(o), ctypes.byref(srv)) == -1
    assert L.bsvd_server_create(0x100000, big, None, None) == -1
    rid = ctypes.c_longlong()
    assert L.bsvd_server_submit(None, b"d", 4, 4, 0x1000, 4, 1, 1, ctypes.byref(rid)) == -1
    assert L.bsvd_server_test(None, 1) == -1
    assert L.bsvd_server_release(None, 1) == -1
    assert L.bsvd_server_pause(None, 1) == -1
    assert L.bsvd_server_cancel(None) == -1
    assert L.bsvd_server_destroy(None) == -1
    assert L.bsvd_server_collect(None, 4, 1, None, None, None, None, None, None) == -1
    assert L.bsvd_server_clock() > 0


def test_qr_workspace_query(L):
    """QR pre-processing needs workspace (reflectors, R, U_R) even where the
    on-chip path alone needs none; the pointer-array form refuses it."""
    plain = binding.workspace_bytes("d", [(1000, 16)], True, batch=10)
    qr = binding.workspace_bytes("d", [(1000, 16)], True, batch=10, flags=binding.FLAG_QR)
    assert qr >= 10 * (1000 * 16 + 16 + 16 * 16 + 16 * 16) * 8 > plain
    with pytest.raises(binding.BsvdError, match="NOT_IMPLEMENTED"):
        binding.workspace_bytes("d", [(1000, 16), (900, 16)], False, flags=binding.FLAG_QR)
    with pytest.raises(binding.BsvdError, match="NOT_IMPLEMENTED"):
        binding.workspace_bytes("d", [(1000, 16)], True, batch=2, flags=binding.FLAG_QR, prec="mixed")


def test_flat_outputs_layout():
    """The pointer-array binding puts every matrix's output in one allocation:
    each output starts 256 bytes after a boundary of the previous one's end,
    pointers match the views, and empty outputs take no room."""
    import numpy as np
    import torch
    from paper_2601_17979_gb300.binding import _flat_outputs
    m = np.array([5, 0, 7, 3, 64]); k = np.minimum(m, np.array([3, 4, 7, 1, 64]))
    for dt in (torch.float32, torch.complex128):
        flat, off, ptr = _flat_outputs(m * k, dt, "cpu")
        elt = flat.element_size()
        assert ((off * elt) % 256 == 0).all()
        ends = off + m * k
        assert (ends[:-1] <= off[1:]).all() and ends[-1] <= flat.numel()
        assert (ptr.numpy() - flat.data_ptr() == off * elt).all()


def test_split_workspace_query(L):
    """Flags bit 6 on a persistent complex64 batch adds the variable-shape
    multi-kernel workspace for the matrices with min(m, n) >= 112 only;
    batches of the other types ignore the flag."""
    h = bsvd.handle()
    n = ctypes.c_size_t()
    ms = (ctypes.c_int * 4)(300, 40, 200, 512)
    ns = (ctypes.c_int * 4)(150, 30, 90, 256)
    pers = binding.make_opts(path="persistent")
    split = binding.make_opts(path="persistent", flags=binding.FLAG_SPLIT_LARGE)
    sizes = {}
    for t in (b"s", b"c", b"d", b"z"):
        for name, o in (("pers", pers), ("split", split)):
            assert L.bsvd_gesvj_workspace(h, t, 4, ms, ns, 0, 1, 1, ctypes.byref(o), ctypes.byref(n)) == 0
            sizes[t, name] = n.value
    # the two large matrices' W, V and finalisation scratch at least
    big = sum(M * N + N * N * 2 + M for M, N in ((300, 150), (512, 256)))
    assert sizes[b"c", "split"] > big * 8
    for t in (b"s", b"d", b"z"):
        assert sizes[t, "split"] == sizes[t, "pers"]
    small = (ctypes.c_int * 2)(100, 60)
    assert L.bsvd_gesvj_workspace(h, b"c", 2, small, small, 0, 1, 1, ctypes.byref(pers), ctypes.byref(n)) == 0
    a = n.value
    assert L.bsvd_gesvj_workspace(h, b"c", 2, small, small, 0, 1, 1, ctypes.byref(split), ctypes.byref(n)) == 0
    assert n.value == a                          # nothing reaches the multi-kernel path


def test_persistent_plan_host_logic():
    """The per-matrix decision of a persistent batch, computed on the host
    (no GPU needed): the block width follows min(m, n) (>= 48: 16, >= 12: 8,
    else 4) unless opts.nb is given; small matrices keep W and V in shared
    memory, large ones in global slots; empty matrices are not planned;
    with flags bit 6 complex64 sends min(m, n) >= 112 to the multi-kernel
    batch, and with bits 6 and 10 real FP32 sends min(m, n) >= 144."""
    import numpy as np
    import paper_2601_17979_gb300 as bsvd
    shapes = [(8, 8), (30, 20), (100, 64), (512, 400), (0, 5), (12, 300), (47, 47)]
    nb, where, launches = bsvd.persistent_plan("s", shapes)
    assert nb.tolist() == [4, 8, 16, 16, 0, 8, 8]
    assert where[0] == 1 and where[1] == 1 and where[2] == 1 and where[3] == 0 and where[4] == -1
    assert launches == len({(int(a), int(b)) for a, b in zip(nb, where) if b >= 0})
    nb2, where2, _ = bsvd.persistent_plan("s", shapes, nb=8)
    assert all(x == 8 for x, w in zip(nb2, where2) if w >= 0)
    _, where3, launches3 = bsvd.persistent_plan("s", shapes, flags=bsvd.FLAG_NO_ONCHIP)
    assert set(where3.tolist()) == {0, -1}
    _, where4, _ = bsvd.persistent_plan("c", [(300, 150), (40, 30), (128, 128), (112, 300), (200, 111)],
                                        flags=bsvd.FLAG_SPLIT_LARGE)
    assert where4.tolist()[0] == 2 and where4.tolist()[2] == 2 and where4.tolist()[3] == 2
    assert where4.tolist()[1] == 1 and where4.tolist()[4] in (0, 1)
    split32 = bsvd.FLAG_SPLIT_LARGE | bsvd.FLAG_SPLIT_F32
    _, where5, _ = bsvd.persistent_plan("s", [(300, 144), (300, 143), (144, 144), (500, 160)], flags=split32)
    assert where5.tolist()[0] == 2 and where5.tolist()[2] == 2 and where5.tolist()[3] == 2
    assert where5.tolist()[1] in (0, 1)
    _, where6, _ = bsvd.persistent_plan("s", [(300, 200)], flags=bsvd.FLAG_SPLIT_LARGE)   # FP32 needs bit 10
    assert where6.tolist()[0] in (0, 1)
    assert np.all(nb >= 0)


def test_flag_range(L):
    """bsvd_opts.flags takes bits 0-12 (bit 12: three kernels per round
    instead of the pair step); a higher bit is an invalid option."""
    assert binding.workspace_bytes("s", [(300, 200)], True, batch=2, flags=8191) > 0
    # the pair step and the three kernels share one workspace layout
    assert (binding.workspace_bytes("s", [(300, 200)], True, batch=2, flags=4096)
            == binding.workspace_bytes("s", [(300, 200)], True, batch=2))
    with pytest.raises(binding.BsvdError, match="INVALID"):
        binding.workspace_bytes("s", [(300, 200)], True, batch=2, flags=8192)
