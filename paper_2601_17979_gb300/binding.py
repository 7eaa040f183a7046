"""Python binding of libbsvd (ctypes): argument marshalling only.

Every step of the SVD runs in the CUDA kernels behind the C-ABI declared in
``include/bsvd.h``; this module allocates outputs with torch, passes device
pointers and the current CUDA stream, and checks status codes.  There is no
CPU fallback: if the library is missing or no CUDA device is present the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading
from collections import namedtuple

import numpy as np
import torch

from . import buildlib as _build

BSVD_OK = 0
STATUS = {0: "BSVD_OK", -1: "BSVD_ERR_INVALID", -2: "BSVD_ERR_WORKSPACE", -3: "BSVD_ERR_CUDA",
          -4: "BSVD_ERR_TIMEOUT", -5: "BSVD_ERR_NOT_IMPLEMENTED", -6: "BSVD_ERR_NOMEM",
          -7: "BSVD_ERR_CANCELLED"}
PATHS = {"auto": 0, "fused": 1, "plain": 2, "blocked": 3, "persistent": 4}
PATH_NAMES = {v: k for k, v in PATHS.items()}
FLAG_NO_V_CORRECTION, FLAG_TWO_STAGE, FLAG_NO_MASKS, FLAG_NO_GRAPH, FLAG_SYNC_CHECK, FLAG_QR = 1, 2, 4, 8, 16, 32
FLAG_SPLIT_LARGE = 64
FLAG_F32_FFMA, FLAG_WIDE_ANGLES, FLAG_NO_ONCHIP, FLAG_SPLIT_F32, FLAG_HOST_LOOP = 128, 256, 512, 1024, 2048
FLAG_THREE_KERNELS = 4096
DTYPES = {torch.float32: "s", torch.float64: "d", torch.complex64: "c", torch.complex128: "z"}
REAL = {torch.float32: torch.float32, torch.float64: torch.float64,
        torch.complex64: torch.float32, torch.complex128: torch.float64}

SVDResult = namedtuple("SVDResult", "S U V info sweeps")

EXPORTS = (
    "bsvd_create", "bsvd_destroy", "bsvd_status_string", "bsvd_last_arg", "bsvd_last_cuda",
    "bsvd_version", "bsvd_gesvj_workspace",
    "bsvd_sgesvj_strided", "bsvd_dgesvj_strided", "bsvd_cgesvj_strided", "bsvd_zgesvj_strided",
    "bsvd_sgesvj_batched", "bsvd_dgesvj_batched", "bsvd_cgesvj_batched", "bsvd_zgesvj_batched",
    "bsvd_dgesvj_strided_noalloc", "bsvd_autotune_workspace", "bsvd_autotune", "bsvd_persistent_plan",
    "bsvd_autotune_batched_workspace", "bsvd_autotune_batched",
    "bsvd_gesvj_host_workspace", "bsvd_sgesvj_strided_host", "bsvd_dgesvj_strided_host",
    "bsvd_cgesvj_strided_host", "bsvd_zgesvj_strided_host",
    "bsvd_server_clock", "bsvd_server_create", "bsvd_server_submit", "bsvd_server_replay",
    "bsvd_server_test", "bsvd_server_wait", "bsvd_server_result", "bsvd_server_fetch",
    "bsvd_server_release", "bsvd_server_collect", "bsvd_server_cancel", "bsvd_server_pause",
    "bsvd_server_stats",
    "bsvd_server_destroy",
)


class BsvdError(RuntimeError):
    def __init__(self, status: int, where: str, arg: int = 0, cuda: int = 0):
        self.status, self.arg, self.cuda = status, arg, cuda
        extra = f" (argument {arg})" if arg else ""
        extra += f" (cudaError {cuda})" if status == -3 else ""
        super().__init__(f"{where}: {STATUS.get(status, status)}{extra}")


class ServerOpts(ctypes.Structure):
    _fields_ = [("max_inflight", ctypes.c_int), ("max_batch", ctypes.c_int), ("big_k", ctypes.c_int),
                ("max_big_batch", ctypes.c_int), ("fp64_prec", ctypes.c_int), ("big_flags", ctypes.c_int),
                ("big_k_fp64", ctypes.c_int), ("reserved", ctypes.c_int * 1)]


class Opts(ctypes.Structure):
    _fields_ = [("nb", ctypes.c_int), ("max_sweeps", ctypes.c_int), ("tol", ctypes.c_double),
                ("inner_sweeps", ctypes.c_int), ("path", ctypes.c_int), ("flags", ctypes.c_int),
                ("prec", ctypes.c_int), ("reserved", ctypes.c_int * 5)]


_lock = threading.Lock()
_lib = None
_handles = threading.local()


def lib_path() -> str:
    return _build.LIB


def load() -> ctypes.CDLL:
    """Load libbsvd.so (built by ``build.build()``); raise if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"{_build.LIB} is not built; run paper_2601_17979_gb300.build()")
            L = ctypes.CDLL(_build.LIB)
            P, I, LL, SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_longlong, ctypes.c_size_t
            L.bsvd_create.argtypes = [ctypes.POINTER(P)]
            L.bsvd_destroy.argtypes = [P]
            L.bsvd_status_string.argtypes = [I]
            L.bsvd_status_string.restype = ctypes.c_char_p
            L.bsvd_last_arg.argtypes = [P]
            L.bsvd_last_cuda.argtypes = [P]
            L.bsvd_gesvj_workspace.argtypes = [P, ctypes.c_char, I, P, P, I, I, I, ctypes.POINTER(Opts),
                                               ctypes.POINTER(SZ)]
            for t in "sdcz":
                getattr(L, f"bsvd_{t}gesvj_strided").argtypes = [
                    P, I, I, I, I, I, P, I, LL, P, LL, P, I, LL, P, I, LL, P, P, P, SZ,
                    ctypes.POINTER(Opts), P]
                getattr(L, f"bsvd_{t}gesvj_batched").argtypes = [
                    P, I, I, I, P, P, P, P, P, P, P, P, P, P, P, P, SZ, ctypes.POINTER(Opts), P]
            L.bsvd_autotune_workspace.argtypes = [P, ctypes.c_char, I, I, I, I, I, ctypes.POINTER(Opts),
                                                  ctypes.POINTER(SZ)]
            L.bsvd_gesvj_host_workspace.argtypes = [P, ctypes.c_char, I, I, I, I, I, ctypes.POINTER(Opts),
                                                    ctypes.POINTER(SZ)]
            for t in "sdcz":
                getattr(L, f"bsvd_{t}gesvj_strided_host").argtypes = [
                    P, I, I, I, I, I, P, I, LL, P, LL, P, I, LL, P, I, LL, P, P, P, SZ,
                    ctypes.POINTER(Opts), P]
            L.bsvd_autotune.argtypes = [P, ctypes.c_char, I, I, I, I, I, P, I, LL, P, SZ,
                                        ctypes.POINTER(Opts), ctypes.POINTER(Opts), P, P]
            L.bsvd_persistent_plan.argtypes = [P, ctypes.c_char, I, P, P, I, I, ctypes.POINTER(Opts), P, P,
                                               ctypes.POINTER(I)]
            L.bsvd_autotune_batched_workspace.argtypes = [P, ctypes.c_char, I, P, P, I, I, ctypes.POINTER(Opts),
                                                          I, ctypes.POINTER(SZ)]
            L.bsvd_autotune_batched.argtypes = [P, ctypes.c_char, I, I, I, P, P, P, P, P, SZ,
                                                ctypes.POINTER(Opts), I, I, P, P, P, ctypes.POINTER(I), P]
            D = ctypes.c_double
            L.bsvd_server_clock.restype = D
            L.bsvd_server_create.argtypes = [P, SZ, ctypes.POINTER(ServerOpts), ctypes.POINTER(P)]
            L.bsvd_server_submit.argtypes = [P, ctypes.c_char, I, I, P, I, I, I, ctypes.POINTER(LL)]
            L.bsvd_server_replay.argtypes = [P, I, P, P, P, P, P, P, I, I, P, ctypes.POINTER(D)]
            L.bsvd_server_test.argtypes = [P, LL]
            L.bsvd_server_wait.argtypes = [P, LL, D, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(D)]
            L.bsvd_server_result.argtypes = [P, LL, ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(I),
                                             ctypes.POINTER(P), ctypes.POINTER(I)]
            L.bsvd_server_fetch.argtypes = [P, LL, P, P, I, P, I]
            L.bsvd_server_release.argtypes = [P, LL]
            L.bsvd_server_collect.argtypes = [P, I, I, P, P, P, P, P, P]
            L.bsvd_server_pause.argtypes = [P, I]
            L.bsvd_server_cancel.argtypes = [P]
            L.bsvd_server_stats.argtypes = [P, P]
            L.bsvd_server_destroy.argtypes = [P]
            _lib = L
    return _lib


def handle() -> ctypes.c_void_p:
    """This thread's library handle (a handle is not thread-safe, so each
    host thread gets its own; autotuned choices live in the handle that
    recorded them)."""
    h = getattr(_handles, "h", None)
    if h is None:
        L = load()
        h = ctypes.c_void_p()
        st = L.bsvd_create(ctypes.byref(h))
        if st != BSVD_OK:
            raise BsvdError(st, "bsvd_create")
        _handles.h = h
    return h


def _check(st: int, where: str):
    if st != BSVD_OK:
        L, h = load(), handle()
        raise BsvdError(st, where, L.bsvd_last_arg(h), L.bsvd_last_cuda(h))


PRECS = {"native": 0, "mixed": 1}


def make_opts(nb=0, tol=0.0, max_sweeps=0, inner_sweeps=0, path="auto", flags=0, prec="native") -> Opts:
    o = Opts()
    o.nb, o.tol, o.max_sweeps, o.inner_sweeps = int(nb), float(tol), int(max_sweeps), int(inner_sweeps)
    o.path, o.flags = PATHS[path] if isinstance(path, str) else int(path), int(flags)
    o.prec = PRECS[prec] if isinstance(prec, str) else int(prec)
    return o


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def column_major(A: torch.Tensor) -> torch.Tensor:
    """(batch, m, n) view whose matrices are column-major (stride(-2) == 1)."""
    if A.stride(-2) == 1 and (A.stride(-1) >= max(1, A.shape[-2]) or A.shape[-1] == 1):
        return A
    return A.transpose(-1, -2).contiguous().transpose(-1, -2)


def leading_dim(X: torch.Tensor) -> int:
    """Leading dimension of a column-major matrix view; a single column's
    stride is meaningless (torch may report 1), so it is taken as the rows."""
    rows = X.shape[-2]
    if X.shape[-1] <= 1:
        return max(1, rows)
    return max(1, X.stride(-1))


def empty_column_major(batch: int, rows: int, cols: int, dtype, device) -> torch.Tensor:
    return torch.empty((batch, cols, rows), dtype=dtype, device=device).transpose(1, 2)


def workspace_bytes(dtype, shapes, uniform: bool, compute_u=True, compute_v=True, **opts) -> int:
    """Device workspace (bytes) a call needs; shapes = [(m, n)] (uniform) or a list."""
    L, h = load(), handle()
    B = len(shapes) if not uniform else opts.pop("batch", 1)
    ms = (ctypes.c_int * max(len(shapes), 1))(*[m for m, _ in shapes])
    ns = (ctypes.c_int * max(len(shapes), 1))(*[n for _, n in shapes])
    o = make_opts(**opts)
    nbytes = ctypes.c_size_t()
    t = DTYPES[dtype] if not isinstance(dtype, str) else dtype
    _check(L.bsvd_gesvj_workspace(h, t.encode(), B, ctypes.cast(ms, ctypes.c_void_p),
                                  ctypes.cast(ns, ctypes.c_void_p), int(uniform), int(compute_u),
                                  int(compute_v), ctypes.byref(o), ctypes.byref(nbytes)),
           "bsvd_gesvj_workspace")
    return int(nbytes.value)


def gesvj(A: torch.Tensor, compute_u: bool = True, compute_v: bool = True, *, nb: int = 0,
          tol: float = 0.0, max_sweeps: int = 0, inner_sweeps: int = 0, path="auto",
          flags: int = 0, prec="native", out=None, work=None, stream=None) -> SVDResult:
    """SVD of every matrix of a CUDA tensor A (batch, m, n) or (m, n).

    A may be float32, float64, complex64 or complex128; matrices are read
    column-major (a copy is made if A is not).  Returns S (batch, k), U
    (batch, m, k), V (batch, n, k) with k = min(m, n) (U/V None when not
    requested), and int32 info and sweeps (batch,).  ``out`` may pass
    preallocated (S, U, V, info, sweeps) in that layout.
    """
    if A.dtype not in DTYPES:
        raise TypeError(f"unsupported dtype {A.dtype}")
    if not A.is_cuda:
        raise ValueError("A must be a CUDA tensor")
    squeeze = A.dim() == 2
    if squeeze:
        A = A.unsqueeze(0)
    A = column_major(A)
    batch, m, n = A.shape
    k = min(m, n)
    dev = A.device
    if out is None:
        S = torch.empty((batch, k), dtype=REAL[A.dtype], device=dev)
        U = empty_column_major(batch, m, k, A.dtype, dev) if compute_u else None
        V = empty_column_major(batch, n, k, A.dtype, dev) if compute_v else None
        info = torch.empty(batch, dtype=torch.int32, device=dev)
        sweeps = torch.empty(batch, dtype=torch.int32, device=dev)
    else:
        S, U, V, info, sweeps = out
    o = make_opts(nb, tol, max_sweeps, inner_sweeps, path, flags, prec)
    t = DTYPES[A.dtype]
    L = load()
    if work is None:
        nbytes = workspace_bytes(A.dtype, [(m, n)], True, compute_u, compute_v, batch=batch, nb=nb,
                                 tol=tol, max_sweeps=max_sweeps, inner_sweeps=inner_sweeps,
                                 path=path, flags=flags, prec=prec)
        work = torch.empty(nbytes, dtype=torch.uint8, device=dev) if nbytes else None
    f = getattr(L, f"bsvd_{t}gesvj_strided")
    st = f(handle(), int(compute_u), int(compute_v), batch, m, n,
           A.data_ptr(), leading_dim(A), A.stride(0),
           S.data_ptr(), S.stride(0) if batch > 1 else k,
           U.data_ptr() if U is not None else None, leading_dim(U) if U is not None else 1,
           U.stride(0) if U is not None else 0,
           V.data_ptr() if V is not None else None, leading_dim(V) if V is not None else 1,
           V.stride(0) if V is not None else 0,
           info.data_ptr(), sweeps.data_ptr() if sweeps is not None else None,
           work.data_ptr() if work is not None else None, work.numel() if work is not None else 0,
           ctypes.byref(o), _stream_ptr(stream))
    _check(st, f"bsvd_{t}gesvj_strided")
    if squeeze:
        return SVDResult(S[0], U[0] if U is not None else None, V[0] if V is not None else None,
                         info, sweeps)
    return SVDResult(S, U, V, info, sweeps)


def host_workspace_bytes(dtype, batch: int, m: int, n: int, compute_u=True, compute_v=True, **opts) -> int:
    """Device workspace (bytes) of ``gesvj_host`` for a (batch, m, n) batch."""
    L, h = load(), handle()
    o = make_opts(**opts)
    nbytes = ctypes.c_size_t()
    t = DTYPES[dtype] if not isinstance(dtype, str) else dtype
    _check(L.bsvd_gesvj_host_workspace(h, t.encode(), batch, m, n, int(compute_u), int(compute_v),
                                       ctypes.byref(o), ctypes.byref(nbytes)), "bsvd_gesvj_host_workspace")
    return max(int(nbytes.value), 256)


def gesvj_host(A: torch.Tensor, compute_u: bool = True, compute_v: bool = True, *, nb: int = 0,
               tol: float = 0.0, max_sweeps: int = 0, inner_sweeps: int = 0, path="auto", flags: int = 0,
               prec="native", out=None, work=None, stream=None, sync: bool = True) -> SVDResult:
    """SVD of a batch in HOST memory (batch, m, n), through the library's
    chunked copy / compute pipeline (``bsvd_?gesvj_strided_host``).

    A is read column-major (a page-locked copy is made if it is pageable or
    not column-major); the results are page-locked CPU tensors in the layout of
    ``gesvj`` (``out`` may pass them preallocated, page-locked).  With
    sync=False the call returns once the work is queued on `stream`.
    """
    if A.dtype not in DTYPES:
        raise TypeError(f"unsupported dtype {A.dtype}")
    if A.is_cuda:
        raise ValueError("gesvj_host takes a CPU tensor; use gesvj for device memory")
    if A.dim() == 2:
        A = A.unsqueeze(0)
    A = column_major(A)
    if not A.is_pinned():
        A = A.transpose(1, 2).contiguous().pin_memory().transpose(1, 2)
    batch, m, n = A.shape
    k = min(m, n)
    dev = torch.device("cuda", torch.cuda.current_device())
    if out is None:
        S = torch.empty((batch, k), dtype=REAL[A.dtype]).pin_memory()
        U = torch.empty((batch, k, m), dtype=A.dtype).pin_memory().transpose(1, 2) if compute_u else None
        V = torch.empty((batch, k, n), dtype=A.dtype).pin_memory().transpose(1, 2) if compute_v else None
        info = torch.empty(batch, dtype=torch.int32).pin_memory()
        sweeps = torch.empty(batch, dtype=torch.int32).pin_memory()
    else:
        S, U, V, info, sweeps = out
    o = make_opts(nb, tol, max_sweeps, inner_sweeps, path, flags, prec)
    t = DTYPES[A.dtype]
    L, h = load(), handle()
    if work is None:
        nbytes = ctypes.c_size_t()
        _check(L.bsvd_gesvj_host_workspace(h, t.encode(), batch, m, n, int(compute_u), int(compute_v),
                                           ctypes.byref(o), ctypes.byref(nbytes)), "bsvd_gesvj_host_workspace")
        work = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=dev)
    st = getattr(L, f"bsvd_{t}gesvj_strided_host")(
        h, int(compute_u), int(compute_v), batch, m, n, A.data_ptr(), leading_dim(A), A.stride(0),
        S.data_ptr(), S.stride(0) if batch > 1 else k,
        U.data_ptr() if U is not None else None, leading_dim(U) if U is not None else 1,
        U.stride(0) if U is not None else 0,
        V.data_ptr() if V is not None else None, leading_dim(V) if V is not None else 1,
        V.stride(0) if V is not None else 0,
        info.data_ptr(), sweeps.data_ptr() if sweeps is not None else None,
        work.data_ptr(), work.numel(), ctypes.byref(o), _stream_ptr(stream))
    _check(st, f"bsvd_{t}gesvj_strided_host")
    if sync:
        (stream or torch.cuda.current_stream()).synchronize()
    return SVDResult(S, U, V, info, sweeps)


def _flat_outputs(sizes, dtype, device):
    """One allocation for a list of outputs of `sizes` elements each, every
    output starting on a 256-byte boundary (as separate allocations would).
    Returns the flat tensor, the element offsets and the device pointers."""
    elt = torch.empty((), dtype=dtype).element_size()
    step = max(1, 256 // elt)
    sizes = np.asarray(sizes, dtype=np.int64)
    padded = (sizes + step - 1) // step * step
    off = np.zeros(len(sizes), dtype=np.int64)
    if len(sizes) > 1:
        np.cumsum(padded[:-1], out=off[1:])
    flat = torch.empty(max(int(padded.sum()), 1), dtype=dtype, device=device)
    ptr = torch.from_numpy(flat.data_ptr() + off * elt).to(device, non_blocking=False)
    return flat, off, ptr


def gesvj_batched(mats, compute_u: bool = True, compute_v: bool = True, *, nb: int = 0,
                  tol: float = 0.0, max_sweeps: int = 0, inner_sweeps: int = 0, path="auto",
                  flags: int = 0, prec="native", stream=None):
    """SVD of a list of CUDA matrices of any shapes (one dtype) through the
    pointer-array entry point.  Returns lists S, U, V and info, sweeps.

    The outputs of all matrices share one allocation per array (views into
    it); the call returns once the work is queued on the stream, like any
    torch operation."""
    mats = [column_major(x) if x.dim() == 2 else None for x in mats]
    if any(x is None for x in mats):
        raise ValueError("every matrix must be 2-D")
    dt = mats[0].dtype
    if any(x.dtype != dt for x in mats) or dt not in DTYPES:
        raise TypeError("all matrices must share one supported dtype")
    dev = mats[0].device
    B = len(mats)
    m_np = np.fromiter((x.shape[0] for x in mats), dtype=np.int64, count=B)
    n_np = np.fromiter((x.shape[1] for x in mats), dtype=np.int64, count=B)
    k_np = np.minimum(m_np, n_np)
    lda_np = np.fromiter((leading_dim(x) for x in mats), dtype=np.int64, count=B)

    def cints(v):
        return (ctypes.c_int * max(B, 1))(*v.tolist())

    ms, ns, lda = cints(m_np), cints(n_np), cints(lda_np)
    ldu, ldv = cints(np.maximum(m_np, 1)), cints(np.maximum(n_np, 1))
    pA = torch.from_numpy(np.fromiter((x.data_ptr() for x in mats), dtype=np.int64, count=B)).to(dev)
    Sf, offS, pS = _flat_outputs(k_np, REAL[dt], dev)
    Uf = Vf = pU = pV = None
    if compute_u:
        Uf, offU, pU = _flat_outputs(m_np * k_np, dt, dev)
    if compute_v:
        Vf, offV, pV = _flat_outputs(n_np * k_np, dt, dev)
    info = torch.empty(B, dtype=torch.int32, device=dev)
    sweeps = torch.empty(B, dtype=torch.int32, device=dev)
    o = make_opts(nb, tol, max_sweeps, inner_sweeps, path, flags, prec)
    L, h = load(), handle()
    t = DTYPES[dt]
    nbytes = ctypes.c_size_t()
    _check(L.bsvd_gesvj_workspace(h, t.encode(), B, ctypes.cast(ms, ctypes.c_void_p),
                                  ctypes.cast(ns, ctypes.c_void_p), 0, int(compute_u),
                                  int(compute_v), ctypes.byref(o), ctypes.byref(nbytes)),
           "bsvd_gesvj_workspace")
    work = torch.empty(max(nbytes.value, 16), dtype=torch.uint8, device=dev)
    f = getattr(L, f"bsvd_{t}gesvj_batched")
    st = f(h, int(compute_u), int(compute_v), B, ctypes.cast(ms, ctypes.c_void_p),
           ctypes.cast(ns, ctypes.c_void_p), pA.data_ptr(), ctypes.cast(lda, ctypes.c_void_p),
           pS.data_ptr(), pU.data_ptr() if pU is not None else None,
           ctypes.cast(ldu, ctypes.c_void_p), pV.data_ptr() if pV is not None else None,
           ctypes.cast(ldv, ctypes.c_void_p), info.data_ptr(), sweeps.data_ptr(),
           work.data_ptr(), work.numel(), ctypes.byref(o), _stream_ptr(stream))
    _check(st, f"bsvd_{t}gesvj_batched")
    if stream is not None:
        # the temporaries return to torch's allocator when this call returns:
        # tie their reuse to the stream the kernels run on
        for x in [pA, pS, pU, pV, work, Sf, Uf, Vf, info, sweeps] + mats:
            if x is not None:
                x.record_stream(stream)
    # views into the flat outputs, formed while the GPU works
    S = [Sf.narrow(0, int(o_), int(k)) for o_, k in zip(offS, k_np)]
    U = [Uf.narrow(0, int(o_), int(m * k)).view(int(k), int(m)).t() for o_, m, k in zip(offU, m_np, k_np)] \
        if compute_u else None
    V = [Vf.narrow(0, int(o_), int(n * k)).view(int(k), int(n)).t() for o_, n, k in zip(offV, n_np, k_np)] \
        if compute_v else None
    return SVDResult(S, U, V, info, sweeps)


_NP_CHAR = {np.dtype(np.float32): "s", np.dtype(np.float64): "d", np.dtype(np.complex64): "c",
            np.dtype(np.complex128): "z"}


def type_char(dtype) -> str:
    """'s', 'd', 'c' or 'z' for a torch dtype, a numpy dtype or the character itself."""
    if isinstance(dtype, str):
        return dtype
    if dtype in DTYPES:
        return DTYPES[dtype]
    return _NP_CHAR[np.dtype(dtype)]


def persistent_plan(dtype, shapes, compute_u: bool = True, compute_v: bool = True, **opts):
    """How a path="persistent" batch of these (m, n) shapes would run each
    matrix: returns (nb, where, launches) with nb and where per matrix (where:
    1 shared memory, 0 global slot, 2 the variable-shape multi-kernel batch,
    -1 empty).  Host only (``bsvd_persistent_plan``)."""
    B = len(shapes)
    ms = (ctypes.c_int * max(B, 1))(*[int(s[0]) for s in shapes])
    ns = (ctypes.c_int * max(B, 1))(*[int(s[1]) for s in shapes])
    nb = (ctypes.c_int * max(B, 1))()
    where = (ctypes.c_int * max(B, 1))()
    launches = ctypes.c_int(0)
    opts.setdefault("path", "persistent")
    o = make_opts(**opts)
    t = type_char(dtype)
    L, h = load(), handle()
    _check(L.bsvd_persistent_plan(h, t.encode(), B, ctypes.cast(ms, ctypes.c_void_p), ctypes.cast(ns, ctypes.c_void_p),
                                  int(compute_u), int(compute_v), ctypes.byref(o), ctypes.cast(nb, ctypes.c_void_p),
                                  ctypes.cast(where, ctypes.c_void_p), ctypes.byref(launches)),
           "bsvd_persistent_plan")
    return np.array(nb[:B], dtype=np.int32), np.array(where[:B], dtype=np.int32), int(launches.value)


def autotune_batched(mats, compute_u: bool = True, compute_v: bool = True, *, sample: int = 64, stream=None,
                     **opts):
    """Per-bucket autotuning of a list of CUDA matrices of mixed shapes (one
    dtype) for path="persistent" (``bsvd_autotune_batched``): times block
    widths 4, 8, 16 on a sample of each (type, M, N rounded to powers of two,
    jobs) bucket and records the winners in the library handle.  Returns a
    list of {"M", "N", "nb", "ms": {nb: ms}} per bucket."""
    mats = [column_major(x) for x in mats]
    dt = mats[0].dtype
    dev = mats[0].device
    B = len(mats)
    ms = (ctypes.c_int * max(B, 1))(*[int(x.shape[0]) for x in mats])
    ns = (ctypes.c_int * max(B, 1))(*[int(x.shape[1]) for x in mats])
    lda = (ctypes.c_int * max(B, 1))(*[leading_dim(x) for x in mats])
    pA = torch.tensor([x.data_ptr() for x in mats], dtype=torch.int64, device=dev)
    o = make_opts(**opts)
    L, h = load(), handle()
    t = DTYPES[dt]
    nbytes = ctypes.c_size_t()
    _check(L.bsvd_autotune_batched_workspace(h, t.encode(), B, ctypes.cast(ms, ctypes.c_void_p),
                                             ctypes.cast(ns, ctypes.c_void_p), int(compute_u), int(compute_v),
                                             ctypes.byref(o), int(sample), ctypes.byref(nbytes)),
           "bsvd_autotune_batched_workspace")
    work = torch.empty(max(nbytes.value, 256), dtype=torch.uint8, device=dev)
    cap = 4096
    mn = (ctypes.c_int * (2 * cap))()
    nb = (ctypes.c_int * cap)()
    tm = (ctypes.c_float * (3 * cap))()
    nbk = ctypes.c_int(0)
    _check(L.bsvd_autotune_batched(h, t.encode(), int(compute_u), int(compute_v), B, ctypes.cast(ms, ctypes.c_void_p),
                                   ctypes.cast(ns, ctypes.c_void_p), pA.data_ptr(), ctypes.cast(lda, ctypes.c_void_p),
                                   work.data_ptr(), work.numel(), ctypes.byref(o), int(sample), cap,
                                   ctypes.cast(mn, ctypes.c_void_p), ctypes.cast(nb, ctypes.c_void_p),
                                   ctypes.cast(tm, ctypes.c_void_p), ctypes.byref(nbk), _stream_ptr(stream)),
           "bsvd_autotune_batched")
    return [{"M": mn[2 * i], "N": mn[2 * i + 1], "nb": nb[i],
             "ms": {w: tm[3 * i + c] for c, w in enumerate((4, 8, 16))}} for i in range(min(nbk.value, cap))]


def autotune(A: torch.Tensor, compute_u: bool = True, compute_v: bool = True, *, stream=None, **opts):
    """Time the path x block-width candidates on (up to 512 of) A's matrices,
    record the winner in the library handle for this (type, size bucket, jobs)
    and return (best, times): best = {"path", "nb"}, times = {(path, nb): ms}.
    Later gesvj calls on that bucket with path "auto" and no nb follow it."""
    if A.dim() == 2:
        A = A.unsqueeze(0)
    A = column_major(A)
    batch, m, n = A.shape
    L, h = load(), handle()
    t = DTYPES[A.dtype]
    base = make_opts(**opts)
    nbytes = ctypes.c_size_t()
    _check(L.bsvd_autotune_workspace(h, t.encode(), batch, m, n, int(compute_u), int(compute_v),
                                     ctypes.byref(base), ctypes.byref(nbytes)), "bsvd_autotune_workspace")
    work = torch.empty(max(nbytes.value, 16), dtype=torch.uint8, device=A.device)
    best = Opts()
    times = (ctypes.c_float * 8)()
    _check(L.bsvd_autotune(h, t.encode(), int(compute_u), int(compute_v), batch, m, n, A.data_ptr(),
                           leading_dim(A), A.stride(0), work.data_ptr(), work.numel(), ctypes.byref(base),
                           ctypes.byref(best), ctypes.cast(times, ctypes.c_void_p), _stream_ptr(stream)),
           "bsvd_autotune")
    nbs = [4, 4, 8, 8, 16, 16, 32, 32]
    names = ["fused", "blocked"] * 4
    tt = {(names[c], nbs[c]): times[c] for c in range(8) if times[c] >= 0}
    return {"path": PATH_NAMES[best.path], "nb": best.nb}, tt


STATS_KEYS = ("submitted", "completed", "failed", "queued", "running", "running_batches", "arena_used",
              "arena_peak", "cancelled", "batches")


class Server:
    """Continuous-batching SVD server on a CUDA device (``bsvd_server_*`` in
    include/bsvd.h): single-matrix requests are queued, batched by type and
    block width, admitted within a device-memory arena of ``arena_bytes``
    (allocated here with torch and owned by this object) and solved by the
    persistent kernel, each request completing as soon as its matrix has.

    Inputs must be CUDA tensors or page-locked CPU tensors (a pageable CPU
    tensor is copied to page-locked memory first); they are kept alive here
    until their request is released.
    """

    def __init__(self, arena_bytes: int, *, max_inflight: int = 0, max_batch: int = 0, big_k: int = 0,
                 max_big_batch: int = 0, fp64_prec="native", big_flags: int = 0, big_k_fp64: int = 0,
                 device=None):
        self.lib = load()
        dev = torch.device(device) if device is not None else torch.device("cuda", torch.cuda.current_device())
        self.device = dev
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=dev)
        o = ServerOpts()
        o.max_inflight, o.max_batch, o.big_k = int(max_inflight), int(max_batch), int(big_k)
        o.max_big_batch = int(max_big_batch)
        o.fp64_prec = PRECS[fp64_prec] if isinstance(fp64_prec, str) else int(fp64_prec)
        o.big_flags = int(big_flags)
        o.big_k_fp64 = int(big_k_fp64)
        srv = ctypes.c_void_p()
        with torch.cuda.device(dev):
            st = self.lib.bsvd_server_create(self.arena.data_ptr(), self.arena.numel(), ctypes.byref(o),
                                             ctypes.byref(srv))
        if st != BSVD_OK:
            raise BsvdError(st, "bsvd_server_create")
        self.srv = srv
        self._keep = {}
        self._meta = {}

    # -- requests --------------------------------------------------------
    def _input(self, A: torch.Tensor) -> torch.Tensor:
        if A.dim() != 2 or A.dtype not in DTYPES:
            raise TypeError("a request is one 2-D float32/float64/complex64/complex128 matrix")
        A = column_major(A.unsqueeze(0))[0]
        if not A.is_cuda and not A.is_pinned():
            A = A.t().contiguous().pin_memory().t()       # column-major, page-locked
        return A

    def submit(self, A: torch.Tensor, compute_u: bool = True, compute_v: bool = True) -> int:
        A = self._input(A)
        m, n = A.shape
        rid = ctypes.c_longlong()
        st = self.lib.bsvd_server_submit(self.srv, DTYPES[A.dtype].encode(), m, n, A.data_ptr(),
                                         leading_dim(A), int(compute_u), int(compute_v), ctypes.byref(rid))
        if st != BSVD_OK:
            raise BsvdError(st, "bsvd_server_submit")
        self._keep[rid.value] = A
        self._meta[rid.value] = (A.dtype, m, n, compute_u, compute_v)
        return rid.value

    def replay(self, t_offset, mats, compute_u: bool = True, compute_v: bool = True, keep: bool = True):
        """Submit mats[i] at t0 + t_offset[i] (seconds) from the calling thread,
        each stamped with its scheduled time; returns (ids, t0).  With
        keep=False the caller keeps the inputs alive until their requests
        complete (and fetch() is not available for them)."""
        import numpy as np
        seen = {}
        mats = [seen[id(A)] if id(A) in seen else seen.setdefault(id(A), self._input(A)) for A in mats]
        B = len(mats)
        t = np.ascontiguousarray(np.asarray(t_offset, dtype=np.float64))
        dt = np.frombuffer(b"".join(DTYPES[A.dtype].encode() for A in mats), dtype=np.uint8).copy()
        m = np.array([A.shape[0] for A in mats], dtype=np.int32)
        n = np.array([A.shape[1] for A in mats], dtype=np.int32)
        lda = np.array([leading_dim(A) for A in mats], dtype=np.int32)
        ptr = np.array([A.data_ptr() for A in mats], dtype=np.uint64)
        ids = np.zeros(B, dtype=np.int64)
        t0 = ctypes.c_double()
        st = self.lib.bsvd_server_replay(self.srv, B, t.ctypes.data, dt.ctypes.data, m.ctypes.data, n.ctypes.data,
                                         ptr.ctypes.data, lda.ctypes.data, int(compute_u), int(compute_v),
                                         ids.ctypes.data, ctypes.byref(t0))
        for i, A in zip(ids.tolist(), mats if keep else []):
            if i > 0 and self.lib.bsvd_server_test(self.srv, i) >= 0:    # not collected and released yet
                self._keep[i] = A
                self._meta[i] = (A.dtype, A.shape[0], A.shape[1], compute_u, compute_v)
        if st != BSVD_OK:
            raise BsvdError(st, "bsvd_server_replay")
        return ids, t0.value

    def test(self, rid: int) -> int:
        return self.lib.bsvd_server_test(self.srv, rid)

    def wait(self, rid: int, timeout: float = -1.0):
        """Block until request rid completes; returns (info, sweeps, t_done)."""
        info, sweeps, t_done = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
        st = self.lib.bsvd_server_wait(self.srv, rid, float(timeout), ctypes.byref(info), ctypes.byref(sweeps),
                                       ctypes.byref(t_done))
        if st != BSVD_OK:
            raise BsvdError(st, "bsvd_server_wait")
        return info.value, sweeps.value, t_done.value

    def fetch(self, rid: int, device="cpu", release: bool = True) -> SVDResult:
        """Copy request rid's results into new tensors on `device` (waits for it)."""
        info, sweeps, _ = self.wait(rid)
        dt, m, n, cu, cv = self._meta[rid]
        k = min(m, n)
        dev = torch.device(device)
        S = torch.empty(k, dtype=REAL[dt], device=dev)
        U = torch.empty((k, m), dtype=dt, device=dev).t() if cu else None
        V = torch.empty((k, n), dtype=dt, device=dev).t() if cv else None
        st = self.lib.bsvd_server_fetch(self.srv, rid, S.data_ptr(), U.data_ptr() if cu else None, max(m, 1),
                                        V.data_ptr() if cv else None, max(n, 1))
        if st != BSVD_OK:
            raise BsvdError(st, "bsvd_server_fetch")
        if release:
            self.release(rid)
        return SVDResult(S, U, V, info, sweeps)

    def release(self, rid: int):
        st = self.lib.bsvd_server_release(self.srv, rid)
        if st != BSVD_OK:
            raise BsvdError(st, "bsvd_server_release")
        self._keep.pop(rid, None)
        self._meta.pop(rid, None)

    def collect(self, max_count: int = 65536, release: bool = True):
        """Requests completed since the last collect: dict of numpy arrays
        id, status, info, sweeps, t_submit, t_done (released if asked)."""
        import numpy as np
        out = {"id": np.zeros(max_count, np.int64), "status": np.zeros(max_count, np.int32),
               "info": np.zeros(max_count, np.int32), "sweeps": np.zeros(max_count, np.int32),
               "t_submit": np.zeros(max_count, np.float64), "t_done": np.zeros(max_count, np.float64)}
        k = self.lib.bsvd_server_collect(self.srv, max_count, int(release), *(out[x].ctypes.data for x in
                                         ("id", "status", "info", "sweeps", "t_submit", "t_done")))
        if k < 0:
            raise BsvdError(k, "bsvd_server_collect")
        out = {key: v[:k] for key, v in out.items()}
        if release:
            for i in out["id"].tolist():
                self._keep.pop(i, None)
                self._meta.pop(i, None)
        return out

    def cancel(self):
        """Cancel queued requests and stop running persistent batches early."""
        _ok(self.lib.bsvd_server_cancel(self.srv), "bsvd_server_cancel")

    def pause(self, paused: bool = True):
        _ok(self.lib.bsvd_server_pause(self.srv, int(paused)), "bsvd_server_pause")

    def stats(self) -> dict:
        c = (ctypes.c_longlong * 10)()
        _ok(self.lib.bsvd_server_stats(self.srv, ctypes.cast(c, ctypes.c_void_p)), "bsvd_server_stats")
        return dict(zip(STATS_KEYS, list(c)))

    def clock(self) -> float:
        return self.lib.bsvd_server_clock()

    def close(self):
        if getattr(self, "srv", None):
            st = self.lib.bsvd_server_destroy(self.srv)
            self.srv = None
            self._keep.clear()
            self._meta.clear()
            if st != BSVD_OK:
                raise BsvdError(st, "bsvd_server_destroy")

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _ok(st: int, where: str):
    if st != BSVD_OK:
        raise BsvdError(st, where)
