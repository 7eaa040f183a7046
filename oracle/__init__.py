"""CPU FP64 oracle for the batched one-sided Jacobi SVD -- TEST INFRASTRUCTURE.

A plain, slow restatement of the method of "An Efficient Batch Solver for the
Singular Value Decomposition on GPUs" (Abdelfattah and Fasi), in C
(``oracle.c`` + ``oracle_core.h``), built with gcc (no fast-math, no FMA
contraction) and loaded with ctypes.  Only the test suite,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import
this package.  It shares no code with the CUDA path and never imports it.

Parity status (pins in ``tests/test_oracle_pins.py``):

* ``gesvj``           Alg. 2 -- pinned: 2x2 closed form, diagonal and
                      permuted-diagonal inputs (bitwise), Q1 diag(sigma) Q2^H
                      with known sigma, mpmath brute force, LAPACK cross-check.
* ``heevj``           Alg. 1 -- pinned: mpmath eigenvalues, the 2x2 closed
                      form, the off-norm contraction of one sweep (P2).
* ``gesvj_blocked``   blocked method of Sec. 3 / Sec. 4 -- pinned: the states
                      A^(1), A^(2), G^(2) printed in the worked example of
                      Sec. 5.1; sigma agrees with Alg. 2.
* ``rr_pair``         round-robin ordering -- pinned: the l = 4 sequence of
                      Sec. 5.1; every pair exactly once per sweep, disjoint
                      slots within a round.
* ``gesvj_qr``        QR pre-processing (Sec. "Pre-processing the SVD using a
                      QR Factorization"): Householder QR (numpy / LAPACK
                      geqrf), the oracle's SVD of R, U = Q U_R -- pinned:
                      sigma against Alg. 2 and LAPACK on tall, wide and square
                      inputs, reconstruction and orthogonality, a planted
                      mistake (U without Q) caught.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ("oracle.c", "oracle_core.h")
DEFAULT_SO = os.path.join(_HERE, "liboracle.so")

U64 = 2.0 ** -53   # unit roundoff of binary64 (u = 2^-s, s = 53 significand bits; Sec. 3)
U32 = 2.0 ** -24   # unit roundoff of binary32


def build(src_dir: str = _HERE, out: str = DEFAULT_SO, force: bool = False) -> str:
    """Compile the oracle with gcc: -O2, no fast-math, no FMA contraction, OpenMP."""
    srcs = [os.path.join(src_dir, s) for s in SOURCES]
    newest = max(os.path.getmtime(p) for p in srcs)
    if force or not os.path.exists(out) or os.path.getmtime(out) < newest:
        tmp = f"{out}.{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fno-fast-math", "-ffp-contract=off", "-fopenmp",
               "-fPIC", "-shared", "-o", tmp, srcs[0], "-lm"]
        subprocess.run(cmd, check=True, cwd=src_dir)
        os.replace(tmp, out)
    return out


class Oracle:
    """ctypes view of one build of the oracle library."""

    def __init__(self, so_path: str):
        L = ctypes.CDLL(so_path)
        I, D, P = ctypes.c_int, ctypes.c_double, ctypes.c_void_p
        L.oracle_rr_pair.argtypes = [I, I, I, ctypes.POINTER(I), ctypes.POINTER(I)]
        L.oracle_rr_pair.restype = None
        for name in ("oracle_dheevj", "oracle_zheevj"):
            f = getattr(L, name)
            f.argtypes = [I, P, I, P, I, D, I, ctypes.POINTER(I)]
            f.restype = I
        L.oracle_gesvj_blocked_rounds.argtypes = [ctypes.c_char, I, I, P, I, I, I, D, I, P, I]
        L.oracle_gesvj_blocked_rounds.restype = I
        L.oracle_gesvj_batch.argtypes = [ctypes.c_char, I, P, P, P, P, I, I, P, I, P, P, P,
                                         P, P, P, P, I]
        L.oracle_gesvj_batch.restype = I
        self.L = L

    # -- round-robin ordering ------------------------------------------------
    def rr_pair(self, l: int, r: int, q: int) -> tuple[int, int]:
        """Slot q of round r of the round-robin ordering of l (even) players."""
        i, j = ctypes.c_int(), ctypes.c_int()
        self.L.oracle_rr_pair(l, r, q, ctypes.byref(i), ctypes.byref(j))
        return i.value, j.value

    # -- Alg. 1 --------------------------------------------------------------
    def heevj(self, G, tol: float = 30 * U64, max_sweeps: int = 60):
        """Alg. 1 on a Hermitian positive semi-definite G.

        Returns (G_out, Z, sweeps, converged), G_out = Z^H G Z."""
        G = np.asarray(G)
        cplx = np.iscomplexobj(G)
        dt = np.complex128 if cplx else np.float64
        n = G.shape[0]
        Gf = np.asfortranarray(G.astype(dt, copy=True))
        Z = np.zeros((n, n), dtype=dt, order="F")
        conv = ctypes.c_int()
        f = self.L.oracle_zheevj if cplx else self.L.oracle_dheevj
        sw = f(n, Gf.ctypes.data, max(n, 1), Z.ctypes.data, max(n, 1), tol, max_sweeps,
               ctypes.byref(conv))
        return Gf, Z, sw, bool(conv.value)

    # -- the blocked method, stopped after k rounds ------------------------------
    def blocked_rounds(self, A, nb: int, rounds: int, inner_sweeps: int = 60,
                       tol: float = 30 * U64) -> np.ndarray:
        """A^(k) after the first ``rounds`` round-robin iterations (m >= n)."""
        A = np.asarray(A)
        cplx = np.iscomplexobj(A)
        dt = np.complex128 if cplx else np.float64
        Af = np.asfortranarray(A.astype(dt))
        m, n = Af.shape
        W = np.zeros((max(m, n), min(m, n)), dtype=dt, order="F")
        self.L.oracle_gesvj_blocked_rounds(b"z" if cplx else b"d", m, n, Af.ctypes.data,
                                           max(m, 1), nb, inner_sweeps, tol, rounds,
                                           W.ctypes.data, max(W.shape[0], 1))
        return W

    # -- Alg. 2 and the blocked method, batched ------------------------------------
    def gesvj(self, A, tol=None, max_sweeps: int = 60, nb: int = 0, inner_sweeps: int = 1,
              want_u: bool = True, want_v: bool = True, nthreads: int = 0):
        """SVD of one matrix (2-D array) or a list of matrices.

        nb = 0 runs Alg. 2 (unblocked, row-cyclic); nb > 0 runs the blocked
        method with ``inner_sweeps`` sweeps of Alg. 1 per block pair.  Real
        input of any float type is widened to float64 exactly, complex to
        complex128.  ``tol`` is the per-pair rotation threshold: a scalar, a
        per-matrix sequence, or None for n * 2^-53 (n = min(m, n)).

        Returns a dict: S, U, V (lists, or arrays for a 2-D input), sweeps,
        info, threads (OpenMP threads used).
        """
        single = isinstance(A, np.ndarray) and A.ndim == 2
        mats = [A] if single else list(A)
        B = len(mats)
        cplx = any(np.iscomplexobj(a) for a in mats)
        dt = np.complex128 if cplx else np.float64
        work = [np.asfortranarray(np.asarray(a).astype(dt)) for a in mats]
        ms = np.array([a.shape[0] for a in work], dtype=np.int32)
        ns = np.array([a.shape[1] for a in work], dtype=np.int32)
        ks = np.minimum(ms, ns)
        if tol is None:
            tols = np.array([max(k, 1) * U64 for k in ks], dtype=np.float64)
        elif np.ndim(tol) == 0:
            tols = np.full(B, float(tol), dtype=np.float64)
        else:
            tols = np.ascontiguousarray(tol, dtype=np.float64)
        S = [np.zeros(k, dtype=np.float64) for k in ks]
        U = [np.zeros((m, k), dtype=dt, order="F") for m, k in zip(ms, ks)] if want_u else None
        V = [np.zeros((n, k), dtype=dt, order="F") for n, k in zip(ns, ks)] if want_v else None
        sweeps = np.zeros(B, dtype=np.int32)
        info = np.zeros(B, dtype=np.int32)

        def parr(arrs):
            return (ctypes.c_void_p * max(B, 1))(*[a.ctypes.data for a in arrs])

        lda = np.maximum(ms, 1).astype(np.int32)
        ldv = np.maximum(ns, 1).astype(np.int32)
        pA, pS = parr(work), parr(S)
        pU = parr(U) if U is not None else None
        pV = parr(V) if V is not None else None
        vp = ctypes.c_void_p
        threads = self.L.oracle_gesvj_batch(
            b"z" if cplx else b"d", B, ms.ctypes.data, ns.ctypes.data, ctypes.cast(pA, vp),
            lda.ctypes.data, int(nb), int(inner_sweeps), tols.ctypes.data, int(max_sweeps),
            ctypes.cast(pS, vp), ctypes.cast(pU, vp) if pU is not None else None,
            lda.ctypes.data, ctypes.cast(pV, vp) if pV is not None else None, ldv.ctypes.data,
            sweeps.ctypes.data, info.ctypes.data, int(nthreads))
        if single:
            return {"S": S[0], "U": U[0] if U else None, "V": V[0] if V else None,
                    "sweeps": int(sweeps[0]), "info": int(info[0]), "threads": threads}
        return {"S": S, "U": U, "V": V, "sweeps": sweeps, "info": info, "threads": threads}


_default = None
_lock = threading.Lock()


def default() -> Oracle:
    global _default
    with _lock:
        if _default is None:
            _default = Oracle(build())
    return _default


def rr_pair(l, r, q):
    return default().rr_pair(l, r, q)


def heevj(G, **kw):
    return default().heevj(G, **kw)


def blocked_rounds(A, nb, rounds, **kw):
    return default().blocked_rounds(A, nb, rounds, **kw)


def gesvj(A, **kw):
    return default().gesvj(A, **kw)


def gesvj_qr(A, **kw):
    """SVD after QR pre-processing (Sec. "Pre-processing the SVD using a QR
    Factorization"), for one matrix or a list.

    A' = A (m >= n) or A^H (m < n) is factored A' = Q [R; 0] by Householder
    QR (numpy's reduced QR, LAPACK geqrf/orgqr: a library step), R is
    decomposed by ``gesvj`` (same keyword arguments), and the left vectors of
    A' are Q U_R; for m < n the roles of U and V swap back (A = V Sigma U^H
    of A').  Returns the same dict as ``gesvj``.
    """
    single = isinstance(A, np.ndarray) and A.ndim == 2
    mats = [A] if single else list(A)
    Rs, Qs, trans = [], [], []
    for a in mats:
        cplx = np.iscomplexobj(a)
        w = np.asarray(a).astype(np.complex128 if cplx else np.float64)
        t = w.shape[0] < w.shape[1]
        if t:
            w = w.conj().T
        Q, R = np.linalg.qr(w, mode="reduced")
        Qs.append(Q)
        Rs.append(R)
        trans.append(t)
    want_u, want_v = kw.pop("want_u", True), kw.pop("want_v", True)
    r = default().gesvj(Rs, want_u=True, want_v=True, **kw)
    S, U, V = [], [], []
    for i, (Q, t) in enumerate(zip(Qs, trans)):
        left = Q @ r["U"][i]            # left vectors of A'
        right = r["V"][i]               # right vectors of A'
        u, v = (right, left) if t else (left, right)
        S.append(r["S"][i])
        U.append(u)
        V.append(v)
    out = {"S": S, "U": U if want_u else None, "V": V if want_v else None, "sweeps": r["sweeps"],
           "info": r["info"], "threads": r["threads"]}
    if single:
        return {"S": S[0], "U": U[0] if want_u else None, "V": V[0] if want_v else None,
                "sweeps": int(r["sweeps"][0]), "info": int(r["info"][0]), "threads": r["threads"]}
    return out
