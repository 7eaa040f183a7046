"""Accuracy measures for an SVD result -- TEST INFRASTRUCTURE.

Plain numpy in FP64 (complex128), no part of the SVD method.

Gating bounds (u = unit roundoff of the working precision, n = column count):
    max_k |sigma_k - sigma_ref_k| / sigma_ref_max  <= 50 n u
    ||A - U Sigma V^H||_F / ||A||_F                <= 20 n u
    ||U^H U - I||_F,  ||V^H V - I||_F              <= 20 n u
Reported beside them, the paper's measures e1-e4 of Sec. 8.1 (LAPACK BDT01 /
UNT01 style, 1-norms), whose threshold is k u with k = 30:
    e1 = ||A - U S V^H||_1 / (n ||A||_1)
    e2 = ||I - U^H U||_1 / m
    e3 = ||I - V^H V||_1 / n
    e4 = ||Sigma - Sigma_ref||_F / (min(m, n) ||Sigma_ref||_F)
"""
from __future__ import annotations

import numpy as np

U64 = 2.0 ** -53
U32 = 2.0 ** -24


def unit_roundoff(dtype) -> float:
    dt = np.dtype(dtype)
    return U32 if dt in (np.float32, np.complex64) else U64


def measures(A, S, U, V, S_ref=None) -> dict:
    """All measures for one matrix; U or V may be None (then skipped)."""
    A = np.asarray(A)
    wide = np.complex128 if np.iscomplexobj(A) or (U is not None and np.iscomplexobj(U)) \
        or (V is not None and np.iscomplexobj(V)) else np.float64
    A64 = A.astype(wide)
    m, n = A64.shape
    k = min(m, n)
    S64 = np.asarray(S, dtype=np.float64)
    out = {"m": m, "n": n}
    if S_ref is not None:
        Sr = np.asarray(S_ref, dtype=np.float64)
        smax = Sr.max() if Sr.size else 0.0
        out["sigma_err"] = float(np.abs(S64 - Sr).max() / smax) if smax > 0 else float(np.abs(S64 - Sr).max())
        nr = np.linalg.norm(Sr)
        out["e4"] = float(np.linalg.norm(S64 - Sr) / (k * nr)) if nr > 0 else 0.0
    out["sorted"] = bool(np.all(S64[:-1] >= S64[1:])) if k > 1 else True
    if U is not None and V is not None:
        U64_ = np.asarray(U).astype(wide)
        V64_ = np.asarray(V).astype(wide)
        R = A64 - (U64_ * S64[None, :]) @ V64_.conj().T
        nA = np.linalg.norm(A64)
        out["resid"] = float(np.linalg.norm(R) / nA) if nA > 0 else float(np.linalg.norm(R))
        n1 = np.abs(A64).sum(axis=0).max() if A64.size else 0.0
        out["e1"] = float(np.abs(R).sum(axis=0).max() / (n * n1)) if n1 > 0 else 0.0
    if U is not None:
        U64_ = np.asarray(U).astype(wide)
        EU = U64_.conj().T @ U64_ - np.eye(k)
        out["orth_u"] = float(np.linalg.norm(EU))
        out["e2"] = float(np.abs(EU).sum(axis=0).max() / m) if m else 0.0
    if V is not None:
        V64_ = np.asarray(V).astype(wide)
        EV = V64_.conj().T @ V64_ - np.eye(k)
        out["orth_v"] = float(np.linalg.norm(EV))
        out["e3"] = float(np.abs(EV).sum(axis=0).max() / n) if n else 0.0
    return out


def bounds(n: int, u: float) -> dict:
    return {"sigma_err": 50 * n * u, "resid": 20 * n * u, "orth_u": 20 * n * u, "orth_v": 20 * n * u}


def violations(meas: dict, u: float) -> list[str]:
    """Names of the gating measures that exceed their bound (empty = pass)."""
    b = bounds(meas["n"], u)
    bad = [k for k, lim in b.items() if k in meas and not (meas[k] <= lim)]
    if not meas.get("sorted", True):
        bad.append("sorted")
    return bad
