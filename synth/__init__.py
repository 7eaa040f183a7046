"""Seeded synthetic inputs for the batched SVD workloads.

This module holds no arithmetic of the SVD method itself: it draws random
numbers, builds Haar-distributed orthonormal factors by QR of Gaussian
matrices (sign-fixed, Mezzadri 2007), and multiplies them by a prescribed
singular-value vector.  Both the CPU oracle checks and the CUDA path take
their inputs from here, so the two sides see identical matrices.

Every matrix has its own random stream, keyed by (seed, matrix index), so
matrix ``i`` of a workload can be rebuilt alone (``matrices(cfg, [i])``)
to check sampled outputs of a full-size run.

Singular-value families follow Table "svd_dist" (Sec. 8.1) of Abdelfattah and
Fasi: random, arith, cluster0, cluster1, logrand, geo.  Workload recipes:

* ``square32_f64``      1,000 matrices 32x32, iid N(0,1), FP64.
* ``tall128x64``        10,000 matrices 128x64 = Q1 diag(sigma) Q2^T, Haar
                        Q1 (128x64 orthonormal columns) and Q2 (64x64), sigma
                        geometric from 1 to 1e-6 (FP64) or 1e-3 (FP32); the FP32
                        matrix is built in FP64 and rounded once.
* ``mixed96``           4,000 square 96x96 matrices, half real FP64 and half
                        complex128 (Haar unitary factors from complex normal
                        QR), sigma in 48 clustered pairs (c_k, c_k (1 - 1e-6)),
                        c_k = 10^(-8 (k-1)/47): condition number about 1e8.
* ``uneven``            m ~ U{8..512}, n ~ U{8..m}, entries iid U(-1,1); half
                        complex64 (real and imaginary parts each U(-1,1)).
* ``random01``          entries iid U[0,1], the distribution of LAPACK larnv
                        that the paper's timings use (Sec. 5.4, Sec. 8.2).
"""
from __future__ import annotations

import numpy as np
import torch

SEED_BASE = 0xB5D00000

FAMILIES = ("random", "arith", "cluster0", "cluster1", "logrand", "geo")


def rng_for(seed: int, index: int) -> np.random.Generator:
    """Independent stream for matrix ``index`` of the workload ``seed``."""
    return np.random.Generator(np.random.Philox(key=[int(seed) & 0xFFFFFFFFFFFFFFFF, int(index)]))


def gaussian(rng: np.random.Generator, m: int, n: int, complex_: bool = False) -> np.ndarray:
    """iid N(0,1) entries; complex: (x + i y)/sqrt(2) with x, y iid N(0,1)."""
    if complex_:
        return (rng.standard_normal((m, n)) + 1j * rng.standard_normal((m, n))) / np.sqrt(2.0)
    return rng.standard_normal((m, n))


def haar(rng: np.random.Generator, m: int, n: int, complex_: bool = False) -> np.ndarray:
    """m x n (m >= n) with orthonormal columns, Haar distributed.

    QR of a Gaussian matrix with R's diagonal phases moved into Q (Mezzadri).
    """
    return _haar_from(gaussian(rng, m, n, complex_)[None])[0]


def _haar_from(Z: np.ndarray) -> np.ndarray:
    """Stacked QR (torch CPU, LAPACK geqrf per matrix) with the sign fix."""
    Q, R = torch.linalg.qr(torch.from_numpy(np.ascontiguousarray(Z)))
    Q, R = Q.numpy(), R.numpy()
    d = np.diagonal(R, axis1=-2, axis2=-1)
    ph = d / np.where(np.abs(d) == 0, 1.0, np.abs(d))
    return Q * ph[..., None, :]


def sigma_family(name: str, n: int, kappa: float, rng: np.random.Generator | None = None) -> np.ndarray:
    """Singular values of Table svd_dist, sigma_1 = 1, sigma_n = 1/kappa."""
    i = np.arange(1, n + 1, dtype=np.float64)
    if n == 1:
        return np.ones(1)
    if name == "arith":
        return 1.0 - (i - 1) / (n - 1) * (1.0 - 1.0 / kappa)
    if name == "cluster0":
        s = np.full(n, 1.0 / kappa)
        s[0] = 1.0
        return s
    if name == "cluster1":
        s = np.ones(n)
        s[-1] = 1.0 / kappa
        return s
    if name == "logrand":
        assert rng is not None
        s = np.exp(rng.uniform(np.log(1.0 / kappa), 0.0, size=n))
        s[0], s[-1] = 1.0, 1.0 / kappa
        return np.sort(s)[::-1].copy()
    if name == "geo":
        return kappa ** ((1.0 - i) / (n - 1))
    raise ValueError(name)


def with_sigma(rng: np.random.Generator, m: int, n: int, sigma: np.ndarray,
               complex_: bool = False) -> np.ndarray:
    """Q1 diag(sigma) Q2^H with Haar Q1 (m x k) and Q2 (n x k), k = min(m, n)."""
    k = min(m, n)
    Q1 = haar(rng, m, k, complex_)
    Q2 = haar(rng, n, k, complex_)
    return torch.matmul(torch.from_numpy(Q1 * np.asarray(sigma)[None, :k]),
                        torch.from_numpy(Q2.conj().T.copy())).numpy()


def clustered_pairs(n: int, gap: float = 1e-6, kappa: float = 1e8) -> np.ndarray:
    """n/2 pairs (c_k, c_k (1 - gap)), c_k = kappa^(-(k-1)/(n/2-1))."""
    h = n // 2
    c = kappa ** (-np.arange(h) / max(h - 1, 1))
    s = np.empty(n)
    s[0:2 * h:2] = c
    s[1:2 * h:2] = c * (1.0 - gap)
    if n % 2:
        s[-1] = c[-1] * (1.0 - gap) ** 2
    return s


# --------------------------------------------------------------------------
# Workloads.  Each returns (list of matrices, meta) for the requested indices.
# --------------------------------------------------------------------------
WORKLOADS = {
    "square32_f64": dict(seed=SEED_BASE + 0, batch=1000, m=32, n=32, dtype="d", nb=8),
    "tall128x64_f64": dict(seed=SEED_BASE + 1, batch=10000, m=128, n=64, dtype="d", nb=16, kappa=1e6),
    "tall128x64_f32": dict(seed=SEED_BASE + 2, batch=10000, m=128, n=64, dtype="s", nb=16, kappa=1e3),
    "mixed96": dict(seed=SEED_BASE + 3, batch=4000, m=96, n=96, dtype="d+z", nb=16, kappa=1e8),
    "uneven": dict(seed=SEED_BASE + 4, batch=20000, dtype="s+c"),
}


def matrix(name: str, index: int) -> np.ndarray:
    """Matrix ``index`` of workload ``name`` (numpy, logical shape m x n)."""
    w = WORKLOADS[name]
    rng = rng_for(w["seed"], index)
    if name == "square32_f64":
        return rng.standard_normal((w["m"], w["n"]))
    if name.startswith("tall128x64"):
        sig = sigma_family("geo", w["n"], w["kappa"])
        A = with_sigma(rng, w["m"], w["n"], sig)
        return A.astype(np.float32) if w["dtype"] == "s" else A
    if name == "mixed96":
        cplx = index % 2 == 1
        return with_sigma(rng, w["m"], w["n"], clustered_pairs(w["n"], 1e-6, w["kappa"]), cplx)
    if name == "uneven":
        m = int(rng.integers(8, 513))
        n = int(rng.integers(8, m + 1))
        cplx = index % 2 == 1
        if cplx:
            A = rng.uniform(-1, 1, (m, n)) + 1j * rng.uniform(-1, 1, (m, n))
            return A.astype(np.complex64)
        return rng.uniform(-1, 1, (m, n)).astype(np.float32)
    raise ValueError(name)


def matrices(name: str, indices) -> list[np.ndarray]:
    return [matrix(name, int(i)) for i in indices]


def uniform_batch(name: str, count: int | None = None, start: int = 0) -> np.ndarray:
    """A (count, m, n) stack for a uniform-shape workload, built fast.

    The same matrices as ``matrix(name, i)`` for i in [start, start+count):
    every matrix draws from its own stream, then the QRs run stacked
    (torch's CPU QR runs LAPACK per matrix, so the bits match).
    """
    w = WORKLOADS[name]
    count = w["batch"] if count is None else count
    idx = range(start, start + count)
    if name == "square32_f64":
        return np.stack([rng_for(w["seed"], i).standard_normal((w["m"], w["n"])) for i in idx])
    if name.startswith("tall128x64"):
        return _tall_chunk(w, list(idx))
    return np.stack(matrices(name, idx))


def _tall_chunk(w: dict, idx: list) -> np.ndarray:
    m, n, count = w["m"], w["n"], len(idx)
    Z1 = np.empty((count, m, n))
    Z2 = np.empty((count, n, n))
    for t, i in enumerate(idx):
        rng = rng_for(w["seed"], i)
        Z1[t] = rng.standard_normal((m, n))
        Z2[t] = rng.standard_normal((n, n))
    Q1 = _haar_from(Z1)
    Q2 = _haar_from(Z2)
    sig = sigma_family("geo", n, w["kappa"])
    A = torch.matmul(torch.from_numpy(Q1 * sig[None, None, :]),
                     torch.from_numpy(Q2).transpose(1, 2)).numpy()
    return A.astype(np.float32) if w["dtype"] == "s" else A


def random01(rng: np.random.Generator, m: int, n: int, dtype=np.float64) -> np.ndarray:
    """Entries iid U[0,1] (complex: both parts), like LAPACK larnv(1, ...)."""
    if np.issubdtype(np.dtype(dtype), np.complexfloating):
        return (rng.uniform(0, 1, (m, n)) + 1j * rng.uniform(0, 1, (m, n))).astype(dtype)
    return rng.uniform(0, 1, (m, n)).astype(dtype)


# --------------------------------------------------------------------------
# Serving stream: Poisson arrivals of single-matrix requests.
# --------------------------------------------------------------------------
SERVING = dict(seed=SEED_BASE + 5, rate=50000.0, seconds=10.0, m_lo=16, m_hi=1024, bins=64, variants=2,
               dtypes=("s", "d", "c"), dtype_p=(0.5, 0.3, 0.2), kappa_lo=1e2, kappa_hi=1e6)
_NP = {"s": np.float32, "d": np.float64, "c": np.complex64, "z": np.complex128}


def serving_sizes(cfg: dict = SERVING) -> np.ndarray:
    """The larger dimension of each size bin: log-spaced from m_lo to m_hi."""
    return np.unique(np.rint(np.geomspace(cfg["m_lo"], cfg["m_hi"], cfg["bins"])).astype(int))


def serving_shape(b: int, tall: bool, cfg: dict = SERVING) -> tuple[int, int]:
    m = int(serving_sizes(cfg)[b])
    return m, (-(-m // 2) if tall else m)


def serving_matrix(b: int, tall: bool, t: str, v: int, cfg: dict = SERVING) -> np.ndarray:
    """Pool matrix (size bin b, 2:1 tall or square, type t, variant v):
    Q1 diag(sigma) Q2^H with Haar factors and logrand sigma (sigma_1 = 1,
    sigma_n = 1/kappa, the rest log-uniform), kappa log-uniform in
    [kappa_lo, kappa_hi]."""
    m, n = serving_shape(b, tall, cfg)
    key = ((b * 2 + int(tall)) * 4 + "sdcz".index(t)) * 64 + v
    rng = rng_for(cfg["seed"], key)
    kappa = float(np.exp(rng.uniform(np.log(cfg["kappa_lo"]), np.log(cfg["kappa_hi"]))))
    sig = sigma_family("logrand", min(m, n), kappa, rng)
    return with_sigma(rng, m, n, sig, t in "cz").astype(_NP[t])


def serving_trace(rate: float, seconds: float, stream: int = 0, cfg: dict = SERVING) -> dict:
    """Arrivals of a Poisson stream (seeded exponential gaps) over `seconds`:
    per request its arrival offset t, size bin (m log-uniform in
    [m_lo, m_hi], rounded to the nearest bin in log scale), shape (half
    square, half 2:1 tall), type (by dtype_p) and pool variant."""
    rng = rng_for(cfg["seed"] + 1, stream)
    n_est = int(rate * seconds * 1.2 + 100)
    t = np.cumsum(rng.exponential(1.0 / rate, n_est))
    while t[-1] < seconds:
        t = np.concatenate([t, t[-1] + np.cumsum(rng.exponential(1.0 / rate, n_est))])
    t = t[t < seconds]
    N = len(t)
    lo, hi = np.log(cfg["m_lo"]), np.log(cfg["m_hi"])
    u = rng.uniform(lo, hi, N)
    sizes = serving_sizes(cfg)
    ls = np.log(sizes)
    b = np.searchsorted((ls[:-1] + ls[1:]) / 2, u)          # nearest bin in log scale
    tall = rng.random(N) < 0.5
    dt = rng.choice(len(cfg["dtypes"]), size=N, p=cfg["dtype_p"])
    v = rng.integers(0, cfg["variants"], N)
    return {"t": t, "bin": b, "tall": tall, "dtype": np.array(cfg["dtypes"])[dt], "variant": v}
