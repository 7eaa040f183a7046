"""Batched one-sided Jacobi SVD for NVIDIA GB300 (sm_103a).

The method of Abdelfattah and Fasi, "An Efficient Batch Solver for the
Singular Value Decomposition on GPUs": blocked one-sided Jacobi with one
inner Jacobi sweep per Gram block, fused vector updates and per-matrix
masking, as hand-written CUDA kernels behind the C-ABI of include/bsvd.h.

    import paper_2601_17979_gb300 as bsvd
    bsvd.build()                         # nvcc, once
    res = bsvd.gesvj(A)                  # A: CUDA tensor (batch, m, n)
    res.S, res.U, res.V, res.info, res.sweeps
"""
from .buildlib import build
from .binding import (BsvdError, SVDResult, Server, gesvj, gesvj_host, host_workspace_bytes, gesvj_batched,
                      autotune, autotune_batched, persistent_plan, load, handle, make_opts,
                      column_major, empty_column_major, workspace_bytes, EXPORTS,
                      FLAG_NO_V_CORRECTION, FLAG_TWO_STAGE, FLAG_NO_MASKS, FLAG_NO_GRAPH,
                      FLAG_SYNC_CHECK, FLAG_QR, FLAG_SPLIT_LARGE, FLAG_F32_FFMA, FLAG_WIDE_ANGLES, FLAG_NO_ONCHIP, FLAG_SPLIT_F32, FLAG_HOST_LOOP, FLAG_THREE_KERNELS)

__all__ = ["build", "BsvdError", "SVDResult", "Server", "gesvj", "gesvj_host", "host_workspace_bytes", "gesvj_batched", "autotune", "autotune_batched", "persistent_plan", "load", "handle",
           "make_opts", "column_major", "empty_column_major", "workspace_bytes", "EXPORTS",
           "FLAG_NO_V_CORRECTION", "FLAG_TWO_STAGE", "FLAG_NO_MASKS", "FLAG_NO_GRAPH",
           "FLAG_SYNC_CHECK", "FLAG_QR", "FLAG_SPLIT_LARGE", "FLAG_F32_FFMA", "FLAG_WIDE_ANGLES", "FLAG_NO_ONCHIP", "FLAG_SPLIT_F32", "FLAG_HOST_LOOP", "FLAG_THREE_KERNELS"]
