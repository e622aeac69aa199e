"""GB300 (sm_103a) memory-constrained SpGEMM -- Python binding.

Thin marshalling over the C ABI in include/spgemm.h: every step of the
product (flop count, symbolic count, batch plan, hash / dense numeric, merge,
backward) runs in the library's CUDA kernels. torch supplies device memory
and streams. There is no CPU fallback: without the built library or a GPU,
calls raise.

Main entry points
-----------------
``Csc``                 device CSC matrix (torch tensors)
``Plan``                symbolic step, batch plan, numeric per batch
``spgemm(A, B)``        C = A*B (all batches concatenated)
``merge(parts)``        sort-free hash merge of partial products
``prune(C, thr, k)``    column-wise threshold / top-k prune of a result batch
``run_batched(...)``    batch loop streaming C to pinned host memory
``transpose(A)``        A^T on the device; ``spgemm_aat(A)`` = A A^T
``run_row_batched(..)`` row-by-row batches of C (column batches of C^T)
``SpGEMMFn``            autograd Function (masked-SpGEMM backward)
``Multi``               many independent products in one pass (CUDA graph)
"""
from __future__ import annotations

from ._capi import SpgemmError, load
from .core import (
    Csc,
    Plan,
    Tuning,
    spgemm,
    merge,
    merge_noalloc,
    prune,
    run_batched,
    transpose,
    spgemm_aat,
    run_row_batched,
    backward,
    SpGEMMFn,
    Multi,
    TorchAllocator,
)

__all__ = [
    "SpgemmError", "load", "Csc", "Plan", "Tuning", "spgemm", "merge", "merge_noalloc", "prune", "run_batched", "transpose",
    "spgemm_aat", "run_row_batched",
    "backward", "SpGEMMFn", "Multi", "TorchAllocator",
]
