"""CPU oracle for the SpGEMM hot path -- TEST INFRASTRUCTURE ONLY.

The plain definition of everything the CUDA path computes, used to check it:
only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. It shares no code with the library
(``paper_2010_08526_gb300``) and never imports it.

Arithmetic lives in ``spgemm_oracle.c`` (loaded through ctypes); this module
widens indices to int64, upcasts float32 values to float64 (exact), and holds
the few closed-form formulas of the paper that are plain arithmetic on counts
(the memory model of Eq. (1) and the batch-count bound of Eq. (2)).

Parity status of each function is pinned by ``tests/test_oracle_pins.py``:
every function below has at least one independent pin (dense products, brute
force, closed forms, invariants); none is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from workloads.csc import CSC

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


class _OCSC(ctypes.Structure):
    _fields_ = [
        ("nrows", ctypes.c_int64),
        ("ncols", ctypes.c_int64),
        ("colptr", ctypes.c_void_p),
        ("rowidx", ctypes.c_void_p),
        ("vals", ctypes.c_void_p),
    ]


def _lib():
    global _LIB
    if _LIB is None:
        from . import build as _b
        path = _b.build()
        lib = ctypes.CDLL(path)
        P = ctypes.POINTER
        i64 = ctypes.c_int64
        vp = ctypes.c_void_p
        lib.oracle_flops.argtypes = [P(_OCSC), P(_OCSC), i64, i64, vp]
        lib.oracle_symbolic.argtypes = [P(_OCSC), P(_OCSC), i64, i64, i64, i64, vp]
        lib.oracle_spgemm.argtypes = [P(_OCSC), P(_OCSC), ctypes.c_int, i64, i64, i64, i64,
                                      vp, vp, vp, vp, vp]
        lib.oracle_merge.argtypes = [P(_OCSC), ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                     vp, vp, vp]
        lib.oracle_backward.argtypes = [P(_OCSC), P(_OCSC), P(_OCSC), vp, vp]
        lib.oracle_plan_batches.argtypes = [vp, i64, i64, vp]
        lib.oracle_prune.argtypes = [P(_OCSC), ctypes.c_int, ctypes.c_double, i64, ctypes.c_int,
                                     vp, vp, vp]
        lib.oracle_plan_batches.restype = i64
        lib.oracle_num_threads.restype = ctypes.c_int
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _LIB = lib
    return _LIB


def num_threads() -> int:
    return int(_lib().oracle_num_threads())


def set_threads(n: int) -> None:
    _lib().oracle_set_threads(int(n))


def _vtype(dtype) -> int:
    dt = np.dtype(dtype)
    if np.issubdtype(dt, np.integer):
        return 2
    return 0


class _Held:
    """Keeps the widened arrays alive while the C side points at them."""

    def __init__(self, a: CSC, vtype: int):
        self.colptr = np.ascontiguousarray(a.colptr, dtype=np.int64)
        self.rowidx = np.ascontiguousarray(a.rowidx, dtype=np.int64)
        vt = np.int64 if vtype in (2, 5) else np.float64
        self.vals = np.ascontiguousarray(a.vals, dtype=vt)
        self.s = _OCSC(a.nrows, a.ncols, self.colptr.ctypes.data, self.rowidx.ctypes.data,
                       self.vals.ctypes.data)


def _ptr(x: np.ndarray):
    return ctypes.c_void_p(x.ctypes.data)


def stage_ranges(k: int, s: int):
    """Contiguous k-stages K_t = [floor(t k / s), floor((t+1) k / s)),
    t = 0..s-1: A split by columns and B by rows (Sec. III-B, Fig. 1(c),(f))."""
    return [(t * k // s, (t + 1) * k // s) for t in range(s)]


def flops_per_column(A: CSC, B: CSC, krange=None) -> np.ndarray:
    """f_j = number of multiplications forming C(:, j) (Sec. II-A)."""
    k0, k1 = (0, A.ncols) if krange is None else krange
    vt = _vtype(A.vals.dtype)
    ha, hb = _Held(A, vt), _Held(B, vt)
    f = np.zeros(B.ncols, dtype=np.int64)
    _lib().oracle_flops(ctypes.byref(ha.s), ctypes.byref(hb.s), k0, k1, _ptr(f))
    return f


def symbolic(A: CSC, B: CSC, krange=None, cols=None) -> np.ndarray:
    """nnz(C(:, j)) for j in ``cols`` (LocalSymbolic of Algorithm 3)."""
    k0, k1 = (0, A.ncols) if krange is None else krange
    c0, c1 = (0, B.ncols) if cols is None else cols
    vt = _vtype(A.vals.dtype)
    ha, hb = _Held(A, vt), _Held(B, vt)
    cnt = np.zeros(c1 - c0, dtype=np.int64)
    _lib().oracle_symbolic(ctypes.byref(ha.s), ctypes.byref(hb.s), k0, k1, c0, c1, _ptr(cnt))
    return cnt


def _sr_vtype(dtype, semiring: str) -> int:
    if semiring == "plus_times":
        return _vtype(dtype)
    if semiring == "min_plus":
        if _vtype(dtype) != 0:
            raise ValueError("min_plus is defined for floating-point values")
        return 3
    if semiring == "or_and":
        return 5 if _vtype(dtype) == 2 else 4
    raise ValueError(f"unknown semiring {semiring!r}")


def spgemm(A: CSC, B: CSC, krange=None, cols=None, with_absterm: bool = False,
           semiring: str = "plus_times", with_nterm: bool = False):
    """C(:, c0:c1) = A(:, K) B(K, c0:c1) by column Gustavson (Sec. II-C).

    semiring "min_plus": C(i, j) = min over k of A(i, k) + B(k, j) on the same
    structure (the algorithms hold over any semiring, Sec. II); NaN products
    are ignored. "or_and": C(i, j) = 1 if A(i, k) != 0 and B(k, j) != 0 for
    some k, else 0 (Boolean values in the input's value type).

    Returns a CSC (int64 indices, float64 or int64 values, rows sorted) and,
    if asked, the per-entry rounding-error scale: sum |products| (plus-times)
    or the largest |a| + |b| over the entry's candidates (min-plus); and, with
    ``with_nterm``, the per-entry number of products n_ij that reach (i, j)
    (the n of that entry's own summation error bound). The result is
    C, then absterm if asked, then nterm if asked.
    """
    if A.ncols != B.nrows:
        raise ValueError("inner dimensions differ")
    k0, k1 = (0, A.ncols) if krange is None else krange
    c0, c1 = (0, B.ncols) if cols is None else cols
    vt = _sr_vtype(A.vals.dtype, semiring)
    ha, hb = _Held(A, vt), _Held(B, vt)
    lib = _lib()
    cnt = np.zeros(c1 - c0, dtype=np.int64)
    lib.oracle_symbolic(ctypes.byref(ha.s), ctypes.byref(hb.s), k0, k1, c0, c1, _ptr(cnt))
    colptr = np.zeros(c1 - c0 + 1, dtype=np.int64)
    np.cumsum(cnt, out=colptr[1:])
    nnz = int(colptr[-1])
    rowidx = np.zeros(nnz, dtype=np.int64)
    vals = np.zeros(nnz, dtype=np.int64 if vt in (2, 5) else np.float64)
    absterm = np.zeros(nnz, dtype=np.float64) if (with_absterm and vt in (0, 3)) else None
    nterm = np.zeros(nnz, dtype=np.int64) if with_nterm else None
    lib.oracle_spgemm(ctypes.byref(ha.s), ctypes.byref(hb.s), vt, k0, k1, c0, c1,
                      _ptr(colptr), _ptr(rowidx), _ptr(vals),
                      _ptr(absterm) if absterm is not None else None,
                      _ptr(nterm) if nterm is not None else None)
    C = CSC(A.nrows, c1 - c0, colptr, rowidx, vals)
    out = (C,)
    if with_absterm:
        out += (absterm,)
    if with_nterm:
        out += (nterm,)
    return out if len(out) > 1 else C


def merge(parts, semiring: str = "plus_times") -> CSC:
    """Add entries of equal (row, col) across ``parts`` (Sec. III-A merge;
    column j of the result formed from column j of every part, Sec. IV-D);
    "min_plus" takes their minimum, "or_and" their OR (1 if one is nonzero)."""
    parts = list(parts)
    if not parts:
        raise ValueError("no parts")
    m, n = parts[0].nrows, parts[0].ncols
    for p in parts:
        if p.nrows != m or p.ncols != n:
            raise ValueError("parts differ in shape")
    vt = _sr_vtype(parts[0].vals.dtype, semiring)
    held = [_Held(p, vt) for p in parts]
    arr = (_OCSC * len(parts))(*[h.s for h in held])
    lib = _lib()
    colptr = np.zeros(n + 1, dtype=np.int64)
    lib.oracle_merge(arr, len(parts), vt, 1, _ptr(colptr), None, None)
    nnz = int(colptr[-1])
    rowidx = np.zeros(nnz, dtype=np.int64)
    vals = np.zeros(nnz, dtype=np.int64 if vt in (2, 5) else np.float64)
    lib.oracle_merge(arr, len(parts), vt, 0, _ptr(colptr), _ptr(rowidx), _ptr(vals))
    return CSC(m, n, colptr, rowidx, vals)


def prune(C: CSC, threshold: float = float("-inf"), topk: int = 0) -> CSC:
    """Column-wise prune of a result batch (the Markov-clustering consumer the
    column batches of Sec. III are formed for; HipMCL prunes each batch,
    Sec. V-F): per column keep the entries with value >= threshold, then, if
    topk > 0, only the topk largest of them (equal values: the earlier stored
    entry wins), written in their input order. Integer values compare against
    the smallest integer >= threshold."""
    vt = _vtype(C.vals.dtype)
    h = _Held(C, vt)
    lib = _lib()
    colptr = np.zeros(C.ncols + 1, dtype=np.int64)
    lib.oracle_prune(ctypes.byref(h.s), vt, float(threshold), int(topk), 1, _ptr(colptr), None, None)
    nnz = int(colptr[-1])
    rowidx = np.zeros(nnz, dtype=np.int64)
    vals = np.zeros(nnz, dtype=np.int64 if vt == 2 else np.float64)
    lib.oracle_prune(ctypes.byref(h.s), vt, float(threshold), int(topk), 0, _ptr(colptr), _ptr(rowidx),
                     _ptr(vals))
    return CSC(C.nrows, C.ncols, colptr, rowidx, vals)


def backward(A: CSC, B: CSC, G: CSC):
    """(dA, dB) for loss = sum(C * G) with G on pattern(C): dA = (G B^T) on
    pattern(A), dB = (A^T G) on pattern(B); float64, in A's / B's storage
    order."""
    ha, hb, hg = _Held(A, 0), _Held(B, 0), _Held(G, 0)
    dA = np.zeros(A.nnz, dtype=np.float64)
    dB = np.zeros(B.nnz, dtype=np.float64)
    _lib().oracle_backward(ctypes.byref(ha.s), ctypes.byref(hb.s), ctypes.byref(hg.s),
                           _ptr(dA), _ptr(dB))
    return dA, dB


# ---------------------------------------------------------------------------
# Memory model and batch count (Sec. IV-A)
# ---------------------------------------------------------------------------

def mem_bytes(r: int, unmerged_nnz_per_stage) -> int:
    """mem(C) = r * sum_k nnz(D^(k)) (Sec. IV-A, below Eq. (1))."""
    return int(r) * int(sum(int(x) for x in unmerged_nnz_per_stage))


def batch_lower_bound(mem_c: int, M: int, r: int, nnz_a: int, nnz_b: int) -> int:
    """Eq. (2): b >= ceil(mem(C) / (M - r (nnz(A) + nnz(B)))). Returns -1 when
    the inputs alone do not fit (denominator <= 0)."""
    den = int(M) - int(r) * (int(nnz_a) + int(nnz_b))
    if den <= 0:
        return -1
    return max(1, -(-int(mem_c) // den))


def column_bytes(W: np.ndarray, r: int, ptr_bytes: int) -> np.ndarray:
    """Bytes one output column occupies in a batch buffer: r per stored
    nonzero (r = index bytes + value bytes for CSC) plus one colptr entry."""
    return np.asarray(W, dtype=np.int64) * int(r) + int(ptr_bytes)


def plan_batches(w: np.ndarray, cap: int):
    """Contiguous column ranges, each holding at most ``cap`` bytes, cut
    greedily (smallest b for contiguous ranges: Sec. V-C picks the smallest b
    that fits). Returns the list of range starts plus n, or None when one
    column alone exceeds ``cap``."""
    w = np.ascontiguousarray(w, dtype=np.int64)
    begin = np.zeros(w.size + 2, dtype=np.int64)
    b = _lib().oracle_plan_batches(_ptr(w), w.size, int(cap), _ptr(begin))
    if b < 0:
        return None
    return begin[: b + 1].copy()


def plan_ranges(cost, n: int, cap: int):
    """The same greedy cut for a batch cost that is not a sum over columns:
    cost(c0, c1) = bytes a batch over columns [c0, c1) needs, non-decreasing
    as the range grows. Starting at column 0, each range is extended while
    the next column still fits under ``cap`` (Sec. V-C: the smallest b whose
    batches fit). Returns the range starts plus n, or None when a single
    column alone exceeds ``cap``. Plain Python; for the small plans of tests."""
    begin = [0]
    c = 0
    if n == 0:
        return np.array([0, 0], dtype=np.int64)
    while c < n:
        if cost(c, c + 1) > cap:
            return None
        x = c + 1
        while x < n and cost(c, x + 1) <= cap:
            x += 1
        begin.append(x)
        c = x
    return np.array(begin, dtype=np.int64)


def canonical(C: CSC) -> CSC:
    """Sort each column by row (the comparison form for sort-free outputs:
    Sec. IV-D keeps intermediate columns unsorted). Pure permutation."""
    cp = np.asarray(C.colptr, dtype=np.int64)
    cols = np.repeat(np.arange(C.ncols, dtype=np.int64), np.diff(cp))
    order = np.lexsort((np.asarray(C.rowidx, dtype=np.int64), cols))
    return CSC(C.nrows, C.ncols, cp.copy(), np.asarray(C.rowidx, dtype=np.int64)[order],
               np.asarray(C.vals)[order])
