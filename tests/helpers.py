"""Shared test helpers: device transfer and element-by-element comparison of a
library result with the oracle."""
from __future__ import annotations

import numpy as np

import oracle
from workloads.csc import CSC

# float32 unit roundoff; float64 unit roundoff
U32 = 2.0 ** -24
U64 = 2.0 ** -53


def to_dev(h: CSC):
    import paper_2010_08526_gb300 as spg
    return spg.Csc.from_host(h, device="cuda")


def host_csc(c, nrows=None) -> CSC:
    """A library Csc (or (colptr, rowidx, vals) tensors) as a host CSC."""
    if isinstance(c, tuple):
        cp, ri, va = (x.cpu().numpy() for x in c)
        return CSC(nrows, cp.size - 1, cp.astype(np.int64), ri.astype(np.int64), va)
    _, ncols, cp, ri, va = c.to_host()
    return CSC(c.nrows, ncols, cp.astype(np.int64), ri.astype(np.int64), va)


def tol_of(dtype, f=None):
    """Allowed |gpu - ref| per unit of sum|terms| for one output entry.

    float64: 1e-12. float32 with float32 accumulation: 1e-5, or the bound for
    recursive summation in any order, gamma_f ~ f * u32, for columns whose
    f_j terms make that larger (any summation order of f terms may err by up
    to (f-1) u sum|terms|, plus u sum|terms| for the products). int64: exact.
    """
    dt = np.dtype(dtype)
    if dt == np.float64:
        base = 1e-12
        return base if f is None else np.maximum(base, (f + 1) * U64 * 1.01)
    if dt == np.float32:
        base = 1e-5
        return base if f is None else np.maximum(base, (f + 1) * U32 * 1.01)
    return 0.0


def assert_matches(gpu: CSC, ref: CSC, absterm=None, f_col=None, *, exact=False, label=""):
    """Structure and per-column nnz bit-exact after the canonical per-column
    sort; values exact (int) or within tol * sum|terms| (float)."""
    g = oracle.canonical(gpu)
    assert g.ncols == ref.ncols, label
    assert np.array_equal(np.asarray(g.colptr, np.int64), np.asarray(ref.colptr, np.int64)), \
        f"{label}: per-column nnz differs"
    assert np.array_equal(np.asarray(g.rowidx, np.int64), np.asarray(ref.rowidx, np.int64)), \
        f"{label}: row structure differs"
    gv = np.asarray(g.vals)
    rv = np.asarray(ref.vals)
    if exact or np.issubdtype(gv.dtype, np.integer):
        assert np.array_equal(gv.astype(np.int64), rv.astype(np.int64)), f"{label}: int values differ"
        return 0.0
    err = np.abs(gv.astype(np.float64) - rv.astype(np.float64))
    scale = absterm if absterm is not None else np.abs(rv)
    if f_col is not None:
        fe = np.repeat(np.asarray(f_col, np.float64), np.diff(np.asarray(ref.colptr, np.int64)))
        tol = tol_of(gv.dtype, fe)
    else:
        tol = tol_of(gv.dtype)
    bad = err > tol * scale + 1e-300
    if bad.any():
        i = int(np.flatnonzero(bad)[0])
        raise AssertionError(f"{label}: value mismatch at entry {i}: gpu {gv[i]!r} ref {rv[i]!r} "
                             f"err {err[i]:.3e} scale {scale[i]:.3e} ({int(bad.sum())} bad)")
    rel = err / np.maximum(np.abs(rv), 1e-300)
    return float(rel.max()) if rel.size else 0.0
