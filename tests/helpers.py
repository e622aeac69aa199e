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


def tol_of(dtype, nterm=None):
    """Allowed |gpu - ref| per unit of sum|terms| for one output entry.

    float64: 1e-12; float32 with float32 accumulation: 1e-5 (the north-star
    tolerances). An entry formed from n products (``nterm``, the oracle's
    per-entry count n_ij) may, summed in any order, err by up to
    (n - 1) u sum|terms| from the additions plus u sum|terms| from rounding
    the products (the recursive-summation bound, which holds for every
    summation order and tree), so the allowance per entry is
    max(base, (n + 1) u * 1.01). int64: exact.
    """
    dt = np.dtype(dtype)
    if dt == np.float64:
        base, u = 1e-12, U64
    elif dt == np.float32:
        base, u = 1e-5, U32
    else:
        return 0.0
    if nterm is None:
        return base
    return np.maximum(base, (np.asarray(nterm, np.float64) + 1.0) * u * 1.01)


# Largest plain-relative error |gpu - ref| / |ref| of every float check, per
# test (printed by conftest.py at the end of the run).
REL_ERRORS: dict = {}


def record_rel(label: str, rel: float) -> None:
    import os
    test = os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]
    key = f"{test} [{label}]" if label else test
    REL_ERRORS[key] = max(rel, REL_ERRORS.get(key, 0.0))


def assert_matches(gpu: CSC, ref: CSC, absterm=None, nterm=None, *, exact=False, label=""):
    """Structure and per-column nnz bit-exact after the canonical per-column
    sort; values exact (int) or within tol_of(dtype, n_ij) * sum|terms| per
    entry (float). Returns the largest plain-relative error and records it."""
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
    tol = tol_of(gv.dtype, nterm)
    bad = err > tol * scale + 1e-300
    if bad.any():
        i = int(np.flatnonzero(bad)[0])
        t = tol[i] if np.ndim(tol) else tol
        raise AssertionError(f"{label}: value mismatch at entry {i}: gpu {gv[i]!r} ref {rv[i]!r} "
                             f"err {err[i]:.3e} scale {scale[i]:.3e} tol {t:.3e} "
                             f"({int(bad.sum())} bad)")
    nz = np.abs(rv) > 0
    rel = err[nz] / np.abs(rv[nz])
    worst = float(rel.max()) if rel.size else 0.0
    record_rel(label, worst)
    return worst
