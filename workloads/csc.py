"""A plain compressed-sparse-column container used to hand inputs around.

``CSC`` holds host numpy arrays: ``colptr`` (ncols+1), ``rowidx`` (nnz) and
``vals`` (nnz). Rows inside a column may be in any order (the kernels and the
oracle are both sort-free on input), but a (row, col) pair appears at most once.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np


@dataclass
class CSC:
    nrows: int
    ncols: int
    colptr: np.ndarray
    rowidx: np.ndarray
    vals: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.colptr[-1]) if len(self.colptr) else 0

    @property
    def index_dtype(self):
        return self.rowidx.dtype

    @property
    def value_dtype(self):
        return self.vals.dtype

    def col_counts(self) -> np.ndarray:
        return np.diff(self.colptr.astype(np.int64))

    def astype(self, index_dtype=None, value_dtype=None) -> "CSC":
        it = self.rowidx.dtype if index_dtype is None else np.dtype(index_dtype)
        vt = self.vals.dtype if value_dtype is None else np.dtype(value_dtype)
        return CSC(self.nrows, self.ncols, self.colptr.astype(it),
                   self.rowidx.astype(it), self.vals.astype(vt))

    def bytes(self) -> int:
        return self.colptr.nbytes + self.rowidx.nbytes + self.vals.nbytes

    def to_dense(self) -> np.ndarray:
        out = np.zeros((self.nrows, self.ncols), dtype=self.vals.dtype)
        cols = np.repeat(np.arange(self.ncols), self.col_counts())
        out[self.rowidx.astype(np.int64), cols] = self.vals
        return out

    def validate(self) -> None:
        cp = self.colptr.astype(np.int64)
        assert cp.shape == (self.ncols + 1,)
        assert cp[0] == 0 and np.all(np.diff(cp) >= 0)
        assert self.rowidx.shape == (cp[-1],) and self.vals.shape == (cp[-1],)
        if cp[-1]:
            r = self.rowidx.astype(np.int64)
            assert r.min() >= 0 and r.max() < self.nrows
            cols = np.repeat(np.arange(self.ncols, dtype=np.int64), np.diff(cp))
            key = cols * self.nrows + r
            assert np.unique(key).size == key.size, "duplicate (row, col)"


def from_coo(nrows: int, ncols: int, rows, cols, vals, *, dup: str = "sum",
             index_dtype=np.int32, value_dtype=None, sort_rows: bool = True) -> CSC:
    """Assemble CSC from coordinate triples.

    ``dup`` says what happens to repeated (row, col): ``"sum"`` adds the values
    (in float64 / int64, then casts), ``"max"`` keeps the largest, ``"error"``
    raises. Rows come out ascending within each column when ``sort_rows``.
    """
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals)
    vt = vals.dtype if value_dtype is None else np.dtype(value_dtype)
    key = cols * np.int64(nrows) + rows
    order = np.argsort(key, kind="stable")
    key = key[order]
    v = vals[order]
    if key.size:
        first = np.empty(key.size, dtype=bool)
        first[0] = True
        np.not_equal(key[1:], key[:-1], out=first[1:])
        starts = np.flatnonzero(first)
        if starts.size != key.size:
            if dup == "error":
                raise ValueError("duplicate (row, col) in COO input")
            if dup == "sum":
                acc = np.int64 if np.issubdtype(v.dtype, np.integer) else np.float64
                v = np.add.reduceat(v.astype(acc), starts)
            elif dup == "max":
                v = np.maximum.reduceat(v, starts)
            else:
                raise ValueError(dup)
            key = key[starts]
    ucols = key // nrows
    urows = key - ucols * nrows
    counts = np.bincount(ucols, minlength=ncols).astype(np.int64)
    colptr = np.zeros(ncols + 1, dtype=np.int64)
    np.cumsum(counts, out=colptr[1:])
    if not sort_rows:
        pass  # already sorted by key; callers shuffle explicitly if they want
    it = np.dtype(index_dtype)
    return CSC(nrows, ncols, colptr.astype(it), urows.astype(it), v.astype(vt))


def transpose(a: CSC) -> CSC:
    """Structural transpose (a permutation of the stored entries)."""
    cols = np.repeat(np.arange(a.ncols, dtype=np.int64), a.col_counts())
    return from_coo(a.ncols, a.nrows, cols, a.rowidx.astype(np.int64), a.vals,
                    dup="error", index_dtype=a.rowidx.dtype, value_dtype=a.vals.dtype)


def shuffle_within_columns(a: CSC, seed: int) -> CSC:
    """Same matrix, rows of each column stored in a random order."""
    rng = np.random.default_rng(seed)
    cols = np.repeat(np.arange(a.ncols, dtype=np.int64), a.col_counts())
    order = np.lexsort((rng.random(a.nnz), cols))
    return CSC(a.nrows, a.ncols, a.colptr.copy(), a.rowidx[order].copy(), a.vals[order].copy())


def column_slice(a: CSC, c0: int, c1: int) -> CSC:
    """Columns [c0, c1) of ``a`` as a standalone CSC (a copy)."""
    p0, p1 = int(a.colptr[c0]), int(a.colptr[c1])
    cp = (a.colptr[c0:c1 + 1].astype(np.int64) - p0).astype(a.colptr.dtype)
    return CSC(a.nrows, c1 - c0, cp, a.rowidx[p0:p1].copy(), a.vals[p0:p1].copy())
