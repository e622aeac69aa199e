"""Seeded generators for the five synthetic workloads.

Recipes (sizes, distributions, seeds) are the ones the design notes state;
each ``configN`` function returns exactly that workload. Seeds are
``CONFIG_SEED_BASE + N``; everything is drawn from numpy ``default_rng``.
"""
from __future__ import annotations

import math

import numpy as np

from .csc import CSC, from_coo

CONFIG_SEED_BASE = 20108526


def config_seed(n: int) -> int:
    return CONFIG_SEED_BASE + n


def _draw_values(rng, n, dist, value_dtype):
    if dist == "uniform":
        return rng.random(n).astype(value_dtype)
    if dist == "normal":
        return rng.standard_normal(n).astype(value_dtype)
    if dist == "ones":
        return np.ones(n, dtype=value_dtype)
    if isinstance(dist, tuple) and dist[0] == "uniform":
        lo, hi = dist[1], dist[2]
        return rng.uniform(lo, hi, n).astype(value_dtype)
    if dist == "smallint":
        return rng.integers(-3, 4, n).astype(value_dtype)
    raise ValueError(dist)


def _distinct_rows(rng, nrows: int, counts: np.ndarray) -> np.ndarray:
    """Per column, ``counts[j]`` distinct rows uniform without replacement,
    returned flat in draw order (not sorted)."""
    counts = counts.astype(np.int64)
    ncols = counts.size
    total = int(counts.sum())
    cols = np.repeat(np.arange(ncols, dtype=np.int64), counts)
    rows = rng.integers(0, nrows, size=total, dtype=np.int64)
    dense = counts * 4 > nrows  # near-dense columns: draw a permutation prefix
    if dense.any():
        starts = np.zeros(ncols + 1, dtype=np.int64)
        np.cumsum(counts, out=starts[1:])
        for j in np.flatnonzero(dense):
            rows[starts[j]:starts[j + 1]] = rng.permutation(nrows)[: counts[j]]
    for _ in range(1000):
        key = cols * nrows + rows
        order = np.argsort(key, kind="stable")
        ks = key[order]
        dup_sorted = np.zeros(total, dtype=bool)
        if total > 1:
            dup_sorted[1:] = ks[1:] == ks[:-1]
        if not dup_sorted.any():
            return rows
        bad = order[dup_sorted]
        rows[bad] = rng.integers(0, nrows, size=bad.size, dtype=np.int64)
    raise RuntimeError("could not draw distinct rows")


def er_exact(nrows: int, ncols: int, d: int, seed: int, *, index_dtype=np.int32,
             value_dtype=np.float64, dist="uniform") -> CSC:
    """Each column: exactly ``min(d, nrows)`` distinct uniform rows, stored in
    draw order (unsorted within columns)."""
    rng = np.random.default_rng(seed)
    d = min(d, nrows)
    counts = np.full(ncols, d, dtype=np.int64)
    rows = _distinct_rows(rng, nrows, counts)
    vals = _draw_values(rng, rows.size, dist, value_dtype)
    colptr = np.arange(ncols + 1, dtype=np.int64) * d
    it = np.dtype(index_dtype)
    return CSC(nrows, ncols, colptr.astype(it), rows.astype(it), vals)


def er_binomial(n: int, dbar: float, seed, *, index_dtype=np.int32,
                value_dtype=np.int64, dist="ones") -> CSC:
    """G(n, p) with p = dbar/n: column counts ~ Binomial(n, p), rows drawn
    without replacement, stored unsorted."""
    rng = seed if isinstance(seed, np.random.Generator) else np.random.default_rng(seed)
    counts = rng.binomial(n, dbar / n, size=n).astype(np.int64)
    rows = _distinct_rows(rng, n, counts)
    vals = _draw_values(rng, rows.size, dist, value_dtype)
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=colptr[1:])
    it = np.dtype(index_dtype)
    return CSC(n, n, colptr.astype(it), rows.astype(it), vals)


def rmat(scale: int, edge_factor: int, seed: int, *, a=0.57, b=0.19, c=0.19,
         index_dtype=np.int32, value_dtype=np.float32) -> CSC:
    """R-MAT: ``edge_factor * 2**scale`` edge draws, each choosing one of the
    four quadrants independently at every level (no noise, no vertex
    permutation). Edge values X ~ U(0,1); the result is A = X + X^T with
    duplicate (row, col) summed, so self-loops are doubled."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    e = edge_factor * n
    r = np.zeros(e, dtype=np.int64)
    cidx = np.zeros(e, dtype=np.int64)
    ab, abc = a + b, a + b + c
    for lvl in range(scale):
        u = rng.random(e)
        bit = np.int64(1) << np.int64(scale - 1 - lvl)
        rbit = u >= ab                      # quadrants c, d: lower half
        cbit = ((u >= a) & (u < ab)) | (u >= abc)  # quadrants b, d: right half
        r += rbit.astype(np.int64) * bit
        cidx += cbit.astype(np.int64) * bit
        del u, rbit, cbit
    x = rng.random(e).astype(np.float32)
    rows = np.concatenate([r, cidx])
    cols = np.concatenate([cidx, r])
    vals = np.concatenate([x, x])
    del r, cidx, x
    return from_coo(n, n, rows, cols, vals, dup="sum", index_dtype=index_dtype,
                    value_dtype=value_dtype)


def lognormal_symmetric(n: int, seed: int, *, mean=40.0, sigma=1.2, cap=5000,
                        index_dtype=np.int64, value_dtype=np.float32,
                        lo=0.3, hi=1.0) -> CSC:
    """Symmetric matrix with lognormal target degrees.

    d_i = clip(round(Lognormal(mu, sigma)), 1, cap) with mu = ln(mean) -
    sigma^2/2 (so ``mean`` is the distribution mean). Vertex i draws
    ceil(d_i/2) partners j != i with probability proportional to d_j
    (Chung-Lu). Each drawn unordered pair gets a value U(lo, hi); repeated
    pairs keep the largest value; both (i,j) and (j,i) are stored with it.
    """
    rng = np.random.default_rng(seed)
    mu = math.log(mean) - sigma * sigma / 2.0
    d = np.clip(np.rint(rng.lognormal(mu, sigma, n)), 1, cap).astype(np.int64)
    k = (d + 1) // 2
    src = np.repeat(np.arange(n, dtype=np.int64), k)
    cw = np.cumsum(d.astype(np.float64))
    dst = np.searchsorted(cw, rng.random(src.size) * cw[-1], side="right")
    np.minimum(dst, n - 1, out=dst)
    keep = dst != src
    src, dst = src[keep], dst[keep]
    val = rng.uniform(lo, hi, src.size).astype(value_dtype)
    lo_i = np.minimum(src, dst)
    hi_i = np.maximum(src, dst)
    del src, dst, keep
    # unordered pairs, duplicates keep their max value
    half = from_coo(n, n, lo_i, hi_i, val, dup="max", index_dtype=np.int64,
                    value_dtype=value_dtype)
    del lo_i, hi_i, val
    hcols = np.repeat(np.arange(n, dtype=np.int64), half.col_counts())
    hrows = half.rowidx.astype(np.int64)
    rows = np.concatenate([hrows, hcols])
    cols = np.concatenate([hcols, hrows])
    vals = np.concatenate([half.vals, half.vals])
    del half, hcols, hrows
    return from_coo(n, n, rows, cols, vals, dup="error", index_dtype=index_dtype,
                    value_dtype=value_dtype)


def multi_problem_set(count: int, seed: int, *, nmin=1000, nmax=200000, dmin=2.0,
                      dmax=32.0, index_dtype=np.int32, value_dtype=np.int64):
    """``count`` independent G(n_i, d_i/n_i) matrices, n_i log-uniform in
    [nmin, nmax] (rounded), d_i ~ U(dmin, dmax), all values 1."""
    rng = np.random.default_rng(seed)
    ns = np.rint(np.exp(rng.uniform(math.log(nmin), math.log(nmax), count))).astype(np.int64)
    ds = rng.uniform(dmin, dmax, count)
    return [er_binomial(int(n), float(dd), rng, index_dtype=index_dtype,
                        value_dtype=value_dtype) for n, dd in zip(ns, ds)]


def values_on_pattern(pattern: CSC, seed: int, *, dist="normal", value_dtype=None) -> CSC:
    """A CSC with ``pattern``'s structure and fresh seeded values."""
    rng = np.random.default_rng(seed)
    vt = pattern.vals.dtype if value_dtype is None else np.dtype(value_dtype)
    vals = _draw_values(rng, pattern.nnz, dist, vt)
    return CSC(pattern.nrows, pattern.ncols, pattern.colptr.copy(), pattern.rowidx.copy(), vals)


# ---------------------------------------------------------------------------
# The five workloads (small-case variants take the same recipe at other sizes)
# ---------------------------------------------------------------------------

def config1(n: int = 4096, d: int = 8) -> CSC:
    """Erdos-Renyi, exactly 8 distinct rows per column, fp64 U(0,1), int32."""
    return er_exact(n, n, d, config_seed(1), index_dtype=np.int32, value_dtype=np.float64)


def config2(scale: int = 20, edge_factor: int = 16) -> CSC:
    """R-MAT scale 20, edge factor 16, symmetrised with duplicates summed,
    fp32 U(0,1), int32."""
    return rmat(scale, edge_factor, config_seed(2), index_dtype=np.int32, value_dtype=np.float32)


def config3(n: int = 2_000_000) -> CSC:
    """Protein-similarity stand-in: symmetric, lognormal degrees (mean 40,
    sigma 1.2, cap 5000), values U(0.3, 1.0) fp32, int64 indices."""
    return lognormal_symmetric(n, config_seed(3), index_dtype=np.int64, value_dtype=np.float32)


def config4(count: int = 512, nmax: int = 200000):
    """512 uneven G(n, p) problems, int64 values all 1, int32 indices."""
    return multi_problem_set(count, config_seed(4), nmax=nmax)


def config5(m: int = 200_000, k: int = 200_000, n: int = 100_000, da: int = 16,
            db: int = 8, value_dtype=np.float32):
    """A (m x k, 16 distinct rows per column) and B (k x n, 8 per column),
    N(0,1) values, int32. G's values are drawn later on C's pattern."""
    s = config_seed(5)
    a = er_exact(m, k, da, s, index_dtype=np.int32, value_dtype=value_dtype, dist="normal")
    b = er_exact(k, n, db, s + 1000, index_dtype=np.int32, value_dtype=value_dtype, dist="normal")
    return a, b
