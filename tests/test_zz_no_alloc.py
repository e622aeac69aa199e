"""spgemm_merge_noalloc: the merge for callers that may not allocate device
memory (for example code running under another framework's fixed device-memory
pool). It must give the same result as spgemm_merge, the allocating entry
point, on consecutive calls that share its one static scratch array.

This file is collected last on purpose; it passes alone in a fresh process
and after the other tests.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from workloads.csc import CSC, from_coo, shuffle_within_columns

from helpers import host_csc, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_08526_gb300 as spg  # noqa: E402


def parts_of(m, n, nparts, density, seed, value_dtype=np.float64, index_dtype=np.int32):
    rng = np.random.default_rng(seed)
    out = []
    for t in range(nparts):
        nnz = int(m * n * density)
        r = rng.integers(0, m, nnz)
        c = rng.integers(0, n, nnz)
        if np.dtype(value_dtype) == np.int64:
            v = rng.integers(-9, 10, nnz).astype(np.int64)
        else:
            v = rng.standard_normal(nnz)
        p = from_coo(m, n, r, c, v, dup="sum", index_dtype=index_dtype, value_dtype=value_dtype)
        out.append(shuffle_within_columns(p, seed + t))
    return out


def same_result(a: CSC, b: CSC, exact: bool):
    """Structure and per-column counts bit-exact after the canonical sort;
    values exact for integers, within 1e-12 of each other for float64 (the
    two entry points may add a row's few terms in different orders)."""
    ca, cb = oracle.canonical(a), oracle.canonical(b)
    assert np.array_equal(ca.colptr, cb.colptr)
    assert np.array_equal(ca.rowidx, cb.rowidx)
    if exact:
        assert np.array_equal(ca.vals, cb.vals)
    else:
        np.testing.assert_allclose(ca.vals, cb.vals, rtol=1e-12, atol=1e-12)


def test_noalloc_merge_matches_allocating_merge_on_consecutive_calls():
    first = parts_of(3000, 2500, 4, 0.002, 1)
    second = parts_of(1200, 4100, 3, 0.004, 2)       # other shape: stale scratch must not leak
    for parts in (first, second, first):
        dev = [to_dev(p) for p in parts]
        got = spg.merge_noalloc(dev)
        ref = spg.merge(dev)
        torch.cuda.synchronize()
        same_result(host_csc(got), host_csc(ref), exact=False)
        same_result(host_csc(got), oracle.merge(parts), exact=False)


def test_noalloc_merge_int64_and_int64_indices():
    parts = parts_of(2000, 1800, 3, 0.003, 5, value_dtype=np.int64, index_dtype=np.int64)
    dev = [to_dev(p) for p in parts]
    for _ in range(2):
        got = spg.merge_noalloc(dev)
        ref = spg.merge(dev)
        torch.cuda.synchronize()
        same_result(host_csc(got), host_csc(ref), exact=True)


def test_noalloc_merge_rejects_inputs_beyond_its_scratch():
    n = 2_000_000                      # 29 B per column: more than the 32 MiB array
    empty = CSC(10, n, np.zeros(n + 1, np.int32), np.zeros(0, np.int32), np.zeros(0))
    with pytest.raises(spg.SpgemmError, match="scratch"):
        spg.merge_noalloc([to_dev(empty)])
    # a column above the largest shared-memory hash table is refused, not run
    rng = np.random.default_rng(3)
    rows = rng.choice(50_000, 9000, replace=False)
    dense_col = from_coo(50_000, 2, rows, np.zeros(rows.size, np.int64), np.ones(rows.size))
    with pytest.raises(spg.SpgemmError, match="8192"):
        spg.merge_noalloc([to_dev(dense_col)])
    # and the entry point still works afterwards
    parts = parts_of(500, 400, 2, 0.01, 7)
    dev = [to_dev(p) for p in parts]
    same_result(host_csc(spg.merge_noalloc(dev)), host_csc(spg.merge(dev)), exact=False)


def _same_rows_parts(nrows, rows_per_part, nparts, seed):
    """nparts parts of one column, each holding the same rows_per_part rows
    (different values): they merge to rows_per_part rows, while the entries
    summed over the parts are nparts * rows_per_part."""
    rng = np.random.default_rng(seed)
    rows = rng.choice(nrows, rows_per_part, replace=False)
    out = []
    for t in range(nparts):
        v = rng.standard_normal(rows.size)
        p = from_coo(nrows, 3, rows, np.ones(rows.size, np.int64), v)
        out.append(shuffle_within_columns(p, seed + t))
    return out


def test_noalloc_limit_is_entries_over_parts_not_distinct_rows():
    """The documented limit: per column, entries summed over the parts (capped
    at nrows) at most 8192. 4 parts of the same 2,000 rows (8,000 entries) are
    merged; 4 parts of the same 3,000 rows (12,000 entries, still 3,000
    distinct rows) are refused."""
    ok = _same_rows_parts(50_000, 2000, 4, 11)
    dev = [to_dev(p) for p in ok]
    got = spg.merge_noalloc(dev)
    torch.cuda.synchronize()
    same_result(host_csc(got), oracle.merge(ok), exact=False)
    assert int(got.nnz) == 2000
    over = _same_rows_parts(50_000, 3000, 4, 12)
    with pytest.raises(spg.SpgemmError, match="8192"):
        spg.merge_noalloc([to_dev(p) for p in over])
    # the row-count cap: with nrows <= 8192 every column is accepted
    small = _same_rows_parts(6000, 3000, 4, 13)
    got = spg.merge_noalloc([to_dev(p) for p in small])
    torch.cuda.synchronize()
    same_result(host_csc(got), oracle.merge(small), exact=False)


def test_noalloc_merge_of_k_stage_partials():
    """The k-split use: the parts are the 4 stage products D_t = A(:, K_t)
    A(K_t, :) of a small R-MAT A*A (Algorithm 1's stages), which share most
    of their rows column by column; the merge must equal A*A (oracle) and
    spgemm_merge, on two calls in a row."""
    import workloads as W
    A = W.rmat(11, 8, 20108599, index_dtype=np.int32, value_dtype=np.float64)
    stages = [oracle.spgemm(A, A, krange=kr) for kr in oracle.stage_ranges(A.ncols, 4)]
    parts = [CSC(p.nrows, p.ncols, p.colptr.astype(np.int32), p.rowidx.astype(np.int32), p.vals)
             for p in stages]
    ref, ab = oracle.spgemm(A, A, with_absterm=True)
    dev = [to_dev(p) for p in parts]
    for _ in range(2):
        got = spg.merge_noalloc(dev)
        alloc = spg.merge(dev)
        torch.cuda.synchronize()
        same_result(host_csc(got), host_csc(alloc), exact=False)
        g = oracle.canonical(host_csc(got))
        assert np.array_equal(g.colptr, ref.colptr) and np.array_equal(g.rowidx, ref.rowidx)
        assert np.all(np.abs(g.vals - ref.vals) <= 1e-12 * ab + 1e-300)
