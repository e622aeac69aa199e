"""The hybrid accumulator (Tuning(hybrid_sort=True)): a column of the CTA
hash tiers whose products fit its table, i.e. a low compression factor, is
accumulated by sorting its products by row and summing equal rows; other
columns keep the hash. Same results as the oracle in every semiring.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as W
from workloads.csc import CSC

from helpers import assert_matches, host_csc, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_08526_gb300 as spg  # noqa: E402

HYB = spg.Tuning(hybrid_sort=True)


def low_cf(n=8000, d=40, seed=3, value_dtype=np.float64, ints=False):
    """40 uniform rows per column: f_j = 1600 products on ~1450 distinct rows
    (cf ~1.1), so every column sits in a CTA tier with room for its products."""
    A = W.er_exact(n, n, d, seed, value_dtype=np.float64)
    rng = np.random.default_rng(seed + 1)
    v = rng.integers(-9, 10, A.nnz).astype(value_dtype) if ints else A.vals.astype(value_dtype)
    return CSC(A.nrows, A.ncols, A.colptr, A.rowidx, v)


def check_exact(C, ref, sorted_rows, label):
    got = host_csc(C)
    if not sorted_rows:
        got = oracle.canonical(got)
    assert np.array_equal(np.asarray(got.colptr, np.int64), ref.colptr), label
    assert np.array_equal(np.asarray(got.rowidx, np.int64), ref.rowidx), label
    assert np.array_equal(np.asarray(got.vals).astype(np.float64), np.asarray(ref.vals, np.float64)), label


@pytest.mark.parametrize("vt", [np.float64, np.float32])
def test_hybrid_plus_times_floats(vt):
    A = low_cf(value_dtype=vt)
    Ad = to_dev(A)
    C = spg.spgemm(Ad, Ad, tuning=HYB)
    torch.cuda.synchronize()
    ref, ab, nt = oracle.spgemm(A, A, with_absterm=True, with_nterm=True)
    assert_matches(host_csc(C), ref, ab, nt, label=f"hybrid {vt.__name__}")


@pytest.mark.parametrize("semiring,vt", [("plus_times", np.int64), ("min_plus", np.float64),
                                         ("min_plus", np.float32), ("or_and", np.float32),
                                         ("or_and", np.int64)])
def test_hybrid_exact_semirings(semiring, vt):
    """Integer-valued inputs: every semiring's result is exact."""
    A = low_cf(value_dtype=vt, ints=True)
    Ad = to_dev(A)
    C = spg.spgemm(Ad, Ad, tuning=HYB, semiring=semiring)
    torch.cuda.synchronize()
    check_exact(C, oracle.spgemm(A, A, semiring=semiring), False, f"hybrid {semiring} {vt.__name__}")


def test_hybrid_output_is_row_sorted_and_mixed_columns():
    """The sorted path writes rows in order (no sort pass asked for), and a
    skewed product mixes sorted (low cf) and hashed (high cf) columns."""
    A = low_cf(n=6000, d=40, seed=9, value_dtype=np.int64, ints=True)
    C = spg.spgemm(to_dev(A), to_dev(A), tuning=HYB)
    torch.cuda.synchronize()
    got = host_csc(C)
    cp = np.asarray(got.colptr, np.int64)
    r = np.asarray(got.rowidx, np.int64)
    # every column of this product takes the sorted path: ascending rows
    assert all(np.all(np.diff(r[cp[j]:cp[j + 1]]) > 0) for j in range(0, A.ncols, 97))
    check_exact(C, oracle.spgemm(A, A), True, "hybrid sorted rows")
    # skewed: hub columns with cf well above 2 stay on the hash
    rng = np.random.default_rng(4)
    m = 5000
    rows = np.concatenate([rng.choice(m, 30, replace=False) for _ in range(m)] +
                          [rng.choice(m, 2500, replace=False) for _ in range(3)])
    cols = np.concatenate([np.repeat(np.arange(m), 30), np.repeat(rng.integers(0, m, 3), 2500)])
    S = W.csc.from_coo(m, m, rows, cols, rng.integers(-5, 6, rows.size).astype(np.int64), dup="sum")
    Cs = spg.spgemm(to_dev(S), to_dev(S), tuning=HYB)
    torch.cuda.synchronize()
    check_exact(Cs, oracle.spgemm(S, S), False, "hybrid skewed")


@pytest.mark.parametrize("merge", ["end", "incremental"])
def test_hybrid_ksplit_merge(merge):
    """The merge passes read the stage partials through the same CTA tiers."""
    A = low_cf(n=6000, d=40, seed=11, value_dtype=np.int64, ints=True)
    C = spg.spgemm(to_dev(A), to_dev(A), tuning=HYB, kstages=3, merge=merge)
    torch.cuda.synchronize()
    check_exact(C, oracle.spgemm(A, A), False, f"hybrid k-split {merge}")


def test_hybrid_with_sort_output():
    A = low_cf(n=6000, d=40, seed=13, value_dtype=np.float64)
    C = spg.spgemm(to_dev(A), to_dev(A), tuning=HYB, sort_output=True)
    torch.cuda.synchronize()
    ref, ab, nt = oracle.spgemm(A, A, with_absterm=True, with_nterm=True)
    got = host_csc(C)
    assert np.array_equal(np.asarray(got.rowidx, np.int64), ref.rowidx)
    assert_matches(got, ref, ab, nt, label="hybrid sorted output")
