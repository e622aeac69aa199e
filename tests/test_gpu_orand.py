"""The Boolean or-and semiring (C(i,j) = OR_k A(i,k) AND B(k,j), a value true
when nonzero; the paper's algorithms hold over any semiring, Sec. II) against
the oracle. Every result is 0 or 1, so the comparison is exact. The inputs
carry explicit false entries (0 and -0.0) and NaN (true), so that C holds
both truth values on its structure.
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


def graph(m, n, seed, hubs=3, hub_deg=None, base=4, index_dtype=np.int32, value_dtype=np.float64,
          false_frac=0.4):
    """Random columns plus hub rows and columns; about false_frac of the
    stored values false (0, and -0.0 for floats), one NaN."""
    rng = np.random.default_rng(seed)
    hub_deg = hub_deg or max(1, m // 3)
    rows, cols = [], []
    counts = rng.integers(0, base * 2 + 1, n)
    for j in range(n):
        rows.append(rng.choice(m, size=min(m, int(counts[j])), replace=False))
        cols.append(np.full(rows[-1].size, j))
    for _ in range(hubs):
        j = int(rng.integers(0, n))
        r = rng.choice(m, size=min(m, hub_deg), replace=False)
        rows.append(r); cols.append(np.full(r.size, j))
        i = int(rng.integers(0, m))
        c = rng.choice(n, size=min(n, hub_deg), replace=False)
        rows.append(np.full(c.size, i)); cols.append(c)
    r = np.concatenate(rows); c = np.concatenate(cols)
    a = from_coo(m, n, r, c, np.ones(r.size), dup="max", index_dtype=index_dtype, value_dtype=np.float64)
    v = rng.integers(1, 5, a.nnz).astype(np.float64)
    z = rng.random(a.nnz) < false_frac
    v[z] = 0.0
    if np.issubdtype(np.dtype(value_dtype), np.floating):
        v[z & (rng.random(a.nnz) < 0.5)] = -0.0
        v[np.flatnonzero(~z)[:1]] = np.nan
    a = CSC(a.nrows, a.ncols, a.colptr, a.rowidx, v.astype(value_dtype))
    return shuffle_within_columns(a, seed + 1)


def compare(C, ref, *, sorted_rows=False, label=""):
    got = host_csc(C)
    if not sorted_rows:
        got = oracle.canonical(got)
    assert np.array_equal(np.asarray(got.colptr, np.int64), ref.colptr), label
    assert np.array_equal(np.asarray(got.rowidx, np.int64), ref.rowidx), label
    gv = np.asarray(got.vals)
    assert np.array_equal(gv.astype(np.float64), np.asarray(ref.vals, np.float64)), label
    assert np.all((gv == 0) | (gv == 1)), label


@pytest.mark.parametrize("vt", [np.float64, np.float32, np.int64])
@pytest.mark.parametrize("case", ["light", "heavy", "ksplit", "incremental", "sorted"])
def test_orand_exact(vt, case):
    kw = {}
    A = graph(4000, 4000, 5, hubs=3, hub_deg=1600, base=6, value_dtype=vt)
    if case != "light":
        kw["tuning"] = spg.Tuning(hash_max_cap=256, panel_rows=1024)
    if case in ("ksplit", "incremental"):
        kw["kstages"] = 3
        kw["merge"] = "end" if case == "ksplit" else "incremental"
    if case == "sorted":
        kw["sort_output"] = True
    Ad = to_dev(A)
    C = spg.spgemm(Ad, Ad, semiring="or_and", **kw)
    torch.cuda.synchronize()
    if case != "light":
        assert C.plan_info["heavy_columns"] > 0
    ref = oracle.spgemm(A, A, semiring="or_and")
    assert 0 < int((ref.vals == 0).sum()) < ref.nnz      # both truth values occur
    compare(C, ref, sorted_rows=(case == "sorted"), label=f"or-and {case} {vt.__name__}")


def test_orand_int64_indices_rectangular():
    A = graph(3000, 2500, 7, hubs=2, hub_deg=1000, base=5, index_dtype=np.int64)
    B = graph(2500, 2800, 8, hubs=2, hub_deg=900, base=5, index_dtype=np.int64)
    C = spg.spgemm(to_dev(A), to_dev(B), semiring="or_and", tuning=spg.Tuning(hash_max_cap=512, panel_rows=1024))
    torch.cuda.synchronize()
    compare(C, oracle.spgemm(A, B, semiring="or_and"), label="or-and int64 indices")


def test_orand_run_batched_streams_the_product():
    A = graph(3000, 3000, 9, hubs=2, hub_deg=1200, base=5, value_dtype=np.float32)
    Ad = to_dev(A)
    ref = oracle.spgemm(A, A, semiring="or_and")
    budget = A.bytes() * 3 + (1 << 20) + ref.nnz * 8 // 2
    plan = spg.Plan(Ad, Ad, budget=budget, semiring="or_and", host_slot_bytes=1 << 15, host_slots=2)
    info = plan.symbolic()
    assert info["nbatches"] >= 2
    pieces = []
    spg.run_batched(plan, lambda b, c0, c1, arrs: pieces.append((c0, c1) + tuple(x.copy() for x in arrs)) or 0)
    plan.close()
    colptr = [0]
    for c0, c1, cp, ri, va in pieces:
        colptr.extend((cp[1:] + colptr[-1]).tolist())
    got = CSC(A.nrows, A.ncols, np.array(colptr, np.int64), np.concatenate([p[3] for p in pieces]).astype(np.int64),
              np.concatenate([p[4] for p in pieces]))
    g = oracle.canonical(got)
    assert np.array_equal(g.colptr, ref.colptr) and np.array_equal(g.rowidx, ref.rowidx)
    assert np.array_equal(np.asarray(g.vals, np.float64), ref.vals)


@pytest.mark.parametrize("k", [3, 50])
def test_orand_sorted_topk_stream(k):
    """Sorted output with a top-k prune in the batch loop: among equal values
    (every kept value is 1) the smaller rows win, as after sorting; k = 3 and
    50 reach the warp and block sorts after the prune. Equal to the oracle's
    prune of the whole sorted or-and product."""
    A = graph(3000, 3000, 13, hubs=2, hub_deg=1200, base=6, value_dtype=np.float32)
    Ad = to_dev(A)
    full = oracle.spgemm(A, A, semiring="or_and")
    ref = oracle.prune(full, 0.5, k)          # true entries only, then the first k rows
    tun = spg.Tuning(hash_max_cap=256, panel_rows=1024)
    budget = A.bytes() * 3 + (2 << 20) + full.nnz * 8
    plan = spg.Plan(Ad, Ad, budget=budget, semiring="or_and", sort_output=True, prune=(0.5, k), tuning=tun,
                    host_slot_bytes=1 << 15, host_slots=2)
    info = plan.symbolic()
    assert info["heavy_columns"] > 0
    pieces = []
    spg.run_batched(plan, lambda b, c0, c1, arrs: pieces.append((c0, c1) + tuple(x.copy() for x in arrs)) or 0)
    plan.close()
    colptr = [0]
    for c0, c1, cp, ri, va in pieces:
        colptr.extend((cp[1:] + colptr[-1]).tolist())
    got_rows = np.concatenate([p[3] for p in pieces]).astype(np.int64)
    got_vals = np.concatenate([p[4] for p in pieces]).astype(np.float64)
    assert np.array_equal(np.array(colptr, np.int64), ref.colptr)
    assert np.array_equal(got_rows, ref.rowidx)                  # sorted, smallest rows kept
    assert np.all(got_vals == 1.0) and np.array_equal(got_vals, ref.vals)


def test_orand_backward_refused():
    A = graph(500, 500, 3, hubs=1, hub_deg=100)
    Ad = to_dev(A)
    plan = spg.Plan(Ad, Ad, semiring="or_and")
    plan.symbolic()
    Cd = spg.spgemm(Ad, Ad, semiring="or_and")
    with pytest.raises(spg.SpgemmError, match="plus-times"):
        plan.backward(Cd)
    plan.close()
