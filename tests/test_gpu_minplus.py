"""The min-plus semiring (C(i,j) = min_k A(i,k) + B(k,j); the paper's
algorithms hold over any semiring, Sec. II) against the oracle.

Integer-valued floats keep every sum exact, so those cases compare bit for
bit; random reals compare within the rounding of one addition (the minimum of
rounded sums is within u * max(|a| + |b|) of the exact minimum).
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
          ints=True):
    """Random columns plus hub rows and columns; integer or N(0,1) weights."""
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
    v = rng.integers(-500, 1000, r.size).astype(np.float64) if ints else rng.standard_normal(r.size)
    a = from_coo(m, n, r, c, v, dup="max", index_dtype=index_dtype, value_dtype=value_dtype)
    return shuffle_within_columns(a, seed + 1)


def compare(C, ref, *, exact, scale=None, sorted_rows=False, label=""):
    got = host_csc(C)
    if not sorted_rows:
        got = oracle.canonical(got)
    assert np.array_equal(np.asarray(got.colptr, np.int64), ref.colptr), label
    assert np.array_equal(np.asarray(got.rowidx, np.int64), ref.rowidx), label
    gv = np.asarray(got.vals).astype(np.float64)
    if exact:
        assert np.array_equal(gv, ref.vals), label
    else:
        u = 2.0 ** -24 if np.asarray(got.vals).dtype == np.float32 else 2.0 ** -53
        assert np.all(np.abs(gv - ref.vals) <= 2 * u * scale + 1e-300), label


@pytest.mark.parametrize("vt", [np.float64, np.float32])
@pytest.mark.parametrize("case", ["light", "heavy", "ksplit", "incremental", "sorted"])
def test_minplus_exact_on_integer_weights(vt, case):
    kw = {}
    A = graph(4000, 4000, 5, hubs=3, hub_deg=1600, base=6, value_dtype=vt)
    if case in ("heavy", "ksplit", "incremental", "sorted"):
        kw["tuning"] = spg.Tuning(hash_max_cap=256, panel_rows=1024)
    if case in ("ksplit", "incremental"):
        kw["kstages"] = 3 if case == "ksplit" else 4
        kw["merge"] = "end" if case == "ksplit" else "incremental"
    if case == "sorted":
        kw["sort_output"] = True
    Ad = to_dev(A)
    C = spg.spgemm(Ad, Ad, semiring="min_plus", **kw)
    torch.cuda.synchronize()
    if case != "light":
        assert C.plan_info["heavy_columns"] > 0
    ref = oracle.spgemm(A, A, semiring="min_plus")
    compare(C, ref, exact=True, sorted_rows=(case == "sorted"), label=f"min-plus {case} {vt.__name__}")


@pytest.mark.parametrize("vt", [np.float64, np.float32])
def test_minplus_real_weights_within_rounding(vt):
    A = graph(3000, 2500, 7, hubs=2, hub_deg=1000, base=5, value_dtype=vt, ints=False)
    B = graph(2500, 2800, 8, hubs=2, hub_deg=900, base=5, value_dtype=vt, ints=False)
    Ad, Bd = to_dev(A), to_dev(B)
    C = spg.spgemm(Ad, Bd, semiring="min_plus", tuning=spg.Tuning(hash_max_cap=512, panel_rows=1024))
    torch.cuda.synchronize()
    ref, scale = oracle.spgemm(A, B, semiring="min_plus", with_absterm=True)
    compare(C, ref, exact=False, scale=scale, label=f"min-plus reals {vt.__name__}")


def test_minplus_run_batched_streams_the_product():
    A = graph(3000, 3000, 9, hubs=2, hub_deg=1200, base=5)
    Ad = to_dev(A)
    ref = oracle.spgemm(A, A, semiring="min_plus")
    budget = A.bytes() * 3 + (1 << 20) + ref.nnz * 12 // 2
    plan = spg.Plan(Ad, Ad, budget=budget, semiring="min_plus", host_slot_bytes=1 << 15, host_slots=2)
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


def test_minplus_refusals():
    A = graph(500, 500, 3, hubs=1, hub_deg=100)
    Ad = to_dev(A)
    plan = spg.Plan(Ad, Ad, semiring="min_plus")
    plan.symbolic()
    Cd = spg.spgemm(Ad, Ad, semiring="min_plus")
    with pytest.raises(spg.SpgemmError, match="plus-times"):
        plan.backward(Cd)
    plan.close()
    Ai = CSC(A.nrows, A.ncols, A.colptr, A.rowidx, A.vals.astype(np.int64))
    with pytest.raises(spg.SpgemmError, match="floating-point"):
        spg.Plan(to_dev(Ai), to_dev(Ai), semiring="min_plus")


def test_minplus_dense_items_after_hash_items_on_one_cta():
    """Many heavy columns, half with dense low panels and sparse high ones and
    half mirrored, so that in the panel-major item order the CTAs of the heavy
    kernel run dense items after hash-range items in the same shared memory
    (which must come back as the min-plus identity)."""
    rng = np.random.default_rng(12)
    m, n = 16384, 4096
    r = (m * rng.random(n * 60) ** 3).astype(np.int64)
    c = np.repeat(np.arange(n), 60)
    r = np.where(c % 2 == 1, m - 1 - r, r)
    A = from_coo(m, n, r, c, rng.integers(0, 1000, r.size).astype(np.float64), dup="max", index_dtype=np.int32,
                 value_dtype=np.float32)
    rb = rng.integers(0, n, n * 12)
    cb = np.repeat(np.arange(n), 12)
    B = from_coo(n, n, rb, cb, rng.integers(0, 1000, rb.size).astype(np.float64), dup="max", index_dtype=np.int32,
                 value_dtype=np.float32)
    Ad, Bd = to_dev(A), to_dev(B)
    C = spg.spgemm(Ad, Bd, semiring="min_plus", tuning=spg.Tuning(hash_max_cap=256, panel_rows=1024))
    torch.cuda.synchronize()
    assert C.plan_info["heavy_columns"] > 1000
    ref = oracle.spgemm(A, B, semiring="min_plus")
    compare(C, ref, exact=True, label="min-plus dense after hash")


@pytest.mark.parametrize("thr,k", [(float("-inf"), 5), (300.0, 0), (100.0, 40)])
def test_minplus_sorted_prune_stream(thr, k):
    """The batch loop's prune over min-plus values (the prune rule is the
    same: values >= threshold, then the k largest, ties to the smaller row
    once sorted). Integer weights keep every sum exact, so the streamed
    selection equals the oracle's prune of the sorted product."""
    A = graph(3000, 3000, 21, hubs=2, hub_deg=1200, base=6)
    Ad = to_dev(A)
    full = oracle.spgemm(A, A, semiring="min_plus")
    ref = oracle.prune(full, thr, k)
    budget = A.bytes() * 3 + (2 << 20) + full.nnz * 12
    plan = spg.Plan(Ad, Ad, budget=budget, semiring="min_plus", sort_output=True, prune=(thr, k),
                    tuning=spg.Tuning(hash_max_cap=256, panel_rows=1024), host_slot_bytes=1 << 15,
                    host_slots=2)
    assert plan.symbolic()["heavy_columns"] > 0
    pieces = []
    spg.run_batched(plan, lambda b, c0, c1, arrs: pieces.append((c0, c1) + tuple(x.copy() for x in arrs)) or 0)
    plan.close()
    colptr = [0]
    for c0, c1, cp, ri, va in pieces:
        colptr.extend((cp[1:] + colptr[-1]).tolist())
    assert np.array_equal(np.array(colptr, np.int64), ref.colptr)
    assert np.array_equal(np.concatenate([p[3] for p in pieces]).astype(np.int64), ref.rowidx)
    assert np.array_equal(np.concatenate([p[4] for p in pieces]).astype(np.float64), ref.vals)
    assert ref.nnz < full.nnz
