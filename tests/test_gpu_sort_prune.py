"""Sorted final output and the column-wise prune (the batch consumer: keep the
largest entries of every column), against the oracle.

* sort_output: every column of the library's C is in ascending row order and
  equals the oracle's (sorted) product entry for entry, with no canonical
  re-sort on our side; light columns, hash-range items and dense items of
  heavy columns, the k-split merge and all value types.
* spgemm_prune: bit-exact against oracle.prune applied to the same values
  (the library's own product, copied to the host), thresholds, top-k, both,
  ties (int64 path counts), empty columns, int32 colptr input.
* run_batched with opts.prune: the pruned pieces streamed to the host
  concatenate to oracle.prune of the whole sorted product.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from workloads.csc import CSC, from_coo, shuffle_within_columns

from helpers import host_csc, record_rel, tol_of, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_08526_gb300 as spg  # noqa: E402


def skewed(m, n, seed, hubs=3, hub_deg=None, base=4, index_dtype=np.int32, value_dtype=np.float64,
           dist="normal"):
    """Random columns plus a few hub rows and columns (all tiers appear)."""
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
    if dist == "normal":
        v = rng.standard_normal(r.size)
        vt = value_dtype
    else:
        v = np.ones(r.size, dtype=np.int64)
        vt = np.int64
    a = from_coo(m, n, r, c, v, dup="max", index_dtype=index_dtype, value_dtype=vt)
    return shuffle_within_columns(a, seed + 1)


def assert_sorted_equal(got: CSC, ref: CSC, ab=None, nt=None, label=""):
    """Rows ascending in every column and equal to the oracle's, as stored."""
    cp = np.asarray(got.colptr, np.int64)
    ri = np.asarray(got.rowidx, np.int64)
    assert np.array_equal(cp, np.asarray(ref.colptr, np.int64)), f"{label}: column counts"
    cols = np.repeat(np.arange(got.ncols), np.diff(cp))
    inc = np.diff(ri) > 0
    same_col = np.diff(cols) == 0
    assert np.all(inc[same_col]), f"{label}: a column is not in ascending row order"
    assert np.array_equal(ri, np.asarray(ref.rowidx, np.int64)), f"{label}: rows differ"
    gv, rv = np.asarray(got.vals), np.asarray(ref.vals)
    if np.issubdtype(gv.dtype, np.integer):
        assert np.array_equal(gv.astype(np.int64), rv.astype(np.int64)), f"{label}: values"
    else:
        tol = tol_of(gv.dtype, nt)
        err = np.abs(gv.astype(np.float64) - rv)
        assert np.all(err <= tol * ab + 1e-300), f"{label}: max err {err.max()}"
        nz = np.abs(rv) > 0
        if nz.any():
            record_rel(label, float((err[nz] / np.abs(rv[nz])).max()))


@pytest.mark.parametrize("case", ["light", "heavy", "heavy_f32", "ksplit", "int64"])
def test_sort_output_matches_oracle_order(case):
    kw = {}
    if case == "light":
        A = skewed(2500, 2500, 3, hubs=2, hub_deg=600, base=5)
    elif case in ("heavy", "ksplit"):
        A = skewed(6000, 6000, 11, hubs=4, hub_deg=2500, base=6)
        kw["tuning"] = spg.Tuning(hash_max_cap=256, panel_rows=1024)
        if case == "ksplit":
            kw["kstages"] = 4
    elif case == "heavy_f32":
        A = skewed(5000, 5000, 21, hubs=3, hub_deg=2000, base=5, value_dtype=np.float32)
        kw["tuning"] = spg.Tuning(hash_max_cap=512, panel_rows=2048)
    else:
        A = skewed(5000, 5000, 22, hubs=3, hub_deg=2000, base=5, dist="ones", index_dtype=np.int64)
        kw["tuning"] = spg.Tuning(hash_max_cap=512, panel_rows=2048)
    Ad = to_dev(A)
    C = spg.spgemm(Ad, Ad, sort_output=True, **kw)
    torch.cuda.synchronize()
    if case in ("heavy", "ksplit"):
        assert C.plan_info["heavy_columns"] > 0
    ref, ab, nt = oracle.spgemm(A, A, with_absterm=True, with_nterm=True)
    assert_sorted_equal(host_csc(C), ref, ab, nt, label=f"sorted {case}")


def _gpu_product(A, **kw):
    Ad = to_dev(A)
    C = spg.spgemm(Ad, Ad, sort_output=True, **kw)
    torch.cuda.synchronize()
    return C


def _same(got: CSC, ref: CSC, label):
    assert np.array_equal(np.asarray(got.colptr, np.int64), np.asarray(ref.colptr, np.int64)), label
    assert np.array_equal(np.asarray(got.rowidx, np.int64), np.asarray(ref.rowidx, np.int64)), label
    gv, rv = np.asarray(got.vals), np.asarray(ref.vals)
    if np.issubdtype(gv.dtype, np.integer):
        assert np.array_equal(gv.astype(np.int64), rv.astype(np.int64)), label
    else:
        assert np.array_equal(gv.astype(np.float64), rv.astype(np.float64)), label


@pytest.mark.parametrize("vt", [np.float64, np.float32, np.int64])
@pytest.mark.parametrize("thr,k", [(float("-inf"), 5), (0.5, 0), (0.25, 3), (float("-inf"), 1),
                                   (float("-inf"), 10**9), (1e30, 4)])
def test_prune_matches_oracle_bit_exact(vt, thr, k):
    dist = "ones" if vt == np.int64 else "normal"
    A = skewed(3000, 3000, 5, hubs=3, hub_deg=800, base=5, value_dtype=vt, dist=dist)
    if dist == "ones" and np.isfinite(thr) and thr < 1e20:
        thr = 2.0 if thr > 0.3 else 1.5          # path counts are integers >= 1
    C = _gpu_product(A, tuning=spg.Tuning(hash_max_cap=256, panel_rows=1024))
    P = spg.prune(C, thr, k)
    torch.cuda.synchronize()
    ref = oracle.prune(host_csc(C), thr, k)
    _same(host_csc(P), ref, f"prune {vt.__name__} thr={thr} k={k}")


def test_prune_unsorted_input_and_int32_colptr():
    """Ties go to the earlier stored entry, whatever the row order; a 32-bit
    colptr input; empty columns."""
    A = skewed(2000, 2000, 9, hubs=2, hub_deg=500, base=3, dist="ones")
    Ad = to_dev(A)
    C = spg.spgemm(Ad, Ad, ptr_dtype=torch.int32)    # unsorted
    torch.cuda.synchronize()
    assert C.colptr.dtype == torch.int32
    host = host_csc(C)
    assert np.any(np.diff(host.colptr) == 0)         # some empty columns
    for thr, k in ((float("-inf"), 2), (2.0, 0), (1.5, 3)):
        P = spg.prune(C, thr, k)
        torch.cuda.synchronize()
        _same(host_csc(P), oracle.prune(host, thr, k), f"unsorted thr={thr} k={k}")


def test_prune_rejects_bad_arguments():
    A = skewed(300, 300, 2, hubs=1, hub_deg=50)
    C = _gpu_product(A)
    with pytest.raises(spg.SpgemmError):
        spg.prune(C, float("nan"), 3)


@pytest.mark.parametrize("kst,k", [(1, 7), (3, 7), (1, 40), (3, 2000), (1, 0), (3, 0)])
def test_run_batched_prunes_before_the_copy(kst, k):
    """int64 path counts: the product is exact, so the streamed selection must
    equal the oracle's bit for bit (and ties are everywhere). With sorted
    output and 0 < k <= 8192 the loop prunes the unsorted batch (ties go to
    the smaller rows) and then sorts the kept entries: k = 7, 40 and 2000
    reach the warp sort and both block sorts of that step; k = 0 keeps the
    threshold only, after the full sort."""
    A = skewed(4000, 4000, 17, hubs=3, hub_deg=1500, base=6, dist="ones")
    Ad = to_dev(A)
    tun = spg.Tuning(hash_max_cap=256, panel_rows=1024)
    full = spg.spgemm(Ad, Ad, sort_output=True, tuning=tun, kstages=kst)
    torch.cuda.synchronize()
    thr = 2.0
    ref = oracle.prune(host_csc(full), thr, k)
    budget = A.bytes() * 3 + (1 << 20) + full.nnz * 12 // 2
    plan = spg.Plan(Ad, Ad, budget=budget, kstages=kst, tuning=tun, sort_output=True, prune=(thr, k),
                    host_slot_bytes=1 << 14, host_slots=2)
    info = plan.symbolic()
    assert info["nbatches"] >= 2
    pieces = []

    def sink(batch, c0, c1, arrs):
        cp, ri, va = arrs
        pieces.append((c0, c1, cp.copy(), ri.copy(), va.copy()))
        return 0

    spg.run_batched(plan, sink)
    plan.close()
    colptr = [0]
    for c0, c1, cp, ri, va in pieces:
        colptr.extend((cp[1:] + colptr[-1]).tolist())
    got = CSC(A.nrows, A.ncols, np.array(colptr, np.int64),
              np.concatenate([p[3] for p in pieces]).astype(np.int64),
              np.concatenate([p[4] for p in pieces]))
    assert pieces[0][0] == 0 and pieces[-1][1] == A.ncols
    _same(got, ref, f"run_batched prune s={kst} k={k}")
    assert ref.nnz < full.nnz                        # the prune did remove entries


# ------------------------------------------------------- transpose, A A^T, row batches
from workloads.csc import transpose as host_transpose  # noqa: E402
from helpers import assert_matches  # noqa: E402


@pytest.mark.parametrize("it,vt,ptr", [(np.int32, np.float32, torch.int32), (np.int32, np.float64, torch.int64),
                                       (np.int64, np.int64, torch.int64), (np.int64, np.float32, torch.int32)])
def test_transpose_moves_every_entry(it, vt, ptr):
    dist = "ones" if vt == np.int64 else "normal"
    A = skewed(1700, 2300, 31, hubs=2, hub_deg=700, base=4, index_dtype=it, value_dtype=vt, dist=dist)
    Ad = to_dev(A)
    T = spg.transpose(Ad, ptr_dtype=ptr)
    torch.cuda.synchronize()
    assert (T.nrows, T.ncols, T.nnz) == (A.ncols, A.nrows, A.nnz)
    got = oracle.canonical(host_csc(T))
    ref = oracle.canonical(host_transpose(A))
    assert np.array_equal(got.colptr, ref.colptr)
    assert np.array_equal(got.rowidx, ref.rowidx)
    assert np.array_equal(np.asarray(got.vals), np.asarray(ref.vals).astype(np.asarray(got.vals).dtype))
    # dense check on a corner
    d = np.zeros((A.nrows, A.ncols))
    cols = np.repeat(np.arange(A.ncols), np.diff(A.colptr))
    d[A.rowidx.astype(np.int64), cols] = A.vals
    dt = np.zeros((A.ncols, A.nrows))
    tcols = np.repeat(np.arange(got.ncols), np.diff(got.colptr))
    dt[got.rowidx, tcols] = got.vals
    assert np.array_equal(dt, d.T)


def test_transpose_rejects_rows_out_of_range():
    A = CSC(10, 3, np.array([0, 2, 3, 4], np.int32), np.array([1, 12, 4, 9], np.int32), np.ones(4))
    Ad = to_dev(A)
    with pytest.raises(spg.SpgemmError, match="outside"):
        spg.transpose(Ad)


def test_aat_matches_oracle():
    """A A^T (Sec. V's overlap product) on a k-mer-like matrix: few nonzeros
    per column, skewed rows."""
    rng = np.random.default_rng(44)
    m, n = 6000, 20000
    r = np.minimum((rng.pareto(1.3, 2 * n) * 50).astype(np.int64), m - 1)
    c = np.repeat(np.arange(n), 2)
    A = from_coo(m, n, r, c, rng.random(2 * n), dup="sum", index_dtype=np.int32)
    Ad = to_dev(A)
    C = spg.spgemm_aat(Ad)
    torch.cuda.synchronize()
    At = host_transpose(A)
    ref, ab, nt = oracle.spgemm(A, At, with_absterm=True, with_nterm=True)
    assert_matches(host_csc(C), ref, ab, nt, label="A A^T")


def test_row_batched_blocks_reassemble_to_the_product():
    A = skewed(3000, 2500, 41, hubs=2, hub_deg=900, base=5)
    B = skewed(2500, 2800, 42, hubs=2, hub_deg=700, base=5)
    Ad, Bd = to_dev(A), to_dev(B)
    ref, ab, nt = oracle.spgemm(A, B, with_absterm=True, with_nterm=True)
    blocks = []

    def sink(batch, r0, r1, arrs):
        rp, ci, va = arrs
        blocks.append((r0, r1, rp.copy(), ci.copy(), va.copy()))
        return 0

    budget = (A.bytes() + B.bytes()) * 4 + (1 << 20) + ref.nnz * 12 // 2
    spg.run_row_batched(Ad, Bd, sink, budget=budget, host_slot_bytes=1 << 15, host_slots=2)
    assert blocks[0][0] == 0 and blocks[-1][1] == A.nrows and len(blocks) >= 2
    rowptr = [0]
    for r0, r1, rp, ci, va in blocks:
        rowptr.extend((rp[1:] + rowptr[-1]).tolist())
    # the rows of C in CSR = the CSC of C^T; transpose back on the host
    CT = CSC(B.ncols, A.nrows, np.array(rowptr, np.int64), np.concatenate([b[3] for b in blocks]).astype(np.int64),
             np.concatenate([b[4] for b in blocks]))
    assert_matches(host_transpose(CT), ref, ab, nt, label="row batches")
