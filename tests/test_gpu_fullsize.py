"""Parity at the full workload sizes, in the launch configuration the
benchmark times, on outputs the oracle can compute one column (or one
problem) at a time.

* R-MAT scale 20 (C = A*A, fp32): sampled columns, including the heaviest.
* Protein-similarity stand-in (2M x 2M, int64 indices, fp32) under a 24 GB
  budget: at least 4 batches, streamed to pinned host memory by the batch
  loop; sampled columns checked inside the sink, per-column counts checked
  for every streamed column against the oracle's symbolic count on samples.
* 512 uneven G(n,p) products (int64 ones): sampled problems bit-exact.
* Differentiation workload (A 200k x 200k, B 200k x 100k, fp32): the whole
  forward product and both gradients against the oracle.
* R-MAT scale 20 through the batch loop with sorted output and a top-1000
  prune per column (sampled columns, by properties), and over the min-plus
  semiring (sampled columns).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as W
from workloads.csc import CSC, column_slice

from helpers import assert_matches, host_csc, to_dev, tol_of

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_08526_gb300 as spg  # noqa: E402


def check_column(A, B, j, rows, vals, label):
    ref, ab, nt = oracle.spgemm(A, column_slice(B, j, j + 1), with_absterm=True, with_nterm=True)
    got = CSC(A.nrows, 1, np.array([0, rows.size], np.int64), rows.astype(np.int64), vals)
    assert_matches(got, ref, ab, nt, label=f"{label} column {j}")


def wide(A: CSC) -> CSC:
    """The oracle's own index and value widths (its wrapper then copies nothing)."""
    return A.astype(index_dtype=np.int64, value_dtype=np.float64)


def test_rmat_scale20_sampled_columns():
    A = W.config2()
    Ad = to_dev(A)
    A = wide(A)
    plan = spg.Plan(Ad, Ad)
    info = plan.symbolic()
    f = oracle.flops_per_column(A, A)
    assert info["flops"] == int(f.sum())
    rng = np.random.default_rng(2)
    cols = sorted(set(rng.choice(A.ncols, 24, replace=False).tolist() + np.argsort(-f)[:3].tolist()))
    cnt = plan.column_counts().cpu().numpy()
    for t in range(plan.nbatches):
        c0, c1, _ = plan.batch(t)
        C = plan.numeric(t)
        torch.cuda.synchronize()
        for j in cols:
            if c0 <= j < c1:
                a, b = C.colptr[j - c0].item(), C.colptr[j - c0 + 1].item()
                rows = C.rowidx[a:b].cpu().numpy()
                vals = C.vals[a:b].cpu().numpy()
                assert b - a == cnt[j]
                check_column(A, A, j, rows, vals, "rmat20")
        del C
        torch.cuda.empty_cache()
    plan.check_errors()
    plan.close()


def test_protein_2M_budget_24GB_streamed():
    A = W.config3()
    Ad = to_dev(A)
    A = wide(A)
    plan = spg.Plan(Ad, Ad, budget=24 * 10**9, host_slot_bytes=1 << 30, host_slots=3)
    info = plan.symbolic()
    assert info["nbatches"] >= 4, info
    rng = np.random.default_rng(3)
    f = oracle.flops_per_column(A, A)
    cols = set(rng.choice(A.ncols, 12, replace=False).tolist() + np.argsort(-f)[:2].tolist())
    sample_cnt = {j: int(oracle.symbolic(A, column_slice(A, j, j + 1))[0]) for j in sorted(cols)}
    seen = {"cols": 0, "checked": 0, "nnz": 0}

    def sink(batch, c0, c1, arrs):
        cp, ri, va = arrs
        assert c0 == seen["cols"]
        seen["cols"] = c1
        seen["nnz"] += int(cp[-1])
        for j in cols:
            if c0 <= j < c1:
                a, b = int(cp[j - c0]), int(cp[j - c0 + 1])
                assert b - a == sample_cnt[j]
                check_column(A, A, j, ri[a:b].copy(), va[a:b].copy(), "protein")
                seen["checked"] += 1
        return 0

    spg.run_batched(plan, sink)
    assert seen["cols"] == A.ncols
    assert seen["nnz"] == info["nnz_c"]
    assert seen["checked"] == len(cols)
    plan.close()


def test_512_problems_sampled_exact():
    probs = W.config4()
    dev = [to_dev(p) for p in probs]
    M = spg.Multi(dev, dev)
    M.run(use_graph=True)
    torch.cuda.synchronize()
    cp, ri, va = M.output()
    cp = cp.cpu().numpy()
    col = 0
    starts = []
    for p in probs:
        starts.append(col)
        col += p.ncols
    rng = np.random.default_rng(4)
    for i in sorted(rng.choice(len(probs), 8, replace=False).tolist() + [0, len(probs) - 1]):
        p = probs[i]
        s = starts[i]
        a, b = int(cp[s]), int(cp[s + p.ncols])
        ref = oracle.spgemm(p, p)
        got = CSC(p.nrows, p.ncols, cp[s:s + p.ncols + 1] - a, ri[a:b].cpu().numpy().astype(np.int64),
                  va[a:b].cpu().numpy())
        assert_matches(got, ref, exact=True, label=f"problem {i}")
    M.close()


def test_differentiation_full_size_forward_and_gradients():
    A, B = W.config5()
    Ad, Bd = to_dev(A), to_dev(B)
    a = Ad.vals.clone().requires_grad_(True)
    b = Bd.vals.clone().requires_grad_(True)
    plan = spg.Plan(Ad, Bd)
    plan.symbolic()
    Cl = plan.numeric(0)
    torch.cuda.synchronize()
    C_host = host_csc(Cl)
    ref, ab, nt = oracle.spgemm(A, B, with_absterm=True, with_nterm=True)
    assert_matches(C_host, ref, ab, nt, label="forward")
    # G drawn on the oracle's pattern, handed to the library in its own layout
    G = W.values_on_pattern(ref, 5, dist="normal", value_dtype=np.float32)
    Gi = G.astype(index_dtype=np.int32)
    dA, dB = plan.backward(to_dev(Gi))
    torch.cuda.synchronize()
    rA, rB = oracle.backward(A, B, G)
    # each gradient entry sums up to 8 (dA) or 16 (dB) products of fp32 values
    absA, absB = oracle.backward(CSC(A.nrows, A.ncols, A.colptr, A.rowidx, np.abs(A.vals)),
                                 CSC(B.nrows, B.ncols, B.colptr, B.rowidx, np.abs(B.vals)),
                                 CSC(G.nrows, G.ncols, G.colptr, G.rowidx, np.abs(G.vals)))
    for got, ref_g, scale in ((dA.cpu().numpy(), rA, absA), (dB.cpu().numpy(), rB, absB)):
        err = np.abs(got.astype(np.float64) - ref_g)
        assert np.all(err <= tol_of(np.float32, 17) * scale + 1e-30)
    plan.close()


def test_rmat_scale20_sorted_topk_stream_sampled_columns():
    """The batch consumer at full size: every batch sorted and pruned to its
    1000 largest entries per column on the device, streamed to the host.
    Sampled columns against the oracle's column (float64): rows ascending, as
    many entries as min(1000, nnz), rows a subset of the column, and the kept
    values the column's largest within fp32 rounding (sum |terms| bound)."""
    k = 1000
    A = W.config2()
    Ad = to_dev(A)
    A = wide(A)
    f = oracle.flops_per_column(A, A)
    rng = np.random.default_rng(6)
    cols = set(rng.choice(A.ncols, 10, replace=False).tolist() + np.argsort(-f)[:3].tolist())
    plan = spg.Plan(Ad, Ad, host_slot_bytes=1 << 30, host_slots=3, sort_output=True, prune=(float("-inf"), k))
    plan.symbolic()
    seen = {"cols": 0, "checked": 0}

    def sink(batch, c0, c1, arrs):
        cp, ri, va = arrs
        assert c0 == seen["cols"]
        seen["cols"] = c1
        for j in cols:
            if c0 <= j < c1:
                a, b = int(cp[j - c0]), int(cp[j - c0 + 1])
                rows = ri[a:b].astype(np.int64)
                vals = va[a:b].astype(np.float64)
                ref, ab, nt = oracle.spgemm(A, column_slice(A, j, j + 1), with_absterm=True,
                                            with_nterm=True)
                rr, rv = ref.rowidx, ref.vals
                err_bound = tol_of(np.float32, nt) * ab
                assert b - a == min(k, rr.size)
                assert np.all(np.diff(rows) > 0)
                pos = np.searchsorted(rr, rows)
                assert np.all(rr[np.minimum(pos, rr.size - 1)] == rows)
                assert np.all(np.abs(vals - rv[pos]) <= err_bound[pos] + 1e-30)
                if rr.size > k:
                    cut = np.sort(rv)[::-1][k - 1]
                    # kept values reach the oracle's k-th largest, up to the
                    # largest rounding bound of any entry of the column
                    assert vals.min() >= cut - err_bound.max() - 1e-30
                seen["checked"] += 1
        return 0

    spg.run_batched(plan, sink)
    assert seen["cols"] == A.ncols and seen["checked"] == len(cols)
    plan.close()


def test_rmat_scale20_min_plus_sampled_columns():
    A = W.config2()
    Ad = to_dev(A)
    A = wide(A)
    plan = spg.Plan(Ad, Ad, semiring="min_plus")
    plan.symbolic()
    f = oracle.flops_per_column(A, A)
    rng = np.random.default_rng(8)
    cols = sorted(set(rng.choice(A.ncols, 12, replace=False).tolist() + np.argsort(-f)[:2].tolist()))
    for t in range(plan.nbatches):
        c0, c1, _ = plan.batch(t)
        C = plan.numeric(t)
        torch.cuda.synchronize()
        for j in cols:
            if c0 <= j < c1:
                a, b = C.colptr[j - c0].item(), C.colptr[j - c0 + 1].item()
                rows = C.rowidx[a:b].cpu().numpy().astype(np.int64)
                vals = C.vals[a:b].cpu().numpy().astype(np.float64)
                ref, scale = oracle.spgemm(A, column_slice(A, j, j + 1), with_absterm=True, semiring="min_plus")
                order = np.argsort(rows)
                assert np.array_equal(rows[order], ref.rowidx)
                assert np.all(np.abs(vals[order] - ref.vals) <= 2 * 2.0 ** -24 * scale + 1e-30)
        del C
        torch.cuda.empty_cache()
    plan.check_errors()
    plan.close()
