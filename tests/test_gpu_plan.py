"""The batch plan of the library against the oracle's (Algorithm 3's b and
Algorithm 4's column ranges, Eq. (2); Sec. V-C takes the smallest b whose
batches fit).

The library cuts the output columns into contiguous ranges whose bytes fit
its per-batch cap. These tests read every range and the cap through the C
ABI, rebuild each column's (or range's) bytes from the oracle's own counts
with the byte model the header documents for spgemm_symbolic, and require the
ranges to equal the oracle's greedy cut bit for bit:

  s = 1             w_j = r nnz(C(:,j)) + 8
  s > 1, at end     w_j = r (nnz(C(:,j)) + sum_t nnz(D_t(:,j))) + 8
  s > 1, incremental
                    cost(c0, c1) = sum_j (r nnz(C(:,j)) + 8)
                                   + r (max_{t>=1} sum_j nnz(D_t(:,j))
                                        + m max_{u<=s-2} sum_j nnz(M_u(:,j)))
                    (M_u = the product over stages 0..u, M_0 = D_0; m = 2
                    running sums, 1 when s = 2)
  prune             w_j += r min(nnz(C(:,j)), topk) + 8 + 40

with r = index bytes + value bytes.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle

from helpers import to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_08526_gb300 as spg  # noqa: E402
from test_gpu_parity import skewed  # noqa: E402

PTR_BYTES = 8
PRUNE_WS_PER_COL = 40


def _ranges(plan):
    info = plan.query()
    starts = [plan.batch(t)[0] for t in range(info["nbatches"])]
    return np.array(starts + [plan.batch(info["nbatches"] - 1)[1]], np.int64), info


def _plan_with_batches(Ad, Bd, total_bytes, want, **kw):
    """A plan whose cap is about total_bytes / want: the workspace is learnt
    from a plan with a large budget (it does not depend on the budget)."""
    big = 1 << 34
    ring = kw.get("ring_depth", 0) or 2
    probe = spg.Plan(Ad, Bd, budget=big, **kw)
    cap0 = probe.symbolic()["batch_cap_bytes"]
    probe.close()
    target = max(1, total_bytes // want)
    plan = spg.Plan(Ad, Bd, budget=big - ring * (cap0 - target), **kw)
    plan.symbolic()
    return plan


def _stage_counts(A, B, s):
    k = A.ncols
    return [oracle.symbolic(A, B, krange=kr) for kr in oracle.stage_ranges(k, s)]


@pytest.mark.parametrize("case", ["s1", "s3_end", "s3_incremental", "s4_incremental",
                                  "s2_incremental", "prune", "s3_end_prune_i64"])
def test_batch_ranges_equal_oracle_plan(case):
    idx = np.int64 if case.endswith("i64") else np.int32
    A = skewed(3000, 2600, 301, hubs=3, hub_deg=900, base=5, index_dtype=idx)
    B = skewed(2600, 3200, 302, hubs=2, hub_deg=800, base=5, index_dtype=idx)
    s = 1
    merge = "end"
    prune = None
    if case.startswith("s3") or case.startswith("s4") or case.startswith("s2"):
        s = int(case[1])
    if "incremental" in case:
        merge = "incremental"
    if "prune" in case:
        prune = (0.25, 7)
    r = (8 if idx == np.int64 else 4) + 8
    nnzc = oracle.symbolic(A, B)
    n = B.ncols
    stage = _stage_counts(A, B, s) if s > 1 else []
    w = r * nnzc + PTR_BYTES
    if s > 1 and merge == "end":
        w = w + r * np.sum(stage, axis=0)
    if prune is not None:
        k = prune[1]
        w = w + r * np.minimum(nnzc, k) + PTR_BYTES + PRUNE_WS_PER_COL
    if merge == "incremental":
        pre_w = np.concatenate([[0], np.cumsum(w)])
        pre_d = [np.concatenate([[0], np.cumsum(d)]) for d in stage]
        # running sums M_u over stages 0..u (u = 1..s-2); M_0 = D_0
        kr = oracle.stage_ranges(A.ncols, s)
        pre_m = [pre_d[0]] + [np.concatenate([[0], np.cumsum(oracle.symbolic(A, B, krange=(0, kr[u][1])))])
                              for u in range(1, s - 1)]
        m = 2 if s > 2 else 1

        def cost(c0, c1):
            dmax = max(int(p[c1] - p[c0]) for p in pre_d[1:])
            mmax = max(int(p[c1] - p[c0]) for p in pre_m)
            return int(pre_w[c1] - pre_w[c0]) + r * (dmax + m * mmax)
        total = cost(0, n)
    else:
        cost = None
        total = int(w.sum())
    Ad, Bd = to_dev(A), to_dev(B)
    plan = _plan_with_batches(Ad, Bd, total, 5, kstages=s, merge=merge, prune=prune)
    got, info = _ranges(plan)
    cap = info["batch_cap_bytes"]
    plan.close()
    assert info["nbatches"] >= 3, (case, info)
    if cost is None:
        ref = oracle.plan_batches(w, cap)
    else:
        ref = oracle.plan_ranges(cost, n, cap)
    assert ref is not None
    assert np.array_equal(got, ref), (case, got, ref)
    # the batch nnz the library reports are the oracle's counts over each range
    pre = np.concatenate([[0], np.cumsum(nnzc)])
    plan = _plan_with_batches(Ad, Bd, total, 5, kstages=s, merge=merge, prune=prune)
    for t in range(plan.nbatches):
        c0, c1, nnz = plan.batch(t)
        assert nnz == int(pre[c1] - pre[c0])
    plan.close()


def test_single_column_over_the_cap_is_refused():
    """A column whose own bytes exceed the cap: the oracle's plan is None and
    the library returns SPGEMM_ERR_BUDGET."""
    A = skewed(3000, 3000, 303, hubs=1, hub_deg=2500, base=2)
    nnzc = oracle.symbolic(A, A)
    w = 12 * nnzc + PTR_BYTES
    Ad = to_dev(A)
    big = 1 << 34
    probe = spg.Plan(Ad, Ad, budget=big)
    cap0 = probe.symbolic()["batch_cap_bytes"]
    probe.close()
    cap = int(w.max()) - 1
    assert oracle.plan_batches(w, cap) is None
    plan = spg.Plan(Ad, Ad, budget=big - 2 * (cap0 - cap))
    with pytest.raises(spg.SpgemmError):
        plan.symbolic()
    plan.close()
