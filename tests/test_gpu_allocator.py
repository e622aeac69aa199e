"""Plan workspace through the caller's allocator (spgemm_opts.allocator).

The library takes its workspace, and the pinned host ring of
spgemm_run_batched, from the spgemm_allocator callbacks when a plan is given
them; the Python binding passes PyTorch's allocators by default. These tests
check that the results are the same as with the library's own cudaMalloc,
that the memory is visible to torch while the plan lives and is returned
when it is destroyed, and that an allocation refused in the middle of a call
surfaces as SPGEMM_ERR_OOM with every block that was handed out given back.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle

from helpers import assert_matches, host_csc, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_08526_gb300 as spg  # noqa: E402
from paper_2010_08526_gb300 import _capi  # noqa: E402
from test_gpu_parity import skewed  # noqa: E402


class FailingAllocator(spg.TorchAllocator):
    """Refuses the allocation with ordinal fail_at (1-based), serves the others."""

    def __init__(self, fail_at):
        super().__init__()
        self.fail_at = fail_at
        self.calls = 0

    def allocate(self, nbytes, kind):
        self.calls += 1
        if self.calls == self.fail_at:
            return None
        return super().allocate(nbytes, kind)


def _product(A, **kw):
    Ad = to_dev(A)
    plan = spg.Plan(Ad, Ad, **kw)
    plan.symbolic()
    outs = [plan.numeric(t) for t in range(plan.nbatches)]
    torch.cuda.synchronize()
    got = host_csc(spg.Csc(A.nrows, A.ncols, *_concat(outs)))
    return plan, got


def _concat(outs):
    cps, rows, vals = [], [], []
    base = 0
    for i, o in enumerate(outs):
        cp = o.colptr.to(torch.int64)
        cps.append(cp[(0 if i == 0 else 1):] + base)
        base += int(cp[-1].item())
        rows.append(o.rowidx)
        vals.append(o.vals)
    return torch.cat(cps), torch.cat(rows), torch.cat(vals)


def test_torch_allocator_holds_the_workspace_and_gives_it_back():
    A = skewed(5000, 5000, 501, hubs=3, hub_deg=2000, base=5)
    tun = spg.Tuning(hash_max_cap=512, panel_rows=2048)
    ref, ab, nt = oracle.spgemm(A, A, with_absterm=True, with_nterm=True)
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    al = spg.TorchAllocator()
    plan, got = _product(A, tuning=tun, allocator=al)
    assert plan.info["heavy_columns"] > 0
    assert al.n_alloc > 0 and al.live > 0
    assert torch.cuda.memory_allocated() - before >= al.bytes_live - sum(
        t.numel() for t in al.blocks.values() if not t.is_cuda)
    assert_matches(got, ref, ab, nt, label="torch allocator")
    plan.close()
    assert al.live == 0 and al.n_free == al.n_alloc and al.bytes_live == 0
    # the same product with the library's own cudaMalloc
    plan2, got2 = _product(A, tuning=tun, allocator=None)
    plan2.close()
    assert np.array_equal(oracle.canonical(got2).rowidx, oracle.canonical(got).rowidx)


def test_run_batched_pinned_ring_from_torch():
    A = skewed(3000, 3000, 502, hubs=2, hub_deg=1000)
    Ad = to_dev(A)
    ref, ab, nt = oracle.spgemm(A, A, with_absterm=True, with_nterm=True)
    al = spg.TorchAllocator()
    budget = A.bytes() * 2 + (1 << 20) + ref.nnz * 12
    plan = spg.Plan(Ad, Ad, budget=budget, host_slot_bytes=1 << 16, host_slots=2, allocator=al)
    plan.symbolic()
    pieces = []

    def sink(batch, c0, c1, arrs):
        cp, ri, va = arrs
        pieces.append((cp.copy(), ri.copy(), va.copy()))
        return 0

    spg.run_batched(plan, sink)
    pinned = [t for t in al.blocks.values() if not t.is_cuda]
    assert pinned and all(t.is_pinned() for t in pinned)
    colptr = [0]
    for cp, _, _ in pieces:
        colptr.extend((cp[1:] + colptr[-1]).tolist())
    from workloads.csc import CSC
    got = CSC(A.nrows, A.ncols, np.array(colptr, np.int64), np.concatenate([p[1] for p in pieces]).astype(np.int64),
              np.concatenate([p[2] for p in pieces]))
    assert_matches(got, ref, ab, nt, label="run_batched, torch allocator")
    plan.close()
    assert al.live == 0


@pytest.mark.parametrize("fail_at", [1, 2, 5, 9, 14, 25, 40])
def test_allocator_failure_is_oom_and_leaks_nothing(fail_at):
    """Refuse one allocation somewhere in plan creation, the symbolic step or
    the numeric step: the call that needed it fails with SPGEMM_ERR_OOM, and
    after the plan is destroyed every block handed out has been given back.
    The device stays usable: the same product then succeeds."""
    A = skewed(4000, 4000, 503, hubs=3, hub_deg=1800, base=5)
    tun = spg.Tuning(hash_max_cap=256, panel_rows=1024)
    Ad = to_dev(A)
    al = FailingAllocator(fail_at)
    failed = None
    plan = None
    try:
        plan = spg.Plan(Ad, Ad, tuning=tun, allocator=al)
        plan.symbolic()
        for t in range(plan.nbatches):
            plan.numeric(t)
        torch.cuda.synchronize()
    except spg.SpgemmError as e:
        failed = e
    finally:
        if plan is not None:
            plan.close()
    if al.calls >= fail_at:
        assert failed is not None and failed.status == 2, failed   # SPGEMM_ERR_OOM
    else:
        assert failed is None   # fewer allocations than fail_at: nothing was refused
    assert al.live == 0 and al.n_free == al.n_alloc, (al.n_alloc, al.n_free)
    # the context is intact
    ref = oracle.spgemm(A, A)
    plan2, got = _product(A, tuning=tun)
    plan2.close()
    assert np.array_equal(oracle.canonical(got).rowidx, ref.rowidx)


def test_allocator_without_free_is_rejected():
    A = skewed(500, 500, 504)
    Ad = to_dev(A)
    al = spg.TorchAllocator()
    al.struct = _capi.SpgemmAllocator(al._alloc_cb, _capi.FREE_FN(), None)
    with pytest.raises(spg.SpgemmError) as ei:
        spg.Plan(Ad, Ad, allocator=al)
    assert ei.value.status == 1   # SPGEMM_ERR_INVALID
