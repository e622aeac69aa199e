"""Autotuner for the kernel knobs (spgemm_tuning).

Times the real product for each candidate setting with CUDA events on the
current stream and returns the fastest. The knobs:

* hash_max_cap        -- largest column kept in a shared-memory hash table;
                         columns above it use the dense row-panel path
                         (which bins columns into tiers: the bin thresholds);
* panel_rows          -- rows of one dense panel (shared-memory accumulator
                         size);
* block_tier_threads  -- CTA size of the hash tiers (block shape).

For the batched products (Multi) the knobs are those of its persistent
passes: hash_max_cap (the largest shared-memory table, so the split between
CTA items and global-table items and the shared memory each CTA holds),
warp_max_cap (the largest column one warp takes with a private table) and
block_tier_threads (CTA width, 128, 256 or 512); multi_candidates() is the grid.

Every candidate is checked to give the same nnz(C) as the first one; a
candidate that fails (for example an invalid combination) is skipped.
"""
from __future__ import annotations

import itertools
from dataclasses import asdict
from typing import Callable, Iterable, List, Optional, Sequence, Tuple

import torch

from .core import Csc, Multi, Plan, Tuning
from ._capi import SpgemmError

DEFAULT_CAPS = (2048, 4096, 8192)
DEFAULT_PANELS = (8192, 16384, 32768)
DEFAULT_THREADS = (0, 256, 512)


def candidates(caps: Sequence[int] = DEFAULT_CAPS, panels: Sequence[int] = DEFAULT_PANELS,
               threads: Sequence[int] = DEFAULT_THREADS) -> List[Tuning]:
    return [Tuning(hash_max_cap=c, panel_rows=p, block_tier_threads=t)
            for c, p, t in itertools.product(caps, panels, threads)]


def _time(fn: Callable[[], None], reps: int) -> float:
    st = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def tune_plan(A: Csc, B: Csc, cands: Optional[Iterable[Tuning]] = None, reps: int = 2,
              budget: Optional[int] = None) -> Tuple[Tuning, list]:
    """Symbolic + numeric of C = A*B for each candidate; returns the fastest
    Tuning and the (tuning, ms) list."""
    cands = list(cands) if cands is not None else candidates()
    results = []
    ref_nnz = None
    for tun in cands:
        try:
            plan = Plan(A, B, budget=budget, tuning=tun)
        except SpgemmError:
            continue
        try:
            info = plan.symbolic()
            if ref_nnz is None:
                ref_nnz = info["nnz_c"]
            elif info["nnz_c"] != ref_nnz:
                raise RuntimeError(f"candidate {tun} changed nnz(C)")
            outs = [plan.alloc_batch(t) for t in range(plan.nbatches)]

            def step():
                plan.symbolic()
                for t in range(plan.nbatches):
                    plan.numeric(t, out=outs[t])
            ms = _time(step, reps)
            plan.check_errors()
            results.append((tun, ms))
            del outs
        except SpgemmError:
            pass
        finally:
            plan.close()
            torch.cuda.empty_cache()
    if not results:
        raise RuntimeError("no tuning candidate ran")
    best = min(results, key=lambda r: r[1])[0]
    return best, results


MULTI_CAPS = (1024, 2048, 4096, 8192)
MULTI_WARP_CAPS = (128, 256, 512)
MULTI_THREADS = (128, 256, 512)


def multi_candidates(caps: Sequence[int] = MULTI_CAPS, warp_caps: Sequence[int] = MULTI_WARP_CAPS,
                     threads: Sequence[int] = MULTI_THREADS) -> List[Tuning]:
    """The grid of the batched passes' knobs (combinations whose tables do
    not fit are refused by the library and skipped)."""
    return [Tuning(hash_max_cap=c, warp_max_cap=w, block_tier_threads=t)
            for c, w, t in itertools.product(caps, warp_caps, threads) if w <= c]


def tune_multi(As: List[Csc], Bs: List[Csc], cands: Optional[Iterable[Tuning]] = None,
               reps: int = 2) -> Tuple[Tuning, list]:
    """The batched multi-problem pass (CUDA graph) for each candidate; the
    fastest Tuning and the (tuning, ms) list."""
    if cands is None:
        cands = multi_candidates()
    results = []
    for tun in cands:
        try:
            M = Multi(As, Bs, tuning=tun)
        except SpgemmError:
            continue
        try:
            ms = _time(lambda: M.run(use_graph=True), reps)
            results.append((tun, ms))
        finally:
            M.close()
            torch.cuda.empty_cache()
    if not results:
        raise RuntimeError("no tuning candidate ran")
    best = min(results, key=lambda r: r[1])[0]
    return best, results


def describe(results) -> list:
    return [{**asdict(t), "ms": round(ms, 3)} for t, ms in results]
