"""Python objects over the C ABI: argument marshalling and output allocation.

All arithmetic of the product runs in the CUDA library; this module only
builds descriptors from torch tensors, allocates outputs with torch, and
passes the current CUDA stream.
"""
from __future__ import annotations

import ctypes
from dataclasses import dataclass
from typing import Callable, List, Optional

import numpy as np
import torch

from . import _capi as C
from ._capi import check, load

_IDX = {torch.int32: C.I32, torch.int64: C.I64}
_VAL = {torch.float64: C.F64, torch.float32: C.F32, torch.int64: C.INT64}
_NP2T = {np.dtype(np.int32): torch.int32, np.dtype(np.int64): torch.int64,
         np.dtype(np.float32): torch.float32, np.dtype(np.float64): torch.float64}


def _stream_handle(stream: Optional[torch.cuda.Stream]) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


@dataclass
class Csc:
    """A CSC matrix held in torch tensors (device tensors for library calls).

    colptr: ncols+1 offsets; rowidx / vals: nnz entries. Rows inside a
    column may be in any order.
    """
    nrows: int
    ncols: int
    colptr: torch.Tensor
    rowidx: torch.Tensor
    vals: torch.Tensor

    @property
    def nnz(self) -> int:
        return int(self.rowidx.numel())

    @property
    def device(self):
        return self.colptr.device

    @classmethod
    def from_host(cls, h, device="cuda", pin: bool = False) -> "Csc":
        """From any object with nrows/ncols/colptr/rowidx/vals numpy arrays."""
        def t(x):
            a = torch.from_numpy(np.ascontiguousarray(x))
            if pin:
                a = a.pin_memory()
            return a.to(device, non_blocking=pin) if device is not None else a
        return cls(int(h.nrows), int(h.ncols), t(h.colptr), t(h.rowidx), t(h.vals))

    def to_host(self):
        """(nrows, ncols, colptr, rowidx, vals) as numpy arrays."""
        return (self.nrows, self.ncols, self.colptr.cpu().numpy(), self.rowidx.cpu().numpy(),
                self.vals.cpu().numpy())

    def struct(self) -> C.SpgemmCsc:
        for name, x in (("colptr", self.colptr), ("rowidx", self.rowidx), ("vals", self.vals)):
            if not x.is_contiguous():
                raise ValueError(f"{name} must be contiguous")
        if self.colptr.numel() != self.ncols + 1:
            raise ValueError("colptr must have ncols+1 entries")
        if self.rowidx.numel() != self.vals.numel():
            raise ValueError("rowidx and vals differ in length")
        s = C.SpgemmCsc()
        s.nrows, s.ncols, s.nnz = self.nrows, self.ncols, self.nnz
        s.colptr = self.colptr.data_ptr()
        s.rowidx = self.rowidx.data_ptr() if self.nnz else 0
        s.vals = self.vals.data_ptr() if self.nnz else 0
        s.ptr_type = _IDX[self.colptr.dtype]
        s.idx_type = _IDX[self.rowidx.dtype]
        s.val_type = _VAL[self.vals.dtype]
        return s


@dataclass
class Tuning:
    """Kernel knobs (0 = library default); see spgemm_tuning in the header."""
    hash_max_cap: int = 0
    panel_rows: int = 0
    short_seg: int = 0
    huge_seg: int = 0
    block_tier_threads: int = 0
    hybrid_sort: bool = False
    warp_max_cap: int = 0

    def struct(self) -> C.SpgemmTuning:
        t = C.SpgemmTuning()
        t.hash_max_cap, t.panel_rows = self.hash_max_cap, self.panel_rows
        t.short_seg, t.huge_seg = self.short_seg, self.huge_seg
        t.block_tier_threads = self.block_tier_threads
        t.hybrid_sort = int(bool(self.hybrid_sort))
        t.warp_max_cap = self.warp_max_cap
        return t


_SEMIRINGS = {"plus_times": 0, "min_plus": 1, "or_and": 2}


_MERGES = {"end": 0, "incremental": 1}


class TorchAllocator:
    """Plan workspace from PyTorch (the spgemm_allocator callbacks): device
    blocks from torch's caching allocator, pinned host blocks from its pinned
    memory allocator. Each block is a uint8 tensor kept alive here until the
    library frees it, so the memory shows up in torch's accounting
    (torch.cuda.memory_allocated) and returns to torch's pool afterwards.
    Counters: n_alloc, n_free, live (blocks held), bytes_live."""

    def __init__(self, device=None):
        self.device = torch.device(device) if device is not None else torch.device(
            "cuda", torch.cuda.current_device())
        self.blocks = {}
        self.n_alloc = 0
        self.n_free = 0
        self.bytes_live = 0
        self._alloc_cb = C.ALLOC_FN(self._alloc)
        self._free_cb = C.FREE_FN(self._free)
        self.struct = C.SpgemmAllocator(self._alloc_cb, self._free_cb, None)

    def allocate(self, nbytes: int, kind: int):
        """A tensor of nbytes bytes of the kind asked for, or None when it
        cannot be had (subclasses may refuse on purpose)."""
        if kind == C.MEM_DEVICE:
            return torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        return torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)

    def _alloc(self, ctx, nbytes, kind):
        try:
            t = self.allocate(int(nbytes), int(kind))
        except Exception:   # out of memory: the library reports SPGEMM_ERR_OOM
            t = None
        if t is None:
            return None
        p = int(t.data_ptr())
        self.blocks[p] = t
        self.n_alloc += 1
        self.bytes_live += int(nbytes)
        return p

    def _free(self, ctx, p, nbytes, kind):
        t = self.blocks.pop(int(p or 0), None)
        if t is not None:
            self.n_free += 1
            self.bytes_live -= int(nbytes)

    @property
    def live(self) -> int:
        return len(self.blocks)


def _allocator_of(allocator, device):
    """allocator: "torch" (default) for a TorchAllocator on the plan's
    device, None for the library's own cudaMalloc / cudaHostAlloc, or an
    object with a .struct (a TorchAllocator or one built the same way)."""
    if allocator is None:
        return None
    if isinstance(allocator, str):
        if allocator != "torch":
            raise ValueError(f"unknown allocator {allocator!r}")
        return TorchAllocator(device)
    return allocator


def _opts(budget=None, kstages=1, tuning: Optional[Tuning] = None, ring_depth=0,
          host_slot_bytes=0, host_slots=0, sort_output=False, prune=None, semiring="plus_times",
          merge="end", allocator=None):
    o = C.SpgemmOpts()
    if allocator is not None:
        o.allocator = ctypes.pointer(allocator.struct)
    o.budget_bytes = int(budget or 0)
    o.kstages = int(kstages)
    o.ring_depth = int(ring_depth)
    o.host_slot_bytes = int(host_slot_bytes)
    o.host_slots = int(host_slots)
    o.sort_output = int(bool(sort_output))
    if prune is not None:
        thr, topk = prune
        o.prune = 1
        o.prune_threshold = float(thr)
        o.prune_topk = int(topk)
    else:
        o.prune = 0
        o.prune_threshold = float("-inf")
        o.prune_topk = 0
    if semiring not in _SEMIRINGS:
        raise ValueError(f"unknown semiring {semiring!r}")
    o.semiring = _SEMIRINGS[semiring]
    if merge not in _MERGES:
        raise ValueError(f"unknown merge mode {merge!r}")
    o.merge_mode = _MERGES[merge]
    keep = None
    if tuning is not None:
        keep = tuning.struct()
        o.tuning = ctypes.pointer(keep)
    return o, keep


class Plan:
    """One product C = A*B: symbolic step, batch plan, numeric per batch.

    A and B must stay alive and unchanged while the plan exists.
    """

    def __init__(self, A: Csc, B: Csc, *, budget: Optional[int] = None, kstages: int = 1,
                 tuning: Optional[Tuning] = None, validate: bool = False, ring_depth: int = 0,
                 host_slot_bytes: int = 0, host_slots: int = 0, sort_output: bool = False,
                 prune: Optional[tuple] = None, semiring: str = "plus_times", merge: str = "end",
                 stream: Optional[torch.cuda.Stream] = None, allocator="torch"):
        """sort_output: rows sorted inside every column of C. prune = (threshold,
        topk): run_batched prunes each batch on the device before the copy
        (see prune()). semiring: "plus_times", "min_plus" (C(i,j) = min_k
        A(i,k) + B(k,j), float values) or "or_and" (Boolean: 1 where some k
        has A(i,k) != 0 and B(k,j) != 0, else 0, any value type). merge (kstages > 1): "end" keeps the
        s stage partials of a batch and merges them once; "incremental"
        merges each stage into the running sum as it is produced (less memory
        when the stages overlap, more merge work). allocator: where the plan's
        workspace comes from: "torch" (PyTorch's allocators, the default),
        None (the library's cudaMalloc / cudaHostAlloc) or a TorchAllocator."""
        lib = load()
        self._lib = lib
        self.A, self.B = A, B
        self._sa, self._sb = A.struct(), B.struct()
        self.allocator = _allocator_of(allocator, A.device)
        self._opts, self._tun = _opts(budget, kstages, tuning, ring_depth, host_slot_bytes,
                                      host_slots, sort_output, prune, semiring, merge, self.allocator)
        h = ctypes.c_void_p()
        check(lib.spgemm_plan_create(ctypes.byref(self._sa), ctypes.byref(self._sb),
                                     ctypes.byref(self._opts), int(validate),
                                     _stream_handle(stream), ctypes.byref(h)))
        self._h = h
        self.info = None

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.spgemm_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- symbolic -------------------------------------------------------------
    def symbolic(self, stream=None) -> dict:
        check(self._lib.spgemm_symbolic(self._h, _stream_handle(stream)))
        return self.query()

    def query(self) -> dict:
        inf = C.SpgemmPlanInfo()
        check(self._lib.spgemm_plan_query(self._h, ctypes.byref(inf)))
        self.info = {f: getattr(inf, f) for f, _ in C.SpgemmPlanInfo._fields_}
        return self.info

    def batch(self, t: int):
        c0, c1, nnz = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        check(self._lib.spgemm_plan_batch(self._h, t, ctypes.byref(c0), ctypes.byref(c1),
                                          ctypes.byref(nnz)))
        return c0.value, c1.value, nnz.value

    @property
    def nbatches(self) -> int:
        return int(self.info["nbatches"]) if self.info else 0

    def column_counts(self, stream=None) -> torch.Tensor:
        out = torch.empty(self.B.ncols, dtype=torch.int64, device=self.A.device)
        check(self._lib.spgemm_plan_column_counts(self._h, ctypes.c_void_p(out.data_ptr()),
                                                  _stream_handle(stream)))
        return out

    def set_timing(self, enable: bool = True):
        check(self._lib.spgemm_plan_set_timing(self._h, int(enable)))

    def stats(self, reset: bool = False) -> dict:
        """Kernel launches and per-phase device milliseconds."""
        s = C.SpgemmStats()
        check(self._lib.spgemm_plan_stats(self._h, int(reset), ctypes.byref(s)))
        return {"launches": int(s.launches),
                "ms": {C.PHASES[i]: float(s.ms[i]) for i in range(C.NUM_PHASES)},
                "count": {C.PHASES[i]: int(s.count[i]) for i in range(C.NUM_PHASES)}}

    def check_errors(self, stream=None):
        """Synchronise and raise if a kernel recorded an error flag."""
        check(self._lib.spgemm_plan_check(self._h, _stream_handle(stream)))

    # -- numeric --------------------------------------------------------------
    def alloc_batch(self, t: int, ptr_dtype=torch.int64) -> Csc:
        c0, c1, nnz = self.batch(t)
        dev = self.A.device
        return Csc(self.A.nrows, c1 - c0,
                   torch.empty(c1 - c0 + 1, dtype=ptr_dtype, device=dev),
                   torch.empty(nnz, dtype=self.A.rowidx.dtype, device=dev),
                   torch.empty(nnz, dtype=self.A.vals.dtype, device=dev))

    def numeric(self, t: int, out: Optional[Csc] = None, ptr_dtype=torch.int64,
                stream=None) -> Csc:
        if out is None:
            out = self.alloc_batch(t, ptr_dtype)
        s = out.struct()
        check(self._lib.spgemm_numeric(self._h, t, ctypes.byref(s), _stream_handle(stream)))
        return out

    def numeric_into(self, t: int, colptr: torch.Tensor, rowidx: torch.Tensor,
                     vals: torch.Tensor, stream=None):
        """Batch t into caller views (rowidx / vals slices of a larger C)."""
        c0, c1, nnz = self.batch(t)
        out = Csc(self.A.nrows, c1 - c0, colptr, rowidx, vals)
        s = out.struct()
        check(self._lib.spgemm_numeric(self._h, t, ctypes.byref(s), _stream_handle(stream)))

    # -- backward -------------------------------------------------------------
    def backward(self, G: Csc, dA: Optional[torch.Tensor] = None,
                 dB: Optional[torch.Tensor] = None, stream=None):
        if dA is None:
            dA = torch.empty_like(self.A.vals)
        if dB is None:
            dB = torch.empty_like(self.B.vals)
        sg = G.struct()
        check(self._lib.spgemm_backward(self._h, ctypes.byref(sg), ctypes.c_void_p(dA.data_ptr()),
                                        ctypes.c_void_p(dB.data_ptr()), _stream_handle(stream)))
        return dA, dB


def spgemm(A: Csc, B: Csc, *, budget: Optional[int] = None, kstages: int = 1,
           tuning: Optional[Tuning] = None, validate: bool = False, stream=None,
           ptr_dtype=torch.int64, sort_output: bool = False, semiring: str = "plus_times",
           merge: str = "end") -> Csc:
    """C = A*B as one device CSC (batches computed one after another into
    slices of the full output). Rows inside columns are unsorted unless
    sort_output. ptr_dtype torch.int32 gives a colptr of the input index type
    (if nnz(C) fits). semiring "min_plus": C(i,j) = min_k A(i,k) + B(k,j);
    "or_and": the Boolean product (1 or 0 on C's structure).
    merge: how a k-split sums its stages ("end" or "incremental", see Plan)."""
    plan = Plan(A, B, budget=budget, kstages=kstages, tuning=tuning, validate=validate,
                sort_output=sort_output, semiring=semiring, merge=merge, stream=stream)
    try:
        info = plan.symbolic(stream)
        nnz = int(info["nnz_c"])
        dev = A.device
        rows = torch.empty(nnz, dtype=A.rowidx.dtype, device=dev)
        vals = torch.empty(nnz, dtype=A.vals.dtype, device=dev)
        colptr = torch.empty(B.ncols + 1, dtype=ptr_dtype, device=dev)
        scratch = torch.empty(int(info["max_batch_cols"]) + 1, dtype=torch.int64, device=dev)
        off = 0
        for t in range(plan.nbatches):
            c0, c1, bn = plan.batch(t)
            plan.numeric_into(t, scratch[: c1 - c0 + 1], rows[off:off + bn], vals[off:off + bn],
                              stream)
            off += bn
        check(plan._lib.spgemm_plan_colptr(plan._h, ctypes.c_void_p(colptr.data_ptr()),
                                           _IDX[ptr_dtype], _stream_handle(stream)))
        out = Csc(A.nrows, B.ncols, colptr, rows, vals)
        out.plan_info = info
        return out
    finally:
        plan.close()


def merge(parts: List[Csc], ptr_dtype=torch.int64, stream=None, _entry="spgemm_merge") -> Csc:
    """Sort-free hash merge: out(:, j) = sum_i parts[i](:, j)."""
    lib = load()
    fn = getattr(lib, _entry)
    if not parts:
        raise ValueError("no parts")
    p0 = parts[0]
    arr = (C.SpgemmCsc * len(parts))(*[p.struct() for p in parts])
    colptr = torch.empty(p0.ncols + 1, dtype=ptr_dtype, device=p0.device)
    out = Csc(p0.nrows, p0.ncols, colptr, p0.rowidx[:0], p0.vals[:0])
    so = out.struct()
    so.rowidx = 0
    so.vals = 0
    so.nnz = 0
    st = _stream_handle(stream)
    check(fn(arr, len(parts), ctypes.byref(so), st))
    nnz = int(so.nnz)
    out.rowidx = torch.empty(nnz, dtype=p0.rowidx.dtype, device=p0.device)
    out.vals = torch.empty(nnz, dtype=p0.vals.dtype, device=p0.device)
    so2 = out.struct()
    if nnz == 0:
        return out
    check(fn(arr, len(parts), ctypes.byref(so2), st))
    return out


def prune(Cm: Csc, threshold: float = float("-inf"), topk: int = 0, stream=None) -> Csc:
    """Column-wise prune (spgemm_prune): per column keep the entries with
    value >= threshold, then at most topk of the largest (topk <= 0: no
    limit; equal values: the earlier stored entry wins), in input order."""
    lib = load()
    colptr = torch.empty(Cm.ncols + 1, dtype=torch.int64, device=Cm.device)
    out = Csc(Cm.nrows, Cm.ncols, colptr, Cm.rowidx[:0], Cm.vals[:0])
    so = out.struct()
    so.rowidx = 0
    so.vals = 0
    so.nnz = 0
    sin = Cm.struct()
    st = _stream_handle(stream)
    check(lib.spgemm_prune(ctypes.byref(sin), float(threshold), int(topk), ctypes.byref(so), st))
    nnz = int(so.nnz)
    out.rowidx = torch.empty(nnz, dtype=Cm.rowidx.dtype, device=Cm.device)
    out.vals = torch.empty(nnz, dtype=Cm.vals.dtype, device=Cm.device)
    if nnz == 0:
        return out
    so2 = out.struct()
    check(lib.spgemm_prune(ctypes.byref(sin), float(threshold), int(topk), ctypes.byref(so2), st))
    return out


def merge_noalloc(parts: List[Csc], ptr_dtype=torch.int64, stream=None) -> Csc:
    """The same merge through spgemm_merge_noalloc, which allocates no device
    memory of its own (the output buffers are still allocated here, by torch)."""
    return merge(parts, ptr_dtype, stream, _entry="spgemm_merge_noalloc")


def run_batched(plan: Plan, sink: Callable[[int, int, int, tuple], Optional[int]],
                compute: Optional[torch.cuda.Stream] = None,
                copy: Optional[torch.cuda.Stream] = None) -> None:
    """Algorithm 4's batch loop: sink(batch, col_begin, col_end, (colptr,
    rowidx, vals)) receives numpy views of pinned host memory that are valid
    only during the call. Returning a non-zero value stops the run."""
    lib = load()
    err: list = []

    def _cb(ctx, batch, c0, c1, piece):
        try:
            p = piece.contents
            n = int(p.ncols)
            nnz = int(p.nnz)
            idt = ctypes.c_int64 if p.idx_type == C.I64 else ctypes.c_int32
            vdt = {C.F64: ctypes.c_double, C.F32: ctypes.c_float, C.INT64: ctypes.c_int64}[p.val_type]
            cp = np.ctypeslib.as_array(ctypes.cast(p.colptr, ctypes.POINTER(ctypes.c_int64)), (n + 1,))
            if nnz:
                ri = np.ctypeslib.as_array(ctypes.cast(p.rowidx, ctypes.POINTER(idt)), (nnz,))
                va = np.ctypeslib.as_array(ctypes.cast(p.vals, ctypes.POINTER(vdt)), (nnz,))
            else:
                ri = np.zeros(0, dtype=np.int64)
                va = np.zeros(0)
            r = sink(int(batch), int(c0), int(c1), (cp, ri, va))
            return int(r or 0)
        except BaseException as e:  # surfaces after the library drains
            err.append(e)
            return 1

    cb = C.SINK_FN(_cb)
    comp = compute if compute is not None else torch.cuda.current_stream()
    cpy = copy if copy is not None else torch.cuda.Stream()
    st = lib.spgemm_run_batched(plan._h, cb, None, ctypes.c_void_p(comp.cuda_stream),
                                ctypes.c_void_p(cpy.cuda_stream))
    if err:
        raise err[0]
    check(st)


def transpose(A: Csc, ptr_dtype=torch.int64, stream=None) -> Csc:
    """A^T as a device CSC (spgemm_transpose; rows inside a column unsorted)."""
    lib = load()
    dev = A.device
    out = Csc(A.ncols, A.nrows, torch.empty(A.nrows + 1, dtype=ptr_dtype, device=dev),
              torch.empty(A.nnz, dtype=A.rowidx.dtype, device=dev),
              torch.empty(A.nnz, dtype=A.vals.dtype, device=dev))
    si, so = A.struct(), out.struct()
    check(lib.spgemm_transpose(ctypes.byref(si), ctypes.byref(so), _stream_handle(stream)))
    return out


def spgemm_aat(A: Csc, **kw) -> Csc:
    """C = A A^T (the BELLA overlap product of Sec. V): the transpose on the
    device, then the column-batched product."""
    At = transpose(A, ptr_dtype=A.colptr.dtype, stream=kw.get("stream"))
    C = spgemm(A, At, **kw)
    C.transposed_operand = At
    return C


def run_row_batched(A: Csc, B: Csc, sink: Callable[[int, int, int, tuple], Optional[int]], *,
                    budget: Optional[int] = None, sort_output: bool = False, prune: Optional[tuple] = None,
                    host_slot_bytes: int = 0, host_slots: int = 0, compute=None, copy=None) -> None:
    """Row-by-row batching of C = A B (Sec. IV-B, for when nnz(A) >> nnz(B)):
    the column batch loop on C^T = B^T A^T. sink(batch, row_begin, row_end,
    (rowptr, colidx, vals)) receives a block of rows of C in CSR form (the
    CSC of that column block of C^T), pinned host memory valid during the
    call. With prune, the rule applies to the rows of C."""
    Bt = transpose(B, ptr_dtype=B.colptr.dtype)
    At = transpose(A, ptr_dtype=A.colptr.dtype)
    plan = Plan(Bt, At, budget=budget, sort_output=sort_output, prune=prune,
                host_slot_bytes=host_slot_bytes, host_slots=host_slots)
    try:
        plan.symbolic()
        run_batched(plan, sink, compute=compute, copy=copy)
    finally:
        plan.close()
        del Bt, At


def backward(A: Csc, B: Csc, G: Csc, stream=None):
    """(dA, dB) for loss = sum over pattern(C) of C * G."""
    plan = Plan(A, B, stream=stream)
    try:
        return plan.backward(G, stream=stream)
    finally:
        plan.close()


class SpGEMMFn(torch.autograd.Function):
    """C_vals = SpGEMM(A_vals, B_vals) on fixed patterns.

    forward(A_vals, B_vals, A_pattern, B_pattern) returns the values of C in
    the layout of ``ctx.C`` (unsorted rows). backward receives dC on that
    layout and returns (dA_vals, dB_vals) from the masked-SpGEMM kernels:
    dA = (dC B^T) on pattern(A), dB = (A^T dC) on pattern(B). The symbolic
    plan is kept between forward and backward unless ``recompute_plan``.
    """

    @staticmethod
    def forward(ctx, a_vals, b_vals, A: Csc, B: Csc, recompute_plan: bool = False,
                budget: Optional[int] = None):
        Ad = Csc(A.nrows, A.ncols, A.colptr, A.rowidx, a_vals.detach().contiguous())
        Bd = Csc(B.nrows, B.ncols, B.colptr, B.rowidx, b_vals.detach().contiguous())
        plan = Plan(Ad, Bd, budget=budget)
        info = plan.symbolic()
        if info["nbatches"] != 1:
            plan.close()
            raise ValueError("SpGEMMFn needs the product to fit one batch")
        Cout = plan.numeric(0)
        ctx.C = Cout
        ctx.shapes = (A, B)
        ctx.save_for_backward(a_vals, b_vals)
        if recompute_plan:
            plan.close()
            ctx.plan = None
        else:
            ctx.plan = plan
        return Cout.vals

    @staticmethod
    def backward(ctx, dc_vals):
        a_vals, b_vals = ctx.saved_tensors
        A, B = ctx.shapes
        Ad = Csc(A.nrows, A.ncols, A.colptr, A.rowidx, a_vals.detach().contiguous())
        Bd = Csc(B.nrows, B.ncols, B.colptr, B.rowidx, b_vals.detach().contiguous())
        plan = ctx.plan if ctx.plan is not None else Plan(Ad, Bd)
        Cl = ctx.C
        G = Csc(Cl.nrows, Cl.ncols, Cl.colptr, Cl.rowidx, dc_vals.contiguous())
        dA, dB = plan.backward(G)
        plan.close()
        ctx.plan = None
        return dA, dB, None, None, None, None


class Multi:
    """Many independent products C_i = A_i * B_i in one pass.

    The output is one arena: the C_i concatenated column by column (rows stay
    local to each problem) with an int64 colptr over all columns.
    """

    def __init__(self, As: List[Csc], Bs: List[Csc], *, tuning: Optional[Tuning] = None,
                 stream=None, allocator="torch"):
        lib = load()
        self._lib = lib
        self.As, self.Bs = As, Bs
        n = len(As)
        self._sa = (C.SpgemmCsc * n)(*[a.struct() for a in As])
        self._sb = (C.SpgemmCsc * n)(*[b.struct() for b in Bs])
        self.allocator = _allocator_of(allocator, As[0].device)
        self._opts, self._tun = _opts(tuning=tuning, allocator=self.allocator)
        h = ctypes.c_void_p()
        check(lib.spgemm_multi_create(n, self._sa, self._sb, ctypes.byref(self._opts),
                                      _stream_handle(stream), ctypes.byref(h)))
        self._h = h
        cp = ctypes.POINTER(ctypes.c_int64)()
        ri, va = ctypes.c_void_p(), ctypes.c_void_p()
        tc, cap = ctypes.c_int64(), ctypes.c_int64()
        check(lib.spgemm_multi_output(self._h, ctypes.byref(cp), ctypes.byref(ri),
                                      ctypes.byref(va), ctypes.byref(tc), ctypes.byref(cap)))
        self.total_cols = tc.value
        self.capacity = cap.value
        self._out_ptrs = (ctypes.cast(cp, ctypes.c_void_p).value, ri.value, va.value)

    def run(self, use_graph: bool = True, stream=None):
        check(self._lib.spgemm_multi_run(self._h, int(use_graph), _stream_handle(stream)))

    def output(self):
        """(colptr, rowidx, vals) torch views of the arena (after run)."""
        dev = self.As[0].device
        cp_ptr, ri_ptr, va_ptr = self._out_ptrs
        colptr = _wrap_device(cp_ptr, self.total_cols + 1, torch.int64, dev)
        nnz = int(colptr[-1].item())
        rowidx = _wrap_device(ri_ptr, nnz, self.As[0].rowidx.dtype, dev)
        vals = _wrap_device(va_ptr, nnz, self.As[0].vals.dtype, dev)
        return colptr, rowidx, vals

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.spgemm_multi_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class _DevView:
    """Exposes library-owned device memory through __cuda_array_interface__."""

    _TYPESTR = {torch.int64: "<i8", torch.int32: "<i4", torch.float32: "<f4",
                torch.float64: "<f8"}

    def __init__(self, ptr: int, n: int, dtype):
        self.__cuda_array_interface__ = {
            "shape": (n,), "typestr": self._TYPESTR[dtype], "data": (ptr, False),
            "version": 3, "strides": None, "stream": None,
        }


def _wrap_device(ptr: int, n: int, dtype, device) -> torch.Tensor:
    """A zero-copy torch view of library-owned device memory; valid while the
    owning library object lives."""
    if n == 0:
        return torch.empty(0, dtype=dtype, device=device)
    return torch.as_tensor(_DevView(ptr, n, dtype), device=device)
