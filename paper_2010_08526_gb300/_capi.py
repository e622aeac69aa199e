"""ctypes declarations of the C ABI in include/spgemm.h (marshalling only)."""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libspgemm_gb300.so")

SPGEMM_OK = 0
STATUS = {
    0: "SPGEMM_OK", 1: "SPGEMM_ERR_INVALID", 2: "SPGEMM_ERR_OOM", 3: "SPGEMM_ERR_BUDGET",
    4: "SPGEMM_ERR_OVERFLOW", 5: "SPGEMM_ERR_INDEX_OVERFLOW", 6: "SPGEMM_ERR_CUDA",
    7: "SPGEMM_ERR_TIMEOUT", 8: "SPGEMM_ERR_SINK", 9: "SPGEMM_ERR_STATE",
}
I32, I64 = 0, 1
F64, F32, INT64 = 0, 1, 2


class SpgemmCsc(ctypes.Structure):
    _fields_ = [
        ("nrows", ctypes.c_int64), ("ncols", ctypes.c_int64), ("nnz", ctypes.c_int64),
        ("colptr", ctypes.c_void_p), ("rowidx", ctypes.c_void_p), ("vals", ctypes.c_void_p),
        ("ptr_type", ctypes.c_int), ("idx_type", ctypes.c_int), ("val_type", ctypes.c_int),
    ]


class SpgemmTuning(ctypes.Structure):
    _fields_ = [
        ("hash_max_cap", ctypes.c_int), ("panel_rows", ctypes.c_int), ("short_seg", ctypes.c_int),
        ("huge_seg", ctypes.c_int), ("block_tier_threads", ctypes.c_int),
        ("hybrid_sort", ctypes.c_int), ("warp_max_cap", ctypes.c_int), ("reserved", ctypes.c_int * 1),
    ]


MEM_DEVICE, MEM_PINNED_HOST = 0, 1
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int)


class SpgemmAllocator(ctypes.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", ctypes.c_void_p)]


class SpgemmOpts(ctypes.Structure):
    _fields_ = [
        ("budget_bytes", ctypes.c_size_t), ("kstages", ctypes.c_int), ("ring_depth", ctypes.c_int),
        ("host_slot_bytes", ctypes.c_size_t), ("host_slots", ctypes.c_int),
        ("sort_output", ctypes.c_int), ("tuning", ctypes.POINTER(SpgemmTuning)),
        ("prune", ctypes.c_int), ("prune_threshold", ctypes.c_double), ("prune_topk", ctypes.c_int64),
        ("semiring", ctypes.c_int), ("merge_mode", ctypes.c_int),
        ("allocator", ctypes.POINTER(SpgemmAllocator)),
    ]


class SpgemmPlanInfo(ctypes.Structure):
    _fields_ = [
        ("flops", ctypes.c_int64), ("nnz_c", ctypes.c_int64), ("unmerged_nnz", ctypes.c_int64),
        ("nbatches", ctypes.c_int64), ("max_batch_nnz", ctypes.c_int64),
        ("max_batch_cols", ctypes.c_int64), ("bytes_per_nnz", ctypes.c_int64),
        ("batch_cap_bytes", ctypes.c_int64), ("heavy_columns", ctypes.c_int64),
        ("stage_buffer_nnz", ctypes.c_int64),
    ]


NUM_PHASES = 9
PHASES = ["flops_bin", "sym_hash", "sym_heavy", "scan", "panels", "num_hash", "num_dense",
          "merge", "backward"]


class SpgemmStats(ctypes.Structure):
    _fields_ = [
        ("launches", ctypes.c_int64), ("ms", ctypes.c_double * NUM_PHASES),
        ("count", ctypes.c_int64 * NUM_PHASES),
    ]


SINK_FN = ctypes.CFUNCTYPE(ctypes.c_int, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                           ctypes.c_int64, ctypes.POINTER(SpgemmCsc))

# name -> (restype, argtypes); every symbol the header declares
P = ctypes.POINTER
vp = ctypes.c_void_p
i64 = ctypes.c_int64
SIGNATURES = {
    "spgemm_last_error": (ctypes.c_char_p, []),
    "spgemm_version": (ctypes.c_char_p, []),
    "spgemm_plan_create": (ctypes.c_int, [P(SpgemmCsc), P(SpgemmCsc), P(SpgemmOpts), ctypes.c_int,
                                          vp, P(vp)]),
    "spgemm_plan_destroy": (ctypes.c_int, [vp]),
    "spgemm_symbolic": (ctypes.c_int, [vp, vp]),
    "spgemm_plan_query": (ctypes.c_int, [vp, P(SpgemmPlanInfo)]),
    "spgemm_plan_batch": (ctypes.c_int, [vp, i64, P(i64), P(i64), P(i64)]),
    "spgemm_plan_column_counts": (ctypes.c_int, [vp, vp, vp]),
    "spgemm_plan_check": (ctypes.c_int, [vp, vp]),
    "spgemm_plan_colptr": (ctypes.c_int, [vp, vp, ctypes.c_int, vp]),
    "spgemm_plan_set_timing": (ctypes.c_int, [vp, ctypes.c_int]),
    "spgemm_plan_stats": (ctypes.c_int, [vp, ctypes.c_int, P(SpgemmStats)]),
    "spgemm_numeric": (ctypes.c_int, [vp, i64, P(SpgemmCsc), vp]),
    "spgemm_merge": (ctypes.c_int, [P(SpgemmCsc), ctypes.c_int, P(SpgemmCsc), vp]),
    "spgemm_prune": (ctypes.c_int, [P(SpgemmCsc), ctypes.c_double, ctypes.c_int64, P(SpgemmCsc), vp]),
    "spgemm_transpose": (ctypes.c_int, [P(SpgemmCsc), P(SpgemmCsc), vp]),
    "spgemm_merge_noalloc": (ctypes.c_int, [P(SpgemmCsc), ctypes.c_int, P(SpgemmCsc), vp]),
    "spgemm_run_batched": (ctypes.c_int, [vp, SINK_FN, vp, vp, vp]),
    "spgemm_backward": (ctypes.c_int, [vp, P(SpgemmCsc), vp, vp, vp]),
    "spgemm_multi_create": (ctypes.c_int, [ctypes.c_int, P(SpgemmCsc), P(SpgemmCsc),
                                           P(SpgemmOpts), vp, P(vp)]),
    "spgemm_multi_destroy": (ctypes.c_int, [vp]),
    "spgemm_multi_run": (ctypes.c_int, [vp, ctypes.c_int, vp]),
    "spgemm_multi_output": (ctypes.c_int, [vp, P(P(i64)), P(vp), P(vp), P(i64), P(i64)]),
}

_LIB = None


class SpgemmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


def load(path: str = LIB_PATH):
    """Load the CUDA library; raises if it has not been built."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(path):
        raise RuntimeError(
            f"{path} is missing: build the sm_103a library first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def check(status: int):
    if status != SPGEMM_OK:
        raise SpgemmError(status, load().spgemm_last_error().decode())
