"""Benchmark of the memory-constrained SpGEMM hot path on one GB300.

Workload (one step): C = A*A for A = R-MAT scale 20 (1,048,576 x 1,048,576,
edge factor 16, a=0.57 b=c=0.19 d=0.05, symmetrised, duplicates summed),
float32 values accumulated in float32, int32 CSC. A step runs the whole
path: flop count and tier binning, symbolic count per column, batch plan for
the HBM budget, row-panel copy of A, and the numeric hash / dense kernels for
every batch. Inputs (250 MB) and outputs (~190 GB) are far larger than L2, so
no flush is needed between steps.

value : SpGEMM GFLOP/s (2 x multiplications / step time), inputs resident.
e2e   : the same metric through the C ABI with host buffers: every step copies
        A from pinned host memory, runs symbolic + the batch loop that streams
        every column batch of C to pinned host slots (spgemm_run_batched), and
        reads the result back on the host.

Extra keys: the k-split path (4 stages + sort-free hash merge) on the same
workload, the batched persistent launch (512 uneven products in one CUDA
graph) vs 512 plain per-matrix launches, and forward + masked backward vs
gradients formed by plain SpGEMMs.

--impl reference times the CPU oracle (the plain Gustavson definition) on the
host cores on a bounded column sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "SpGEMM GFLOP/s (2 x multiplies / s)"
UNIT = "GFLOP/s"
WORKLOAD = ("C = A*A, A R-MAT scale 20 (1,048,576^2, edge factor 16, a=.57 b=c=.19 d=.05), "
            "symmetrised, duplicates summed, fp32 U(0,1) accumulated in fp32, int32 CSC")


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", os.environ.get("BENCH_GPU_INDEX", "0")],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------- helpers
def algorithmic_bytes_dense(A, f, cnt, cap, si=4, sv=4):
    """Column-Gustavson bytes of the dense (heavy) numeric kernel: per dense
    column j, its B entries (index + value) and two colptr reads of A per B
    entry, every gathered A entry (index + value), and every written C entry
    (index + value)."""
    dense = cnt > cap
    nnzb = np.diff(A.colptr.astype(np.int64))
    b_bytes = int(nnzb[dense].sum()) * (si + sv + 2 * si)
    a_bytes = int(f[dense].sum()) * (si + sv)
    c_bytes = int(cnt[dense].sum()) * (si + sv)
    return b_bytes + a_bytes + c_bytes, int(dense.sum())


def flops_host_ab(A, B):
    """Multiplications per column of A*B."""
    deg = np.diff(A.colptr.astype(np.int64))
    cols = np.repeat(np.arange(B.ncols), np.diff(B.colptr.astype(np.int64)))
    return np.bincount(cols, weights=deg[B.rowidx.astype(np.int64)].astype(np.float64),
                       minlength=B.ncols).astype(np.int64)


def flops_host(A):
    deg = np.diff(A.colptr.astype(np.int64))
    cols = np.repeat(np.arange(A.ncols), deg)
    return np.bincount(cols, weights=deg[A.rowidx.astype(np.int64)].astype(np.float64),
                       minlength=A.ncols).astype(np.int64)


def dist_init(n_gpus):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo"
        dist.init_process_group(backend)
    return rank, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- reference arm
def cpu_oracle_sample(A, f, target_flops, threads=None):
    """Time the oracle (as it stands) on a contiguous column range of about
    target_flops multiplications; returns (GFLOP/s, sample description, cores).
    threads: run it on that many OpenMP threads (default: all)."""
    import oracle
    from workloads.csc import column_slice
    if threads:
        saved = oracle.num_threads()
        oracle.set_threads(threads)
        try:
            return cpu_oracle_sample(A, f, target_flops)
        finally:
            oracle.set_threads(saved)
    rng = np.random.default_rng(0)
    c0 = int(rng.integers(0, A.ncols // 2))
    cs = np.cumsum(f[c0:])
    c1 = c0 + int(np.searchsorted(cs, target_flops)) + 1
    c1 = min(c1, A.ncols)
    fl = int(f[c0:c1].sum())
    cores = oracle.num_threads()
    # the range in pieces of at most ~1.5e9 multiplies, each product freed
    # before the next, so host memory holds one piece's output (~10 GB), not
    # the whole sample's; only the oracle calls are timed
    piece = 1.5e9
    cuts = [c0]
    acc = 0
    for j in range(c0, c1):
        acc += int(f[j])
        if acc >= piece and j + 1 < c1:
            cuts.append(j + 1)
            acc = 0
    cuts.append(c1)
    dt = 0.0
    nnz = 0
    for a, b in zip(cuts, cuts[1:]):
        Bs = column_slice(A, a, b)
        t0 = time.perf_counter()
        C = oracle.spgemm(A, Bs)
        dt += time.perf_counter() - t0
        nnz += C.nnz
        del C, Bs
    desc = (f"columns [{c0}, {c1}) of the workload ({c1 - c0} columns, {fl:.3e} multiplies, "
            f"nnz(C) {nnz}, in {len(cuts) - 1} column pieces), oracle symbolic + numeric, "
            f"float64 accumulation")
    return 2 * fl / dt / 1e9, desc, cores, dt


def run_reference(args):
    rank, world = dist_init(args.gpus)
    if rank != 0:
        return
    A = W.config2()
    f = flops_host(A)
    vals = []
    desc = cores = None
    # every step is a bounded sample: about 2 minutes of oracle work over the
    # whole run (at ~1 GFLOP/s on 16 cores), and never more than --ref-flops
    per_step = max(2e8, min(args.ref_flops, 6e10 / max(1, args.warmup + args.steps)))
    for i in range(args.warmup + args.steps):
        v, desc, cores, _ = cpu_oracle_sample(A, f, per_step)
        if i >= args.warmup:
            vals.append(v)
    v = float(np.mean(vals))
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "higher_is_better": True,
        "scaling": "weak", "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "oracle": "plain CPU Gustavson with a dense accumulator"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "vs_baseline": None,
    }
    print(json.dumps(line))


# ---------------------------------------------------------------- GPU arm
def pinned_d2h_peak(torch, dev):
    """GB/s of a plain device-to-pinned-host copy (4 x 1 GiB, best of 3)."""
    GB = 1 << 30
    src = torch.empty(4 * GB, dtype=torch.uint8, device=f"cuda:{dev}")
    src.fill_(1)
    host = torch.empty(GB, dtype=torch.uint8, pin_memory=True)
    best = 0.0
    for _ in range(3):
        torch.cuda.synchronize()
        t = time.perf_counter()
        for i in range(4):
            host.copy_(src[i * GB:(i + 1) * GB], non_blocking=True)
        torch.cuda.synchronize()
        best = max(best, 4 * GB / (time.perf_counter() - t) / 1e9)
    del src, host
    torch.cuda.empty_cache()
    return best


def run_gpu(args):
    import torch
    import paper_2010_08526_gb300 as spg

    rank, world = dist_init(args.gpus)
    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    os.environ["BENCH_GPU_INDEX"] = str(dev)
    A = W.config2(scale=args.scale)
    f = flops_host(A)
    F = int(f.sum())
    st = torch.cuda.current_stream()

    Ad = spg.Csc.from_host(A, device=f"cuda:{dev}")
    plan = spg.Plan(Ad, Ad)
    plan.set_timing(True)
    info = plan.symbolic()
    assert info["flops"] == F
    outs = [plan.alloc_batch(t) for t in range(plan.nbatches)]

    def step():
        plan.symbolic()
        for t in range(plan.nbatches):
            plan.numeric(t, out=outs[t])

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    plan.stats(reset=True)
    plan.check_errors()
    clk = ClockSampler()
    barrier(world)
    torch.cuda.synchronize()
    clk.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    ms = e0.elapsed_time(e1) / args.steps
    ms = max_over_ranks(ms, world)
    stats = plan.stats(reset=True)
    plan.check_errors()
    value = world * 2 * F / (ms / 1e3) / 1e9

    # roofline of the dominant kernel (dense row-panel numeric)
    cnt = plan.column_counts().cpu().numpy()
    hbm, peak_kind = peaks()
    dense_ms = stats["ms"]["num_dense"] / max(1, stats["count"]["num_dense"])
    bytes_dense, ndense = algorithmic_bytes_dense(A, f, cnt, 8192)
    launches_dense = max(1, stats["count"]["num_dense"] // args.steps)
    bytes_per_launch = bytes_dense / launches_dense
    achieved = bytes_per_launch / (dense_ms / 1e3) / 1e9 if dense_ms > 0 else 0.0
    phase_ms = {k: round(v / args.steps, 3) for k, v in stats["ms"].items() if v}
    traffic = None
    tf = os.path.join(ROOT, "profiles", "traffic_num_heavy32.txt")
    if os.path.exists(tf) and args.scale == 20:
        for line in open(tf):
            if line.startswith("bytes_per_full_launch"):
                traffic = float(line.split()[1])

    # ---- k-split (4 stages + hash merge) on the same workload
    ks = None
    if not args.quick:
        del outs
        torch.cuda.empty_cache()
        kplan = spg.Plan(Ad, Ad, kstages=4)
        kplan.set_timing(True)
        kinfo = kplan.symbolic()
        kouts = [kplan.alloc_batch(t) for t in range(kplan.nbatches)]

        def kstep():
            kplan.symbolic()
            for t in range(kplan.nbatches):
                kplan.numeric(t, out=kouts[t])
        kstep()
        torch.cuda.synchronize()
        ks_steps = max(1, args.steps // 2)
        k0 = torch.cuda.Event(enable_timing=True)
        k1 = torch.cuda.Event(enable_timing=True)
        kplan.stats(reset=True)
        k0.record(st)
        for _ in range(ks_steps):
            kstep()
        k1.record(st)
        torch.cuda.synchronize()
        kms = k0.elapsed_time(k1) / ks_steps
        kstats = kplan.stats(reset=True)
        kplan.check_errors()
        # the sort-free hash merge (Sec. IV-D) on the HBM roofline: it reads
        # every stage partial entry and writes every entry of C
        mbytes = (int(kinfo["unmerged_nnz"]) + int(kinfo["nnz_c"])) * (4 + 4)
        mms = kstats["ms"]["merge"] / ks_steps
        ks = {"value": 2 * F / (kms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": kms,
              "stages": 4, "nbatches": kinfo["nbatches"], "unmerged_nnz": kinfo["unmerged_nnz"],
              "stage_buffer_nnz": kinfo["stage_buffer_nnz"], "merge": "end",
              "phase_ms_per_step": {k: round(v / ks_steps, 3) for k, v in kstats["ms"].items() if v},
              "merge_roofline": {"bound": "hbm", "algorithmic_bytes": mbytes, "merge_ms": mms,
                                 "achieved": mbytes / (mms / 1e3) / 1e9 if mms else 0.0,
                                 "peak": peaks()[0], "unit": "GB/s",
                                 "frac": (mbytes / (mms / 1e3) / 1e9) / peaks()[0] if mms else 0.0,
                                 "note": "sum_t nnz(D_t) + nnz(C) entries of (index + value)"}}
        del kouts
        kplan.close()
        torch.cuda.empty_cache()
        outs = None

    # ---- e2e through the C ABI with host buffers
    e2e = None
    if not args.no_e2e:
        if outs is not None:
            del outs
            torch.cuda.empty_cache()
        hostA = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory()
                 for x in (A.colptr, A.rowidx, A.vals)]
        dA = spg.Csc(A.nrows, A.ncols, *[torch.empty_like(h, device=f"cuda:{dev}") for h in hostA])
        for h, d in zip(hostA, (dA.colptr, dA.rowidx, dA.vals)):
            d.copy_(h)
        # one plan object serves every step (same shapes); each step copies new
        # input values in and redoes the symbolic analysis
        # batches of ~24 GB keep the copy engine busy from early in the step
        # (a copy of batch t overlaps the multiply of batch t+1)
        ebudget = 2 * (24 << 30) + 4 * A.bytes() + (4 << 30)
        eplan = spg.Plan(dA, dA, budget=ebudget, host_slot_bytes=1 << 30, host_slots=4)
        copy_stream = torch.cuda.Stream()
        got = {"bytes": 0, "check": 0.0}

        def sink(batch, c0, c1, arrs):
            cp, ri, va = arrs
            got["bytes"] += cp.nbytes + ri.nbytes + va.nbytes
            if va.size:
                got["check"] += float(va[0])
            return 0

        def estep():
            for h, d in zip(hostA, (dA.colptr, dA.rowidx, dA.vals)):
                d.copy_(h, non_blocking=True)
            eplan.symbolic()
            got["bytes"] = 0
            spg.run_batched(eplan, sink, copy=copy_stream)
            return got["bytes"]

        estep()
        torch.cuda.synchronize()
        e_steps = max(1, min(args.steps, 3))
        t0 = time.perf_counter()
        bo = 0
        for _ in range(e_steps):
            bo = estep()
        torch.cuda.synchronize()
        edt = (time.perf_counter() - t0) / e_steps
        bi = sum(h.numel() * h.element_size() for h in hostA)
        eplan.close()
        # the D2H roofline: a plain pinned copy of 4 GiB from HBM, same box
        peak_d2h = pinned_d2h_peak(torch, dev)
        e2e = {"value": world * 2 * F / edt / 1e9, "unit": UNIT, "h2d_bytes_per_step": bi,
               "d2h_bytes_per_step": bo, "ms_per_step": edt * 1e3,
               "d2h_gbs": bo / edt / 1e9, "d2h_peak_gbs": peak_d2h,
               "d2h_frac": (bo / edt / 1e9) / peak_d2h if peak_d2h else None}

    # ---- batched persistent launch vs plain per-matrix path; fwd+bwd vs plain
    extras = {}
    if not args.quick:
        extras["batched_vs_plain"] = bench_multi(spg, torch, args)
        extras["fwdbwd_vs_plain"] = bench_fwdbwd(spg, torch, args)
        extras["sorted_and_topk"] = bench_sorted_topk(spg, torch, args, A, F, dev)
        extras["min_plus"] = bench_step(spg, torch, args, A, dev, semiring="min_plus",
                                        note="the same product over the min-plus semiring")
        extras["min_plus"].pop("_counts")
        extras["or_and"] = bench_step(spg, torch, args, A, dev, semiring="or_and",
                                      note="the same product over the Boolean or-and semiring")
        extras["or_and"].pop("_counts")
        extras["protein_2M"] = bench_protein(spg, torch, args, dev)
        extras["kmerge"] = bench_kmerge(spg, torch, args, A, dev)
        extras["er4096"] = bench_config1(spg, torch, args, dev)
        extras["aat_kmer"] = bench_aat(spg, torch, args, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        v, desc, cores, dt = cpu_oracle_sample(A, f, args.ref_flops)
        v1, desc1, _, dt1 = cpu_oracle_sample(A, f, args.ref_flops / 16, threads=1)
        cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
               "seconds": dt,
               "single_thread": {"value": v1, "unit": UNIT, "cores": 1, "sample": desc1, "seconds": dt1}}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD if args.scale == 20 else
                       WORKLOAD.replace("scale 20 (1,048,576^2", f"scale {args.scale} ({1 << args.scale:,}^2"),
                       "flops_per_step": F, "nnz_c": info["nnz_c"],
                       "nbatches": info["nbatches"], "budget": "80% of free HBM",
                       "l2": "inputs and outputs larger than L2 (no flush needed)",
                       "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"},
            "roofline": {"bound": "hbm", "kernel": "k_num_heavy32 (heavy-column numeric: dense row panels + hash row ranges)",
                         "achieved": achieved, "peak": hbm, "peak_kind": peak_kind, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "algorithmic_bytes_per_launch": bytes_per_launch,
                         "launch_ms": dense_ms, "dense_columns": ndense},
            "phase_ms_per_step": phase_ms,
            "gpu_launches": stats["launches"],
            "clocks": clocks,
            "e2e": e2e,
            "ksplit4": ks,
            "cpu_baseline": cpu,
        }
        line.update(extras)
        if extras:
            line["configs"] = configs_summary(line)
        print(json.dumps(line))


def configs_summary(line):
    """One entry per benchmark configuration (the five workloads the
    benchmark is specified on), with the GPU figure, its roofline where the
    HBM bound applies, and the CPU oracle beside it."""
    def pick(d, *keys):
        return {k: d[k] for k in keys if d is not None and k in d}
    p = line.get("protein_2M") or {}
    return {
        "1_er4096_fp64": pick(line.get("er4096"), "us_per_product", "value", "unit", "cpu_baseline", "note"),
        "2_rmat20_fp32": {"value": line["value"], "unit": line["unit"], "ms_per_step": line["ms_per_step"],
                          "roofline": line["roofline"], "e2e": line.get("e2e"),
                          "ksplit4": line.get("ksplit4"), "cpu_baseline": line.get("cpu_baseline")},
        "3_protein2M_24GB": pick(p, "value", "unit", "ms_per_step", "nbatches", "roofline_numeric", "e2e",
                                 "cpu_baseline"),
        "4_batched512_int64": pick(line.get("batched_vs_plain"), "multi_gflops", "multi_ms", "plain_ms",
                                   "speedup", "cpu_baseline"),
        "5_fwdbwd": pick(line.get("fwdbwd_vs_plain"), "fused_ms", "plain_ms", "speedup", "cpu_baseline"),
    }


def bench_multi(spg, torch, args):
    """512 uneven G(n,p) products (int64 ones semiring): one CUDA-graph
    launch of the device-driven multi-problem pass vs 512 plain plans."""
    from paper_2010_08526_gb300 import autotune
    n = 512 if not args.small_extras else 64
    probs = W.config4(count=n, nmax=200000 if not args.small_extras else 20000)
    dev = [spg.Csc.from_host(p) for p in probs]
    flops = sum(int(flops_host(p).sum()) for p in probs)
    # table caps (CTA / warp) and CTA width of the persistent passes picked by
    # the autotuner over its grid, on the first 64 problems
    best, trials = autotune.tune_multi(dev[:64], dev[:64], autotune.multi_candidates(), reps=2)
    M = spg.Multi(dev, dev, tuning=best)
    M.run(use_graph=True)
    torch.cuda.synchronize()
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        M.run(use_graph=True)
    torch.cuda.synchronize()
    t_multi = (time.perf_counter() - t0) / reps
    M.close()
    torch.cuda.empty_cache()

    # the per-matrix path with its plans and outputs made once and reused:
    # every call redoes symbolic (one host synchronisation) and numeric
    plans = [spg.Plan(d, d) for d in dev]
    outs = []
    for p in plans:
        p.symbolic()
        outs.append([p.alloc_batch(t) for t in range(p.nbatches)])

    def plain():
        for p, o in zip(plans, outs):
            p.symbolic()
            for t in range(p.nbatches):
                p.numeric(t, out=o[t])
    plain()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain()
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    for p in plans:
        p.close()
    del outs, plans
    torch.cuda.empty_cache()
    r = {"problems": n, "flops": flops, "multi_ms": t_multi * 1e3, "plain_ms": t_plain * 1e3,
         "speedup": t_plain / t_multi, "multi_gflops": 2 * flops / t_multi / 1e9,
         "launches_per_run": "flop count, tier binning, 1 symbolic pass, 3-kernel scan, 1 numeric pass",
         "plain_path": "512 plans made once and reused: symbolic + numeric per product per run",
         "tuning": autotune.describe([(best, 0.0)])[0], "autotune_trials": autotune.describe(trials)}
    if not args.no_cpu:
        import oracle
        sample = probs[:48]
        sf = sum(int(flops_host(p).sum()) for p in sample)
        t0 = time.perf_counter()
        for p in sample:
            oracle.spgemm(p, p)
        dt = time.perf_counter() - t0
        r["cpu_baseline"] = {"value": 2 * sf / dt / 1e9, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "seconds": dt,
                             "sample": f"the first {len(sample)} of the {n} problems ({sf:.3e} multiplies), "
                                       "int64 path counts"}
    return r


def bench_step(spg, torch, args, A, dev, note, B=None, **plan_kw):
    """Device time of one symbolic + numeric step of A*B (B = A by default)
    with plan options."""
    st = torch.cuda.current_stream()
    Ad = spg.Csc.from_host(A, device=f"cuda:{dev}")
    Bd = Ad if B is None else spg.Csc.from_host(B, device=f"cuda:{dev}")
    plan = spg.Plan(Ad, Bd, **plan_kw)
    plan.set_timing(True)
    info = plan.symbolic()
    outs = [plan.alloc_batch(t) for t in range(plan.nbatches)]

    def step():
        plan.symbolic()
        for t in range(plan.nbatches):
            plan.numeric(t, out=outs[t])
    step()
    torch.cuda.synchronize()
    plan.stats(reset=True)
    n = max(1, min(args.steps, 3))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(n):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    stats = plan.stats(reset=True)
    plan.check_errors()
    cnt = plan.column_counts().cpu().numpy()
    del outs
    plan.close()
    torch.cuda.empty_cache()
    F = int(info["flops"])
    r = {"value": 2 * F / (ms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": ms, "flops_per_step": F,
         "nnz_c": int(info["nnz_c"]), "nbatches": int(info["nbatches"]),
         "phase_ms_per_step": {k: round(v / n, 3) for k, v in stats["ms"].items() if v},
         "note": note, "_counts": cnt}
    if plan_kw.get("kstages", 1) > 1:
        r["unmerged_nnz"] = int(info["unmerged_nnz"])
        r["stage_buffer_nnz"] = int(info["stage_buffer_nnz"])
    return r


def bench_kmerge(spg, torch, args, A, dev):
    """The k-split's two ways of summing the stage partials: merge at the end
    (the paper's choice) against the incremental merge M_t = M_{t-1} + D_t.
    On the headline product (4 stages), and on a saturated product where
    every stage partial already fills most of C (8 stages): A 2048 x 262144
    with 8 uniform rows per column, B 262144 x 16384 with 2048."""
    out = {"rmat20_s4": bench_step(spg, torch, args, A, dev, kstages=4, merge="incremental",
                                   note="incremental merge, headline product, 4 stages")}
    out["rmat20_s4"].pop("_counts")
    Ao = W.er_exact(2048, 262144, 8, 11, value_dtype=np.float32)
    Bo = W.er_exact(262144, 16384, 2048, 12, value_dtype=np.float32)
    for mode in ("end", "incremental"):
        r = bench_step(spg, torch, args, Ao, dev, B=Bo, kstages=8, merge=mode,
                       note=f"merge {mode}, saturated product, 8 stages")
        r.pop("_counts")
        out[f"overlap_s8_{mode}"] = r
    return out


def bench_protein(spg, torch, args, dev):
    """Config 3, the protein-similarity stand-in (2M x 2M, int64 indices,
    fp32, mean degree 40, compression ~1) at its 24 GB HBM output budget,
    which forces b >= 4 column batches: the device step (symbolic + every
    batch's numeric), the numeric phases against the HBM roofline, and the
    batch loop end to end (A from pinned host memory, every batch streamed to
    pinned host slots on a copy stream while the next one is computed)."""
    A = W.config3()
    budget = 24 << 30
    r = bench_step(spg, torch, args, A, dev, budget=budget,
                   note="C = A*A, protein-similarity stand-in, 2,000,000^2, lognormal degrees "
                        "(mean 40), int64 CSC, fp32; 24 GB budget")
    cnt = r.pop("_counts")
    r["budget_bytes"] = budget
    f = flops_host(A)
    nnzb = np.diff(A.colptr).astype(np.int64)
    si, sv = 8, 4
    model = float(nnzb.sum() * (si + sv + 2 * si) + f.sum() * (si + sv) + cnt.sum() * (si + sv))
    num_ms = sum(v for k, v in r["phase_ms_per_step"].items() if k.startswith("num_"))
    hbm, _ = peaks()
    achieved = model / (num_ms / 1e3) / 1e9 if num_ms else 0.0
    r["roofline_numeric"] = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                             "frac": achieved / hbm, "algorithmic_bytes": model, "numeric_ms": num_ms}
    # end to end through the batch loop, at the same budget
    F = int(f.sum())
    hostA = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in (A.colptr, A.rowidx, A.vals)]
    dA = spg.Csc(A.nrows, A.ncols, *[torch.empty_like(h, device=f"cuda:{dev}") for h in hostA])
    eplan = spg.Plan(dA, dA, budget=budget, host_slot_bytes=1 << 30, host_slots=4)
    cs = torch.cuda.Stream()
    got = {"bytes": 0}

    def sink(batch, c0, c1, arrs):
        cp, ri, va = arrs
        got["bytes"] += cp.nbytes + ri.nbytes + va.nbytes
        return 0

    def estep():
        for h, d in zip(hostA, (dA.colptr, dA.rowidx, dA.vals)):
            d.copy_(h, non_blocking=True)
        eplan.symbolic()
        got["bytes"] = 0
        spg.run_batched(eplan, sink, copy=cs)
        return got["bytes"]
    estep()
    torch.cuda.synchronize()
    n = max(1, min(args.steps, 2))
    t0 = time.perf_counter()
    bo = 0
    for _ in range(n):
        bo = estep()
    torch.cuda.synchronize()
    edt = (time.perf_counter() - t0) / n
    einfo = eplan.query()
    eplan.close()
    del dA
    torch.cuda.empty_cache()
    r["e2e"] = {"value": 2 * F / edt / 1e9, "unit": UNIT, "ms_per_step": edt * 1e3,
                "nbatches": int(einfo["nbatches"]),
                "h2d_bytes_per_step": sum(h.numel() * h.element_size() for h in hostA),
                "d2h_bytes_per_step": bo, "d2h_gbs": bo / edt / 1e9,
                "note": "A copied from pinned host memory, symbolic, then every batch streamed to "
                        "pinned host slots by spgemm_run_batched"}
    # the hybrid accumulator on the same product: CTA-tier columns whose
    # products fit their table are sorted by row instead of hashed
    h = bench_step(spg, torch, args, A, dev, budget=budget, tuning=spg.Tuning(hybrid_sort=True),
                   note="hybrid accumulator (sort-based for low-cf CTA-tier columns)")
    h.pop("_counts")
    r["hybrid_sort"] = {k: h[k] for k in ("value", "unit", "ms_per_step", "phase_ms_per_step", "note")}
    if not args.no_cpu:
        v, desc, cores, dt = cpu_oracle_sample(A, f, 4e9)
        r["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
                             "seconds": dt}
    return r


def bench_config1(spg, torch, args, dev):
    """Config 1: C = A*A for a 4,096^2 Erdos-Renyi matrix with exactly 8 rows
    per column, fp64, int32 -- a latency case (the inputs fit in L2): one
    plain single-batch symbolic + numeric, in microseconds per product."""
    A = W.config1()
    st = torch.cuda.current_stream()
    Ad = spg.Csc.from_host(A, device=f"cuda:{dev}")
    plan = spg.Plan(Ad, Ad)
    info = plan.symbolic()
    out = plan.alloc_batch(0)

    def step():
        plan.symbolic()
        plan.numeric(0, out=out)
    for _ in range(5):
        step()
    torch.cuda.synchronize()
    n = 50
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(n):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    us = e0.elapsed_time(e1) / n * 1e3
    plan.check_errors()
    plan.close()
    F = int(info["flops"])
    r = {"us_per_product": us, "value": 2 * F / (us / 1e6) / 1e9, "unit": UNIT, "flops": F,
         "nnz_c": int(info["nnz_c"]), "nbatches": int(info["nbatches"]),
         "note": "symbolic (one host synchronisation) + numeric; inputs fit in L2, so the HBM "
                 "roofline does not apply"}
    if not args.no_cpu:
        import oracle
        t0 = time.perf_counter()
        for _ in range(5):
            oracle.spgemm(A, A)
        dt = (time.perf_counter() - t0) / 5
        r["cpu_baseline"] = {"value": 2 * F / dt / 1e9, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "us_per_product": dt * 1e6,
                             "sample": "the whole product, 5 runs"}
    return r


def bench_aat(spg, torch, args, dev):
    """A*A^T and row-wise batching on a k-mer-like matrix (2 nonzeros per
    column, the Rice-kmers shape the paper's A*A^T runs use): A 1,000,000 x
    4,000,000, fp32, int32. The transpose, the product, and the row-batched
    stream of C (column batches of C^T = A A^T, handed over as rows)."""
    import oracle  # noqa: F401  (inputs only)
    A = W.er_exact(1_000_000, 4_000_000, 2, W.config_seed(6), index_dtype=np.int32,
                   value_dtype=np.float32)
    Ad = spg.Csc.from_host(A, device=f"cuda:{dev}")
    st = torch.cuda.current_stream()
    spg.spgemm_aat(Ad)
    torch.cuda.synchronize()
    n = 3
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(n):
        C = spg.spgemm_aat(Ad)
        del C
    e1.record(st)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / n
    F = 4 * A.ncols   # every column of A (2 entries) gives 4 products of A A^T
    rows = {"blocks": 0}

    def sink(batch, r0, r1, arrs):
        rows["blocks"] += 1
        return 0
    At = spg.transpose(Ad, ptr_dtype=Ad.colptr.dtype)
    budget = (A.bytes() * 6) + (256 << 20)
    t0 = time.perf_counter()
    spg.run_row_batched(Ad, At, sink, budget=budget, host_slot_bytes=1 << 28, host_slots=3)
    torch.cuda.synchronize()
    rb = time.perf_counter() - t0
    del At, Ad
    torch.cuda.empty_cache()
    return {"value": 2 * F / (ms / 1e3) / 1e9, "unit": UNIT, "ms_per_product": ms, "flops": F,
            "row_batched_ms": rb * 1e3, "row_blocks": rows["blocks"],
            "note": "A*A^T (device transpose + product) and the same product streamed by row blocks"}


def bench_sorted_topk(spg, torch, args, A, F, dev, topk=1000):
    """The paper's final form of C (rows sorted in every column, Sec. IV-D) on
    the device, and the batch consumer of Sec. III / V-F end to end: every
    batch sorted and pruned to its topk largest entries per column on the
    device before the copy to pinned host memory."""
    st = torch.cuda.current_stream()
    Ad = spg.Csc.from_host(A, device=f"cuda:{dev}")
    plan = spg.Plan(Ad, Ad, sort_output=True)
    plan.symbolic()
    outs = [plan.alloc_batch(t) for t in range(plan.nbatches)]

    def step():
        plan.symbolic()
        for t in range(plan.nbatches):
            plan.numeric(t, out=outs[t])
    step()
    torch.cuda.synchronize()
    n = max(1, min(args.steps, 3))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(n):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    sms = e0.elapsed_time(e1) / n
    plan.check_errors()
    del outs
    plan.close()
    torch.cuda.empty_cache()

    hostA = [torch.from_numpy(np.ascontiguousarray(x)).pin_memory() for x in (A.colptr, A.rowidx, A.vals)]
    # pruned batches copy little, so the default budget (fewest batches) fits
    eplan = spg.Plan(Ad, Ad, host_slot_bytes=1 << 30, host_slots=4, sort_output=True,
                     prune=(float("-inf"), topk))
    cs = torch.cuda.Stream()
    got = {"bytes": 0, "nnz": 0}

    def sink(batch, c0, c1, arrs):
        cp, ri, va = arrs
        got["bytes"] += cp.nbytes + ri.nbytes + va.nbytes
        got["nnz"] += int(va.size)
        return 0

    def estep():
        for h, d in zip(hostA, (Ad.colptr, Ad.rowidx, Ad.vals)):
            d.copy_(h, non_blocking=True)
        eplan.symbolic()
        got["bytes"] = got["nnz"] = 0
        spg.run_batched(eplan, sink, copy=cs)
    estep()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n):
        estep()
    torch.cuda.synchronize()
    edt = (time.perf_counter() - t0) / n
    info = eplan.query()
    eplan.close()
    torch.cuda.empty_cache()
    return {
        "sorted_device": {"value": 2 * F / (sms / 1e3) / 1e9, "unit": UNIT, "ms_per_step": sms,
                          "note": "symbolic + numeric with rows sorted in every column"},
        "e2e_topk": {"value": 2 * F / edt / 1e9, "unit": UNIT, "ms_per_step": edt * 1e3, "topk": topk,
                     "kept_nnz": got["nnz"], "d2h_bytes_per_step": got["bytes"],
                     "h2d_bytes_per_step": sum(h.numel() * h.element_size() for h in hostA),
                     "nbatches": info["nbatches"],
                     "note": "each batch sorted and pruned to its top-k per column on the device, "
                             "then streamed to pinned host memory"},
    }


def bench_fwdbwd(spg, torch, args):
    """Forward + masked backward (SpGEMMFn) vs gradients formed by plain
    SpGEMMs G*B^T and A^T*G on explicit transposes, masked afterwards."""
    import oracle  # noqa: F401  (not used: inputs only)
    from workloads.csc import transpose
    A, B = W.config5()
    Ad, Bd = spg.Csc.from_host(A), spg.Csc.from_host(B)
    At, Bt = spg.Csc.from_host(transpose(A)), spg.Csc.from_host(transpose(B))
    # G: N(0,1) values on C's pattern (seeded), the same for both paths
    gen = torch.Generator(device=Ad.vals.device)
    gen.manual_seed(W.config_seed(5))
    nnz_c = spg.spgemm(Ad, Bd, ptr_dtype=torch.int32).nnz
    gvals = torch.randn(nnz_c, generator=gen, device=Ad.vals.device, dtype=Ad.vals.dtype)

    def fused():
        a = Ad.vals.detach().clone().requires_grad_(True)
        b = Bd.vals.detach().clone().requires_grad_(True)
        c = spg.SpGEMMFn.apply(a, b, Ad, Bd)
        c.backward(gvals)
        return a.grad, b.grad

    def plain():
        C = spg.spgemm(Ad, Bd, ptr_dtype=torch.int32)
        G = spg.Csc(C.nrows, C.ncols, C.colptr, C.rowidx, gvals)
        gb = spg.spgemm(G, Bt)          # G * B^T  (m x k), masked to pattern(A) by the caller
        ag = spg.spgemm(At, G)          # A^T * G  (k x n), masked to pattern(B)
        return gb, ag

    for fn in (fused, plain):
        fn()
    torch.cuda.synchronize()
    reps = 5
    t0 = time.perf_counter()
    for _ in range(reps):
        fused()
    torch.cuda.synchronize()
    tf = (time.perf_counter() - t0) / reps
    t0 = time.perf_counter()
    for _ in range(reps):
        plain()
    torch.cuda.synchronize()
    tp = (time.perf_counter() - t0) / reps
    r = {"fused_ms": tf * 1e3, "plain_ms": tp * 1e3, "speedup": tp / tf,
         "flops_forward": int(flops_host_ab(A, B).sum()),
         "note": "plain path = forward SpGEMM + two full SpGEMMs on transposes (mask not applied); "
                 "G = N(0,1) values on C's pattern"}
    if not args.no_cpu:
        import oracle
        t0 = time.perf_counter()
        Cr = oracle.spgemm(A, B)
        G = W.values_on_pattern(Cr, 5, dist="normal", value_dtype=np.float32)
        t1 = time.perf_counter()
        oracle.backward(A, B, G)
        t2 = time.perf_counter()
        r["cpu_baseline"] = {"fwd_bwd_ms": (t1 - t0 + t2 - t1) * 1e3, "fwd_ms": (t1 - t0) * 1e3,
                             "bwd_ms": (t2 - t1) * 1e3, "cores": oracle.num_threads(), "kind": "oracle",
                             "speedup_of_fused": (t2 - t0) / tf,
                             "sample": "the whole forward product and both gradients (the backward "
                                       "oracle runs on one thread)"}
    return r


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--quick", action="store_true", help="skip the k-split and extra sections")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--small-extras", action="store_true")
    ap.add_argument("--scale", type=int, default=20,
                    help="R-MAT scale of the timed product (profiling small cases; the "
                         "benchmark workload is 20; other scales imply --quick --no-e2e --no-cpu)")
    ap.add_argument("--ref-flops", type=float, default=1.2e10,
                    help="multiplications in the CPU oracle sample")
    args = ap.parse_args()
    if args.scale != 20:
        args.quick = args.no_e2e = args.no_cpu = True
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
