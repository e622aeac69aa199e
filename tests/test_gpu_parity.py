"""Parity of the CUDA path with the CPU oracle, element by element.

Every test here calls the sm_103a library through its C ABI (via the thin
Python binding) and compares with the oracle on the same seeded inputs:
structure and per-column nnz bit-exact after the canonical per-column sort,
integers bit-exact, floats within the stated tolerance (tests/helpers.py).
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads as W
from workloads.csc import CSC, from_coo, shuffle_within_columns, column_slice

from helpers import assert_matches, host_csc, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

import paper_2010_08526_gb300 as spg  # noqa: E402


def run(A: CSC, B: CSC, **kw):
    Ad, Bd = to_dev(A), to_dev(B)
    C = spg.spgemm(Ad, Bd, validate=True, **kw)
    torch.cuda.synchronize()
    return host_csc(C), C.plan_info


def check_product(A, B, label, **kw):
    got, info = run(A, B, **kw)
    ref, ab, nt = oracle.spgemm(A, B, with_absterm=True, with_nterm=True)
    f = oracle.flops_per_column(A, B)
    assert info["flops"] == int(f.sum()), f"{label}: flops"
    assert info["nnz_c"] == ref.nnz, f"{label}: nnz"
    assert_matches(got, ref, ab, nt, label=label)
    return info


def rand_csc(m, n, density, seed, vals="normal", index_dtype=np.int32, value_dtype=np.float64):
    rng = np.random.default_rng(seed)
    nnz = int(m * n * density)
    r = rng.integers(0, m, nnz)
    c = rng.integers(0, n, nnz)
    if vals == "normal":
        v = rng.standard_normal(nnz)
    elif vals == "ones":
        v = np.ones(nnz, dtype=np.int64)
    else:
        v = rng.integers(-4, 5, nnz).astype(np.int64)
    a = from_coo(m, n, r, c, v, dup="sum", index_dtype=index_dtype,
                 value_dtype=value_dtype if vals == "normal" else np.int64)
    return shuffle_within_columns(a, seed + 3)


def skewed(m, n, seed, hubs=3, hub_deg=None, base=4, index_dtype=np.int32, value_dtype=np.float64,
           dist="normal"):
    """Random columns plus a few hub rows/columns, so that every tier appears."""
    rng = np.random.default_rng(seed)
    hub_deg = hub_deg or max(1, m // 3)
    rows, cols = [], []
    counts = rng.integers(0, base * 2 + 1, n)
    for j in range(n):
        rows.append(rng.choice(m, size=min(m, int(counts[j])), replace=False))
        cols.append(np.full(rows[-1].size, j))
    for h in range(hubs):
        j = int(rng.integers(0, n))
        r = rng.choice(m, size=min(m, hub_deg), replace=False)
        rows.append(r); cols.append(np.full(r.size, j))
        i = int(rng.integers(0, m))
        c = rng.choice(n, size=min(n, hub_deg), replace=False)
        rows.append(np.full(c.size, i)); cols.append(c)
    r = np.concatenate(rows); c = np.concatenate(cols)
    if dist == "normal":
        v = rng.standard_normal(r.size)
    else:
        v = np.ones(r.size, dtype=np.int64)
    a = from_coo(m, n, r, c, v, dup="max", index_dtype=index_dtype,
                 value_dtype=value_dtype if dist == "normal" else np.int64)
    return shuffle_within_columns(a, seed + 1)


# ------------------------------------------------------------------ plain path

def test_config1_full_size_fp64():
    A = W.config1()
    info = check_product(A, A, "config1")
    assert info["nbatches"] == 1


@pytest.mark.parametrize("vt", [np.float64, np.float32, np.int64])
@pytest.mark.parametrize("it", [np.int32, np.int64])
def test_types_small(vt, it):
    dist = "normal" if vt != np.int64 else "int"
    A = rand_csc(300, 257, 0.03, 5, vals=dist, index_dtype=it, value_dtype=vt)
    B = rand_csc(257, 301, 0.03, 6, vals=dist, index_dtype=it, value_dtype=vt)
    check_product(A, B, f"types {vt.__name__} {it.__name__}")


@pytest.mark.parametrize("cap", [256, 1024, 8192])
def test_all_tiers_and_heavy_path(cap):
    """Skewed matrix: warp, block and heavy tiers in one product; a small
    hash cap and small panels push many columns through the dense path."""
    A = skewed(6000, 6000, 11, hubs=4, hub_deg=2500, base=6)
    tun = spg.Tuning(hash_max_cap=cap, panel_rows=1024)
    info = check_product(A, A, f"tiers cap={cap}", tuning=tun)
    if cap == 256:
        assert info["heavy_columns"] > 0


def test_heavy_path_symbolic_panels():
    """More rows than one symbolic bitmap panel with tiny numeric panels."""
    A = skewed(3000, 2000, 12, hubs=3, hub_deg=1500, base=3)
    B = skewed(2000, 500, 13, hubs=2, hub_deg=1000, base=8)
    tun = spg.Tuning(hash_max_cap=256, panel_rows=1024)
    check_product(A, B, "rect heavy", tuning=tun)


@pytest.mark.parametrize("vt", [np.float32, np.int64])
def test_heavy_types(vt):
    dist = "normal" if vt != np.int64 else "ones"
    A = skewed(5000, 5000, 21, hubs=3, hub_deg=2000, base=5, value_dtype=vt, dist=dist,
               index_dtype=np.int64)
    tun = spg.Tuning(hash_max_cap=512, panel_rows=2048)
    check_product(A, A, f"heavy {vt.__name__}", tuning=tun)


@pytest.mark.parametrize("vt", [np.float32, np.float64, np.int64])
def test_heavy_dense_items_with_cancelling_sums(vt):
    """Dense row-panel items whose sums cancel to exactly zero, and explicit
    zero entries: the structural nonzeros of C include entries whose value is
    0 (every (i, j) reached by a product is kept), so these items cannot be
    compacted by value; the exact per-panel counts decide. Values in
    {-1, 0, 1}: every sum is an exact integer in any order."""
    rng = np.random.default_rng(61)
    A = skewed(4000, 4000, 62, hubs=4, hub_deg=3000, base=6, index_dtype=np.int32)
    vals = rng.choice(np.array([-1.0, 1.0, 1.0, -1.0, 0.0]), A.nnz)
    A = CSC(A.nrows, A.ncols, A.colptr, A.rowidx, vals.astype(vt))
    tun = spg.Tuning(hash_max_cap=256, panel_rows=1024)
    got, info = run(A, A, tuning=tun)
    assert info["heavy_columns"] > 0
    ref = oracle.spgemm(A, A)
    assert int((np.asarray(ref.vals) == 0).sum()) > 1000   # many exact zeros are structural
    assert_matches(got, ref, exact=True, label=f"cancelling heavy {np.dtype(vt).name}")
    # all-zero values: every entry of C is structural and zero
    Z = CSC(A.nrows, A.ncols, A.colptr, A.rowidx, np.zeros(A.nnz, vt))
    gz, _ = run(Z, Z, tuning=tun)
    rz = oracle.spgemm(Z, Z)
    assert_matches(gz, rz, exact=True, label="all-zero heavy")


def test_tuning_variants():
    A = skewed(4000, 3000, 31, hubs=2, hub_deg=1500)
    B = skewed(3000, 3500, 32, hubs=2, hub_deg=1200)
    for tun in [spg.Tuning(short_seg=1), spg.Tuning(short_seg=64, huge_seg=64),
                spg.Tuning(block_tier_threads=128), spg.Tuning(block_tier_threads=1024)]:
        check_product(A, B, f"tuning {tun}", tuning=tun)


def test_edge_cases():
    # empty product
    Z = CSC(5, 4, np.zeros(5, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B = CSC(4, 3, np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0))
    got, info = run(Z, B)
    assert info["nnz_c"] == 0 and got.nnz == 0 and got.ncols == 3
    # 1x1
    A1 = from_coo(1, 1, [0], [0], [3.0])
    check_product(A1, A1, "1x1")
    # identity and empty columns
    A = rand_csc(200, 200, 0.02, 41)
    I = from_coo(200, 200, np.arange(200), np.arange(200), np.ones(200))
    check_product(A, I, "A*I")
    check_product(I, A, "I*A")
    # zero-sum cancellation stays structural
    Ac = from_coo(2, 2, [0, 1, 0, 1], [0, 0, 1, 1], [1.0, 1.0, 1.0, -1.0])
    Bc = from_coo(2, 1, [0, 1], [0, 0], [1.0, 1.0])
    got, _ = run(Ac, Bc)
    assert got.nnz == 2
    # large row indices (sparse rows near the top of the 32-bit key range)
    rng = np.random.default_rng(7)
    m = 1 << 26
    r = rng.integers(m - 5000, m, 3000)
    c = rng.integers(0, 300, 3000)
    Ab = from_coo(m, 300, r, c, rng.standard_normal(3000), dup="sum")
    Bb = rand_csc(300, 50, 0.05, 8)
    check_product(Ab, Bb, "large rows")


@pytest.mark.parametrize("heavy", [False, True])
def test_int64_rows_at_the_top_of_the_key_range(heavy):
    """int64 indices with A's rows up to 2^31 - 2, the largest row the header
    allows (the hash keys are 32-bit and 0xffffffff marks an empty slot).
    The oracle's dense accumulator cannot span 2^31 rows, so it runs on A with
    its occupied rows relabelled 0..u-1 in order; relabelling the rows of A
    relabels the rows of C = A*B and changes nothing else."""
    rng = np.random.default_rng(17)
    m = (1 << 31) - 1
    k, n = 400, 300
    top = np.arange(m - 6000, m, dtype=np.int64)          # ..., 2^31 - 2
    pool = np.concatenate([top, rng.integers(0, m - 6000, 2000), [0, 1, (1 << 30), (1 << 31) - 3]])
    nnz = 6000
    r = rng.choice(pool, nnz)
    c = rng.integers(0, k, nnz)
    if heavy:   # a few dense columns of A reach the heavy tier
        hub = rng.choice(top, 3000, replace=False)
        r = np.concatenate([r, hub, hub[:2500]])
        c = np.concatenate([c, np.full(3000, 7), np.full(2500, 11)])
    r = np.concatenate([r, [m - 1, m - 1, m - 2]])       # row 2^31 - 2 present
    c = np.concatenate([c, [0, 5, 5]])
    A = from_coo(m, k, r, c, rng.standard_normal(r.size), dup="sum", index_dtype=np.int64)
    B = rand_csc(k, n, 0.05, 18, index_dtype=np.int64)
    assert int(A.rowidx.max()) == (1 << 31) - 2
    kw = {"tuning": spg.Tuning(hash_max_cap=256)} if heavy else {}
    got, info = run(A, B, **kw)
    if heavy:
        assert info["heavy_columns"] > 0
    # oracle on the relabelled rows
    uniq, inv = np.unique(np.asarray(A.rowidx, np.int64), return_inverse=True)
    Ac = CSC(uniq.size, k, A.colptr.astype(np.int64), inv.astype(np.int64), A.vals)
    ref, ab, nt = oracle.spgemm(Ac, B, with_absterm=True, with_nterm=True)
    ref = CSC(m, n, ref.colptr, uniq[ref.rowidx], ref.vals)
    assert_matches(got, ref, ab, nt, label=f"rows near 2^31 heavy={heavy}")


@pytest.mark.parametrize("kst,merge", [(2, "end"), (3, "incremental"), (5, "incremental"), (2, "incremental")])
def test_edge_cases_with_stages(kst, merge):
    """The degenerate inputs through the k-split, both merge modes: stages
    with no entries, more stages than some columns have entries, and the
    running sums' buffers at their smallest."""
    Z = CSC(5, 4, np.zeros(5, np.int32), np.zeros(0, np.int32), np.zeros(0))
    B = CSC(4, 3, np.zeros(4, np.int32), np.zeros(0, np.int32), np.zeros(0))
    got, info = run(Z, B, kstages=kst, merge=merge)
    assert info["nnz_c"] == 0 and got.nnz == 0 and got.ncols == 3
    A1 = from_coo(1, 1, [0], [0], [3.0])
    check_product(A1, A1, f"1x1 s={kst} {merge}", kstages=kst, merge=merge)
    A = rand_csc(200, 200, 0.02, 41)
    I = from_coo(200, 200, np.arange(200), np.arange(200), np.ones(200))
    check_product(A, I, f"A*I s={kst} {merge}", kstages=kst, merge=merge)
    check_product(I, A, f"I*A s={kst} {merge}", kstages=kst, merge=merge)
    # B with empty columns and a k smaller than the number of stages
    Ak = rand_csc(300, 3, 0.5, 42)
    Bk = from_coo(3, 6, [0, 2, 1], [0, 0, 4], [1.0, -2.0, 0.5])
    check_product(Ak, Bk, f"k=3 s={kst} {merge}", kstages=kst, merge=merge)


def test_hybrid_with_int64_indices():
    """The sort-based accumulator with 64-bit indices (rows < 2^31 as keys)."""
    A = W.er_exact(6000, 6000, 40, 17, index_dtype=np.int64)
    check_product(A, A, "hybrid int64 indices", tuning=spg.Tuning(hybrid_sort=True))


def test_row_order_invariance_on_gpu():
    A = W.config1(n=1024)
    A2 = shuffle_within_columns(A, 99)
    g1, _ = run(A, A)
    g2, _ = run(A2, A2)
    c1, c2 = oracle.canonical(g1), oracle.canonical(g2)
    assert np.array_equal(c1.rowidx, c2.rowidx)
    np.testing.assert_allclose(c1.vals, c2.vals, rtol=1e-12)


def test_symbolic_counts_and_invalid_inputs():
    A = rand_csc(500, 400, 0.01, 51)
    B = rand_csc(400, 450, 0.01, 52)
    plan = spg.Plan(to_dev(A), to_dev(B))
    info = plan.symbolic()
    cnt = plan.column_counts().cpu().numpy()
    assert np.array_equal(cnt, oracle.symbolic(A, B))
    assert info["flops"] == int(oracle.flops_per_column(A, B).sum())
    plan.check_errors()
    plan.close()
    # corrupt column pointers are rejected by validation
    bad = CSC(A.nrows, A.ncols, A.colptr.copy(), A.rowidx.copy(), A.vals.copy())
    bad.colptr[5] = bad.colptr[6] + 1
    with pytest.raises(spg.SpgemmError):
        spg.Plan(to_dev(bad), to_dev(B), validate=True)
    badr = CSC(A.nrows, A.ncols, A.colptr.copy(), A.rowidx.copy(), A.vals.copy())
    badr.rowidx[3] = A.nrows + 5
    with pytest.raises(spg.SpgemmError):
        spg.Plan(to_dev(badr), to_dev(B), validate=True)
    # shape mismatch
    with pytest.raises(spg.SpgemmError):
        spg.Plan(to_dev(A), to_dev(A))


# --------------------------------------------------------------- k-split + merge

@pytest.mark.parametrize("s", [2, 3, 4, 7])
def test_ksplit_merge_equals_unsplit(s):
    A = skewed(3000, 3000, 61, hubs=3, hub_deg=1200)
    info = check_product(A, A, f"ksplit s={s}", kstages=s)
    parts = [oracle.spgemm(A, A, krange=kr) for kr in oracle.stage_ranges(3000, s)]
    assert info["unmerged_nnz"] == sum(p.nnz for p in parts)
    assert info["flops"] >= info["unmerged_nnz"] >= info["nnz_c"]   # Eq. (1)


def test_repeated_symbolic_keeps_the_batch_plan():
    A = skewed(3000, 3000, 63, hubs=3, hub_deg=1200)
    Ad = to_dev(A)
    ref = oracle.spgemm(A, A)
    for kst in (1, 3):
        plan = spg.Plan(Ad, Ad, kstages=kst, budget=A.bytes() * 2 + (1 << 20) + ref.nnz * 12)
        first = [plan.batch(t) for t in range(plan.symbolic()["nbatches"])]
        outs = [plan.alloc_batch(t) for t in range(len(first))]
        for _ in range(2):
            info = plan.symbolic()
            assert [plan.batch(t) for t in range(info["nbatches"])] == first
            for t in range(len(first)):
                plan.numeric(t, out=outs[t])
        plan.check_errors()
        plan.close()


@pytest.mark.parametrize("vt", [np.float32, np.int64])
def test_ksplit_heavy_dense_merge(vt):
    dist = "normal" if vt != np.int64 else "ones"
    A = skewed(5000, 5000, 71, hubs=4, hub_deg=2500, base=6, value_dtype=vt, dist=dist)
    tun = spg.Tuning(hash_max_cap=256, panel_rows=1024)
    check_product(A, A, f"ksplit heavy {vt.__name__}", kstages=4, tuning=tun)


# ------------------------------------------- incremental (per-stage) merge

def _stage_nnz(A, B, s):
    """Oracle counts: nnz(D_t) per stage and nnz(M_u) of the running sums
    M_u = D_0 + ... + D_u (the product over k in [0, k1_u))."""
    kr = oracle.stage_ranges(A.ncols, s)
    d = [int(oracle.symbolic(A, B, krange=r).sum()) for r in kr]
    m = [int(oracle.symbolic(A, B, krange=(0, r[1])).sum()) for r in kr]
    return d, m


@pytest.mark.parametrize("s", [2, 3, 4, 7])
def test_incremental_merge_equals_unsplit(s):
    """merge="incremental" sums the stages as they come (M_t = M_{t-1} + D_t)
    and must give the unsplit product; one batch holds the largest D_t
    (t >= 1) plus one or two running sums sized by the largest M_u, u <= s-2."""
    A = skewed(3000, 3000, 61, hubs=3, hub_deg=1200)
    info = check_product(A, A, f"incremental s={s}", kstages=s, merge="incremental")
    d, m = _stage_nnz(A, A, s)
    assert info["unmerged_nnz"] == sum(d)
    assert m[-1] == info["nnz_c"]
    assert info["nbatches"] == 1
    runs = [d[0]] + m[1:s - 1]
    assert info["stage_buffer_nnz"] == max(d[1:]) + (2 if s > 2 else 1) * max(runs)


@pytest.mark.parametrize("vt,it", [(np.float32, np.int32), (np.int64, np.int32), (np.float64, np.int64)])
def test_incremental_heavy_dense_merge(vt, it):
    """Heavy columns: the stage partials and the running sums are grouped by
    the heavy items' panel ranges; dense-panel and hash-range merge items."""
    dist = "normal" if vt != np.int64 else "ones"
    A = skewed(5000, 5000, 71, hubs=4, hub_deg=2500, base=6, index_dtype=it, value_dtype=vt, dist=dist)
    tun = spg.Tuning(hash_max_cap=256, panel_rows=1024)
    info = check_product(A, A, f"incremental heavy {vt.__name__} {it.__name__}", kstages=4, tuning=tun,
                         merge="incremental")
    assert info["heavy_columns"] > 0


def _overlapping(m=240, k=3200, n=240, seed=5):
    """Every stage partial is already most of C (cf high): 10 entries per
    column of A, 160 per column of B, so D_t fills ~2/3 of each column."""
    rng = np.random.default_rng(seed)
    ra = np.concatenate([rng.choice(m, 10, replace=False) for _ in range(k)])
    A = from_coo(m, k, ra, np.repeat(np.arange(k), 10), rng.standard_normal(ra.size))
    rb = np.concatenate([rng.choice(k, 160, replace=False) for _ in range(n)])
    B = from_coo(k, n, rb, np.repeat(np.arange(n), 160), rng.standard_normal(rb.size))
    return shuffle_within_columns(A, seed + 1), shuffle_within_columns(B, seed + 2)


def test_incremental_merge_needs_less_memory_when_stages_overlap():
    A, B = _overlapping()
    s = 8
    end = check_product(A, B, "overlap end", kstages=s)
    inc = check_product(A, B, "overlap incremental", kstages=s, merge="incremental")
    d, m = _stage_nnz(A, B, s)
    assert end["stage_buffer_nnz"] == sum(d)
    assert inc["stage_buffer_nnz"] == max(d[1:]) + 2 * max([d[0]] + m[1:s - 1])
    assert inc["stage_buffer_nnz"] < 0.6 * end["stage_buffer_nnz"]
    # a budget whose batch cap (half of what the inputs and the workspace
    # leave, two batches in flight) just holds C plus the incremental buffers
    # in one batch: the s partials do not fit, so merging at the end needs
    # more batches
    Ad, Bd = to_dev(A), to_dev(B)
    big = 1 << 30
    probe = spg.Plan(Ad, Bd, budget=big, kstages=s, merge="incremental")
    cap0 = probe.symbolic()["batch_cap_bytes"]
    probe.close()
    r = 12
    target = r * (inc["nnz_c"] + inc["stage_buffer_nnz"]) + 8 * (B.ncols + 1) + 4096
    budget = big - 2 * (cap0 - target)
    pe = spg.Plan(Ad, Bd, budget=budget, kstages=s)
    pi = spg.Plan(Ad, Bd, budget=budget, kstages=s, merge="incremental")
    ne, ni = pe.symbolic()["nbatches"], pi.symbolic()["nbatches"]
    pe.close(); pi.close()
    assert ni == 1 and ne > 1, (ni, ne)


@pytest.mark.parametrize("kst", [3, 5])
def test_incremental_merge_over_batches(kst):
    """Several batches (budget-limited) through plan.numeric and run_batched."""
    A = skewed(4000, 4000, 83, hubs=3, hub_deg=1500, base=6)
    ref, ab, nt = oracle.spgemm(A, A, with_absterm=True, with_nterm=True)
    Ad = to_dev(A)
    tun = spg.Tuning(hash_max_cap=256, panel_rows=1024)
    budget = A.bytes() * 2 + (4 << 20) + ref.nnz * 12
    plan = spg.Plan(Ad, Ad, budget=budget, kstages=kst, tuning=tun, merge="incremental",
                    host_slot_bytes=1 << 16, host_slots=2)
    info = plan.symbolic()
    assert info["nbatches"] >= 2
    pieces = []

    def sink(batch, c0, c1, arrs):
        cp, ri, va = arrs
        pieces.append((c0, c1, cp.copy(), ri.copy(), va.copy()))
        return 0

    spg.run_batched(plan, sink)
    outs = [host_csc(plan.numeric(t)) for t in range(plan.nbatches)]
    torch.cuda.synchronize()
    plan.close()

    def assemble(chunks):
        colptr = [0]
        for cp in chunks[0]:
            colptr.extend((np.asarray(cp, np.int64)[1:] + colptr[-1]).tolist())
        return CSC(A.nrows, A.ncols, np.array(colptr, np.int64),
                   np.concatenate(chunks[1]).astype(np.int64), np.concatenate(chunks[2]))

    got = assemble(([p[2] for p in pieces], [p[3] for p in pieces], [p[4] for p in pieces]))
    assert pieces[0][0] == 0 and pieces[-1][1] == A.ncols
    assert_matches(got, ref, ab, nt, label=f"incremental run_batched s={kst}")
    got2 = assemble(([o.colptr for o in outs], [o.rowidx for o in outs], [o.vals for o in outs]))
    assert_matches(got2, ref, ab, nt, label=f"incremental numeric s={kst}")


def test_merge_api():
    parts = [rand_csc(700, 300, 0.02, 80 + t) for t in range(4)]
    M = spg.merge([to_dev(p) for p in parts])
    torch.cuda.synchronize()
    ref = oracle.merge(parts)
    # the scale of each merged entry's rounding is the sum of |part values|
    ab = oracle.merge([CSC(p.nrows, p.ncols, p.colptr, p.rowidx, np.abs(p.vals)) for p in parts]).vals
    assert_matches(host_csc(M), ref, ab, label="merge")
    # heavy merge columns
    big = [skewed(20000, 40, 90 + t, hubs=0, base=1) for t in range(3)]
    for i, b in enumerate(big):
        rng = np.random.default_rng(i)
        r = rng.choice(20000, 12000, replace=False)
        extra = from_coo(20000, 40, r, np.zeros(r.size, np.int64), rng.standard_normal(r.size))
        big[i] = oracle.merge([b, extra])
        big[i] = CSC(20000, 40, big[i].colptr.astype(np.int32), big[i].rowidx.astype(np.int32),
                     big[i].vals)
    M = spg.merge([to_dev(p) for p in big])
    torch.cuda.synchronize()
    ref = oracle.merge(big)
    ab = oracle.merge([CSC(p.nrows, p.ncols, p.colptr, p.rowidx, np.abs(p.vals)) for p in big]).vals
    assert_matches(host_csc(M), ref, ab, label="heavy merge")


# ---------------------------------------------------------------- batching

def test_batches_concatenate_to_unbatched():
    A = W.config1(n=2048)
    r = 12
    nnz = int(oracle.symbolic(A, A).sum())
    inputs = (A.nnz * 2) * r + 2 * (A.ncols + 1) * 4
    budget = inputs + (1 << 20) + (nnz * r) // 2
    got, info = run(A, A, budget=budget)
    assert info["nbatches"] >= 2, info
    ref, ab, nt = oracle.spgemm(A, A, with_absterm=True, with_nterm=True)
    assert_matches(got, ref, ab, nt, label="batched")


@pytest.mark.parametrize("nb_target", [1, 2, 20])
def test_heavy_items_over_many_batches(nb_target):
    """Heavy columns spread over 1, about 2 and about 20 batches: after the
    plan the items are ordered batch-major (by batch, kind and panel; by batch
    and kind when the scratch lacks room for the panel histogram; left in
    panel order when it lacks room for that), and each batch's launch takes
    its own run of them. With 24 heavy columns and 6 panels the three cases
    take the three orders."""
    A = skewed(6000, 6000, 11, hubs=4, hub_deg=2500, base=6)
    tun = spg.Tuning(hash_max_cap=256, panel_rows=1024)
    ref, ab, nt = oracle.spgemm(A, A, with_absterm=True, with_nterm=True)
    cnt = np.diff(ref.colptr)
    Ad = to_dev(A)
    big = 1 << 30
    probe = spg.Plan(Ad, Ad, budget=big, tuning=tun)
    cap0 = probe.symbolic()["batch_cap_bytes"]
    probe.close()
    r = 12
    total = r * ref.nnz + 8 * A.ncols
    target = max(int((r * int(cnt.max()) + 8) * 1.5), total // nb_target + 4096)
    budget = big - 2 * (cap0 - target)
    got, info = run(A, A, budget=budget, tuning=tun)
    assert info["heavy_columns"] > 0
    assert info["nbatches"] >= (nb_target + 1) // 2, info
    assert_matches(got, ref, ab, nt, label=f"heavy items, {info['nbatches']} batches")


def test_budget_too_small():
    A = W.config1(n=1024)
    with pytest.raises(spg.SpgemmError):
        run(A, A, budget=1 << 10)


def test_run_batched_streams_to_host():
    A = skewed(3000, 3000, 101, hubs=2, hub_deg=1000)
    Ad = to_dev(A)
    ref, ab, nt = oracle.spgemm(A, A, with_absterm=True, with_nterm=True)
    budget = A.bytes() * 2 + (1 << 20) + ref.nnz * 12
    for kst in (1, 3):
        plan = spg.Plan(Ad, Ad, budget=budget, kstages=kst, host_slot_bytes=1 << 16, host_slots=2)
        info = plan.symbolic()
        pieces = []

        def sink(batch, c0, c1, arrs):
            cp, ri, va = arrs
            pieces.append((batch, c0, c1, cp.copy(), ri.copy(), va.copy()))
            return 0

        spg.run_batched(plan, sink)
        assert pieces[0][1] == 0 and pieces[-1][2] == A.ncols
        for a, b in zip(pieces, pieces[1:]):
            assert a[2] == b[1] and b[0] >= a[0]
        colptr = [0]
        for _, c0, c1, cp, ri, va in pieces:
            colptr.extend((cp[1:] + colptr[-1]).tolist())
        got = CSC(A.nrows, A.ncols, np.array(colptr, np.int64),
                  np.concatenate([p[4] for p in pieces]).astype(np.int64),
                  np.concatenate([p[5] for p in pieces]))
        assert_matches(got, ref, ab, nt, label=f"run_batched s={kst}")
        assert len({p[0] for p in pieces}) == info["nbatches"]
        plan.close()


def test_sink_error_stops_cleanly():
    A = skewed(2000, 2000, 111, hubs=2, hub_deg=800)
    Ad = to_dev(A)
    plan = spg.Plan(Ad, Ad, host_slot_bytes=1 << 14, host_slots=2)
    plan.symbolic()
    calls = []

    def sink(batch, c0, c1, arrs):
        calls.append(c0)
        return 1 if len(calls) == 2 else 0

    with pytest.raises(spg.SpgemmError):
        spg.run_batched(plan, sink)
    assert len(calls) == 2
    # the plan stays usable
    C = plan.numeric(0)
    torch.cuda.synchronize()
    assert C.nnz == plan.batch(0)[2]
    plan.close()


# ---------------------------------------------------------------- backward

def test_backward_matches_oracle():
    A, B = W.config5(m=3000, k=3000, n=1500, value_dtype=np.float64)
    C = oracle.spgemm(A, B)
    G = shuffle_within_columns(W.values_on_pattern(C, 17, dist="normal", value_dtype=np.float64), 5)
    G = G.astype(index_dtype=np.int32)
    dA, dB = spg.backward(to_dev(A), to_dev(B), to_dev(G))
    torch.cuda.synchronize()
    rA, rB = oracle.backward(A, B, G)
    np.testing.assert_allclose(dA.cpu().numpy(), rA, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(dB.cpu().numpy(), rB, rtol=1e-11, atol=1e-11)


def test_backward_heavy_columns():
    A = skewed(4000, 3000, 121, hubs=2, hub_deg=2000)
    B = skewed(3000, 200, 122, hubs=1, hub_deg=2500)
    C = oracle.spgemm(A, B)
    G = W.values_on_pattern(C, 18, dist="normal", value_dtype=np.float64).astype(index_dtype=np.int32)
    Ad, Bd = to_dev(A), to_dev(B)
    plan = spg.Plan(Ad, Bd, tuning=spg.Tuning(hash_max_cap=256, panel_rows=1024))
    dA, dB = plan.backward(to_dev(G))
    torch.cuda.synchronize()
    rA, rB = oracle.backward(A, B, G)
    np.testing.assert_allclose(dA.cpu().numpy(), rA, rtol=1e-10, atol=1e-10)
    np.testing.assert_allclose(dB.cpu().numpy(), rB, rtol=1e-10, atol=1e-10)
    plan.close()


def test_backward_rejects_mismatched_g():
    A, B = W.config5(m=300, k=300, n=200, value_dtype=np.float64)
    C = oracle.spgemm(A, B)      # int64 indices
    G = W.values_on_pattern(C, 3, dist="normal", value_dtype=np.float64)
    with pytest.raises(spg.SpgemmError):
        spg.backward(to_dev(A), to_dev(B), to_dev(G))


def test_autograd_function_fp64_finite_differences():
    A, B = W.config5(m=64, k=64, n=64, value_dtype=np.float64)
    Ad, Bd = to_dev(A), to_dev(B)
    a = Ad.vals.clone().requires_grad_(True)
    b = Bd.vals.clone().requires_grad_(True)
    c = spg.SpGEMMFn.apply(a, b, Ad, Bd)
    torch.manual_seed(0)
    gvals = torch.randn(c.shape, dtype=torch.float64, device="cuda")
    (c * gvals).sum().backward()
    for recompute in (False, True):
        a2 = Ad.vals.clone().requires_grad_(True)
        b2 = Bd.vals.clone().requires_grad_(True)
        c2 = spg.SpGEMMFn.apply(a2, b2, Ad, Bd, recompute)
        (c2 * gvals).sum().backward()
        torch.testing.assert_close(a2.grad, a.grad, rtol=1e-12, atol=1e-12)
    # central differences of the bilinear loss are exact up to rounding
    h = 1e-3
    with torch.no_grad():
        for q in range(0, A.nnz, 97):
            ap = Ad.vals.clone(); ap[q] += h
            am = Ad.vals.clone(); am[q] -= h
            lp = (spg.SpGEMMFn.apply(ap, Bd.vals, Ad, Bd) * gvals).sum()
            lm = (spg.SpGEMMFn.apply(am, Bd.vals, Ad, Bd) * gvals).sum()
            fd = float((lp - lm) / (2 * h))
            assert abs(fd - float(a.grad[q])) <= 1e-9 * max(1.0, abs(fd))
    # and the gradient equals the oracle's masked products, with G in the
    # library's (unsorted) layout of C, which is the layout of SpGEMMFn's output
    plan = spg.Plan(Ad, Bd)
    plan.symbolic()
    Cl = plan.numeric(0)
    Gl = CSC(Cl.nrows, Cl.ncols, Cl.colptr.cpu().numpy().astype(np.int64),
             Cl.rowidx.cpu().numpy().astype(np.int64), gvals.cpu().numpy())
    rA, rB = oracle.backward(A, B, Gl)
    np.testing.assert_allclose(a.grad.cpu().numpy(), rA, rtol=1e-11, atol=1e-11)
    np.testing.assert_allclose(b.grad.cpu().numpy(), rB, rtol=1e-11, atol=1e-11)
    plan.close()


def test_autotuner_picks_a_working_candidate():
    from paper_2010_08526_gb300 import autotune
    A = skewed(3000, 3000, 131, hubs=2, hub_deg=1500)
    Ad = to_dev(A)
    cands = autotune.candidates(caps=(1024, 8192), panels=(8192, 16384), threads=(0, 256))
    best, res = autotune.tune_plan(Ad, Ad, cands, reps=1)
    assert best in [r[0] for r in res] and len(res) == len(cands)
    check_product(A, A, "autotuned", tuning=best)
    probs = [to_dev(p) for p in W.config4(count=6, nmax=3000)]
    bm, rm = autotune.tune_multi(probs, probs, reps=1)
    assert bm in [r[0] for r in rm]


# ---------------------------------------------------------------- batched problems

def _check_multi(probs, Bs=None, **kw):
    Bs = Bs if Bs is not None else probs
    dev = [to_dev(p) for p in probs]
    devb = dev if Bs is probs else [to_dev(b) for b in Bs]
    for use_graph in (False, True):
        M = spg.Multi(dev, devb, **kw)
        M.run(use_graph=use_graph)
        M.run(use_graph=use_graph)   # replay
        torch.cuda.synchronize()
        cp, ri, va = M.output()
        cp = cp.cpu().numpy(); ri = ri.cpu().numpy(); va = va.cpu().numpy()
        col = 0
        for p, b in zip(probs, Bs):
            ref = oracle.spgemm(p, b)
            lo, hi = cp[col], cp[col + b.ncols]
            got = CSC(p.nrows, b.ncols, cp[col:col + b.ncols + 1] - lo, ri[lo:hi].astype(np.int64), va[lo:hi])
            assert_matches(got, ref, exact=True, label="multi")
            col += b.ncols
        M.close()


def test_multi_path_counting_exact():
    _check_multi(W.config4(count=24, nmax=5000))


@pytest.mark.parametrize("tun", [dict(hash_max_cap=1024, warp_max_cap=128, block_tier_threads=256),
                                 dict(hash_max_cap=4096, warp_max_cap=32, block_tier_threads=512),
                                 dict(hash_max_cap=8192, warp_max_cap=512, block_tier_threads=512)])
def test_multi_tuning_variants(tun):
    _check_multi(W.config4(count=16, nmax=8000), tuning=spg.Tuning(**tun))


def test_multi_heavy_columns_use_global_tables():
    """Problems with hub columns above the largest shared-memory table (the
    refusal of earlier versions): their columns take global-memory tables in
    the same persistent launch as the small ones. int64 path counts, exact."""
    probs = W.config4(count=6, nmax=3000)
    hubs = [skewed(5000, 5000, 900 + i, hubs=2, hub_deg=3000, base=3, dist="ones") for i in range(3)]
    allp = probs[:3] + hubs + probs[3:]
    _check_multi(allp, tuning=spg.Tuning(hash_max_cap=1024))
    # rectangular problems with heavy columns and an empty one
    A1 = skewed(4000, 300, 911, hubs=1, hub_deg=3500, base=4, dist="ones")
    B1 = skewed(300, 700, 912, hubs=2, hub_deg=250, base=8, dist="ones")
    Z = CSC(50, 40, np.zeros(41, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64))
    Zb = CSC(40, 30, np.zeros(31, np.int32), np.zeros(0, np.int32), np.zeros(0, np.int64))
    _check_multi([A1, Z] + probs[:2], Bs=[B1, Zb] + probs[:2], tuning=spg.Tuning(hash_max_cap=256, warp_max_cap=128))


# ------------------------------------------------------ every output slot written

@pytest.mark.parametrize("kst,sort_output", [(1, False), (3, False), (1, True)])
def test_poisoned_outputs_are_fully_written(kst, sort_output):
    """Output buffers filled with a poison (row -7, value NaN) before the
    numeric: after every batch no poison is left, and the result is the
    oracle's. Catches slots no kernel writes, which fresh or reused memory
    could otherwise hide. Heavy columns included (small tables and panels)."""
    A = skewed(4000, 4000, 91, hubs=3, hub_deg=1500, base=6)
    Ad = to_dev(A)
    ref, ab, nt = oracle.spgemm(A, A, with_absterm=True, with_nterm=True)
    tun = spg.Tuning(hash_max_cap=256, panel_rows=1024)
    plan = spg.Plan(Ad, Ad, kstages=kst, tuning=tun, sort_output=sort_output,
                    budget=A.bytes() * 2 + (2 << 20) + ref.nnz * 12 * kst)
    info = plan.symbolic()
    assert info["nbatches"] >= 2 and info["heavy_columns"] > 0
    nnz = int(info["nnz_c"])
    rows = torch.full((nnz,), -7, dtype=torch.int32, device="cuda")
    vals = torch.full((nnz,), float("nan"), dtype=torch.float64, device="cuda")
    scratch = torch.full((int(info["max_batch_cols"]) + 1,), -7, dtype=torch.int64, device="cuda")
    off = 0
    for t in range(plan.nbatches):
        c0, c1, bn = plan.batch(t)
        plan.numeric_into(t, scratch[: c1 - c0 + 1], rows[off:off + bn], vals[off:off + bn])
        assert int(scratch[c1 - c0].item()) == bn        # the batch colptr is written too
        off += bn
    torch.cuda.synchronize()
    counts = plan.column_counts().cpu().numpy()
    plan.close()
    r = rows.cpu().numpy()
    v = vals.cpu().numpy()
    assert off == nnz and (r >= 0).all() and not np.isnan(v).any()
    got = CSC(A.nrows, A.ncols, np.concatenate([[0], np.cumsum(counts)]).astype(np.int64), r, v)
    if sort_output:
        assert np.array_equal(got.rowidx.astype(np.int64), ref.rowidx)
    assert_matches(got, ref, ab, nt, label=f"poisoned s={kst} sorted={sort_output}")
