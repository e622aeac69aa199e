"""Pins for the CPU oracle: each check is independent of the oracle's own code
(dense numpy products, brute force in Python, closed forms, invariants, the
paper's printed numbers), chosen so that a dropped term, a wrong index or a
transposed operand in the oracle fails at least one of them.
"""
from __future__ import annotations

import itertools
import os

import numpy as np
import pytest

import oracle
import workloads as W
from workloads.csc import CSC, from_coo, transpose, shuffle_within_columns, column_slice

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rand_csc(m, n, density, seed, *, vals="normal", index_dtype=np.int32, shuffle=True):
    rng = np.random.default_rng(seed)
    mask = rng.random((m, n)) < density
    r, c = np.nonzero(mask)
    if vals == "normal":
        v = rng.standard_normal(r.size)
    elif vals == "int":
        v = rng.integers(-5, 6, r.size).astype(np.int64)
    elif vals == "ones":
        v = np.ones(r.size, dtype=np.int64)
    else:
        raise ValueError(vals)
    a = from_coo(m, n, r, c, v, dup="error", index_dtype=index_dtype)
    return shuffle_within_columns(a, seed + 7) if shuffle else a


def dense_structure(A: CSC):
    d = np.zeros((A.nrows, A.ncols), dtype=np.int64)
    cols = np.repeat(np.arange(A.ncols), A.col_counts())
    d[A.rowidx.astype(np.int64), cols] = 1
    return d


def read_golden_triples(path):
    sections, cur = {}, None
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("["):
            cur = line.strip("[]")
            sections[cur] = []
            continue
        sections[cur].append([int(x) for x in line.split()])
    return sections


# --------------------------------------------------------------------------- c1

@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("shape", [(7, 5, 6), (13, 17, 11), (32, 24, 40), (1, 9, 3)])
def test_product_matches_dense_fp64(seed, shape):
    m, k, n = shape
    A = rand_csc(m, k, 0.3, seed)
    B = rand_csc(k, n, 0.3, seed + 100)
    C = oracle.spgemm(A, B)
    Cd = A.to_dense().astype(np.float64) @ B.to_dense().astype(np.float64)
    got = np.zeros((m, n))
    cols = np.repeat(np.arange(n), C.col_counts())
    got[C.rowidx, cols] = C.vals
    np.testing.assert_allclose(got, Cd, rtol=1e-13, atol=1e-13)
    # structure: exactly the entries reached by some product (boolean product)
    S = (dense_structure(A) @ dense_structure(B)) > 0
    sgot = np.zeros((m, n), dtype=bool)
    sgot[C.rowidx, cols] = True
    assert np.array_equal(S, sgot)
    # rows sorted inside each column
    for j in range(n):
        seg = C.rowidx[C.colptr[j]:C.colptr[j + 1]]
        assert np.all(np.diff(seg) > 0)


@pytest.mark.parametrize("seed", range(4))
def test_product_matches_dense_int64(seed):
    A = rand_csc(20, 15, 0.35, seed, vals="int")
    B = rand_csc(15, 18, 0.35, seed + 50, vals="int")
    C = oracle.spgemm(A, B)
    assert C.vals.dtype == np.int64
    Cd = A.to_dense().astype(np.int64) @ B.to_dense().astype(np.int64)
    got = np.zeros_like(Cd)
    cols = np.repeat(np.arange(C.ncols), C.col_counts())
    got[C.rowidx, cols] = C.vals
    assert np.array_equal(got, Cd)


def test_zero_sums_are_kept_structurally():
    # A(:,0) = [1, 1], A(:,1) = [1, -1]; B(:,0) = [1, 1]^T -> C(:,0) = [2, 0]
    A = from_coo(2, 2, [0, 1, 0, 1], [0, 0, 1, 1], [1.0, 1.0, 1.0, -1.0])
    B = from_coo(2, 1, [0, 1], [0, 0], [1.0, 1.0])
    C = oracle.spgemm(A, B)
    assert C.nnz == 2
    assert list(C.rowidx) == [0, 1]
    assert list(C.vals) == [2.0, 0.0]


def test_int64_wraps_like_twos_complement():
    big = (1 << 62) + 12345
    A = from_coo(1, 3, [0, 0, 0], [0, 1, 2], np.array([big, big, -7], dtype=np.int64))
    B = from_coo(3, 1, [0, 1, 2], [0, 0, 0], np.array([3, 5, 1 << 61], dtype=np.int64))
    C = oracle.spgemm(A, B)
    exact = big * 3 + big * 5 + (-7) * (1 << 61)
    wrapped = (exact + (1 << 63)) % (1 << 64) - (1 << 63)
    assert int(C.vals[0]) == wrapped


def test_identity_is_neutral():
    A = rand_csc(30, 20, 0.2, 3)
    I_k = from_coo(20, 20, np.arange(20), np.arange(20), np.ones(20))
    I_m = from_coo(30, 30, np.arange(30), np.arange(30), np.ones(30))
    for C in (oracle.spgemm(A, I_k), oracle.spgemm(I_m, A)):
        ref = oracle.canonical(A)
        assert np.array_equal(C.colptr, ref.colptr)
        assert np.array_equal(C.rowidx, ref.rowidx)
        assert np.array_equal(C.vals, ref.vals.astype(np.float64))


def test_path_counting_brute_force():
    """Ones semiring: C(i,j) = #{k : A(i,k) != 0 and A(k,j) != 0}."""
    A = rand_csc(14, 14, 0.25, 11, vals="ones")
    C = oracle.spgemm(A, A)
    S = dense_structure(A)
    for j in range(14):
        got = dict(zip(C.rowidx[C.colptr[j]:C.colptr[j + 1]].tolist(),
                       C.vals[C.colptr[j]:C.colptr[j + 1]].tolist()))
        for i in range(14):
            paths = sum(1 for k in range(14) if S[i, k] and S[k, j])
            assert got.get(i, 0) == paths
            assert (i in got) == (paths > 0)


def test_golden_worked_example():
    g = read_golden_triples(os.path.join(GOLDEN, "worked_3x3.txt"))
    def mk(rows):
        r, c, v = zip(*rows)
        return from_coo(3, 3, r, c, np.array(v, dtype=np.int64))
    A, B, Cref = mk(g["A"]), mk(g["B"]), mk(g["C"])
    C = oracle.spgemm(A, B)
    assert np.array_equal(C.colptr, Cref.colptr.astype(np.int64))
    assert np.array_equal(C.rowidx, Cref.rowidx.astype(np.int64))
    assert np.array_equal(C.vals, Cref.vals)


# ----------------------------------------------------------------- flops / c2/c3

def test_flops_brute_force_and_cf():
    A = rand_csc(25, 30, 0.2, 5)
    B = rand_csc(30, 22, 0.2, 6)
    f = oracle.flops_per_column(A, B)
    SA, SB = dense_structure(A), dense_structure(B)
    brute = np.array([sum(SA[:, k].sum() for k in range(30) if SB[k, j]) for j in range(22)])
    assert np.array_equal(f, brute)
    nnzc = oracle.symbolic(A, B)
    assert np.all(nnzc <= f)          # cf >= 1 per column (Sec. II-A)
    assert f.sum() >= nnzc.sum() > 0


@pytest.mark.parametrize("s", [1, 2, 3, 4, 7])
def test_eq1_inequalities_and_stage_merge(s):
    """Eq. (1): flops >= sum_t nnz(D_t) >= nnz(C); merging the stage products
    gives the unsplit product."""
    A = rand_csc(40, 35, 0.15, 21 + s)
    B = rand_csc(35, 30, 0.15, 31 + s)
    F = int(oracle.flops_per_column(A, B).sum())
    C = oracle.spgemm(A, B)
    parts = [oracle.spgemm(A, B, krange=kr) for kr in oracle.stage_ranges(A.ncols, s)]
    U = sum(p.nnz for p in parts)
    assert F >= U >= C.nnz
    assert sum(int(oracle.flops_per_column(A, B, kr).sum())
               for kr in oracle.stage_ranges(A.ncols, s)) == F
    M = oracle.merge(parts)
    assert np.array_equal(M.colptr, C.colptr) and np.array_equal(M.rowidx, C.rowidx)
    np.testing.assert_allclose(M.vals, C.vals, rtol=1e-12, atol=1e-14)
    # stage ranges tile [0, k) contiguously
    kr = oracle.stage_ranges(A.ncols, s)
    assert kr[0][0] == 0 and kr[-1][1] == A.ncols
    assert all(kr[i][1] == kr[i + 1][0] for i in range(s - 1))


def test_merge_matches_dense_sum_int():
    parts = [rand_csc(12, 9, 0.3, 70 + t, vals="int") for t in range(3)]
    M = oracle.merge(parts)
    ref = sum(p.to_dense().astype(np.int64) for p in parts)
    got = np.zeros_like(ref)
    cols = np.repeat(np.arange(9), M.col_counts())
    got[M.rowidx, cols] = M.vals
    assert np.array_equal(got, ref)
    S = sum(dense_structure(p) for p in parts) > 0
    assert M.nnz == int(S.sum())


def test_symbolic_equals_numeric_nnz_and_boolean_popcount():
    A = rand_csc(50, 45, 0.08, 41)
    B = rand_csc(45, 60, 0.08, 42)
    cnt = oracle.symbolic(A, B)
    C = oracle.spgemm(A, B)
    assert np.array_equal(cnt, C.col_counts())
    S = (dense_structure(A) @ dense_structure(B)) > 0
    assert np.array_equal(cnt, S.sum(axis=0))


def test_column_ranges_concatenate_to_whole():
    """ColConcat of batches equals the unbatched product (Algorithm 4)."""
    A = rand_csc(30, 30, 0.15, 51)
    C = oracle.spgemm(A, A)
    pieces = [oracle.spgemm(A, A, cols=(c0, c1)) for c0, c1 in [(0, 7), (7, 8), (8, 8), (8, 30)]]
    rows = np.concatenate([p.rowidx for p in pieces])
    vals = np.concatenate([p.vals for p in pieces])
    counts = np.concatenate([p.col_counts() for p in pieces])
    assert np.array_equal(counts, C.col_counts())
    assert np.array_equal(rows, C.rowidx) and np.array_equal(vals, C.vals)


def test_row_order_invariance():
    """Sort-free inputs (Sec. IV-D): shuffling rows inside input columns
    changes nothing after the canonical sort."""
    A = rand_csc(35, 28, 0.2, 61, vals="int", shuffle=False)
    B = rand_csc(28, 33, 0.2, 62, vals="int", shuffle=False)
    C0 = oracle.spgemm(A, B)
    C1 = oracle.spgemm(shuffle_within_columns(A, 1), shuffle_within_columns(B, 2))
    assert np.array_equal(C0.rowidx, C1.rowidx) and np.array_equal(C0.vals, C1.vals)


def test_semiring_invariants():
    A = rand_csc(26, 19, 0.2, 71)
    B = rand_csc(19, 23, 0.2, 72)
    C = oracle.spgemm(A, B)
    ones = np.ones(23)
    Cd = np.zeros((26, 23))
    cols = np.repeat(np.arange(23), C.col_counts())
    Cd[C.rowidx, cols] = C.vals
    lhs = Cd @ ones
    rhs = A.to_dense() @ (B.to_dense() @ ones)
    np.testing.assert_allclose(lhs, rhs, rtol=1e-12, atol=1e-12)
    # (AB)^T = B^T A^T
    Ct = oracle.spgemm(transpose(B), transpose(A))
    CT = transpose(CSC(C.nrows, C.ncols, C.colptr, C.rowidx, C.vals))
    assert np.array_equal(Ct.colptr, CT.colptr.astype(np.int64))
    assert np.array_equal(Ct.rowidx, CT.rowidx.astype(np.int64))
    np.testing.assert_allclose(Ct.vals, CT.vals, rtol=1e-13, atol=1e-13)


def test_absterm_bounds_value():
    A = rand_csc(20, 20, 0.3, 81)
    C, ab = oracle.spgemm(A, A, with_absterm=True)
    assert np.all(np.abs(C.vals) <= ab * (1 + 1e-12))
    Ad = np.abs(A.to_dense())
    Sd = Ad @ Ad
    cols = np.repeat(np.arange(20), C.col_counts())
    np.testing.assert_allclose(ab, Sd[C.rowidx, cols], rtol=1e-13)


def test_nterm_is_structure_product():
    # n_ij = |{k : A(i,k) != 0 and B(k,j) != 0}| = (S_A S_B)(i, j), the dense
    # integer product of the 0/1 structure matrices; over a k-stage the
    # product of the stage's slices. Values are chosen so that some sums
    # cancel to zero (the count still holds: structure, not value).
    for seed, (m, k, n, d) in enumerate([(20, 20, 20, 0.3), (37, 11, 23, 0.5), (9, 40, 5, 0.2)]):
        A = rand_csc(m, k, d, 300 + seed)
        B = rand_csc(k, n, d, 400 + seed)
        A.vals[::3] *= -1.0
        SA = (A.to_dense() != 0).astype(np.int64)
        SB = (B.to_dense() != 0).astype(np.int64)
        for krange in (None, (k // 3, k - k // 4)):
            C, nt = oracle.spgemm(A, B, krange=krange, with_nterm=True)
            k0, k1 = (0, k) if krange is None else krange
            N = SA[:, k0:k1] @ SB[k0:k1, :]
            cols = np.repeat(np.arange(n), C.col_counts())
            assert np.array_equal(nt, N[C.rowidx, cols])
            assert np.all(nt >= 1)
            # every reached entry is listed once: the structure is N > 0
            assert int((N > 0).sum()) == C.nnz
            # the counts of a column add up to its flops
            f = oracle.flops_per_column(A, B, krange)
            assert np.array_equal(np.bincount(cols, weights=nt, minlength=n).astype(np.int64), f)
            # the three-tuple form returns the same C and scale
            C2, ab, nt2 = oracle.spgemm(A, B, krange=krange, with_absterm=True, with_nterm=True)
            assert np.array_equal(C2.rowidx, C.rowidx) and np.array_equal(nt2, nt)


# ----------------------------------------------------------------------- c3 plan

def test_plan_ranges_additive_equals_plan_batches():
    rng = np.random.default_rng(93)
    for trial in range(300):
        n = int(rng.integers(0, 12))
        w = rng.integers(0, 10, n)
        cap = int(rng.integers(1, 25))
        pre = np.concatenate([[0], np.cumsum(w)])
        got = oracle.plan_ranges(lambda a, b: int(pre[b] - pre[a]), n, cap)
        ref = oracle.plan_batches(w, cap)
        if ref is None:
            assert got is None
        else:
            assert np.array_equal(got, ref)


def test_plan_ranges_minimal_for_max_costs():
    # a cost with a maximum over "stages" (like a batch that keeps the largest
    # of several partial products): monotone under range growth but not a sum;
    # greedy extension still gives the fewest contiguous ranges (brute force)
    import itertools
    rng = np.random.default_rng(94)
    for trial in range(200):
        n = int(rng.integers(1, 8))
        s = int(rng.integers(1, 4))
        base = rng.integers(0, 6, n)
        d = rng.integers(0, 6, (s, n))
        cap = int(rng.integers(3, 30))

        def cost(a, b):
            return int(base[a:b].sum() + max(d[t, a:b].sum() for t in range(s)))

        got = oracle.plan_ranges(cost, n, cap)
        best = None
        for cuts in itertools.product([0, 1], repeat=n - 1):
            starts = [0] + [i + 1 for i in range(n - 1) if cuts[i]] + [n]
            if all(cost(starts[i], starts[i + 1]) <= cap for i in range(len(starts) - 1)):
                if best is None or len(starts) < best:
                    best = len(starts)
        if best is None:
            assert got is None
        else:
            assert got is not None and len(got) == best
            assert got[0] == 0 and got[-1] == n
            assert all(cost(got[i], got[i + 1]) <= cap for i in range(len(got) - 1))


def test_plan_batches_greedy_is_minimal_and_valid():
    rng = np.random.default_rng(91)
    for trial in range(200):
        n = int(rng.integers(1, 9))
        w = rng.integers(0, 10, n)
        cap = int(rng.integers(1, 20))
        begin = oracle.plan_batches(w, cap)
        if w.max() > cap:
            assert begin is None
            continue
        b = len(begin) - 1
        assert begin[0] == 0 and begin[-1] == n
        for t in range(b):
            seg = w[begin[t]:begin[t + 1]]
            assert seg.sum() <= cap and begin[t + 1] > begin[t]
            if t + 1 < b:  # greedy: the next column would not have fit
                assert seg.sum() + w[begin[t + 1]] > cap
        # brute force: no contiguous partition uses fewer ranges
        best = n + 1
        for mask in range(1 << (n - 1)):
            cuts = [0] + [i + 1 for i in range(n - 1) if mask >> i & 1] + [n]
            if all(w[cuts[i]:cuts[i + 1]].sum() <= cap for i in range(len(cuts) - 1)):
                best = min(best, len(cuts) - 1)
        assert b == best
        assert b >= -(-int(w.sum()) // cap)   # Eq. (2)-style lower bound


def test_eq2_bound_and_paper_memory_example():
    vals = {}
    for line in open(os.path.join(GOLDEN, "paper_memory_example.txt")):
        if line.strip() and not line.startswith("#"):
            k, v = line.split()
            vals[k] = float(v)
    r = int(vals["r"])
    assert oracle.mem_bytes(r, [int(vals["nnz_c"])]) == int(vals["final_output_bytes"])
    assert oracle.mem_bytes(r, [int(vals["flops"])]) == int(vals["worst_case_bytes"])
    # Eq. (2) with the paper's printed sizes: 2208 TB over 1.09 PB minus inputs
    b = oracle.batch_lower_bound(int(vals["worst_case_bytes"]), int(vals["aggregate_memory_bytes"]),
                                 r, int(vals["nnz_a"]), int(vals["nnz_a"]))
    den = vals["aggregate_memory_bytes"] - r * 2 * vals["nnz_a"]
    assert b == int(np.ceil(vals["worst_case_bytes"] / den)) == 3
    assert oracle.batch_lower_bound(10, 5, 1, 3, 3) == -1
    assert oracle.batch_lower_bound(0, 100, 1, 1, 1) == 1
    assert oracle.batch_lower_bound(101, 102, 1, 1, 0) == 1
    assert oracle.batch_lower_bound(102, 102, 1, 1, 0) == 2


# ----------------------------------------------------------------------- c7

def _loss(A, B, G):
    C = oracle.spgemm(A, B)
    Gc = oracle.canonical(G)
    assert np.array_equal(C.rowidx, Gc.rowidx)
    return float(np.dot(C.vals, Gc.vals))


def test_backward_finite_differences_exact_for_bilinear_loss():
    A, B = W.config5(m=64, k=64, n=64, value_dtype=np.float64)
    C = oracle.spgemm(A, B)
    G = W.values_on_pattern(C, 5, dist="normal", value_dtype=np.float64)
    G = shuffle_within_columns(G, 3)
    dA, dB = oracle.backward(A, B, G)
    h = 1e-3
    rng = np.random.default_rng(0)
    for q in rng.choice(A.nnz, 40, replace=False):
        Ap = CSC(A.nrows, A.ncols, A.colptr, A.rowidx, A.vals.copy()); Ap.vals[q] += h
        Am = CSC(A.nrows, A.ncols, A.colptr, A.rowidx, A.vals.copy()); Am.vals[q] -= h
        fd = (_loss(Ap, B, G) - _loss(Am, B, G)) / (2 * h)
        assert abs(fd - dA[q]) <= 1e-9 * max(1.0, abs(dA[q]))
    for p in rng.choice(B.nnz, 40, replace=False):
        Bp = CSC(B.nrows, B.ncols, B.colptr, B.rowidx, B.vals.copy()); Bp.vals[p] += h
        Bm = CSC(B.nrows, B.ncols, B.colptr, B.rowidx, B.vals.copy()); Bm.vals[p] -= h
        fd = (_loss(A, Bp, G) - _loss(A, Bm, G)) / (2 * h)
        assert abs(fd - dB[p]) <= 1e-9 * max(1.0, abs(dB[p]))


def test_backward_matches_dense_masked_products():
    A = rand_csc(18, 14, 0.3, 101)
    B = rand_csc(14, 16, 0.3, 102)
    C = oracle.spgemm(A, B)
    G = W.values_on_pattern(C, 9, dist="normal", value_dtype=np.float64)
    dA, dB = oracle.backward(A, B, G)
    Gd = G.to_dense()
    dAd = Gd @ B.to_dense().T
    dBd = A.to_dense().T @ Gd
    colsA = np.repeat(np.arange(A.ncols), A.col_counts())
    colsB = np.repeat(np.arange(B.ncols), B.col_counts())
    np.testing.assert_allclose(dA, dAd[A.rowidx, colsA], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(dB, dBd[B.rowidx, colsB], rtol=1e-12, atol=1e-12)


# ----------------------------------------------------------------- generators

def test_generators_shapes_and_recipes():
    A1 = W.config1(n=256)
    A1.validate()
    assert np.all(A1.col_counts() == 8)
    assert A1.vals.dtype == np.float64 and A1.rowidx.dtype == np.int32
    A2 = W.config2(scale=10, edge_factor=16)
    A2.validate()
    d2 = A2.to_dense()
    assert np.allclose(d2, d2.T)          # X + X^T is symmetric
    A3 = W.config3(n=5000)
    A3.validate()
    d3 = A3.to_dense()
    assert np.array_equal(d3, d3.T)
    assert A3.rowidx.dtype == np.int64
    assert 0.3 <= A3.vals.min() and A3.vals.max() <= 1.0
    probs = W.config4(count=6, nmax=3000)
    for P in probs:
        P.validate()
        assert np.all(P.vals == 1)
    A5, B5 = W.config5(m=300, k=300, n=150)
    assert np.all(A5.col_counts() == 16) and np.all(B5.col_counts() == 8)
    # determinism
    assert np.array_equal(W.config1(n=256).rowidx, A1.rowidx)


# ---------------------------------------------------------------- prune
def _col(C, j):
    a, b = int(C.colptr[j]), int(C.colptr[j + 1])
    return np.asarray(C.rowidx[a:b], dtype=np.int64), np.asarray(C.vals[a:b])


@pytest.mark.parametrize("vals", ["normal", "int"])
@pytest.mark.parametrize("topk,thr", [(0, 0.0), (3, float("-inf")), (2, -0.5), (1, 0.25), (50, 0.0)])
def test_prune_properties(vals, topk, thr):
    """Prune (the per-column top-k / threshold step of the batches' consumer):
    every output column is an order-preserving subsequence of the input, all
    kept values pass the threshold, the count is min(topk, candidates), no
    dropped candidate beats a kept one, and among equal values at the cut the
    earlier stored entries are the ones kept."""
    C = rand_csc(40, 30, 0.3, 11, vals=vals)
    P = oracle.prune(C, thr, topk)
    int_vals = vals == "int"
    t = np.ceil(thr) if (int_vals and np.isfinite(thr)) else thr
    for j in range(C.ncols):
        r, v = _col(C, j)
        pr, pv = _col(P, j)
        cand = np.nonzero(v >= t)[0]
        want = len(cand) if topk <= 0 else min(topk, len(cand))
        assert len(pr) == want
        # subsequence, in order
        pos = []
        for x in pr:
            pos.append(int(np.nonzero(r == x)[0][0]))
        assert pos == sorted(pos)
        assert np.array_equal(v[pos], pv)
        assert np.all(pv >= t)
        dropped = np.setdiff1d(cand, pos)
        if len(pv) and len(dropped):
            assert v[dropped].max() <= pv.min()
            cut = pv.min()
            kept_at_cut = [p for p in pos if v[p] == cut]
            dropped_at_cut = [p for p in dropped if v[p] == cut]
            if kept_at_cut and dropped_at_cut:
                assert max(kept_at_cut) < min(dropped_at_cut)


def test_prune_special_cases():
    """No threshold and no limit is the identity; topk = 1 with no threshold is
    the column argmax (first occurrence, numpy's rule); a threshold alone keeps
    exactly the entries numpy selects; top-k maximises the kept sum."""
    C = rand_csc(60, 25, 0.25, 5)
    ident = oracle.prune(C, float("-inf"), 0)
    assert np.array_equal(ident.colptr, C.colptr)
    assert np.array_equal(ident.rowidx, C.rowidx.astype(np.int64))
    assert np.array_equal(ident.vals, C.vals)
    top1 = oracle.prune(C, float("-inf"), 1)
    for j in range(C.ncols):
        r, v = _col(C, j)
        pr, pv = _col(top1, j)
        if len(v):
            assert pr[0] == r[np.argmax(v)] and pv[0] == v.max()
        else:
            assert len(pr) == 0
    thr = oracle.prune(C, 0.3, 0)
    for j in range(C.ncols):
        r, v = _col(C, j)
        pr, pv = _col(thr, j)
        assert np.array_equal(pr, r[v >= 0.3]) and np.array_equal(pv, v[v >= 0.3])
    k = 4
    topk = oracle.prune(C, float("-inf"), k)
    for j in range(C.ncols):
        _, v = _col(C, j)
        _, pv = _col(topk, j)
        assert np.isclose(pv.sum(), np.sort(v)[::-1][:k].sum())


def test_prune_ties_keep_earlier_entries():
    """All-equal column: top-k keeps the first k stored entries."""
    n = 10
    C = CSC(20, 1, np.array([0, n], np.int64), np.arange(19, 19 - n, -1, dtype=np.int64), np.full(n, 0.5))
    P = oracle.prune(C, float("-inf"), 3)
    assert np.array_equal(P.rowidx, [19, 18, 17])


# ---------------------------------------------------------------- min-plus
def _dense_minplus(A: CSC, B: CSC):
    """Brute force over all k with +inf for absent entries; structure from the
    boolean product."""
    da = np.full((A.nrows, A.ncols), np.inf)
    ca = np.repeat(np.arange(A.ncols), A.col_counts())
    da[A.rowidx.astype(np.int64), ca] = A.vals
    db = np.full((B.nrows, B.ncols), np.inf)
    cb = np.repeat(np.arange(B.ncols), B.col_counts())
    db[B.rowidx.astype(np.int64), cb] = B.vals
    vals = np.min(da[:, :, None] + db[None, :, :], axis=1)
    struct = dense_structure(A) @ dense_structure(B) > 0
    return vals, struct


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_minplus_matches_dense_brute_force(seed):
    """Min-plus (the paper's algorithms hold over any semiring, Sec. II):
    C(i,j) = min_k A(i,k) + B(k,j) on the boolean product's structure."""
    A = rand_csc(25, 18, 0.25, seed)
    B = rand_csc(18, 21, 0.25, seed + 10)
    C = oracle.spgemm(A, B, semiring="min_plus")
    vals, struct = _dense_minplus(A, B)
    assert np.array_equal(dense_structure(C) > 0, struct)
    cc = np.repeat(np.arange(C.ncols), C.col_counts())
    assert np.array_equal(C.vals, vals[C.rowidx, cc])


def test_minplus_identity_and_nan_and_stages():
    A = rand_csc(30, 30, 0.2, 7)
    n = A.ncols
    Z = CSC(n, n, np.arange(n + 1, dtype=np.int64), np.arange(n, dtype=np.int64), np.zeros(n))
    C = oracle.spgemm(A, Z, semiring="min_plus")          # 0 is the (x) identity
    ref = oracle.canonical(A)
    assert np.array_equal(C.colptr, ref.colptr) and np.array_equal(C.rowidx, ref.rowidx)
    assert np.array_equal(C.vals, ref.vals)
    # a NaN product is ignored by the min
    An = CSC(2, 2, np.array([0, 2, 2]), np.array([0, 1]), np.array([np.nan, 1.0]))
    Bn = CSC(2, 1, np.array([0, 1]), np.array([0]), np.array([2.0]))
    Cn = oracle.spgemm(An, Bn, semiring="min_plus")
    assert np.array_equal(Cn.rowidx, [0, 1]) and np.isinf(Cn.vals[0]) and Cn.vals[1] == 3.0
    # stages merged with min equal the unsplit product
    B = rand_csc(30, 40, 0.2, 8)
    full = oracle.spgemm(A, B, semiring="min_plus")
    parts = [oracle.spgemm(A, B, krange=r, semiring="min_plus") for r in oracle.stage_ranges(30, 3)]
    merged = oracle.merge(parts, semiring="min_plus")
    assert np.array_equal(merged.colptr, full.colptr) and np.array_equal(merged.rowidx, full.rowidx)
    assert np.array_equal(merged.vals, full.vals)


# ---------------------------------------------------------------- or-and
def _with_false_entries(A: CSC, seed, as_int=False):
    """About a third of the stored values set to false (0, and -0.0 for
    floats), one to NaN (true): explicit zeros are stored entries that
    carry no truth."""
    rng = np.random.default_rng(seed)
    v = A.vals.astype(np.int64 if as_int else np.float64).copy()
    z = rng.random(v.size) < 0.35
    v[z] = 0
    if not as_int:
        v[z & (rng.random(v.size) < 0.5)] = -0.0
        v[np.flatnonzero(~z)[:1]] = np.nan
    return CSC(A.nrows, A.ncols, A.colptr, A.rowidx, v)


@pytest.mark.parametrize("seed,as_int", [(1, False), (2, False), (3, True), (4, True)])
def test_orand_matches_dense_boolean_product(seed, as_int):
    """Or-and (the algorithms hold over any semiring, Sec. II): on the
    structure of the product, C(i,j) = 1 iff some k has A(i,k) != 0 and
    B(k,j) != 0 -- a dense integer product of the truth matrices."""
    A = _with_false_entries(rand_csc(25, 18, 0.3, seed), seed + 20, as_int)
    B = _with_false_entries(rand_csc(18, 21, 0.3, seed + 10), seed + 30, as_int)
    C = oracle.spgemm(A, B, semiring="or_and")

    def truth(X):
        d = np.zeros((X.nrows, X.ncols), np.int64)
        cx = np.repeat(np.arange(X.ncols), X.col_counts())
        d[X.rowidx.astype(np.int64), cx] = (X.vals != 0).astype(np.int64)   # NaN != 0 is true
        return d

    struct = dense_structure(A) @ dense_structure(B) > 0
    val = (truth(A) @ truth(B)) > 0
    assert np.array_equal(dense_structure(C) > 0, struct)
    cc = np.repeat(np.arange(C.ncols), C.col_counts())
    assert np.array_equal(C.vals, val[C.rowidx, cc].astype(C.vals.dtype))
    assert C.vals.dtype == (np.int64 if as_int else np.float64)
    assert 0 < int((C.vals == 0).sum()) < C.nnz          # both truth values occur


def test_orand_stages_merge_and_all_true_inputs():
    A = _with_false_entries(rand_csc(30, 30, 0.2, 7), 9)
    B = _with_false_entries(rand_csc(30, 40, 0.2, 8), 10)
    full = oracle.spgemm(A, B, semiring="or_and")
    parts = [oracle.spgemm(A, B, krange=r, semiring="or_and") for r in oracle.stage_ranges(30, 3)]
    merged = oracle.merge(parts, semiring="or_and")
    assert np.array_equal(merged.colptr, full.colptr) and np.array_equal(merged.rowidx, full.rowidx)
    assert np.array_equal(merged.vals, full.vals)
    # inputs without false entries: every entry of C is true, on C's structure
    P = rand_csc(30, 30, 0.2, 11)
    Q = rand_csc(30, 40, 0.2, 12)
    Cb = oracle.spgemm(P, Q, semiring="or_and")
    assert np.array_equal(Cb.colptr[1:] - Cb.colptr[:-1], oracle.symbolic(P, Q))
    assert np.all(Cb.vals == 1.0)
