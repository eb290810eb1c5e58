"""Pins of the CPU oracle to things other than itself (no GPU needed).

Each test checks the oracle against an independent statement of the same
result: a dense brute-force triple loop written here, hand-worked fixtures,
closed forms, or an external library (scipy, networkx).  A wrong sign, a dropped
term, a transposed operand or a wrong additive operator in the oracle fails at
least one of them.
"""
import math
import os

import networkx as nx
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse import csgraph

import oracle as O
import workloads as W

GOLD = os.path.join(os.path.dirname(__file__), "golden")
INF32 = np.float32(np.inf)


# ------------------------------------------------------------ helpers (tests only)

def dense_of(m: W.Csr):
    """(present mask, dense values) of a CSR matrix."""
    pres = np.zeros((m.nrows, m.ncols), dtype=bool)
    rows = np.repeat(np.arange(m.nrows), np.diff(m.rowptr))
    pres[rows, m.col] = True
    if m.val is None:
        return pres, None
    vals = np.zeros((m.nrows, m.ncols), dtype=m.val.dtype)
    vals[rows, m.col] = m.val
    return pres, vals


def brute_force(alg, A: W.Csr, B: W.Csr):
    """Dense triple loop: for every (i, j), gather f over all k present in both."""
    pa, va = dense_of(A)
    pb, vb = dense_of(B)
    out = {}
    for i in range(A.nrows):
        for j in range(B.ncols):
            ks = [k for k in range(A.ncols) if pa[i, k] and pb[k, j]]
            if not ks:
                continue
            if alg in (O.PT_F32, O.PT_F64):
                terms = [float(va[i, k]) * float(vb[k, j]) for k in ks]
                out[(i, j)] = (math.fsum(terms), sum(abs(t) for t in terms))
            elif alg == O.MP_I32:
                out[(i, j)] = min(int(va[i, k]) + int(vb[k, j]) for k in ks)
            elif alg == O.MP_F32:
                out[(i, j)] = min(np.float32(va[i, k]) + np.float32(vb[k, j]) for k in ks)
            elif alg == O.BOOL:
                out[(i, j)] = int(any(bool(va[i, k]) and bool(vb[k, j]) for k in ks))
            elif alg == O.MULTPATH:
                cand = [(int(va[i, k]) + int(vb[k, j]["d"]), float(vb[k, j]["s"])) for k in ks]
                dmin = min(c[0] for c in cand)
                out[(i, j)] = (dmin, sum(c[1] for c in cand if c[0] == dmin))
    return out


def values_for(alg, nnz, seed, operand="A"):
    rng = np.random.default_rng(seed)
    if alg == O.PT_F32:
        return rng.standard_normal(nnz).astype(np.float32)
    if alg == O.PT_F64:
        return rng.standard_normal(nnz)
    if alg == O.MP_I32:
        return rng.integers(-50, 1000, nnz).astype(np.int32)
    if alg == O.MP_F32:
        return (rng.random(nnz) * 10 - 1).astype(np.float32)
    if alg == O.BOOL:
        return rng.integers(0, 2, nnz).astype(np.uint8)
    if alg == O.MULTPATH:
        if operand == "A":
            return rng.integers(1, 6, nnz).astype(np.int32)
        return W.multpath_values(nnz, 6, 4, seed)
    raise ValueError


def as_dict(ptr, col, val, rows=None, ab=None):
    out = {}
    nrow = ptr.size - 1
    for t in range(nrow):
        i = t if rows is None else int(rows[t])
        for p in range(ptr[t], ptr[t + 1]):
            out[(i, int(col[p]))] = (val[p], None if ab is None else ab[p])
    return out


ALL_ALGS = [O.PT_F32, O.PT_F64, O.MP_I32, O.MP_F32, O.BOOL, O.MULTPATH]


# ------------------------------------------------------------ SpGEMM

@pytest.mark.parametrize("alg", ALL_ALGS)
@pytest.mark.parametrize("shape", [(17, 23, 19), (24, 24, 24), (1, 5, 1), (9, 1, 7)])
def test_spgemm_vs_brute_force(alg, shape):
    m, k, n = shape
    for seed in range(3):
        A = W.random_csr(m, k, 6, seed * 7 + 1, empty_frac=0.2)
        B = W.random_csr(k, n, 6, seed * 7 + 2, empty_frac=0.2)
        A.val = values_for(alg, A.nnz, seed * 7 + 3, "A")
        B.val = values_for(alg, B.nnz, seed * 7 + 4, "B")
        ptr, col, val, ab = O.spgemm(alg, A, B, want_abs=True)
        # sorted ascending, unique inside each row
        for i in range(m):
            c = col[ptr[i]:ptr[i + 1]]
            assert np.all(np.diff(c) > 0)
        got = as_dict(ptr, col, val, ab=ab)
        exp = brute_force(alg, A, B)
        assert set(got) == set(exp)
        for key, e in exp.items():
            g, gabs = got[key]
            if alg in (O.PT_F32, O.PT_F64):
                assert abs(g - e[0]) <= 1e-14 * e[1] + 1e-300
                assert abs(gabs - e[1]) <= 1e-14 * e[1]
            elif alg == O.MP_F32:
                assert np.float32(g).tobytes() == np.float32(e).tobytes()
            elif alg == O.MULTPATH:
                assert int(g["d"]) == e[0] and float(g["s"]) == e[1]
            else:
                assert int(g) == int(e)


def _load_gold():
    ent = {}
    with open(os.path.join(GOLD, "hand_4x4.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            ent.setdefault(parts[0], []).append([int(x) for x in parts[1:]])
    return ent


def _csr4(entries, dtype):
    rows = np.array([e[0] for e in entries])
    cols = np.array([e[1] for e in entries])
    m = W.csr_from_coo(rows, cols, 4, 4)
    order = np.lexsort((cols, rows))
    if dtype is W.MULTPATH_DTYPE:
        v = np.zeros(len(entries), dtype=dtype)
        v["d"] = [entries[o][2] for o in order]
        v["s"] = [entries[o][3] for o in order]
    else:
        v = np.array([entries[o][2] for o in order]).astype(dtype)
    m.val = v
    return m


def test_spgemm_hand_worked_4x4():
    g = _load_gold()
    for alg, key, dt in [(O.MP_I32, "CMINPLUS", np.int32), (O.PT_F64, "CPLUSTIMES", np.float64),
                         (O.PT_F32, "CPLUSTIMES", np.float32), (O.BOOL, "CMINPLUS", np.uint8)]:
        A = _csr4(g["A"], dt if alg != O.BOOL else np.int64)
        if alg == O.BOOL:
            A.val = np.ones(A.nnz, np.uint8)
        ptr, col, val, _ = O.spgemm(alg, A, A)
        got = {(i, int(col[p])): val[p] for i in range(4) for p in range(ptr[i], ptr[i + 1])}
        exp = {(e[0], e[1]): e[2] for e in g[key]}
        assert set(got) == set(exp), alg
        for kk, v in exp.items():
            assert (got[kk] == 1) if alg == O.BOOL else (got[kk] == v), (alg, kk)
    A = _csr4(g["A"], np.int32)
    B = _csr4(g["BMULT"], W.MULTPATH_DTYPE)
    ptr, col, val, _ = O.spgemm(O.MULTPATH, A, B)
    got = {(i, int(col[p])): (int(val[p]["d"]), float(val[p]["s"])) for i in range(4)
           for p in range(ptr[i], ptr[i + 1])}
    exp = {(e[0], e[1]): (e[2], float(e[3])) for e in g["CMULT"]}
    assert got == exp


def test_spgemm_plus_times_matches_scipy_rmat():
    A = W.rmat(10, seed=3)
    A.val = W.weights_unit01(A.nnz, 4)
    S = sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.nrows, A.ncols))
    R = (S @ S).tocsr()
    R.sort_indices()
    ptr, col, val, _ = O.spgemm(O.PT_F64, A, A)
    assert np.array_equal(ptr, R.indptr) and np.array_equal(col, R.indices)
    assert np.max(np.abs(val - R.data) / R.data) < 1e-13
    ptr32, col32, val32, _ = O.spgemm(O.PT_F32, A.with_val(A.val.astype(np.float32)),
                                      A.with_val(A.val.astype(np.float32)))
    assert np.array_equal(col32, col) and np.max(np.abs(val32 - R.data) / R.data) < 1e-13


def test_spgemm_ones_counts_two_paths():
    """With all values 1, C_ij under (+,x) is the number of 2-step paths i->k->j."""
    A = W.random_csr(30, 30, 8, 11)
    A.val = np.ones(A.nnz)
    pa, _ = dense_of(A)
    paths = pa.astype(np.int64) @ pa.astype(np.int64)
    ptr, col, val, _ = O.spgemm(O.PT_F64, A, A)
    for i in range(30):
        for p in range(ptr[i], ptr[i + 1]):
            assert val[p] == paths[i, col[p]]
    assert (ptr[-1]) == np.count_nonzero(paths)


def test_spgemm_structure_same_for_all_algebras_and_counts():
    A = W.random_csr(40, 40, 7, 5, empty_frac=0.1)
    counts = O.spgemm_count(A, A)
    pa, _ = dense_of(A)
    struct = (pa.astype(np.int64) @ pa.astype(np.int64)) > 0
    assert np.array_equal(counts, struct.sum(axis=1))
    cols = None
    for alg in ALL_ALGS:
        A.val = values_for(alg, A.nnz, 1, "A")
        B = A.with_val(values_for(alg, A.nnz, 2, "B"))
        ptr, col, _, _ = O.spgemm(alg, A, B)
        if cols is None:
            cols = (ptr, col)
        assert np.array_equal(ptr, cols[0]) and np.array_equal(col, cols[1])


def test_spgemm_row_subset_matches_full():
    A = W.rmat(9, seed=2)
    A.val = W.weights_unit01(A.nnz, 5)
    full = O.spgemm(O.PT_F64, A, A)
    rows = np.array([5, 0, 511, 17, 17, 100])
    sub = O.spgemm(O.PT_F64, A, A, rows=rows)
    for t, i in enumerate(rows):
        a = slice(full[0][i], full[0][i + 1])
        b = slice(sub[0][t], sub[0][t + 1])
        assert np.array_equal(full[1][a], sub[1][b]) and np.array_equal(full[2][a], sub[2][b])


def test_tropical_identity_matrix_is_neutral():
    """I (x) A = A with I holding the multiplicative identity 0 on the diagonal only."""
    A = W.random_csr(25, 25, 6, 9)
    A.val = values_for(O.MP_I32, A.nnz, 3)
    I = W.csr_from_coo(np.arange(25), np.arange(25), 25, 25)
    I.val = np.zeros(25, np.int32)
    ptr, col, val, _ = O.spgemm(O.MP_I32, I, A)
    assert np.array_equal(ptr, A.rowptr) and np.array_equal(col, A.col) and np.array_equal(val, A.val)
    ptr, col, val, _ = O.spgemm(O.MP_I32, A, I)
    assert np.array_equal(col, A.col) and np.array_equal(val, A.val)


def test_path_doubling_closure_equals_floyd_warshall_and_scipy():
    """Repeated squaring of (I + A) over (min,+) reaches the all-pairs distances."""
    n = 40
    A = W.random_csr(n, n, 3, 21)
    A.val = np.random.default_rng(1).integers(1, 100, A.nnz).astype(np.int32)
    # I + A : add the zero diagonal (min with existing diagonal)
    pa, va = dense_of(A)
    D = np.full((n, n), O.TROP_I32_ID, np.int32)
    D[pa] = va[pa]
    np.fill_diagonal(D, np.minimum(np.diag(D), 0))
    rows, cols = np.nonzero(D < O.TROP_I32_ID)
    M = W.csr_from_coo(rows, cols, n, n)
    M.val = D[rows, cols].astype(np.int32)
    l = 1
    while l < n:
        ptr, col, val, _ = O.spgemm(O.MP_I32, M, M)
        M = W.Csr(n, n, ptr, col, val)
        l <<= 1
    pm, vm = dense_of(M)
    closure = np.where(pm, vm, O.TROP_I32_ID)
    fw = O.floyd_warshall_i32(D)
    assert np.array_equal(closure, fw)
    S = sp.csr_matrix((A.val.astype(np.float64), A.col, A.rowptr), shape=(n, n))
    ref = csgraph.floyd_warshall(S, directed=True)
    ref = np.where(np.isinf(ref), O.TROP_I32_ID, ref).astype(np.int64)
    assert np.array_equal(fw.astype(np.int64), ref)


def test_boolean_structure_matches_scipy():
    A = W.rmat(9, seed=7)
    A.val = np.ones(A.nnz, np.uint8)
    S = sp.csr_matrix((np.ones(A.nnz), A.col, A.rowptr), shape=(A.nrows, A.ncols))
    R = (S @ S).tocsr()
    R.sort_indices()
    ptr, col, val, _ = O.spgemm(O.BOOL, A, A)
    assert np.array_equal(ptr, R.indptr) and np.array_equal(col, R.indices) and np.all(val == 1)


# ------------------------------------------------------------ SpMM / SpMV

@pytest.mark.parametrize("alg", ALL_ALGS)
def test_spmm_vs_brute_force(alg):
    A = W.random_csr(13, 11, 5, 31, empty_frac=0.2)
    A.val = values_for(alg, A.nnz, 32, "A")
    ncol = 3
    Xf = W.Csr(11, ncol, np.arange(0, 11 * ncol + 1, ncol, dtype=np.int64),
               np.tile(np.arange(ncol, dtype=np.int32), 11),
               values_for(alg, 11 * ncol, 33, "B"))
    X = Xf.val.reshape(11, ncol)
    Y = O.spmm(alg, A, X)
    exp = brute_force(alg, A, Xf)
    for i in range(13):
        for c in range(ncol):
            e = exp.get((i, c))
            y = Y[i, c]
            if alg == O.PT_F32:
                ref = 0.0 if e is None else e[0]
                assert y == np.float32(ref) or abs(float(y) - ref) <= 2e-7 * (e[1] if e else 0) + 1e-30
            elif alg == O.PT_F64:
                ref = 0.0 if e is None else e[0]
                assert abs(y - ref) <= 1e-14 * (e[1] if e else 0)
            elif alg == O.MP_I32:
                assert y == (O.TROP_I32_ID if e is None else e)
            elif alg == O.MP_F32:
                assert y == (INF32 if e is None else e)
            elif alg == O.BOOL:
                assert y == (0 if e is None else e)
            else:
                if e is None:
                    assert y["d"] == O.TROP_I32_ID and y["s"] == 0
                else:
                    assert (int(y["d"]), float(y["s"])) == e
    # accumulate: Y0 (+) A(x)X equals elementwise (+) of Y0 and the plain result
    if alg == O.MP_I32:
        Y0 = np.random.default_rng(4).integers(0, 2000, (13, ncol)).astype(np.int32)
        assert np.array_equal(O.spmm(alg, A, X, Y0), np.minimum(Y0, Y))


def test_spmv_matches_scipy_plus_times():
    A = W.rmat(11, seed=4)
    A.val = W.weights_unit01(A.nnz, 1)
    x = np.random.default_rng(0).standard_normal(A.ncols)
    S = sp.csr_matrix((A.val, A.col, A.rowptr), shape=(A.nrows, A.ncols))
    y = O.spmv(O.PT_F64, A, x)
    assert np.allclose(y, S @ x, rtol=1e-13, atol=1e-13)


# ------------------------------------------------------------ Bellman-Ford / Dijkstra

def test_bellman_ford_matches_scipy_and_dijkstra_int():
    G = W.rmat(12, seed=5)
    G.val = W.weights_int(G.nnz, 1, 1000, 6)
    d, rounds = O.bellman_ford(O.MP_I32, G, 0)
    S = sp.csr_matrix((G.val.astype(np.float64), G.col, G.rowptr), shape=(G.nrows, G.ncols))
    ref = csgraph.dijkstra(S, directed=True, indices=0)
    ref = np.where(np.isinf(ref), O.TROP_I32_ID, ref).astype(np.int64)
    assert np.array_equal(d.astype(np.int64), ref)
    assert np.array_equal(O.dijkstra(O.MP_I32, G, 0), d)
    assert rounds > 0


def test_bellman_ford_fp32_bits_equal_dijkstra():
    G = W.rmat(12, seed=8)
    G.val = W.weights_unit01(G.nnz, 9).astype(np.float32)
    d, rounds = O.bellman_ford(O.MP_F32, G, 0)
    dj = O.dijkstra(O.MP_F32, G, 0)
    assert d.tobytes() == dj.tobytes()
    S = sp.csr_matrix((G.val.astype(np.float64), G.col, G.rowptr), shape=(G.nrows, G.ncols))
    ref = csgraph.dijkstra(S, directed=True, indices=0)
    fin = np.isfinite(ref)
    assert np.array_equal(np.isfinite(d), fin)
    assert np.max(np.abs(d[fin] - ref[fin]) / np.maximum(ref[fin], 1e-30)) < 1e-5


def test_bellman_ford_line_graph_closed_form():
    n = 50
    G = W.csr_from_coo(np.arange(n - 1), np.arange(1, n), n, n)
    G.val = np.full(n - 1, 3, np.int32)
    d, rounds = O.bellman_ford(O.MP_I32, G, 0)
    assert np.array_equal(d, 3 * np.arange(n)) and rounds == n - 1
    d, rounds = O.bellman_ford(O.MP_I32, G, 10)
    assert np.all(d[:10] == O.TROP_I32_ID) and np.array_equal(d[10:], 3 * np.arange(n - 10))
    G.val = np.full(n - 1, 0.5, np.float32)
    d, _ = O.bellman_ford(O.MP_F32, G, 0)
    assert np.array_equal(d, 0.5 * np.arange(n, dtype=np.float32))


def test_bellman_ford_negative_weights_and_cycle():
    # negative edges without a negative cycle: compare with scipy's Bellman-Ford
    n = 60
    G = W.random_csr(n, n, 3, 13)
    rng = np.random.default_rng(2)
    pa, _ = dense_of(G)
    pot = rng.integers(0, 50, n)
    rows = np.repeat(np.arange(n), np.diff(G.rowptr))
    G.val = (rng.integers(1, 20, G.nnz) + pot[G.col] - pot[rows]).astype(np.int32)  # reduced costs
    d, rounds = O.bellman_ford(O.MP_I32, G, 0)
    S = sp.csr_matrix((G.val.astype(np.float64), G.col, G.rowptr), shape=(n, n))
    ref = csgraph.bellman_ford(S, directed=True, indices=0)
    ref = np.where(np.isinf(ref), O.TROP_I32_ID, ref).astype(np.int64)
    assert rounds >= 0 and np.array_equal(d.astype(np.int64), ref)
    # a reachable negative cycle: 0 -> 1 -> 2 -> 1 with 1->2->1 summing to -1
    C = W.csr_from_coo([0, 1, 2], [1, 2, 1], 3, 3)
    C.val = np.array([4, 2, -3], np.int32)
    _, r = O.bellman_ford(O.MP_I32, C, 0)
    assert r == -1
    # unreachable negative cycle does not fail
    _, r = O.bellman_ford(O.MP_I32, W.csr_from_coo([1, 2], [2, 1], 3, 3).with_val(np.array([2, -3], np.int32)), 0)
    assert r == 0


# ------------------------------------------------------------ Brandes

def _nx_graph(G: W.Csr, weighted):
    g = nx.DiGraph()
    g.add_nodes_from(range(G.nrows))
    rows = np.repeat(np.arange(G.nrows), np.diff(G.rowptr))
    for u, v, w in zip(rows.tolist(), G.col.tolist(), (G.val if weighted else np.ones(G.nnz)).tolist()):
        g.add_edge(u, v, weight=w)
    return g


@pytest.mark.parametrize("weighted", [False, True])
def test_brandes_matches_networkx(weighted):
    G = W.rmat(8, seed=12)
    G.val = W.weights_int(G.nnz, 1, 5, 13)
    allsrc = np.arange(G.nrows, dtype=np.int32)
    bc = O.brandes(G, allsrc, weighted)
    ref = nx.betweenness_centrality(_nx_graph(G, weighted), normalized=False,
                                    weight="weight" if weighted else None)
    ref = np.array([ref[v] for v in range(G.nrows)])
    assert np.allclose(bc, ref, rtol=1e-12, atol=1e-9)
    # a source subset equals the sum of single-source dependencies
    srcs = W.sample_sources(G, 20, 0)
    sub = nx.betweenness_centrality_subset(_nx_graph(G, weighted), sources=srcs.tolist(),
                                           targets=list(range(G.nrows)), normalized=False,
                                           weight="weight" if weighted else None)
    sub = np.array([sub[v] for v in range(G.nrows)])
    assert np.allclose(O.brandes(G, srcs, weighted), sub, rtol=1e-12, atol=1e-9)


def test_brandes_all_pairs_definition_small():
    """BC(v) = sum over s != v != t of sigma_sv * sigma_vt / sigma_st on shortest paths."""
    n = 24
    G = W.random_csr(n, n, 4, 17)
    G.val = np.random.default_rng(5).integers(1, 4, G.nnz).astype(np.int32)
    pa, va = dense_of(G)
    INF = 10 ** 9
    D = np.full((n, n), INF, np.int64)
    D[pa] = va[pa]
    np.fill_diagonal(D, 0)
    for k in range(n):
        D = np.minimum(D, D[:, k:k + 1] + D[k:k + 1, :])
    # path counts sigma[s, t] by increasing distance
    sig = np.zeros((n, n))
    for s in range(n):
        sig[s, s] = 1
        for t in sorted(range(n), key=lambda t: D[s, t]):
            if t == s or D[s, t] >= INF:
                continue
            sig[s, t] = sum(sig[s, u] for u in range(n) if pa[u, t] and D[s, u] + va[u, t] == D[s, t])
    bc = np.zeros(n)
    for v in range(n):
        for s in range(n):
            for t in range(n):
                if len({s, v, t}) < 3 or D[s, t] >= INF:
                    continue
                if D[s, v] + D[v, t] == D[s, t]:
                    bc[v] += sig[s, v] * sig[v, t] / sig[s, t]
    got = O.brandes(G, np.arange(n, dtype=np.int32), True)
    assert np.allclose(got, bc, rtol=1e-12, atol=1e-12)
    d, s = O.sssp_counts(G, 3, True)
    fin = D[3] < INF
    assert np.array_equal(d[fin], D[3][fin]) and np.all(d[~fin] == -1)
    assert np.array_equal(s, sig[3])


def test_brandes_closed_forms():
    m = 9  # star, both directions: centre lies on every leaf-to-leaf path
    rows = np.r_[np.zeros(m, int), np.arange(1, m + 1)]
    cols = np.r_[np.arange(1, m + 1), np.zeros(m, int)]
    G = W.csr_from_coo(rows, cols, m + 1, m + 1)
    bc = O.brandes(G, np.arange(m + 1, dtype=np.int32), False)
    assert bc[0] == m * (m - 1) and np.all(bc[1:] == 0)
    n = 12  # directed path 0 -> 1 -> ... -> n-1
    P = W.csr_from_coo(np.arange(n - 1), np.arange(1, n), n, n)
    bc = O.brandes(P, np.arange(n, dtype=np.int32), False)
    assert np.array_equal(bc, np.array([v * (n - 1 - v) for v in range(n)], float))
