"""All-pairs shortest paths by path doubling (repeated (min,+) squaring of I + G)
through the C ABI against the oracle's Floyd-Warshall, entry by entry (exact)."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu

INF = O.TROP_I32_ID


@pytest.fixture(scope="module")
def H():
    need_gpu()
    import paper_1512_00066_b300 as stc
    return stc.Handle()


def dense_lengths(G):
    """I + G as a dense matrix, the identity where there is no edge."""
    n = G.nrows
    D = np.full((n, n), INF, np.int32)
    rows = np.repeat(np.arange(n), np.diff(G.rowptr))
    D[rows, G.col] = G.val
    np.fill_diagonal(D, np.minimum(np.diag(D), 0))
    return D


def check(H, G, tiskin=False):
    if tiskin:
        P, sq, _ = H.apsp_tiskin(to_dev(G))
    else:
        P, sq = H.apsp(to_dev(G))
    rp, col, val = P.to_host()
    n = G.nrows
    got = np.full((n, n), INF, np.int32)
    rows = np.repeat(np.arange(n), np.diff(rp))
    got[rows, col] = val
    ref = O.floyd_warshall_i32(dense_lengths(G))
    assert np.array_equal(got, ref)
    # only reachable pairs are stored
    assert P.nnz == int((ref < INF).sum())
    return sq


def test_sparse_random_graph(H):
    G = W.random_csr(600, 600, 6, seed=81, empty_frac=0.1)
    G.val = W.weights_int(G.nnz, 1, 1000, seed=82)
    sq = check(H, G)
    assert 1 <= sq <= 11


def test_paper_workload_dense_2048(H):
    """The paper's APSP workload: dense graph, n = 2048, lengths U[1, n^2]."""
    n = 2048
    rng = np.random.default_rng(83)
    rows = np.repeat(np.arange(n), n)
    cols = np.tile(np.arange(n), n)
    keep = rows != cols
    G = W.csr_from_coo(rows[keep], cols[keep], n, n)
    G.val = rng.integers(1, n * n + 1, G.nnz).astype(np.int32)
    check(H, G)


def test_negative_lengths_without_negative_cycle(H):
    n = 400
    G = W.random_csr(n, n, 5, seed=84)
    rng = np.random.default_rng(85)
    pot = rng.integers(0, 100, n)
    rows = np.repeat(np.arange(n), np.diff(G.rowptr))
    G.val = (rng.integers(1, 50, G.nnz) + pot[G.col] - pot[rows]).astype(np.int32)
    assert (G.val < 0).any()
    check(H, G)


def test_negative_cycle_and_edge_cases(H):
    import paper_1512_00066_b300 as stc
    C = W.csr_from_coo([0, 1, 2, 3], [1, 2, 1, 0], 4, 4)
    C.val = np.array([4, 2, -3, 1], np.int32)
    with pytest.raises(stc.StcError) as e:
        H.apsp(to_dev(C))
    assert e.value.status == 7
    # the handle stays usable; a graph with no edges gives the zero diagonal
    E = W.Csr(5, 5, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32))
    P, sq = H.apsp(to_dev(E))
    rp, col, val = P.to_host()
    assert np.array_equal(col, np.arange(5)) and np.all(val == 0)
    # a directed path: the closure is the upper triangle
    n = 50
    L = W.csr_from_coo(np.arange(n - 1), np.arange(1, n), n, n)
    L.val = np.full(n - 1, 3, np.int32)
    sq = check(H, L)
    assert sq <= 7  # 2^6 >= 49 hops, plus the squaring that changes nothing
    R = W.random_csr(6, 7, 2, seed=1)
    R.val = np.ones(R.nnz, np.int32)
    with pytest.raises(stc.StcError) as e:
        H.apsp(to_dev(R))
    assert e.value.status == 2


# ----------------------------------------------------------------- Tiskin's path doubling

def test_tiskin_sparse_and_negative_lengths(H):
    G = W.random_csr(600, 600, 6, seed=91, empty_frac=0.1)
    G.val = W.weights_int(G.nnz, 1, 1000, seed=92)
    check(H, G, tiskin=True)
    n = 400
    N = W.random_csr(n, n, 5, seed=93)
    rng = np.random.default_rng(94)
    pot = rng.integers(0, 100, n)
    rows = np.repeat(np.arange(n), np.diff(N.rowptr))
    N.val = (rng.integers(1, 50, N.nnz) + pot[N.col] - pot[rows]).astype(np.int32)
    check(H, N, tiskin=True)


def test_tiskin_paper_workload_fewer_products(H):
    """Dense n = 2048, lengths U[1, n^2]: the same distances as Floyd-Warshall with
    fewer path products than dense path doubling (n^3 per squaring)."""
    n = 2048
    rng = np.random.default_rng(95)
    rows = np.repeat(np.arange(n), n)
    cols = np.tile(np.arange(n), n)
    keep = rows != cols
    G = W.csr_from_coo(rows[keep], cols[keep], n, n)
    G.val = rng.integers(1, n * n + 1, G.nnz).astype(np.int32)
    check(H, G, tiskin=True)
    _, rounds, prods = H.apsp_tiskin(to_dev(G))
    _, sq = H.apsp(to_dev(G))
    assert 0 < prods < sq * n ** 3


def test_tiskin_cycles_and_long_paths(H):
    import paper_1512_00066_b300 as stc
    C = W.csr_from_coo([0, 1, 2, 3], [1, 2, 1, 0], 4, 4)
    C.val = np.array([4, 2, -3, 1], np.int32)
    with pytest.raises(stc.StcError) as e:
        H.apsp_tiskin(to_dev(C))
    assert e.value.status == 7
    # a directed path of 300 vertices plus shortcuts (many least paths of equal weight)
    n = 300
    r = np.r_[np.arange(n - 1), np.arange(0, n - 3, 3)]
    c = np.r_[np.arange(1, n), np.arange(3, n, 3)]
    L = W.csr_from_coo(r, c, n, n)
    rows = np.repeat(np.arange(n), np.diff(L.rowptr))
    L.val = np.where(L.col - rows == 3, 6, 2).astype(np.int32)
    check(H, L, tiskin=True)
