"""GPU betweenness centrality (multiplicity-monoid shortest paths + Brandes
accumulation) through the C ABI against the CPU oracle.

Forward distances and path counts are exact integers (fp64 counts below 2^53) and
must match bit for bit; centrality is held to relative 1e-12 (absolute 1e-9 on
entries the oracle gives as exactly zero).
"""
import functools

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


@functools.lru_cache(maxsize=2)
def _structure(scale, seed):
    return W.rmat(scale, seed=seed)


def graph(scale, seed, weighted):
    S = _structure(scale, seed)
    G = W.Csr(S.nrows, S.ncols, S.rowptr, S.col)
    G.val = W.weights_int(G.nnz, 1, 255, seed + 1) if weighted else None
    return G


def check_forward(H, G, sources, weighted):
    d, sig, rounds = H.mfbc_sssp(to_dev(G), sources)
    d = d.cpu().numpy()
    sig = sig.cpu().numpy()
    assert rounds >= 1
    for j, s in enumerate(sources):
        rd, rs = O.sssp_counts(G, int(s), weighted)
        exp_d = np.where(rd < 0, INF, rd)
        assert np.array_equal(d[:, j], exp_d), f"distances differ for source {s}"
        assert np.array_equal(sig[:, j], rs), f"path counts differ for source {s}"


def bc_close(got, ref):
    assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref) + 1e-9 * (ref == 0))


@pytest.mark.parametrize("weighted", [False, True])
def test_forward_exact_rmat12(H, weighted):
    G = graph(12, 3, weighted)
    src = W.sample_sources(G, 37, seed=4)  # ragged: not a multiple of 32
    check_forward(H, G, src, weighted)


@pytest.mark.parametrize("weighted", [False, True])
@pytest.mark.parametrize("batch", [256, 96])
def test_bc_matches_brandes_rmat12(H, weighted, batch):
    G = graph(12, 5, weighted)
    src = W.sample_sources(G, 300, seed=6)  # several batches, the last one partial
    bc = H.mfbc(to_dev(G), src, batch=batch).cpu().numpy()
    bc_close(bc, O.brandes(G, src, weighted))


def test_bc_all_sources_small_and_closed_forms(H):
    G = graph(9, 7, True)
    allsrc = np.arange(G.nrows, dtype=np.int32)
    bc = H.mfbc(to_dev(G), allsrc, batch=200).cpu().numpy()
    bc_close(bc, O.brandes(G, allsrc, True))
    m = 9  # star, both directions
    rows = np.r_[np.zeros(m, int), np.arange(1, m + 1)]
    cols = np.r_[np.arange(1, m + 1), np.zeros(m, int)]
    S = W.csr_from_coo(rows, cols, m + 1, m + 1)
    bc = H.mfbc(to_dev(S), np.arange(m + 1, dtype=np.int32)).cpu().numpy()
    assert bc[0] == m * (m - 1) and np.all(bc[1:] == 0)
    n = 12  # directed path
    P = W.csr_from_coo(np.arange(n - 1), np.arange(1, n), n, n)
    bc = H.mfbc(to_dev(P), np.arange(n, dtype=np.int32)).cpu().numpy()
    assert np.array_equal(bc, np.array([v * (n - 1 - v) for v in range(n)], float))


def test_equal_length_paths_multiply(H):
    """A ladder of k diamonds has 2^k shortest paths end to end."""
    k = 40
    rows, cols = [], []
    for i in range(k):
        a, b, c, d = 3 * i, 3 * i + 1, 3 * i + 2, 3 * i + 3
        rows += [a, a, b, c]
        cols += [b, c, d, d]
    n = 3 * k + 1
    G = W.csr_from_coo(rows, cols, n, n)
    G.val = np.full(G.nnz, 2, np.int32)
    d, sig, _ = H.mfbc_sssp(to_dev(G), [0])
    assert int(d[n - 1, 0]) == 4 * k and float(sig[n - 1, 0]) == 2.0 ** k


def test_invalid_lengths_are_rejected(H):
    import paper_1512_00066_b300 as stc
    G = graph(8, 9, True)
    G.val[5] = 0
    with pytest.raises(stc.StcError) as e:
        H.mfbc(to_dev(G), [0, 1])
    assert e.value.status == 1
    with pytest.raises(stc.StcError):
        H.mfbc(to_dev(G), [G.nrows])  # source out of range (host check)


def test_rmat22_full_size_forward_sampled(H):
    """R-MAT scale 22, int32 lengths U[1,255], a 256-source batch: distances and
    path counts of 4 of the sources against the oracle, element by element."""
    G = graph(22, 0, True)
    src = W.sample_sources(G, 256, seed=0)
    d, sig, rounds = H.mfbc_sssp(to_dev(G), src)
    for j in (0, 77, 150, 255):
        rd, rs = O.sssp_counts(G, int(src[j]), True)
        dj = d[:, j].cpu().numpy()
        sj = sig[:, j].cpu().numpy()
        assert np.array_equal(dj, np.where(rd < 0, INF, rd))
        assert np.array_equal(sj, rs)


@pytest.mark.parametrize("weighted", [False, True])
def test_rmat22_centrality_on_a_source_sample(H, weighted):
    """The centrality workload at full size: R-MAT scale 22 with unit lengths and
    with int32 lengths U[1,255], over 64 sources (every 64th of the seeded
    4096-source sample, in one batch of 64): every vertex's centrality against
    Brandes' algorithm (Section 4.2, geodetic semiring) within relative 1e-12."""
    G = graph(22, 0, weighted)
    src = W.sample_sources(G, 4096, seed=0)[::64]
    assert src.size == 64
    bc = H.mfbc(to_dev(G), src, batch=64).cpu().numpy()
    bc_close(bc, O.brandes(G, src, weighted))


@pytest.mark.parametrize("weighted", [False, True])
def test_round_drivers_agree(H, weighted):
    """Host-driven rounds and the one-graph-per-batch driver give identical
    results; the graph driver counts each of its nodes once per batch."""
    G = graph(12, 11, weighted)
    src = W.sample_sources(G, 70, seed=12)
    dG = to_dev(G)
    out = {}
    try:
        for drv in ("host", "graph"):
            H.set_round_driver(drv)
            k0 = H.kernel_launches()
            d, sig, rounds = H.mfbc_sssp(dG, src[:40])
            k1 = H.kernel_launches()
            bc = H.mfbc(dG, src, batch=32).cpu().numpy()  # 3 batches, the last one partial
            k2 = H.kernel_launches()
            out[drv] = (d.cpu().numpy(), sig.cpu().numpy(), rounds, bc, k1 - k0, k2 - k1)
    finally:
        H.set_round_driver("graph")
    h, g = out["host"], out["graph"]
    assert np.array_equal(h[0], g[0]) and np.array_equal(h[1], g[1]) and h[2] == g[2]
    bc_close(g[3], O.brandes(G, src, weighted))
    bc_close(h[3], g[3])
    # host: 5 kernels per forward round (3 with unit lengths: bitset push, update,
    # check); graph: one node each
    assert h[4] >= 2 + (5 if weighted else 3) * h[2] and g[4] < h[4]
    assert g[5] < h[5]


def test_unit_lengths_fall_back_when_the_bitset_kernels_give_up(H):
    """Unit lengths run on bitset frontiers, which keep every round's work items and
    at most 4096 rounds.  A path of 5000 vertices needs more rounds, and a cycle with
    sources all around it puts every vertex on hundreds of levels (more items than
    kept): both batches are recomputed by the general kernels, with the oracle's
    centrality and the exact distances and path counts."""
    n = 5000
    P = W.csr_from_coo(np.arange(n - 1), np.arange(1, n), n, n)
    src = np.array([0, 3, 4000], np.int32)
    bc_close(H.mfbc(to_dev(P), src).cpu().numpy(), O.brandes(P, src, False))
    check_forward(H, P, src, False)
    m = 600
    Cy = W.csr_from_coo(np.arange(m), (np.arange(m) + 1) % m, m, m)
    src = np.arange(0, m, 2, dtype=np.int32)[:256]
    bc_close(H.mfbc(to_dev(Cy), src).cpu().numpy(), O.brandes(Cy, src, False))
    check_forward(H, Cy, src[:100], False)


@pytest.mark.parametrize("driver", ["host", "graph"])
def test_unit_lengths_bitset_kernels_match_brandes_rmat14(H, driver):
    """The bitset-frontier path on a skewed graph, both round drivers, a ragged last
    batch: centrality against Brandes and forward distances/path counts exact."""
    G = graph(14, 21, False)
    src = W.sample_sources(G, 300, seed=22)
    try:
        H.set_round_driver(driver)
        bc = H.mfbc(to_dev(G), src, batch=128).cpu().numpy()
        check_forward(H, G, src[:70], False)
    finally:
        H.set_round_driver("graph")
    bc_close(bc, O.brandes(G, src, False))
