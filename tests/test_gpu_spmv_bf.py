"""GPU SpMV / SpMM and Bellman-Ford through the C ABI against the CPU oracle."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from gpu_util import compare_values, dsig_from_raw, need_gpu, to_dev

pytestmark = pytest.mark.gpu

ALL = [O.PT_F32, O.PT_F64, O.MP_I32, O.MP_F32, O.BOOL, O.MULTPATH]


@pytest.fixture(scope="module")
def H():
    need_gpu()
    import paper_1512_00066_b300 as stc
    return stc.Handle()


def dense_vals(alg, shape, seed):
    rng = np.random.default_rng(seed)
    n = int(np.prod(shape))
    if alg == O.PT_F32:
        return rng.standard_normal(n).astype(np.float32).reshape(shape)
    if alg == O.PT_F64:
        return rng.standard_normal(n).reshape(shape)
    if alg == O.MP_I32:
        return rng.integers(0, 5000, n).astype(np.int32).reshape(shape)
    if alg == O.MP_F32:
        return (rng.random(n) * 50).astype(np.float32).reshape(shape)
    if alg == O.BOOL:
        return rng.integers(0, 2, n).astype(np.uint8).reshape(shape)
    return W.multpath_values(n, 30, 6, seed).reshape(shape)


def a_vals(alg, nnz, seed):
    rng = np.random.default_rng(seed)
    if alg in (O.PT_F32,):
        return rng.standard_normal(nnz).astype(np.float32)
    if alg == O.PT_F64:
        return rng.standard_normal(nnz)
    if alg in (O.MP_I32, O.MULTPATH):
        return rng.integers(1, 100, nnz).astype(np.int32)
    if alg == O.MP_F32:
        return rng.random(nnz).astype(np.float32)
    return rng.integers(0, 2, nnz).astype(np.uint8)


def dev_dense(alg, X):
    if alg == O.MULTPATH:
        raw = np.ascontiguousarray(X).view(np.uint8).reshape(X.shape + (16,))
        return torch.from_numpy(raw.copy()).cuda()
    return torch.from_numpy(np.ascontiguousarray(X)).cuda()


def host_out(alg, Y):
    y = Y.cpu().numpy()
    if alg == O.MULTPATH:
        return dsig_from_raw(y).reshape(y.shape[:-1])
    return y


@pytest.mark.parametrize("alg", ALL)
@pytest.mark.parametrize("ncol", [1, 5, 37, 300])
@pytest.mark.parametrize("accumulate", [False, True])
def test_spmm_all_algebras(H, alg, ncol, accumulate):
    A = W.random_csr(2049, 1500, 70, seed=11, empty_frac=0.1)
    A.val = a_vals(alg, A.nnz, 12)
    shape = (1500,) if ncol == 1 else (1500, ncol)
    X = dense_vals(alg, shape, 13)
    Y0 = dense_vals(alg, (2049,) if ncol == 1 else (2049, ncol), 14) if accumulate else None
    Yd = dev_dense(alg, Y0) if accumulate else None
    Y = H.spmm(alg, to_dev(A), dev_dense(alg, X), Yd, accumulate=accumulate)
    torch.cuda.synchronize()
    H.check_device_status()
    got = host_out(alg, Y)
    ref = O.spmm(alg, A, X, Y0)
    if alg in (O.PT_F32, O.PT_F64):
        # bound relative to the sum of |terms| (signed values cancel)
        absA = A.with_val(np.abs(A.val).astype(np.float64))
        absX = np.abs(X).astype(np.float64)
        scale = O.spmm(O.PT_F64, absA, absX, None if Y0 is None else np.abs(Y0).astype(np.float64))
        tol = 1e-12 if alg == O.PT_F64 else 1e-5
        assert np.all(np.abs(got.astype(np.float64) - ref.astype(np.float64)) <= tol * np.abs(ref) + 1e-14 * scale + 1e-30)
    elif alg == O.MULTPATH:
        assert np.array_equal(got["d"], ref["d"]) and np.array_equal(got["s"], ref["s"])
    else:
        assert got.tobytes() == ref.tobytes()


@pytest.mark.parametrize("persistent", [True, False, "graph"])
def test_bellman_ford_rmat14(H, persistent):
    G = W.rmat(14, seed=21)
    G.val = W.weights_int(G.nnz, 1, 1000, 22)
    d, r = H.bellman_ford(O.MP_I32, to_dev(G), 0, persistent=persistent)
    ref, rref = O.bellman_ford(O.MP_I32, G, 0)
    assert np.array_equal(d.cpu().numpy(), ref)
    assert 1 <= r <= rref
    G.val = W.weights_unit01(G.nnz, 23).astype(np.float32)
    d, r = H.bellman_ford(O.MP_F32, to_dev(G), 0, persistent=persistent)
    ref, rref = O.bellman_ford(O.MP_F32, G, 0)
    assert d.cpu().numpy().tobytes() == ref.tobytes()
    assert 1 <= r <= rref


def test_bellman_ford_rmat18_full_size(H):
    """R-MAT scale 18 from vertex 0, (min,+) fp32, persistent launch: bit-exact."""
    G = W.rmat(18, seed=0)
    G.val = W.weights_unit01(G.nnz, seed=1).astype(np.float32)
    d, r = H.bellman_ford(O.MP_F32, to_dev(G), 0, persistent=True)
    ref = O.dijkstra(O.MP_F32, G, 0)
    assert d.cpu().numpy().tobytes() == ref.tobytes()
    d2, r2 = H.bellman_ford(O.MP_F32, to_dev(G), 0, persistent=False)
    assert d2.cpu().numpy().tobytes() == ref.tobytes()
    d3, r3 = H.bellman_ford(O.MP_F32, to_dev(G), 0, persistent="graph")
    assert d3.cpu().numpy().tobytes() == ref.tobytes()


def test_bellman_ford_closed_forms_and_cycles(H):
    import paper_1512_00066_b300 as stc
    n = 1000
    L = W.csr_from_coo(np.arange(n - 1), np.arange(1, n), n, n)
    L.val = np.full(n - 1, 7, np.int32)
    for persistent in (True, False, "graph"):
        d, r = H.bellman_ford(O.MP_I32, to_dev(L), 0, persistent=persistent)
        assert np.array_equal(d.cpu().numpy(), 7 * np.arange(n)) and r == n - 1
        d, r = H.bellman_ford(O.MP_I32, to_dev(L), 500, persistent=persistent)
        assert np.all(d.cpu().numpy()[:500] == O.TROP_I32_ID)
    # negative weights, no negative cycle
    G = W.random_csr(3000, 3000, 4, seed=31)
    rng = np.random.default_rng(3)
    pot = rng.integers(0, 100, 3000)
    rows = np.repeat(np.arange(3000), np.diff(G.rowptr))
    G.val = (rng.integers(1, 50, G.nnz) + pot[G.col] - pot[rows]).astype(np.int32)
    ref, _ = O.bellman_ford(O.MP_I32, G, 0)
    for persistent in (True, False, "graph"):
        d, _ = H.bellman_ford(O.MP_I32, to_dev(G), 0, persistent=persistent)
        assert np.array_equal(d.cpu().numpy(), ref)
    # reachable negative cycle -> status
    C = W.csr_from_coo([0, 1, 2], [1, 2, 1], 3, 3)
    C.val = np.array([4, 2, -3], np.int32)
    for persistent in (True, False, "graph"):
        with pytest.raises(stc.StcError) as e:
            H.bellman_ford(O.MP_I32, to_dev(C), 0, persistent=persistent)
        assert e.value.status == 7
    # the handle stays usable
    d, _ = H.bellman_ford(O.MP_I32, to_dev(L), 0)
    assert np.array_equal(d.cpu().numpy(), 7 * np.arange(n))


def test_bellman_ford_graph_is_reused_across_calls(H):
    """The graph driver instantiates its CUDA graph once per handle and algebra and
    rewrites only its parameter block per call: graphs of different sizes, both
    algebras interleaved, many sources in a row, each call against the oracle.
    A graph with a negative cycle in between leaves later calls correct."""
    cases = []
    for scale, seed in ((10, 31), (13, 32), (8, 33)):
        G = W.rmat(scale, seed=seed)
        gi = G.with_val(W.weights_int(G.nnz, 1, 100, seed + 1))
        gf = G.with_val(W.weights_unit01(G.nnz, seed + 2).astype(np.float32))
        cases.append((gi, to_dev(gi), gf, to_dev(gf), W.sample_sources(G, 4, seed=seed + 3)))
    n = 50
    C = W.csr_from_coo(np.arange(n), (np.arange(n) + 1) % n, n, n)
    C.val = np.full(n, -1, np.int32)
    for rep in range(2):
        for gi, dgi, gf, dgf, srcs in cases:
            for v in srcs:
                d, _ = H.bellman_ford(O.MP_I32, dgi, int(v), persistent="graph")
                ref, _ = O.bellman_ford(O.MP_I32, gi, int(v))
                assert np.array_equal(d.cpu().numpy(), ref)
                d, _ = H.bellman_ford(O.MP_F32, dgf, int(v), persistent="graph")
                ref, _ = O.bellman_ford(O.MP_F32, gf, int(v))
                assert d.cpu().numpy().tobytes() == ref.tobytes()
        if rep == 0:
            import paper_1512_00066_b300 as stc
            with pytest.raises(stc.StcError) as e:
                H.bellman_ford(O.MP_I32, to_dev(C), 0, persistent="graph")
            assert e.value.status == 7


def test_bellman_ford_drivers_are_distinct(H):
    """Each driver runs its own launch pattern: the host loop launches one kernel
    per round, the cooperative form one kernel in all, and the graph form counts
    the two kernels of its WHILE body once (the device repeats them)."""
    n = 1000
    L = W.csr_from_coo(np.arange(n - 1), np.arange(1, n), n, n)
    L.val = np.full(n - 1, 7, np.int32)
    G = to_dev(L)
    launches = {}
    for persistent in (True, False, "graph"):
        k0 = H.kernel_launches()
        d, r = H.bellman_ford(O.MP_I32, G, 0, persistent=persistent)
        launches[persistent] = H.kernel_launches() - k0
        assert np.array_equal(d.cpu().numpy(), 7 * np.arange(n)) and r == n - 1
    assert launches["graph"] == launches[True] + 1
    assert launches[False] >= launches[True] + n - 2


def test_bounded_barrier_times_out_with_a_status(H):
    """A grid barrier waiting for a block that never arrives gives up after its
    poll limit: the call returns STC_ERR_TIMEOUT (8), no kernel hangs, and the
    handle keeps working."""
    assert H.selftest_barrier(0) == 0
    assert H.selftest_barrier(1, spin_limit=4096) == 8
    assert H.selftest_barrier(0) == 0
    n = 500
    L = W.csr_from_coo(np.arange(n - 1), np.arange(1, n), n, n)
    L.val = np.full(n - 1, 3, np.int32)
    d, r = H.bellman_ford(O.MP_I32, to_dev(L), 0, persistent=True)
    assert np.array_equal(d.cpu().numpy(), 3 * np.arange(n)) and r == n - 1


def test_spmm_paper_e1_shape_sampled(H):
    """The paper's SpMM shape: a 16384 x 16384 sparse matrix with independent 1%
    density times a dense 16384 x 8192 block, fp64, at full size: 64 sampled rows
    element by element against the oracle (run on those rows of A)."""
    n, k = 16384, 8192
    rng = np.random.default_rng(101)
    A = W.distinct_columns(rng, rng.binomial(n, 0.01, size=n), n)
    A.val = W.weights_unit01(A.nnz, 102)
    X = np.random.default_rng(103).random((n, k))
    Y = H.spmm(O.PT_F64, to_dev(A), torch.from_numpy(X).cuda())
    rows = np.unique(np.r_[np.random.default_rng(104).choice(n, 62, replace=False), 0, n - 1])
    sub_ptr = np.r_[0, np.cumsum(np.diff(A.rowptr)[rows])].astype(np.int64)
    sel = np.concatenate([np.arange(A.rowptr[i], A.rowptr[i + 1]) for i in rows])
    S = W.Csr(len(rows), n, sub_ptr, A.col[sel], A.val[sel])
    ref = O.spmm(O.PT_F64, S, X, None)
    got = Y[torch.from_numpy(rows).cuda()].cpu().numpy()
    assert np.all(np.abs(got - ref) <= 1e-12 * np.abs(ref))
