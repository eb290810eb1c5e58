"""GPU SpGEMM through the C ABI against the CPU oracle, element by element.

Integer, boolean, (min,+) and multiplicity results must be bit-exact; (+,x) is
held to rel 1e-12 (fp64) and rel 1e-5 (fp32 against the fp64 oracle).  The
output structure (row pointers and sorted columns) must be identical.
"""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from gpu_util import compare_values, need_gpu, to_dev

pytestmark = pytest.mark.gpu

ALL = [O.PT_F32, O.PT_F64, O.MP_I32, O.MP_F32, O.BOOL, O.MULTPATH]


@pytest.fixture(scope="module")
def H():
    need_gpu()
    import paper_1512_00066_b300 as stc
    return stc.Handle()


def vals(alg, nnz, seed, operand):
    rng = np.random.default_rng(seed)
    if alg == O.PT_F32:
        return rng.standard_normal(nnz).astype(np.float32)
    if alg == O.PT_F64:
        return rng.standard_normal(nnz)
    if alg == O.MP_I32:
        return rng.integers(-1000, 100000, nnz).astype(np.int32)
    if alg == O.MP_F32:
        return (rng.random(nnz) * 100 - 10).astype(np.float32)
    if alg == O.BOOL:
        return rng.integers(0, 2, nnz).astype(np.uint8)
    if operand == "A":
        return rng.integers(1, 8, nnz).astype(np.int32)
    return W.multpath_values(nnz, 20, 5, seed)


def check(H, alg, A, B, rows=None, window_cols=0, light_rows=0):
    C = H.spgemm(alg, to_dev(A), to_dev(B), window_cols=window_cols, light_rows=light_rows)
    torch.cuda.synchronize()
    H.check_device_status()
    rp, col, val = C.to_host()
    if rows is None:
        ptr, rcol, rval, rabs = O.spgemm(alg, A, B, want_abs=True)
        assert np.array_equal(rp, ptr), "row pointers differ"
        assert np.array_equal(col, rcol), "columns differ"
        compare_values(alg, val, rval, rabs, where=f"alg {alg}")
    else:
        counts = O.spgemm_count(A, B)
        assert np.array_equal(np.diff(rp), counts), "row counts differ"
        ptr, rcol, rval, rabs = O.spgemm(alg, A, B, rows=rows, want_abs=True)
        sel = np.concatenate([np.arange(rp[i], rp[i + 1]) for i in rows]) if len(rows) else np.zeros(0, int)
        assert np.array_equal(col[sel], rcol)
        v = val[sel] if alg != O.MULTPATH else val[sel]
        compare_values(alg, v, rval, rabs, where=f"alg {alg} sampled")
    return C


def test_er4096_min_plus_exact(H):
    """ER n=4096, exactly 8 distinct columns per row, int32 U[1,1000]: C = A (x) A."""
    A = W.er_fixed_degree(4096, 8, seed=0)
    A.val = W.weights_int(A.nnz, 1, 1000, seed=0)
    check(H, O.MP_I32, A, A)


@pytest.mark.parametrize("alg", ALL)
def test_random_rectangular_all_algebras(H, alg):
    A = W.random_csr(3001, 2500, 40, seed=1, empty_frac=0.1)
    B = W.random_csr(2500, 3999, 60, seed=2, empty_frac=0.1)
    A.val = vals(alg, A.nnz, 3, "A")
    B.val = vals(alg, B.nnz, 4, "B")
    check(H, alg, A, B)


@pytest.mark.parametrize("alg", ALL)
def test_small_windows_multi_window_path(H, alg):
    """Force 1024-column windows so every row spans several windows."""
    A = W.random_csr(700, 900, 80, seed=5, empty_frac=0.05)
    B = W.random_csr(900, 5000, 120, seed=6, empty_frac=0.05)
    A.val = vals(alg, A.nnz, 7, "A")
    B.val = vals(alg, B.nnz, 8, "B")
    check(H, alg, A, B, window_cols=1024)


@pytest.mark.parametrize("alg", ALL)
def test_wide_rows_many_rank_windows(H, alg):
    """Output rows with tens of thousands of entries: several rank windows per row."""
    A = W.random_csr(150, 300, 300, seed=15, empty_frac=0.05)
    B = W.random_csr(300, 60000, 400, seed=16)
    A.val = vals(alg, A.nnz, 17, "A")
    B.val = vals(alg, B.nnz, 18, "B")
    check(H, alg, A, B)


@pytest.mark.parametrize("alg", ALL)
def test_rmat14_square(H, alg):
    """R-MAT scale 14: hub rows longer than one chunk of A, several windows."""
    A = W.rmat(14, seed=3)
    A.val = vals(alg, A.nnz, 9, "A")
    B = A.with_val(vals(alg, A.nnz, 10, "B"))
    check(H, alg, A, B)


@pytest.mark.parametrize("alg", ALL)
@pytest.mark.parametrize("light", [8, 10])
def test_light_row_launch(H, alg, light):
    """Rows with fewer than 2^light products in their own launch of smaller CTAs
    on a second stream, beside the wide launch: R-MAT 14, all algebras."""
    A = W.rmat(14, seed=13)
    A.val = vals(alg, A.nnz, 19, "A")
    B = A.with_val(vals(alg, A.nnz, 20, "B"))
    check(H, alg, A, B, light_rows=light)


def test_autotuner_and_tuning_file(H, tmp_path):
    """The autotuner times its candidates, caches the fastest, and later calls
    with the default option give the same product; the cache survives a save and
    load, and a file for another device is refused."""
    import paper_1512_00066_b300 as stc
    A = W.rmat(13, seed=21)
    A.val = W.weights_unit01(A.nnz, 2).astype(np.float32)
    dA = to_dev(A)
    res = H.autotune_spgemm(O.PT_F32, dA, dA)
    assert res["best"] in res["candidates"] and -1 in res["candidates"] and len(res["candidates"]) >= 2
    assert all(t > 0 for t in res["candidates"].values())
    assert res["candidates"][res["best"]] == min(res["candidates"].values())
    C = H.spgemm(O.PT_F32, dA, dA)
    R = H.spgemm(O.PT_F32, dA, dA, light_rows=-1)
    assert np.array_equal(C.rowptr.cpu().numpy(), R.rowptr.cpu().numpy())
    assert np.array_equal(C.col.cpu().numpy(), R.col.cpu().numpy())
    assert np.allclose(C.val.cpu().numpy(), R.val.cpu().numpy(), rtol=1e-5)
    f = tmp_path / "tune.txt"
    H.tune_save(f)
    lines = f.read_text().splitlines()
    assert lines[0].startswith("stc-tune 1 ") and any(l.split()[:2] == [str(O.PT_F32), "13"] for l in lines[1:])
    H2 = stc.Handle()
    H2.tune_load(f)
    H2.tune_save(tmp_path / "tune2.txt")
    assert (tmp_path / "tune2.txt").read_text() == f.read_text()
    bad = tmp_path / "other.txt"
    bad.write_text("stc-tune 1 3 Some_Other_GPU\n1 13 8\n")
    with pytest.raises(stc.StcError):
        H2.tune_load(bad)
    bad.write_text(lines[0] + "\n1 13 0\n")
    with pytest.raises(stc.StcError):
        H2.tune_load(bad)


def test_rmat14_plus_times_unit_weights_relative(H):
    A = W.rmat(14, seed=4)
    A.val = W.weights_unit01(A.nnz, 1)
    for alg in (O.PT_F64, O.PT_F32):
        a = A.with_val(A.val.astype(np.float32 if alg == O.PT_F32 else np.float64))
        C = H.spgemm(alg, to_dev(a), to_dev(a))
        rp, col, val = C.to_host()
        ptr, rcol, rval, _ = O.spgemm(alg, a, a)
        assert np.array_equal(col, rcol)
        tol = 1e-12 if alg == O.PT_F64 else 1e-5
        assert np.max(np.abs(val.astype(np.float64) - rval) / rval) <= tol


@pytest.mark.parametrize("alg", ALL)
def test_wide_output_column_slabs(H, alg):
    """More than 2^18 output columns: three full column slabs and a ragged fourth."""
    A = W.random_csr(700, 1200, 30, seed=41, empty_frac=0.05)
    B = W.random_csr(1200, 3 * (1 << 18) + 12345, 150, seed=42, empty_frac=0.05)
    A.val = vals(alg, A.nnz, 43, "A")
    B.val = vals(alg, B.nnz, 44, "B")
    check(H, alg, A, B)


def test_column_slab_boundaries(H):
    """Entries on both sides of every slab boundary, single-entry rows of A (copy
    path) next to multi-entry rows, and rows whose products all fall in one slab."""
    W_ = 1 << 18
    ncols = 2 * W_ + 1
    edges = [0, W_ - 1, W_, 2 * W_ - 1, 2 * W_]
    rows, cols = [], []
    for k in range(40):
        picks = sorted(set([edges[k % 5], edges[(k + 2) % 5], (k * 7919) % ncols, (k * 104729) % ncols]))
        rows += [k] * len(picks)
        cols += picks
    B = W.csr_from_coo(np.array(rows), np.array(cols), 40, ncols)
    B.val = np.arange(1, B.nnz + 1, dtype=np.int32)
    arow = [0, 1, 1, 2, 2, 2] + [3 + i // 2 for i in range(30)]
    acol = [5, 0, 9, 1, 2, 3] + [(7 * i) % 40 for i in range(30)]
    A = W.csr_from_coo(np.array(arow), np.array(acol), 20, 40)
    A.val = np.arange(1, A.nnz + 1, dtype=np.int32)
    check(H, O.MP_I32, A, B)
    check(H, O.PT_F64, A.with_val(A.val.astype(np.float64)), B.with_val(B.val.astype(np.float64)))


def test_edge_cases(H):
    import paper_1512_00066_b300 as stc
    # empty A, empty B, 1x1, rows with ub == 0, single column
    empty = W.Csr(5, 7, np.zeros(6, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32))
    B = W.random_csr(7, 9, 3, seed=1)
    B.val = np.arange(B.nnz, dtype=np.int32)
    C = H.spgemm(O.MP_I32, to_dev(empty), to_dev(B))
    assert C.nnz == 0 and np.array_equal(C.rowptr.cpu().numpy(), np.zeros(6))
    one = W.Csr(1, 1, np.array([0, 1], np.int64), np.array([0], np.int32), np.array([3], np.int32))
    C = H.spgemm(O.MP_I32, to_dev(one), to_dev(one))
    assert C.to_host()[2].tolist() == [6]
    A = W.random_csr(50, 7, 3, seed=2, empty_frac=0.5)
    A.val = np.ones(A.nnz, np.int32)
    Bz = W.Csr(7, 1, np.zeros(8, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32))
    C = H.spgemm(O.MP_I32, to_dev(A), to_dev(Bz))
    assert C.nnz == 0
    col1 = W.random_csr(7, 1, 1, seed=3)
    col1.val = np.arange(col1.nnz, dtype=np.int32) + 1
    check(H, O.MP_I32, A, col1)
    # columns 0 and n-1 present
    n = 300
    E = W.csr_from_coo(np.r_[np.arange(n), np.arange(n)], np.r_[np.zeros(n, int), np.full(n, n - 1)], n, n)
    E.val = np.arange(E.nnz, dtype=np.int32)
    check(H, O.MP_I32, E, E)


def test_errors_are_statuses(H):
    import paper_1512_00066_b300 as stc
    A = W.random_csr(10, 8, 3, seed=1)
    A.val = np.ones(A.nnz, np.int32)
    B = W.random_csr(9, 8, 3, seed=2)
    B.val = np.ones(B.nnz, np.int32)
    with pytest.raises(stc.StcError) as e:
        H.spgemm(O.MP_I32, to_dev(A), to_dev(B))
    assert e.value.status == 2  # shape
    # unsorted columns
    U = W.Csr(2, 8, np.array([0, 2, 3], np.int64), np.array([5, 1, 2], np.int32), np.ones(3, np.int32))
    S = W.random_csr(8, 8, 3, seed=3)
    S.val = np.ones(S.nnz, np.int32)
    with pytest.raises(stc.StcError) as e:
        H.spgemm(O.MP_I32, to_dev(U), to_dev(S))
    assert e.value.status == 3
    # column out of range
    R = W.Csr(1, 8, np.array([0, 1], np.int64), np.array([8], np.int32), np.ones(1, np.int32))
    with pytest.raises(stc.StcError) as e:
        H.spgemm(O.MP_I32, to_dev(R), to_dev(S))
    assert e.value.status == 3
    # bad row pointers
    P = W.Csr(2, 8, np.array([0, 3, 2], np.int64), np.array([1, 2], np.int32), np.ones(2, np.int32))
    with pytest.raises(stc.StcError) as e:
        H.spgemm(O.MP_I32, to_dev(P), to_dev(S))
    assert e.value.status == 2
    # the handle stays usable after errors
    check(H, O.MP_I32, S, S)


@pytest.mark.parametrize("alg", [O.MP_I32, O.MP_F32, O.BOOL, O.PT_F32, O.PT_F64])
def test_repeatable(H, alg):
    """Two runs of the same product.  The structure is the symbolic union and
    (min,+) / boolean values are order-independent, so those repeat bit for bit.
    (+,x) sums are accumulated by shared-memory atomics in an order that depends
    on scheduling: their structure repeats exactly and their values only within
    the algebra's tolerance (each run is also within it of the fp64 oracle)."""
    A = W.rmat(12, seed=8)
    A.val = vals(alg, A.nnz, 1, "A")
    d = to_dev(A)
    C1 = H.spgemm(alg, d, d).to_host()
    C2 = H.spgemm(alg, d, d).to_host()
    assert np.array_equal(C1[0], C2[0]) and np.array_equal(C1[1], C2[1])
    if alg in (O.PT_F32, O.PT_F64):
        ptr, col, val, ab = O.spgemm(alg, A, A, want_abs=True)
        compare_values(alg, C1[2], val, ab, "run 1")
        compare_values(alg, C2[2], val, ab, "run 2")
    else:
        assert C1[2].tobytes() == C2[2].tobytes()


@pytest.mark.parametrize("alg", [O.PT_F64, O.PT_F32])
def test_rmat18_full_size_sampled(H, alg):
    """R-MAT scale 18 A.A at full size: every row count against the oracle's
    exact counts, and every 64th row plus the 256 heaviest rows element by element."""
    A = W.rmat(18, seed=0)
    w = W.weights_unit01(A.nnz, seed=0)
    A.val = w.astype(np.float32 if alg == O.PT_F32 else np.float64)
    lens = np.diff(A.rowptr)
    ub = np.zeros(A.nrows, np.int64)
    np.add.at(ub, np.repeat(np.arange(A.nrows), lens), lens[A.col])
    rows = np.unique(np.r_[np.arange(0, A.nrows, 64), np.argsort(ub)[-256:]])
    check(H, alg, A, A, rows=rows)


def test_rmat20_column_slabs_full_size_sampled(H):
    """R-MAT scale 20 A.A in fp32 (2^20 output columns: four column slabs) at full
    size: every row count against the oracle's exact counts, and every 256th row
    plus the 64 heaviest rows element by element."""
    A = W.rmat(20, seed=0)
    A.val = W.weights_unit01(A.nnz, seed=0).astype(np.float32)
    lens = np.diff(A.rowptr)
    ub = np.zeros(A.nrows, np.int64)
    np.add.at(ub, np.repeat(np.arange(A.nrows), lens), lens[A.col])
    rows = np.unique(np.r_[np.arange(0, A.nrows, 256), np.argsort(ub)[-64:]])
    d = to_dev(A)
    C = H.spgemm(O.PT_F32, d, d)
    torch.cuda.synchronize()
    H.check_device_status()
    rp = C.rowptr.cpu().numpy()
    assert np.array_equal(np.diff(rp), O.spgemm_count(A, A)), "row counts differ"
    # gather the sampled rows on the device (C itself is ~78 GB)
    sel = np.concatenate([np.arange(rp[i], rp[i + 1]) for i in rows])
    idx = torch.from_numpy(sel).to(C.col.device)
    col = C.col[idx].cpu().numpy()
    val = C.val[idx].cpu().numpy()
    del C
    torch.cuda.empty_cache()
    ptr, rcol, rval, rabs = O.spgemm(O.PT_F32, A, A, rows=rows, want_abs=True)
    assert np.array_equal(col, rcol)
    compare_values(O.PT_F32, val, rval, rabs, where="rmat20 sampled")


# ----------------------------------------------------------------- masked product

def masked_expected(alg, A, B, M):
    """C<M> from the oracle's full product: its entries at M's positions, the
    additive identity where the product has none."""
    ptr, col, val, absv = O.spgemm(alg, A, B, want_abs=True)
    rows = np.repeat(np.arange(A.nrows, dtype=np.int64), np.diff(ptr))
    keys = rows * B.ncols + col.astype(np.int64)
    mrows = np.repeat(np.arange(M.nrows, dtype=np.int64), np.diff(M.rowptr))
    mkeys = mrows * B.ncols + M.col.astype(np.int64)
    if len(keys):
        pos = np.minimum(np.searchsorted(keys, mkeys), len(keys) - 1)
        hit = keys[pos] == mkeys
    else:
        pos = np.zeros(len(mkeys), np.int64)
        hit = np.zeros(len(mkeys), bool)
    out = np.zeros(len(mkeys), dtype=val.dtype)
    if alg == O.MULTPATH:
        out["d"] = O.TROP_I32_ID
    elif alg == O.MP_I32:
        out[:] = O.TROP_I32_ID
    elif alg == O.MP_F32:
        out[:] = np.inf
    out[hit] = val[pos[hit]]
    ab = np.zeros(len(mkeys))
    if absv is not None:
        ab[hit] = absv[pos[hit]]
    return out, ab, hit


def mask_from(A, B, keep, extra_per_row, seed, empty_frac=0.1):
    """Part of the product's structure (fraction `keep`) plus random columns."""
    rng = np.random.default_rng(seed)
    ptr, col, _, _ = O.spgemm(O.BOOL, A.with_val(np.ones(A.nnz, np.uint8)), B.with_val(np.ones(B.nnz, np.uint8)))
    rows = np.repeat(np.arange(A.nrows), np.diff(ptr))
    sel = rng.random(len(col)) < keep
    er = rng.integers(0, A.nrows, extra_per_row * A.nrows)
    ec = rng.integers(0, B.ncols, extra_per_row * A.nrows)
    r = np.r_[rows[sel], er]
    c = np.r_[col[sel], ec]
    drop = rng.random(A.nrows) < empty_frac
    k = ~drop[r]
    return W.csr_from_coo(r[k], c[k], A.nrows, B.ncols)


def check_masked(H, alg, A, B, M, where=""):
    C = H.spgemm_masked(alg, to_dev(A), to_dev(B), to_dev(M))
    torch.cuda.synchronize()
    H.check_device_status()
    assert np.array_equal(C.rowptr.cpu().numpy(), M.rowptr) and np.array_equal(C.col.cpu().numpy(), M.col)
    exp, ab, hit = masked_expected(alg, A, B, M)
    got = C.val.cpu().numpy()
    compare_values(alg, got, exp, ab, where=where or f"masked alg {alg}")
    return hit


@pytest.mark.parametrize("alg", ALL)
def test_masked_all_algebras(H, alg):
    """A mask holding half of the product's entries, foreign entries (identity) and
    empty rows, over rows of A that are empty or not."""
    A = W.random_csr(400, 500, 30, seed=61, empty_frac=0.15)
    B = W.random_csr(500, 3000, 40, seed=62, empty_frac=0.1)
    A.val = vals(alg, A.nnz, 63, "A")
    B.val = vals(alg, B.nnz, 64, "B")
    M = mask_from(A, B, 0.5, 5, seed=65)
    hit = check_masked(H, alg, A, B, M)
    assert hit.any() and not hit.all()


@pytest.mark.parametrize("alg", [O.PT_F64, O.MP_I32, O.MULTPATH])
def test_masked_by_own_structure_rmat14(H, alg):
    """C<A> = A (x) A masked by A (the triangle-counting shape), R-MAT scale 14."""
    A = W.rmat(14, seed=31)
    A.val = vals(alg, A.nnz, 32, "A")
    B = A.with_val(vals(alg, A.nnz, 33, "B"))
    M = W.Csr(A.nrows, A.ncols, A.rowptr, A.col, None)
    check_masked(H, alg, A, B, M)


@pytest.mark.parametrize("alg", [O.PT_F32, O.MP_F32, O.BOOL])
def test_masked_rows_over_several_rank_windows(H, alg):
    """Mask rows with tens of thousands of entries (several rank windows each)."""
    A = W.random_csr(120, 300, 300, seed=71, empty_frac=0.05)
    B = W.random_csr(300, 60000, 400, seed=72)
    A.val = vals(alg, A.nnz, 73, "A")
    B.val = vals(alg, B.nnz, 74, "B")
    M = mask_from(A, B, 0.8, 2000, seed=75, empty_frac=0.05)
    assert np.diff(M.rowptr).max() > 30000
    check_masked(H, alg, A, B, M)


def test_masked_rmat18_full_size_sampled(H):
    """The benchmark's masked product, C<A> = A.A in fp64 at R-MAT scale 18: C has
    exactly A's structure, and every 64th row plus the 256 heaviest rows hold the
    oracle's product read at the mask's positions (0 where no product lands)."""
    A = W.rmat(18, seed=0)
    A.val = W.weights_unit01(A.nnz, seed=0)
    M = W.Csr(A.nrows, A.ncols, A.rowptr, A.col, None)
    d = to_dev(A)
    C = H.spgemm_masked(O.PT_F64, d, d, to_dev(M))
    torch.cuda.synchronize()
    H.check_device_status()
    assert np.array_equal(C.rowptr.cpu().numpy(), M.rowptr) and np.array_equal(C.col.cpu().numpy(), M.col)
    lens = np.diff(A.rowptr)
    ub = np.zeros(A.nrows, np.int64)
    np.add.at(ub, np.repeat(np.arange(A.nrows), lens), lens[A.col])
    rows = np.unique(np.r_[np.arange(0, A.nrows, 64), np.argsort(ub)[-256:]])
    sel = np.concatenate([np.arange(M.rowptr[i], M.rowptr[i + 1]) for i in rows])
    got = C.val.cpu().numpy()[sel]
    ptr, col, val, absv = O.spgemm(O.PT_F64, A, A, rows=rows, want_abs=True)
    mrow = np.repeat(np.arange(len(rows), dtype=np.int64), lens[rows])
    pkeys = np.repeat(np.arange(len(rows), dtype=np.int64), np.diff(ptr)) * A.ncols + col.astype(np.int64)
    mkeys = mrow * A.ncols + M.col[sel].astype(np.int64)
    pos = np.minimum(np.searchsorted(pkeys, mkeys), max(len(pkeys) - 1, 0))
    hit = pkeys[pos] == mkeys
    exp = np.where(hit, val[pos], 0.0)
    ab = np.where(hit, absv[pos], 0.0)
    assert hit.any() and not hit.all()
    compare_values(O.PT_F64, got, exp, ab, where="masked rmat18 sampled")


def test_masked_errors(H):
    import paper_1512_00066_b300 as stc
    A = W.random_csr(10, 8, 3, seed=1)
    A.val = np.ones(A.nnz, np.int32)
    B = W.random_csr(8, 9, 3, seed=2)
    B.val = np.ones(B.nnz, np.int32)
    Mbad = W.random_csr(10, 10, 3, seed=3)  # 10 columns, the product has 9
    with pytest.raises(stc.StcError) as e:
        H.spgemm_masked(O.MP_I32, to_dev(A), to_dev(B), to_dev(Mbad))
    assert e.value.status == 2
    U = W.Csr(10, 9, np.r_[0, 2, np.full(9, 2)].astype(np.int64), np.array([5, 1], np.int32), None)
    with pytest.raises(stc.StcError) as e:
        H.spgemm_masked(O.MP_I32, to_dev(A), to_dev(B), to_dev(U))
    assert e.value.status == 3
    E = W.Csr(10, 9, np.zeros(11, np.int64), np.zeros(0, np.int32), None)
    C = H.spgemm_masked(O.MP_I32, to_dev(A), to_dev(B), to_dev(E))
    assert C.nnz == 0


def _hub_case(K, ncols, per_b, hub_lens, light_rows, light_len, seed):
    """A with the given hub row lengths (stored entries) followed by light rows;
    B with per_b distinct columns a row; positive values U[0.5, 2) (no cancellation:
    the relative error of a sum is its rounding error)."""
    rng = np.random.default_rng(seed)
    rows, cols = [], []
    lens = list(hub_lens) + [light_len] * light_rows
    for i, n in enumerate(lens):
        rows.append(np.full(n, i))
        cols.append(rng.choice(K, n, replace=False))
    A = W.csr_from_coo(np.concatenate(rows), np.concatenate(cols), len(lens), K)
    A.val = rng.uniform(0.5, 2.0, A.nnz).astype(np.float32)
    br = np.repeat(np.arange(K), per_b)
    bc = np.concatenate([rng.choice(ncols, per_b, replace=False) for _ in range(K)])
    B = W.csr_from_coo(br, bc, K, ncols)
    B.val = rng.uniform(0.5, 2.0, B.nnz).astype(np.float32)
    return A, B


def _check_wide_rows(A, B, rp, col, val, wide_len=1024):
    """Rows of A with more than wide_len stored entries (summed with compensation):
    within one fp32 ulp (2^-23 relative) of the fp64 oracle, which plain fp32
    summation of their hundreds of terms per entry misses; the other rows within
    the fp32 tolerance."""
    ptr, rcol, rval, rabs = O.spgemm(O.PT_F32, A, B, want_abs=True)
    assert np.array_equal(rp, ptr) and np.array_equal(col, rcol)
    alen = np.diff(A.rowptr)
    wide = np.repeat(alen > wide_len, np.diff(ptr))
    got = val.astype(np.float64)
    rel = np.abs(got - rval) / rval
    assert wide.any()
    assert rel[wide].max() <= 2.0 ** -23, rel[wide].max()
    compare_values(O.PT_F32, val[~wide], rval[~wide], rabs[~wide], "narrow rows")


def test_fp32_hub_rows_are_summed_with_compensation(H):
    import paper_1512_00066_b300 as stc
    # narrow output (warp-per-row path, hub rows split off to the CTA kernel):
    # row 0 has 3000 entries (about 375 terms per output entry), row 2 has 1025
    A, B = _hub_case(4096, 64, 8, [3000, 1024, 1025], 200, 40, seed=3)
    C = H.spgemm(stc.PLUS_TIMES_F32, to_dev(A), to_dev(B))
    _check_wide_rows(A, B, *C.to_host())
    # the same pair in a batch, and through the learned single pass
    Cs = H.spgemm_batched(stc.PLUS_TIMES_F32, [to_dev(A)] * 3, [to_dev(B)] * 3)
    _check_wide_rows(A, B, *Cs[1].to_host())
    C2, _ = H.spgemm_learned(stc.PLUS_TIMES_F32, to_dev(A), to_dev(B))
    _check_wide_rows(A, B, *C2.to_host())
    # a wide output (2^17 columns): the hub rows' outputs span several half-width
    # rank windows
    A, B = _hub_case(20000, 1 << 17, 16, [3000, 6000], 100, 30, seed=4)
    C = H.spgemm(stc.PLUS_TIMES_F32, to_dev(A), to_dev(B))
    rp, col, val = C.to_host()
    assert np.diff(rp)[1] > 40000
    _check_wide_rows(A, B, rp, col, val)
    C2, _ = H.spgemm_learned(stc.PLUS_TIMES_F32, to_dev(A), to_dev(B))
    _check_wide_rows(A, B, *C2.to_host())
