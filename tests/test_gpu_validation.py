"""Device-side CSR validation: every stored entry and row pointer is checked.

The check runs over a flat index of each matrix's rows and entries in tiles of
2048 elements; these cases put the fault on and beside tile boundaries, deep in a
large matrix and in one matrix of a batch, and check that valid inputs whose rows
restart at a smaller column (the usual case between rows) pass.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_util import need_gpu, to_dev

pytestmark = pytest.mark.gpu

TILE = 2048


@pytest.fixture(scope="module")
def H():
    need_gpu()
    import paper_1512_00066_b300 as stc
    return stc.Handle()


def _ones(m):
    m.val = np.ones(m.nnz, np.int32)
    return m


def _inner_positions(A):
    """Entries p that are not the first of their row, chosen at and beside the
    tile boundaries of the flat index (nrows + p) and at the array's end."""
    starts = set(A.rowptr[:-1].tolist())
    first = A.nrows // TILE + 1  # first tile boundary inside the column part
    last = (A.nrows + A.nnz) // TILE
    want = [A.nnz - 1]
    for k in (first, first + 1, (first + last) // 2, last):
        for d in (-1, 0, 1):
            want.append(k * TILE + d - A.nrows)
    out = set()
    for p in want:
        for q in list(range(p, min(p + 64, A.nnz))) + list(range(p - 1, max(p - 64, 0), -1)):
            if 0 < q < A.nnz and q not in starts:
                out.add(q)
                break
    return sorted(out)


def test_valid_rmat_with_empty_rows_passes(H):
    import paper_1512_00066_b300 as stc
    A = _ones(W.rmat(13, seed=3))
    assert (np.diff(A.rowptr) == 0).any()  # empty rows present
    C = H.spgemm(stc.MIN_PLUS_I32, to_dev(A), to_dev(A))
    ptr, _, _, _ = O.spgemm(O.MP_I32, A, A)
    assert C.nnz == int(ptr[-1])


@pytest.mark.parametrize("fault", ["swap", "duplicate", "range"])
def test_column_faults_anywhere_are_found(H, fault):
    import paper_1512_00066_b300 as stc
    A = _ones(W.rmat(13, seed=3))
    B = _ones(W.rmat(13, seed=4))
    ps = _inner_positions(A)
    assert len(ps) >= 8
    for p in ps:
        col = A.col.copy()
        if fault == "swap":
            col[p - 1], col[p] = col[p], col[p - 1]
        elif fault == "duplicate":
            col[p] = col[p - 1]
        else:
            col[p] = A.ncols
        bad = W.Csr(A.nrows, A.ncols, A.rowptr, col, A.val)
        with pytest.raises(stc.StcError) as e:
            H.spgemm(stc.MIN_PLUS_I32, to_dev(bad), to_dev(B))
        assert e.value.status == 3, p
        # and as the right operand
        with pytest.raises(stc.StcError) as e:
            H.spgemm(stc.MIN_PLUS_I32, to_dev(B), to_dev(bad))
        assert e.value.status == 3, p


def test_row_pointer_faults_are_found(H):
    import paper_1512_00066_b300 as stc
    A = _ones(W.rmat(13, seed=3))
    nz_rows = np.flatnonzero(np.diff(A.rowptr) > 1)
    for i in (int(nz_rows[0]), int(nz_rows[len(nz_rows) // 2]), TILE - 1, TILE, int(nz_rows[-1])):
        rp = A.rowptr.copy()
        rp[i + 1] = rp[i] - 1  # pointer runs backwards
        bad = W.Csr(A.nrows, A.ncols, rp, A.col, A.val)
        with pytest.raises(stc.StcError) as e:
            H.spgemm(stc.MIN_PLUS_I32, to_dev(bad), to_dev(A))
        assert e.value.status == 2, i
    # the last pointer disagrees with the number of stored entries
    rp = A.rowptr.copy()
    rp[-1] -= 1
    bad = W.Csr(A.nrows, A.ncols, rp, A.col, A.val)
    with pytest.raises(stc.StcError) as e:
        H.spgemm(stc.MIN_PLUS_I32, to_dev(bad), to_dev(A))
    assert e.value.status == 2


def test_batched_validation_finds_one_bad_matrix_among_many(H):
    import paper_1512_00066_b300 as stc
    rng = np.random.default_rng(5)
    As, Bs = [], []
    for b in range(40):
        m, k = int(rng.integers(0, 3000)), int(rng.integers(1, 900))
        n = int(rng.integers(1, 5000))
        As.append(_ones(W.random_csr(m, k, int(rng.integers(1, 30)), seed=100 + b, empty_frac=0.1)))
        Bs.append(_ones(W.random_csr(k, n, int(rng.integers(1, 30)), seed=200 + b, empty_frac=0.1)))
    dA = [to_dev(a) for a in As]
    dB = [to_dev(b) for b in Bs]
    Cs = H.spgemm_batched(stc.MIN_PLUS_I32, dA, dB)
    for b in (0, 17, 39):
        ptr, _, _, _ = O.spgemm(O.MP_I32, As[b], Bs[b])
        assert Cs[b].nnz == int(ptr[-1])
    # one bad entry in the middle of B_29
    Bb = Bs[29]
    assert Bb.nnz > 4
    p = next(q for q in range(Bb.nnz // 2, Bb.nnz) if q not in set(Bb.rowptr.tolist()))
    col = Bb.col.copy()
    col[p] = col[p - 1]
    dB_bad = list(dB)
    dB_bad[29] = to_dev(W.Csr(Bb.nrows, Bb.ncols, Bb.rowptr, col, Bb.val))
    with pytest.raises(stc.StcError) as e:
        H.spgemm_batched(stc.MIN_PLUS_I32, dA, dB_bad)
    assert e.value.status == 3
    # a bad row pointer in the first non-empty A from the fourth on
    ia = next(b for b in range(3, 40) if As[b].nnz > 0)
    Ab = As[ia]
    rp = Ab.rowptr.copy()
    i = int(np.flatnonzero(np.diff(rp) > 0)[0])
    rp[i + 1] = -1
    dA_bad = list(dA)
    dA_bad[ia] = to_dev(W.Csr(Ab.nrows, Ab.ncols, rp, Ab.col, Ab.val))
    with pytest.raises(stc.StcError) as e:
        H.spgemm_batched(stc.MIN_PLUS_I32, dA_bad, dB)
    assert e.value.status == 2
    # and the handle still works
    Cs = H.spgemm_batched(stc.MIN_PLUS_I32, dA, dB)
    assert Cs[5].nnz == int(O.spgemm(O.MP_I32, As[5], Bs[5])[0][-1])


def test_empty_operands_pass(H):
    import paper_1512_00066_b300 as stc
    Z = W.Csr(0, 5, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32))
    E = W.Csr(4, 5, np.zeros(5, np.int64), np.zeros(0, np.int32), np.zeros(0, np.int32))
    B = _ones(W.random_csr(5, 7, 3, seed=9))
    for A in (Z, E):
        C = H.spgemm(stc.MIN_PLUS_I32, to_dev(A), to_dev(B))
        assert C.nrows == A.nrows and C.nnz == 0
    Cs = H.spgemm_batched(stc.MIN_PLUS_I32, [to_dev(Z), to_dev(E), to_dev(B)],
                          [to_dev(B), to_dev(B), to_dev(_ones(W.random_csr(7, 3, 2, seed=10)))])
    assert Cs[0].nnz == 0 and Cs[1].nnz == 0 and Cs[2].nnz > 0
