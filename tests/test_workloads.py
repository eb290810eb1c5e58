"""The seeded synthetic inputs that the benchmark and the profiles are quoted on
(CPU only): a change to a generator changes every published number, so the
statistics the design notes state are pinned here."""
import numpy as np

import workloads as W


def _stats(A):
    lens = np.diff(A.rowptr)
    return A.nnz, int(lens.max()), int((lens == 0).sum()), int(lens[A.col].sum())


def test_rmat_benchmark_graphs():
    # R-MAT scale 16 (profiles), 18 (the benchmark step) and 20 (slabs, perceptron form):
    # edges, maximum out-degree, vertices without out-edges, products of A.A
    assert _stats(W.rmat(16, seed=0)) == (954632, 6259, 25264, 401053578)
    A = W.rmat(18, seed=0)
    assert _stats(A) == (3939728, 15767, 113727, 2932766381)
    # structure: sorted, unique columns per row, in range
    assert A.rowptr[0] == 0 and A.rowptr[-1] == A.nnz and np.all(np.diff(A.rowptr) >= 0)
    rows = np.repeat(np.arange(A.nrows), np.diff(A.rowptr))
    key = rows.astype(np.int64) * A.ncols + A.col
    assert np.all(np.diff(key) > 0) and A.col.min() >= 0 and A.col.max() < A.ncols


def test_weights_are_seeded_and_in_range():
    w = W.weights_unit01(100000, seed=0)
    assert np.array_equal(w, W.weights_unit01(100000, seed=0))
    assert w.min() > 0.0 and w.max() <= 1.0
    wi = W.weights_int(100000, 1, 255, seed=1)
    assert wi.min() >= 1 and wi.max() <= 255 and wi.dtype == np.int32
