"""Pins of the oracle's learned-sizing functions (CPU only)."""
import numpy as np

import oracle as O
import workloads as W


def test_splitmix64_published_outputs():
    # first outputs of the SplitMix64 generator seeded with 0 (state advanced by
    # the golden gamma before each mix)
    assert O.splitmix64(0) == 0xE220A8397B1DCDAF
    assert O.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4


def _single_row(k, K):
    return W.Csr(1, K, np.array([0, 1], np.int64), np.array([k], np.int32))


def test_feature_scalars_and_union_sketch():
    A = W.random_csr(60, 80, 12, seed=1, empty_frac=0.1)
    B = W.random_csr(80, 500, 40, seed=2, empty_frac=0.1)
    F = O.row_features(A, B)
    blen = np.diff(B.rowptr)
    for i in range(A.nrows):
        ks = A.col[A.rowptr[i]:A.rowptr[i + 1]]
        ub = int(blen[ks].sum())
        mx = int(blen[ks].max()) if ks.size else 0
        assert F[i, 0] == np.log2(1 + ub) and F[i, 1] == np.log2(1 + ks.size) and F[i, 2] == np.log2(1 + mx)
        # the sketch of a union is the bucket-wise minimum of the sketches of its parts
        parts = [O.row_features(_single_row(int(k), A.ncols), B)[0] for k in ks]
        if parts:
            mins = np.min([p[3::2] for p in parts], axis=0)
            empt = np.min([p[4::2] for p in parts], axis=0)
            assert np.array_equal(F[i, 3::2], mins) and np.array_equal(F[i, 4::2], empt)
        else:
            assert np.all(F[i, 3::2] == 1.0) and np.all(F[i, 4::2] == 1.0)
    # empty flags agree with the buckets actually hit by the union's columns
    i = int(np.argmax(np.diff(A.rowptr)))
    cols = set()
    for k in A.col[A.rowptr[i]:A.rowptr[i + 1]]:
        cols |= set(B.col[B.rowptr[k]:B.rowptr[k + 1]].tolist())
    hit = {O.splitmix64(c) >> 59 for c in cols}
    assert {b for b in range(32) if F[i, 4 + 2 * b] == 0.0} == hit


def test_mlp_gradient_matches_finite_differences():
    rng = np.random.default_rng(0)
    nw = O.mlp_num_weights()
    w = rng.standard_normal(nw) * 0.2
    x = rng.standard_normal((9, O.NFEAT))
    t = rng.standard_normal(9)
    g, L = O.mlp_grad(w, x, t)
    loss = lambda ww: float(np.mean((O.mlp_forward(ww, x) - t) ** 2))
    assert abs(L - loss(w)) < 1e-12
    idx = rng.choice(nw, 60, replace=False).tolist() + [nw - 1, 0, 64 * 67, 64 * 67 + 64]
    for k in idx:
        e = np.zeros(nw)
        e[k] = 1e-6
        fd = (loss(w + e) - loss(w - e)) / 2e-6
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(fd)), k


def test_mlp_closed_form_bias_only():
    nw = O.mlp_num_weights()
    w = np.zeros(nw)
    w[-1] = 2.5  # only the output bias
    x = np.random.default_rng(1).standard_normal((5, O.NFEAT))
    t = np.arange(5.0)
    assert np.all(O.mlp_forward(w, x) == 2.5)
    g, L = O.mlp_grad(w, x, t)
    assert abs(g[-1] - 2 * np.mean(2.5 - t)) < 1e-12 and np.all(g[:-1] == 0)
    assert abs(L - np.mean((2.5 - t) ** 2)) < 1e-12


def test_min_hash_key_of_a_single_column_from_the_published_output():
    """A row whose column union is {0}: SplitMix64's first published output for
    seed 0 is 0xE220A8397B1DCDAF, so the column lands in bucket 0xE220... >> 59 = 28
    with key 0x7B1DCDAF (the low word), normalised by 2^32; every other bucket is
    empty (1, 1).  Taking the high word or dropping the normalisation fails here."""
    B = W.Csr(1, 4, np.array([0, 1], np.int64), np.array([0], np.int32))
    F = O.row_features(_single_row(0, 1), B)[0]
    assert (0xE220A8397B1DCDAF >> 59) == 28
    for b in range(32):
        if b == 28:
            assert F[3 + 2 * b] == 0x7B1DCDAF / 2.0 ** 32 and F[4 + 2 * b] == 0.0
        else:
            assert F[3 + 2 * b] == 1.0 and F[4 + 2 * b] == 1.0


def test_min_hash_keys_restated_on_random_rows():
    """Bucket-wise minimum of (low 32 bits of SplitMix64(j)) / 2^32 over the union
    of the B rows' columns, written out with Python integers."""
    A = W.random_csr(12, 40, 6, seed=7, empty_frac=0.0)
    B = W.random_csr(40, 3000, 50, seed=8, empty_frac=0.0)
    F = O.row_features(A, B)
    for i in range(A.nrows):
        cols = set()
        for k in A.col[A.rowptr[i]:A.rowptr[i + 1]]:
            cols |= set(B.col[B.rowptr[k]:B.rowptr[k + 1]].tolist())
        mins = [None] * 32
        for j in cols:
            h = O.splitmix64(int(j))
            b, key = h >> 59, h & 0xFFFFFFFF
            mins[b] = key if mins[b] is None else min(mins[b], key)
        for b in range(32):
            if mins[b] is None:
                assert F[i, 3 + 2 * b] == 1.0 and F[i, 4 + 2 * b] == 1.0
            else:
                assert F[i, 3 + 2 * b] == mins[b] / 2.0 ** 32 and F[i, 4 + 2 * b] == 0.0
