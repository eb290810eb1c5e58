"""Batched SpGEMM (many independent pairs in one call) against the oracle and
against one call per pair."""
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
        return rng.integers(-100, 10000, nnz).astype(np.int32)
    if alg == O.MP_F32:
        return (rng.random(nnz) * 100).astype(np.float32)
    if alg == O.BOOL:
        return rng.integers(0, 2, nnz).astype(np.uint8)
    if operand == "A":
        return rng.integers(1, 8, nnz).astype(np.int32)
    return W.multpath_values(nnz, 20, 5, seed)


def check_pair(alg, A, B, C):
    rp, col, val = C.to_host()
    ptr, rcol, rval, rabs = O.spgemm(alg, A, B, want_abs=True)
    assert np.array_equal(rp, ptr) and np.array_equal(col, rcol)
    compare_values(alg, val, rval, rabs, where=f"alg {alg}")


@pytest.mark.parametrize("alg", ALL)
def test_batched_mixed_sizes_all_algebras(H, alg):
    rng = np.random.default_rng(alg)
    As, Bs = [], []
    for b in range(23):
        m, k, n = rng.integers(0, 300, 3)
        if b == 5:
            m = 0  # empty matrix in the middle
        A = W.random_csr(int(m), int(k) + 1, 30, seed=100 * alg + 2 * b, empty_frac=0.1)
        B = W.random_csr(int(k) + 1, int(n) + 1, 30, seed=100 * alg + 2 * b + 1, empty_frac=0.1)
        A.val = vals(alg, A.nnz, b, "A")
        B.val = vals(alg, B.nnz, b + 1000, "B")
        As.append(A)
        Bs.append(B)
    Cs = H.spgemm_batched(alg, [to_dev(a) for a in As], [to_dev(b) for b in Bs])
    for A, B, C in zip(As, Bs, Cs):
        check_pair(alg, A, B, C)


def test_batched_equals_per_call_min_plus(H):
    sizes, As, Bs = W.powerlaw_batch(40, 64, 2048, 2.1, 4, 64, seed=3)
    for m in As + Bs:
        m.val = (np.abs(m.val) * 1000).astype(np.int32)
    dA = [to_dev(a) for a in As]
    dB = [to_dev(b) for b in Bs]
    Cs = H.spgemm_batched(O.MP_I32, dA, dB)
    for a, b, c in zip(dA, dB, Cs):
        ref = H.spgemm(O.MP_I32, a, b)
        for x, y in zip(c.to_host(), ref.to_host()):
            assert np.array_equal(x, y)


def test_single_pair_batch_and_wide_rows(H):
    A = W.random_csr(100, 300, 300, seed=15)
    B = W.random_csr(300, 60000, 400, seed=16)
    A.val = vals(O.PT_F32, A.nnz, 1, "A")
    B.val = vals(O.PT_F32, B.nnz, 2, "B")
    C = H.spgemm_batched(O.PT_F32, [to_dev(A), to_dev(A)], [to_dev(B), to_dev(B)])
    check_pair(O.PT_F32, A, B, C[0])
    check_pair(O.PT_F32, A, B, C[1])


def test_config_4096_pairs_sampled(H):
    """4096 pairs, rows power-law in [64, 16384] (exponent 2.1), U{4..64} entries
    per row, N(0,1) fp32: 40 sampled pairs (incl. the largest) element by element."""
    sizes, As, Bs = W.powerlaw_batch(4096, 64, 16384, 2.1, 4, 64, seed=0)
    Cs = H.spgemm_batched(O.PT_F32, [to_dev(a) for a in As], [to_dev(b) for b in Bs])
    rng = np.random.default_rng(1)
    pick = set(rng.choice(4096, 36, replace=False).tolist()) | set(np.argsort(sizes)[-4:].tolist())
    for b in sorted(pick):
        check_pair(O.PT_F32, As[b], Bs[b], Cs[b])


@pytest.mark.parametrize("light", [7, 10])
def test_batched_light_row_launch(H, light):
    """Light rows of the whole batch in their own launch: same result as one call
    per pair without it."""
    sizes, As, Bs = W.powerlaw_batch(30, 64, 4096, 2.1, 4, 64, seed=7)
    for m in As + Bs:
        m.val = (np.abs(m.val) * 1000).astype(np.int32)
    dA = [to_dev(a) for a in As]
    dB = [to_dev(b) for b in Bs]
    Cs = H.spgemm_batched(O.MP_I32, dA, dB, light_rows=light)
    for a, b, c in zip(dA, dB, Cs):
        ref = H.spgemm(O.MP_I32, a, b, light_rows=-1)
        for x, y in zip(c.to_host(), ref.to_host()):
            assert np.array_equal(x, y)
