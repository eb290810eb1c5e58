"""Learned output sizing on the GPU: features, perceptron forward/gradient and
training against the fp64 oracle, and the learned single-pass SpGEMM against the
plain two-pass one (identical structure whatever the model predicts)."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W
from gpu_util import compare_values, mlp_tc_tolerance, need_gpu, to_dev

pytestmark = pytest.mark.gpu

ALL = [O.PT_F32, O.PT_F64, O.MP_I32, O.MP_F32, O.BOOL, O.MULTPATH]


@pytest.fixture(scope="module")
def H():
    need_gpu()
    import paper_1512_00066_b300 as stc
    return stc.Handle()


def bf16_weights(w: torch.Tensor) -> np.ndarray:
    return w.to(torch.bfloat16).to(torch.float64).cpu().numpy()


def test_features_match_oracle(H):
    A = W.rmat(11, seed=2)
    B = W.rmat(11, seed=3)
    f = H.row_features(to_dev(A), to_dev(B)).cpu().numpy()
    ref = O.row_features(A, B)
    assert np.array_equal(f[:, 3:67], ref[:, 3:].astype(np.float32))  # sketch: exact
    assert np.allclose(f[:, :3], ref[:, :3], rtol=1e-6, atol=1e-6)
    assert np.all(f[:, 67] == 0)


def test_mlp_forward_and_gradient_match_oracle(H):
    import paper_1512_00066_b300 as stc
    w = stc.mlp_init(seed=5)
    A = W.rmat(10, seed=4)
    feat = H.row_features(to_dev(A), to_dev(A))
    n = feat.shape[0]
    target = torch.linspace(0, 8, n, device="cuda")
    wd = bf16_weights(w)
    x = feat[:, :67].double().cpu().numpy()
    y = H.mlp_forward(w, feat).cpu().numpy()
    yr = O.mlp_forward(wd, x)
    assert np.all(np.abs(y - yr) <= 1e-4 * (1 + np.abs(yr)))
    g, loss = H.mlp_grad(w, feat, target)
    gr, Lr = O.mlp_grad(wd, x, target.double().cpu().numpy())
    g = g.double().cpu().numpy()
    assert np.linalg.norm(g - gr) <= 1e-3 * np.linalg.norm(gr)
    assert abs(float(loss) / n - Lr) <= 1e-4 * Lr


@pytest.mark.parametrize("n", [1, 129, 1024, 131072 - 37])
def test_mlp_forward_tensor_cores(H, n):
    """tcgen05 forward against the fp64 oracle (tolerance derived from the hi/lo
    bf16 arithmetic, gpu_util.mlp_tc_tolerance) and the CUDA-core kernel: one row,
    a tile plus one row, whole tiles, and more tiles than resident CTAs with a
    ragged last tile."""
    import paper_1512_00066_b300 as stc
    w = stc.mlp_init(seed=6)
    A = W.rmat(17, seed=8)
    feat = H.row_features(to_dev(A), to_dev(A))[:n]
    y = H.mlp_forward_tc(w, feat).cpu().numpy()
    wd = bf16_weights(w)
    x = feat[:, :67].double().cpu().numpy()
    yr = O.mlp_forward(wd, x)
    assert np.all(np.abs(y - yr) <= mlp_tc_tolerance(wd, x, yr))
    # the CUDA-core kernel (fp32 inputs, error far below 1e-5) within the same bound
    yc = H.mlp_forward(w, feat).cpu().numpy()
    assert np.all(np.abs(y - yc) <= mlp_tc_tolerance(wd, x, yc) + 1e-5 * (1 + np.abs(yc)))


def test_mlp_forward_tensor_cores_full_size(H):
    """The workload the benchmark times: features of every row of A.A for R-MAT
    scale 20 (2^20 rows), every row against the fp64 oracle."""
    import paper_1512_00066_b300 as stc
    w = stc.mlp_init(seed=1)
    A = W.rmat(20, seed=0)
    dA = stc.DeviceCsr.from_host(A.nrows, A.ncols, A.rowptr, A.col, np.ones(A.nnz, np.float32))
    feat = H.row_features(dA, dA)
    assert feat.shape[0] == 1 << 20
    y = H.mlp_forward_tc(w, feat).cpu().numpy()
    wd = bf16_weights(w)
    x = feat[:, :67].double().cpu().numpy()
    yr = O.mlp_forward(wd, x)
    assert np.all(np.abs(y - yr) <= mlp_tc_tolerance(wd, x, yr))


def test_mlp_forward_tensor_cores_signed_inputs(H):
    """Inputs of both signs and wide range (the hi/lo split of negative values),
    a non-zero padding column (ignored), and an empty batch."""
    import paper_1512_00066_b300 as stc
    w = stc.mlp_init(seed=7)
    g = torch.Generator(device="cuda").manual_seed(9)
    feat = torch.randn(5000, 68, device="cuda", generator=g) * 8.0
    y = H.mlp_forward_tc(w, feat).cpu().numpy()
    wd = bf16_weights(w)
    x = feat[:, :67].double().cpu().numpy()
    yr = O.mlp_forward(wd, x)
    assert np.all(np.abs(y - yr) <= mlp_tc_tolerance(wd, x, yr))
    assert H.mlp_forward_tc(w, feat[:0]).numel() == 0


def _pairs(stc, seeds):
    """Training matrices: R-MAT scales 11-14 (seeds >= 1; the evaluation graph is
    seed 0), ER and banded matrices."""
    out = []
    for s in seeds:
        for m in (W.rmat(11 + s % 4, seed=s), W.er_fixed_degree(2048 << (s % 2), 4 + 4 * (s % 4), seed=s),
                  W.banded(4096, 1 + 8 * (s % 4), 0.5, seed=s)):
            d = to_dev(m)
            out.append((d, d))
    return out


@pytest.fixture(scope="module")
def trained(H):
    import paper_1512_00066_b300 as stc
    feat, target = stc.training_rows(H, _pairs(stc, range(1, 9)))
    w = stc.mlp_init(seed=1)
    losses = H.mlp_train(w, feat, target, batch=2048, epochs=40, lr=2e-3, seed=3)
    return w, losses


def test_training_lowers_the_loss(trained):
    w, losses = trained
    assert losses[-1] < 0.2 * losses[0] and losses[-1] < 0.5


def _same(alg, C, R):
    rp, col, val = C.to_host()
    rp2, col2, val2 = R.to_host()
    assert np.array_equal(rp, rp2) and np.array_equal(col, col2)
    if alg in (O.PT_F32, O.PT_F64):
        # same products, possibly another summation order
        assert np.allclose(val.astype(np.float64), val2.astype(np.float64), rtol=1e-4 if alg == O.PT_F32 else 1e-12,
                           atol=1e-5)
    else:
        assert val.tobytes() == val2.tobytes()


def _vals(alg, nnz, seed):
    rng = np.random.default_rng(seed)
    if alg in (O.PT_F32, O.MP_F32):
        return rng.random(nnz).astype(np.float32)
    if alg == O.PT_F64:
        return rng.random(nnz)
    if alg == O.BOOL:
        return rng.integers(0, 2, nnz).astype(np.uint8)
    return rng.integers(1, 100, nnz).astype(np.int32)


@pytest.mark.parametrize("alg", ALL)
def test_learned_equals_plain_for_any_model(H, trained, alg):
    import paper_1512_00066_b300 as stc
    w, _ = trained
    A = W.rmat(13, seed=9)
    A.val = _vals(alg, A.nnz, 1)
    B = A.with_val(_vals(alg if alg != O.MULTPATH else O.MP_I32, A.nnz, 2)) if alg != O.MULTPATH else \
        A.with_val(W.multpath_values(A.nnz, 20, 5, 2))
    dA, dB = to_dev(A), to_dev(B)
    plain = H.spgemm(alg, dA, dB)
    under = torch.zeros(stc.MLP_NUM_WEIGHTS, dtype=torch.float32, device="cuda")  # predicts 0: capacity 8
    for weights, margin in ((w, 0.25), (None, 0.0), (under, 0.0)):
        C, st = H.spgemm_learned(alg, dA, dB, weights, margin)
        _same(alg, C, plain)
        assert st["nnz"] == plain.nnz
    C, st = H.spgemm_learned(alg, dA, dB, under, 0.0)
    assert st["recomputed_rows"] > 0  # the exact recomputation really ran
    # a trained model with no margin: rows above their capacity land in the
    # overflow pool instead of being recomputed
    C, st = H.spgemm_learned(alg, dA, dB, w, 0.0)
    _same(alg, C, plain)
    assert st["overflow_rows"] > st["recomputed_rows"]


def test_learned_rows_against_oracle(H, trained):
    w, _ = trained
    A = W.rmat(12, seed=11)
    A.val = W.weights_unit01(A.nnz, 1).astype(np.float32)
    C, st = H.spgemm_learned(O.PT_F32, to_dev(A), to_dev(A), w, 0.25)
    rp, col, val = C.to_host()
    ptr, rcol, rval, rabs = O.spgemm(O.PT_F32, A, A, want_abs=True)
    assert np.array_equal(rp, ptr) and np.array_equal(col, rcol)
    compare_values(O.PT_F32, val, rval, rabs)


def test_what_the_model_gains(H, trained):
    """Trained model vs the upper-bound single pass on a held-out R-MAT: the model
    sizes the scratch far below the bound while few rows overflow."""
    w, _ = trained
    A = W.rmat(14, seed=0)
    A.val = W.weights_unit01(A.nnz, 0).astype(np.float32)
    dA = to_dev(A)
    _, st_ub = H.spgemm_learned(O.PT_F32, dA, dA, None, 0.0)
    _, st_ml = H.spgemm_learned(O.PT_F32, dA, dA, w, 0.5)
    print("scratch ub", st_ub["scratch_entries"], "model", st_ml["scratch_entries"], "nnz", st_ml["nnz"],
          "overflow", st_ml["overflow_rows"], "/", st_ml["rows"], "err", st_ml["mean_abs_log2_error"])
    assert st_ub["overflow_rows"] == 0
    # scratch beyond the exact size: the model removes at least half of the bound's
    excess_ub = st_ub["scratch_entries"] - st_ub["nnz"]
    excess_ml = st_ml["scratch_entries"] - st_ml["nnz"]
    assert excess_ml <= 0.5 * excess_ub
    assert st_ml["overflow_rows"] <= 0.05 * st_ml["rows"]
    assert 0 <= st_ml["mean_abs_log2_error"] < 0.5


@pytest.mark.parametrize("alg", ALL)
def test_learned_column_slabs_equal_plain(H, trained, alg):
    """More than 2^18 output columns: every column slab is its own learned pass;
    the result equals the plain product under any model, and the oracle's."""
    import paper_1512_00066_b300 as stc
    w, _ = trained
    A = W.random_csr(500, 900, 40, seed=51, empty_frac=0.05)
    B = W.random_csr(900, 2 * (1 << 18) + 777, 300, seed=52, empty_frac=0.05)
    A.val = _vals(alg, A.nnz, 53)
    B.val = _vals(alg if alg != O.MULTPATH else O.MP_I32, B.nnz, 54) if alg != O.MULTPATH else \
        W.multpath_values(B.nnz, 20, 5, 54)
    dA, dB = to_dev(A), to_dev(B)
    plain = H.spgemm(alg, dA, dB)
    under = torch.zeros(stc.MLP_NUM_WEIGHTS, dtype=torch.float32, device="cuda")
    for weights, margin in ((w, 0.25), (None, 0.0), (under, 0.0)):
        C, st = H.spgemm_learned(alg, dA, dB, weights, margin)
        _same(alg, C, plain)
        assert st["nnz"] == plain.nnz and st["rows"] > A.nrows  # (row, slab) units
    C, st = H.spgemm_learned(alg, dA, dB, under, 0.0)
    assert st["overflow_rows"] > 0 and st["recomputed_rows"] > 0
    if alg == O.PT_F32:
        rp, col, val = C.to_host()
        ptr, rcol, rval, rabs = O.spgemm(alg, A, B, want_abs=True)
        assert np.array_equal(rp, ptr) and np.array_equal(col, rcol)
        compare_values(alg, val, rval, rabs)


def test_training_rows_are_features_and_exact_log_counts(H):
    """stc_training_rows: the features of stc_row_features and targets
    log2(1 + nnz(C_i)) from the symbolic phase; stc_row_counts equals the oracle's
    row counts, also past 2^18 output columns (counted slab by slab)."""
    import paper_1512_00066_b300 as stc
    for A, B in ((W.rmat(12, seed=21), None),
                 (W.random_csr(300, 700, 30, seed=22, empty_frac=0.1),
                  W.random_csr(700, 3 * (1 << 18) + 5, 200, seed=23, empty_frac=0.1))):
        B = A if B is None else B
        dA = stc.DeviceCsr.from_host(A.nrows, A.ncols, A.rowptr, A.col, None)
        dB = stc.DeviceCsr.from_host(B.nrows, B.ncols, B.rowptr, B.col, None)
        cnt = O.spgemm_count(A, B)
        assert np.array_equal(H.row_counts(dA, dB).cpu().numpy(), cnt)
        f, t = H.training_rows_of(dA, dB)
        assert torch.equal(f, H.row_features(dA, dB))
        assert np.array_equal(t.cpu().numpy(), np.log2(1.0 + cnt).astype(np.float32))


def test_model_file_round_trip_and_rejections(H, trained, tmp_path):
    import paper_1512_00066_b300 as stc
    w, _ = trained
    p = tmp_path / "model.stc"
    stc.model_save(p, w)
    assert torch.equal(stc.model_load(p), w)
    raw = bytearray(p.read_bytes())
    assert len(raw) == 32 + 4 * stc.MLP_NUM_WEIGHTS and raw[:8] == b"STCMLP1\0"
    for bad in (raw[:-4], raw + b"\0", raw[:40] + bytes([raw[40] ^ 1]) + raw[41:], b"XXXXXXX\0" + raw[8:]):
        q = tmp_path / "bad.stc"
        q.write_bytes(bytes(bad))
        with pytest.raises(stc.StcError):
            stc.model_load(q)
    with pytest.raises(stc.StcError):
        stc.model_load(tmp_path / "missing.stc")


def _block_hashes(col: torch.Tensor, block: int = 1 << 27):
    """64-bit hash of every block of `block` consecutive entries: sum of col * w
    with fixed odd random weights w, in wrapping int64 arithmetic."""
    g = torch.Generator(device="cuda").manual_seed(12345)
    w = torch.randint(-(1 << 62), 1 << 62, (block,), dtype=torch.int64, device="cuda", generator=g) | 1
    out = []
    for s in range(0, col.numel(), block):
        c = col[s:s + block].to(torch.int64)
        out.append(int((c * w[:c.numel()]).sum()))
    return out


def _rows_of(C, rows):
    """(row pointers, columns, values) of the listed rows of device CSR C, on the host."""
    r = torch.from_numpy(rows).cuda()
    start = C.rowptr[r]
    lens = C.rowptr[r + 1] - start
    ptr = torch.zeros(rows.size + 1, dtype=torch.int64, device="cuda")
    ptr[1:] = torch.cumsum(lens, 0)
    idx = torch.repeat_interleave(start - ptr[:-1], lens) + torch.arange(int(ptr[-1]), device="cuda")
    return ptr.cpu().numpy(), C.col[idx].cpu().numpy(), C.val[idx].cpu().numpy()


def test_rmat20_learned_full_size_structure_and_sampled_values(H, trained):
    """The learned-sizing workload at full size: (+,x) fp32 A.A on R-MAT scale 20
    (2^20 output columns, four slabs).  The learned result has the plain result's
    row pointers exactly and the same column array (64-bit hash of every block of
    2^27 entries); values of every 64th row and of the 1024 longest rows against
    the fp64 oracle within relative 1e-5."""
    import paper_1512_00066_b300 as stc
    w, _ = trained
    A = W.rmat(20, seed=0)
    A.val = W.weights_unit01(A.nnz, seed=0).astype(np.float32)
    dA = to_dev(A)
    plain = H.spgemm(O.PT_F32, dA, dA)
    p_ptr = plain.rowptr.cpu().numpy()
    p_hash = _block_hashes(plain.col)
    lens = np.diff(p_ptr)
    rows = np.unique(np.r_[np.arange(0, A.nrows, 64), np.argsort(lens)[-1024:]]).astype(np.int64)
    del plain
    torch.cuda.empty_cache()
    C, st = H.spgemm_learned(O.PT_F32, dA, dA, w, 0.5)
    assert st["nnz"] == int(p_ptr[-1]) and st["rows"] > A.nrows
    assert np.array_equal(C.rowptr.cpu().numpy(), p_ptr)
    assert _block_hashes(C.col) == p_hash
    gptr, gcol, gval = _rows_of(C, rows)
    del C
    torch.cuda.empty_cache()
    ptr, rcol, rval, rabs = O.spgemm(O.PT_F32, A, A, rows=rows, want_abs=True)
    assert np.array_equal(gptr, ptr) and np.array_equal(gcol, rcol)
    compare_values(O.PT_F32, gval, rval, rabs, "rmat20 learned rows")
