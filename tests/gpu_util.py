"""Helpers shared by the GPU parity tests: oracle comparison with the stated tolerances."""
import numpy as np
import pytest
import torch

import oracle as O
import workloads as W

# (+,x): fp64 within rel 1e-12 of the fp64 oracle, fp32 within rel 1e-5; for
# signed values the bound is taken relative to the sum of |products| as well.
TOL_F64 = 1e-12
TOL_F32 = 1e-5


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def to_dev(m: W.Csr):
    import paper_1512_00066_b300 as stc
    return stc.DeviceCsr.from_host(m.nrows, m.ncols, m.rowptr, m.col, m.val)


def dsig_from_raw(raw: np.ndarray) -> np.ndarray:
    return np.ascontiguousarray(raw).view(np.uint8).reshape(-1).view(W.MULTPATH_DTYPE)


def compare_values(alg, got, ref, ref_abs=None, where=""):
    """Elementwise comparison of one contraction's values against the oracle's.

    (+,x): |got - ref| <= tol * max(|ref|, sum of |products|).  On positive data the
    two are equal (plain relative error); on signed data a cancelled sum is judged
    against the magnitude of its terms, which is what bounds rounding error.
    """
    if alg == O.PT_F64 or alg == O.PT_F32:
        tol = TOL_F64 if alg == O.PT_F64 else TOL_F32
        got = got.astype(np.float64)
        err = np.abs(got - ref)
        scale = np.abs(ref) if ref_abs is None else np.maximum(np.abs(ref), ref_abs)
        bad = err > tol * scale
        assert not bad.any(), f"{where}: {bad.sum()} values off, worst {np.max(err / np.maximum(scale, 1e-300))}"
    elif alg == O.MULTPATH:
        g = dsig_from_raw(got)
        assert np.array_equal(g["d"], ref["d"]), where
        assert np.array_equal(g["s"], ref["s"]), where
    elif alg == O.MP_F32:
        assert got.astype(np.float32).tobytes() == ref.astype(np.float32).tobytes(), where
    else:
        assert np.array_equal(got.astype(np.int64), ref.astype(np.int64)), where


# ----------------------------------------------------------------- tensor-core perceptron
MLP_NF, MLP_NH = 67, 64


def mlp_unpack(w: np.ndarray):
    """W1, b1, W2, b2, w3, b3 of the perceptron's flat weight vector."""
    NF, NH = MLP_NF, MLP_NH
    W1 = w[:NH * NF].reshape(NH, NF)
    b1 = w[NH * NF:NH * NF + NH]
    W2 = w[NH * NF + NH:NH * NF + NH + NH * NH].reshape(NH, NH)
    b2 = w[NH * NF + NH + NH * NH:NH * NF + 2 * NH + NH * NH]
    w3 = w[NH * NF + 2 * NH + NH * NH:NH * NF + 3 * NH + NH * NH]
    return W1, b1, W2, b2, w3, w[-1]


def mlp_tc_tolerance(wd: np.ndarray, x: np.ndarray, yr: np.ndarray) -> np.ndarray:
    """Per-row tolerance of the tensor-core perceptron against the fp64 oracle.

    The kernel carries every fp32 input of both hidden layers as bf16 hi + lo, an
    error of at most 2^-16 of the value, and sums in fp32.  Rounding errors add up
    like independent terms, so their scale is the root-sum-square of each input's
    2^-16 |value| carried to y through the weights (wd: the bf16-rounded weights, x:
    the fp64 inputs, yr: the oracle's outputs):
        e1 = 2^-16 sqrt((W1e^2) (xe^2)),  xe = (x, 1), W1e = (W1, b1)
        e2 = sqrt((W2^2) (e1^2 + (2^-16 h1)^2)),  h1 = relu(W1e xe)
        ey = sqrt((w3^2) . e2^2)
    The tolerance is 4 ey, plus 2^-20 (1 + |y|) for the fp32 sums and output.  Exact
    emulation of the arithmetic stays within 0.6 ey; leaving out the lo halves puts
    the median row above 20 ey."""
    W1, b1, W2, b2, w3, _ = mlp_unpack(np.asarray(wd, np.float64))
    W1e = np.concatenate([W1, b1[:, None]], axis=1)
    xe = np.concatenate([np.asarray(x, np.float64), np.ones((x.shape[0], 1))], axis=1)
    s = 2.0 ** -16
    h1 = np.maximum(xe @ W1e.T, 0.0)
    e1 = s * np.sqrt((xe ** 2) @ (W1e ** 2).T)
    e2 = np.sqrt((e1 ** 2 + (s * h1) ** 2) @ (W2 ** 2).T)
    ey = np.sqrt((e2 ** 2) @ (w3 ** 2))
    return 4.0 * ey + 2.0 ** -20 * (1.0 + np.abs(yr))
