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
