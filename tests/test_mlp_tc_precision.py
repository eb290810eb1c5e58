"""Host model of the tensor-core perceptron's arithmetic (CPU only).

The tcgen05 kernel feeds every fp32 activation to bf16 MMAs as hi = bf16(x) plus
lo = bf16(x - hi) against bf16 weights, accumulates in fp32, adds b1 through a
constant-1 input and evaluates the 64 -> 1 output layer in fp32.  These tests pin
the split's error bound, check the worst-case error bound of that arithmetic, and
check that the GPU parity tolerance (gpu_util.mlp_tc_tolerance, a root-sum-square
rounding-error scale) holds for the arithmetic with a margin and fails when the lo
halves are left out.
"""
import numpy as np
import torch

import oracle as O
from gpu_util import MLP_NF as NF, MLP_NH as NH, mlp_tc_tolerance, mlp_unpack as unpack


def bf16(x: np.ndarray) -> np.ndarray:
    """Round fp32 values to bf16 (nearest, ties to even) and back to fp32."""
    return torch.from_numpy(np.ascontiguousarray(x, dtype=np.float32)).to(torch.bfloat16).to(torch.float32).numpy()


def split(x: np.ndarray):
    hi = bf16(x)
    lo = bf16(x.astype(np.float32) - hi)
    return hi, lo


def test_hi_lo_split_error_bound():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(200000) * 10.0 ** rng.integers(-6, 6, 200000),
                        rng.random(50000), -rng.random(50000) * 40.0]).astype(np.float32)
    hi, lo = split(x)
    err = np.abs(x.astype(np.float64) - hi.astype(np.float64) - lo.astype(np.float64))
    assert np.all(err <= 2.0 ** -16 * np.abs(x.astype(np.float64)))
    # bf16 alone (one MMA per operand) would be far outside the parity tolerance
    assert np.max(np.abs(x - hi) / np.maximum(np.abs(x), 1e-30)) > 2.0 ** -10


def emulate_tc_forward(w: np.ndarray, x: np.ndarray):
    """The kernel's arithmetic: bf16 weights (b1 as column 67), hi/lo inputs, fp32
    sums.  Returns y and the error bound that this arithmetic implies against the
    exact evaluation with the same bf16 weights."""
    W1, b1, W2, b2, w3, b3 = unpack(bf16(w.astype(np.float32)).astype(np.float64))
    W1e = np.concatenate([W1, b1[:, None]], axis=1)  # input 67 is the constant 1
    xe = np.concatenate([x, np.ones((x.shape[0], 1))], axis=1).astype(np.float32)
    hi, lo = split(xe)
    # products of bf16 values are exact in fp32; the sums are rounded to fp32
    d1 = (hi.astype(np.float64) @ W1e.T + lo.astype(np.float64) @ W1e.T).astype(np.float32)
    h1 = np.maximum(d1, 0.0)
    hhi, hlo = split(h1)
    d2 = (hhi.astype(np.float64) @ W2.T + hlo.astype(np.float64) @ W2.T).astype(np.float32)
    h2 = np.maximum(d2 + b2.astype(np.float32), 0.0).astype(np.float32)
    y = (h2.astype(np.float64) @ w3 + b3).astype(np.float32)
    # error bound: the split's 2^-16 per input, fp32 rounding of every sum (a K-term
    # sum in any order: K 2^-24 of the sum of magnitudes); ReLU is 1-Lipschitz
    u, s16 = 2.0 ** -24, 2.0 ** -16
    ax = np.abs(xe.astype(np.float64))
    e1 = (s16 + 80 * u) * (ax @ np.abs(W1e).T)
    ah1 = np.abs(h1.astype(np.float64))
    e2 = np.abs(W2) @ (e1 + s16 * ah1).T
    e2 = e2.T + 65 * u * (ah1 @ np.abs(W2).T + np.abs(b2))
    ey = e2 @ np.abs(w3) + 65 * u * (np.abs(h2.astype(np.float64)) @ np.abs(w3) + abs(b3))
    return y, ey


def he_weights(rng) -> np.ndarray:
    """He-normal layers and zero biases, the initialisation of stc_mlp_init."""
    W1 = rng.standard_normal((NH, NF)) * np.sqrt(2.0 / NF)
    W2 = rng.standard_normal((NH, NH)) * np.sqrt(2.0 / NH)
    w3 = rng.standard_normal(NH) * np.sqrt(2.0 / NH)
    return np.concatenate([W1.ravel(), np.zeros(NH), W2.ravel(), np.zeros(NH), w3, [0.0]]).astype(np.float32)


def test_emulated_kernel_within_derived_bound():
    """Stress weights (every weight and bias N(0, 1/16)) and signed inputs: the
    emulation stays inside the bound derived from its arithmetic."""
    rng = np.random.default_rng(3)
    w = (rng.standard_normal(O.mlp_num_weights()) / 4).astype(np.float32)
    x = np.concatenate([np.column_stack([rng.random((3000, 3)) * 30, rng.random((3000, NF - 3))]),
                        rng.standard_normal((3000, NF)) * 8]).astype(np.float32)
    y, ey = emulate_tc_forward(w, x)
    yr = O.mlp_forward(bf16(w).astype(np.float64), x.astype(np.float64))
    assert np.all(np.abs(y - yr) <= ey + 1e-30)


def test_emulated_kernel_within_gpu_tolerance():
    """He-initialised and stress weights, feature-like and signed inputs: the
    arithmetic stays well inside the tolerance of the GPU parity tests."""
    rng = np.random.default_rng(5)
    for trial in range(4):
        w = he_weights(rng) if trial < 2 else (rng.standard_normal(O.mlp_num_weights()) / 4).astype(np.float32)
        x = np.concatenate([np.column_stack([rng.random((3000, 3)) * 30, rng.random((3000, NF - 3))]),
                            rng.standard_normal((3000, NF)) * 8]).astype(np.float32)
        y, _ = emulate_tc_forward(w, x)
        wd = bf16(w).astype(np.float64)
        yr = O.mlp_forward(wd, x.astype(np.float64))
        assert np.max(np.abs(y - yr) / mlp_tc_tolerance(wd, x, yr)) <= 0.25


def test_emulation_detects_a_dropped_lo_half():
    """Without the lo halves (plain bf16 inputs) most rows fail the GPU tolerance,
    so the tolerance can tell the split from its absence."""
    rng = np.random.default_rng(4)
    for trial in range(2):
        w = he_weights(rng) if trial == 0 else (rng.standard_normal(O.mlp_num_weights()) / 4).astype(np.float32)
        x = np.concatenate([np.column_stack([rng.random((2000, 3)) * 30, rng.random((2000, NF - 3))]),
                            rng.standard_normal((2000, NF)) * 8]).astype(np.float32)
        wd = bf16(w).astype(np.float64)
        yr = O.mlp_forward(wd, x.astype(np.float64))
        W1, b1, W2, b2, w3, b3 = unpack(wd)
        h1 = np.maximum(bf16(x).astype(np.float64) @ W1.T + b1, 0.0)
        y_hi_only = np.maximum(bf16(h1.astype(np.float32)).astype(np.float64) @ W2.T + b2, 0.0) @ w3 + b3
        assert np.mean(np.abs(y_hi_only - yr) > mlp_tc_tolerance(wd, x, yr)) > 0.9
