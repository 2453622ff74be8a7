"""Pins of the numpy emulation that the tensor-core network tests compare
with (no GPU): its BF16 rounding against torch's round-to-nearest-even
conversion and hand-checked ties, and its forward pass and gradient, with the
rounding switched off, against the FP64 oracle (so every term, index and
sign of the emulation is the oracle's)."""
import numpy as np
import pytest
import torch

import oracle
import test_gpu_warm as W


def test_bf16_rounding_is_nearest_even():
    one = np.float32(1.0)
    ulp = np.float32(2.0 ** -7)          # BF16 spacing in [1, 2)
    x = np.array([one + ulp / 2, one + 3 * ulp / 2, one + ulp / 4, -(one + 3 * ulp / 2), 0.0, 3.0e38],
                 dtype=np.float32)
    got = W._bf16(x)
    assert got[0] == 1.0                 # tie to the even neighbour 1
    assert got[1] == 1.0 + 2 * ulp       # tie to the even neighbour 1 + 2^-6
    assert got[2] == 1.0
    assert got[3] == -(1.0 + 2 * ulp)
    assert got[4] == 0.0
    r = np.random.default_rng(0).standard_normal(100000).astype(np.float32) * np.float32(7.0)
    ref = torch.from_numpy(r).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(W._bf16(r), ref)


@pytest.mark.parametrize("widths", [[9, 128, 128, 128, 128, 1], [9, 128, 128, 1], [5, 128, 128, 128, 1]])
def test_emulation_without_rounding_is_the_oracle(monkeypatch, widths):
    monkeypatch.setattr(W, "_bf16", lambda a: np.asarray(a, dtype=np.float64))
    th = W._net(widths, 3, scale=0.3)
    rng = np.random.default_rng(1)
    X = rng.uniform(-1, 1, (37, widths[0])).astype(np.float32)
    T = rng.standard_normal(37).astype(np.float32)
    y = W._forward_bf16(widths, th, X)
    y_o = oracle.mlp_forward(widths, th.astype(np.float64), X.astype(np.float64))
    assert np.abs(y - y_o).max() <= 1e-13 * np.abs(y_o).max()
    lo, g = W._grad_bf16(widths, th, X, T)
    lo_o, g_o = oracle.mlp_grad(widths, th.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    assert lo == pytest.approx(lo_o, rel=1e-13)
    assert np.abs(g - g_o).max() <= 1e-13 * np.abs(g_o).max()


def test_emulation_with_rounding_stays_near_the_oracle():
    """With the BF16 roundings the emulated gradient moves from the oracle's by
    about 1e-2 normwise (8 significant bits per operand), not more."""
    widths = [9, 128, 128, 128, 128, 1]
    th = W._net(widths, 4, scale=0.3)
    rng = np.random.default_rng(2)
    X = rng.uniform(-1, 1, (300, 9)).astype(np.float32)
    T = rng.standard_normal(300).astype(np.float32)
    _, g = W._grad_bf16(widths, th, X, T)
    _, g_o = oracle.mlp_grad(widths, th.astype(np.float64), X.astype(np.float64), T.astype(np.float64))
    rel = np.linalg.norm(g - g_o) / np.linalg.norm(g_o)
    assert 1e-4 < rel < 5e-2
