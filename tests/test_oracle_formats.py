"""Pins of the oracle's storage formats against torch's / numpy's own casts."""

import numpy as np
import pytest
import torch

from oracle import formats


def _probe_values(rng, n=20000):
    x = rng.standard_normal(n).astype(np.float32) * np.float32(10.0) ** rng.integers(-8, 4, n).astype(np.float32)
    # exact ties for bf16 (lower 16 bits == 0x8000) and for fp16
    mant = rng.integers(0, 2**7, 500).astype(np.uint32) << np.uint32(16)
    expo = rng.integers(100, 150, 500).astype(np.uint32) << np.uint32(23)
    ties = (expo | mant | np.uint32(0x8000)).view(np.float32)
    return np.concatenate([x, ties, -ties, np.array([0.0, -0.0, 1.0, 448.0, 447.0, 460.0, 1e-12],
                                                     dtype=np.float32)])


def test_bf16_matches_torch():
    x = _probe_values(np.random.default_rng(1))
    ref = torch.from_numpy(x).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(formats.round_bf16(x), ref)


def test_f16_matches_torch():
    x = _probe_values(np.random.default_rng(2))
    x = x[np.abs(x) < 60000]
    ref = torch.from_numpy(x).to(torch.float16).to(torch.float32).numpy()
    np.testing.assert_array_equal(formats.round_f16(x), ref)


def test_fp8_matches_torch_in_range():
    rng = np.random.default_rng(3)
    x = (rng.standard_normal(50000) * 100).astype(np.float32)
    x = np.concatenate([x, (rng.standard_normal(5000) * 1e-3).astype(np.float32)])
    x = x[np.abs(x) <= 448]
    ref = torch.from_numpy(x).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    np.testing.assert_array_equal(formats.round_fp8_e4m3(x), ref)


def test_fp8_saturates():
    x = np.array([449.0, 470.0, 1e6, -1e6], dtype=np.float32)
    np.testing.assert_array_equal(formats.round_fp8_e4m3(x), [448.0, 448.0, 448.0, -448.0])


@pytest.mark.parametrize("fmt", ["f16", "fp8e4m3"])
def test_row_scaled_formats_cover_rows(fmt):
    rng = np.random.default_rng(4)
    K = rng.uniform(0, 1, (64, 200)) / 32768.0          # below fp16's normal range unscaled
    K[5] = 0.0
    q, s = formats.quantize(K, fmt)
    assert s[5] == 1.0 and np.all(q[5] == 0)
    rec = s[:, None].astype(np.float64) * q
    rel = np.abs(rec - K) / np.max(np.abs(K), axis=1, keepdims=True).clip(1e-300)
    bound = 2.0 ** -11 if fmt == "f16" else 2.0 ** -4   # half an ulp at the row maximum
    assert np.max(rel[np.arange(64) != 5]) <= bound
    if fmt == "f16":
        amax = np.max(np.abs(q), axis=1)
        assert np.all((amax[np.arange(64) != 5] >= 2 ** 14) & (amax[np.arange(64) != 5] <= 2 ** 15))
    else:
        assert np.max(np.abs(q)) <= 448.0
