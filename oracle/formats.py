"""Storage formats for the coupling weights (test infrastructure).

The paper's own solvers hold the weights in S or D (Sec. 2.3).  The extension
to bfloat16 / fp16 / fp8 named in its conclusion (Sec. 4) is defined here as:

1. round the weights to FP32 (round to nearest even);
2. choose a per-row scale s_i:
   * f64, f32, bf16: s_i = 1;
   * f16: s_i = 2^max(e_i - 14, -126), where 2^e_i <= max_j |K_ij| < 2^(e_i+1),
     so every row maps into [2^14, 2^15) without fp16 overflow or underflow;
   * fp8 (E4M3): s_i = fp32(max_j |K_ij| / 448);
   * an all-zero row has s_i = 1;
3. q_ij = round_nearest_even(fp32(K_ij / s_i)) in the target format
   (fp8 saturates to +-448).

The weight actually used is s_i * q_ij.  Every routine is written from the
IEEE-754 / OCP-FP8 format definitions; they are pinned against torch's and
numpy's own conversions in tests/test_oracle_formats.py.
"""

from __future__ import annotations

import numpy as np

FORMATS = ("f64", "f32", "bf16", "f16", "fp8e4m3")

FP8_E4M3_MAX = 448.0


def round_bf16(x32: np.ndarray) -> np.ndarray:
    """FP32 -> bfloat16 (round to nearest even), returned as exact FP32 values."""
    x32 = np.ascontiguousarray(x32, dtype=np.float32)
    bits = x32.view(np.uint32).astype(np.uint64)
    lsb = (bits >> np.uint64(16)) & np.uint64(1)
    rounded = ((bits + np.uint64(0x7FFF) + lsb) >> np.uint64(16)) << np.uint64(16)
    return rounded.astype(np.uint32).view(np.float32).reshape(x32.shape)


def round_f16(x32: np.ndarray) -> np.ndarray:
    """FP32 -> IEEE binary16 (round to nearest even), as exact FP32 values."""
    return np.asarray(x32, dtype=np.float32).astype(np.float16).astype(np.float32)


def round_fp8_e4m3(x32: np.ndarray) -> np.ndarray:
    """FP32 -> OCP E4M3 (bias 7, 3 mantissa bits, max 448), nearest even, saturating.

    Normal numbers 2^-6 <= |x| have spacing 2^(e-3); below 2^-6 the subnormal
    spacing is 2^-9.  Returned as exact FP32 values.
    """
    x = np.asarray(x32, dtype=np.float32).astype(np.float64)
    a = np.abs(x)
    _, k = np.frexp(a)                      # a = m 2^k, m in [0.5, 1)
    e = np.maximum(k - 1, -6)               # exponent of the binade, subnormals share -6
    spacing = np.ldexp(1.0, e - 3)
    q = np.rint(a / spacing) * spacing      # rint: ties to even
    q = np.minimum(q, FP8_E4M3_MAX)
    return (np.sign(x) * q).astype(np.float32)


def row_scales(k32: np.ndarray, fmt: str) -> np.ndarray:
    """Per-row scales s_i (exact FP32 values, returned as float32)."""
    n = k32.shape[0]
    if fmt in ("f64", "f32", "bf16"):
        return np.ones(n, dtype=np.float32)
    amax = np.max(np.abs(k32), axis=1).astype(np.float32)
    s = np.ones(n, dtype=np.float32)
    nz = amax > 0
    if fmt == "f16":
        _, k = np.frexp(amax[nz].astype(np.float64))
        s[nz] = np.ldexp(1.0, np.maximum(k - 1 - 14, -126)).astype(np.float32)
    elif fmt == "fp8e4m3":
        s[nz] = amax[nz] / np.float32(FP8_E4M3_MAX)   # float32 / float32: IEEE RN
    else:
        raise ValueError(fmt)
    return s


def quantize(K: np.ndarray, fmt: str):
    """Return (q, s): q holds exact stored values (float32, or float64 for f64)."""
    if fmt not in FORMATS:
        raise ValueError(fmt)
    if fmt == "f64":
        return np.asarray(K, dtype=np.float64), np.ones(K.shape[0], dtype=np.float32)
    k32 = np.asarray(K, dtype=np.float32)
    s = row_scales(k32, fmt)
    if fmt == "f32":
        return k32.copy(), s
    q = np.empty_like(k32)
    B = 1024
    for r0 in range(0, k32.shape[0], B):
        r1 = min(k32.shape[0], r0 + B)
        y = k32[r0:r1] / s[r0:r1, None]            # float32 division, RN
        if fmt == "bf16":
            q[r0:r1] = round_bf16(y)
        elif fmt == "f16":
            q[r0:r1] = round_f16(y)
        else:
            q[r0:r1] = round_fp8_e4m3(y)
    return q, s
