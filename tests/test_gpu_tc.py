"""Tensor-core (tcgen05) split-bfloat16 product against the oracle's
definition: C = A_hi B_hi^T + A_hi B_lo^T + A_lo B_hi^T in binary64."""

import numpy as np
import pytest

from oracle.formats import round_bf16
from tests.gpu_helpers import library, torch_cuda

pytestmark = pytest.mark.gpu


def _split(x):
    x = x.astype(np.float32)
    hi = round_bf16(x)
    lo = round_bf16((x - hi).astype(np.float32))
    return hi.astype(np.float64), lo.astype(np.float64)


def _run(A, B):
    bs3 = library()
    torch = torch_cuda()
    Ad = torch.tensor(A, dtype=torch.float32, device="cuda")
    Bd = torch.tensor(B, dtype=torch.float32, device="cuda")
    C = torch.full((A.shape[0], B.shape[0]), float("nan"), dtype=torch.float32, device="cuda")
    rc = bs3.bs3_tc_gemm(A.shape[0], B.shape[0], A.shape[1], Ad, Bd, C)
    assert rc == bs3.OK, bs3.bs3_status_string(rc)
    return C.cpu().numpy().astype(np.float64)


def test_permutation_rows_are_exact():
    """A = permutation: each output is b_hi + b_lo of one row of B (exact in binary32)."""
    rng = np.random.default_rng(0)
    M, Nc, K = 128, 256, 128
    perm = rng.permutation(K)[:M]
    A = np.zeros((M, K), dtype=np.float32)
    A[np.arange(M), perm] = 1.0
    B = rng.standard_normal((Nc, K)).astype(np.float32)
    C = _run(A, B)
    bh, bl = _split(B)
    np.testing.assert_array_equal(C, (bh + bl)[:, perm].T)


@pytest.mark.parametrize("M,Nc,K", [(128, 256, 64), (256, 512, 320), (512, 256, 2048)])
def test_matches_split_definition(M, Nc, K):
    rng = np.random.default_rng(M + Nc + K)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.uniform(-1, 1, (Nc, K)).astype(np.float32)
    C = _run(A, B)
    ah, al = _split(A)
    bh, bl = _split(B)
    ref = ah @ bh.T + ah @ bl.T + al @ bh.T
    mag = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    # binary32 accumulation of 3K products (any order): <= (3K) u32 sum|a||b|
    assert np.all(np.abs(C - ref) <= 3 * K * 2.0 ** -24 * mag + 1e-30)
    # the split keeps about 16 significant bits of each operand
    exact = A.astype(np.float64) @ B.astype(np.float64).T
    assert np.max(np.abs(C - exact) / mag) < 2.0 ** -14


@pytest.mark.parametrize("tile_n,max_ctas", [(128, 0), (128, 37), (256, 19)])
def test_persistent_product_matches_split_definition(tile_n, max_ctas):
    """The ensembles' form of the product (persistent CTAs, two tensor-memory
    accumulators) at the shared-K size: M = K = 8192, Nc = 512.  With 37 (19)
    CTAs every CTA takes about 7 tiles, so both accumulators are reused and the
    operand ring runs on across tiles; every output is written (no NaN left)."""
    bs3 = library()
    torch = torch_cuda()
    M, Nc, K = 8192, 512, 8192
    rng = np.random.default_rng(tile_n + max_ctas)
    A = rng.standard_normal((M, K)).astype(np.float32)
    B = rng.uniform(-1, 1, (Nc, K)).astype(np.float32)
    Ad = torch.tensor(A, device="cuda")
    Bd = torch.tensor(B, device="cuda")
    C = torch.full((M, Nc), float("nan"), dtype=torch.float32, device="cuda")
    rc = bs3.bs3_tc_gemm_persistent(M, Nc, K, Ad, Bd, C, tile_n, max_ctas)
    assert rc == bs3.OK, bs3.bs3_status_string(rc)
    C = C.cpu().numpy().astype(np.float64)
    assert np.all(np.isfinite(C))
    ah, al = _split(A)
    bh, bl = _split(B)
    ref = ah @ (bh + bl).T + al @ bh.T          # bh + bl is exact in binary64
    mag = np.abs(A).astype(np.float64) @ np.abs(B).astype(np.float64).T
    assert np.all(np.abs(C - ref) <= 3 * K * 2.0 ** -24 * mag + 1e-30)
    exact = A.astype(np.float64) @ B.astype(np.float64).T
    assert np.max(np.abs(C - exact) / mag) < 2.0 ** -14


def _persistent(A, B, tile_n, max_ctas):
    bs3 = library()
    torch = torch_cuda()
    Ad = torch.tensor(A, dtype=torch.float32, device="cuda")
    Bd = torch.tensor(B, dtype=torch.float32, device="cuda")
    C = torch.full((A.shape[0], B.shape[0]), float("nan"), dtype=torch.float32, device="cuda")
    rc = bs3.bs3_tc_gemm_persistent(A.shape[0], B.shape[0], A.shape[1], Ad, Bd, C, tile_n, max_ctas)
    assert rc == bs3.OK, bs3.bs3_status_string(rc)
    return C.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("tile_n,max_ctas", [(128, 37), (256, 19)])
def test_persistent_one_hot_products_are_exact(tile_n, max_ctas):
    """Every output of a one-hot product is one split pair, hi + lo, with no
    rounding in the accumulation, so it must equal the split exactly:
    B one-hot (row n selects column k_n of A): C = A_hi + A_lo at (m, k_n),
    which needs the A_lo B_hi product; A one-hot: C = B_hi + B_lo, which needs
    A_hi B_lo.  The selected columns lie in every 64-deep K block, so the
    accumulation across blocks (and a tile placed at the wrong offset) shows
    exactly, at the shared-K size with about 7 tiles per CTA."""
    rng = np.random.default_rng(tile_n)
    M, Nc, K = 8192, 512, 8192
    X = rng.standard_normal((M, K)).astype(np.float32)
    cols = rng.permutation(K)[:Nc]
    sel = np.zeros((Nc, K), dtype=np.float32)
    sel[np.arange(Nc), cols] = 1.0
    xh, xl = _split(X)
    C = _persistent(X, sel, tile_n, max_ctas)
    np.testing.assert_array_equal(C, (xh + xl)[:, cols])
    rows = rng.permutation(K)[:M] if M <= K else rng.integers(0, K, M)
    selA = np.zeros((M, K), dtype=np.float32)
    selA[np.arange(M), rows] = 1.0
    Y = rng.uniform(-1, 1, (Nc, K)).astype(np.float32)
    yh, yl = _split(Y)
    C = _persistent(selA, Y, tile_n, max_ctas)
    np.testing.assert_array_equal(C, (yh + yl)[:, rows].T)


def test_plain_product_one_hot_B_is_exact():
    """bs3_tc_gemm with B one-hot: C = A_hi + A_lo exactly (the A_lo B_hi term)."""
    rng = np.random.default_rng(1)
    M, Nc, K = 256, 512, 1024
    X = rng.standard_normal((M, K)).astype(np.float32)
    cols = rng.integers(0, K, Nc)
    sel = np.zeros((Nc, K), dtype=np.float32)
    sel[np.arange(Nc), cols] = 1.0
    xh, xl = _split(X)
    np.testing.assert_array_equal(_run(X, sel), (xh + xl)[:, cols])
