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
