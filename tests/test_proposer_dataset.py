"""The library's training-pair builder (host code of libbs3.so) against the
oracle's, on a synthetic step history (no GPU needed)."""

import numpy as np
import pytest

from oracle import mlp


@pytest.fixture(scope="module")
def bs3():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_23727_gb300 import bs3 as b
    b.load()
    return b


def test_dataset_matches_oracle(bs3):
    rng = np.random.default_rng(3)
    n = 300
    hist = np.zeros((n, 8))
    hist[:, 0] = np.cumsum(rng.uniform(0.01, 0.02, n))
    hist[:, 1] = rng.uniform(0.005, 0.05, n)
    hist[:, 2] = 10 ** rng.uniform(-9, -5.8, n)
    hist[:, 3] = (hist[:, 2] <= 1e-6).astype(float)
    hist[5, 2] = 0.0                                   # E = 0 is clamped
    hist[5, 3] = 1.0
    rc, X, y = bs3.bs3_mlp_dataset(hist, 1e-6)
    assert rc == bs3.OK
    Xo, yo = mlp.dataset_from_history(hist, 1e-6)
    assert X.shape == Xo.shape and X.shape[0] == int(hist[:, 3].sum()) - 1
    np.testing.assert_allclose(X, Xo.astype(np.float32), rtol=1e-6, atol=1e-6)
    np.testing.assert_allclose(y, yo.astype(np.float32), rtol=1e-6, atol=1e-6)
