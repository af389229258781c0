"""Training pipeline of the learned step-size proposer, through the C ABI:
solves with step recording (bs3_set_history / bs3_get_history) -> training
pairs (bs3_mlp_dataset) -> GPU training (bs3_mlp_train) -> a model for
bs3_set_proposer.  Only argument marshalling happens here."""

from __future__ import annotations

from typing import Iterable, Tuple

import numpy as np

from . import bs3


def histories(workloads: Iterable[Tuple[object, str, str, float]], capacity: int = 200000):
    """Yields (history records, rtol) for (workload, stored weights, variant, rtol)."""
    for w, store, variant, rtol in workloads:
        s = bs3.System.from_workload(w, store)
        rc = bs3.bs3_set_history(s.handle, capacity)
        if rc != bs3.OK:
            raise RuntimeError(bs3.bs3_status_string(rc))
        rc, st, _, _ = s.solve(w.t0, w.t1, w.y0, rtol, rtol, variant, "float2")
        if rc != bs3.OK:
            raise RuntimeError(bs3.bs3_status_string(rc))
        rc, hist = bs3.bs3_get_history(s.handle, capacity)
        s.close()
        yield hist, rtol


def dataset(workloads):
    Xs, ys = [], []
    for hist, rtol in histories(workloads):
        rc, X, y = bs3.bs3_mlp_dataset(hist, rtol)
        if rc != bs3.OK:
            raise RuntimeError(bs3.bs3_status_string(rc))
        Xs.append(X)
        ys.append(y)
    return np.concatenate(Xs), np.concatenate(ys)


def init_params(seed: int) -> np.ndarray:
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights, zero biases (1313 binary32)."""
    rng = np.random.default_rng(seed)
    p = np.zeros(bs3.MLP_PARAMS, dtype=np.float32)
    o = 0
    for fan_in, fan_out in ((6, 32), (32, 32), (32, 1)):
        a = 1.0 / np.sqrt(fan_in)
        p[o:o + fan_in * fan_out] = rng.uniform(-a, a, fan_in * fan_out)
        o += fan_in * fan_out + fan_out
    return p


def train(X, y, epochs: int = 200, batch: int = 256, lr: float = 2e-3, seed: int = 0):
    rc, model, loss = bs3.bs3_mlp_train(X, y, init_params(seed), epochs, batch, lr, seed)
    if rc != bs3.OK:
        raise RuntimeError(bs3.bs3_status_string(rc))
    return model, loss
