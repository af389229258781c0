"""Dormand-Prince 5(4) reference integrator (binary64).

The paper's reference solutions come from an ode45 (Dormand-Prince 5(4))
solve in double precision at a tight tolerance (Sec. 2.4, Eq. Metric).  This
is a plain restatement: tableau of oracle.tableau (Dormand & Prince 1980),
local extrapolation (the fifth-order solution is kept), FSAL, the error norm
sqrt(mean((err_k / (atol + rtol max(|y_k|, |ynew_k|)))^2)), and the standard
controller h <- h min(5, max(0.2, 0.9 err^(-1/5))).  Pinned against closed
forms and against scipy's RK45 in tests/test_oracle_solver.py.
"""

from __future__ import annotations

import numpy as np

from . import models
from .tableau import DP5_A, DP5_B, DP5_BSTAR, DP5_C, as_float

_A = as_float(DP5_A)
_B = np.array(as_float(DP5_B))
_E = np.array(as_float(DP5_B)) - np.array(as_float(DP5_BSTAR))
_C = as_float(DP5_C)


def integrate(f, t0, t1, y0, rtol=1e-12, atol=1e-12, max_steps=2_000_000):
    """Integrate y' = f(t, y) from t0 to t1; returns (y(t1), accepted, rejected)."""
    y = np.asarray(y0, dtype=np.float64).copy()
    t = float(t0)
    k = [None] * 7
    k[0] = f(t, y)
    # starting step (Hairer-Norsett-Wanner II.4, RMS norm, order 5)
    sc = atol + rtol * np.abs(y)
    d0 = np.sqrt(np.mean((y / sc) ** 2))
    d1 = np.sqrt(np.mean((k[0] / sc) ** 2))
    h0 = 0.01 * d0 / d1 if (d0 >= 1e-5 and d1 >= 1e-5) else 1e-6
    f1 = f(t + h0, y + h0 * k[0])
    d2 = np.sqrt(np.mean(((f1 - k[0]) / sc) ** 2)) / h0
    m = max(d1, d2)
    h1 = (0.01 / m) ** 0.2 if m > 1e-15 else max(1e-6, h0 * 1e-3)
    h = min(100 * h0, h1, abs(t1 - t0))
    acc = rej = 0
    while t < t1:
        if acc + rej > max_steps:
            raise RuntimeError("DOPRI5 reference: too many steps")
        if t + h >= t1:
            h = t1 - t
        for s in range(1, 7):
            ys = y + h * sum(_A[s][m] * k[m] for m in range(s))
            k[s] = f(t + _C[s] * h, ys)
        ynew = ys  # the seventh stage argument is the fifth-order solution (FSAL)
        err_v = h * sum(_E[m] * k[m] for m in range(7))
        sc = atol + rtol * np.maximum(np.abs(y), np.abs(ynew))
        err = float(np.sqrt(np.mean((err_v / sc) ** 2)))
        if err <= 1.0:
            t = t1 if t + h >= t1 else t + h
            y = ynew
            k[0] = k[6]
            acc += 1
            h = h * (5.0 if err == 0 else min(5.0, max(0.2, 0.9 * err ** -0.2)))
        else:
            rej += 1
            h = h * max(0.2, 0.9 * err ** -0.2)
    return y, acc, rej


def reference_solution(sysm: models.System, t0, t1, y0, rtol=1e-12, atol=1e-12):
    """Binary64 DOPRI5 solution of a benchmark system at t1."""
    f = lambda t, y: models.rhs(sysm, t, y, ("D", "D", "D"))  # noqa: E731
    y, _, _ = integrate(f, t0, t1, y0, rtol, atol)
    return y
