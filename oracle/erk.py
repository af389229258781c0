"""Adaptive embedded Runge-Kutta pairs with the paper's precision variants
(test infrastructure).

The solver of oracle/bs3.py written for any explicit FSAL pair, here the
Bogacki-Shampine 3(2) pair itself and Dormand-Prince 5(4): the paper notes
that its mixed-precision approach carries over to other explicit schemes
(Sec. 4); this module is that extension, step by step:

* stages K_l = f(t + c_l h, Y_l), Y_l = X^n + h (sum_{m<l} a_lm K_m) with the
  sum taken over the nonzero a_lm in increasing m, in the state precision;
* FSAL: the last stage argument is X^{n+1} (a_s = b), K_s = f(t+h, X^{n+1})
  is the next K_1 after an accepted step;
* error as Eq. ERROR-O23: Dv = h (sum_m e_m K_m), e = b - b_hat, nonzero e_m in
  increasing m, E = max_k |Dv_k| / max(|X^n_k|, |X^{n+1}_k|, Ab/Rel), accept
  when E <= Rel;
* failure conditions, h_max, the stretched last step, the starting step and
  dense output (cubic Hermite on X^n, K_1, X^{n+1}, K_s) as in oracle/bs3.py.

Readings where the paper is silent (parity unpinned; the paper runs BS3
only): the controller exponent and the starting-step exponent are 1/(q+1)
with q the order of the embedded solution (BS3: q = 2, DP5: q = 4), the other
controller constants as for BS3; the precision table extends Table
MP-Distrib stage by stage: Single all stages (S, S, S); Mixed1 every stage
(S, S, S) except the last, FSAL stage (D, D, S); Mixed2 every stage (D, D, S);
Double (D, D, D).  The first K_1 and the starting-step evaluation use the
last stage's row.

Pinned in tests/test_oracle_erk.py: with the BS3 pair it takes the same steps
as oracle/bs3.py; the DP5 pair shows order 5 on fixed steps and tracks the
closed form of the second-order oscillators under error control.
"""

from __future__ import annotations

import dataclasses
import time
from typing import Optional, Sequence

import numpy as np

from . import models
from .bs3 import (ERR_MAX_REJECTS, ERR_MAX_STEPS, ERR_NONFINITE, ERR_STEP_TOO_SMALL, ERR_TIMEOUT,
                  GROW_MAX, HMAX_FRACTION, OK, SAFETY, SHRINK_FIRST_MIN, SHRINK_REPEAT, STRETCH,
                  Limits, Result, error_norm, hermite)
from .tableau import (BS3_A, BS3_B, BS3_BTILDE, BS3_C, DP5_A, DP5_B, DP5_BSTAR, DP5_C)


@dataclasses.dataclass(frozen=True)
class Pair:
    name: str
    c: tuple          # nodes c_1..c_s (floats)
    a: tuple          # rows a_l (l = 1..s), each a tuple of l-1 floats
    e: tuple          # b - b_hat (floats)
    q: int            # order of the embedded solution

    @property
    def stages(self) -> int:
        return len(self.c)


def _pair(name, C, A, B, BH, q):
    e = tuple(float(b - bh) for b, bh in zip(B, BH))
    return Pair(name, tuple(float(x) for x in C), tuple(tuple(float(x) for x in row) for row in A), e, q)


PAIRS = {
    "bs3": _pair("bs3", BS3_C, BS3_A, BS3_B, BS3_BTILDE, 2),
    "dp5": _pair("dp5", DP5_C, DP5_A, DP5_B, DP5_BSTAR, 4),
}

_S, _MIX, _D = ("S", "S", "S"), ("D", "D", "S"), ("D", "D", "D")


def stage_precision(variant: str, l: int, s: int):
    """(F, Sigma, G) of stage l (2..s) of an s-stage pair."""
    if variant == "single":
        return _S
    if variant == "mixed1":
        return _MIX if l == s else _S
    if variant == "mixed2":
        return _MIX
    if variant == "double":
        return _D
    raise ValueError(variant)


def _comb(coefs, K, st):
    """sum_m coefs[m] K_m over the nonzero coefficients, in increasing m,
    in the state precision st."""
    acc = None
    for m, a in enumerate(coefs):
        if a == 0.0:
            continue
        term = st(a) * K[m]
        acc = term if acc is None else acc + term
    return acc


def attempt(pair: Pair, sysm, t, X, K1, h, variant, rtol, atol):
    """One attempt: returns (X^{n+1}, K_s, E, K)."""
    s = pair.stages
    st = X.dtype.type
    hs = st(h)
    K = [K1]
    Y = X
    for l in range(2, s + 1):
        Y = X + hs * _comb(pair.a[l - 1], K, st)
        K.append(models.rhs(sysm, t + pair.c[l - 1] * h, Y, stage_precision(variant, l, s)))
    Xn = Y                                  # a_s = b: the last stage argument
    Dv = hs * _comb(pair.e, K, st)
    return Xn, K[-1], error_norm(X, Xn, Dv, rtol, atol), K


def initial_step(pair, sysm, t0, y0, f0, rtol, atol, hmax, prec):
    sc = rtol * np.maximum(np.abs(y0.astype(np.float64)), atol / rtol)
    d0 = float(np.max(np.abs(y0.astype(np.float64)) / sc))
    d1 = float(np.max(np.abs(f0.astype(np.float64)) / sc))
    h0 = 0.01 * d0 / d1 if (d0 >= 1e-5 and d1 >= 1e-5) else 1e-6
    st = y0.dtype.type
    f1 = models.rhs(sysm, t0 + h0, y0 + st(h0) * f0, prec)
    d2 = float(np.max(np.abs(f1.astype(np.float64) - f0.astype(np.float64)) / sc)) / h0
    m = max(d1, d2)
    h1 = (0.01 / m) ** (1.0 / (pair.q + 1)) if m > 1e-15 else max(1e-6, h0 * 1e-3)
    return min(100.0 * h0, h1, hmax)


def solve(pair: Pair, sysm: models.System, t0: float, t1: float, y0: np.ndarray, rtol: float, atol: float,
          variant: str = "double", t_out: Optional[Sequence[float]] = None,
          limits: Optional[Limits] = None) -> Result:
    lim = limits or Limits()
    s = pair.stages
    expo = 1.0 / (pair.q + 1)
    state_t = np.float32 if variant == "single" else np.float64
    hmin = lim.hmin_factor * float(np.finfo(state_t).eps)
    hmax = HMAX_FRACTION * abs(t1 - t0)
    t_out = np.asarray([] if t_out is None else t_out, dtype=np.float64)
    y_out = np.full((len(t_out), sysm.d * sysm.N), np.nan)
    next_out = 0
    while next_out < len(t_out) and t_out[next_out] <= t0:
        y_out[next_out] = y0
        next_out += 1
    X = np.asarray(y0, dtype=np.float64).astype(state_t)
    if not np.all(np.isfinite(X)):
        return Result(X.astype(np.float64), t0, y_out, 0, 0, 0, ERR_NONFINITE, 0.0)
    last_prec = stage_precision(variant, s, s)
    K1 = models.rhs(sysm, t0, X, last_prec)
    h = initial_step(pair, sysm, t0, X, K1, rtol, atol, hmax, last_prec)
    n_rhs = 2
    t = float(t0)
    n_acc = n_rej = 0
    status = OK if np.all(np.isfinite(K1)) else ERR_NONFINITE
    rejected_this_step = False
    started = time.monotonic()
    while status == OK and t < t1:
        if n_rej > lim.max_rejects:
            status = ERR_MAX_REJECTS
            break
        if n_acc + n_rej >= lim.max_attempts:
            status = ERR_MAX_STEPS
            break
        elapsed = time.monotonic() - started
        if elapsed > lim.wall_limit_s or (elapsed > lim.slow_limit_s and
                                          (t - t0) < lim.slow_fraction * (t1 - t0)):
            status = ERR_TIMEOUT
            break
        h = min(h, hmax)
        if h <= hmin:
            status = ERR_STEP_TOO_SMALL
            break
        last = t + STRETCH * h >= t1
        if last:
            h = t1 - t
        Xn, Ks, err, _ = attempt(pair, sysm, t, X, K1, h, variant, rtol, atol)
        n_rhs += s - 1
        if not (np.isfinite(err) and np.all(np.isfinite(Xn))):
            status = ERR_NONFINITE
            n_rej += 1
            break
        if err <= rtol:
            t_new = t1 if last else t + h
            while next_out < len(t_out) and t_out[next_out] <= t_new:
                y_out[next_out] = hermite((t_out[next_out] - t) / h, h, X, Xn, K1, Ks)
                next_out += 1
            fac = GROW_MAX if err == 0.0 else min(GROW_MAX, SAFETY * (rtol / err) ** expo)
            if rejected_this_step:
                fac = min(1.0, fac)
            t, X, K1 = t_new, Xn, Ks
            n_acc += 1
            rejected_this_step = False
            h = h * fac
        else:
            n_rej += 1
            if not rejected_this_step:
                h = h * max(SHRINK_FIRST_MIN, SAFETY * (rtol / err) ** expo)
            else:
                h = h * SHRINK_REPEAT
            rejected_this_step = True
    return Result(X.astype(np.float64), t, y_out, n_acc, n_rej, n_rhs, status, h)


def fixed_step(pair: Pair, sysm, t0, y0, h, n_steps, variant="double"):
    """n_steps steps of constant size h without error control: X^{n}."""
    st = np.float32 if variant == "single" else np.float64
    X = np.asarray(y0, dtype=np.float64).astype(st)
    K1 = models.rhs(sysm, t0, X, stage_precision(variant, pair.stages, pair.stages))
    t = t0
    for _ in range(n_steps):
        X, K1, _, _ = attempt(pair, sysm, t, X, K1, h, variant, 1.0, 1.0)
        t += h
    return X
