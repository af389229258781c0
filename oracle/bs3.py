"""Adaptive Bogacki-Shampine 3(2) solver with the paper's precision variants.

Follows Sec. 2.2-2.3 step by step:

* stages K_l = f(t + c_l h, X^n + h sum_{m<l} a_lm K_m) with the tableau of
  Table Butcher-O23 (Eq. Stage-ODE23); X^{n+1} = X^n + h sum b_l K_l is kept,
  the embedded X~^{n+1} only measures the error;
* FSAL: K_4 = f(t+h, X^{n+1}) is the next K_1 when the step is accepted, and
  is discarded (K_1 reused) when it is rejected;
* the error of Eq. ERROR-O23: W_k = max(|X^n_k|, |X^{n+1}_k|, Ab/Rel),
  V_k = |X^{n+1}_k - X~^{n+1}_k| / W_k, E = max_k V_k, with
  X^{n+1} - X~^{n+1} = h sum_l (b_l - b~_l) K_l;
* accept when E <= Rel (the paper: "smaller than"; equality has measure zero);
* failure conditions of Sec. 2.2: attempts (accepted + failed) limited to
  I_max = 1e5, failed steps to 0.85 I_max, h > h_min = 100 eps_m, and the
  two wall-clock limits;
* Table MP-Distrib: per stage k2, k3, k4 the precision of (F, Sigma, G);
  stage linear combinations and the state in binary64 for Mixed1/Mixed2/
  Double.

Readings where the paper is silent (parity unpinned: the paper prints no
controller and no step sequence; the solver is pinned only through its stage
arithmetic, its error norm and its global accuracy):

* controller (standard 3(2) controller with exponent 1/3, safety 0.8):
  accepted: h <- h min(5, 0.8 (Rel/E)^(1/3)), growth capped at 1 when this
  step had a rejected attempt; first rejection: h <- h max(0.5, 0.8 (Rel/E)^(1/3));
  further rejections of the same step: h <- h/2; h <= h_max = |t1 - t0|/10;
  when t + 1.1 h >= t1 the step is stretched to end exactly at t1;
* initial step: Hairer-Norsett-Wanner II.4 starting-step algorithm with
  exponent 1/3, in the norm of the acceptance test (max_k |v_k| / (Rel W_k),
  W_k = max(|y0_k|, Ab/Rel)); its extra evaluation is counted;
* the first K_1 and the starting-step evaluation use the k4 row of the table;
* Single keeps the state, the stages and their combinations in binary32,
  with t, h, E and the controller in binary64; eps_m of h_min is the epsilon
  of the state format;
* dense output at requested times: cubic Hermite on (t_n, X^n, K_1) and
  (t_{n+1}, X^{n+1}, K_4).
"""

from __future__ import annotations

import dataclasses
import time
from typing import Callable, List, Optional, Sequence

import numpy as np

from . import models
from .tableau import BS3_A, BS3_B, BS3_C, BS3_E, as_float

# status codes of a solve
OK = 0
ERR_INVALID_ARG = 1
ERR_CUDA = 2
ERR_MAX_STEPS = 3
ERR_MAX_REJECTS = 4
ERR_STEP_TOO_SMALL = 5
ERR_TIMEOUT = 6
ERR_DEVICE_WAIT = 7
ERR_NONFINITE = 8

STATUS_NAMES = {
    OK: "OK", ERR_INVALID_ARG: "ERR_INVALID_ARG", ERR_CUDA: "ERR_CUDA",
    ERR_MAX_STEPS: "ERR_MAX_STEPS", ERR_MAX_REJECTS: "ERR_MAX_REJECTS",
    ERR_STEP_TOO_SMALL: "ERR_STEP_TOO_SMALL", ERR_TIMEOUT: "ERR_TIMEOUT",
    ERR_DEVICE_WAIT: "ERR_DEVICE_WAIT", ERR_NONFINITE: "ERR_NONFINITE",
}

# Table MP-Distrib: (F, Sigma, G) for stages k2, k3, k4.
VARIANTS = {
    "single": {2: ("S", "S", "S"), 3: ("S", "S", "S"), 4: ("S", "S", "S")},
    "mixed1": {2: ("S", "S", "S"), 3: ("S", "S", "S"), 4: ("D", "D", "S")},
    "mixed2": {2: ("D", "D", "S"), 3: ("D", "D", "S"), 4: ("D", "D", "S")},
    "double": {2: ("D", "D", "D"), 3: ("D", "D", "D"), 4: ("D", "D", "D")},
    # ensembles sharing K on the tensor cores (models.rhs_tensor), state in binary64
    "tensor": {2: "T", 3: "T", 4: "T"},
}

PAPER_VARIANTS = ("single", "mixed1", "mixed2", "double")

C = as_float(BS3_C)
A = as_float(BS3_A)
B = as_float(BS3_B)
E = as_float(BS3_E)

SAFETY = 0.8
GROW_MAX = 5.0
SHRINK_FIRST_MIN = 0.5
SHRINK_REPEAT = 0.5
STRETCH = 1.1
HMAX_FRACTION = 0.1


@dataclasses.dataclass
class Limits:
    max_attempts: int = 100_000          # I_max
    max_rejects: int = 85_000            # 0.85 I_max
    hmin_factor: float = 100.0           # h_min = 100 eps_m
    wall_limit_s: float = 1.5 * 3600.0
    slow_limit_s: float = 45 * 60.0
    slow_fraction: float = 0.10


@dataclasses.dataclass
class Result:
    y: np.ndarray                 # state at t_reached (float64 copy)
    t_reached: float
    y_out: np.ndarray             # [n_out, d*N]
    n_accepted: int
    n_rejected: int
    n_rhs: int
    status: int
    h_last: float
    history: Optional[List[tuple]] = None   # (t, h, E, accepted) per attempt


def hermite(theta, h, y0, y1, f0, f1):
    """Cubic Hermite on [t_n, t_n + h] at fraction theta (binary64)."""
    y0 = y0.astype(np.float64); y1 = y1.astype(np.float64)
    f0 = f0.astype(np.float64); f1 = f1.astype(np.float64)
    return (1 - theta) * y0 + theta * y1 + theta * (theta - 1) * (
        (1 - 2 * theta) * (y1 - y0) + (theta - 1) * h * f0 + theta * h * f1)


def error_norm(X, Xn, Dv, rtol, atol):
    """Eq. ERROR-O23 with Dv = X^{n+1} - X~^{n+1}; computed in binary64."""
    W = np.maximum(np.maximum(np.abs(X.astype(np.float64)), np.abs(Xn.astype(np.float64))),
                   atol / rtol)
    return float(np.max(np.abs(Dv.astype(np.float64)) / W)) if X.size else 0.0


def _rhs(sysm, t, y, prec):
    return models.rhs_tensor(sysm, t, y) if prec == "T" else models.rhs(sysm, t, y, prec)


def attempt(sysm, t, X, K1, h, variant, rtol, atol):
    """One BS3 attempt: returns (Xn, K4, E, (K2, K3)).  State dtype decides the
    precision of the stage combinations (binary32 for Single)."""
    prec = VARIANTS[variant]
    st = X.dtype.type
    hs = st(h)
    # the scalar a_lm h is formed in the state precision
    Y2 = X + (st(A[1][0]) * hs) * K1
    K2 = _rhs(sysm, t + C[1] * h, Y2, prec[2])
    Y3 = X + (st(A[2][1]) * hs) * K2
    K3 = _rhs(sysm, t + C[2] * h, Y3, prec[3])
    Xn = X + hs * (st(B[0]) * K1 + st(B[1]) * K2 + st(B[2]) * K3)
    K4 = _rhs(sysm, t + h, Xn, prec[4])
    Dv = hs * (st(E[0]) * K1 + st(E[1]) * K2 + st(E[2]) * K3 + st(E[3]) * K4)
    return Xn, K4, error_norm(X, Xn, Dv, rtol, atol), (K2, K3)


def initial_step(sysm, t0, y0, f0, rtol, atol, hmax, prec):
    """Starting step (reading stated in the module docstring); returns (h, f1)."""
    sc = rtol * np.maximum(np.abs(y0.astype(np.float64)), atol / rtol)
    d0 = float(np.max(np.abs(y0.astype(np.float64)) / sc))
    d1 = float(np.max(np.abs(f0.astype(np.float64)) / sc))
    h0 = 0.01 * d0 / d1 if (d0 >= 1e-5 and d1 >= 1e-5) else 1e-6
    st = y0.dtype.type
    y1 = y0 + st(h0) * f0
    f1 = _rhs(sysm, t0 + h0, y1, prec)
    d2 = float(np.max(np.abs(f1.astype(np.float64) - f0.astype(np.float64)) / sc)) / h0
    m = max(d1, d2)
    h1 = (0.01 / m) ** (1.0 / 3.0) if m > 1e-15 else max(1e-6, h0 * 1e-3)
    return min(100.0 * h0, h1, hmax)


def solve(sysm: models.System, t0: float, t1: float, y0: np.ndarray, rtol: float, atol: float,
          variant: str = "double", t_out: Optional[Sequence[float]] = None,
          limits: Optional[Limits] = None, proposer: Optional[Callable] = None,
          record_history: bool = False, h_init: Optional[float] = None) -> Result:
    """Integrate from t0 to t1 > t0.  ``proposer(hist, h, rtol) -> h_new`` may
    replace the controller's proposal after an accepted attempt (the error test
    is unchanged, and a rejected proposal falls back to the controller)."""
    if variant not in VARIANTS:
        raise ValueError(variant)
    lim = limits or Limits()
    prec = VARIANTS[variant]
    state_t = np.float32 if variant == "single" else np.float64
    eps_m = float(np.finfo(state_t).eps)
    hmin = lim.hmin_factor * eps_m
    hmax = HMAX_FRACTION * abs(t1 - t0)
    t_out = np.asarray([] if t_out is None else t_out, dtype=np.float64)
    dN = sysm.d * sysm.N
    y_out = np.full((len(t_out), dN), np.nan)
    next_out = 0
    while next_out < len(t_out) and t_out[next_out] <= t0:
        y_out[next_out] = y0
        next_out += 1

    X = np.asarray(y0, dtype=np.float64).astype(state_t)
    if not np.all(np.isfinite(X)):
        return Result(X.astype(np.float64), t0, y_out, 0, 0, 0, ERR_NONFINITE, 0.0)
    K1 = _rhs(sysm, t0, X, prec[4])
    n_rhs = 1
    if h_init is None:
        h = initial_step(sysm, t0, X, K1, rtol, atol, hmax, prec[4])
        n_rhs += 1
    else:
        h = float(h_init)
    t = float(t0)
    n_acc = n_rej = 0
    status = OK
    hist = [] if (record_history or proposer is not None) else None
    err_hist: List[float] = []
    rejected_this_step = False
    started = time.monotonic()
    if not np.all(np.isfinite(K1)):
        status = ERR_NONFINITE

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
        Xn, K4, err, _ = attempt(sysm, t, X, K1, h, variant, rtol, atol)
        n_rhs += 3
        if not (np.isfinite(err) and np.all(np.isfinite(Xn))):
            status = ERR_NONFINITE
            n_rej += 1
            break
        accepted = err <= rtol
        if hist is not None:
            hist.append((t, h, err, accepted))
        if accepted:
            t_new = t1 if last else t + h
            while next_out < len(t_out) and t_out[next_out] <= t_new:
                theta = (t_out[next_out] - t) / h
                y_out[next_out] = hermite(theta, h, X, Xn, K1, K4)
                next_out += 1
            fac = GROW_MAX if err == 0.0 else min(GROW_MAX, SAFETY * (rtol / err) ** (1.0 / 3.0))
            if rejected_this_step:
                fac = min(1.0, fac)
            h_new = h * fac
            err_hist.append(err)
            if proposer is not None and not rejected_this_step:
                h_new = proposer(err_hist, h, rtol, h_new)
            t, X, K1 = t_new, Xn, K4
            n_acc += 1
            rejected_this_step = False
            h = h_new
        else:
            n_rej += 1
            if not rejected_this_step:
                h = h * max(SHRINK_FIRST_MIN, SAFETY * (rtol / err) ** (1.0 / 3.0))
            else:
                h = h * SHRINK_REPEAT
            rejected_this_step = True
    return Result(X.astype(np.float64), t, y_out, n_acc, n_rej, n_rhs, status, h,
                  hist if record_history else None)


def fixed_step(sysm, t0, y0, h, n_steps, variant="double"):
    """n_steps BS3 steps of constant size h (no error control): returns
    (X^{n}, X~^{n} of the last step).  Used for the observed-order pins."""
    st = np.float32 if variant == "single" else np.float64
    X = np.asarray(y0, dtype=np.float64).astype(st)
    K1 = models.rhs(sysm, t0, X, VARIANTS[variant][4])
    t = t0
    Xt = X
    for _ in range(n_steps):
        Xn, K4, _, (K2, K3) = attempt(sysm, t, X, K1, h, variant, 1.0, 1.0)
        Dv = h * (E[0] * K1 + E[1] * K2 + E[2] * K3 + E[3] * K4)
        Xt = Xn - Dv
        X, K1, t = Xn, K4, t + h
    return X, Xt
