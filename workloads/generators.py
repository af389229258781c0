"""Seeded synthetic workloads shaped like the paper's three benchmarks.

Every generator draws from ``numpy.random.default_rng(seed)`` and returns a
:class:`Workload`.  Nothing here evaluates the ODE: the right-hand sides, the
scheme and the controller live in the oracle and in the CUDA library, which
share no code with each other.

State vectors are structure-of-arrays: component ``k`` of agent ``i`` sits at
``y[k * N + i]``.  Coupling matrices are dense, row-major ``N x N``.

Distributions (the paper's own parameter tables, Sec. 2.1 and App. A, made
heterogeneous and enlarged as the measured configurations require):

* coupled linear oscillators, second-order form: ``A = (G + G^T)/sqrt(2)/N``,
  ``G_ij ~ N(0,1)``; ``omega_i ~ U(0.5, 1.5)``; ``x0, v0 ~ N(0,1)``.
* coupled linear oscillators, paper form (Eq. LCO): ``M_ij = 1/N`` or a
  heterogeneous ``U(0.5,1.5)/N``; initial state ``2 * U(0,1)`` (App. A.1).
* Kuramoto (Eq. Kuramoto): ``omega_i ~ N(0, sigma^2)``;
  ``K_ij = (k/N)(1 + U(-1/2, 1/2))``; ``theta0 ~ U(0, 2 pi)`` (App. A.2).
* circadian clock (Eq. CC): fixed constants of Sec. 2.1; per-cell
  ``k1_i = 0.339278 (1 + U(-0.1, 0.1))``; weights ``W_ij ~ U(0,1)/N`` times
  the coupling coefficient; initial state
  ``(1, 1, -1.19, -0.62) + 0.2 U(-1/2, 1/2)^4`` (App. A.3).
"""

from __future__ import annotations

import dataclasses
import math
from typing import Dict, List, Optional

import numpy as np

# Fixed constants of the circadian clock / cell cycle model (Sec. 2.1, Eq. CC).
# The Hill exponent is 4; the per-cell k1 is drawn by ``circadian``.
CIRCADIAN_GLOBALS: Dict[str, float] = {
    "k0": 2.0,
    "k2": 0.144832,
    "k3": 2.0,
    "a": 2.0,
    "b": 0.7,
    "c": 0.8,
    "eps": 0.228249,
    "I0": 0.228249,
}
CIRCADIAN_K1_MEAN = 0.339278
CIRCADIAN_K1_STD = 0.090909
CIRCADIAN_Y0_CENTER = (1.0, 1.0, -1.19, -0.62)


@dataclasses.dataclass
class Workload:
    """One seeded problem instance.

    kind      -- "lco_cfg", "lco_paper", "kuramoto" or "circadian"
    N, d      -- number of agents and components per agent
    params    -- per-agent parameters (omega_i or k1_i), float64 [N] (or None)
    globals   -- kind-wide constants (circadian only)
    coupling  -- dense row-major N x N weights, float64 or float32
    y0        -- initial state, float64, structure-of-arrays [d*N]
    t0, t1    -- integration interval
    rtol, atol
    """

    kind: str
    N: int
    d: int
    params: Optional[np.ndarray]
    coupling: np.ndarray
    y0: np.ndarray
    t0: float
    t1: float
    rtol: float
    atol: float
    globals: Optional[Dict[str, float]] = None
    seed: int = 0
    name: str = ""


def _matrix_dtype(N: int, dtype) -> np.dtype:
    if dtype is not None:
        return np.dtype(dtype)
    return np.dtype(np.float64 if N <= 8192 else np.float32)


def _symmetric_normal(rng: np.random.Generator, N: int, dtype) -> np.ndarray:
    """(G + G^T)/sqrt(2) with G_ij ~ N(0,1), built in place in blocks."""
    G = rng.standard_normal((N, N), dtype=np.float64 if dtype == np.float64 else np.float32)
    G = G.astype(dtype, copy=False)
    inv = dtype.type(1.0 / math.sqrt(2.0))
    B = 2048
    for i0 in range(0, N, B):
        i1 = min(N, i0 + B)
        # diagonal block
        blk = G[i0:i1, i0:i1]
        sym = (blk + blk.T) * inv
        G[i0:i1, i0:i1] = sym
        for j0 in range(i1, N, B):
            j1 = min(N, j0 + B)
            up = G[i0:i1, j0:j1]
            lo = G[j0:j1, i0:i1]
            s = (up + lo.T) * inv
            G[i0:i1, j0:j1] = s
            G[j0:j1, i0:i1] = s.T
    return G


def lco_config(N: int = 256, seed: int = 0, t1: float = 10.0, rtol: float = 1e-6,
               atol: Optional[float] = None, dtype=None) -> Workload:
    """Second-order linear oscillators x'' = -omega_i^2 x_i + sum_j A_ij x_j."""
    rng = np.random.default_rng(seed)
    dt = _matrix_dtype(N, dtype)
    A = _symmetric_normal(rng, N, dt)
    A *= dt.type(1.0 / N)
    omega = rng.uniform(0.5, 1.5, N)
    x0 = rng.standard_normal(N)
    v0 = rng.standard_normal(N)
    y0 = np.concatenate([x0, v0]).astype(np.float64)
    return Workload("lco_cfg", N, 2, omega.astype(np.float64), A, y0, 0.0, float(t1),
                    rtol, rtol if atol is None else atol, seed=seed,
                    name=f"lco_cfg_N{N}_seed{seed}")


def lco_paper(N: int = 1000, seed: int = 0, t1: float = 10 * math.pi, rtol: float = 1e-6,
              atol: Optional[float] = None, heterogeneous: bool = False, dtype=None) -> Workload:
    """Paper form of Benchmark 1: x' = v + sum_j M_ij (x_j - x_i), v' = -x."""
    rng = np.random.default_rng(seed)
    dt = _matrix_dtype(N, dtype)
    if heterogeneous:
        M = (rng.uniform(0.5, 1.5, (N, N)) / N).astype(dt)
    else:
        M = np.full((N, N), 1.0 / N, dtype=dt)
    y0 = (2.0 * rng.uniform(0.0, 1.0, 2 * N)).astype(np.float64)
    return Workload("lco_paper", N, 2, None, M, y0, 0.0, float(t1), rtol,
                    rtol if atol is None else atol, seed=seed,
                    name=f"lco_paper_N{N}_seed{seed}")


def kuramoto(N: int = 4096, seed: int = 0, t1: float = 50.0, rtol: float = 1e-6,
             atol: Optional[float] = None, sigma: float = 1.0, k: float = 2.0,
             spread: float = 1.0, dtype=None) -> Workload:
    """theta_i' = omega_i + sum_j K_ij sin(theta_j - theta_i).

    K_ij = (k/N)(1 + spread * U(-1/2, 1/2)); spread=0 gives the paper's
    homogeneous K/N weights, k=0 the uncoupled case.
    """
    rng = np.random.default_rng(seed)
    dt = _matrix_dtype(N, dtype)
    omega = sigma * rng.standard_normal(N)
    K = ((k / N) * (1.0 + spread * rng.uniform(-0.5, 0.5, (N, N)))).astype(dt)
    theta0 = rng.uniform(0.0, 2.0 * math.pi, N)
    return Workload("kuramoto", N, 1, omega.astype(np.float64), K, theta0.astype(np.float64),
                    0.0, float(t1), rtol, rtol if atol is None else atol, seed=seed,
                    name=f"kuramoto_N{N}_seed{seed}")


def circadian(N: int = 16384, seed: int = 0, t1: float = 240.0, rtol: float = 1e-6,
              atol: Optional[float] = None, kc: float = 1.0, k1_mode: str = "jitter",
              dtype=None) -> Workload:
    """Circadian clock / cell-cycle cells with dense weights W_ij = kc U(0,1)/N.

    k1_mode "jitter": k1_i = 0.339278 (1 + U(-0.1,0.1));
    k1_mode "normal": the paper's N(0.339278, 0.090909), clipped to [0.05, 1.9].
    """
    rng = np.random.default_rng(seed)
    dt = _matrix_dtype(N, dtype)
    if k1_mode == "jitter":
        k1 = CIRCADIAN_K1_MEAN * (1.0 + rng.uniform(-0.1, 0.1, N))
    elif k1_mode == "normal":
        k1 = np.clip(rng.normal(CIRCADIAN_K1_MEAN, CIRCADIAN_K1_STD, N), 0.05, 1.9)
    else:
        raise ValueError(k1_mode)
    W = (rng.uniform(0.0, 1.0, (N, N)) * (kc / N)).astype(dt)
    center = np.asarray(CIRCADIAN_Y0_CENTER)
    y0 = center[:, None] + 0.2 * rng.uniform(-0.5, 0.5, (4, N))
    return Workload("circadian", N, 4, k1.astype(np.float64), W, y0.reshape(-1).astype(np.float64),
                    0.0, float(t1), rtol, rtol if atol is None else atol,
                    globals=dict(CIRCADIAN_GLOBALS), seed=seed,
                    name=f"circadian_N{N}_seed{seed}")


def kuramoto_ensemble(T: int = 256, N: int = 8192, seed: int = 0, t1: float = 50.0,
                      rtol: float = 1e-6, dtype=np.float32):
    """T Kuramoto trajectories sharing one K: returns (K, omega[T,N], theta0[T,N])."""
    rng = np.random.default_rng(seed)
    K = ((2.0 / N) * (1.0 + rng.uniform(-0.5, 0.5, (N, N)))).astype(dtype)
    omega = rng.standard_normal((T, N))
    theta0 = rng.uniform(0.0, 2.0 * math.pi, (T, N))
    return K, omega, theta0


def lco_ragged_batch(count: int = 1000, n_min: int = 64, n_max: int = 4096, seed: int = 0,
                     t1: float = 10.0, rtol: float = 1e-6) -> List[Workload]:
    """Independent second-order oscillator systems, N log-uniform in [n_min, n_max]."""
    rng = np.random.default_rng(seed)
    sizes = np.rint(np.exp(rng.uniform(math.log(n_min), math.log(n_max), count))).astype(int)
    seeds = rng.integers(0, 2**31 - 1, count)
    return [lco_config(int(n), int(s), t1=t1, rtol=rtol, dtype=np.float32) for n, s in zip(sizes, seeds)]
