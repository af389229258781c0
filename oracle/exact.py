"""Closed-form solutions used to pin the oracle (binary64).

* second-order oscillators x'' = -(Omega^2 - A) x with symmetric A: through
  the eigendecomposition S = Omega^2 - A = Q diag(lam) Q^T (lam > 0);
* the paper's Benchmark 1 (Eq. LCO), a linear system y' = B y: y = expm(B t) y0
  (the paper notes it has an analytic solution, Sec. 2.1);
* Kuramoto with zero coupling: theta_i(t) = theta_i(0) + omega_i t;
* Kuramoto with two oscillators and symmetric weight k: the phase difference
  phi = theta_2 - theta_1 obeys Adler's equation phi' = dw - 2 k sin(phi),
  and theta_1 + theta_2 = (omega_1 + omega_2) t + const.  phi(t) is found by
  inverting t = int_{phi0}^{phi} dpsi / (dw - 2k sin psi) (quadrature + root
  finding), valid while dw - 2k sin(phi) keeps one sign.
"""

from __future__ import annotations

import numpy as np
import scipy.integrate
import scipy.linalg
import scipy.optimize


def lco_cfg_exact(omega, A, x0, v0, t):
    S = np.diag(np.asarray(omega, dtype=np.float64) ** 2) - np.asarray(A, dtype=np.float64)
    lam, Q = np.linalg.eigh(S)
    if np.min(lam) <= 0:
        raise ValueError("Omega^2 - A must be positive definite")
    w = np.sqrt(lam)
    c = Q.T @ x0
    d = Q.T @ v0
    x = Q @ (np.cos(w * t) * c + np.sin(w * t) / w * d)
    v = Q @ (-w * np.sin(w * t) * c + np.cos(w * t) * d)
    return np.concatenate([x, v])


def lco_paper_exact(M, y0, t):
    M = np.asarray(M, dtype=np.float64)
    N = M.shape[0]
    B = np.zeros((2 * N, 2 * N))
    B[:N, :N] = M - np.diag(M.sum(axis=1))
    B[:N, N:] = np.eye(N)
    B[N:, :N] = -np.eye(N)
    return scipy.linalg.expm(B * t) @ np.asarray(y0, dtype=np.float64)


def kuramoto_uncoupled(theta0, omega, t):
    return np.asarray(theta0, dtype=np.float64) + np.asarray(omega, dtype=np.float64) * t


def adler_pair(theta0, omega, k, t):
    """Two oscillators with K_12 = K_21 = k, requires |dw| > 2|k| (drifting)."""
    dw = omega[1] - omega[0]
    if abs(dw) <= 2 * abs(k):
        raise ValueError("phase-locked case not supported")
    phi0 = theta0[1] - theta0[0]
    rate = lambda p: 1.0 / (dw - 2 * k * np.sin(p))  # noqa: E731
    period = abs(scipy.integrate.quad(rate, 0.0, 2 * np.pi, epsabs=1e-13, epsrel=1e-13, limit=200)[0])
    turns = np.floor(t / period)
    rem = t - turns * period
    direction = np.sign(dw)

    def g(phi):
        return scipy.integrate.quad(rate, phi0, phi, epsabs=1e-13, epsrel=1e-13, limit=200)[0] - rem

    lo, hi = phi0, phi0 + direction * 2 * np.pi
    a, b = (lo, hi) if lo < hi else (hi, lo)
    phi_rem = scipy.optimize.brentq(g, a, b, xtol=1e-15, rtol=1e-15, maxiter=200)
    phi = phi_rem + direction * 2 * np.pi * turns
    s = theta0[0] + theta0[1] + (omega[0] + omega[1]) * t
    return np.array([(s - phi) / 2, (s + phi) / 2])
