"""Brute-force pins of the right-hand sides (pairwise definitions, long double)."""

import numpy as np
import pytest

import workloads as W
from oracle import models


def _small(kind, N=24, seed=0):
    if kind == "lco_cfg":
        return W.lco_config(N, seed)
    if kind == "lco_paper":
        return W.lco_paper(N, seed, heterogeneous=True)
    if kind == "kuramoto":
        w = W.kuramoto(N, seed)
        w.y0 = w.y0 + 40.0 * np.random.default_rng(seed).standard_normal(N)   # large phases
        return w
    return W.circadian(N, seed)


@pytest.mark.parametrize("kind", models.KINDS)
def test_gemv_form_equals_pairwise_definition(kind):
    w = _small(kind)
    S = models.from_workload(w, "f64")
    y = w.y0
    f = models.rhs(S, 0.0, y, ("D", "D", "D")).reshape(S.d, S.N)
    ref = models.agent_term(S, y)
    c = models.COUPLED_COMPONENT[kind]
    ref[c] = ref[c] + models.pairwise_coupling(S, y).astype(np.float64)
    scale = np.max(np.abs(ref)) + 1.0
    np.testing.assert_allclose(f, ref, rtol=0, atol=1e-13 * scale)


@pytest.mark.parametrize("kind", models.KINDS)
@pytest.mark.parametrize("prec", [("S", "S", "S"), ("D", "D", "S")])
def test_low_precision_within_unit_roundoff_bound(kind, prec):
    """S evaluations differ from the exact sum by at most a few binary32 ulps of
    sum_j |w_ij g_ij| (plus the phase-reduction term for Kuramoto)."""
    w = _small(kind, N=40)
    S = models.from_workload(w, "f64")
    y = w.y0
    f = models.rhs(S, 0.0, y, prec).reshape(S.d, S.N)
    ref = models.rhs(S, 0.0, y, ("D", "D", "D")).reshape(S.d, S.N)
    u = 2.0 ** -24
    absK = np.abs(S.s[:, None] * S.q)
    mag = absK.sum(axis=1) + np.abs(models.agent_term(S, y)).max(axis=0) + 1e-30
    if kind == "circadian":
        mag = mag * 6.0
    err = np.max(np.abs(f - ref), axis=0)
    assert np.all(err <= (S.N + 16) * u * mag * 4)


def test_dropped_term_is_detected():
    """A right-hand side with one weight zeroed misses the bound above."""
    w = _small("lco_cfg", N=40)
    S = models.from_workload(w, "f64")
    ref = models.rhs(S, 0.0, w.y0, ("D", "D", "D"))
    S.q = S.q.copy()
    S.q[3, 7] = 0.0
    bad = models.rhs(S, 0.0, w.y0, ("D", "D", "D"))
    assert abs(bad[40 + 3] - ref[40 + 3]) > 1e-6


def test_permutation_coupling_is_exact_gather():
    N = 33
    rng = np.random.default_rng(5)
    perm = rng.permutation(N)
    P = np.zeros((N, N)); P[np.arange(N), perm] = 1.0
    S = models.make_system("lco_cfg", N, np.zeros(N), P, "bf16")
    y = np.concatenate([rng.standard_normal(N), np.zeros(N)])
    f = models.rhs(S, 0.0, y, ("S", "S", "S"))
    np.testing.assert_array_equal(f[N:], y[:N][perm].astype(np.float32).astype(np.float64))


def test_kuramoto_sum_invariant_symmetric():
    """sum_i theta_i' = sum_i omega_i for symmetric weights (pairwise antisymmetry)."""
    N = 64
    rng = np.random.default_rng(6)
    K = rng.uniform(0, 2 / N, (N, N)); K = (K + K.T) / 2
    omega = rng.standard_normal(N)
    S = models.make_system("kuramoto", N, omega, K, "f64")
    f = models.rhs(S, 0.0, rng.uniform(0, 50, N))
    assert abs(f.sum() - omega.sum()) < 1e-12


def test_circadian_synchronous_cells_have_no_coupling():
    N = 16
    w = W.circadian(N, 0)
    w.params[:] = w.params[0]
    y = np.repeat(w.y0.reshape(4, N)[:, :1], N, axis=1).reshape(-1)
    S = models.from_workload(w)
    f = models.rhs(S, 0.0, y).reshape(4, N)
    F = models.agent_term(S, y)
    np.testing.assert_allclose(f, F, rtol=1e-15, atol=0)
