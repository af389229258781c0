"""Pins of the oracle's BS3 solver against closed forms, a library routine and
the paper's printed statistics."""

import math
import os

import numpy as np
import pytest
import scipy.integrate._ivp.rk as scipy_rk

import workloads as W
from oracle import bs3, dopri5, exact, metrics, models

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _lco(N=32, seed=1, t1=10.0):
    w = W.lco_config(N, seed, t1=t1)
    return w, models.from_workload(w)


def test_observed_order_three_and_embedded_order_two():
    w, S = _lco(16)
    T = 2.0
    ex = exact.lco_cfg_exact(w.params, w.coupling, w.y0[:16], w.y0[16:], T)
    errs, errs_t = [], []
    for n in (20, 40, 80, 160):
        X, Xt = bs3.fixed_step(S, 0.0, w.y0, T / n, n)
        errs.append(np.max(np.abs(X - ex)))
        # one embedded step from the exact state: local error O(h^3)
        h = T / n
        y_mid = exact.lco_cfg_exact(w.params, w.coupling, w.y0[:16], w.y0[16:], T - h)
        _, Xt1 = bs3.fixed_step(S, T - h, y_mid, h, 1)
        errs_t.append(np.max(np.abs(Xt1 - ex)))
    p = [math.log2(errs[i] / errs[i + 1]) for i in range(3)]
    q = [math.log2(errs_t[i] / errs_t[i + 1]) for i in range(3)]
    assert all(abs(x - 3.0) < 0.1 for x in p), p
    assert all(abs(x - 3.0) < 0.15 for x in q), q   # local error of the 2nd-order pair ~ h^3


def test_one_step_matches_scipy_rk23():
    """scipy's RK23 is the same Bogacki-Shampine pair: the stage arithmetic and
    the embedded difference of one step must agree to rounding."""
    w, S = _lco(24)
    f = lambda t, y: models.rhs(S, t, y)  # noqa: E731
    y0 = w.y0
    f0 = f(0.0, y0)
    h = 0.137
    K = np.empty((4, y0.size))
    y_new, f_new = scipy_rk.rk_step(f, 0.0, y0, f0, h, scipy_rk.RK23.A, scipy_rk.RK23.B,
                                    scipy_rk.RK23.C, K)
    err_scipy = h * (K.T @ scipy_rk.RK23.E)        # scipy: y_new - y_embedded with E = b~ - b sign
    Xn, K4, _, (K2, K3) = bs3.attempt(S, 0.0, y0, f0, h, "double", 1.0, 1.0)
    Dv = h * (bs3.E[0] * f0 + bs3.E[1] * K2 + bs3.E[2] * K3 + bs3.E[3] * K4)
    np.testing.assert_allclose(Xn, y_new, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(K4, f_new, rtol=1e-14, atol=1e-14)
    np.testing.assert_allclose(np.abs(Dv), np.abs(err_scipy), rtol=1e-9, atol=1e-16)


@pytest.mark.parametrize("rtol", [1e-4, 1e-6, 1e-8])
def test_lco_cfg_global_error_tracks_tolerance(rtol):
    w, S = _lco(48)
    r = bs3.solve(S, 0.0, w.t1, w.y0, rtol, rtol, "double")
    ex = exact.lco_cfg_exact(w.params, w.coupling, w.y0[:48], w.y0[48:], w.t1)
    err = metrics.normalized_final_error(ex, r.y, 48)
    assert r.status == bs3.OK and r.t_reached == w.t1
    assert rtol * 0.3 < err < rtol * 30


def test_lco_paper_form_against_expm():
    w = W.lco_paper(40, 2, t1=10 * math.pi, heterogeneous=True)
    S = models.from_workload(w)
    r = bs3.solve(S, 0.0, w.t1, w.y0, 1e-8, 1e-8, "double")
    ex = exact.lco_paper_exact(w.coupling, w.y0, w.t1)
    assert metrics.normalized_final_error(ex, r.y, 40) < 3e-6


def test_kuramoto_uncoupled_is_exact():
    w = W.kuramoto(64, 3, k=0.0, t1=50.0)
    S = models.from_workload(w)
    r = bs3.solve(S, 0.0, w.t1, w.y0, 1e-9, 1e-9, "double", record_history=True)
    np.testing.assert_allclose(r.y, exact.kuramoto_uncoupled(w.y0, w.params, w.t1), rtol=0, atol=1e-12)
    # zero error estimate: every step accepted, h grows x5 up to h_max = 5
    hs = [h for (_, h, _, _) in r.history]
    assert r.n_rejected == 0 and max(hs) == pytest.approx(5.0)
    assert all(e <= 1e-12 for (_, _, e, _) in r.history)


def test_adler_pair_against_quadrature():
    theta0 = np.array([0.3, 1.1])
    omega = np.array([-0.4, 0.9])
    k = 0.25
    K = np.array([[0.0, k], [k, 0.0]])
    S = models.make_system("kuramoto", 2, omega, K, "f64")
    r = bs3.solve(S, 0.0, 20.0, theta0, 1e-9, 1e-9, "double")
    ex = exact.adler_pair(theta0, omega, k, 20.0)
    np.testing.assert_allclose(r.y, ex, atol=2e-7)


def test_kuramoto_symmetric_invariant_through_solve():
    N = 50
    rng = np.random.default_rng(7)
    K = rng.uniform(0, 4 / N, (N, N)); K = (K + K.T) / 2
    omega = rng.standard_normal(N); th0 = rng.uniform(0, 2 * np.pi, N)
    S = models.make_system("kuramoto", N, omega, K, "f64")
    r = bs3.solve(S, 0.0, 30.0, th0, 1e-7, 1e-7, "double")
    assert abs((r.y.sum() - 30.0 * omega.sum()) - th0.sum()) < 1e-9


def test_lco_energy_drift_bounded():
    w, S = _lco(40)
    Smat = np.diag(w.params ** 2) - w.coupling

    def energy(y):
        x, v = y[:40], y[40:]
        return 0.5 * v @ v + 0.5 * x @ Smat @ x

    r = bs3.solve(S, 0.0, w.t1, w.y0, 1e-8, 1e-8, "double")
    assert abs(energy(r.y) - energy(w.y0)) / energy(w.y0) < 1e-6


def test_circadian_synchronous_population_equals_single_cell():
    N = 12
    w = W.circadian(N, 1, t1=48.0)
    w.params[:] = w.params[0]
    y0 = np.repeat(w.y0.reshape(4, N)[:, :1], N, axis=1).reshape(-1)
    S = models.from_workload(w)
    one = models.make_system("circadian", 1, w.params[:1], np.zeros((1, 1)), "f64", w.globals)
    r = bs3.solve(S, 0.0, 48.0, y0, 1e-7, 1e-7, "double")
    r1 = bs3.solve(one, 0.0, 48.0, y0.reshape(4, N)[:, 0].copy(), 1e-7, 1e-7, "double")
    assert (r.n_accepted, r.n_rejected) == (r1.n_accepted, r1.n_rejected)
    np.testing.assert_allclose(r.y.reshape(4, N), np.repeat(r1.y.reshape(4, 1), N, axis=1), rtol=1e-12)


def test_accepted_attempts_satisfy_tolerance_and_rejections_happen():
    w = W.circadian(32, 2, t1=72.0)
    S = models.from_workload(w)
    r = bs3.solve(S, 0.0, w.t1, w.y0, 1e-5, 1e-5, "double", record_history=True)
    assert r.status == bs3.OK
    assert all(e <= 1e-5 for (_, _, e, a) in r.history if a)
    assert all(e > 1e-5 for (_, _, e, a) in r.history if not a)
    assert r.n_rhs == 2 + 3 * (r.n_accepted + r.n_rejected)


def test_dense_output_hits_closed_form_and_endpoint():
    w, S = _lco(20)
    ts = np.linspace(0.0, w.t1, 11)
    r = bs3.solve(S, 0.0, w.t1, w.y0, 1e-8, 1e-8, "double", t_out=ts)
    for i, t in enumerate(ts):
        ex = exact.lco_cfg_exact(w.params, w.coupling, w.y0[:20], w.y0[20:], t)
        assert np.max(np.abs(r.y_out[i] - ex)) < 2e-6
    np.testing.assert_array_equal(r.y_out[0], w.y0)
    np.testing.assert_array_equal(r.y_out[-1], r.y)


def test_failure_conditions():
    w, S = _lco(16)
    r = bs3.solve(S, 0.0, w.t1, w.y0, 1e-6, 1e-6, "double", limits=bs3.Limits(max_attempts=10))
    assert r.status == bs3.ERR_MAX_STEPS and r.n_accepted + r.n_rejected == 10
    r = bs3.solve(S, 0.0, w.t1, w.y0, 1e-30, 1e-30, "double",
                  limits=bs3.Limits(max_rejects=5))
    assert r.status in (bs3.ERR_MAX_REJECTS, bs3.ERR_STEP_TOO_SMALL)
    r = bs3.solve(S, 0.0, w.t1, w.y0, 1e-30, 1e-30, "double")
    assert r.status == bs3.ERR_STEP_TOO_SMALL
    y = w.y0.copy(); y[3] = np.nan
    r = bs3.solve(S, 0.0, w.t1, y, 1e-6, 1e-6, "double")
    assert r.status == bs3.ERR_NONFINITE


def test_precision_plateaus_follow_the_paper():
    """Sec. 3.2: at tight tolerance Single plateaus, Mixed1 is limited on
    Benchmark 1 below 1e-7, Mixed2 stays close to Double."""
    w, S = _lco(64)
    ex = exact.lco_cfg_exact(w.params, w.coupling, w.y0[:64], w.y0[64:], w.t1)
    err = {v: metrics.normalized_final_error(ex, bs3.solve(S, 0.0, w.t1, w.y0, 1e-9, 1e-9, v).y, 64)
           for v in bs3.PAPER_VARIANTS}
    assert err["double"] < 2e-8
    assert err["mixed2"] < 10 * err["double"] + 5e-8
    assert err["mixed1"] > 3 * err["mixed2"]
    assert err["single"] > 3 * err["mixed1"]


def test_beta_within_papers_printed_range():
    rows = {}
    with open(os.path.join(GOLDEN, "beta_lco_paper.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                v, *vals = line.split()
                rows[v] = [float(x) for x in vals]
    w = W.lco_paper(100, 4, heterogeneous=False)
    S = models.from_workload(w)
    rd = bs3.solve(S, 0.0, w.t1, w.y0, 1e-6, 1e-6, "double")
    for v, (lo, _, _, _, hi) in rows.items():
        r = bs3.solve(S, 0.0, w.t1, w.y0, 1e-6, 1e-6, v)
        b = metrics.beta(rd.n_accepted + rd.n_rejected, r.n_accepted + r.n_rejected)
        assert lo <= b <= hi, (v, b)


def test_dopri5_reference_against_closed_forms_and_scipy():
    w, S = _lco(24)
    ex = exact.lco_cfg_exact(w.params, w.coupling, w.y0[:24], w.y0[24:], w.t1)
    y = dopri5.reference_solution(S, 0.0, w.t1, w.y0)
    assert np.max(np.abs(y - ex)) < 1e-10
    wk = W.kuramoto(40, 5, t1=10.0)
    Sk = models.from_workload(wk)
    yk = dopri5.reference_solution(Sk, 0.0, 10.0, wk.y0)
    sp = scipy.integrate.solve_ivp(lambda t, y: models.rhs(Sk, t, y), (0.0, 10.0), wk.y0,
                                   method="RK45", rtol=1e-12, atol=1e-12)
    assert np.max(np.abs(yk - sp.y[:, -1])) < 1e-9


import scipy.integrate  # noqa: E402
