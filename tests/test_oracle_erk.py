"""Pins of the embedded-pair oracle (oracle/erk.py): with the BS3 pair it is
the pinned BS3 solver; the DP5 pair has order 5 and tracks closed forms."""

import math

import numpy as np
import pytest

import workloads as W
from oracle import bs3 as obs3
from oracle import dopri5, erk, exact, metrics, models


@pytest.mark.parametrize("variant", ["double", "mixed2", "mixed1"])
def test_bs3_pair_takes_the_bs3_solvers_steps(variant):
    w = W.lco_config(24, 3, t1=4.0)
    sysm = models.from_workload(w, "f64" if variant == "double" else "f32")
    a = obs3.solve(sysm, w.t0, w.t1, w.y0, 1e-7, 1e-7, variant)
    b = erk.solve(erk.PAIRS["bs3"], sysm, w.t0, w.t1, w.y0, 1e-7, 1e-7, variant)
    assert (a.n_accepted, a.n_rejected, a.n_rhs) == (b.n_accepted, b.n_rejected, b.n_rhs)
    np.testing.assert_allclose(b.y, a.y, rtol=1e-11, atol=1e-12)


def test_dp5_pair_is_consistent():
    p = erk.PAIRS["dp5"]
    assert p.stages == 7 and p.q == 4
    for l in range(1, 7):
        assert math.isclose(sum(p.a[l]), p.c[l], rel_tol=0, abs_tol=1e-15)
    assert abs(sum(p.e)) < 1e-15
    assert p.a[6] == tuple(float(x) for x in (35 / 384, 0, 500 / 1113, 125 / 192, -2187 / 6784, 11 / 84))


def test_dp5_observed_order_five():
    w = W.lco_config(8, 1, t1=1.0)
    sysm = models.from_workload(w, "f64")
    ex = exact.lco_cfg_exact(w.params, np.asarray(w.coupling, np.float64), w.y0[:8], w.y0[8:], 1.0)
    errs = []
    for n in (10, 20, 40):
        y = erk.fixed_step(erk.PAIRS["dp5"], sysm, 0.0, w.y0, 1.0 / n, n)
        errs.append(np.max(np.abs(y - ex)))
    orders = [math.log2(errs[i] / errs[i + 1]) for i in range(2)]
    assert all(abs(o - 5.0) < 0.3 for o in orders), orders


@pytest.mark.parametrize("rtol", [1e-5, 1e-8])
def test_dp5_tracks_closed_form(rtol):
    w = W.lco_config(32, 2, t1=10.0)
    sysm = models.from_workload(w, "f64")
    ex = exact.lco_cfg_exact(w.params, np.asarray(w.coupling, np.float64), w.y0[:32], w.y0[32:], w.t1)
    r = erk.solve(erk.PAIRS["dp5"], sysm, w.t0, w.t1, w.y0, rtol, rtol, "double")
    assert r.status == obs3.OK and r.t_reached == w.t1
    e = metrics.normalized_final_error(ex, r.y, w.N)
    assert e < 20 * rtol, e
    # fewer evaluations than BS3 at a tight tolerance (higher order)
    if rtol <= 1e-8:
        b = obs3.solve(sysm, w.t0, w.t1, w.y0, rtol, rtol, "double")
        assert r.n_rhs < b.n_rhs
    # and the reference integrator (its own controller and norm) lands on the same solution
    f = lambda t, y: models.rhs(sysm, t, y, ("D", "D", "D"))  # noqa: E731
    yr, _, _ = dopri5.integrate(f, w.t0, w.t1, w.y0, rtol=rtol * 1e-3, atol=rtol * 1e-3)
    assert metrics.normalized_final_error(yr, r.y, w.N) < 20 * rtol


def test_dp5_precision_plateaus():
    """Single stalls near binary32 resolution, Mixed2 follows Double."""
    w = W.lco_config(32, 4, t1=5.0)
    ex = exact.lco_cfg_exact(w.params, np.asarray(w.coupling, np.float32).astype(np.float64), w.y0[:32],
                             w.y0[32:], w.t1)
    errs = {}
    for v in ("single", "mixed2", "double"):
        sysm = models.from_workload(w, "f64" if v == "double" else "f32")
        r = erk.solve(erk.PAIRS["dp5"], sysm, w.t0, w.t1, w.y0, 1e-10, 1e-10, v)
        errs[v] = metrics.normalized_final_error(ex, r.y, w.N)
    assert errs["single"] > 1e-7
    assert errs["mixed2"] < 1e-8
