"""Dormand-Prince 5(4) on the GPU (bs3_set_method) against the embedded-pair
oracle (oracle/erk.py) on the same seeded inputs."""

import numpy as np
import pytest

import workloads as W
from oracle import bs3 as obs3
from oracle import erk, exact, metrics, models
from tests.gpu_helpers import library, torch_cuda

pytestmark = pytest.mark.gpu

DP5 = erk.PAIRS["dp5"]


def _solve(w, store, variant, rtol, t_out=None):
    bs3 = library()
    torch_cuda()
    sysm = bs3.System.from_workload(w, store)
    sysm.set_method("dp54")
    rc, st, y, y_out = sysm.solve(w.t0, w.t1, w.y0, rtol, rtol, variant, "float2", t_out)
    sysm.close()
    assert rc == bs3.OK, bs3.bs3_status_string(rc)
    assert st.t_reached == w.t1
    ref = erk.solve(DP5, models.from_workload(w, store), w.t0, w.t1, w.y0, rtol, rtol, variant, t_out=t_out)
    assert ref.status == obs3.OK
    n_gpu, n_ref = st.n_accepted + st.n_rejected, ref.n_accepted + ref.n_rejected
    assert abs(n_gpu - n_ref) <= max(2, 0.05 * n_ref), (n_gpu, n_ref)
    assert st.n_rhs_evals == 2 + 6 * n_gpu
    return st, y, y_out, ref


@pytest.mark.parametrize("variant,store", [("double", "f64"), ("mixed2", "f32"), ("mixed1", "f32"),
                                           ("single", "f32")])
def test_dp5_oscillators_against_closed_form(variant, store):
    """Second-order oscillators N = 256 (t in [0, 10], rtol 1e-6): the GPU's
    global error against the closed form is the oracle's within a factor 2."""
    w = W.lco_config(256, 0, t1=10.0)
    st, y, _, ref = _solve(w, store, variant, 1e-6)
    A = np.asarray(w.coupling, dtype=np.float32 if store == "f32" else np.float64).astype(np.float64)
    ex = exact.lco_cfg_exact(w.params, A, w.y0[:w.N], w.y0[w.N:], w.t1)
    e_gpu = metrics.normalized_final_error(ex, y, w.N)
    e_ref = metrics.normalized_final_error(ex, ref.y, w.N)
    assert 0.5 <= e_gpu / e_ref <= 2.0, (e_gpu, e_ref)


@pytest.mark.parametrize("kind,variant,store", [("kuramoto", "mixed2", "f32"), ("kuramoto", "double", "f64"),
                                                ("circadian", "mixed1", "f32"), ("lco_paper", "mixed2", "f32")])
def test_dp5_kinds_match_oracle(kind, variant, store):
    w = {"kuramoto": lambda: W.kuramoto(200, 5, t1=10.0), "circadian": lambda: W.circadian(64, 5, t1=24.0),
         "lco_paper": lambda: W.lco_paper(100, 5, heterogeneous=True)}[kind]()
    _, y, _, ref = _solve(w, store, variant, 1e-7)
    assert metrics.normalized_final_error(ref.y, y, w.N) < 1e-5


def test_dp5_dense_output_and_fewer_evaluations():
    bs3 = library()
    w = W.lco_paper(100, 6, heterogeneous=True, rtol=1e-9)
    ts = np.linspace(0.0, w.t1, 33)
    st, y, y_out, ref = _solve(w, "f64", "double", 1e-9, t_out=ts)
    assert st.n_out_written == len(ts)
    np.testing.assert_array_equal(y_out[0], w.y0)
    np.testing.assert_allclose(y_out, ref.y_out, atol=1e-7)
    # the fifth-order pair needs fewer evaluations than BS3 at this tolerance
    sysm = bs3.System.from_workload(w, "f64")
    rc, st3, _, _ = sysm.solve(w.t0, w.t1, w.y0, 1e-9, 1e-9, "double", "float2")
    sysm.close()
    assert rc == bs3.OK and st.n_rhs_evals < st3.n_rhs_evals


def test_single_attempt_entry_is_bs3_only():
    bs3 = library()
    torch_cuda()
    w = W.kuramoto(64, 1, t1=1.0)
    sysm = bs3.System.from_workload(w, "f32")
    sysm.set_method("dp54")
    x = np.ascontiguousarray(w.y0)
    out = np.zeros_like(x)
    rc, _ = bs3.bs3_attempt(sysm.handle, 0.0, 0.01, x, x, 1e-6, 1e-6, bs3.MIXED1, bs3.ACC_FLOAT2, out, out)
    assert rc == bs3.ERR_INVALID_ARG
    assert bs3.bs3_set_method(sysm.handle, 7) == bs3.ERR_INVALID_ARG
    sysm.close()
