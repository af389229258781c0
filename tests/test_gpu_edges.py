"""Edge cases of the GPU path: a single agent, an uncoupled system (closed
form), many dense outputs inside one step, ragged batches of tiny systems,
and argument validation (host-side, nothing reaches the GPU)."""

import ctypes

import numpy as np
import pytest

import workloads as W
from oracle import bs3 as obs3
from oracle import exact, metrics, models
from tests.gpu_helpers import library, torch_cuda

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("kind", ["lco_cfg", "lco_paper", "kuramoto", "circadian"])
@pytest.mark.parametrize("variant,store", [("double", "f64"), ("mixed1", "f32"), ("single", "f32")])
def test_single_agent(kind, variant, store):
    bs3 = library()
    torch_cuda()
    make = {"lco_cfg": lambda: W.lco_config(1, 3, t1=5.0), "lco_paper": lambda: W.lco_paper(1, 3),
            "kuramoto": lambda: W.kuramoto(1, 3, t1=5.0), "circadian": lambda: W.circadian(1, 3, t1=24.0)}
    w = make[kind]()
    sysm = bs3.System.from_workload(w, store)
    rc, st, y, _ = sysm.solve(w.t0, w.t1, w.y0, w.rtol, w.atol, variant, "float2")
    sysm.close()
    ref = obs3.solve(models.from_workload(w, store), w.t0, w.t1, w.y0, w.rtol, w.atol, variant)
    assert rc == bs3.OK and ref.status == obs3.OK
    assert st.t_reached == w.t1
    n_gpu, n_ref = st.n_accepted + st.n_rejected, ref.n_accepted + ref.n_rejected
    assert abs(n_gpu - n_ref) <= max(2, 0.05 * n_ref), (n_gpu, n_ref)
    tol = 1e-4 if variant == "single" else 1e-7
    np.testing.assert_allclose(y, ref.y, rtol=tol, atol=tol)


@pytest.mark.parametrize("variant,store", [("double", "f64"), ("mixed2", "f32"), ("mixed2", "bf16")])
def test_uncoupled_kuramoto_is_exact(variant, store):
    """K = 0: theta(t) = theta0 + omega t.  Every stage sees the constant
    omega (F in binary64 in these variants; Mixed1 and Single round omega to
    binary32 in F), so the method is exact up to rounding, E = 0 and h grows
    to hmax."""
    bs3 = library()
    torch_cuda()
    w = W.kuramoto(333, 11, t1=20.0, k=0.0)
    sysm = bs3.System.from_workload(w, store)
    rc, st, y, _ = sysm.solve(w.t0, w.t1, w.y0, 1e-8, 1e-8, variant, "float2")
    sysm.close()
    assert rc == bs3.OK
    ex = exact.kuramoto_uncoupled(w.y0, w.params, w.t1)
    assert np.max(np.abs(y - ex)) <= 1e-12 * (1.0 + np.max(np.abs(ex)))
    # the step grows to hmax = (t1 - t0) / 10 after the starting step
    assert st.n_rejected == 0 and st.n_accepted <= 20


def test_many_dense_outputs_inside_one_step():
    """500 output times over 10 steps of the uncoupled system (50 per step,
    more than the solver batches at once); the cubic Hermite interpolant of
    a linear solution is the solution itself."""
    bs3 = library()
    torch_cuda()
    w = W.kuramoto(64, 12, t1=10.0, k=0.0)
    ts = np.linspace(0.0, w.t1, 500)
    sysm = bs3.System.from_workload(w, "f64")
    rc, st, y, y_out = sysm.solve(w.t0, w.t1, w.y0, 1e-9, 1e-9, "double", "float2", t_out=ts)
    sysm.close()
    assert rc == bs3.OK and st.n_out_written == len(ts)
    ex = np.stack([exact.kuramoto_uncoupled(w.y0, w.params, t) for t in ts])
    assert np.max(np.abs(y_out - ex)) <= 1e-11 * (1.0 + np.max(np.abs(ex)))
    np.testing.assert_array_equal(y_out[-1], y)


def test_ragged_batch_of_tiny_systems():
    """Systems of 1, 2 and 3 agents next to larger ones in one launch."""
    bs3 = library()
    torch_cuda()
    systems = [W.lco_config(n, 40 + n, t1=3.0) for n in (1, 2, 3, 200, 1, 17)]
    Ns = [w.N for w in systems]
    K = np.concatenate([np.asarray(w.coupling, dtype=np.float32).ravel() for w in systems])
    rc, yf, stats, _ = bs3.bs3_batch_solve(bs3.LCO_CFG, Ns, np.concatenate([w.params for w in systems]), K,
                                           bs3.F64, np.concatenate([w.y0 for w in systems]),
                                           np.zeros(len(systems)), np.full(len(systems), 3.0), 1e-6, 1e-6,
                                           bs3.DOUBLE, bs3.ACC_FLOAT2)
    assert rc == bs3.OK
    o = 0
    for k, w in enumerate(systems):
        ref = obs3.solve(models.from_workload(w, "f64"), w.t0, w.t1, w.y0, 1e-6, 1e-6, "double")
        assert stats[k].status == 0 and stats[k].t_reached == w.t1
        n_gpu, n_ref = stats[k].n_accepted + stats[k].n_rejected, ref.n_accepted + ref.n_rejected
        assert abs(n_gpu - n_ref) <= max(2, 0.05 * n_ref), (k, w.N, n_gpu, n_ref)
        # step sequences may part at roundoff (a stretched last step, say):
        # compare global errors against the closed form, as for single solves
        ex = exact.lco_cfg_exact(w.params, np.asarray(w.coupling, dtype=np.float64), w.y0[:w.N], w.y0[w.N:], w.t1)
        e_gpu = metrics.normalized_final_error(ex, yf[o:o + 2 * w.N], w.N)
        e_ref = metrics.normalized_final_error(ex, ref.y, w.N)
        assert 0.5 * e_ref <= e_gpu <= 2.0 * e_ref + 1e-12, (k, w.N, e_gpu, e_ref)
        o += 2 * w.N


def test_invalid_arguments_are_rejected():
    bs3 = library()
    torch_cuda()
    lib = bs3.load()
    out = ctypes.c_void_p()
    assert lib.bs3_create_system(bs3.KURAMOTO, 0, None, 0, 0, None, ctypes.byref(out)) == bs3.ERR_INVALID_ARG
    assert lib.bs3_create_system(bs3.KURAMOTO, 4, None, 0, 0, None, ctypes.byref(out)) == bs3.ERR_INVALID_ARG
    assert lib.bs3_create_system(9, 4, None, 0, 0, None, ctypes.byref(out)) == bs3.ERR_INVALID_ARG
    w = W.kuramoto(40, 1, t1=1.0)
    sysm = bs3.System.from_workload(w, "f32")
    h = sysm.handle
    y0 = np.ascontiguousarray(w.y0)
    yo = np.zeros_like(y0)
    for t0, t1, rtol, atol, variant, accum in ((1.0, 1.0, 1e-6, 1e-6, bs3.MIXED1, bs3.ACC_FLOAT2),
                                               (0.0, 1.0, 0.0, 1e-6, bs3.MIXED1, bs3.ACC_FLOAT2),
                                               (0.0, 1.0, 1e-6, -1.0, bs3.MIXED1, bs3.ACC_FLOAT2),
                                               (0.0, 1.0, 1e-6, 1e-6, 7, bs3.ACC_FLOAT2),
                                               (0.0, 1.0, 1e-6, 1e-6, bs3.MIXED1, 5),
                                               (0.0, float("inf"), 1e-6, 1e-6, bs3.MIXED1, bs3.ACC_FLOAT2)):
        rc, st = bs3.bs3_solve(h, t0, t1, y0, rtol, atol, variant, accum, None, 0, None, yo, bs3.HOST_IO)
        assert rc == bs3.ERR_INVALID_ARG and st.status == bs3.ERR_INVALID_ARG
    # output times outside the span, or not ascending
    for ts in (np.array([0.5, 1.5]), np.array([0.5, 0.2])):
        y_out = np.zeros((len(ts), w.N))
        rc, _ = bs3.bs3_solve(h, 0.0, 1.0, y0, 1e-6, 1e-6, bs3.MIXED1, bs3.ACC_FLOAT2, ts, len(ts), y_out, yo,
                              bs3.HOST_IO)
        assert rc == bs3.ERR_INVALID_ARG
    assert bs3.bs3_set_tuning(h, 99, 1) == bs3.ERR_INVALID_ARG
    assert bs3.bs3_set_tuning(h, bs3.TUNE_RESIDENT_WEIGHTS, 2) == bs3.ERR_INVALID_ARG
    assert bs3.bs3_set_coupling(h, np.zeros((40, 40), np.float32), bs3.BF16, bs3.F32, False) == bs3.ERR_INVALID_ARG
    sysm.close()
    # ensembles: T must fill whole 128-column tiles (64 trajectories), N whole 128-row tiles
    torch = torch_cuda()
    for N, T in ((256, 100), (200, 128)):
        K = torch.zeros((N, N), dtype=torch.float32, device="cuda")
        om = torch.zeros((T, N), dtype=torch.float64, device="cuda")
        th = torch.zeros((T, N), dtype=torch.float64, device="cuda")
        rc, *_ = bs3.bs3_ensemble_solve(K, N, T, om, th, 0.0, 1.0, 1e-6, 1e-6, th)
        assert rc == bs3.ERR_INVALID_ARG
