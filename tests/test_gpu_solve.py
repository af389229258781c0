"""GPU parity of whole adaptive solves (controller, FSAL, dense output,
failure conditions) against the oracle on the same seeded inputs."""

import numpy as np
import pytest

import workloads as W
from oracle import bs3 as obs3
from oracle import exact, metrics, models
from tests.gpu_helpers import library, torch_cuda

pytestmark = pytest.mark.gpu


def _compare(w, store, variant, accum="float2", t_out=None, exact_y=None, resident=False):
    bs3 = library()
    torch_cuda()
    sysm = bs3.System.from_workload(w, store, resident=resident)
    rc, st, y, y_out = sysm.solve(w.t0, w.t1, w.y0, w.rtol, w.atol, variant, accum, t_out)
    sysm.close()
    osys = models.from_workload(w, store)
    ref = obs3.solve(osys, w.t0, w.t1, w.y0, w.rtol, w.atol, variant, t_out=t_out)
    assert rc == bs3.OK and ref.status == obs3.OK, bs3.bs3_status_string(rc)
    assert st.t_reached == w.t1
    n_gpu, n_ref = st.n_accepted + st.n_rejected, ref.n_accepted + ref.n_rejected
    assert abs(n_gpu - n_ref) <= max(2, 0.05 * n_ref), (n_gpu, n_ref)
    assert st.n_rhs_evals == 2 + 3 * n_gpu
    diff = metrics.normalized_final_error(ref.y, y, w.N)
    if exact_y is not None:
        e_gpu = metrics.normalized_final_error(exact_y, y, w.N)
        e_ref = metrics.normalized_final_error(exact_y, ref.y, w.N)
        assert 0.5 <= e_gpu / e_ref <= 2.0, (e_gpu, e_ref)
        assert diff <= 0.5 * e_ref + 1e-12, (diff, e_ref)
    return st, y, y_out, ref, diff


@pytest.mark.parametrize("variant", list(obs3.PAPER_VARIANTS))
@pytest.mark.parametrize("accum", ["float2", "f64"])
def test_lco_config_n256_all_variants(variant, accum):
    """Second-order oscillators, N = 256, rtol = atol = 1e-6, t in [0, 10]."""
    w = W.lco_config(256, 0)
    ex = exact.lco_cfg_exact(w.params, w.coupling, w.y0[:256], w.y0[256:], w.t1)
    store = "f64" if variant == "double" else "f32"
    _compare(w, store, variant, accum, exact_y=ex)


@pytest.mark.parametrize("variant,store", [("single", "f32"), ("mixed1", "f32"), ("mixed2", "f32"),
                                           ("double", "f64"), ("mixed1", "bf16"), ("mixed2", "f16"),
                                           ("mixed2", "fp8e4m3")])
@pytest.mark.parametrize("resident", [True, False])
def test_kuramoto_small(variant, store, resident):
    w = W.kuramoto(300, 2, t1=20.0)
    st, y, _, ref, diff = _compare(w, store, variant, resident=resident)
    # both follow the same trajectory to well within the tolerance
    assert diff < 1e-3


@pytest.mark.parametrize("variant,store", [("mixed1", "f32"), ("mixed2", "bf16"), ("double", "f64"),
                                           ("single", "f32")])
def test_circadian_small(variant, store):
    w = W.circadian(64, 2, t1=48.0)
    _, _, _, _, diff = _compare(w, store, variant)
    assert diff < 1e-3


def test_lco_paper_form_and_dense_output():
    w = W.lco_paper(100, 5, heterogeneous=True, rtol=1e-8)
    ts = np.linspace(0.0, w.t1, 17)
    ex = exact.lco_paper_exact(w.coupling, w.y0, w.t1)
    st, y, y_out, ref, _ = _compare(w, "f64", "double", t_out=ts, exact_y=ex)
    assert st.n_out_written == len(ts)
    np.testing.assert_array_equal(y_out[0], w.y0)
    np.testing.assert_allclose(y_out, ref.y_out, atol=1e-7)
    np.testing.assert_allclose(y_out[-1], y, atol=0, rtol=0)


@pytest.mark.parametrize("variant,store", [("mixed1", "bf16"), ("mixed1", "f32"), ("mixed2", "f32")])
def test_full_size_kuramoto_short_span(variant, store):
    """Benchmark workload (N = 4096) in the benchmark's launch configuration
    (resident bf16 weights; streamed f32 weights) over t in [0, 1]."""
    w = W.kuramoto(4096, 0, t1=1.0)
    _, _, _, _, diff = _compare(w, store, variant)
    assert diff < 1e-6


def test_device_and_host_io_agree():
    bs3 = library()
    torch = torch_cuda()
    w = W.kuramoto(200, 7, t1=10.0)
    sysm = bs3.System.from_workload(w, "f32")
    rc, st, y_host, _ = sysm.solve(w.t0, w.t1, w.y0, 1e-7, 1e-7, "mixed2", "float2")
    y0d = torch.tensor(w.y0, device="cuda")
    yfd = torch.empty_like(y0d)
    rc2, st2 = bs3.bs3_solve(sysm.handle, w.t0, w.t1, y0d, 1e-7, 1e-7, bs3.MIXED2, bs3.ACC_FLOAT2, None, 0,
                             None, yfd, 0)
    sysm.close()
    assert rc == rc2 == bs3.OK
    assert (st.n_accepted, st.n_rejected) == (st2.n_accepted, st2.n_rejected)
    np.testing.assert_array_equal(y_host, yfd.cpu().numpy())


def _solve_status(w, store="f64", variant="double", rtol=None, y0=None, **lim):
    bs3 = library()
    torch_cuda()
    limits = bs3.bs3_default_limits()
    for k, v in lim.items():
        setattr(limits, k, v)
    sysm = bs3.System.from_workload(w, store)
    r = rtol if rtol is not None else w.rtol
    rc, st, y, _ = sysm.solve(w.t0, w.t1, w.y0 if y0 is None else y0, r, r, variant, "float2", limits=limits)
    sysm.close()
    return bs3, rc, st


def test_failure_max_steps():
    w = W.lco_config(64, 1)
    bs3, rc, st = _solve_status(w, max_attempts=10)
    assert rc == bs3.ERR_MAX_STEPS and st.n_accepted + st.n_rejected == 10 and st.t_reached < w.t1


def test_failure_step_too_small():
    w = W.lco_config(64, 1)
    bs3, rc, st = _solve_status(w, rtol=1e-30)
    assert rc == bs3.ERR_STEP_TOO_SMALL


def test_failure_nonfinite_state():
    w = W.lco_config(64, 1)
    y0 = w.y0.copy()
    y0[5] = np.nan
    bs3, rc, st = _solve_status(w, y0=y0)
    assert rc == bs3.ERR_NONFINITE


def test_failure_bounded_device_wait():
    """A grid-barrier wait limited to one poll runs out; the launch returns
    BS3_ERR_DEVICE_WAIT and the context stays usable.  With one poll allowed,
    every one of the solve's thousands of barriers of 152 CTAs would have to
    find all arrivals at once; the first that does not ends the solve."""
    w = W.lco_config(4096, 1, dtype=np.float32)
    bs3, rc, st = _solve_status(w, store="bf16", variant="mixed1", spin_limit=1)
    assert rc == bs3.ERR_DEVICE_WAIT
    w2 = W.lco_config(64, 1)
    bs3, rc2, st2 = _solve_status(w2)
    assert rc2 == bs3.OK


def test_failure_wall_clock_watchdog():
    w = W.kuramoto(2048, 1, t1=50.0)
    bs3, rc, st = _solve_status(w, store="f32", variant="mixed1", wall_limit_s=0.0)
    assert rc == bs3.ERR_TIMEOUT and st.t_reached < w.t1
