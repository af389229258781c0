"""bs3_solve_noalloc, the entry point for callers that cannot allocate device
memory at solve time, against the allocating bs3_solve on the same inputs.

Collected last on purpose: a failure here leaves every other test already run.
"""

import numpy as np
import pytest

import workloads as W
from oracle import metrics
from tests.gpu_helpers import library, torch_cuda

def _padded(K, dtype):
    N = K.shape[0]
    ld = (N + 15) // 16 * 16
    Kp = np.zeros((N, ld), dtype=dtype)
    Kp[:, :N] = K
    return Kp, ld


@pytest.mark.gpu
@pytest.mark.parametrize("kind,store,variant", [("kuramoto", "f32", "mixed2"), ("lco_paper", "f64", "double"),
                                                ("circadian", "f32", "mixed1")])
def test_noalloc_matches_solve_twice(kind, store, variant):
    bs3 = library()
    torch = torch_cuda()
    if kind == "kuramoto":
        w = W.kuramoto(1000, 12, t1=10.0)
    elif kind == "lco_paper":
        w = W.lco_paper(333, 12, heterogeneous=True, t1=10.0)
    else:
        w = W.circadian(200, 12, t1=24.0)
    ts = np.linspace(w.t0, w.t1, 5)

    # the existing entry point
    sysm = bs3.System.from_workload(w, store)
    rc, st_ref, y_ref, yo_ref = sysm.solve(w.t0, w.t1, w.y0, w.rtol, w.atol, variant, "float2", t_out=ts)
    sysm.close()
    assert rc == bs3.OK

    npdt = np.float64 if store == "f64" else np.float32
    Kp, ld = _padded(w.coupling, npdt)
    dev = lambda a: torch.tensor(a, device="cuda")  # noqa: E731
    wd = dev(Kp)
    par = None if w.params is None else dev(w.params)
    g = None
    if kind == "circadian":
        gl = w.globals
        g = [gl["k0"], gl["k2"], gl["k3"], gl["a"], gl["b"], gl["c"], gl["eps"], gl["I0"]]
    y0 = dev(w.y0)
    tod = dev(ts)
    for call in range(2):                       # the scratch keeps the last call's contents
        yo = torch.full((len(ts), w.y0.size), float("nan"), dtype=torch.float64, device="cuda")
        yf = torch.full_like(y0, float("nan"))
        rc, st = bs3.bs3_solve_noalloc(bs3.KIND_IDS[kind], w.N, par, g, wd, bs3.DTYPE_IDS[store], ld, w.t0, w.t1,
                                       y0, w.rtol, w.atol, bs3.VARIANT_IDS[variant], bs3.ACC_FLOAT2, tod,
                                       len(ts), yo, yf)
        assert rc == bs3.OK, (call, bs3.bs3_status_string(rc))
        n_ref = st_ref.n_accepted + st_ref.n_rejected
        assert abs(st.n_accepted + st.n_rejected - n_ref) <= max(2, 0.05 * n_ref)
        assert st.t_reached == w.t1 and st.n_out_written == len(ts)
        diff = metrics.normalized_final_error(y_ref, yf.cpu().numpy(), w.N)
        assert diff < 1e-6, (call, diff)
        np.testing.assert_allclose(yo.cpu().numpy(), yo_ref, rtol=0, atol=1e-6)


@pytest.mark.gpu
def test_noalloc_rejects_sizes_beyond_its_scratch():
    bs3 = library()
    torch = torch_cuda()
    N = bs3.NOALLOC_MAX_N + 1
    y0 = torch.zeros(N, dtype=torch.float64, device="cuda")
    wd = torch.zeros(16, dtype=torch.float32, device="cuda")
    rc, st = bs3.bs3_solve_noalloc(bs3.KURAMOTO, N, y0, None, wd, bs3.F32, (N + 15) // 16 * 16, 0.0, 1.0, y0,
                                   1e-6, 1e-6, bs3.MIXED1, bs3.ACC_FLOAT2, None, 0, None, None)
    assert rc == bs3.ERR_INVALID_ARG


def test_noalloc_rejects_a_row_stride_beyond_its_scratch():
    """A row stride ld above the scratch's j-vector capacity is refused before
    any CUDA call (so this runs without a GPU): N = 16 agents, ld = max + 16."""
    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_23727_gb300 import bs3
    bs3.load()
    ld = bs3.NOALLOC_MAX_N + 16
    host = np.zeros(64, dtype=np.float64)    # never read: the arguments are refused first
    rc, st = bs3.bs3_solve_noalloc(bs3.KURAMOTO, 16, host, None, host, bs3.F32, ld, 0.0, 1.0, host, 1e-6, 1e-6,
                                   bs3.MIXED1, bs3.ACC_FLOAT2, None, 0, None, None)
    assert rc == bs3.ERR_INVALID_ARG and st.status == bs3.ERR_INVALID_ARG


@pytest.mark.gpu
def test_noalloc_rejects_circadian_k1_outside_its_range():
    """k1_i must lie in (0, k0) (Theta_i = k1_i / (k0 - k1_i) > 0), as for
    bs3_create_system: one cell with k1 = k0 is refused before the solve."""
    bs3 = library()
    torch = torch_cuda()
    w = W.circadian(32, 3, t1=1.0)
    gl = w.globals
    g = [gl["k0"], gl["k2"], gl["k3"], gl["a"], gl["b"], gl["c"], gl["eps"], gl["I0"]]
    Kp, ld = _padded(w.coupling, np.float32)
    par = np.array(w.params, dtype=np.float64)
    par[7] = gl["k0"]
    dev = lambda a: torch.tensor(a, device="cuda")  # noqa: E731
    yf = torch.zeros(w.y0.size, dtype=torch.float64, device="cuda")
    rc, st = bs3.bs3_solve_noalloc(bs3.CIRCADIAN, w.N, dev(par), g, dev(Kp), bs3.F32, ld, w.t0, w.t1, dev(w.y0),
                                   w.rtol, w.atol, bs3.MIXED1, bs3.ACC_FLOAT2, None, 0, None, yf)
    assert rc == bs3.ERR_INVALID_ARG and st.status == bs3.ERR_INVALID_ARG
    # the next call with valid parameters runs normally
    rc, st = bs3.bs3_solve_noalloc(bs3.CIRCADIAN, w.N, dev(w.params), g, dev(Kp), bs3.F32, ld, w.t0, w.t1,
                                   dev(w.y0), w.rtol, w.atol, bs3.MIXED1, bs3.ACC_FLOAT2, None, 0, None, yf)
    assert rc == bs3.OK and st.t_reached == w.t1
