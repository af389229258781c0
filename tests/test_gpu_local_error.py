"""Real local error against the embedded estimate on the GPU (the local-error
comparison of Sec. 3 for the second-order oscillators, whose exact flow is
known): a solve records its steps, an identical solve writes the state at the
end of every accepted step (dense output at theta = 1), and each step's real
local error is the distance between the GPU's X_{n+1} and the exact flow
X_ex of X_n over h_n, normalised as Eq. LCO-Local-Error does:
max_k |X_{n+1,k} - X_ex,k| / max(|X_ex,k|, delta), delta = Ab/Rel.  The paper's finding: in binary32
state (Single) the error control fails at tight tolerances -- the estimate
stays below Rel while the real local error does not -- and the mixed
solvers, whose state is binary64, keep it under control."""

import numpy as np
import pytest

import workloads as W
from oracle import exact
from tests.gpu_helpers import library, torch_cuda

pytestmark = pytest.mark.gpu


def _local_errors(w, variant, store, rtol):
    bs3 = library()
    torch_cuda()
    N = w.N
    sysm = bs3.System.from_workload(w, store)
    cap = 1 << 16
    assert bs3.bs3_set_history(sysm.handle, cap) == bs3.OK
    rc, st, _, _ = sysm.solve(w.t0, w.t1, w.y0, rtol, rtol, variant, "float2")
    assert rc == bs3.OK
    rc, H = bs3.bs3_get_history(sysm.handle, cap)
    acc = H[H[:, 3] == 1.0]
    ends = acc[:, 0] + acc[:, 1]
    ends[-1] = w.t1
    ts = np.concatenate([[w.t0], ends])
    rc, st2, _, X = sysm.solve(w.t0, w.t1, w.y0, rtol, rtol, variant, "float2", t_out=ts)
    sysm.close()
    assert rc == bs3.OK and st2.n_accepted == st.n_accepted == len(acc)
    # the exact flow of the system the solver integrates (its stored weights)
    A = np.asarray(w.coupling, dtype=np.float32 if store == "f32" else np.float64).astype(np.float64)
    real = np.empty(len(acc))
    for k in range(len(acc)):
        x0, x1 = X[k], X[k + 1]
        ex = exact.lco_cfg_exact(w.params, A, x0[:N], x0[N:], ts[k + 1] - ts[k])
        real[k] = np.max(np.abs(x1 - ex) / np.maximum(np.abs(ex), w.atol / w.rtol))
    return real / rtol, acc[:, 2] / rtol


@pytest.mark.parametrize("rtol", [1e-5, 1e-9])
def test_real_local_error_against_estimate(rtol):
    w = W.lco_config(256, 0, t1=5.0)
    out = {}
    for variant, store in (("double", "f64"), ("mixed2", "f32"), ("mixed1", "f32"), ("single", "f32")):
        real, est = _local_errors(w, variant, store, rtol)
        out[variant] = (np.median(real), np.max(real), np.mean(real > 1.0), np.median(est))
        print(f"rtol {rtol:.0e} {variant:7s}: real/Rel median {out[variant][0]:.3g} max {out[variant][1]:.3g} "
              f"steps above Rel {100 * out[variant][2]:.0f} %, estimate/Rel median {out[variant][3]:.3g}")
        assert out[variant][3] < 1.0    # accepted steps: E <= Rel
    for variant in ("double", "mixed2"):
        assert out[variant][1] < 1.0, variant
    assert out["mixed1"][0] < 1.0
    if rtol >= 1e-5:
        assert out["single"][1] < 1.0
    else:
        # binary32 state: rounding alone exceeds the tolerance at every step
        assert out["single"][0] > 10.0 and out["single"][2] > 0.9
