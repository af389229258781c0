"""GPU parity of one BS3 attempt (stages, X^{n+1}, K4 and the error E)."""

import numpy as np
import pytest

import workloads as W
from oracle import bs3 as obs3
from oracle import models
from tests.gpu_helpers import U32, U64, library, rhs_tolerance, torch_cuda

pytestmark = pytest.mark.gpu


def _wl(kind, N):
    if kind == "lco_cfg":
        return W.lco_config(N, 4)
    if kind == "lco_paper":
        return W.lco_paper(N, 4, heterogeneous=True)
    if kind == "kuramoto":
        return W.kuramoto(N, 4)
    return W.circadian(N, 4)


@pytest.mark.parametrize("kind", models.KINDS)
@pytest.mark.parametrize("variant", list(obs3.PAPER_VARIANTS))
@pytest.mark.parametrize("accum", ["float2", "f64"])
def test_attempt_matches_oracle(kind, variant, accum):
    bs3 = library()
    torch = torch_cuda()
    N = 203
    w = _wl(kind, N)
    store = "f64" if variant == "double" else "f32"
    sysm = bs3.System.from_workload(w, store)
    osys = models.from_workload(w, store)
    st = np.float32 if variant == "single" else np.float64
    X = w.y0.astype(st)
    K1 = models.rhs(osys, 0.0, X, obs3.VARIANTS[variant][4])
    h, rtol, atol = 0.05, 1e-6, 1e-6
    Xn, K4, E, _ = obs3.attempt(osys, 0.0, X, K1, h, variant, rtol, atol)
    xd = torch.tensor(X.astype(np.float64), device="cuda")
    kd = torch.tensor(K1.astype(np.float64), device="cuda")
    xn = torch.empty_like(xd)
    k4 = torch.empty_like(xd)
    rc, err = bs3.bs3_attempt(sysm.handle, 0.0, h, xd, kd, rtol, atol, bs3.VARIANT_IDS[variant],
                              bs3.ACCUM_IDS[accum], xn, k4)
    sysm.close()
    assert rc == bs3.OK
    xn = xn.cpu().numpy(); k4 = k4.cpu().numpy()
    # stage values differ by at most one right-hand-side tolerance per stage
    worst = max((rhs_tolerance(osys, X, obs3.VARIANTS[variant][s], accum) for s in (2, 3, 4)),
                key=lambda v: v.sum())
    u = U32 if variant == "single" else U64
    # a difference in one component reaches the others through the stage arguments
    worst = np.full_like(worst, worst.max())
    tol_x = 2 * h * worst + 8 * u * (np.abs(Xn) + 1)
    assert np.all(np.abs(xn - Xn) <= tol_x)
    assert np.all(np.abs(k4 - K4) <= 4 * worst + 4 * u * (np.abs(K4) + 1))
    Wk = np.maximum(np.maximum(np.abs(X.astype(np.float64)), np.abs(Xn.astype(np.float64))), atol / rtol)
    tol_e = np.max((h * 0.5 * 4 * worst + 8 * u * np.abs(Xn)) / Wk) + 1e-12
    assert abs(err - E) <= tol_e, (err, E, tol_e)
