"""Lock-step ensembles sharing K on the tensor cores against per-trajectory
oracle solves of the same method (oracle variant "tensor")."""

import numpy as np
import pytest

import workloads as W
from oracle import bs3 as obs3
from oracle import metrics, models
from tests.gpu_helpers import library, torch_cuda

pytestmark = pytest.mark.gpu


def _ensemble(N, T, t1, rtol, seed):
    bs3 = library()
    torch = torch_cuda()
    K, omega, theta0 = W.kuramoto_ensemble(T=T, N=N, seed=seed, t1=t1, rtol=rtol)
    Kd = torch.tensor(K, dtype=torch.float32, device="cuda")
    om = torch.tensor(omega, dtype=torch.float64, device="cuda")
    th0 = torch.tensor(theta0, dtype=torch.float64, device="cuda")
    out = torch.full_like(th0, float("nan"))
    rc, n_acc, n_rej, status, steps = bs3.bs3_ensemble_solve(Kd, N, T, om, th0, 0.0, t1, rtol, rtol, out)
    assert rc == bs3.OK, bs3.bs3_status_string(rc)
    return K, omega, theta0, out.cpu().numpy(), n_acc, n_rej, status, steps


def test_ensemble_matches_oracle_per_trajectory():
    N, T, t1, rtol = 256, 128, 10.0, 1e-6
    K, omega, theta0, y, n_acc, n_rej, status, steps = _ensemble(N, T, t1, rtol, 3)
    assert np.all(status == 0) and np.all(np.isfinite(y))
    assert steps >= np.max(n_acc + n_rej)
    for b in (0, 63, 127):
        osys = models.make_system("kuramoto", N, omega[b], K, "f32")
        ref = obs3.solve(osys, 0.0, t1, theta0[b], rtol, rtol, "tensor")
        n_gpu, n_ref = n_acc[b] + n_rej[b], ref.n_accepted + ref.n_rejected
        assert abs(n_gpu - n_ref) <= max(2, 0.05 * n_ref), (b, n_gpu, n_ref)
        # the tensor cores accumulate each 16-wide step in binary32 with a bias
        # toward zero (about 0.5 ulp of the running sum per instruction; the
        # oracle sums exactly, then rounds), so compare global errors against a
        # tight binary64 solve of the same trajectory instead of the solutions
        tight = obs3.solve(models.make_system("kuramoto", N, omega[b], K, "f64"), 0.0, t1, theta0[b],
                           1e-10, 1e-10, "double")
        e_gpu = metrics.normalized_final_error(tight.y, y[b], N)
        e_tensor = metrics.normalized_final_error(tight.y, ref.y, N)
        print(f"trajectory {b}: global error gpu {e_gpu:.3e}, oracle tensor variant {e_tensor:.3e}")
        assert e_gpu <= 20.0 * e_tensor + 1e-6, (b, e_gpu, e_tensor)


def test_ensemble_trajectories_are_independent():
    """Trajectory b of an ensemble equals the same trajectory solved in another
    ensemble whose other members differ (per-trajectory h, t, decisions)."""
    bs3 = library()
    torch = torch_cuda()
    N, T, t1 = 256, 128, 5.0
    K, omega, theta0 = W.kuramoto_ensemble(T=T, N=N, seed=4)
    omega2, theta2 = omega.copy(), theta0.copy()
    omega2[1:] = np.random.default_rng(9).standard_normal((T - 1, N)) * 3.0
    outs = []
    for om_, th_ in ((omega, theta0), (omega2, theta2)):
        Kd = torch.tensor(K, dtype=torch.float32, device="cuda")
        out = torch.empty((T, N), dtype=torch.float64, device="cuda")
        rc, n_acc, n_rej, status, steps = bs3.bs3_ensemble_solve(
            Kd, N, T, torch.tensor(om_, device="cuda"), torch.tensor(th_, device="cuda"), 0.0, t1, 1e-6, 1e-6, out)
        assert rc == bs3.OK
        outs.append((out.cpu().numpy()[0], n_acc[0], n_rej[0]))
    assert outs[0][1:] == outs[1][1:]
    np.testing.assert_array_equal(outs[0][0], outs[1][0])


def test_tile_widths_agree():
    """128- and 256-column output tiles give the same trajectories (each output
    is the same sum over K in the same order) and the same decisions."""
    bs3 = library()
    torch = torch_cuda()
    N, T, t1 = 256, 128, 5.0
    K, omega, theta0 = W.kuramoto_ensemble(T=T, N=N, seed=6)
    Kd = torch.tensor(K, dtype=torch.float32, device="cuda")
    om = torch.tensor(omega, dtype=torch.float64, device="cuda")
    th = torch.tensor(theta0, dtype=torch.float64, device="cuda")
    res = {}
    for tile in (256, 128):
        out = torch.empty_like(th)
        rc, n_acc, n_rej, status, _ = bs3.bs3_ensemble_solve(Kd, N, T, om, th, 0.0, t1, 1e-6, 1e-6, out, tile_n=tile)
        assert rc == bs3.OK and np.all(status == 0)
        res[tile] = (out.cpu().numpy(), n_acc, n_rej)
    np.testing.assert_array_equal(res[128][1], res[256][1])
    np.testing.assert_array_equal(res[128][2], res[256][2])
    np.testing.assert_allclose(res[128][0], res[256][0], rtol=0, atol=1e-9)


def test_tile_autotuner_and_narrow_ensembles():
    bs3 = library()
    torch = torch_cuda()
    N, T = 256, 64   # only the 128-column tile fits 2T = 128
    K, omega, theta0 = W.kuramoto_ensemble(T=T, N=N, seed=7)
    Kd = torch.tensor(K, dtype=torch.float32, device="cuda")
    om = torch.tensor(omega, dtype=torch.float64, device="cuda")
    th = torch.tensor(theta0, dtype=torch.float64, device="cuda")
    out = torch.empty_like(th)
    rc, tile, us = bs3.bs3_ensemble_autotune(Kd, N, T, om, th, 0.0, 5.0, 1e-6, 1e-6, 16, out)
    assert rc == bs3.OK and tile == 128 and us > 0.0
    assert bs3.bs3_ensemble_solve(Kd, N, T, om, th, 0.0, 5.0, 1e-6, 1e-6, out, tile_n=256)[0] == bs3.ERR_INVALID_ARG
    rc, n_acc, n_rej, status, _ = bs3.bs3_ensemble_solve(Kd, N, T, om, th, 0.0, 5.0, 1e-6, 1e-6, out)
    assert rc == bs3.OK and np.all(status == 0)
    # a bounded solve stops early with MAX_STEPS
    rc, *_ = bs3.bs3_ensemble_solve(Kd, N, T, om, th, 0.0, 5.0, 1e-6, 1e-6, out, max_lockstep=8)
    assert rc == bs3.ERR_MAX_STEPS
    # the autotuner chooses between both widths when both fit
    T2 = 128
    K2, om2, th2 = W.kuramoto_ensemble(T=T2, N=N, seed=8)
    out2 = torch.empty((T2, N), dtype=torch.float64, device="cuda")
    rc, tile, _ = bs3.bs3_ensemble_autotune(torch.tensor(K2, dtype=torch.float32, device="cuda"), N, T2,
                                            torch.tensor(om2, device="cuda"), torch.tensor(th2, device="cuda"),
                                            0.0, 5.0, 1e-6, 1e-6, 16, out2)
    assert rc == bs3.OK and tile in (128, 256)
