"""Lock-step ensembles sharing K on the tensor cores against per-trajectory
oracle solves of the same method (oracle variant "tensor")."""

import numpy as np
import pytest

import workloads as W
from oracle import bs3 as obs3
from oracle import models
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
    """Per trajectory against the oracle's tensor variant solved alone: over
    t in [0, 10] the attempt counts agree within 5 %; over t in [0, 0.5] the
    final phases agree within the bound derived from the one place the two
    differ (the tensor cores round each of the 3N/16 accumulations of an
    output toward zero, at most one binary32 ulp of a running sum bounded by
    R_i = sum_j |K_ij|; the coupling then differs by at most
    d = 2 (3N/16) 2^-23 max_i R_i, and the phases by d (e^{L t} - 1) / L with
    the Lipschitz constant L = 2 max_i R_i)."""
    N, T, rtol = 256, 128, 1e-6
    K, omega, theta0, y, n_acc, n_rej, status, steps = _ensemble(N, T, 10.0, rtol, 3)
    assert np.all(status == 0) and np.all(np.isfinite(y))
    assert steps >= np.max(n_acc + n_rej)
    for b in (0, 63, 127):
        osys = models.make_system("kuramoto", N, omega[b], K, "f32")
        ref = obs3.solve(osys, 0.0, 10.0, theta0[b], rtol, rtol, "tensor")
        n_gpu, n_ref = n_acc[b] + n_rej[b], ref.n_accepted + ref.n_rejected
        assert abs(n_gpu - n_ref) <= max(2, 0.05 * n_ref), (b, n_gpu, n_ref)
    t1 = 0.5
    K, omega, theta0, y, n_acc, n_rej, status, steps = _ensemble(N, T, t1, rtol, 3)
    R = float(np.max(np.abs(K.astype(np.float64)).sum(axis=1)))
    d = 2.0 * (3 * N / 16) * 2.0 ** -23 * R
    L = 2.0 * R
    bound = d * (np.exp(L * t1) - 1.0) / L
    for b in (0, 63, 127):
        osys = models.make_system("kuramoto", N, omega[b], K, "f32")
        ref = obs3.solve(osys, 0.0, t1, theta0[b], rtol, rtol, "tensor")
        n_gpu, n_ref = n_acc[b] + n_rej[b], ref.n_accepted + ref.n_rejected
        assert abs(n_gpu - n_ref) <= max(2, 0.05 * n_ref), (b, n_gpu, n_ref)
        dev = float(np.max(np.abs(y[b] - ref.y)))
        print(f"trajectory {b}: max |dtheta| {dev:.3e} (bound {bound:.3e})")
        assert dev <= bound, (b, dev, bound)


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
