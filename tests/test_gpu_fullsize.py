"""Full-size workloads in the launch configurations the benchmarks time, checked
on outputs the oracle can compute one by one or through properties that hold at
any size: the 256-trajectory ensemble at N = 8192 (closed form when K = 0, and
trajectory independence) and at N = 16384 (several tiles per persistent CTA),
the N = 32768 binary16 oscillators (sampled rows of one evaluation), and the
1000-system ragged batch (sampled systems against their own solves)."""

import numpy as np
import pytest

import workloads as W
from oracle import exact, models
from tests.gpu_helpers import library, rhs_tolerance, torch_cuda

pytestmark = pytest.mark.gpu


def test_ensemble_256x8192_uncoupled_closed_form():
    bs3 = library()
    torch = torch_cuda()
    T, N, t1 = 256, 8192, 10.0
    _, omega, theta0 = W.kuramoto_ensemble(T=T, N=N, seed=11)
    Kd = torch.zeros((N, N), dtype=torch.float32, device="cuda")
    om = torch.tensor(omega, device="cuda")
    th = torch.tensor(theta0, device="cuda")
    out = torch.empty_like(th)
    rc, n_acc, n_rej, status, _ = bs3.bs3_ensemble_solve(Kd, N, T, om, th, 0.0, t1, 1e-8, 1e-8, out)
    assert rc == bs3.OK and np.all(status == 0) and np.all(n_rej == 0)
    ex = exact.kuramoto_uncoupled(theta0, omega, t1)
    assert np.max(np.abs(out.cpu().numpy() - ex)) <= 1e-12 * (1.0 + np.max(np.abs(ex)))


def test_ensemble_256x8192_members_are_independent():
    """Trajectory 0 of the full-size ensemble is the same when every other
    trajectory starts elsewhere (per-trajectory step sizes and decisions)."""
    bs3 = library()
    torch = torch_cuda()
    T, N, t1 = 256, 8192, 2.0
    K, omega, theta0 = W.kuramoto_ensemble(T=T, N=N, seed=12)
    Kd = torch.tensor(K, dtype=torch.float32, device="cuda")
    om = torch.tensor(omega, device="cuda")
    first = None
    for shift in (0.0, 1.0):
        th0 = theta0.copy()
        th0[1:] += shift
        th = torch.tensor(th0, device="cuda")
        out = torch.empty_like(th)
        rc, n_acc, n_rej, status, _ = bs3.bs3_ensemble_solve(Kd, N, T, om, th, 0.0, t1, 1e-6, 1e-6, out)
        assert rc == bs3.OK and np.all(status == 0)
        res = (out[0].cpu().numpy(), int(n_acc[0]), int(n_rej[0]))
        if first is None:
            first = res
        else:
            assert res[1:] == first[1:]
            np.testing.assert_array_equal(res[0], first[0])


def test_ensemble_persistent_tiles_agree_across_widths():
    """T = 256 trajectories at N = 16384: with 128-column tiles every CTA of the
    persistent product takes three or four tiles (512 tiles on at most 152
    CTAs, both tensor-memory accumulators reused), with 256-column tiles one or
    two.  Each output is the same sum in the same order either way, so the
    trajectories and every decision agree; with K = 0 both reproduce the
    closed form."""
    bs3 = library()
    torch = torch_cuda()
    T, N, t1 = 256, 16384, 0.5
    K, omega, theta0 = W.kuramoto_ensemble(T=T, N=N, seed=13)
    om = torch.tensor(omega, device="cuda")
    th = torch.tensor(theta0, device="cuda")
    for coupled in (True, False):
        Kd = torch.tensor(K, device="cuda") if coupled else torch.zeros((N, N), dtype=torch.float32, device="cuda")
        res = {}
        for tile in (128, 256):
            out = torch.empty_like(th)
            rc, n_acc, n_rej, status, _ = bs3.bs3_ensemble_solve(Kd, N, T, om, th, 0.0, t1, 1e-6, 1e-6, out,
                                                                 tile_n=tile)
            assert rc == bs3.OK and np.all(status == 0), (coupled, tile)
            res[tile] = (out.cpu().numpy(), n_acc, n_rej)
        del Kd
        np.testing.assert_array_equal(res[128][1], res[256][1])
        np.testing.assert_array_equal(res[128][2], res[256][2])
        np.testing.assert_allclose(res[128][0], res[256][0], rtol=0, atol=1e-9)
        if not coupled:
            ex = exact.kuramoto_uncoupled(theta0, omega, t1)
            assert np.max(np.abs(res[128][0] - ex)) <= 1e-12 * (1.0 + np.max(np.abs(ex)))


def test_oscillators_32768_f16_sampled_rows():
    """One evaluation of the N = 32768 binary16 system (the learned-proposer
    workload) in its solve launch configuration: 48 sampled agents against the
    oracle, in the precisions of Single and of the Mixed stages."""
    bs3 = library()
    torch = torch_cuda()
    N = 32768
    w = W.lco_config(N, 7, t1=10.0, dtype=np.float32)
    sysm = bs3.System.from_workload(w, "f16")
    osys = models.from_workload(w, "f16")
    rows = np.sort(np.random.default_rng(3).choice(N, 48, replace=False))
    rows[-1] = N - 1
    for prec in (("S", "S", "S"), ("D", "D", "S")):
        yd = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
        out = torch.empty_like(yd)
        p = [0 if c == "S" else 1 for c in prec]
        assert bs3.bs3_rhs(sysm.handle, 0.0, yd, p[0], p[1], p[2], bs3.ACC_FLOAT2, out) == bs3.OK
        got = out.cpu().numpy().reshape(2, N)[:, rows]
        y_in = w.y0.astype(np.float32) if prec == ("S", "S", "S") else w.y0
        ref = models.rhs(osys, 0.0, y_in, prec, rows=rows)
        tol = rhs_tolerance(osys, w.y0, prec).reshape(2, N)[:, rows]
        assert np.all(np.abs(got - ref) <= tol), prec
    sysm.close()


def test_ragged_1000_sampled_systems_match_single_solves():
    """The 1000-system batch of the benchmark (N log-uniform in [64, 4096],
    f16, Mixed1, t in [0, 2]): sampled systems, the largest and the smallest
    among them, agree with their standalone solves."""
    bs3 = library()
    torch_cuda()
    systems = W.lco_ragged_batch(count=1000, n_min=64, n_max=4096, seed=0, t1=2.0, rtol=1e-6)
    Ns = [w.N for w in systems]
    K = np.concatenate([np.asarray(w.coupling, dtype=np.float32).ravel() for w in systems])
    rc, yf, stats, _ = bs3.bs3_batch_solve(bs3.LCO_CFG, Ns, np.concatenate([w.params for w in systems]), K, bs3.F16,
                                           np.concatenate([w.y0 for w in systems]), np.zeros(1000),
                                           np.full(1000, 2.0), 1e-6, 1e-6, bs3.MIXED1, bs3.ACC_FLOAT2)
    assert rc == bs3.OK and all(s.status == 0 for s in stats)
    offs = np.concatenate([[0], np.cumsum([2 * n for n in Ns])])
    picks = sorted(set([int(np.argmax(Ns)), int(np.argmin(Ns))] + list(np.random.default_rng(4).choice(1000, 6))))
    for k in picks:
        w = systems[k]
        s = bs3.System.from_workload(w, "f16")
        rc, st, y, _ = s.solve(w.t0, 2.0, w.y0, 1e-6, 1e-6, "mixed1", "float2")
        s.close()
        assert rc == bs3.OK
        # the batch and the whole-GPU launch split each row's sum over different
        # thread groups, so their roundoff differs and a decision may part
        n_b = stats[k].n_accepted + stats[k].n_rejected
        assert abs((st.n_accepted + st.n_rejected) - n_b) <= 2, (k, w.N)
        np.testing.assert_allclose(yf[offs[k]:offs[k + 1]], y, rtol=0, atol=1e-6)
