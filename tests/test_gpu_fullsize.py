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


def test_ensemble_256x8192_sampled_trajectories_against_oracle():
    """Three trajectories of the coupled full-size ensemble (T = 256, N = 8192,
    t in [0, 0.5], rtol 1e-6) against the oracle's tensor variant solved one by
    one: attempt counts within 5 %, final phases within a bound derived from
    the one place the two differ.  Both use the same bfloat16 split of K and of
    the sine/cosine; the oracle sums the three split products exactly and
    rounds once, the tensor cores round every accumulation toward zero.  With
    3N/16 accumulations of at most one binary32 ulp of a running sum bounded by
    R_i = sum_j |K_ij| (|sin|, |cos| <= 1), a coupling differs by at most
    d = 2 (3N/16) 2^-23 max_i R_i; over the span, by Gronwall with the
    Lipschitz constant L = 2 max_i R_i, the phases by d (e^{L t} - 1) / L.  A
    wrong stage combination, a stale operand copy or a sign error in the
    epilogue exceeds it; the split itself and the tiling are pinned exactly by
    the one-hot products of tests/test_gpu_tc.py."""
    bs3 = library()
    torch = torch_cuda()
    from oracle import bs3 as obs3
    T, N, t1, rtol = 256, 8192, 0.5, 1e-6
    K, omega, theta0 = W.kuramoto_ensemble(T=T, N=N, seed=14)
    Kd = torch.tensor(K, dtype=torch.float32, device="cuda")
    om = torch.tensor(omega, device="cuda")
    th = torch.tensor(theta0, device="cuda")
    out = torch.empty_like(th)
    rc, n_acc, n_rej, status, _ = bs3.bs3_ensemble_solve(Kd, N, T, om, th, 0.0, t1, rtol, rtol, out)
    assert rc == bs3.OK and np.all(status == 0)
    del Kd
    y = out.cpu().numpy()
    R = float(np.max(np.abs(K.astype(np.float64)).sum(axis=1)))
    d = 2.0 * (3 * N / 16) * 2.0 ** -23 * R
    L = 2.0 * R
    bound = d * (np.exp(L * t1) - 1.0) / L
    osys = models.make_system("kuramoto", N, omega[0], K, "f32")
    for b in (0, 127, 255):
        osys.params = np.asarray(omega[b], dtype=np.float64)
        ref = obs3.solve(osys, 0.0, t1, theta0[b], rtol, rtol, "tensor")
        assert ref.status == obs3.OK
        n_gpu, n_ref = int(n_acc[b] + n_rej[b]), ref.n_accepted + ref.n_rejected
        assert abs(n_gpu - n_ref) <= max(2, 0.05 * n_ref), (b, n_gpu, n_ref)
        dev = float(np.max(np.abs(y[b] - ref.y)))
        print(f"trajectory {b}: attempts gpu {n_gpu} oracle {n_ref}, max |dtheta| {dev:.3e} (bound {bound:.3e})")
        assert dev <= bound, (b, dev, bound)


def test_config4_group_and_1000_systems_in_one_submission():
    """The shared-K batch configuration in one bs3_solve_batch call: 256
    Kuramoto trajectories at N = 8192 sharing K (t in [0, 0.5]) beside 1000
    second-order oscillator systems with N log-uniform in [64, 4096] (binary16
    weights, Mixed1, t in [0, 10]).  The group equals the standalone ensemble
    entry's solve (same products and decisions); the four smallest systems
    match their oracle solves; the largest (solved by a team of CTAs) matches
    its standalone bs3_solve."""
    bs3 = library()
    torch = torch_cuda()
    from oracle import bs3 as obs3
    from oracle import metrics
    systems = W.lco_ragged_batch(count=1000, n_min=64, n_max=4096, seed=0, t1=10.0, rtol=1e-6)
    handles, items, outs = [], [], []
    for w in systems:
        s = bs3.System.from_workload(w, "f16")
        handles.append(s)
        y0 = torch.tensor(w.y0, device="cuda")
        yf = torch.full_like(y0, float("nan"))
        outs.append(yf)
        items.append({"sys": s.handle, "y0": y0, "y_final": yf, "t0": w.t0, "t1": w.t1, "rtol": 1e-6, "atol": 1e-6})
    T, N, t1 = 256, 8192, 0.5
    K, omega, theta0 = W.kuramoto_ensemble(T=T, N=N, seed=15)
    g = {"K": torch.tensor(K, device="cuda"), "N": N, "T": T, "omega": torch.tensor(omega, device="cuda"),
         "theta0": torch.tensor(theta0, device="cuda"), "t0": 0.0, "t1": t1, "rtol": 1e-6, "atol": 1e-6,
         "n_acc": np.zeros(T, dtype=np.int64), "n_rej": np.zeros(T, dtype=np.int64),
         "status": np.zeros(T, dtype=np.int32)}
    g["theta_out"] = torch.full_like(g["theta0"], float("nan"))
    rc, stats, steps, ms = bs3.bs3_solve_batch(items, bs3.MIXED1, bs3.ACC_FLOAT2, 0, g)
    assert rc == bs3.OK, bs3.bs3_status_string(rc)
    assert all(st.status == 0 and st.t_reached == 10.0 for st in stats)
    assert np.all(g["status"] == 0)
    out = torch.empty_like(g["theta0"])
    rc, n_acc, n_rej, status, steps2 = bs3.bs3_ensemble_solve(g["K"], N, T, g["omega"], g["theta0"], 0.0, t1, 1e-6,
                                                              1e-6, out)
    assert rc == bs3.OK and steps == steps2 and np.array_equal(n_acc, g["n_acc"])
    np.testing.assert_array_equal(out.cpu().numpy(), g["theta_out"].cpu().numpy())
    del out, g
    order = np.argsort([w.N for w in systems])
    for k in order[:4]:
        w = systems[k]
        ref = obs3.solve(models.from_workload(w, "f16"), w.t0, w.t1, w.y0, 1e-6, 1e-6, "mixed1")
        n_gpu, n_ref = stats[k].n_accepted + stats[k].n_rejected, ref.n_accepted + ref.n_rejected
        assert abs(n_gpu - n_ref) <= max(2, 0.05 * n_ref), (k, w.N, n_gpu, n_ref)
        assert metrics.normalized_final_error(ref.y, outs[k].cpu().numpy(), w.N) < 1e-5, (k, w.N)
    k = int(order[-1])
    w = systems[k]
    rc, st, y, _ = handles[k].solve(w.t0, w.t1, w.y0, 1e-6, 1e-6, "mixed1", "float2")
    assert rc == bs3.OK
    n_gpu, n_ref = stats[k].n_accepted + stats[k].n_rejected, st.n_accepted + st.n_rejected
    assert abs(n_gpu - n_ref) <= max(2, 0.05 * n_ref)
    assert metrics.normalized_final_error(y, outs[k].cpu().numpy(), w.N) < 1e-5
    for h in handles:
        h.close()
