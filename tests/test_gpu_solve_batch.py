"""bs3_solve_batch: independent systems (system handles, each with its own
span and tolerances) and a shared-K trajectory group in one submission,
against per-system oracle solves and the standalone ensemble entry."""

import numpy as np
import pytest

import workloads as W
from oracle import bs3 as obs3
from oracle import metrics, models
from tests.gpu_helpers import library, torch_cuda

pytestmark = pytest.mark.gpu


def _items(bs3, torch, systems, store, rtols, host=False):
    handles, items, outs = [], [], []
    for w, rt in zip(systems, rtols):
        s = bs3.System.from_workload(w, store)
        handles.append(s)
        if host:
            y0, yf = np.ascontiguousarray(w.y0), np.full(w.y0.size, np.nan)
        else:
            y0 = torch.tensor(w.y0, device="cuda")
            yf = torch.full_like(y0, float("nan"))
        outs.append((y0, yf))
        items.append({"sys": s.handle, "y0": y0, "y_final": yf, "t0": w.t0, "t1": w.t1, "rtol": rt, "atol": rt})
    return handles, items, outs


def _group(torch, T, N, t1, rtol, seed):
    K, omega, theta0 = W.kuramoto_ensemble(T=T, N=N, seed=seed)
    g = {"K": torch.tensor(K, device="cuda"), "N": N, "T": T, "omega": torch.tensor(omega, device="cuda"),
         "theta0": torch.tensor(theta0, device="cuda"), "t0": 0.0, "t1": t1, "rtol": rtol, "atol": rtol,
         "n_acc": np.zeros(T, dtype=np.int64), "n_rej": np.zeros(T, dtype=np.int64),
         "status": np.zeros(T, dtype=np.int32)}
    g["theta_out"] = torch.full_like(g["theta0"], float("nan"))
    return K, omega, theta0, g


@pytest.mark.parametrize("host", [False, True])
def test_items_with_their_own_tolerances_match_the_oracle(host):
    bs3 = library()
    torch = torch_cuda()
    systems = W.lco_ragged_batch(count=12, n_min=16, n_max=300, seed=31, t1=5.0)
    for k, w in enumerate(systems):
        w.t1 = 3.0 + 0.5 * k           # uneven spans
    rtols = [(1e-5, 1e-6, 1e-7)[k % 3] for k in range(len(systems))]
    handles, items, outs = _items(bs3, torch, systems, "f32", rtols, host=host)
    rc, stats, _, ms = bs3.bs3_solve_batch(items, bs3.MIXED2, bs3.ACC_FLOAT2, bs3.HOST_IO if host else 0)
    assert rc == bs3.OK, bs3.bs3_status_string(rc)
    assert ms > 0
    for k, w in enumerate(systems):
        ref = obs3.solve(models.from_workload(w, "f32"), w.t0, w.t1, w.y0, rtols[k], rtols[k], "mixed2")
        n_gpu, n_ref = stats[k].n_accepted + stats[k].n_rejected, ref.n_accepted + ref.n_rejected
        assert stats[k].status == 0 and stats[k].t_reached == w.t1
        assert abs(n_gpu - n_ref) <= max(2, 0.05 * n_ref), (k, w.N, n_gpu, n_ref)
        y = outs[k][1] if host else outs[k][1].cpu().numpy()
        assert metrics.normalized_final_error(ref.y, y, w.N) < 10 * rtols[k], (k, w.N)
    for h in handles:
        h.close()


def test_group_alone_equals_the_ensemble_entry():
    """A batch of only a group runs the same products and decisions as
    bs3_ensemble_solve: identical phases and counts."""
    bs3 = library()
    torch = torch_cuda()
    K, omega, theta0, g = _group(torch, 64, 256, 4.0, 1e-6, 41)
    rc, stats, steps, _ = bs3.bs3_solve_batch([], bs3.MIXED1, bs3.ACC_FLOAT2, 0, g)
    assert rc == bs3.OK, bs3.bs3_status_string(rc)
    out = torch.empty_like(g["theta0"])
    rc, n_acc, n_rej, status, steps2 = bs3.bs3_ensemble_solve(g["K"], 256, 64, g["omega"], g["theta0"], 0.0, 4.0,
                                                              1e-6, 1e-6, out)
    assert rc == bs3.OK
    assert steps == steps2 and np.array_equal(n_acc, g["n_acc"]) and np.array_equal(n_rej, g["n_rej"])
    np.testing.assert_array_equal(out.cpu().numpy(), g["theta_out"].cpu().numpy())


@pytest.mark.parametrize("ctas", [0, 40])
def test_items_and_group_in_one_submission(ctas):
    """Systems and a group together in one graph (ctas = 0: one after the
    other on every SM; ctas = 40: side by side on disjoint CTA budgets): the
    group as bs3_ensemble_solve computes it, sampled trajectories against the
    oracle's tensor variant, sampled systems against their oracle solves."""
    bs3 = library()
    torch = torch_cuda()
    systems = W.lco_ragged_batch(count=40, n_min=16, n_max=400, seed=32, t1=4.0)
    rtols = [1e-6] * len(systems)
    handles, items, outs = _items(bs3, torch, systems, "f32", rtols)
    T, N, t1 = 64, 512, 2.0
    K, omega, theta0, g = _group(torch, T, N, t1, 1e-6, 42)
    g["ctas"] = ctas
    rc, stats, steps, ms = bs3.bs3_solve_batch(items, bs3.MIXED1, bs3.ACC_FLOAT2, 0, g)
    assert rc == bs3.OK, bs3.bs3_status_string(rc)
    assert np.all(g["status"] == 0) and steps >= np.max(g["n_acc"] + g["n_rej"])
    out = torch.empty_like(g["theta0"])
    rc, n_acc, n_rej, status, steps2 = bs3.bs3_ensemble_solve(g["K"], N, T, g["omega"], g["theta0"], 0.0, t1, 1e-6,
                                                              1e-6, out)
    assert rc == bs3.OK and steps == steps2 and np.array_equal(n_acc, g["n_acc"])
    y_group = g["theta_out"].cpu().numpy()
    np.testing.assert_array_equal(out.cpu().numpy(), y_group)
    osys = models.make_system("kuramoto", N, omega[0], K, "f32")
    for b in (0, T - 1):
        osys.params = np.asarray(omega[b], dtype=np.float64)
        ref = obs3.solve(osys, 0.0, t1, theta0[b], 1e-6, 1e-6, "tensor")
        n_gpu, n_ref = int(n_acc[b] + n_rej[b]), ref.n_accepted + ref.n_rejected
        assert abs(n_gpu - n_ref) <= max(2, 0.05 * n_ref)
        assert metrics.normalized_final_error(ref.y, y_group[b], N) < 1e-5
    for k, w in enumerate(systems):
        if k % 4:
            continue
        ref = obs3.solve(models.from_workload(w, "f32"), w.t0, w.t1, w.y0, 1e-6, 1e-6, "mixed1")
        n_gpu, n_ref = stats[k].n_accepted + stats[k].n_rejected, ref.n_accepted + ref.n_rejected
        assert stats[k].status == 0 and abs(n_gpu - n_ref) <= max(2, 0.05 * n_ref), (k, w.N)
        assert metrics.normalized_final_error(ref.y, outs[k][1].cpu().numpy(), w.N) < 1e-5, (k, w.N)
    for h in handles:
        h.close()


def test_mixed_kinds_or_types_are_refused():
    bs3 = library()
    torch = torch_cuda()
    a = W.lco_config(32, 1, t1=1.0)
    b = W.kuramoto(32, 2, t1=1.0)
    ha, items_a, _ = _items(bs3, torch, [a], "f32", [1e-6])
    hb, items_b, _ = _items(bs3, torch, [b], "f32", [1e-6])
    hc, items_c, _ = _items(bs3, torch, [a], "f64", [1e-6])
    rc, stats, _, _ = bs3.bs3_solve_batch(items_a + items_b, bs3.MIXED1, bs3.ACC_FLOAT2)
    assert rc == bs3.ERR_INVALID_ARG
    rc, stats, _, _ = bs3.bs3_solve_batch(items_a + items_c, bs3.MIXED1, bs3.ACC_FLOAT2)
    assert rc == bs3.ERR_INVALID_ARG
    rc, stats, _, _ = bs3.bs3_solve_batch(items_a + items_a, bs3.MIXED1, bs3.ACC_FLOAT2)
    assert rc == bs3.ERR_INVALID_ARG      # one system in two items
    bad = dict(items_a[0], rtol=0.0)
    rc, stats, _, _ = bs3.bs3_solve_batch([bad], bs3.MIXED1, bs3.ACC_FLOAT2)
    assert rc == bs3.ERR_INVALID_ARG and stats[0].status == bs3.ERR_INVALID_ARG
    for h in ha + hb + hc:
        h.close()
