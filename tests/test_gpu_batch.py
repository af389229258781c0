"""Ragged batches of independent systems in one launch (each CTA solves whole
systems) against per-system oracle solves."""

import numpy as np
import pytest

import workloads as W
from oracle import bs3 as obs3
from oracle import metrics, models
from tests.gpu_helpers import library, torch_cuda

pytestmark = pytest.mark.gpu


def _batch(systems, store, variant, kind="lco_cfg"):
    bs3 = library()
    torch_cuda()
    Ns = [w.N for w in systems]
    params = None if kind == "lco_paper" else np.concatenate([w.params for w in systems])
    K = np.concatenate([np.asarray(w.coupling, dtype=np.float32).ravel() for w in systems])
    y0 = np.concatenate([w.y0 for w in systems])
    t0 = np.array([w.t0 for w in systems])
    t1 = np.array([w.t1 for w in systems])
    rc, yf, stats, _ = bs3.bs3_batch_solve(bs3.KIND_IDS[kind], Ns, params, K, bs3.DTYPE_IDS[store], y0, t0, t1,
                                        systems[0].rtol, systems[0].atol, bs3.VARIANT_IDS[variant],
                                        bs3.ACC_FLOAT2)
    assert rc == bs3.OK, bs3.bs3_status_string(rc)
    out, o = [], 0
    for w in systems:
        n = w.d * w.N
        out.append(yf[o:o + n])
        o += n
    return out, stats


@pytest.mark.parametrize("variant,store", [("double", "f64"), ("mixed2", "f32"), ("mixed1", "f16")])
def test_ragged_oscillators_match_oracle(variant, store):
    systems = W.lco_ragged_batch(count=24, n_min=16, n_max=300, seed=5, t1=5.0)
    out, stats = _batch(systems, store, variant)
    for k, w in enumerate(systems):
        ref = obs3.solve(models.from_workload(w, store), w.t0, w.t1, w.y0, w.rtol, w.atol, variant)
        n_gpu, n_ref = stats[k].n_accepted + stats[k].n_rejected, ref.n_accepted + ref.n_rejected
        assert stats[k].status == 0 and stats[k].t_reached == w.t1
        assert abs(n_gpu - n_ref) <= max(2, 0.05 * n_ref), (k, w.N, n_gpu, n_ref)
        assert metrics.normalized_final_error(ref.y, out[k], w.N) < 1e-6, (k, w.N)


def test_ragged_kuramoto_and_single_system_entry_agree():
    bs3 = library()
    systems = [W.kuramoto(n, 20 + n, t1=5.0) for n in (17, 64, 129, 333, 520)]
    out, stats = _batch(systems, "f32", "mixed2", kind="kuramoto")
    for k, w in enumerate(systems):
        s = bs3.System.from_workload(w, "f32")
        rc, st, y, _ = s.solve(w.t0, w.t1, w.y0, w.rtol, w.atol, "mixed2", "float2")
        s.close()
        assert rc == bs3.OK
        assert abs((st.n_accepted + st.n_rejected) - (stats[k].n_accepted + stats[k].n_rejected)) <= 2
        assert metrics.normalized_final_error(y, out[k], w.N) < 1e-6


def test_autotuner_picks_a_valid_plan_and_keeps_results():
    bs3 = library()
    torch = torch_cuda()
    w = W.kuramoto(2048, 8, t1=2.0)
    s = bs3.System.from_workload(w, "bf16")
    y0 = torch.tensor(w.y0, device="cuda")
    rc, y_default, st_default = None, None, None
    rc, st_default = bs3.bs3_solve(s.handle, w.t0, w.t1, y0, 1e-6, 1e-6, bs3.MIXED1, bs3.ACC_FLOAT2, None, 0, None,
                                   yd := torch.empty_like(y0), 0)
    assert rc == bs3.OK
    rc, plan, us = bs3.bs3_autotune(s.handle, y0, w.t0, w.t1, 1e-6, bs3.MIXED1, bs3.ACC_FLOAT2, 20)
    assert rc == bs3.OK and plan[0] in (0, 1) and plan[1] >= 1 and us > 0
    yt = torch.empty_like(y0)
    rc, st = bs3.bs3_solve(s.handle, w.t0, w.t1, y0, 1e-6, 1e-6, bs3.MIXED1, bs3.ACC_FLOAT2, None, 0, None, yt, 0)
    s.close()
    assert rc == bs3.OK
    assert abs((st.n_accepted + st.n_rejected) - (st_default.n_accepted + st_default.n_rejected)) <= 2
    assert metrics.normalized_final_error(yd.cpu().numpy(), yt.cpu().numpy(), w.N) < 1e-6
