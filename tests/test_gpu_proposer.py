"""Learned step-size proposer on the GPU: gradients of the training kernel
against the oracle's backprop, training, solve parity with the proposer
installed, and what the trained proposer gains over the plain controller."""

import numpy as np
import pytest

import workloads as W
from oracle import bs3 as obs3
from oracle import metrics, mlp, models
from tests.gpu_helpers import library, torch_cuda

pytestmark = pytest.mark.gpu


def test_training_gradient_matches_oracle():
    bs3 = library()
    rng = np.random.default_rng(5)
    p = (mlp.init_params(2) + 0.05 * rng.standard_normal(mlp.N_PARAMS)).astype(np.float32)
    X = rng.standard_normal((1000, 6)).astype(np.float32)
    y = rng.standard_normal(1000).astype(np.float32)
    rc, loss, g = bs3.bs3_mlp_grad(p, X, y)
    assert rc == bs3.OK
    loss_ref, g_ref = mlp.loss_and_grad(p.astype(np.float64), X.astype(np.float64), y.astype(np.float64))
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    assert np.max(np.abs(g - g_ref)) <= 1e-4 * np.max(np.abs(g_ref)) + 1e-7


def test_training_fits_a_smooth_target():
    bs3 = library()
    from paper_2605_23727_gb300 import proposer
    rng = np.random.default_rng(6)
    X = rng.standard_normal((4000, 6)).astype(np.float32)
    y = (0.3 * np.tanh(X[:, 0]) - 0.2 * X[:, 4] + 0.1 * X[:, 1] * X[:, 2]).astype(np.float32)
    model, loss = proposer.train(X, y, epochs=150, batch=256, lr=3e-3)
    assert loss[-1] < 0.02 * loss[0]
    Xs = (X - model[1313:1319]) / model[1319:1325]
    pred = mlp.forward(model[:1313].astype(np.float64), Xs.astype(np.float64))
    assert np.sqrt(np.mean((pred - y) ** 2)) < 0.05


def _trained_model():
    from paper_2605_23727_gb300 import proposer
    train_set = []
    for seed in (101, 102, 103):
        for rtol in (1e-4, 1e-5, 1e-6, 1e-7):
            train_set.append((W.lco_config(256, seed), "f64", "double", rtol))
    train_set.append((W.kuramoto(1024, 101, t1=50.0), "f32", "mixed2", 1e-6))
    train_set.append((W.circadian(256, 101, t1=240.0), "f32", "mixed2", 1e-6))
    X, y = proposer.dataset(train_set)
    model, loss = proposer.train(X, y, epochs=120, batch=256, lr=2e-3)
    return model


@pytest.fixture(scope="module")
def model():
    library()
    torch_cuda()
    return _trained_model()


def test_solve_with_proposer_matches_oracle(model):
    bs3 = library()
    w = W.lco_config(256, 0)
    sysm = bs3.System.from_workload(w, "f64")
    assert bs3.bs3_set_proposer(sysm.handle, model) == bs3.OK
    rc, st, y, _ = sysm.solve(w.t0, w.t1, w.y0, w.rtol, w.atol, "double", "float2")
    sysm.close()
    assert rc == bs3.OK
    osys = models.from_workload(w, "f64")
    ref = obs3.solve(osys, w.t0, w.t1, w.y0, w.rtol, w.atol, "double",
                     proposer=mlp.Proposer(model[:1313], model[1313:1319], model[1319:1325]))
    n_gpu, n_ref = st.n_accepted + st.n_rejected, ref.n_accepted + ref.n_rejected
    assert abs(n_gpu - n_ref) <= max(3, 0.05 * n_ref), (n_gpu, n_ref)
    assert metrics.normalized_final_error(ref.y, y, w.N) < 1e-5


def test_trained_proposer_gains_over_plain_controller(model):
    """Second-order oscillators N = 4096, f16 weights, Mixed1, rtol 1e-6 (evaluation
    seed distinct from the training seeds): fewer attempts and RHS evaluations,
    comparable global error against a tight binary64 solve."""
    bs3 = library()
    w = W.lco_config(4096, 7, dtype=np.float32)
    ref_sys = bs3.System.from_workload(w, "f64")
    rc, _, y_ref, _ = ref_sys.solve(w.t0, w.t1, w.y0, 1e-11, 1e-11, "double", "float2")
    ref_sys.close()
    assert rc == bs3.OK
    s = bs3.System.from_workload(w, "f16")
    rc, plain, y_plain, _ = s.solve(w.t0, w.t1, w.y0, 1e-6, 1e-6, "mixed1", "float2")
    assert bs3.bs3_set_proposer(s.handle, model) == bs3.OK
    rc2, learned, y_learned, _ = s.solve(w.t0, w.t1, w.y0, 1e-6, 1e-6, "mixed1", "float2")
    s.close()
    assert rc == rc2 == bs3.OK
    e_plain = metrics.normalized_final_error(y_ref, y_plain, w.N)
    e_learned = metrics.normalized_final_error(y_ref, y_learned, w.N)
    print(f"plain {plain.n_accepted}+{plain.n_rejected} evals {plain.n_rhs_evals} err {e_plain:.3e}; "
          f"learned {learned.n_accepted}+{learned.n_rejected} evals {learned.n_rhs_evals} err {e_learned:.3e}")
    assert learned.n_rhs_evals < plain.n_rhs_evals
    assert e_learned < 3.0 * e_plain
