"""GPU parity of the stored weights and of one right-hand-side evaluation
(every kind x storage format x precision triple) against the oracle."""

import numpy as np
import pytest

import workloads as W
from oracle import formats, models
from tests.gpu_helpers import decode_store, library, rhs_tolerance, torch_cuda

pytestmark = pytest.mark.gpu

STORES = ["f64", "f32", "bf16", "f16", "fp8e4m3"]
PRECS = [("S", "S", "S"), ("D", "D", "S"), ("D", "D", "D")]
ACCUMS = ["f64", "float2"]


def _workload(kind, N, seed=3):
    if kind == "lco_cfg":
        return W.lco_config(N, seed)
    if kind == "lco_paper":
        return W.lco_paper(N, seed, heterogeneous=True)
    if kind == "kuramoto":
        w = W.kuramoto(N, seed)
        w.y0 = w.y0 + 30.0 * np.random.default_rng(seed).standard_normal(N)
        return w
    return W.circadian(N, seed)


def _gpu_rhs(bs3, torch, sysm, y, prec, accum):
    yd = torch.tensor(y, dtype=torch.float64, device="cuda")
    out = torch.empty_like(yd)
    p = [0 if c == "S" else 1 for c in prec]
    rc = bs3.bs3_rhs(sysm.handle, 0.0, yd, p[0], p[1], p[2], bs3.ACCUM_IDS[accum], out)
    assert rc == bs3.OK, bs3.bs3_status_string(rc)
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("store", STORES)
@pytest.mark.parametrize("N", [1, 37, 1000])
def test_quantised_weights_bit_exact(store, N):
    bs3 = library()
    torch_cuda()
    w = W.circadian(N, 1) if N > 1 else W.circadian(1, 1)
    K = w.coupling.copy()
    if N > 5:
        K[5] = 0.0                                    # an all-zero row
    sysm = bs3.System("circadian", N, w.params, w.globals)
    sysm.set_coupling(K, store)
    q, s = sysm.get_coupling()
    sysm.close()
    q_ref, s_ref = formats.quantize(K, store)
    np.testing.assert_array_equal(s, s_ref)
    np.testing.assert_array_equal(decode_store(q, store), q_ref.astype(np.float64))


@pytest.mark.parametrize("kind", models.KINDS)
@pytest.mark.parametrize("store", STORES)
@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("N,resident", [(37, False), (37, True), (523, True), (523, False)])
def test_rhs_matches_oracle(kind, store, prec, N, resident):
    bs3 = library()
    torch = torch_cuda()
    w = _workload(kind, N)
    sysm = bs3.System.from_workload(w, store, resident=resident)
    osys = models.from_workload(w, store)
    for accum in (ACCUMS if prec == ("D", "D", "S") else ["float2"]):
        got = _gpu_rhs(bs3, torch, sysm, w.y0, prec, accum)
        y_in = w.y0.astype(np.float32) if prec == ("S", "S", "S") else w.y0
        ref = models.rhs(osys, 0.0, y_in, prec).astype(np.float64)
        tol = rhs_tolerance(osys, w.y0, prec, accum)
        bad = np.abs(got - ref) > tol
        assert not bad.any(), (accum, np.flatnonzero(bad)[:5], got[bad][:5], ref[bad][:5], tol[bad][:5])
    sysm.close()


@pytest.mark.parametrize("kind", ["kuramoto", "circadian"])
@pytest.mark.parametrize("store", ["f32", "bf16"])
def test_biased_float_float_sums_with_uneven_rows(kind, store):
    """The packed float-float sums start from the largest bias of a CTA's rows:
    a row 1000x heavier than its neighbours loosens their bias, an all-zero
    row has none of its own; both stay within the stated bound."""
    bs3 = library()
    torch = torch_cuda()
    N = 523
    w = _workload(kind, N)
    K = np.array(w.coupling, dtype=np.float64, copy=True)
    K[17] *= 1000.0
    K[18] = 0.0
    K[300] *= 1e-3
    w.coupling = K.astype(w.coupling.dtype)
    prec = ("D", "D", "S")
    sysm = bs3.System.from_workload(w, store)
    osys = models.from_workload(w, store)
    got = _gpu_rhs(bs3, torch, sysm, w.y0, prec, "float2")
    ref = models.rhs(osys, 0.0, w.y0, prec).astype(np.float64)
    tol = rhs_tolerance(osys, w.y0, prec, "float2")
    bad = np.abs(got - ref) > tol
    assert not bad.any(), (np.flatnonzero(bad)[:5], got[bad][:5], ref[bad][:5], tol[bad][:5])
    sysm.close()


def test_permutation_weights_give_exact_gather():
    """A permutation matrix turns the coupling into a gather: exact in every format."""
    bs3 = library()
    torch = torch_cuda()
    N = 301
    rng = np.random.default_rng(9)
    perm = rng.permutation(N)
    P = np.zeros((N, N))
    P[np.arange(N), perm] = 1.0
    y = np.concatenate([rng.standard_normal(N), np.zeros(N)])
    for store in STORES:
        sysm = bs3.System("lco_cfg", N, np.zeros(N))
        sysm.set_coupling(P, store)
        got = _gpu_rhs(bs3, torch, sysm, y, ("D", "D", "D"), "float2")
        sysm.close()
        # one product per row: q_ij x_j is exact, then one rounding by the row scale
        # (a power of two except for fp8, whose scale is fp32(1/448))
        osys = models.make_system("lco_cfg", N, np.zeros(N), P, store)
        ref = models.rhs(osys, 0.0, y, ("D", "D", "D"))
        np.testing.assert_array_equal(got[N:], ref[N:])
        if store != "fp8e4m3":
            np.testing.assert_array_equal(got[N:], y[:N][perm])


@pytest.mark.parametrize("kind,N,store", [("kuramoto", 4096, "bf16"), ("kuramoto", 4096, "f32"),
                                          ("circadian", 16384, "bf16"), ("circadian", 16384, "fp8e4m3")])
def test_full_size_sampled_rows(kind, N, store):
    """Full-size workloads in the launch configuration of the benchmark: 64
    sampled agents evaluated by the oracle one by one."""
    bs3 = library()
    torch = torch_cuda()
    w = W.kuramoto(N, 0) if kind == "kuramoto" else W.circadian(N, 0)
    sysm = bs3.System.from_workload(w, store)
    osys = models.from_workload(w, store)
    rows = np.sort(np.random.default_rng(1).choice(N, 64, replace=False))
    rows[-1] = N - 1
    for prec in (("S", "S", "S"), ("D", "D", "S")):
        got = _gpu_rhs(bs3, torch, sysm, w.y0, prec, "float2").reshape(osys.d, N)[:, rows]
        y_in = w.y0.astype(np.float32) if prec == ("S", "S", "S") else w.y0
        ref = models.rhs(osys, 0.0, y_in, prec, rows=rows)
        tol = rhs_tolerance(osys, w.y0, prec).reshape(osys.d, N)[:, rows]
        assert np.all(np.abs(got - ref) <= tol), prec
    sysm.close()


def test_binary32_sine_cosine_of_binary64_phases_are_rounded_without_bias():
    """The G = S j-vector holds the binary32 sine and cosine of a binary64
    phase (Table MP-Distrib: G in S).  Read back exactly through a
    permutation coupling (row agents at phase 0 or 3 pi/2 gather one phase
    each, Sigma = D), they equal the correctly rounded values in at least 97 %
    of cases and are never more than one ulp away; over 16384 phases their mean
    error is below 0.01 ulp (the rounding noise alone gives a standard error of
    0.0023 ulp), so that oscillators with nearly equal phases do not share a
    systematic error."""
    bs3 = library()
    torch = torch_cuda()
    M = 4096
    N = 2 * M
    P = np.zeros((N, N), dtype=np.float32)
    P[np.arange(M), M + np.arange(M)] = 1.0
    P[M + np.arange(M), np.arange(M)] = 1.0
    for which, row_phase in (("sin", 0.0), ("cos", 1.5 * np.pi)):
        sysm = bs3.System("kuramoto", N, np.zeros(N))
        sysm.set_coupling(P, "f32")
        errs, diffs = [], []
        for seed in range(4):
            theta = np.random.default_rng(seed).uniform(0.0, 2 * np.pi * 50, M)
            y = torch.tensor(np.concatenate([np.full(M, row_phase), theta]), device="cuda")
            out = torch.empty_like(y)
            assert bs3.bs3_rhs(sysm.handle, 0.0, y.data_ptr(), 1, 1, 0, bs3.ACC_F64, out.data_ptr()) == bs3.OK
            got = out.cpu().numpy()[:M]
            exact = np.sin(theta) if which == "sin" else np.cos(theta)
            # (cos(3 pi / 2) in binary64 is -1.8e-16, not 0: the gathered sine leaks in at that size)
            rounded = exact.astype(np.float32).astype(np.float64)
            ulp = np.spacing(np.abs(rounded).astype(np.float32)).astype(np.float64)
            diffs.append(np.rint((got - rounded) / ulp))
            errs.append((got - exact) / ulp)
        sysm.close()
        d, e = np.concatenate(diffs), np.concatenate(errs)
        assert np.max(np.abs(d)) <= 1, which
        assert np.mean(d != 0) <= 0.03, (which, np.mean(d != 0))
        assert abs(np.mean(e)) < 0.01, (which, np.mean(e))
