#!/usr/bin/env python
"""Benchmark: time-to-solution of the mixed-precision BS3 solve at a fixed
global error, against the binary64 GPU path, on Kuramoto N = 4096,
K_ij = (2/N)(1 + U(-1/2, 1/2)), omega ~ N(0,1), theta0 ~ U(0, 2 pi),
t in [0, 50] (seeded synthetic data; the paper's Sobol test suites are not
available).

A step is one complete adaptive solve (every attempt: three coupling
evaluations, stage combinations, the embedded error norm and the controller)
inside one persistent kernel.  Inputs are resident in HBM; the L2 is flushed
between timed steps (a 512 MiB write, then a 512 MiB read of another buffer)
outside the timed events.

Default run: N = 1 GPU.  Under torchrun each rank solves an independent replica
(other seed); the reported time is the maximum over ranks ("replicas only").
``--impl reference`` times the CPU oracle instead (bounded sample, extrapolated).
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

N_AGENTS = 4096
T1 = 50.0
RTOL = 1e-6
ERROR_FACTOR = 2.0          # "fixed global error": within this factor of the binary64 GPU path
# The headline configuration, the same for the GPU arm and the CPU reference
# arm: the paper's Mixed1 with binary32 weights, its Sigma = D stage summed by
# the compensated float-float accumulator (the literal binary64 sum is timed
# beside it).  The survey below checks that its global error stays within
# ERROR_FACTOR of the binary64 path's and that it is the fastest mixed variant
# that does.
HEADLINE = ("mixed1", "f32")
ORACLE_SOLVE_FILE = os.path.join(ROOT, "tests", "golden", "oracle_solve_kuramoto_N4096_mixed1_f32.json")
METRIC = "time-to-solution at fixed global error, mixed vs FP64 GPU; coupling HBM GB/s"
WORKLOAD = "kuramoto_N4096_t50"
REF_FILE = os.path.join(ROOT, "tests", "golden", "ref_kuramoto_N4096_seed0_t50.npy")
STORE_BYTES = {"f64": 8, "f32": 4, "bf16": 2, "f16": 2, "fp8e4m3": 1}
# (variant, stored weights) surveyed; the headline is the fastest of the paper's
# mixed variants (Mixed1, Mixed2) whose global error stays within ERROR_FACTOR
# of the binary64 path.
CANDIDATES = [("double", "f64"), ("mixed2", "f32"), ("mixed1", "f32"), ("mixed2", "bf16"),
              ("mixed1", "bf16"), ("mixed1", "f16"), ("single", "f32")]


# Single-solve cases for profiler captures (one persistent-kernel launch each):
# name -> (workload builder, variant, stored weights)
CASES = {
    "kuramoto4096_mixed1_f32": (lambda: workloads.kuramoto(4096, 0, t1=T1, rtol=RTOL), "mixed1", "f32"),
    "kuramoto4096_mixed1_bf16": (lambda: workloads.kuramoto(4096, 0, t1=T1, rtol=RTOL), "mixed1", "bf16"),
    "kuramoto4096_double_f64": (lambda: workloads.kuramoto(4096, 0, t1=5.0, rtol=RTOL), "double", "f64"),
    "kuramoto4096_mixed2_f32": (lambda: workloads.kuramoto(4096, 0, t1=T1, rtol=RTOL), "mixed2", "f32"),
    "lco16384_mixed1_f16": (lambda: workloads.lco_config(16384, 0, t1=0.5, rtol=RTOL), "mixed1", "f16"),
    "lco32768_mixed1_f16": (lambda: workloads.lco_config(32768, 0, t1=0.2, rtol=RTOL), "mixed1", "f16"),
    "circadian16384_mixed1_bf16": (lambda: workloads.circadian(16384, 0, t1=0.5, rtol=RTOL), "mixed1", "bf16"),
    "circadian16384_mixed1_fp8": (lambda: workloads.circadian(16384, 0, t1=0.5, rtol=RTOL), "mixed1", "fp8e4m3"),
    "ensemble256_kuramoto8192": None,
    "ensemble128_kuramoto1024": None,
    "ensemble128_kuramoto8192": None,
    "ragged1000_lco_mixed1_f16": None,
    "batch_config4": None,
    "ragged_skewed_lco_f16": None,
    "proposer_lco32768_f16": None,
    "proposer_lco8192_f16": None,
    "phases_kuramoto4096_mixed1_f32": None,
    "sweep_kuramoto4096": None,
    "beta_gamma_suite": None,
    "size_vs_error": None,
}

# FP32 instructions per pair of the circadian coupling (own arctangent): the
# difference, reciprocal (above 1) with its selects, z = t*t, 8 polynomial FMAs,
# the product t*P, the pi/2 fold and sign, and the FMA with the weight.
CC_OPS_PER_PAIR = 15
# binary32 lanes per SM and the maximum SM clock of GB300 (nominal ALU peak)
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def run_ensemble_case(name):
    """Shared-K ensemble on the tensor cores: T Kuramoto trajectories, one K."""
    import torch
    from paper_2605_23727_gb300 import bs3
    import __graft_entry__
    __graft_entry__.build()
    bs3.load()
    T, N, t1 = {"ensemble256_kuramoto8192": (256, 8192, T1), "ensemble128_kuramoto8192": (128, 8192, T1),
                "ensemble128_kuramoto1024": (128, 1024, 10.0)}[name]
    K, omega, theta0 = workloads.kuramoto_ensemble(T=T, N=N, seed=0)
    Kd = torch.tensor(K, dtype=torch.float32, device="cuda")
    om = torch.tensor(omega, dtype=torch.float64, device="cuda")
    th = torch.tensor(theta0, dtype=torch.float64, device="cuda")
    out = torch.empty_like(th)
    # tile width by the autotuner (bounded solves of each width)
    rc, tile, us_tile = bs3.bs3_ensemble_autotune(Kd, N, T, om, th, 0.0, t1, RTOL, RTOL, 16, out)
    if rc != bs3.OK:
        raise RuntimeError(bs3.bs3_status_string(rc))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record()
    rc, n_acc, n_rej, status, steps = bs3.bs3_ensemble_solve(Kd, N, T, om, th, 0.0, t1, RTOL, RTOL, out,
                                                             tile_n=tile)
    e1.record()
    e1.synchronize()
    ms = e0.elapsed_time(e1)
    flops = 3 * 3 * 2.0 * N * N * (2 * T) * steps     # 3 stages x 3 split products per lock-step attempt
    print(json.dumps({"case": name, "status": bs3.bs3_status_string(rc), "ms": ms, "T": T, "N": N,
                      "lockstep_attempts": steps, "attempts_max": int((n_acc + n_rej).max()),
                      "attempts_mean": float((n_acc + n_rej).mean()), "all_ok": bool((status == 0).all()),
                      "tensor_tflops": flops / (ms * 1e-3) / 1e12, "tile_n": tile,
                      "autotune_us_per_attempt": us_tile,
                      "ms_per_trajectory": ms / T}))
    if rc != bs3.OK:
        sys.exit(1)


def run_ragged_case(name):
    """1000 independent second-order oscillator systems, N log-uniform in
    [64, 4096], f16 weights, Mixed1, rtol 1e-6, t in [0, 10], one launch."""
    from paper_2605_23727_gb300 import bs3
    import __graft_entry__
    __graft_entry__.build()
    bs3.load()
    count = 1000
    systems = workloads.lco_ragged_batch(count=count, n_min=64, n_max=4096, seed=0, t1=10.0, rtol=RTOL)
    Ns = [w.N for w in systems]
    K = np.concatenate([np.asarray(w.coupling, dtype=np.float32).ravel() for w in systems])
    params = np.concatenate([w.params for w in systems])
    y0 = np.concatenate([w.y0 for w in systems])
    t0 = np.zeros(count)
    t1 = np.full(count, 10.0)
    for _ in range(2):     # the first launch pays the one-time set-up
        rc, yf, stats, kms = bs3.bs3_batch_solve(bs3.LCO_CFG, Ns, params, K, bs3.F16, y0, t0, t1, RTOL, RTOL,
                                                 bs3.MIXED1, bs3.ACC_FLOAT2)
    evals = np.array([st.n_rhs_evals for st in stats], dtype=np.float64)
    nn = np.array(Ns, dtype=np.float64)
    weight_bytes = float(np.sum(evals * nn * nn * 2))
    print(json.dumps({"case": name, "status": bs3.bs3_status_string(rc), "systems": count,
                      "sum_N2": float(np.sum(nn * nn)), "kernel_ms": kms,
                      "attempts_total": int(sum(st.n_accepted + st.n_rejected for st in stats)),
                      "weight_GBs": weight_bytes / (kms * 1e-3) / 1e9, "all_ok": all(st.status == 0 for st in stats)}))
    if rc != bs3.OK:
        sys.exit(1)


def run_batch_config4_case(name):
    """The shared-K batch configuration in one bs3_solve_batch call: 256
    Kuramoto trajectories at N = 8192 sharing one K (t in [0, 50], rtol 1e-6,
    the tensor-core group) beside 1000 second-order oscillator systems with N
    log-uniform in [64, 4096] (binary16 weights, Mixed1, t in [0, 10], rtol
    1e-6).  The one call is timed beside the same two parts submitted alone."""
    import torch
    from paper_2605_23727_gb300 import bs3
    import __graft_entry__
    __graft_entry__.build()
    bs3.load()
    systems = workloads.lco_ragged_batch(count=1000, n_min=64, n_max=4096, seed=0, t1=10.0, rtol=RTOL)
    handles, items = [], []
    for w in systems:
        sy = bs3.System.from_workload(w, "f16")
        handles.append(sy)
        y0 = torch.tensor(w.y0, device="cuda")
        items.append({"sys": sy.handle, "y0": y0, "y_final": torch.empty_like(y0), "t0": w.t0, "t1": w.t1,
                      "rtol": RTOL, "atol": RTOL})
    T, N = 256, 8192
    K, omega, theta0 = workloads.kuramoto_ensemble(T=T, N=N, seed=0)
    g = {"K": torch.tensor(K, device="cuda"), "N": N, "T": T, "omega": torch.tensor(omega, device="cuda"),
         "theta0": torch.tensor(theta0, device="cuda"), "t0": 0.0, "t1": T1, "rtol": RTOL, "atol": RTOL,
         "n_acc": np.zeros(T, dtype=np.int64), "n_rej": np.zeros(T, dtype=np.int64),
         "status": np.zeros(T, dtype=np.int32)}
    g["theta_out"] = torch.empty_like(g["theta0"])
    out = {"case": name}
    for tag, its, grp, ctas in (("items_alone", items, None, 0), ("group_alone", [], g, 0),
                                ("one_call", items, g, 0), ("one_call_side_by_side_48", items, g, 48)):
        if grp is not None:
            grp["ctas"] = ctas
        for _ in range(2):          # the first call pays the one-time set-up
            rc, stats, steps, ms = bs3.bs3_solve_batch(its, bs3.MIXED1, bs3.ACC_FLOAT2, 0, grp)
        rec = {"status": bs3.bs3_status_string(rc), "ms": round(ms, 2)}
        if its:
            evals = np.array([st.n_rhs_evals for st in stats], dtype=np.float64)
            nn = np.array([w.N for w in systems], dtype=np.float64)
            rec["items_attempts"] = int(sum(st.n_accepted + st.n_rejected for st in stats))
            rec["items_weight_GBs"] = round(float(np.sum(evals * nn * nn * 2)) / (ms * 1e-3) / 1e9, 1)
            rec["items_all_ok"] = all(st.status == 0 for st in stats)
        if grp is not None:
            flops = 9 * 2.0 * N * N * (2 * T) * steps
            rec["group_lockstep_attempts"] = int(steps)
            rec["group_tensor_TFLOPs"] = round(flops / (ms * 1e-3) / 1e12, 1)
            rec["group_all_ok"] = bool(np.all(g["status"] == 0))
        out[tag] = rec
    out["one_call_vs_sum_of_parts"] = round(out["one_call"]["ms"] / (out["items_alone"]["ms"] +
                                                                     out["group_alone"]["ms"]), 3)
    for h in handles:
        h.close()
    print(json.dumps(out))


def run_skewed_case(name):
    """A skewed ragged batch: one second-order oscillator system of N=8192
    among 200 of N=256 (f16, Mixed1, t in [0, 2]).  The large system is
    solved by a team of CTAs; its solve alone through bs3_solve (the whole
    GPU) is timed beside the batch."""
    import torch
    from paper_2605_23727_gb300 import bs3
    import __graft_entry__
    __graft_entry__.build()
    bs3.load()
    systems = [workloads.lco_config(8192, 1, t1=2.0, rtol=RTOL)] + \
        [workloads.lco_config(256, 2 + k, t1=2.0, rtol=RTOL) for k in range(200)]
    Ns = [w.N for w in systems]
    K = np.concatenate([np.asarray(w.coupling, dtype=np.float32).ravel() for w in systems])
    params = np.concatenate([w.params for w in systems])
    y0 = np.concatenate([w.y0 for w in systems])
    S = len(systems)
    args = (bs3.LCO_CFG, Ns, params, K, bs3.F16, y0, np.zeros(S), np.full(S, 2.0), RTOL, RTOL, bs3.MIXED1,
            bs3.ACC_FLOAT2)
    bs3.bs3_batch_solve(*args)
    rc, yf, stats, kms = bs3.bs3_batch_solve(*args)
    big = systems[0]
    s = bs3.System.from_workload(big, "f16")
    y0d = torch.tensor(big.y0, device="cuda")
    yo = torch.empty_like(y0d)
    for _ in range(2):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        rc2, st = bs3.bs3_solve(s.handle, big.t0, big.t1, y0d, RTOL, RTOL, bs3.MIXED1, bs3.ACC_FLOAT2, None, 0,
                                None, yo, 0)
        e1.record()
        e1.synchronize()
    s.close()
    print(json.dumps({"case": name, "status": bs3.bs3_status_string(rc), "batch_kernel_ms": kms,
                      "big_alone_ms": e0.elapsed_time(e1), "big_attempts_in_batch": stats[0].n_accepted +
                      stats[0].n_rejected, "big_attempts_alone": st.n_accepted + st.n_rejected,
                      "big_max_abs_diff": float(np.max(np.abs(yf[:2 * 8192] - yo.cpu().numpy())))}))


def run_beta_case(name):
    """The paper's performance parameters (Sec. 2.5, Eq. Beta-2MP and
    Gamma-2MP) measured on the GPU over a seeded synthetic test suite:
    beta = steps of Double / steps of the mixed solver (accepted + rejected),
    gamma = time per step of the mixed solver / of Double, Gamma = gamma / beta
    = time ratio.  Benchmarks: Benchmark 1 (paper form, heterogeneous M),
    Kuramoto, circadian; N in {256, 1024}; rtol = atol in {1e-4, 1e-6, 1e-8};
    seeds 0..3.  Double stores binary64 weights, the other solvers binary32
    (G = S).  Statistics over the tests every solver finished, as in Table
    Beta-values: (min, 1st quartile, median, 3rd quartile, max)."""
    import torch
    from paper_2605_23727_gb300 import bs3
    import __graft_entry__
    __graft_entry__.build()
    bs3.load()
    makers = {
        "LCO": lambda N, seed: workloads.lco_paper(N, seed, heterogeneous=True),
        "Kur": lambda N, seed: workloads.kuramoto(N, seed, t1=10.0),
        "CC": lambda N, seed: workloads.circadian(N, seed, t1=48.0),
    }
    solvers = (("single", "f32"), ("mixed1", "f32"), ("mixed2", "f32"), ("double", "f64"))
    tests = []
    for bench_name, make in makers.items():
        for N in (256, 1024):
            for seed in range(4):
                w = make(N, seed)
                systems = {store: bs3.System.from_workload(w, store) for store in ("f32", "f64")}
                y0 = torch.tensor(w.y0, device="cuda")
                yo = torch.empty_like(y0)
                for rt in (1e-4, 1e-6, 1e-8):
                    rec = {"benchmark": bench_name, "N": N, "seed": seed, "rtol": rt}
                    for variant, store in solvers:
                        best, st, rc = None, None, None
                        for _ in range(2):
                            e0 = torch.cuda.Event(enable_timing=True)
                            e1 = torch.cuda.Event(enable_timing=True)
                            e0.record()
                            rc, st = bs3.bs3_solve(systems[store].handle, w.t0, w.t1, y0, rt, rt,
                                                   bs3.VARIANT_IDS[variant], bs3.ACC_FLOAT2, None, 0, None, yo, 0)
                            e1.record()
                            e1.synchronize()
                            ms = e0.elapsed_time(e1)
                            best = ms if best is None else min(best, ms)
                        rec[variant] = {"ok": rc == bs3.OK, "steps": st.n_accepted + st.n_rejected, "ms": best}
                    tests.append(rec)
                    print(json.dumps(rec), flush=True)
                for sy in systems.values():
                    sy.close()

    def quant(v):
        q = np.quantile(np.asarray(v), [0.0, 0.25, 0.5, 0.75, 1.0])
        return [round(float(x), 3) for x in q]

    summary = {}
    for bench_name in makers:
        done = [t for t in tests if t["benchmark"] == bench_name and all(t[v]["ok"] for v, _ in solvers)]
        row = {"tests_finished_by_all": len(done)}
        for variant, _ in solvers[:3]:
            beta = [t["double"]["steps"] / t[variant]["steps"] for t in done]
            gamma = [(t[variant]["ms"] / t[variant]["steps"]) / (t["double"]["ms"] / t["double"]["steps"])
                     for t in done]
            Gam = [t[variant]["ms"] / t["double"]["ms"] for t in done]
            row[variant] = {"beta": quant(beta), "gamma": quant(gamma), "Gamma": quant(Gam),
                            "Gamma_below_1": sum(g < 1.0 for g in Gam)}
        summary[bench_name] = row
    print(json.dumps({"case": name, "paper_naive_gamma": {"single": 0.5, "mixed1": 0.583, "mixed2": 0.75},
                      "summary": summary}))


def proposer_comparison(N=32768):
    """Second-order oscillators (f16 weights, Mixed1, t in [0, 10]) with and
    without the learned step-size proposer, trained on the GPU on step
    histories of the three smaller workloads (other seeds).  Both at rtol 1e-6;
    the proposer also at 5e-7, so that its time at the plain controller's
    global error is interpolated (log-log) along its own curve.  Global errors
    against a tight solve with the same weights (Mixed2, rtol 1e-9)."""
    import torch
    from paper_2605_23727_gb300 import bs3, proposer
    train = []
    for seed in (101, 102, 103):
        for rtol in (1e-4, 1e-5, 1e-6, 1e-7):
            train.append((workloads.lco_config(256, seed), "f64", "double", rtol))
    train.append((workloads.kuramoto(1024, 101, t1=50.0), "f32", "mixed2", 1e-6))
    train.append((workloads.circadian(256, 101, t1=240.0), "f32", "mixed2", 1e-6))
    X, y = proposer.dataset(train)
    model, loss = proposer.train(X, y, epochs=120, batch=256, lr=2e-3)
    w = workloads.lco_config(N, 7, t1=10.0, dtype=np.float32)
    s = bs3.System.from_workload(w, "f16")
    y0 = torch.tensor(w.y0, device="cuda")

    def run(rtol, variant):
        yo = torch.empty_like(y0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        rc, st = bs3.bs3_solve(s.handle, w.t0, w.t1, y0, rtol, rtol, bs3.VARIANT_IDS[variant], bs3.ACC_FLOAT2,
                               None, 0, None, yo, 0)
        e1.record()
        e1.synchronize()
        if rc != bs3.OK:
            raise RuntimeError(bs3.bs3_status_string(rc))
        return yo.cpu().numpy(), st, e0.elapsed_time(e1)

    y_ref, _, _ = run(1e-9, "mixed2")     # same f16 weights, tight tolerance
    run(RTOL, "mixed1")
    y_plain, st_plain, ms_plain = run(RTOL, "mixed1")
    if bs3.bs3_set_proposer(s.handle, model) != bs3.OK:
        raise RuntimeError("bs3_set_proposer")
    run(RTOL, "mixed1")
    y_learn, st_learn, ms_learn = run(RTOL, "mixed1")
    y_learn2, st_learn2, ms_learn2 = run(5e-7, "mixed1")
    s.close()
    out = {"workload": f"lco_cfg_N{N}_f16_mixed1_t10", "training_samples": int(len(y)),
           "final_train_loss": float(loss[-1])}
    for tag, yv, st, ms, rt in (("plain", y_plain, st_plain, ms_plain, RTOL),
                                ("learned", y_learn, st_learn, ms_learn, RTOL),
                                ("learned_rtol5e-7", y_learn2, st_learn2, ms_learn2, 5e-7)):
        out[tag] = {"rtol": rt, "accepted": st.n_accepted, "rejected": st.n_rejected, "rhs_evals": st.n_rhs_evals,
                    "ms": round(ms, 3), "global_error_vs_tight": normalized_error(y_ref, yv, N)}
    e_plain = out["plain"]["global_error_vs_tight"]
    t_match = time_at([(out["learned"]["global_error_vs_tight"], ms_learn),
                       (out["learned_rtol5e-7"]["global_error_vs_tight"], ms_learn2)], e_plain)
    out["learned_ms_at_plain_error"] = None if t_match is None else round(t_match, 3)
    out["speedup_at_matched_error"] = None if t_match is None else round(ms_plain / t_match, 4)
    return out


def run_size_case(name):
    """Normalized final error against system size at fixed tolerance (Sec. 3.3,
    Fig. Size-VS-Error) on the seeded synthetic benchmarks: Benchmark 1 (paper
    form, heterogeneous M, t in [0, 10 pi]), Kuramoto (t in [0, 10]) and the
    circadian model (t in [0, 48]), N in {256, 1024, 4096}, rtol = atol in
    {1e-3, 1e-6, 1e-8}, seeds 0..2, the four solvers (binary32 weights, Double
    binary64).  The reference is the GPU's binary64 solve at rtol = atol =
    1e-11 of the same system (CPU DOPRI5 at these sizes takes hours; the
    GPU Double path is validated against the oracle by the parity tests).
    Per (benchmark, N, rtol, solver): the errors' (min, median, max)."""
    import torch
    from paper_2605_23727_gb300 import bs3
    import __graft_entry__
    __graft_entry__.build()
    bs3.load()
    makers = {
        "LCO": lambda N, seed: workloads.lco_paper(N, seed, heterogeneous=True),
        "Kur": lambda N, seed: workloads.kuramoto(N, seed, t1=10.0),
        "CC": lambda N, seed: workloads.circadian(N, seed, t1=48.0),
    }
    solvers = (("single", "f32"), ("mixed1", "f32"), ("mixed2", "f32"), ("double", "f64"))
    rows = []
    for bench_name, make in makers.items():
        for N in (256, 1024, 4096):
            errs = {}
            for seed in range(3):
                w = make(N, seed)
                systems = {st: bs3.System.from_workload(w, st) for st in ("f32", "f64")}
                y0 = torch.tensor(w.y0, device="cuda")
                yo = torch.empty_like(y0)
                rc, _ = bs3.bs3_solve(systems["f64"].handle, w.t0, w.t1, y0, 1e-11, 1e-11, bs3.DOUBLE,
                                      bs3.ACC_FLOAT2, None, 0, None, yo, 0)
                if rc != bs3.OK:
                    continue
                y_ref = yo.cpu().numpy()
                for rt in (1e-3, 1e-6, 1e-8):
                    for variant, store in solvers:
                        rc, _ = bs3.bs3_solve(systems[store].handle, w.t0, w.t1, y0, rt, rt,
                                              bs3.VARIANT_IDS[variant], bs3.ACC_FLOAT2, None, 0, None, yo, 0)
                        if rc == bs3.OK:
                            errs.setdefault((rt, variant), []).append(normalized_error(y_ref, yo.cpu().numpy(), N))
                for sy in systems.values():
                    sy.close()
            for (rt, variant), v in sorted(errs.items()):
                rec = {"benchmark": bench_name, "N": N, "rtol": rt, "solver": variant, "tests": len(v),
                       "error_min": min(v), "error_median": float(np.median(v)), "error_max": max(v)}
                rows.append(rec)
                print(json.dumps(rec), flush=True)
    print(json.dumps({"case": name, "reference": "GPU binary64 solve at rtol=atol=1e-11 (GPU-derived)",
                      "rows": rows}))


def run_proposer_case(name):
    from paper_2605_23727_gb300 import bs3
    import __graft_entry__
    __graft_entry__.build()
    bs3.load()
    N = 32768 if name == "proposer_lco32768_f16" else 8192
    print(json.dumps(dict({"case": name}, **proposer_comparison(N))))


def run_phases_case(name):
    """Per-phase device time of the attempts of the benchmark solve (Kuramoto
    N=4096, Mixed1, f32 weights), from the library's step records: the time
    from the start of an attempt to the end of each of its four grid barriers
    (A: Y2 j-vector; B2, B3: stages 2, 3; B4: stage 4 and the error norm), and
    the rest (decision and the next attempt's set-up)."""
    import torch
    from paper_2605_23727_gb300 import bs3
    import __graft_entry__
    __graft_entry__.build()
    bs3.load()
    out = {"case": name}
    for N, t1 in ((4096, T1), (256, 5.0)):
        w = workloads.kuramoto(N, 0, t1=t1, rtol=RTOL)
        s = bs3.System.from_workload(w, "f32")
        y0 = torch.tensor(w.y0, device="cuda")
        yo = torch.empty_like(y0)
        cap = 1 << 15
        bs3.bs3_set_history(s.handle, cap)
        for _ in range(2):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            rc, st = bs3.bs3_solve(s.handle, w.t0, w.t1, y0, RTOL, RTOL, bs3.MIXED1, bs3.ACC_FLOAT2, None, 0,
                                   None, yo, 0)
            e1.record()
            e1.synchronize()
        rc2, H = bs3.bs3_get_history(s.handle, cap)
        s.close()
        att = st.n_accepted + st.n_rejected
        per = 1e3 * e0.elapsed_time(e1) / att
        cum = np.median(H[2:, 4:8], axis=0) / 1e3
        ph = np.diff(np.concatenate([[0.0], cum]))
        out[f"N{N}"] = {"status": bs3.bs3_status_string(rc), "attempts": att, "us_per_attempt": per,
                        "us_A_Y2": ph[0], "us_B2": ph[1], "us_B3": ph[2], "us_B4_error": ph[3],
                        "us_decision_and_setup": per - cum[3]}
    print(json.dumps(out))


def run_sweep_case(name):
    """Time-to-solution against global error: every variant x stored format
    over rtol = atol = 1e-3 .. 1e-9 on the benchmark workload (Kuramoto
    N=4096, t in [0, 50]), global error against the oracle's DOPRI5 reference;
    then each mixed variant's time at the global error the binary64 path
    reaches, by log-log interpolation along the variant's own curve."""
    import torch
    from paper_2605_23727_gb300 import bs3
    import __graft_entry__
    __graft_entry__.build()
    bs3.load()
    w = workloads.kuramoto(4096, 0, t1=T1, rtol=RTOL)
    ref = np.load(REF_FILE)
    y0 = torch.tensor(w.y0, device="cuda")
    yo = torch.empty_like(y0)
    rtols = [1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9]
    combos = [("double", "f64", "bs32"), ("mixed2", "f32", "bs32"), ("mixed1", "f32", "bs32"),
              ("single", "f32", "bs32"), ("mixed2", "bf16", "bs32"), ("mixed1", "bf16", "bs32"),
              ("mixed1", "f16", "bs32"), ("double", "f64", "dp54"), ("mixed1", "f32", "dp54"),
              ("mixed2", "f32", "dp54")]
    curves = {}
    for variant, store, method in combos:
        s = bs3.System.from_workload(w, store)
        s.set_method(method)
        pts = []
        for rt in rtols:
            times = []
            for _ in range(2):
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record()
                rc, st = bs3.bs3_solve(s.handle, w.t0, w.t1, y0, rt, rt, bs3.VARIANT_IDS[variant], bs3.ACC_FLOAT2,
                                       None, 0, None, yo, 0)
                e1.record()
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
            err = normalized_error(yo.cpu().numpy(), ref, w.N) if rc == bs3.OK else None
            rec = {"variant": variant, "weights": store, "method": method, "rtol": rt,
                   "status": bs3.bs3_status_string(rc),
                   "ms": min(times), "global_error": err, "accepted": st.n_accepted, "rejected": st.n_rejected,
                   "rhs_evals": st.n_rhs_evals}
            print(json.dumps(rec), flush=True)
            if rc == bs3.OK:
                pts.append((err, min(times)))
        s.close()
        curves[f"{variant}/{store}" + ("" if method == "bs32" else "/dp54")] = pts

    summary = []
    for e_target, t_double in curves["double/f64"]:
        row = {"global_error": e_target, "double_ms": t_double}
        for key, pts in curves.items():
            if key == "double/f64":
                continue
            t = time_at(pts, e_target)
            row[key] = None if t is None else {"ms": t, "speedup_vs_double": t_double / t}
        summary.append(row)
    print(json.dumps({"case": name, "time_at_double_error": summary}))


def time_at(pts, e):
    """Time at global error e by log-log interpolation between the two points
    (error, time) of a curve that bracket e; None when none does."""
    for (e_a, t_a), (e_b, t_b) in zip(pts, pts[1:]):
        lo, hi = min(e_a, e_b), max(e_a, e_b)
        if lo <= e <= hi and e_a != e_b:
            f = (math.log(e) - math.log(e_a)) / (math.log(e_b) - math.log(e_a))
            return math.exp(math.log(t_a) + f * (math.log(t_b) - math.log(t_a)))
    return None


def run_case(name):
    if name.startswith("ensemble"):
        return run_ensemble_case(name)
    if name.startswith("phases"):
        return run_phases_case(name)
    if name.startswith("sweep"):
        return run_sweep_case(name)
    if name.startswith("beta"):
        return run_beta_case(name)
    if name == "size_vs_error":
        return run_size_case(name)
    if name.startswith("ragged_skewed"):
        return run_skewed_case(name)
    if name == "batch_config4":
        return run_batch_config4_case(name)
    if name.startswith("ragged"):
        return run_ragged_case(name)
    if name.startswith("proposer"):
        return run_proposer_case(name)
    import torch
    from paper_2605_23727_gb300 import bs3
    import __graft_entry__
    __graft_entry__.build()
    bs3.load()
    make, variant, store = CASES[name]
    w = make()
    sysm = bs3.System.from_workload(w, store)
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    y = torch.empty_like(y0)
    # the first solve pays the one-time set-up (module load, launch plan,
    # buffers) between its events; the second is timed
    for _ in range(2):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        rc, st = bs3.bs3_solve(sysm.handle, w.t0, w.t1, y0, w.rtol, w.atol, bs3.VARIANT_IDS[variant],
                               bs3.ACC_FLOAT2, None, 0, None, y, 0)
        e1.record()
        e1.synchronize()
    sysm.close()
    ms = e0.elapsed_time(e1)
    out = {"case": name, "status": bs3.bs3_status_string(rc), "ms": ms,
           "accepted": st.n_accepted, "rejected": st.n_rejected, "rhs_evals": st.n_rhs_evals,
           "us_per_attempt": 1e3 * ms / max(1, st.n_accepted + st.n_rejected),
           "N": w.N, "weights": store, "variant": variant,
           "weight_bytes_per_eval": w.N * w.N * STORE_BYTES[store]}
    if w.kind == "circadian":
        # FP32 ALU roofline of the pairwise arctangent coupling
        ops = float(st.n_rhs_evals) * w.N * w.N * CC_OPS_PER_PAIR
        peak = 152 * FP32_LANES_PER_SM * SM_MAX_MHZ * 1e6
        out["alu"] = {"ops_per_pair": CC_OPS_PER_PAIR, "achieved_Tops": ops / (ms * 1e-3) / 1e12,
                      "peak_Tops": peak / 1e12, "frac": ops / (ms * 1e-3) / peak,
                      "peak_basis": "nominal: 152 SMs x 128 binary32 lanes x 2070 MHz"}
    print(json.dumps(out))
    if rc != bs3.OK:
        sys.exit(1)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="bs3", choices=["bs3", "reference"])
    ap.add_argument("--accum", default="float2", choices=["float2", "f64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-sweep", action="store_true", help="skip the accuracy-against-tolerance sweep")
    ap.add_argument("--no-proposer", action="store_true", help="skip the learned-proposer comparison")
    ap.add_argument("--cpu-sample-attempts", type=int, default=100)
    ap.add_argument("--case", default=None, choices=sorted(CASES),
                    help="run one solve of a named case and print its stats (profiling runs)")
    return ap.parse_args()


def max_over_ranks(value, device=None):
    """Maximum of a per-rank number over the process group (the value itself
    when no group is initialised or the group has one rank)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# Sources that decide the code and launch plan of each profiled kernel; a
# capture's DRAM traffic is reported only while these are unchanged.
KERNEL_SOURCES = {
    "solver": ("bs3_device.cuh", "bs3_solver.cuh", "bs3_mlp.cuh", "bs3_api.cu", "gen_inst.py"),
    "ensemble": ("bs3_device.cuh", "bs3_tc.cuh", "bs3_tc_host.h", "bs3_tc.cu", "bs3_ensemble.cu"),
}


def kernel_sha256(which="solver"):
    import hashlib
    csrc = os.path.join(ROOT, "paper_2605_23727_gb300", "csrc")
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[which]:
        h.update(f.encode())
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()


def recorded_traffic(case):
    """DRAM bytes per launch from the committed ncu capture, or None once the
    kernel sources have changed since that capture."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    rec = json.load(open(path)).get(case)
    if not rec or rec.get("sources_sha256") != kernel_sha256(rec.get("sources", "solver")):
        return None
    return rec["dram_bytes_per_launch"]


def normalized_error(a, b, n):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / math.sqrt(n))


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.proc = None
        self.path = tempfile.mktemp(suffix=".csv")
        self.device_index = device_index

    def __enter__(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device_index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        loaded = [s for s in sm if s > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------- GPU arm
def run_gpu(args):
    import torch
    from paper_2605_23727_gb300 import bs3
    import __graft_entry__

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    __graft_entry__.build()
    bs3.load()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    w = workloads.kuramoto(N_AGENTS, seed=rank, t1=T1, rtol=RTOL)
    n = w.N * w.d
    systems = {}

    def system(store):
        if store not in systems:
            s = bs3.System(w.kind, w.N, w.params, None, device=local, stream=stream.cuda_stream)
            s.set_coupling(w.coupling, store)
            systems[store] = s
        return systems[store]

    y0_d = torch.tensor(w.y0, dtype=torch.float64, device=dev)
    y_d = torch.empty_like(y0_d)
    flush_w = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    flush_r = torch.ones(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    class _Flush:
        """Evicts the L2 between steps: writes a 512 MiB buffer, then reads
        another 512 MiB one so that the written lines are back in DRAM (dirty
        lines left in L2 would otherwise crowd the next step's weights out of it
        for the whole step).  Runs outside the timed events."""

        def zero_(self):
            flush_w.zero_()
            torch.sum(flush_r)

    flush = _Flush()

    def solve_dev(variant, store, rtol=RTOL, accum=None):
        s = system(store)
        rc, st = bs3.bs3_solve(s.handle, w.t0, w.t1, y0_d, rtol, rtol, bs3.VARIANT_IDS[variant],
                               bs3.ACCUM_IDS[accum or args.accum], None, 0, None, y_d, 0)
        if rc != bs3.OK:
            raise RuntimeError(f"{variant}/{store}: {bs3.bs3_status_string(rc)}")
        return st

    def timed(variant, store, reps, accum=None):
        times, st = [], None
        for _ in range(reps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = solve_dev(variant, store, accum=accum)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        return times, st, y_d.cpu().numpy()

    # reference solution for the global error
    if rank == 0 and os.path.exists(REF_FILE):
        y_ref, ref_kind = np.load(REF_FILE), "oracle DOPRI5 rtol=atol=1e-12 (binary64 weights)"
    else:
        solve_dev("double", "f64", rtol=1e-11)
        y_ref, ref_kind = y_d.cpu().numpy(), "GPU-derived: binary64 BS3 at rtol=atol=1e-11"

    survey = {}
    for variant, store in CANDIDATES:
        solve_dev(variant, store)              # warm-up of this configuration
        times, st, y = timed(variant, store, 2)
        survey[f"{variant}/{store}"] = {
            "ms": min(times), "accepted": st.n_accepted, "rejected": st.n_rejected,
            "rhs_evals": st.n_rhs_evals, "global_error": normalized_error(y_ref, y, w.N)}
    e_double = survey["double/f64"]["global_error"]
    ok = [(v["ms"], k) for k, v in survey.items()
          if k.startswith("mixed") and v["global_error"] <= ERROR_FACTOR * e_double]
    fastest_ok = min(ok)[1] if ok else None
    h_variant, h_store = HEADLINE
    head = f"{h_variant}/{h_store}"
    # the literal Sigma = D of the headline's stage 4 (each binary32 product
    # cast to binary64, binary64 sum), timed beside the float-float sum
    solve_dev(h_variant, h_store, accum="f64")
    lit_times, lit_st, lit_y = timed(h_variant, h_store, 2, accum="f64")
    sigma_literal = {"accum": "f64", "ms": min(lit_times), "attempts": lit_st.n_accepted + lit_st.n_rejected,
                     "global_error": normalized_error(y_ref, lit_y, w.N)}
    from paper_2605_23727_gb300 import autotune
    plan, plan_us = autotune.tuned(system(h_store), y0_d, w.t0, w.t1, RTOL, h_variant, args.accum,
                                   torch.cuda.get_device_name(dev))

    # ---------------------------------------------------------------- timed
    for _ in range(args.warmup):
        flush.zero_()
        solve_dev(h_variant, h_store)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    step_ms = []
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        for _ in range(args.steps):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st = solve_dev(h_variant, h_store)
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    clocks = clk.summary()
    ms = max_over_ranks(statistics.mean(step_ms), dev)
    y_head = y_d.cpu().numpy()

    # ---------------------------------------------------- end to end (host)
    s = system(h_store)
    y_host = np.empty(n)
    e2e_ms = []
    for _ in range(max(2, args.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, st2 = bs3.bs3_solve(s.handle, w.t0, w.t1, w.y0, RTOL, RTOL, bs3.VARIANT_IDS[h_variant],
                                bs3.ACCUM_IDS[args.accum], None, 0, None, y_host, bs3.HOST_IO)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
        assert rc == bs3.OK

    # ------------------------------------- the fifth-order pair (extension)
    dp54 = {}
    for variant, store in (("mixed1", "f32"), ("double", "f64")):
        sd = bs3.System(w.kind, w.N, w.params, None, device=local, stream=stream.cuda_stream)
        sd.set_coupling(w.coupling, store)
        sd.set_method("dp54")
        best, std = None, None
        for _ in range(2):
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc, std = bs3.bs3_solve(sd.handle, w.t0, w.t1, y0_d, RTOL, RTOL, bs3.VARIANT_IDS[variant],
                                    bs3.ACCUM_IDS[args.accum], None, 0, None, y_d, 0)
            e1.record(stream)
            e1.synchronize()
            best = e0.elapsed_time(e1) if best is None else min(best, e0.elapsed_time(e1))
        sd.close()
        dp54[f"{variant}/{store}"] = {"status": bs3.bs3_status_string(rc), "ms": round(best, 3),
                                      "attempts": std.n_accepted + std.n_rejected,
                                      "global_error": normalized_error(y_ref, y_d.cpu().numpy(), w.N)}

    # ------------------------------------ accuracy against tolerance (Sec. 3.2)
    sweep = None
    if rank == 0 and not args.no_sweep:
        sweep = accuracy_sweep(bs3, torch, w, y0_d, y_ref, stream, flush, local)
    proposer_line = None
    if rank == 0 and not args.no_proposer:
        proposer_line = proposer_comparison(32768)

    # --------------------------------------------------------------- roofline
    evals = st.n_rhs_evals
    bytes_per_eval = w.N * w.N * STORE_BYTES[h_store] + w.N * 4 * 2 + n * 8 * 6
    achieved_gbs = evals * bytes_per_eval / (ms * 1e-3) / 1e9
    peaks = {}
    pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk):
        peaks = json.load(open(pk))
    hbm_peak = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if "hbm_gbs" in peaks else "fallback 6800 GB/s"
    # the headline's weights (N^2 binary32 = 67 MB) stay in L2 across stages:
    # its bound is the L2 read rate, measured here over a buffer of that size
    # with the coupling pass's own loads
    l2_buf = torch.zeros(w.N * w.N * STORE_BYTES[h_store] // 4, dtype=torch.float32, device=dev)
    rc_l2, l2_gbs = bs3.bs3_read_bandwidth(l2_buf, l2_buf.numel() * 4, 40)
    del l2_buf
    if rc_l2 != bs3.OK:
        raise RuntimeError("bs3_read_bandwidth: " + bs3.bs3_status_string(rc_l2))
    result = {
        "metric": METRIC,
        "value": round(ms, 4),
        "unit": "ms",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(ms, 4),
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"f32": "f32", "bf16": "bf16", "f16": "f16", "f64": "f64", "fp8e4m3": "fp8"}[h_store]
                 + "+f64" if h_variant != "single" else "f32",
        "data": "synthetic (seeded numpy; Kuramoto shaped like the paper's Benchmark 2)",
        "config": {"workload": WORKLOAD, "N": w.N, "t1": T1, "rtol": RTOL, "atol": RTOL,
                   "variant": h_variant, "weights": h_store, "sigma_d_sum": args.accum,
                   "headline_rule": f"fixed {head}; the fastest mixed variant within the error factor in "
                                    f"this run's survey: {fastest_ok}",
                   "launch_plan": {"resident_weights": plan[0], "ctas": plan[1]},
                   "parallelism": "replicas only" if world > 1 else "1 GPU",
                   "l2": "flushed between steps (512 MiB write, then 512 MiB read of another buffer, "
                         "outside the timed events)",
                   "reference_solution": ref_kind, "error_factor": ERROR_FACTOR},
        "global_error": normalized_error(y_ref, y_head, w.N),
        "fp64_gpu_ms": survey["double/f64"]["ms"],
        "fp64_gpu_global_error": e_double,
        "speedup_vs_fp64_gpu": survey["double/f64"]["ms"] / ms,
        "accepted": st.n_accepted, "rejected": st.n_rejected, "rhs_evals": evals,
        "headline_within_error_factor": bool(survey[head]["global_error"] <= ERROR_FACTOR * e_double),
        "parity_unpinned": ["step-size controller formula and constants (the paper gives none; the standard "
                            "3(2) controller with exponent 1/3 and safety 0.8 is read in)",
                            "starting step (the paper gives none; Hairer-Norsett-Wanner II.4 is read in)"],
        "sigma_d_literal": sigma_literal,
        "survey": survey,
        "dormand_prince_54": dp54,
        "accuracy_sweep": sweep,
        "learned_proposer": proposer_line,
        "wall_s_timed_region": wall,
        "clocks": clocks,
        "e2e": {"value": round(statistics.median(e2e_ms), 4), "unit": "ms",
                "h2d_bytes_per_step": n * 8, "d2h_bytes_per_step": n * 8 + 64},
        "gpu_launches": args.steps,
        "roofline": {"bound": "l2", "achieved": round(achieved_gbs, 1), "peak": round(l2_gbs, 1), "unit": "GB/s",
                     "frac": round(achieved_gbs / l2_gbs, 4),
                     "traffic": recorded_traffic(f"kuramoto4096_{h_variant}_{h_store}"),
                     "peak_source": "measured in this run: bs3_read_bandwidth, 40 passes over an L2-resident "
                                    f"{w.N * w.N * STORE_BYTES[h_store] / 1e6:.0f} MB buffer",
                     "hbm_frac": round(achieved_gbs / hbm_peak, 4), "hbm_peak": hbm_peak, "hbm_peak_source": hbm_src,
                     "note": "algorithmic bytes = rhs_evals x (N^2 b_K + vectors) per solve launch; the weights "
                             "stay in L2 (DRAM traffic per launch, ncu, is one read of them), so the L2 read "
                             "rate bounds the pass; roofline_streaming is the HBM-bound case"},
        "roofline_streaming": streaming_roofline(bs3, hbm_peak),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        result["cpu_baseline"] = cpu_baseline(w, h_variant, h_store, st.n_accepted + st.n_rejected,
                                              args.cpu_sample_attempts)
    for s in systems.values():
        s.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(result))


SWEEP_RTOLS = [1e-3, 1e-4, 1e-5, 1e-6, 1e-7, 1e-8, 1e-9]
SWEEP_COMBOS = [("double", "f64"), ("mixed2", "f32"), ("mixed1", "f32"), ("single", "f32")]


def accuracy_sweep(bs3, torch, w, y0_d, y_ref, stream, flush, device):
    """Global error and time-to-solution of each variant over rtol = atol =
    1e-3 .. 1e-9 on the benchmark workload (Sec. 3.2, Fig. Tol-VS-Error):
    per rtol, each mixed variant's error as a factor of the binary64 path's,
    and its time at the binary64 path's error (log-log interpolation along its
    own curve) as a ratio to the binary64 time.  L2 flushed before each timed
    solve; each configuration warmed up once."""
    y_d = torch.empty_like(y0_d)
    curves, rows = {}, []
    for variant, store in SWEEP_COMBOS:
        s = bs3.System(w.kind, w.N, w.params, None, device=device, stream=stream.cuda_stream)
        s.set_coupling(w.coupling, store)
        bs3.bs3_solve(s.handle, w.t0, w.t1, y0_d, 1e-3, 1e-3, bs3.VARIANT_IDS[variant], bs3.ACC_FLOAT2, None, 0,
                      None, y_d, 0)
        pts = []
        for rt in SWEEP_RTOLS:
            flush.zero_()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            rc, st = bs3.bs3_solve(s.handle, w.t0, w.t1, y0_d, rt, rt, bs3.VARIANT_IDS[variant], bs3.ACC_FLOAT2,
                                   None, 0, None, y_d, 0)
            e1.record(stream)
            e1.synchronize()
            ms = e0.elapsed_time(e1)
            err = normalized_error(y_ref, y_d.cpu().numpy(), w.N) if rc == bs3.OK else None
            pts.append({"rtol": rt, "status": bs3.bs3_status_string(rc), "ms": round(ms, 3), "global_error": err,
                        "attempts": st.n_accepted + st.n_rejected})
        s.close()
        curves[f"{variant}/{store}"] = pts
    dbl = curves["double/f64"]
    for k, rt in enumerate(SWEEP_RTOLS):
        e_d, t_d = dbl[k]["global_error"], dbl[k]["ms"]
        row = {"rtol": rt, "double/f64": {"global_error": e_d, "ms": t_d}}
        for key, pts in curves.items():
            if key == "double/f64":
                continue
            p = pts[k]
            ok = [(q["global_error"], q["ms"]) for q in pts if q["global_error"] is not None]
            t = time_at(ok, e_d) if e_d is not None else None
            row[key] = {"global_error": p["global_error"], "ms": p["ms"],
                        "error_factor_vs_double": (None if p["global_error"] is None or not e_d
                                                   else round(p["global_error"] / e_d, 3)),
                        "ms_at_double_error": None if t is None else round(t, 3),
                        "speedup_at_double_error": None if t is None else round(t_d / t, 3)}
        rows.append(row)
    return {"workload": WORKLOAD, "reference": "oracle DOPRI5 rtol=atol=1e-12", "per_rtol": rows,
            "curves": curves}


def streaming_roofline(bs3, hbm_peak):
    """The coupling pass where the weights cannot stay on chip: second-order
    oscillators, N = 16384, f16 weights (537 MB), Mixed1, t in [0, 0.5];
    HBM bytes per solve = rhs_evals x N^2 x 2 B."""
    import torch
    make, variant, store = CASES["lco16384_mixed1_f16"]
    w = make()
    s = bs3.System.from_workload(w, store)
    y0 = torch.tensor(w.y0, dtype=torch.float64, device="cuda")
    y = torch.empty_like(y0)
    best, st = None, None
    for _ in range(3):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        rc, st = bs3.bs3_solve(s.handle, w.t0, w.t1, y0, w.rtol, w.atol, bs3.VARIANT_IDS[variant],
                               bs3.ACC_FLOAT2, None, 0, None, y, 0)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    s.close()
    gbs = st.n_rhs_evals * w.N * w.N * STORE_BYTES[store] / (best * 1e-3) / 1e9
    return {"bound": "hbm", "workload": "lco_cfg_N16384_f16_mixed1_t0.5", "achieved": round(gbs, 1),
            "peak": hbm_peak, "unit": "GB/s", "frac": round(gbs / hbm_peak, 4),
            "traffic": recorded_traffic("lco16384_mixed1_f16"), "ms": round(best, 3)}


# ------------------------------------------------------------- CPU oracle
def cpu_sample(w, variant, store, attempts):
    from oracle import bs3 as obs3
    from oracle import models
    osys = models.from_workload(w, store)
    t0 = time.perf_counter()
    r = obs3.solve(osys, w.t0, w.t1, w.y0, w.rtol, w.atol, variant,
                   limits=obs3.Limits(max_attempts=attempts))
    dt = time.perf_counter() - t0
    return dt, r.n_accepted + r.n_rejected


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def cpu_sample_process(variant, store, attempts, threads=None):
    """The oracle's first `attempts` attempts of the benchmark solve, timed in
    a fresh process whose BLAS/OpenMP threads are limited to `threads` (None:
    the library default, one per core).  Returns (seconds, attempts)."""
    env = dict(os.environ)
    if threads:
        for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
            env[k] = str(threads)
    code = ("import json, bench, workloads; "
            f"w = workloads.kuramoto({N_AGENTS}, seed=0, t1={T1}, rtol={RTOL}); "
            f"print(json.dumps(bench.cpu_sample(w, '{variant}', '{store}', {attempts})))")
    res = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                         timeout=1200)
    if res.returncode != 0:
        raise RuntimeError("CPU oracle sample failed: " + res.stderr[-500:])
    dt, att = json.loads(res.stdout.strip().splitlines()[-1])
    return dt, att


def cpu_baseline(w, variant, store, gpu_attempts, sample_attempts):
    """The oracle on the host cores, all cores and one thread, each a bounded
    sample of the same solve extrapolated per attempt to the GPU solve's
    attempt count (stated as such)."""
    cores = os.cpu_count()
    dt_all, att_all = cpu_sample_process(variant, store, sample_attempts)
    n1 = max(4, sample_attempts // 4)
    dt_one, att_one = cpu_sample_process(variant, store, n1, threads=1)
    per_all, per_one = dt_all / max(att_all, 1), dt_one / max(att_one, 1)
    return {"value": round(per_all * gpu_attempts * 1e3, 1), "unit": "ms", "cores": cores, "kind": "oracle",
            "cpu_model": cpu_model(), "nproc": cores,
            "sample": f"first {att_all} attempts of the same solve ({dt_all:.1f} s, BLAS threads = {cores}; the "
                      f"elementwise numpy steps run on one core), per-attempt time extrapolated to the GPU "
                      f"solve's {gpu_attempts} attempts",
            "single_thread": {"value": round(per_one * gpu_attempts * 1e3, 1), "unit": "ms", "cores": 1,
                              "sample": f"first {att_one} attempts ({dt_one:.1f} s), one thread, extrapolated "
                                        f"likewise"}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    w = workloads.kuramoto(N_AGENTS, seed=0, t1=T1, rtol=RTOL)
    variant, store = HEADLINE
    rec = json.load(open(ORACLE_SOLVE_FILE))
    attempts = int(rec["accepted"] + rec["rejected"])
    sample = 10
    for _ in range(args.warmup):
        cpu_sample(w, variant, store, 2)
    per, step_s = [], []
    t_all = time.perf_counter()
    for _ in range(args.steps):
        dt, att = cpu_sample(w, variant, store, sample)
        per.append(dt / att)
        step_s.append(dt)
    wall = time.perf_counter() - t_all
    value = statistics.mean(per) * attempts * 1e3
    cores = os.cpu_count()
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(value, 1), "unit": "ms", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * statistics.mean(step_s), 1),
        "value_kind": f"extrapolated time-to-solution: each step times the oracle's first {sample} attempts of "
                      f"the solve; per-attempt time x the {attempts} attempts of the oracle's own full solve "
                      f"(tests/golden/{os.path.basename(ORACLE_SOLVE_FILE)})",
        "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "N": N_AGENTS, "t1": T1, "rtol": RTOL, "atol": RTOL,
                                        "variant": variant, "weights": store, "sigma_d_sum": "f64 (numpy)"},
        "cpu_baseline": {"value": round(value, 1), "unit": "ms", "cores": cores, "kind": "oracle",
                         "cpu_model": cpu_model(), "nproc": cores,
                         "sample": f"{sample} attempts per step, per-attempt time x {attempts} attempts"},
        "e2e": {"value": round(value, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s_timed_region": wall,
    }))


if __name__ == "__main__":
    a = parse()
    if a.case:
        run_case(a.case)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)
