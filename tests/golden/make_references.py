"""Writes reference solutions used by the accuracy tests and the benchmark.

Calls only the CPU oracle (binary64 DOPRI5 at rtol = atol = 1e-12, the
paper's ode45-style reference of Sec. 2.4) on seeded synthetic workloads:

  ref_kuramoto_N4096_seed0_t50.npy  Kuramoto, N = 4096, K_ij = (2/N)(1 + U(-1/2,1/2)),
                                   omega ~ N(0,1), theta0 ~ U(0, 2 pi), t in [0, 50]

  oracle_solve_kuramoto_N4096_mixed1_f32.json
                                   the oracle's own BS3 solve of that workload (Mixed1,
                                   binary32 weights, rtol = atol = 1e-6): its attempt and
                                   evaluation counts, which the benchmark's CPU arms
                                   multiply their per-attempt time by

Usage: python tests/golden/make_references.py [reference|oracle-solve]
(the reference takes about an hour on 8 cores, the oracle solve minutes)
"""

import json
import math
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from oracle import bs3, dopri5, models  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    w = workloads.kuramoto(4096, 0, t1=50.0)
    S = models.from_workload(w, "f64")
    t = time.time()
    f = lambda tt, y: models.rhs(S, tt, y, ("D", "D", "D"))  # noqa: E731
    y, acc, rej = dopri5.integrate(f, w.t0, w.t1, w.y0, 1e-12, 1e-12)
    np.save(os.path.join(HERE, "ref_kuramoto_N4096_seed0_t50.npy"), y)
    print(f"kuramoto N=4096: {acc} accepted, {rej} rejected, {time.time() - t:.0f} s")


def oracle_solve():
    w = workloads.kuramoto(4096, 0, t1=50.0, rtol=1e-6)
    S = models.from_workload(w, "f32")
    t = time.time()
    r = bs3.solve(S, w.t0, w.t1, w.y0, 1e-6, 1e-6, "mixed1")
    wall = time.time() - t
    ref = np.load(os.path.join(HERE, "ref_kuramoto_N4096_seed0_t50.npy"))
    out = {"workload": "kuramoto_N4096_t50", "variant": "mixed1", "weights": "f32", "rtol": 1e-6, "atol": 1e-6,
           "status": bs3.STATUS_NAMES[r.status], "accepted": r.n_accepted, "rejected": r.n_rejected,
           "rhs_evals": r.n_rhs, "global_error": float(np.linalg.norm(r.y - ref) / math.sqrt(w.N)),
           "wall_s": round(wall, 1)}
    with open(os.path.join(HERE, "oracle_solve_kuramoto_N4096_mixed1_f32.json"), "w") as fh:
        json.dump(out, fh, indent=1)
    print(out)


if __name__ == "__main__":
    what = sys.argv[1] if len(sys.argv) > 1 else "reference"
    if what == "reference":
        main()
    else:
        oracle_solve()
