"""Writes reference solutions used by the accuracy tests and the benchmark.

Calls only the CPU oracle (binary64 DOPRI5 at rtol = atol = 1e-12, the
paper's ode45-style reference of Sec. 2.4) on seeded synthetic workloads:

  ref_kuramoto_N4096_seed0_t50.npy  Kuramoto, N = 4096, K_ij = (2/N)(1 + U(-1/2,1/2)),
                                   omega ~ N(0,1), theta0 ~ U(0, 2 pi), t in [0, 50]

Usage: python tests/golden/make_references.py   (about an hour on 8 cores)
"""

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402
from oracle import dopri5, models  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))


def main():
    w = workloads.kuramoto(4096, 0, t1=50.0)
    S = models.from_workload(w, "f64")
    t = time.time()
    f = lambda tt, y: models.rhs(S, tt, y, ("D", "D", "D"))  # noqa: E731
    y, acc, rej = dopri5.integrate(f, w.t0, w.t1, w.y0, 1e-12, 1e-12)
    np.save(os.path.join(HERE, "ref_kuramoto_N4096_seed0_t50.npy"), y)
    print(f"kuramoto N=4096: {acc} accepted, {rej} rejected, {time.time() - t:.0f} s")


if __name__ == "__main__":
    main()
