"""CPU oracle for the mixed-precision Bogacki-Shampine 3(2) solver.

TEST INFRASTRUCTURE ONLY.  This package is a plain, slow, FP64 (numpy)
restatement of the method of "Mixed-Precision in adaptive Runge-Kutta method
for large ODE systems": the three benchmark right-hand sides (Sec. 2.1), the
Bogacki-Shampine 3(2) pair with FSAL (Sec. 2.2, Table Butcher-O23), the
embedded error norm (Eq. ERROR-O23), the failure conditions (Sec. 2.2), the
Single/Mixed1/Mixed2/Double precision distribution (Sec. 2.3, Table
MP-Distrib), the error metric (Eq. Metric) and a Dormand-Prince 5(4)
reference integrator (Sec. 2.4).  Only ``tests/``, ``__graft_entry__.smoke()``
and ``bench.py``'s CPU-baseline / reference legs may import it; the product
path never does, and it shares no code with the CUDA library.

Parity status per function (what pins it is listed in each module):
* tableau, right-hand sides, stage arithmetic, error norm, dense output,
  number formats, DOPRI5, closed forms, metrics: pinned.
* step-size controller constants and the initial step size: parity unpinned
  (the paper names no formula; the reading adopted is stated in bs3.py).
"""
