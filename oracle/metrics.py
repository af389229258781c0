"""Accuracy and performance metrics of Sec. 2.4-2.5.

* normalized final error (Eq. Metric): ||X_ref(t_f) - X(t_f)||_2 / sqrt(N),
  N the number of agents (not d N);
* beta = N_step,h / N_step,m (Eq. Beta-2MP), steps counting accepted and
  failed attempts.
"""

import numpy as np


def normalized_final_error(x_ref, x, n_agents):
    d = np.asarray(x_ref, dtype=np.float64) - np.asarray(x, dtype=np.float64)
    return float(np.linalg.norm(d) / np.sqrt(n_agents))


def beta(steps_high, steps_mixed):
    return steps_high / steps_mixed
