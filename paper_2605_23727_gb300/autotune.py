"""Launch-plan cache of the autotuner (bs3_autotune): one JSON table keyed by
(kind, N, stored weights, variant, Sigma mode, GPU name), so that a plan found
once is applied to later systems of the same shape without timing again."""

from __future__ import annotations

import json
import os
from typing import Optional, Tuple

from . import bs3

DEFAULT_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "autotune_cache.json")


def _key(kind, N, store, variant, accum, gpu):
    return f"{kind}|{N}|{store}|{variant}|{accum}|{gpu}"


def tuned(system: "bs3.System", y0_dev, t0: float, t1: float, rtol: float, variant: str, accum: str,
          gpu: str, attempts: int = 40, path: str = DEFAULT_PATH) -> Tuple[Tuple[int, int], Optional[float]]:
    """Applies the cached plan for this shape, or runs the autotuner and caches it."""
    table = json.load(open(path)) if os.path.exists(path) else {}
    key = _key(system.kind, system.N, system.store, variant, accum, gpu)
    if key in table:
        res, ctas = table[key]["plan"]
        for k, v in ((bs3.TUNE_RESIDENT_WEIGHTS, res), (bs3.TUNE_CTAS, ctas)):
            rc = bs3.bs3_set_tuning(system.handle, k, v)
            if rc != bs3.OK:
                raise RuntimeError(bs3.bs3_status_string(rc))
        return (res, ctas), table[key].get("us_per_attempt")
    rc, plan, us = bs3.bs3_autotune(system.handle, y0_dev, t0, t1, rtol, bs3.VARIANT_IDS[variant],
                                    bs3.ACCUM_IDS[accum], attempts)
    if rc != bs3.OK:
        raise RuntimeError(bs3.bs3_status_string(rc))
    table[key] = {"plan": list(plan), "us_per_attempt": us}
    with open(path, "w") as fh:
        json.dump(table, fh, indent=1, sort_keys=True)
    return plan, us
