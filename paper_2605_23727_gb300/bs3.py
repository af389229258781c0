"""ctypes binding of the C ABI in include/bs3.h (argument marshalling only).

Every function keeps the C name.  Pointers are passed as Python ints (device
addresses, e.g. ``tensor.data_ptr()``) or as numpy arrays (host memory).  The
binding never computes any part of the method: a missing library raises.
"""

from __future__ import annotations

import ctypes
import os
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libbs3.so")

# enums of bs3.h
LCO_CFG, LCO_PAPER, KURAMOTO, CIRCADIAN = 0, 1, 2, 3
SINGLE, MIXED1, MIXED2, DOUBLE = 0, 1, 2, 3
F64, F32, BF16, F16, FP8E4M3 = 0, 1, 2, 3, 4
ACC_F32, ACC_FLOAT2, ACC_F64 = 0, 1, 2
HOST_IO = 1
OK = 0
ERR_INVALID_ARG, ERR_CUDA, ERR_MAX_STEPS, ERR_MAX_REJECTS = 1, 2, 3, 4
ERR_STEP_TOO_SMALL, ERR_TIMEOUT, ERR_DEVICE_WAIT, ERR_NONFINITE = 5, 6, 7, 8

KIND_IDS = {"lco_cfg": LCO_CFG, "lco_paper": LCO_PAPER, "kuramoto": KURAMOTO, "circadian": CIRCADIAN}
VARIANT_IDS = {"single": SINGLE, "mixed1": MIXED1, "mixed2": MIXED2, "double": DOUBLE}
DTYPE_IDS = {"f64": F64, "f32": F32, "bf16": BF16, "f16": F16, "fp8e4m3": FP8E4M3}
ACCUM_IDS = {"f32": ACC_F32, "float2": ACC_FLOAT2, "f64": ACC_F64}
STORE_NUMPY = {F64: np.float64, F32: np.float32, BF16: np.uint16, F16: np.float16, FP8E4M3: np.uint8}

EXPORTED = (
    "bs3_default_limits", "bs3_status_string", "bs3_create_system", "bs3_set_coupling",
    "bs3_get_coupling", "bs3_rhs", "bs3_attempt", "bs3_solve", "bs3_destroy_system",
    "bs3_set_history", "bs3_get_history", "bs3_set_tuning", "bs3_solve_noalloc",
    "bs3_mlp_dataset", "bs3_mlp_train", "bs3_mlp_grad", "bs3_set_proposer", "bs3_tc_gemm",
    "bs3_ensemble_solve", "bs3_batch_solve", "bs3_autotune", "bs3_set_method",
    "bs3_ensemble_solve_tiled", "bs3_ensemble_autotune", "bs3_tc_gemm_persistent",
    "bs3_read_bandwidth", "bs3_solve_batch",
)
METHOD_BS32, METHOD_DP54 = 0, 1
METHOD_IDS = {"bs32": METHOD_BS32, "dp54": METHOD_DP54}
TUNE_CTAS = 2
MLP_PARAMS = 1313
MLP_MODEL = 1325
NOALLOC_MAX_N = 16384
TUNE_RESIDENT_WEIGHTS = 1


class bs3_stats(ctypes.Structure):
    _fields_ = [
        ("n_accepted", ctypes.c_int64),
        ("n_rejected", ctypes.c_int64),
        ("n_rhs_evals", ctypes.c_int64),
        ("t_reached", ctypes.c_double),
        ("h_last", ctypes.c_double),
        ("status", ctypes.c_int32),
        ("n_out_written", ctypes.c_int32),
    ]


class bs3_limits(ctypes.Structure):
    _fields_ = [
        ("max_attempts", ctypes.c_int64),
        ("max_rejects", ctypes.c_int64),
        ("hmin_factor", ctypes.c_double),
        ("wall_limit_s", ctypes.c_double),
        ("slow_limit_s", ctypes.c_double),
        ("slow_fraction", ctypes.c_double),
        ("spin_limit", ctypes.c_int64),
    ]


class bs3_batch_item(ctypes.Structure):
    _fields_ = [
        ("sys", ctypes.c_void_p),
        ("y0", ctypes.c_void_p),
        ("y_final", ctypes.c_void_p),
        ("t0", ctypes.c_double),
        ("t1", ctypes.c_double),
        ("rtol", ctypes.c_double),
        ("atol", ctypes.c_double),
        ("stats", bs3_stats),
    ]


class bs3_ensemble_group(ctypes.Structure):
    _fields_ = [
        ("K", ctypes.c_void_p),
        ("N", ctypes.c_int64),
        ("T", ctypes.c_int64),
        ("omega", ctypes.c_void_p),
        ("theta0", ctypes.c_void_p),
        ("theta_out", ctypes.c_void_p),
        ("t0", ctypes.c_double),
        ("t1", ctypes.c_double),
        ("rtol", ctypes.c_double),
        ("atol", ctypes.c_double),
        ("tile_n", ctypes.c_int),
        ("ctas", ctypes.c_int),
        ("n_acc", ctypes.c_void_p),
        ("n_rej", ctypes.c_void_p),
        ("status", ctypes.c_void_p),
        ("lockstep_attempts", ctypes.c_int64),
    ]


_lib: Optional[ctypes.CDLL] = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libbs3.so (raising if it was not built) and declares signatures."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with __graft_entry__.build() "
                           "(the CUDA library is required; there is no fallback)")
    lib = ctypes.CDLL(path)
    P, D, I, I64 = ctypes.c_void_p, ctypes.c_double, ctypes.c_int, ctypes.c_int64
    sig = {
        "bs3_default_limits": (None, [ctypes.POINTER(bs3_limits)]),
        "bs3_status_string": (ctypes.c_char_p, [I]),
        "bs3_create_system": (I, [I, I64, P, I64, I, P, ctypes.POINTER(P)]),
        "bs3_set_coupling": (I, [P, P, I, I, I]),
        "bs3_get_coupling": (I, [P, P, P]),
        "bs3_rhs": (I, [P, D, P, I, I, I, I, P]),
        "bs3_attempt": (I, [P, D, D, P, P, D, D, I, I, P, P, ctypes.POINTER(D)]),
        "bs3_solve": (I, [P, D, D, P, D, D, I, I, P, I64, P, P, I, ctypes.POINTER(bs3_stats),
                          ctypes.POINTER(bs3_limits)]),
        "bs3_destroy_system": (I, [P]),
        "bs3_set_history": (I, [P, I64]),
        "bs3_set_tuning": (I, [P, I, I64]),
        "bs3_mlp_dataset": (I, [P, I64, D, P, P, ctypes.POINTER(I64)]),
        "bs3_mlp_train": (I, [P, P, I64, P, I, I, ctypes.c_float, ctypes.c_uint64, P, P]),
        "bs3_mlp_grad": (I, [P, P, P, I64, P, P]),
        "bs3_set_proposer": (I, [P, P]),
        "bs3_tc_gemm": (I, [I64, I64, I64, P, P, P]),
        "bs3_tc_gemm_persistent": (I, [I64, I64, I64, P, P, P, I, I]),
        "bs3_read_bandwidth": (I, [P, I64, I, ctypes.POINTER(D)]),
        "bs3_solve_batch": (I, [P, I64, I, I, I, ctypes.POINTER(bs3_ensemble_group), I, P, ctypes.POINTER(D)]),
        "bs3_ensemble_solve": (I, [P, I64, I64, P, P, D, D, D, D, P, P, P, P, ctypes.POINTER(I64), P]),
        "bs3_batch_solve": (I, [I, I64, P, P, P, I, P, P, P, D, D, I, I, P, P, ctypes.POINTER(D), I, P]),
        "bs3_autotune": (I, [P, P, D, D, D, I, I, I, P, ctypes.POINTER(D)]),
        "bs3_solve_noalloc": (I, [I, I64, P, P, P, I, I64, D, D, P, D, D, I, I, P, I64, P, P,
                                  ctypes.POINTER(bs3_stats), P]),
        "bs3_get_history": (I, [P, P, ctypes.POINTER(I64)]),
        "bs3_set_method": (I, [P, I]),
        "bs3_ensemble_solve_tiled": (I, [P, I64, I64, P, P, D, D, D, D, I, I64, P, P, P, P, ctypes.POINTER(I64), P]),
        "bs3_ensemble_autotune": (I, [P, I64, I64, P, P, D, D, D, D, I64, P, ctypes.POINTER(I),
                                      ctypes.POINTER(D)]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("host arrays must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    raise TypeError(type(x))


# ---------------------------------------------------------------- C names
def bs3_default_limits() -> bs3_limits:
    lim = bs3_limits()
    load().bs3_default_limits(ctypes.byref(lim))
    return lim


def bs3_status_string(status: int) -> str:
    return load().bs3_status_string(status).decode()


def bs3_create_system(kind: int, N: int, params, device: int = 0, stream: int = 0) -> int:
    p = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    out = ctypes.c_void_p()
    rc = load().bs3_create_system(kind, N, _ptr(p), 0 if p is None else p.size, device, stream or None,
                                  ctypes.byref(out))
    if rc != OK:
        raise RuntimeError(f"bs3_create_system: {bs3_status_string(rc)}")
    return out.value


def bs3_set_coupling(sys_: int, K, src: int, store: int, is_device_ptr: bool) -> int:
    return load().bs3_set_coupling(sys_, _ptr(K), src, store, int(is_device_ptr))


def bs3_get_coupling(sys_: int, q_out, scales_out) -> int:
    return load().bs3_get_coupling(sys_, _ptr(q_out), _ptr(scales_out))


def bs3_rhs(sys_: int, t: float, y, f_prec: int, sigma_prec: int, g_prec: int, accum: int, out) -> int:
    return load().bs3_rhs(sys_, t, _ptr(y), f_prec, sigma_prec, g_prec, accum, _ptr(out))


def bs3_attempt(sys_: int, t: float, h: float, x, k1, rtol: float, atol: float, variant: int, accum: int,
                xn_out, k4_out):
    err = ctypes.c_double()
    rc = load().bs3_attempt(sys_, t, h, _ptr(x), _ptr(k1), rtol, atol, variant, accum, _ptr(xn_out),
                            _ptr(k4_out), ctypes.byref(err))
    return rc, err.value


def bs3_solve(sys_: int, t0: float, t1: float, y0, rtol: float, atol: float, variant: int, accum: int,
              t_out, n_out: int, y_out, final_y, flags: int, limits: Optional[bs3_limits] = None):
    st = bs3_stats()
    rc = load().bs3_solve(sys_, t0, t1, _ptr(y0), rtol, atol, variant, accum, _ptr(t_out), n_out,
                          _ptr(y_out), _ptr(final_y), flags, ctypes.byref(st),
                          None if limits is None else ctypes.byref(limits))
    return rc, st


def bs3_set_method(sys_: int, method: int) -> int:
    return load().bs3_set_method(sys_, method)


def bs3_set_tuning(sys_: int, key: int, value: int) -> int:
    return load().bs3_set_tuning(sys_, key, value)


def bs3_set_history(sys_: int, capacity: int) -> int:
    return load().bs3_set_history(sys_, capacity)


def bs3_get_history(sys_: int, capacity: int):
    """Returns (rc, records[n, 8])."""
    out = np.zeros((max(capacity, 1), 8))
    n = ctypes.c_int64()
    rc = load().bs3_get_history(sys_, _ptr(out), ctypes.byref(n))
    return rc, out[:n.value]


def bs3_solve_noalloc(kind: int, N: int, par, globals_, weights, store: int, ld: int, t0: float, t1: float,
                      y0, rtol: float, atol: float, variant: int, accum: int, t_out, n_out: int, y_out,
                      final_y, stream: int = 0):
    st = bs3_stats()
    g = None if globals_ is None else np.ascontiguousarray(globals_, dtype=np.float64)
    rc = load().bs3_solve_noalloc(kind, N, _ptr(par), _ptr(g), _ptr(weights), store, ld, t0, t1, _ptr(y0), rtol,
                                  atol, variant, accum, _ptr(t_out), n_out, _ptr(y_out), _ptr(final_y),
                                  ctypes.byref(st), stream or None)
    return rc, st


def bs3_mlp_dataset(hist, rtol: float):
    """Returns (rc, X[n, 6] float32, y[n] float32) from history records [n_rec, 8]."""
    hist = np.ascontiguousarray(hist, dtype=np.float64)
    n_rec = hist.shape[0]
    X = np.zeros((max(n_rec, 1), 6), dtype=np.float32)
    y = np.zeros(max(n_rec, 1), dtype=np.float32)
    n = ctypes.c_int64()
    rc = load().bs3_mlp_dataset(_ptr(hist), n_rec, rtol, _ptr(X), _ptr(y), ctypes.byref(n))
    return rc, X[:n.value], y[:n.value]


def bs3_mlp_train(X, y, params_init, epochs: int, batch: int, lr: float, seed: int):
    """Returns (rc, model[1325] float32, loss_hist[epochs] float32)."""
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    p0 = np.ascontiguousarray(params_init, dtype=np.float32)
    model = np.zeros(MLP_MODEL, dtype=np.float32)
    hist = np.zeros(epochs, dtype=np.float32)
    rc = load().bs3_mlp_train(_ptr(X), _ptr(y), X.shape[0], _ptr(p0), epochs, batch, lr, seed, _ptr(model),
                              _ptr(hist))
    return rc, model, hist


def bs3_mlp_grad(params, X, y):
    """Returns (rc, loss, grad[1313] float32)."""
    p = np.ascontiguousarray(params, dtype=np.float32)
    X = np.ascontiguousarray(X, dtype=np.float32)
    y = np.ascontiguousarray(y, dtype=np.float32)
    g = np.zeros(MLP_PARAMS, dtype=np.float32)
    loss = ctypes.c_float()
    rc = load().bs3_mlp_grad(_ptr(p), _ptr(X), _ptr(y), X.shape[0], _ptr(g), ctypes.byref(loss))
    return rc, loss.value, g


def bs3_set_proposer(sys_: int, model) -> int:
    m = None if model is None else np.ascontiguousarray(model, dtype=np.float32)
    return load().bs3_set_proposer(sys_, _ptr(m))


def bs3_tc_gemm(M: int, Nc: int, K: int, A, B, C) -> int:
    return load().bs3_tc_gemm(M, Nc, K, _ptr(A), _ptr(B), _ptr(C))


def bs3_tc_gemm_persistent(M: int, Nc: int, K: int, A, B, C, tile_n: int = 128, max_ctas: int = 0) -> int:
    return load().bs3_tc_gemm_persistent(M, Nc, K, _ptr(A), _ptr(B), _ptr(C), tile_n, max_ctas)


def bs3_ensemble_solve(K, N: int, T: int, omega, theta0, t0: float, t1: float, rtol: float, atol: float,
                       theta_out, stream: int = 0, tile_n: int = 0, max_lockstep: int = 0):
    """Returns (rc, n_acc[T], n_rej[T], status[T], lockstep_attempts)."""
    n_acc = np.zeros(T, dtype=np.int64)
    n_rej = np.zeros(T, dtype=np.int64)
    status = np.zeros(T, dtype=np.int32)
    steps = ctypes.c_int64()
    rc = load().bs3_ensemble_solve_tiled(_ptr(K), N, T, _ptr(omega), _ptr(theta0), t0, t1, rtol, atol, tile_n,
                                         max_lockstep, _ptr(theta_out), _ptr(n_acc), _ptr(n_rej), _ptr(status),
                                         ctypes.byref(steps), stream or None)
    return rc, n_acc, n_rej, status, steps.value


def bs3_ensemble_autotune(K, N: int, T: int, omega, theta0, t0: float, t1: float, rtol: float, atol: float,
                          lockstep_attempts: int, scratch_theta):
    """Returns (rc, tile width, microseconds per lock-step attempt)."""
    tile = ctypes.c_int()
    us = ctypes.c_double()
    rc = load().bs3_ensemble_autotune(_ptr(K), N, T, _ptr(omega), _ptr(theta0), t0, t1, rtol, atol,
                                      lockstep_attempts, _ptr(scratch_theta), ctypes.byref(tile), ctypes.byref(us))
    return rc, tile.value, us.value


def bs3_batch_solve(kind: int, Ns, params, K, store: int, y0, t0, t1, rtol: float, atol: float, variant: int,
                    accum: int, device: int = 0, stream: int = 0):
    """Host arrays in, returns (rc, y_final concat, stats list, kernel ms)."""
    Ns = np.ascontiguousarray(Ns, dtype=np.int64)
    S = Ns.size
    p = None if params is None else np.ascontiguousarray(params, dtype=np.float64)
    K = np.ascontiguousarray(K, dtype=np.float32)
    y0 = np.ascontiguousarray(y0, dtype=np.float64)
    t0 = np.ascontiguousarray(t0, dtype=np.float64)
    t1 = np.ascontiguousarray(t1, dtype=np.float64)
    yf = np.zeros_like(y0)
    stats = (bs3_stats * S)()
    kms = ctypes.c_double()
    rc = load().bs3_batch_solve(kind, S, _ptr(Ns), _ptr(p), _ptr(K), store, _ptr(y0), _ptr(t0), _ptr(t1), rtol, atol,
                                variant, accum, _ptr(yf), ctypes.cast(stats, ctypes.c_void_p), ctypes.byref(kms),
                                device, stream or None)
    return rc, yf, list(stats), kms.value


def bs3_autotune(sys_: int, y0, t0: float, t1: float, rtol: float, variant: int, accum: int, attempts: int):
    """Returns (rc, (resident, ctas), microseconds per attempt)."""
    choice = np.zeros(2, dtype=np.int64)
    us = ctypes.c_double()
    rc = load().bs3_autotune(sys_, _ptr(y0), t0, t1, rtol, variant, accum, attempts, _ptr(choice), ctypes.byref(us))
    return rc, (int(choice[0]), int(choice[1])), us.value


def bs3_solve_batch(items, variant: int, accum: int, flags: int = 0, group=None, device: int = 0,
                    stream: int = 0):
    """items: a sequence of dicts with keys sys (handle), y0, y_final (pointers or arrays), t0, t1, rtol,
    atol; group: None or a dict with the fields of bs3_ensemble_group (pointers/arrays, n_acc etc. numpy
    arrays).  Returns (rc, [bs3_stats per item], lockstep attempts of the group or None, kernel ms)."""
    n = len(items)
    arr = (bs3_batch_item * max(n, 1))()
    for k, it in enumerate(items):
        arr[k].sys = it["sys"]
        arr[k].y0 = _ptr(it["y0"])
        arr[k].y_final = _ptr(it["y_final"])
        arr[k].t0, arr[k].t1 = it["t0"], it["t1"]
        arr[k].rtol, arr[k].atol = it["rtol"], it["atol"]
    g = None
    if group is not None:
        g = bs3_ensemble_group()
        for f in ("K", "omega", "theta0", "theta_out", "n_acc", "n_rej", "status"):
            setattr(g, f, _ptr(group.get(f)))
        for f in ("N", "T", "t0", "t1", "rtol", "atol"):
            setattr(g, f, group[f])
        g.tile_n = group.get("tile_n", 0)
        g.ctas = group.get("ctas", 0)
    ms = ctypes.c_double()
    rc = load().bs3_solve_batch(ctypes.cast(arr, ctypes.c_void_p), n, variant, accum, flags,
                                None if g is None else ctypes.byref(g), device, stream or None, ctypes.byref(ms))
    return rc, [arr[k].stats for k in range(n)], (None if g is None else g.lockstep_attempts), ms.value


def bs3_read_bandwidth(buf, nbytes: int, reps: int):
    """Returns (rc, GB/s)."""
    gbs = ctypes.c_double()
    rc = load().bs3_read_bandwidth(_ptr(buf), nbytes, reps, ctypes.byref(gbs))
    return rc, gbs.value


def bs3_destroy_system(sys_: int) -> int:
    return load().bs3_destroy_system(sys_)


# ------------------------------------------------------------ convenience
class System:
    """Owns one bs3 system; host numpy in, host numpy out (BS3_HOST_IO)."""

    def __init__(self, kind: str, N: int, params=None, globals_=None, device: int = 0, stream: int = 0):
        self.kind = kind
        self.N = N
        self.d = {"lco_cfg": 2, "lco_paper": 2, "kuramoto": 1, "circadian": 4}[kind]
        p = params
        if kind == "circadian":
            g = globals_
            p = np.concatenate([np.asarray(params, dtype=np.float64),
                                [g["k0"], g["k2"], g["k3"], g["a"], g["b"], g["c"], g["eps"], g["I0"]]])
        if kind == "lco_paper":
            p = None
        self.handle = bs3_create_system(KIND_IDS[kind], N, p, device, stream)

    @classmethod
    def from_workload(cls, w, store: str = "f64", device: int = 0, stream: int = 0,
                      resident: bool = False) -> "System":
        s = cls(w.kind, w.N, w.params, w.globals, device, stream)
        s.set_coupling(w.coupling, store)
        if resident:
            rc = bs3_set_tuning(s.handle, TUNE_RESIDENT_WEIGHTS, 1)
            if rc != OK:
                raise RuntimeError(bs3_status_string(rc))
        return s

    def set_coupling(self, K, store: str) -> None:
        if hasattr(K, "data_ptr"):
            src = F64 if str(K.dtype) == "torch.float64" else F32
            rc = bs3_set_coupling(self.handle, K.data_ptr(), src, DTYPE_IDS[store], True)
        else:
            K = np.ascontiguousarray(K)
            if K.dtype not in (np.float64, np.float32):
                K = K.astype(np.float64)
            src = F64 if K.dtype == np.float64 else F32
            rc = bs3_set_coupling(self.handle, K, src, DTYPE_IDS[store], False)
        if rc != OK:
            raise RuntimeError(f"bs3_set_coupling: {bs3_status_string(rc)}")
        self.store = store

    def get_coupling(self):
        st = DTYPE_IDS[self.store]
        q = np.empty((self.N, self.N), dtype=STORE_NUMPY[st])
        s = np.empty(self.N, dtype=np.float32)
        rc = bs3_get_coupling(self.handle, q, s)
        if rc != OK:
            raise RuntimeError(bs3_status_string(rc))
        return q, s

    def set_method(self, method: str) -> None:
        rc = bs3_set_method(self.handle, METHOD_IDS[method])
        if rc != OK:
            raise RuntimeError(bs3_status_string(rc))

    def solve(self, t0, t1, y0, rtol, atol, variant="double", accum="float2", t_out=None,
              limits: Optional[bs3_limits] = None):
        y0 = np.ascontiguousarray(y0, dtype=np.float64)
        t_out = np.ascontiguousarray([] if t_out is None else t_out, dtype=np.float64)
        n = self.d * self.N
        y_out = np.zeros((len(t_out), n))
        final = np.zeros(n)
        rc, st = bs3_solve(self.handle, t0, t1, y0, rtol, atol, VARIANT_IDS[variant], ACCUM_IDS[accum],
                           t_out if len(t_out) else None, len(t_out), y_out if len(t_out) else None,
                           final, HOST_IO, limits)
        return rc, st, final, y_out

    def close(self) -> None:
        if getattr(self, "handle", None):
            bs3_destroy_system(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
