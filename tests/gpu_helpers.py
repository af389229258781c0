"""Helpers shared by the GPU parity tests (CUDA path through the C ABI vs the
CPU oracle on the same seeded inputs)."""

import numpy as np

U32 = 2.0 ** -24     # binary32 unit roundoff
U64 = 2.0 ** -53     # binary64 unit roundoff


def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    return torch


def library():
    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_23727_gb300 import bs3
    bs3.load()
    return bs3


def decode_store(q, store):
    """Stored weights returned by bs3_get_coupling -> exact float64 values."""
    import torch
    if store == "bf16":
        return (q.astype(np.uint32) << np.uint32(16)).view(np.float32).astype(np.float64)
    if store == "f16":
        return q.astype(np.float64)
    if store == "fp8e4m3":
        return torch.from_numpy(q.copy()).view(torch.float8_e4m3fn).to(torch.float64).numpy()
    return q.astype(np.float64)


def jvalues(kind, y, N):
    """binary64 j-side values g_j used for the magnitude bound sum_j |w_ij g_j|."""
    x = np.asarray(y, dtype=np.float64).reshape(-1, N)[0]
    if kind == "kuramoto":
        return [np.abs(np.sin(x)), np.abs(np.cos(x))]
    if kind == "circadian":
        return [np.full(N, np.pi / 2)]
    return [np.abs(x)]


def rhs_tolerance(osys, y, prec, accum="float2"):
    """Per-component bound on |gpu - oracle| for one right-hand side.

    * the j-side values and products agree to a few units of the G
      precision (own arctangent <= 3 ulp, sincos of a reduced phase <= 2 ulp);
    * binary32 sums (Sigma = S) may be ordered differently: at most
      (N + 64) binary32 roundings of sum_j |w_ij g_j|;
    * binary64 / float-float sums: (N + 64) roundings of their own unit, and
      for Kuramoto's biased float-float sums the growth of their low parts;
    * the agent term and the i-side finish: a few roundings of their precision.
    """
    F, S, G = prec
    N, d = osys.N, osys.d
    W = np.abs(osys.s.astype(np.float64)[:, None] * osys.q.astype(np.float64))
    mag = sum(W @ g for g in jvalues(osys.kind, y, N))
    uG = U32 if G == "S" else U64
    if S == "S":
        uS = U32
    else:
        uS = {"f64": U64, "float2": 2.0 ** -44, "f32": U32}[accum] if G == "S" else U64
    uF = U32 if F == "S" else U64
    coupling_bound = (4 * uG + (N + 64) * uS) * mag
    if osys.kind in ("kuramoto", "circadian") and S == "D" and G == "S" and accum == "float2":
        # the packed float-float sums start from the bias B <= 5 sum_j |q_ij| of
        # the CTA's rows (circadian: 2B, |arctan| <= pi/2; Fast2Sum): each of
        # the gt >= 32 threads of a row adds
        # n <= ld/gt + 16 products, and its low part rounds by <= 2^-48 B k at
        # its k-th addition, in all gt n (n + 1) 2^-49 B
        # <= (ld^2/32 + 33 ld + 8192) 2^-49 B
        ld = (N + 15) // 16 * 16
        B = (10 if osys.kind == "circadian" else 5) * W.sum(axis=1).max()
        coupling_bound = coupling_bound + (ld * ld / 32 + 33 * ld + 8192) * 2.0 ** -49 * B
    if osys.kind == "circadian":
        coupling_bound = coupling_bound * 8.0          # pref_i <= k0 a = 4
    Y = np.abs(np.asarray(y, dtype=np.float64).reshape(d, N))
    scale = np.max(Y, axis=0) + 1.0
    if osys.kind == "kuramoto":
        scale = scale + np.abs(osys.params)
    if osys.kind in ("lco_cfg",):
        scale = scale * (1.0 + osys.params ** 2)
    tol = np.zeros((d, N))
    tol[:] = 32 * uF * scale * 4
    from oracle.models import COUPLED_COMPONENT
    tol[COUPLED_COMPONENT[osys.kind]] += coupling_bound * 2 + 16 * uS * mag
    if osys.kind == "circadian":
        tol = tol * 4.0 + 64 * uF * (1 + Y.sum(axis=0)) ** 3
    return tol.reshape(-1)
