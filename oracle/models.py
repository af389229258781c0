"""Right-hand sides of the three benchmark systems, with precision emulation.

General model (Sec. 2.1, Eq. General-Model):
    X_i' = F_i(X_i) + sum_j M_ij (.) G_ij(X_i, X_j).
The dense weights are heterogeneous (the general model allows any M_ij) and
held in a storage format (oracle.formats): weight_ij = s_i q_ij.

Kinds (state is structure-of-arrays, component k of agent i at y[k*N + i]):

* "lco_paper" (Eq. LCO): x_i' = x_{i,2}-part v_i + sum_j M_ij (x_j - x_i),
  v_i' = -x_i.  Evaluated as v_i + s_i (q x)_i - rowsum_i x_i.
* "lco_cfg": the second-order oscillator form of the measured configuration,
  x_i' = v_i, v_i' = -omega_i^2 x_i + s_i (q x)_i.
* "kuramoto" (Eq. Kuramoto): theta_i' = omega_i + sum_j K_ij sin(theta_j - theta_i),
  evaluated as cos(theta_i) s_i (q sin theta)_i - sin(theta_i) s_i (q cos theta)_i.
* "circadian" (Eq. CC): the Goodwin / FitzHugh-Nagumo agent term F with the
  coupling pref_i s_i sum_j q_ij atan(x_{j,1} - x_{i,1}) on component 1,
  pref_i = k0 Theta_i a / (Theta_i + x_{i,2}^4), Theta_i = k1_i / (k0 - k1_i).

Precision emulation (Sec. 2.3, Table MP-Distrib): each evaluation takes a
triple (F, Sigma, G) of 'S' (IEEE binary32) or 'D' (binary64):
* G: the interaction terms, i.e. the j-side values (x_j, sin/cos theta_j,
  atan of the difference) and the products with the weights;
* Sigma: the sum over j (S: binary32 accumulation; D: each binary32 product is
  cast to binary64 before a binary64 sum, Sec. 2.3) and the i-side finish
  (row scale, cos/sin theta_i combination, rowsum term, pref_i);
* F: the agent term F_i.
F + coupling is added in the precision of F (equal to Sigma in every row of
the table).  The j-side sine/cosine in G=S is the binary32 rounding of the
sine of the stored phase.

The GEMV-form evaluations above are algebraic rewrites of the pairwise
definitions; ``pairwise_coupling`` writes the definitions out and the tests
compare the two (brute force, long double, tiny N).
"""

from __future__ import annotations

import dataclasses
from typing import Dict, Optional, Sequence

import numpy as np

from . import formats

KINDS = ("lco_cfg", "lco_paper", "kuramoto", "circadian")
DIMS = {"lco_cfg": 2, "lco_paper": 2, "kuramoto": 1, "circadian": 4}

F32 = np.float32
F64 = np.float64


def _ft(p: str):
    return F32 if p == "S" else F64


@dataclasses.dataclass
class System:
    kind: str
    N: int
    params: Optional[np.ndarray]          # omega_i (lco_cfg, kuramoto) or k1_i (circadian)
    q: np.ndarray                         # stored weights (float32 exact values or float64)
    s: np.ndarray                         # per-row scales (float32)
    fmt: str
    globals: Optional[Dict[str, float]] = None
    rowsum: Optional[np.ndarray] = None   # lco_paper: sum_j s_i q_ij (float64)
    theta_h: Optional[np.ndarray] = None  # circadian: k1/(k0-k1) (float64)
    ksplit: Optional[tuple] = None        # tensor variant: bfloat16 split of q (computed once)

    @property
    def d(self) -> int:
        return DIMS[self.kind]


def make_system(kind: str, N: int, params, coupling, fmt: str = "f64", globals=None) -> System:
    if kind not in KINDS:
        raise ValueError(kind)
    q, s = formats.quantize(np.asarray(coupling), fmt)
    sysm = System(kind, N, None if params is None else np.asarray(params, dtype=F64), q, s, fmt,
                  None if globals is None else dict(globals))
    if kind == "lco_paper":
        sysm.rowsum = s.astype(F64) * q.astype(F64).sum(axis=1)
    if kind == "circadian":
        k0 = sysm.globals["k0"]
        sysm.theta_h = sysm.params / (k0 - sysm.params)
    return sysm


def from_workload(w, fmt: str = "f64") -> System:
    return make_system(w.kind, w.N, w.params, w.coupling, fmt, w.globals)


# --------------------------------------------------------------------------
# The weighted sum over j: sum_j q_ij g_ij in (G, Sigma) precision.
# --------------------------------------------------------------------------

def _sum_products(q_rows: np.ndarray, g: np.ndarray, G: str, Sig: str) -> np.ndarray:
    """Rows of q times a j-vector g (same for every row) or a matrix g[rows, N]."""
    out = np.empty(q_rows.shape[0], dtype=_ft(Sig))
    B = 512
    for r0 in range(0, q_rows.shape[0], B):
        r1 = min(q_rows.shape[0], r0 + B)
        gq = g if g.ndim == 1 else g[r0:r1]
        if G == "S":
            q32 = q_rows[r0:r1].astype(F32)
            g32 = gq.astype(F32)
            if Sig == "S":
                if g.ndim == 1:
                    out[r0:r1] = np.matmul(q32, g32)
                else:
                    out[r0:r1] = (q32 * g32).sum(axis=1, dtype=F32)
            else:
                prod = q32 * g32                           # binary32 products
                out[r0:r1] = prod.astype(F64).sum(axis=1)  # cast, then binary64 sum
        else:
            q64 = q_rows[r0:r1].astype(F64)
            g64 = gq.astype(F64)
            out[r0:r1] = np.matmul(q64, g64) if g.ndim == 1 else (q64 * g64).sum(axis=1)
    return out


def _jvalue(v: np.ndarray, G: str) -> np.ndarray:
    """A j-side state value in G precision (binary32 state stays binary32)."""
    return v.astype(_ft(G)) if v.dtype == F64 else v.astype(_ft(G))


def _trig(theta: np.ndarray, p: str):
    """sin/cos of the stored phase in precision p (rounded from binary64 for
    a binary64 phase, evaluated in binary32 for a binary32 phase)."""
    if theta.dtype == F32 and p == "S":
        return np.sin(theta), np.cos(theta)
    th = theta.astype(F64)
    return np.sin(th).astype(_ft(p)), np.cos(th).astype(_ft(p))


def rhs(sysm: System, t: float, y: np.ndarray, prec: Sequence[str] = ("D", "D", "D"),
        rows: Optional[np.ndarray] = None) -> np.ndarray:
    """f(t, y) in the precision triple prec = (F, Sigma, G).

    Returns an array of y's dtype and shape [d*N]; with ``rows`` given, only
    those agents are evaluated and the result has shape [d, len(rows)].
    """
    Fp, Sp, Gp = prec
    N, d = sysm.N, sysm.d
    Y = y.reshape(d, N)
    idx = np.arange(N) if rows is None else np.asarray(rows)
    q = sysm.q[idx]
    s_row = sysm.s[idx]
    tF, tS = _ft(Fp), _ft(Sp)
    out = np.empty((d, len(idx)), dtype=F64)

    if sysm.kind == "kuramoto":
        th = Y[0]
        sj, cj = _trig(th, Gp)
        S = _sum_products(q, sj, Gp, Sp)
        C = _sum_products(q, cj, Gp, Sp)
        sc = s_row.astype(tS)
        S = S.astype(tS) * sc
        C = C.astype(tS) * sc
        si, ci = _trig(th[idx], Sp)
        coupling = ci * S - si * C
        out[0] = sysm.params[idx].astype(tF) + coupling.astype(tF)
    elif sysm.kind == "lco_cfg":
        x, v = Y[0], Y[1]
        Ax = _sum_products(q, _jvalue(x, Gp), Gp, Sp).astype(tS) * s_row.astype(tS)
        w = sysm.params[idx].astype(tF)
        xi = x[idx].astype(tF)
        out[0] = v[idx].astype(tF)
        out[1] = (-(w * w) * xi) + Ax.astype(tF)
    elif sysm.kind == "lco_paper":
        x, v = Y[0], Y[1]
        Mx = _sum_products(q, _jvalue(x, Gp), Gp, Sp).astype(tS) * s_row.astype(tS)
        coupling = Mx - sysm.rowsum[idx].astype(tS) * x[idx].astype(tS)
        out[0] = v[idx].astype(tF) + coupling.astype(tF)
        out[1] = -(x[idx].astype(tF))
    elif sysm.kind == "circadian":
        g = sysm.globals
        x1, x2, x3, x4 = (Y[k][idx].astype(tF) for k in range(4))
        k0, k2, k3 = tF(g["k0"]), tF(g["k2"]), tF(g["k3"])
        a, b, c = tF(g["a"]), tF(g["b"]), tF(g["c"])
        eps, I0 = tF(g["eps"]), tF(g["I0"])
        k1 = sysm.params[idx].astype(tF)
        Th = sysm.theta_h[idx].astype(tF)
        x2sq = x2 * x2
        hill = (k0 * Th) / (Th + x2sq * x2sq)
        F1 = hill * (a * x1 * x1 + tF(1)) - k1 * x1
        F2 = k2 * (x1 - x2)
        F3 = x3 * (tF(1) - x3 * x3 / tF(3)) - x4 + I0 * (tF(1) - (k3 * k3) / (k3 * k3 + x1 * x1))
        F4 = eps * (x3 + b - c * x4)
        # interaction: atan(x_j1 - x_i1) in G precision, weighted sum in Sigma
        xg = _jvalue(Y[0], Gp)
        xi_g = xg[idx]
        r = np.empty(len(idx), dtype=tS)
        B = 256
        for r0 in range(0, len(idx), B):
            r1 = min(len(idx), r0 + B)
            diff = xg[None, :] - xi_g[r0:r1, None]          # G precision
            at = np.arctan(diff)                             # G precision
            r[r0:r1] = _sum_products(q[r0:r1], at, Gp, Sp)
        tS_ = tS
        x2s = Y[1][idx].astype(tS_)
        x2s2 = x2s * x2s
        pref = (tS_(g["k0"]) * sysm.theta_h[idx].astype(tS_) * tS_(g["a"])) / \
            (sysm.theta_h[idx].astype(tS_) + x2s2 * x2s2)
        coupling = pref * (r * s_row.astype(tS_))
        out[0] = F1 + coupling.astype(tF)
        out[1] = F2
        out[2] = F3
        out[3] = F4
    else:
        raise ValueError(sysm.kind)

    if rows is not None:
        return out
    res = out.reshape(-1)
    return res.astype(y.dtype) if y.dtype == F32 else res


# --------------------------------------------------------------------------
# Tensor-core variant of Kuramoto (ensembles sharing K): the weights and the
# j-side sine/cosine are split into bfloat16 pairs x = x_hi + x_lo, the three
# products K_hi s_hi + K_hi s_lo + K_lo s_hi are exact and summed (here in
# binary64), the sums are held in binary32, the i-side finish is binary32 and
# F = omega in binary64.
# --------------------------------------------------------------------------

def split_bf16(x32: np.ndarray):
    hi = formats.round_bf16(np.asarray(x32, dtype=F32))
    lo = formats.round_bf16((np.asarray(x32, dtype=F32) - hi).astype(F32))
    return hi.astype(F64), lo.astype(F64)


def tensor_sums(sysm: System, y: np.ndarray):
    """The split products of the tensor-core variant: S_i = sum_j (K_hi s_hi
    + K_hi s_lo + K_lo s_hi)_ij and C_i likewise with cos, summed in binary64
    (every product of two bfloat16 values is exact there) and rounded once to
    binary32; also the binary32 sin/cos of the phases.  Returns (S, C, s, c)."""
    if sysm.kind != "kuramoto":
        raise ValueError("the tensor-core variant is defined for Kuramoto ensembles")
    if sysm.ksplit is None:
        sysm.ksplit = split_bf16(sysm.q.astype(F32))
    kh, kl = sysm.ksplit
    th = np.asarray(y, dtype=F64)
    sj, cj = np.sin(th).astype(F32), np.cos(th).astype(F32)
    vh, vl = split_bf16(np.stack([sj, cj], axis=1))     # columns: sine, cosine
    SC = kh @ vh + kh @ vl + kl @ vh
    S = SC[:, 0].astype(F32)
    C = SC[:, 1].astype(F32)
    return S, C, sj, cj


def rhs_tensor(sysm: System, t: float, y: np.ndarray) -> np.ndarray:
    """Kuramoto right-hand side of the tensor-core variant: the i-side finish
    cos(theta_i) S_i - sin(theta_i) C_i in binary32, then omega_i + coupling in
    binary64."""
    S, C, sj, cj = tensor_sums(sysm, y)
    coupling = cj * S - sj * C
    return sysm.params + coupling.astype(F64)


# --------------------------------------------------------------------------
# Pairwise definitions (Eq. LCO, Eq. Kuramoto, Eq. CC) for brute-force pins.
# --------------------------------------------------------------------------

def pairwise_coupling(sysm: System, y: np.ndarray, dtype=np.longdouble) -> np.ndarray:
    """sum_j w_ij G_ij(X_i, X_j) for the coupled component, summed pair by pair
    in ``dtype`` (long double by default).  Returns shape [N]."""
    N = sysm.N
    Y = np.asarray(y, dtype=F64).reshape(sysm.d, N).astype(dtype)
    W = (sysm.s.astype(F64)[:, None] * sysm.q.astype(F64)).astype(dtype)
    x = Y[0]
    out = np.zeros(N, dtype=dtype)
    for i in range(N):
        acc = dtype(0)
        for j in range(N):
            if sysm.kind == "kuramoto":
                gij = np.sin(x[j] - x[i])
            elif sysm.kind == "lco_paper":
                gij = x[j] - x[i]
            elif sysm.kind == "lco_cfg":
                gij = x[j]
            else:
                gij = np.arctan(x[j] - x[i])
            acc += W[i, j] * gij
        out[i] = acc
    if sysm.kind == "circadian":
        g = sysm.globals
        th = sysm.theta_h.astype(dtype)
        x2 = Y[1]
        out = (dtype(g["k0"]) * th * dtype(g["a"]) / (th + x2 ** 4)) * out
    return out


def agent_term(sysm: System, y: np.ndarray) -> np.ndarray:
    """F(X) alone in binary64, shape [d, N] (used with pairwise_coupling)."""
    N = sysm.N
    Y = np.asarray(y, dtype=F64).reshape(sysm.d, N)
    out = np.zeros((sysm.d, N))
    if sysm.kind == "kuramoto":
        out[0] = sysm.params
    elif sysm.kind == "lco_cfg":
        out[0] = Y[1]
        out[1] = -(sysm.params ** 2) * Y[0]
    elif sysm.kind == "lco_paper":
        out[0] = Y[1]
        out[1] = -Y[0]
    else:
        g = sysm.globals
        x1, x2, x3, x4 = Y
        th = sysm.theta_h
        out[0] = g["k0"] * th / (th + x2 ** 4) * (g["a"] * x1 ** 2 + 1) - sysm.params * x1
        out[1] = g["k2"] * (x1 - x2)
        out[2] = x3 * (1 - x3 ** 2 / 3) - x4 + g["I0"] * (1 - g["k3"] ** 2 / (g["k3"] ** 2 + x1 ** 2))
        out[3] = g["eps"] * (x3 + g["b"] - g["c"] * x4)
    return out


COUPLED_COMPONENT = {"lco_cfg": 1, "lco_paper": 0, "kuramoto": 0, "circadian": 0}
