"""Fits the binary32 arctangent polynomial used by the pairwise circadian kernel.

atan(x) = x P(x^2) on [0, 1], P of degree DEG, found by Lawson's algorithm (reweighted
least squares converging to the minimax relative error) of x P(x^2) against arctan (binary64 reference),
then rounded to binary32.  |x| > 1 uses atan(x) = pi/2 - atan(1/x).
Prints the coefficients (c0 first) and the maximum error of the
binary32 Horner evaluation on a dense grid.  Run: python fit_atan.py
"""

import numpy as np

DEG = 8


def fit_minimax(deg, iters=400):
    """Lawson's iteratively reweighted least squares, which converges to the
    minimax polynomial: P(z) ~ atan(sqrt z)/sqrt z on [0, 1]."""
    m = 4000
    z = 0.5 - 0.5 * np.cos(np.pi * (np.arange(m) + 0.5) / m)
    x = np.sqrt(z)
    g = np.arctan(x) / x
    V = np.vander(z, deg + 1, increasing=True)
    w = np.full(m, 1.0 / m)
    for _ in range(iters):
        sw = np.sqrt(w)
        c, *_ = np.linalg.lstsq(V * sw[:, None], g * sw, rcond=None)
        e = np.abs(V @ c - g) / g
        w = w * e
        w /= w.sum()
    return c


def eval32(c32, x):
    x = np.asarray(x, dtype=np.float32)
    ax = np.abs(x)
    big = ax > 1
    t = np.where(big, np.float32(1) / np.where(big, ax, np.float32(1)), ax).astype(np.float32)
    zt = (t * t).astype(np.float32)
    p = np.float32(c32[-1])
    for cj in c32[-2::-1]:
        # fused multiply-add: one rounding of the exact p*z + c
        p = (p.astype(np.float64) * zt.astype(np.float64) + np.float64(cj)).astype(np.float32)
    r = (t * p).astype(np.float32)
    r = np.where(big, np.float32(np.pi / 2) - r, r).astype(np.float32)
    return np.copysign(r, x)


if __name__ == "__main__":
    c = fit_minimax(DEG)
    c32 = c.astype(np.float32)
    x = np.concatenate([np.linspace(-50, 50, 2000001), np.geomspace(1e-6, 1e4, 200001)]).astype(np.float32)
    ref = np.arctan(x.astype(np.float64))
    err = np.abs(eval32(c32, x).astype(np.float64) - ref)
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    print("coefficients c0..c%d:" % DEG)
    for v in c32:
        print("  %.9ef" % v)
    print("max abs err %.3e, max err in ulps %.2f" % (err.max(), (err / ulp).max()))
