"""Pins of the oracle's tensor-core variant (the reference of the shared-K
ensembles): the bfloat16 split of a binary32 value, the three split products
summed exactly, and the Kuramoto right-hand side built on them.

* the split against torch's own bfloat16 conversion and its 2^-16 bound;
* the split sums against a brute-force sum of the three products in exact
  rational arithmetic (tiny N), rounded once to binary32;
* the right-hand side against the binary64 one of the same stored weights,
  within a bound derived from the split (about 3 2^-16 sum_j |K_ij|), tight
  enough that a dropped split term, an unsplit operand or a sign error in the
  i-side finish fails it (planted below in copies of the oracle's routine);
* the solver's tensor variant against the closed form at K = 0.
"""

from fractions import Fraction

import numpy as np
import pytest

import workloads as W
from oracle import bs3 as obs3
from oracle import exact, metrics, models

U16 = 2.0 ** -16
U24 = 2.0 ** -24


def _kuramoto(N, seed, scale=1.0):
    w = W.kuramoto(N, seed, t1=1.0)
    return w, models.make_system("kuramoto", N, w.params, np.asarray(w.coupling) * scale, "f32")


def test_split_is_torch_bf16_rounding_and_keeps_16_bits():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = (rng.standard_normal(20000) * np.exp(rng.uniform(-20, 20, 20000))).astype(np.float32)
    hi, lo = models.split_bf16(x)
    t_hi = torch.from_numpy(x).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(hi, t_hi)
    r = (x.astype(np.float64) - hi).astype(np.float32)        # exact: the residual fits binary32
    assert np.all(r.astype(np.float64) == x.astype(np.float64) - hi)
    np.testing.assert_array_equal(lo, torch.from_numpy(r).to(torch.bfloat16).to(torch.float64).numpy())
    assert np.all(np.abs(x - (hi + lo)) <= U16 * np.abs(x))


def test_split_sums_equal_exact_three_product_sums():
    w, sysm = _kuramoto(7, 3)
    rng = np.random.default_rng(5)
    y = rng.uniform(-40.0, 40.0, 7)
    S, C, sj, cj = models.tensor_sums(sysm, y)
    kh, kl = models.split_bf16(sysm.q.astype(np.float32))
    for vec, got in ((sj, S), (cj, C)):
        vh, vl = models.split_bf16(vec)
        for i in range(7):
            acc = Fraction(0)
            for j in range(7):
                a_h, a_l = Fraction(float(kh[i, j])), Fraction(float(kl[i, j]))
                b_h, b_l = Fraction(float(vh[j])), Fraction(float(vl[j]))
                acc += a_h * b_h + a_h * b_l + a_l * b_h
            assert Fraction(float(acc)) == acc        # the exact sum is a binary64 number here
            assert got[i] == np.float32(float(acc)), (i, got[i], float(acc))


def _bound_ratio(sysm, y, rhs_t):
    """max_i |rhs_t - rhs_DDD| / bound_i for the split's error bound."""
    ref = models.rhs(sysm, 0.0, y, ("D", "D", "D"))
    R = np.abs(sysm.q.astype(np.float64)).sum(axis=1)
    bound = 2.0 * 3.1 * U16 * R + 12.0 * U24 * R + 4 * np.finfo(np.float64).eps * np.abs(ref)
    return float(np.max(np.abs(rhs_t - ref) / bound))


@pytest.mark.parametrize("N,seed", [(64, 1), (300, 2)])
def test_tensor_rhs_within_split_bound_of_binary64(N, seed):
    w, sysm = _kuramoto(N, seed)
    y = np.random.default_rng(seed).uniform(0, 2 * np.pi, N)
    assert _bound_ratio(sysm, y, models.rhs_tensor(sysm, 0.0, y)) <= 1.0


def _planted_rhs(sysm, y, mistake):
    """Copies of the oracle's routine with one plausible mistake each."""
    F32, F64 = np.float32, np.float64
    kh, kl = models.split_bf16(sysm.q.astype(F32))
    th = np.asarray(y, dtype=F64)
    sj, cj = np.sin(th).astype(F32), np.cos(th).astype(F32)
    sh, sl = models.split_bf16(sj)
    ch, cl = models.split_bf16(cj)
    if mistake == "no_lo_hi":
        S = (kh @ sh + kh @ sl).astype(F32)
        C = (kh @ ch + kh @ cl).astype(F32)
    elif mistake == "unsplit_vector":
        S = (kh @ sh + kl @ sh).astype(F32)
        C = (kh @ ch + kl @ ch).astype(F32)
    elif mistake == "bf16_sums":
        from oracle.formats import round_bf16
        S = round_bf16((kh @ sh + kh @ sl + kl @ sh).astype(F32))
        C = round_bf16((kh @ ch + kh @ cl + kl @ ch).astype(F32))
    else:
        S = (kh @ sh + kh @ sl + kl @ sh).astype(F32)
        C = (kh @ ch + kh @ cl + kl @ ch).astype(F32)
    coupling = cj * S + sj * C if mistake == "finish_sign" else cj * S - sj * C
    return sysm.params + coupling.astype(F64)


@pytest.mark.parametrize("mistake", ["no_lo_hi", "unsplit_vector", "bf16_sums", "finish_sign"])
def test_planted_mistakes_break_the_bound(mistake):
    w, sysm = _kuramoto(300, 2)
    y = np.random.default_rng(2).uniform(0, 2 * np.pi, 300)
    assert _bound_ratio(sysm, y, _planted_rhs(sysm, y, "none")) <= 1.0
    assert _bound_ratio(sysm, y, _planted_rhs(sysm, y, mistake)) > 1.0


def test_tensor_solve_uncoupled_is_the_closed_form():
    w, sysm = _kuramoto(48, 4, scale=0.0)
    r = obs3.solve(sysm, 0.0, 3.0, w.y0, 1e-8, 1e-8, "tensor")
    assert r.status == obs3.OK
    ex = exact.kuramoto_uncoupled(w.y0, w.params, 3.0)
    assert metrics.normalized_final_error(ex, r.y, 48) < 1e-12
