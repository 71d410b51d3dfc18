"""Pins of the oracle's special functions (CPU only).

Closed forms (DLMF 8.17, 8.4; textbook t/F/chi-squared tails), symmetry, and
40-digit values from mpmath where it is installed.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O

RNG = np.random.default_rng(12345)


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.abs(a - b) / np.maximum(np.abs(b), 1e-300)


def test_ibeta_closed_forms():
    x = RNG.uniform(0.001, 0.999, 200)
    a = RNG.uniform(0.2, 60.0, 200)
    # I_x(a,1) = x^a ; I_x(1,b) = 1-(1-x)^b  (DLMF 8.17.5)
    assert rel(O.ibeta(a, 1.0, x), x ** a).max() < 1e-13
    assert rel(O.ibeta(1.0, a, x), -np.expm1(a * np.log1p(-x))).max() < 1e-13
    # I_{1/2}(a,a) = 1/2 (symmetry DLMF 8.17.4)
    assert rel(O.ibeta(a, a, 0.5), 0.5).max() < 1e-13
    # I_x(a,b) + I_{1-x}(b,a) = 1
    b = RNG.uniform(0.2, 60.0, 200)
    s = O.ibeta(a, b, x) + O.ibeta(b, a, 1.0 - x)
    assert np.abs(s - 1.0).max() < 1e-13


def test_student_t_closed_forms():
    t = np.concatenate([RNG.uniform(-30, 30, 100), [0.0, 1e-8, 1e3]])
    # df = 1 (Cauchy): p = 1 - 2 atan(|t|)/pi = 2 atan(1/|t|)/pi
    at = np.abs(t)
    p1 = np.where(at > 0, 2.0 * np.arctan(1.0 / np.where(at > 0, at, 1.0)) / np.pi, 1.0)
    assert rel(O.t_p2(t, 1.0), p1).max() < 1e-12
    # df = 2: p = 1 - |t| / sqrt(2 + t^2), written without cancellation
    r = np.sqrt(2.0 + t * t)
    p2 = 2.0 / (r * (r + at))
    assert rel(O.t_p2(t, 2.0), p2).max() < 1e-12


def test_chi2_f_closed_forms():
    x = np.concatenate([RNG.uniform(0, 80, 100), [1e-10, 200.0]])
    # chi2 df = 2: sf = exp(-x/2); df = 1: sf = erfc(sqrt(x/2))
    assert rel(O.chi2_sf(x, 2.0), np.exp(-x / 2)).max() < 1e-13
    e1 = np.array([math.erfc(math.sqrt(v / 2)) for v in x])
    assert rel(O.chi2_sf(x, 1.0), e1).max() < 1e-12
    # F(2, d2): sf = (d2 / (d2 + 2F))^(d2/2)
    F = RNG.uniform(0.0, 30.0, 100)
    d2 = RNG.integers(1, 500, 100).astype(float)
    assert rel(O.f_sf(F, 2.0, d2), (d2 / (d2 + 2 * F)) ** (d2 / 2)).max() < 1e-12
    # normal sf against the closed form erfc
    z = RNG.uniform(-8, 8, 100)
    assert rel(O.norm_sf(z), np.array([0.5 * math.erfc(v / math.sqrt(2)) for v in z])).max() < 1e-15


def test_special_edge_values():
    assert O.t_p2(np.inf, 10.0) == 0.0
    assert math.isnan(O.t_p2(np.nan, 10.0))
    assert O.f_sf(np.inf, 3.0, 10.0) == 0.0
    assert O.f_sf(0.0, 3.0, 10.0) == 1.0
    assert O.chi2_sf(0.0, 3.0) == 1.0
    assert math.isnan(O.chi2_sf(1.0, 0.0))
    assert O.corr_p(1.0, 10) == 0.0 and O.corr_p(-1.0, 10) == 0.0
    assert math.isnan(O.corr_p(0.3, 2))


def test_against_scipy():
    sp = pytest.importorskip("scipy.special")
    a = np.exp(RNG.uniform(np.log(0.5), np.log(2000), 300))
    b = np.exp(RNG.uniform(np.log(0.5), np.log(2000), 300))
    x = RNG.uniform(0.0, 1.0, 300)
    x = np.round(x * 2 ** 30) / 2 ** 30
    ours, ref = O.ibeta(a, b, x), sp.betainc(a, b, x)
    ok = ref > 1e-250
    assert (np.abs(ours - ref)[ok] <= 1e-11 * np.minimum(ref, 1 - ref + 1e-300)[ok] + 1e-300).all() or \
        rel(ours[ok], ref[ok]).max() < 1e-10
    aa = np.exp(RNG.uniform(np.log(0.5), np.log(200), 300))
    xx = aa * np.exp(RNG.normal(0, 0.5, 300))
    assert rel(O.gamma_q(aa, xx), sp.gammaincc(aa, xx)).max() < 1e-11


def test_against_mpmath_high_precision():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    rng = np.random.default_rng(99)
    worst = 0.0
    count = 0
    for _ in range(300):
        r = rng.random()
        if r < 0.4:
            a, b = float(np.exp(rng.uniform(0, np.log(60000)))), float(rng.integers(1, 12)) / 2
        elif r < 0.6:
            b, a = float(np.exp(rng.uniform(0, np.log(60000)))), float(rng.integers(1, 12)) / 2
        else:
            a, b = [float(np.exp(rng.uniform(np.log(0.5), np.log(60000)))) for _ in range(2)]
        m = a / (a + b)
        sd = math.sqrt(a * b / ((a + b) ** 2 * (a + b + 1)))
        x = m + 3 * sd * rng.normal()
        if not 0 < x < 1:
            continue
        x = round(x * 2 ** 30) / 2 ** 30          # x and 1-x both exact doubles
        if not 0 < x < 1:
            continue
        try:
            ex = mp.betainc(a, b, 0, x, regularized=True)
        except Exception:  # mpmath's own convergence limit
            continue
        if ex < 1e-250 or 1 - ex < 1e-250:
            continue
        count += 1
        ours = float(O.ibeta(a, b, x))
        err = abs(ours - float(ex)) / min(float(ex), float(1 - ex))
        # front-factor exponent carries ~eps*|log I| of rounding
        tol = 2e-12 + 8.9e-16 * abs(math.log(float(ex)))
        assert err < tol, (a, b, x, ours, float(ex))
        worst = max(worst, err)
    assert count > 150
    for _ in range(200):
        a = float(np.exp(rng.uniform(np.log(0.5), np.log(300))))
        x = float(a * np.exp(rng.normal(0, 0.6)))
        ex = mp.gammainc(a, x, mp.inf, regularized=True)
        if ex < 1e-250 or 1 - ex < 1e-250:
            continue
        ours = float(O.gamma_q(a, x))
        assert abs(ours - float(ex)) / min(float(ex), float(1 - ex)) < 2e-12 + 8.9e-16 * abs(math.log(float(ex)))


def test_mwu_exact_distribution_by_enumeration():
    """P(U >= u) for tiny groups equals counting all C(n, n0) splits."""
    from itertools import combinations
    for n0, n1 in [(1, 1), (2, 3), (3, 3), (4, 5), (2, 9), (6, 7), (7, 7)]:
        n = n0 + n1
        counts = {}
        total = 0
        for A in combinations(range(n), n0):
            sA = set(A)
            # U counts pairs (a in A, b in B) with a ranked above b
            U = sum(1 for a in A for b in range(n) if b not in sA and a > b)
            counts[U] = counts.get(U, 0) + 1
            total += 1
        for u in range(0, n0 * n1 + 2):
            ref = sum(c for k, c in counts.items() if k >= u) / total
            got = float(O.mwu_exact_sf(float(u), n0, n1))
            assert abs(got - ref) <= 1e-14 * max(ref, 1e-300) + 1e-300, (n0, n1, u, got, ref)
        # symmetry in the group sizes
        assert float(O.mwu_exact_sf(n0 * n1 / 2.0, n0, n1)) == pytest.approx(
            float(O.mwu_exact_sf(n0 * n1 / 2.0, n1, n0)), rel=1e-14)
