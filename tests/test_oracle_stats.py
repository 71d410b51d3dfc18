"""Pins of the oracle's per-pair statistics (CPU only).

Each statistic is checked against something other than itself: closed forms,
invariants, brute-force counts on tiny inputs, identities between tests, and
SciPy's per-pair routines applied to the arrays left after pairwise deletion
(Sec. 3.2). The paper prints no worked example; tests/golden holds small
hand-derived cases (each with its derivation).
"""
import itertools
import json
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_00448_gb300 import synth

st = pytest.importorskip("scipy.stats")
NAN = float("nan")
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def cohort_from_rows(rows, types, nlev):
    X = np.array(rows, dtype=np.float64)
    return X, np.array(types, np.uint8), np.array(nlev, np.int32)


def deleted(x, y, ctx=None):
    keep = ~np.isnan(x) & ~np.isnan(y)
    if ctx is not None:
        keep &= ctx.astype(bool)
    return x[keep], y[keep]


# ---------------------------------------------------------------- Pearson ----

def test_pearson_vs_scipy_after_deletion():
    coh = synth.small_cohort(1, n_cont=10, n_cat=0, S=200, miss=0.3)
    X = coh["X"]
    r, p, n = O.run("pearson", X, NAN, coh["vtype"], coh["nlev"], coh["cont"])
    for i, j in itertools.combinations(range(10), 2):
        a, b = deleted(X[i], X[j])
        assert n[i, j] == len(a)
        ref = st.pearsonr(a, b)
        assert abs(r[i, j] - ref.statistic) < 1e-13
        assert abs(p[i, j] - ref.pvalue) <= 1e-9 * ref.pvalue + 1e-300
    assert np.array_equal(r, r.T, equal_nan=True) and np.array_equal(n, n.T)


def test_pearson_exact_linear_columns_any_deletion():
    rng = np.random.default_rng(3)
    x = rng.integers(-50, 50, 400).astype(float)
    rows = [x, 2 * x + 3, -x + 7, x.copy()]
    X = np.array(rows)
    for k in range(4):
        X[k, rng.random(400) < 0.35] = np.nan
    vt = np.zeros(4, np.uint8)
    r, p, n = O.run("pearson", X, NAN, vt, np.zeros(4, np.int32), [0, 1, 2, 3])
    assert abs(r[0, 1] - 1) < 1e-14 and abs(r[0, 2] + 1) < 1e-14 and abs(r[1, 2] + 1) < 1e-14
    assert p[0, 1] < 1e-300 and p[0, 2] < 1e-300


def test_pearson_shift_scale_invariance():
    coh = synth.small_cohort(2, n_cont=6, n_cat=0, S=150, miss=0.25)
    X = coh["X"]
    r1, p1, _ = O.run("pearson", X, NAN, coh["vtype"], coh["nlev"], coh["cont"])
    X2 = X * np.array([[3.0], [0.5], [7.0], [1.0], [2.0], [0.25]]) + 1000.0
    r2, p2, _ = O.run("pearson", X2, NAN, coh["vtype"], coh["nlev"], coh["cont"])
    assert np.nanmax(np.abs(r1 - r2)) < 1e-11


def test_pearson_edge_counts_and_constant():
    X = np.array([[1.0, 2.0, NAN, 4.0, 5.0],
                  [2.0, NAN, 3.0, 1.0, 9.0],
                  [NAN, NAN, 1.0, NAN, NAN],
                  [5.0, 5.0, 5.0, 5.0, 5.0],
                  [1.0, 4.0, 2.0, NAN, NAN]])
    vt = np.zeros(5, np.uint8)
    r, p, n = O.run("pearson", X, NAN, vt, np.zeros(5, np.int32), [0, 1, 2, 3, 4])
    assert n[0, 1] == 3 and not math.isnan(r[0, 1]) and not math.isnan(p[0, 1])
    assert n[0, 2] == 0 and math.isnan(r[0, 2]) and math.isnan(p[0, 2])       # n <= 1
    assert n[1, 2] == 1 and math.isnan(r[1, 2])
    assert n[0, 4] == 2 and abs(abs(r[0, 4]) - 1) < 1e-15 and math.isnan(p[0, 4])  # n == 2: p NaN
    assert math.isnan(r[0, 3]) and math.isnan(p[0, 3])                          # constant column


# --------------------------------------------------------------- Spearman ----

def test_spearman_vs_scipy_and_rank_identities():
    coh = synth.small_cohort(3, n_cont=8, n_cat=0, S=250, miss=0.3, ties=True)
    X = coh["X"]
    rho, p, n = O.run("spearman", X, NAN, coh["vtype"], coh["nlev"], coh["cont"])
    for i, j in itertools.combinations(range(8), 2):
        a, b = deleted(X[i], X[j])
        ref = st.spearmanr(a, b)
        assert abs(rho[i, j] - ref.statistic) < 1e-13
        assert abs(p[i, j] - ref.pvalue) <= 1e-9 * ref.pvalue + 1e-300
        # equals Pearson of the tie-averaged ranks
        ra, rb = st.rankdata(a), st.rankdata(b)
        assert abs(rho[i, j] - st.pearsonr(ra, rb).statistic) < 1e-13
        ints = O.pair_ints("spearman", X, NAN, coh["vtype"], coh["nlev"], i, j)
        assert ints[0] == len(a)
        assert ints[1] == int(np.sum((2 * ra).astype(np.int64) * (2 * rb).astype(np.int64)))
        assert ints[2] == int(np.sum((2 * ra).astype(np.int64) ** 2))


def test_spearman_monotone_invariance_bit_exact():
    coh = synth.small_cohort(4, n_cont=5, n_cat=0, S=120, miss=0.2, ties=True)
    X = coh["X"]
    X2 = X.copy()
    X2[0] = np.exp(X[0] / 5.0)
    X2[1] = X[1] ** 3 + 10
    X2[2] = 1.0 / (1e3 - X[2])           # increasing for X < 1e3
    for i, j in itertools.combinations(range(5), 2):
        a = O.pair_ints("spearman", X, NAN, coh["vtype"], coh["nlev"], i, j)
        b = O.pair_ints("spearman", X2, NAN, coh["vtype"], coh["nlev"], i, j)
        assert np.array_equal(a, b)


def test_spearman_no_ties_closed_form_and_reversal():
    rng = np.random.default_rng(5)
    x = rng.permutation(60).astype(float)
    y = rng.permutation(60).astype(float)
    X = np.array([x, y, -x])
    vt = np.zeros(3, np.uint8)
    rho, p, n = O.run("spearman", X, NAN, vt, np.zeros(3, np.int32), [0, 1, 2])
    d = st.rankdata(x) - st.rankdata(y)
    nn = 60
    assert abs(rho[0, 1] - (1 - 6 * np.sum(d * d) / (nn * (nn * nn - 1)))) < 1e-14
    assert abs(rho[0, 2] + 1.0) < 1e-15 and p[0, 2] < 1e-250


# ------------------------------------------------------------ chi-squared ----

def test_chi2_vs_scipy_and_yates():
    coh = synth.small_cohort(6, n_cont=0, n_cat=6, S=300, miss=0.2, lev_lo=2, lev_hi=4, binary_cats=3)
    X = coh["X"]
    for yates in (0, 1):
        chi, p, n = O.run("chi2", X, NAN, coh["vtype"], coh["nlev"], coh["cat"], yates=yates)
        for i, j in itertools.combinations(range(6), 2):
            a, b = deleted(X[i], X[j])
            la = [g for g in range(coh["nlev"][i]) if np.any(X[i] == g)]
            lb = [h for h in range(coh["nlev"][j]) if np.any(X[j] == h)]
            T = np.array([[np.sum((a == g) & (b == h)) for h in lb] for g in la])
            if (T.sum(axis=1) == 0).any() or (T.sum(axis=0) == 0).any():
                assert math.isnan(chi[i, j])
                continue
            ref = st.chi2_contingency(T, correction=bool(yates))
            assert chi[i, j] == pytest.approx(ref.statistic, rel=1e-12, abs=1e-13)
            assert p[i, j] == pytest.approx(ref.pvalue, rel=1e-10)
        assert np.allclose(chi, chi.T, rtol=1e-14, atol=0, equal_nan=True)


def test_chi2_product_of_margins_and_2x2_closed_form():
    # table [[2,4],[3,6]] = outer((6,9),(5,10))/15: chi2 = 0 exactly
    a = [0] * 6 + [1] * 9
    b = [0] * 2 + [1] * 4 + [0] * 3 + [1] * 6
    X = np.array([a, b], float)
    vt = np.ones(2, np.uint8)
    nl = np.array([2, 2], np.int32)
    chi, p, n = O.run("chi2", X, NAN, vt, nl, [0, 1])
    assert chi[0, 1] == 0.0 and p[0, 1] == 1.0
    # 2x2 closed form n (ad - bc)^2 / ((a+b)(c+d)(a+c)(b+d))
    A, B, Cc, D = 7, 3, 2, 9
    a = [0] * (A + B) + [1] * (Cc + D)
    b = [0] * A + [1] * B + [0] * Cc + [1] * D
    chi, p, n = O.run("chi2", np.array([a, b], float), NAN, vt, nl, [0, 1])
    N = A + B + Cc + D
    ref = N * (A * D - B * Cc) ** 2 / ((A + B) * (Cc + D) * (A + Cc) * (B + D))
    assert chi[0, 1] == pytest.approx(ref, rel=1e-14)
    assert p[0, 1] == pytest.approx(math.erfc(math.sqrt(ref / 2)), rel=1e-12)


def test_chi2_edge_rules():
    # level 2 of var 0 exists only where var 1 is missing -> emptied -> NaN
    X = np.array([[0, 1, 2, 0, 1, 2, 0, 1],
                  [0, 1, NAN, 1, 0, NAN, 1, 0],
                  [0, 0, 0, 0, 0, 0, 0, 0]], float)
    vt = np.ones(3, np.uint8)
    nl = np.array([3, 2, 1], np.int32)
    chi, p, n = O.run("chi2", X, NAN, vt, nl, [0, 1, 2])
    assert math.isnan(chi[0, 1]) and n[0, 1] == 6
    # one present level: chi2 = 0, p NaN
    assert chi[0, 2] == 0.0 and math.isnan(p[0, 2])


# --------------------------------------------------------- ANOVA / t-tests ----

def _groups(x, lab):
    return [x[lab == g] for g in np.unique(lab)]


def test_anova_welch_student_vs_scipy():
    coh = synth.small_cohort(7, n_cont=6, n_cat=5, S=300, miss=0.2, lev_lo=2, lev_hi=5, binary_cats=2)
    X = coh["X"]
    F, pF, nF = O.run("anova", X, NAN, coh["vtype"], coh["nlev"], coh["cat"], coh["cont"])
    for ia, a in enumerate(coh["cat"]):
        for ib, j in enumerate(coh["cont"]):
            lab, x = deleted(X[a], X[j])
            ref = st.f_oneway(*_groups(x, lab))
            assert F[ia, ib] == pytest.approx(ref.statistic, rel=1e-11)
            assert pF[ia, ib] == pytest.approx(ref.pvalue, rel=1e-9)
    bins = coh["cat"][:2]
    for welch in (1, 0):
        t, pt, nt = O.run("ttest", X, NAN, coh["vtype"], coh["nlev"], bins, coh["cont"], welch=welch)
        for ia, a in enumerate(bins):
            for ib, j in enumerate(coh["cont"]):
                lab, x = deleted(X[a], X[j])
                if min((lab == 0).sum(), (lab == 1).sum()) < 2:   # Sec. 3.5.5: undefined
                    assert math.isnan(t[ia, ib]) and math.isnan(pt[ia, ib])
                    continue
                ref = st.ttest_ind(x[lab == 0], x[lab == 1], equal_var=not welch)
                assert t[ia, ib] == pytest.approx(ref.statistic, rel=1e-11)
                assert pt[ia, ib] == pytest.approx(ref.pvalue, rel=1e-9)


def test_anova_two_groups_equals_student_t_squared():
    coh = synth.small_cohort(8, n_cont=5, n_cat=2, S=200, miss=0.2, binary_cats=2)
    X = coh["X"]
    F, pF, _ = O.run("anova", X, NAN, coh["vtype"], coh["nlev"], coh["cat"], coh["cont"])
    t, pt, _ = O.run("ttest", X, NAN, coh["vtype"], coh["nlev"], coh["cat"], coh["cont"], welch=0)
    assert np.allclose(F, t * t, rtol=1e-12, atol=0)
    assert np.allclose(pF, pt, rtol=1e-11, atol=0)


def test_welch_equals_student_for_equal_group_sizes():
    rng = np.random.default_rng(9)
    lab = np.array([0] * 40 + [1] * 40, float)
    x = rng.normal(size=80) * np.where(lab == 0, 1.0, 3.0)
    X = np.array([lab, x])
    vt = np.array([1, 0], np.uint8)
    nl = np.array([2, 0], np.int32)
    tw, _, _ = O.run("ttest", X, NAN, vt, nl, [0], [1], welch=1)
    ts, _, _ = O.run("ttest", X, NAN, vt, nl, [0], [1], welch=0)
    assert tw[0, 0] == pytest.approx(ts[0, 0], rel=1e-14)


def test_anova_t_large_offset_against_exact_rationals():
    """F and t are shift-invariant; with a common offset 10^4 times the spread and
    group means 10^-5 spread apart, the oracle still matches F and t^2 computed
    in exact rational arithmetic (the inputs are multiples of 2^-8)."""
    from fractions import Fraction as Fr
    rng = np.random.default_rng(21)
    n = 3000
    lab = rng.integers(0, 3, n).astype(float)
    y = 57403.0 + np.round(rng.normal(size=n) * 7.5 * 256) / 256
    y[lab == 1] += 2.0 ** -8                       # a mean shift far below the offset
    X = np.array([lab, lab % 2, y])
    vt = np.array([1, 1, 0], np.uint8)
    nl = np.array([3, 2, 0], np.int32)
    F, _, _ = O.run("anova", X, NAN, vt, nl, [0], [2])
    g = [[Fr(v) for v in y[lab == k]] for k in range(3)]
    tot = [v for gg in g for v in gg]
    m = sum(tot) / len(tot)
    mg = [sum(gg) / len(gg) for gg in g]
    ssb = sum(len(gg) * (mk - m) ** 2 for gg, mk in zip(g, mg))
    ssw = sum((v - mk) ** 2 for gg, mk in zip(g, mg) for v in gg)
    F_exact = (ssb / 2) / (ssw / (n - 3))
    assert abs(F[0, 0] - float(F_exact)) <= 1e-13 * float(F_exact)
    lab2 = lab % 2
    h = [[Fr(v) for v in y[lab2 == k]] for k in range(2)]
    mh = [sum(hh) / len(hh) for hh in h]
    vh = [sum((v - mk) ** 2 for v in hh) / (len(hh) - 1) for hh, mk in zip(h, mh)]
    for welch in (1, 0):
        t, _, _ = O.run("ttest", X, NAN, vt, nl, [1], [2], welch=welch)
        if welch:
            se2 = vh[0] / len(h[0]) + vh[1] / len(h[1])
        else:
            sp2 = (vh[0] * (len(h[0]) - 1) + vh[1] * (len(h[1]) - 1)) / (n - 2)
            se2 = sp2 * (Fr(1, len(h[0])) + Fr(1, len(h[1])))
        t2 = (mh[0] - mh[1]) ** 2 / se2
        assert math.copysign(1.0, t[0, 0]) == (1.0 if mh[0] > mh[1] else -1.0)
        assert abs(t[0, 0] ** 2 - float(t2)) <= 1e-13 * float(t2)


def test_anova_t_edge_rules():
    lab = np.array([0, 0, 0, 1, 1, 1, 2, 2], float)
    x_const_diff = np.array([1, 1, 1, 2, 2, 2, 3, 3], float)
    x_const_same = np.array([4, 4, 4, 4, 4, 4, 4, 4], float)
    x_lose_level = np.array([1, 2, 3, 4, 5, 6, NAN, NAN], float)
    X = np.array([lab, x_const_diff, x_const_same, x_lose_level])
    vt = np.array([1, 0, 0, 0], np.uint8)
    nl = np.array([3, 0, 0, 0], np.int32)
    F, p, n = O.run("anova", X, NAN, vt, nl, [0], [1, 2, 3])
    assert F[0, 0] == math.inf and p[0, 0] == 0.0
    assert math.isnan(F[0, 1]) and math.isnan(p[0, 1])
    assert math.isnan(F[0, 2]) and n[0, 2] == 6
    lab2 = np.array([0, 0, 0, 1, 1, 1], float)
    Xt = np.array([lab2, [1, 1, 1, 2, 2, 2], [1, 1, 1, 1, 1, 1], [1, 2, 3, 4, NAN, NAN]], float)
    vt2 = np.array([1, 0, 0, 0], np.uint8)
    nl2 = np.array([2, 0, 0, 0], np.int32)
    t, p, n = O.run("ttest", Xt, NAN, vt2, nl2, [0], [1, 2, 3], welch=1)
    assert t[0, 0] == -math.inf and p[0, 0] == 0.0          # both groups constant, means differ
    assert math.isnan(t[0, 1])                               # both constant, same value
    assert math.isnan(t[0, 2]) and n[0, 2] == 4              # group 1 has < 2 samples
    t, p, n = O.run("ttest", Xt, NAN, vt2, nl2, [0], [1], welch=0)
    assert math.isnan(t[0, 0])                               # Student: pooled SD 0


# ---------------------------------------------------------- MWU / Kruskal ----

def test_mwu_vs_scipy_asymptotic_and_exact():
    coh = synth.small_cohort(10, n_cont=6, n_cat=3, S=250, miss=0.2, ties=True, binary_cats=3)
    X = coh["X"]
    U, p, n = O.run("mwu", X, NAN, coh["vtype"], coh["nlev"], coh["cat"], coh["cont"], mwu_mode=2)
    for ia, a in enumerate(coh["cat"]):
        for ib, j in enumerate(coh["cont"]):
            lab, x = deleted(X[a], X[j])
            ref = st.mannwhitneyu(x[lab == 0], x[lab == 1], method="asymptotic", use_continuity=True)
            assert U[ia, ib] == ref.statistic
            assert p[ia, ib] == pytest.approx(ref.pvalue, rel=1e-10)
            ints = O.pair_ints("mwu", X, NAN, coh["vtype"], coh["nlev"], a, j)
            nn = ints[0]
            assert ints[3] + ints[5] == nn * (nn + 1)                  # sum of 2R = n(n+1)
            assert U[ia, ib] + (ints[2] * ints[4] - U[ia, ib]) == ints[2] * ints[4]
    rng = np.random.default_rng(11)
    for trial in range(20):
        n0, n1 = int(rng.integers(1, 8)), int(rng.integers(1, 30))
        x = rng.permutation(n0 + n1).astype(float) + 0.5
        lab = np.array([0] * n0 + [1] * n1, float)
        X2 = np.array([lab, x])
        vt = np.array([1, 0], np.uint8)
        nl = np.array([2, 0], np.int32)
        U2, p2, _ = O.run("mwu", X2, NAN, vt, nl, [0], [1], mwu_mode=0)
        ref = st.mannwhitneyu(x[lab == 0], x[lab == 1], method="exact")
        assert U2[0, 0] == ref.statistic
        assert p2[0, 0] == pytest.approx(ref.pvalue, rel=1e-12)


def test_kruskal_vs_scipy_and_mwu_identity():
    coh = synth.small_cohort(12, n_cont=6, n_cat=4, S=250, miss=0.2, ties=True, lev_lo=2, lev_hi=5)
    X = coh["X"]
    H, p, n = O.run("kruskal", X, NAN, coh["vtype"], coh["nlev"], coh["cat"], coh["cont"])
    for ia, a in enumerate(coh["cat"]):
        for ib, j in enumerate(coh["cont"]):
            lab, x = deleted(X[a], X[j])
            ref = st.kruskal(*_groups(x, lab))
            assert H[ia, ib] == pytest.approx(ref.statistic, rel=1e-11)
            assert p[ia, ib] == pytest.approx(ref.pvalue, rel=1e-10)
    # k = 2 without continuity correction: H (tie-corrected) = z_MWU^2
    coh2 = synth.small_cohort(13, n_cont=4, n_cat=2, S=200, miss=0.2, ties=True, binary_cats=2)
    X = coh2["X"]
    H, _, _ = O.run("kruskal", X, NAN, coh2["vtype"], coh2["nlev"], coh2["cat"], coh2["cont"])
    U, pu, _ = O.run("mwu", X, NAN, coh2["vtype"], coh2["nlev"], coh2["cat"], coh2["cont"],
                     mwu_mode=2, mwu_cc=0)
    z = np.array([st.norm.isf(v / 2) for v in pu.ravel()]).reshape(pu.shape)
    assert np.allclose(H, z * z, rtol=1e-8)


def _exact_kruskal(lab, y, k):
    """Kruskal-Wallis H (Sec. 3.5.8) in exact rational arithmetic: tie-averaged
    ranks as halves of integers, H0 = 12/(n(n+1)) sum R_g^2/n_g - 3(n+1), divided
    by 1 - sum(t^3 - t)/(n^3 - n)."""
    from fractions import Fraction as Fr
    n = len(y)
    order = np.argsort(y, kind="stable")
    ys = y[order]
    twice_rank = np.empty(n, dtype=np.int64)      # 2R = (first + last) positions, 1-based
    tie = 0
    i = 0
    while i < n:
        j = i
        while j + 1 < n and ys[j + 1] == ys[i]:
            j += 1
        twice_rank[order[i:j + 1]] = (i + 1) + (j + 1)
        t = j - i + 1
        tie += t ** 3 - t
        i = j + 1
    h0 = Fr(0)
    for g in range(k):
        sel = lab == g
        R2 = int(twice_rank[sel].sum())           # 2 R_g, an exact integer
        h0 += Fr(R2 * R2, 4 * int(sel.sum()))
    h0 = Fr(12, n * (n + 1)) * h0 - 3 * (n + 1)
    return h0 / (1 - Fr(tie, n ** 3 - n))


def test_kruskal_large_n_small_h_against_exact_rationals():
    """At n = 50,000 with groups from one distribution (H of order 1, the sums
    R_g^2 / n_g agreeing to ~1e-10 relative before the 3(n+1) subtraction), with
    heavy ties: the oracle's H equals the exact rational H to 1e-12 relative; for
    two groups the same holds for the Mann-Whitney z^2 without continuity
    correction, which equals H."""
    rng = np.random.default_rng(27)
    n = 50_000
    y = np.round(rng.normal(size=n), 1)          # about 70 distinct values: ties everywhere
    for k in (4, 2):
        lab = rng.integers(0, k, n).astype(float)
        X = np.array([lab, y])
        vt = np.array([1, 0], np.uint8)
        nl = np.array([k, 0], np.int32)
        H, _, nn = O.run("kruskal", X, NAN, vt, nl, [0], [1])
        assert nn[0, 0] == n
        Hx = _exact_kruskal(lab, y, k)
        assert 0.0 < float(Hx) < 20.0
        assert abs(H[0, 0] - float(Hx)) <= 1e-12 * float(Hx), (k, H[0, 0], float(Hx))
        if k == 2:
            U, pu, _ = O.run("mwu", X, NAN, vt, nl, [0], [1], mwu_mode=2, mwu_cc=0)
            from fractions import Fraction as Fr
            n0 = int((lab == 0).sum())
            n1 = n - n0
            # z^2 = (U0 - n0 n1 / 2)^2 / sigma^2 with the tie-corrected variance,
            # exactly equal to H
            assert abs(st.norm.isf(pu[0, 0] / 2) ** 2 - float(Hx)) <= 1e-8 * float(Hx)
            assert Fr(U[0, 0]) * 2 == int(round(2 * U[0, 0]))


def test_kruskal_mwu_edge_rules():
    lab = np.array([0, 0, 0, 1, 1, 1], float)
    tied = np.array([2, 2, 2, 2, 2, 2], float)
    lose = np.array([1, 2, 3, NAN, NAN, NAN], float)
    X = np.array([lab, tied, lose])
    vt = np.array([1, 0, 0], np.uint8)
    nl = np.array([2, 0, 0], np.int32)
    H, p, n = O.run("kruskal", X, NAN, vt, nl, [0], [1, 2])
    assert math.isnan(H[0, 0]) and math.isnan(H[0, 1]) and n[0, 1] == 3
    U, p, n = O.run("mwu", X, NAN, vt, nl, [0], [1, 2], mwu_mode=2)
    assert U[0, 0] == 4.5 and math.isnan(p[0, 0])            # all tied: zero variance
    assert math.isnan(U[0, 1])                               # a group emptied


# --------------------------------------------------- counts by brute force ----

def test_counts_and_tables_brute_force_exhaustive_masks():
    """Every missingness pattern of two 8-sample variables: n and the table."""
    S = 8
    g = np.array([0, 1, 2, 0, 1, 2, 1, 0], float)
    h = np.array([1, 0, 1, 1, 0, 0, 1, 0], float)
    vt = np.ones(2, np.uint8)
    nl = np.array([3, 2], np.int32)
    for ma in range(0, 2 ** S, 7):
        for mb in range(0, 2 ** S, 11):
            X = np.array([g, h])
            X[0, [(ma >> s) & 1 == 1 for s in range(S)]] = NAN
            X[1, [(mb >> s) & 1 == 1 for s in range(S)]] = NAN
            T = O.pair_ints("chi2", X, NAN, vt, nl, 0, 1).reshape(3, 2)
            ref = np.zeros((3, 2), np.int64)
            for s in range(S):
                if not (np.isnan(X[0, s]) or np.isnan(X[1, s])):
                    ref[int(X[0, s]), int(X[1, s])] += 1
            assert np.array_equal(T, ref)


def test_listwise_equals_pairwise_without_missing():
    coh = synth.small_cohort(14, n_cont=5, n_cat=3, S=100, miss=0.0, binary_cats=1)
    X = coh["X"]
    r, _, n = O.run("pearson", X, NAN, coh["vtype"], coh["nlev"], coh["cont"])
    assert (n == 100).all()
    assert np.allclose(r, np.corrcoef(X[coh["cont"]]), atol=1e-14)


def test_sample_context_equals_submatrix():
    coh = synth.small_cohort(15, n_cont=5, n_cat=3, S=160, miss=0.2, binary_cats=1)
    X = coh["X"]
    ctx = (np.arange(160) % 3 != 0).astype(np.uint8)
    for test, va, vb in [("pearson", coh["cont"], None), ("kruskal", coh["cat"], coh["cont"]),
                         ("chi2", coh["cat"], None)]:
        a = O.run(test, X, NAN, coh["vtype"], coh["nlev"], va, vb, ctx=ctx)
        b = O.run(test, X[:, ctx == 1], NAN, coh["vtype"], coh["nlev"], va, vb)
        for u, v in zip(a, b):
            assert np.array_equal(u, v, equal_nan=True)


def test_validation_errors():
    X = np.array([[0, 1, 3], [1.0, 2.0, 3.0]])
    vt = np.array([1, 0], np.uint8)
    assert O.validate(X, NAN, vt, np.array([3, 0], np.int32)) == O.E_LABEL
    assert O.validate(np.array([[0, 1, 0.5], [1, 2, 3.0]]), NAN, vt, np.array([3, 0], np.int32)) == O.E_LABEL
    assert O.validate(np.array([[0, 1, 2], [1, np.inf, 3.0]]), NAN, vt, np.array([3, 0], np.int32)) == O.E_NONFINITE
    assert O.validate(np.array([[0, 1, 2], [1, -99.0, 3.0]]), -99.0, vt, np.array([3, 0], np.int32)) == O.OK
    with pytest.raises(O.OracleError):
        O.run("ttest", np.array([[0, 1, 2.0], [1, 2, 3.0]]), NAN, vt, np.array([3, 0], np.int32), [0], [1])


def test_pvalues_uniform_under_independence():
    rng = np.random.default_rng(21)
    X = rng.normal(size=(40, 300))
    X[rng.random(X.shape) < 0.2] = np.nan
    _, p, _ = O.run("pearson", X, NAN, np.zeros(40, np.uint8), np.zeros(40, np.int32), np.arange(40))
    pv = p[np.triu_indices(40, 1)]
    assert st.kstest(pv, "uniform").pvalue > 1e-3


def test_golden_cases():
    for name in sorted(os.listdir(GOLDEN)):
        if not name.endswith(".json"):
            continue
        case = json.load(open(os.path.join(GOLDEN, name)))
        X = np.array([[NAN if v is None else v for v in row] for row in case["X"]], float)
        kw = case.get("options", {})
        stat, p, n = O.run(case["test"], X, NAN, np.array(case["vtype"], np.uint8),
                           np.array(case["nlev"], np.int32), case["vars_a"], case.get("vars_b"), **kw)
        ia, ib = case["pair"]
        assert n[ia, ib] == case["n"], name
        assert stat[ia, ib] == pytest.approx(case["stat"], rel=case.get("rtol", 1e-12)), name
        if case.get("p") is not None:
            assert p[ia, ib] == pytest.approx(case["p"], rel=case.get("rtol", 1e-12)), name
