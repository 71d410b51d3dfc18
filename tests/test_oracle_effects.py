"""Pins of the oracle's effect sizes (Table 2) and multiple-testing corrections
(Sec. 3.4), CPU only. Each is checked against an independent route: SciPy's
per-pair statistics and association measures on the arrays left after pairwise
deletion, identities between effect sizes and test statistics, sums of squares
formed directly from the groups, and SciPy's false-discovery-rate control.
"""
import math
import statistics

import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_00448_gb300 import synth

st = pytest.importorskip("scipy.stats")
contingency = pytest.importorskip("scipy.stats.contingency")
NAN = float("nan")


def deleted(x, y):
    keep = ~np.isnan(x) & ~np.isnan(y)
    return x[keep], y[keep]


@pytest.fixture(scope="module")
def coh():
    return synth.small_cohort(31, n_cont=7, n_cat=6, S=400, miss=0.2, lev_lo=2, lev_hi=5, binary_cats=2, ties=True)


def test_correlation_effects(coh):
    X = coh["X"]
    cont = coh["cont"]
    r2, _ = O.effects("pearson", X, NAN, coh["vtype"], coh["nlev"], cont)
    rho, _ = O.effects("spearman", X, NAN, coh["vtype"], coh["nlev"], cont)
    for ia, a in enumerate(cont):
        for ib, b in enumerate(cont):
            x, y = deleted(X[a], X[b])
            assert r2[ia, ib] == pytest.approx(st.pearsonr(x, y).statistic ** 2, rel=1e-12, abs=1e-15)
            assert rho[ia, ib] == pytest.approx(st.spearmanr(x, y).statistic, rel=1e-12, abs=1e-15)


def test_phi_and_cramers_v_against_association(coh):
    X = coh["X"]
    cats = coh["cat"]
    phi, V = O.effects("chi2", X, NAN, coh["vtype"], coh["nlev"], cats)
    for ia, a in enumerate(cats):
        for ib, b in enumerate(cats):
            x, y = deleted(X[a], X[b])
            la, lb = np.unique(x), np.unique(y)
            T = np.array([[np.sum((x == g) & (y == h)) for h in lb] for g in la])
            if min(T.shape) < 2:
                assert math.isnan(V[ia, ib])
                continue
            assert V[ia, ib] == pytest.approx(contingency.association(T, method="cramer"), rel=1e-12)
            # Pearson's contingency coefficient C = sqrt(chi2 / (chi2 + n)) gives phi^2 = C^2 / (1 - C^2)
            C = contingency.association(T, method="pearson")
            assert phi[ia, ib] == pytest.approx(math.sqrt(C * C / (1.0 - C * C)), rel=1e-10, abs=1e-14)


def test_single_category_gives_phi_zero_and_v_nan():
    rng = np.random.default_rng(3)
    a = np.zeros(50)
    b = rng.integers(0, 3, 50).astype(float)
    X = np.array([a, b])
    phi, V = O.effects("chi2", X, NAN, np.array([1, 1], np.uint8), np.array([1, 3], np.int32), [0, 1])
    assert phi[0, 1] == 0.0 and math.isnan(V[0, 1])


def test_cohens_d(coh):
    X = coh["X"]
    bins = coh["cat"][:2]
    for welch in (0, 1):
        d, _ = O.effects("ttest", X, NAN, coh["vtype"], coh["nlev"], bins, coh["cont"], welch=welch)
        for ia, a in enumerate(bins):
            for ib, j in enumerate(coh["cont"]):
                lab, x = deleted(X[a], X[j])
                g0, g1 = list(x[lab == 0]), list(x[lab == 1])
                if welch:
                    s = math.sqrt((statistics.variance(g0) + statistics.variance(g1)) / 2)
                    ref = (statistics.fmean(g0) - statistics.fmean(g1)) / s
                else:
                    # Student: d = t sqrt(1/n0 + 1/n1) with SciPy's pooled t
                    t = st.ttest_ind(g0, g1, equal_var=True).statistic
                    ref = t * math.sqrt(1 / len(g0) + 1 / len(g1))
                assert d[ia, ib] == pytest.approx(ref, rel=1e-10)


def test_ttest_degrees_of_freedom_match_scipy(coh):
    """The t-test's second output is the degrees of freedom of its t
    distribution: SciPy's Welch-Satterthwaite df (Welch) and n0 + n1 - 2
    (Student) on the arrays left after deletion; and p is the two-sided t tail
    at that df."""
    X = coh["X"]
    bins = coh["cat"][:2]
    for welch in (0, 1):
        _, df = O.effects("ttest", X, NAN, coh["vtype"], coh["nlev"], bins, coh["cont"], welch=welch)
        t, p, _ = O.run("ttest", X, NAN, coh["vtype"], coh["nlev"], bins, coh["cont"], welch=welch)
        for ia, a in enumerate(bins):
            for ib, j in enumerate(coh["cont"]):
                lab, x = deleted(X[a], X[j])
                g0, g1 = x[lab == 0], x[lab == 1]
                ref = st.ttest_ind(g0, g1, equal_var=not welch)
                assert df[ia, ib] == pytest.approx(float(ref.df), rel=1e-12)
                assert p[ia, ib] == pytest.approx(2 * st.t.sf(abs(t[ia, ib]), float(ref.df)), rel=1e-10)


def test_welch_d_equals_student_d_for_equal_groups():
    rng = np.random.default_rng(5)
    lab = np.array([0] * 30 + [1] * 30, float)
    x = rng.normal(size=60) * np.where(lab == 0, 1.0, 2.5) + lab
    X = np.array([lab, x])
    vt, nl = np.array([1, 0], np.uint8), np.array([2, 0], np.int32)
    dw, _ = O.effects("ttest", X, NAN, vt, nl, [0], [1], welch=1)
    ds, _ = O.effects("ttest", X, NAN, vt, nl, [0], [1], welch=0)
    assert dw[0, 0] == pytest.approx(ds[0, 0], rel=1e-13)
    # constant groups: Cohen's d undefined (Sec. 3.5.5)
    X2 = np.array([lab, np.where(lab == 0, 1.0, 2.0)])
    dw2, _ = O.effects("ttest", X2, NAN, vt, nl, [0], [1], welch=1)
    assert math.isnan(dw2[0, 0])


def test_mwu_r_from_scipy_z(coh):
    X = coh["X"]
    bins = coh["cat"][:2]
    r, _ = O.effects("mwu", X, NAN, coh["vtype"], coh["nlev"], bins, coh["cont"])
    for ia, a in enumerate(bins):
        for ib, j in enumerate(coh["cont"]):
            lab, x = deleted(X[a], X[j])
            p = st.mannwhitneyu(x[lab == 0], x[lab == 1], use_continuity=False, method="asymptotic").pvalue
            z = st.norm.isf(p / 2)
            assert r[ia, ib] == pytest.approx(z / math.sqrt(len(x)), rel=1e-9)


def test_anova_partial_eta2(coh):
    X = coh["X"]
    cats, conts = coh["cat"], coh["cont"]
    eta, _ = O.effects("anova", X, NAN, coh["vtype"], coh["nlev"], cats, conts)
    F_or, _, _ = O.run("anova", X, NAN, coh["vtype"], coh["nlev"], cats, conts)
    for ia, a in enumerate(cats):
        for ib, j in enumerate(conts):
            if math.isnan(F_or[ia, ib]):             # a present level lost all its samples
                assert math.isnan(eta[ia, ib])
                continue
            lab, x = deleted(X[a], X[j])
            groups = [x[lab == g] for g in np.unique(lab)]
            sst = len(x) * np.var(x)
            ssw = sum(len(g) * np.var(g) for g in groups)
            assert eta[ia, ib] == pytest.approx(1.0 - ssw / sst, rel=1e-10, abs=1e-14)
            F = st.f_oneway(*groups).statistic
            d1, d2 = len(groups) - 1, len(x) - len(groups)
            assert eta[ia, ib] == pytest.approx(F * d1 / (F * d1 + d2), rel=1e-10, abs=1e-14)


def test_kruskal_eta2(coh):
    X = coh["X"]
    cats, conts = coh["cat"], coh["cont"]
    eta, _ = O.effects("kruskal", X, NAN, coh["vtype"], coh["nlev"], cats, conts)
    H_or, _, _ = O.run("kruskal", X, NAN, coh["vtype"], coh["nlev"], cats, conts)
    for ia, a in enumerate(cats):
        for ib, j in enumerate(conts):
            if math.isnan(H_or[ia, ib]):
                assert math.isnan(eta[ia, ib])
                continue
            lab, x = deleted(X[a], X[j])
            groups = [x[lab == g] for g in np.unique(lab)]
            H = st.kruskal(*groups).statistic
            k, n = len(groups), len(x)
            assert eta[ia, ib] == pytest.approx((H - k + 1) / (n - k), rel=1e-10, abs=1e-13)
    # n <= k: undefined (Sec. 3.5.8)
    Xs = np.array([[0, 1, 2], [1.0, 2.0, 3.5]])
    e, _ = O.effects("kruskal", Xs, NAN, np.array([1, 0], np.uint8), np.array([3, 0], np.int32), [0], [1])
    assert math.isnan(e[0, 0])


def test_effects_nan_where_statistic_is_nan():
    X = np.array([[0, 0, 1, 1, np.nan], [1.0, np.nan, np.nan, 2.0, 3.0]])
    e, _ = O.effects("ttest", X, NAN, np.array([1, 0], np.uint8), np.array([2, 0], np.int32), [0], [1])
    assert math.isnan(e[0, 0])                     # a group of one sample


def test_bh_by_against_scipy():
    rng = np.random.default_rng(11)
    for m in (1, 2, 7, 100, 1000):
        p = rng.random(m) ** 3
        p[rng.random(m) < 0.2] = p[0]                # ties
        for method in ("bh", "by"):
            ours = O.adjust(p.reshape(1, -1), method, symmetric=False).ravel()
            ref = st.false_discovery_control(p, method=method)
            assert np.allclose(ours, ref, rtol=1e-13, atol=0), (m, method)


def test_symmetric_counts_each_pair_once_and_diagonal_nan():
    rng = np.random.default_rng(12)
    F = 9
    A = rng.random((F, F))
    P = np.triu(A, 1) + np.triu(A, 1).T
    np.fill_diagonal(P, 0.0)
    P[2, 5] = P[5, 2] = NAN                      # an undefined test is not counted
    for method in ("bonferroni", "bh", "by"):
        adj = O.adjust(P, method, symmetric=True)
        assert np.all(np.isnan(np.diag(adj)))
        assert np.array_equal(adj, adj.T, equal_nan=True)
        iu = np.triu_indices(F, 1)
        v = P[iu]
        ok = ~np.isnan(v)
        m = int(ok.sum())
        assert m == F * (F - 1) // 2 - 1
        if method == "bonferroni":
            ref = np.minimum(1.0, v[ok] * m)
        else:
            ref = st.false_discovery_control(v[ok], method=method)
        got = adj[iu][ok]
        assert np.allclose(got, ref, rtol=1e-13, atol=0)
        assert np.isnan(adj[2, 5])


def test_bonferroni_brute_force_and_bounds():
    p = np.array([[0.2, 0.001, NAN], [0.5, 0.04, 0.9]])
    adj = O.adjust(p, "bonferroni", symmetric=False)
    m = 5
    exp = np.array([[min(1, 0.2 * m), 0.001 * m, NAN], [min(1, 0.5 * m), 0.04 * m, min(1, 0.9 * m)]])
    assert np.array_equal(adj, exp, equal_nan=True)
    for method in ("bh", "by"):
        a = O.adjust(p, method, symmetric=False)
        ok = ~np.isnan(p)
        assert np.all(a[ok] >= p[ok]) and np.all(a[ok] <= 1.0)
