"""GPU parity of the effect sizes (Table 2) and of the multiple-testing
correction (Sec. 3.4) against the FP64 oracle.

Effect sizes, plain FP64 form: |d| <= 1e-12 max(1, |value|), NaN patterns equal.
Mixed form: the effect sizes follow their statistics, so the bars follow the
statistics' bars (|dr| <= 1e-6 gives |d r^2| <= 2e-6; F and t within 1e-6 on
their effect scale give partial eta^2 and Cohen's d within a few 1e-6).
Correction: the device applied to the device's own p-values equals the oracle
applied to the same p-values bit for bit (same products, quotients and
running minimum).
"""

import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_00448_gb300 import synth

pytestmark = pytest.mark.gpu
NAN = float("nan")


@pytest.fixture(scope="module")
def napg():
    from paper_2505_00448_gb300 import napg as N
    return N


def ctx_for(N, coh):
    c = N.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    return c


def close(got, ref, tol, what):
    got, ref = np.asarray(got), np.asarray(ref)
    assert got.shape == ref.shape
    bad = np.argwhere(np.isnan(got) != np.isnan(ref))
    assert bad.size == 0, f"{what}: NaN pattern differs at {bad[:5].tolist()}: {got[tuple(bad[0])]} vs {ref[tuple(bad[0])]}"
    ok = ~np.isnan(ref)
    d = np.abs(got[ok] - ref[ok]) / np.maximum(1.0, np.abs(ref[ok]))
    assert d.max(initial=0) <= tol, f"{what}: max difference {d.max()} > {tol}"


def with_edge_columns(coh, rng):
    """Append a constant column and a column observed on three samples."""
    X = coh["X"]
    S = X.shape[1]
    extra = np.full((2, S), np.nan, X.dtype)
    extra[0, rng.random(S) < 0.7] = 2.5
    extra[1, rng.choice(S, 3, replace=False)] = [1.0, 2.0, 4.0]
    Fc = len(coh["cont"])
    Xn = np.concatenate([X[:Fc], extra, X[Fc:]])
    vtype = np.concatenate([coh["vtype"][:Fc], np.zeros(2, np.uint8), coh["vtype"][Fc:]])
    nlev = np.concatenate([coh["nlev"][:Fc], np.zeros(2, np.int32), coh["nlev"][Fc:]])
    out = dict(coh, X=Xn, vtype=vtype, nlev=nlev)
    out["cont"] = np.arange(Fc + 2, dtype=np.int32)
    out["cat"] = np.arange(Fc + 2, Fc + 2 + len(coh["cat"]), dtype=np.int32)
    return out


@pytest.fixture(scope="module")
def cohort():
    rng = np.random.default_rng(41)
    coh = synth.small_cohort(141, n_cont=40, n_cat=16, S=1500 + 7, miss=0.25, lev_lo=2, lev_hi=6, binary_cats=6,
                             ties=True)
    return with_edge_columns(coh, rng)


def oracle_effects(test, coh, va, vb=None, **kw):
    return O.effects(test, coh["X"].astype(np.float64), coh["missing"], coh["vtype"], coh["nlev"], va, vb, **kw)


CASES = [("pearson", "cont", None, {}), ("spearman", "cont", None, {}), ("chi2", "cat", None, {}),
         ("chi2", "cat", None, {"yates": True}), ("anova", "cat", "cont", {}),
         ("ttest", "bins", "cont", {"welch": True}), ("ttest", "bins", "cont", {"welch": False}),
         ("mwu", "bins", "cont", {"mwu_mode": "asymptotic"}), ("mwu", "bins", "cont", {"mwu_mode": "exact"}),
         ("kruskal", "cat", "cont", {})]


@pytest.mark.parametrize("test,a,b,opt", CASES)
def test_effect_sizes_plain(napg, cohort, test, a, b, opt):
    c = ctx_for(napg, cohort)
    sets = {"cont": cohort["cont"], "cat": cohort["cat"], "bins": cohort["cat"][:6]}
    va, vb = sets[a], (sets[b] if b else None)
    if test == "kruskal":
        va = cohort["cat"][6:]
    nb = len(va) if vb is None else len(vb)
    g = {k: np.empty((len(va), nb), np.int32 if k == "n" else np.float64)
         for k in ("stat", "p", "n", "effect", "effect2")}
    try:
        c.run(test, va, vb, outputs=g, effects=True, **opt)
    except napg.NapgError as e:
        # forced exact Mann-Whitney beyond its exact range: p NaN for those pairs
        # and the call says so; the effect size does not depend on the p-value mode
        assert test == "mwu" and opt.get("mwu_mode") == "exact" and e.code == napg.E_UNSUPPORTED
    kw = {}
    if "welch" in opt:
        kw["welch"] = int(opt["welch"])
    if "yates" in opt:
        kw["yates"] = int(opt["yates"])
    e1, e2 = oracle_effects(test, cohort, va, vb, **kw)
    close(g["effect"], e1, 1e-12, f"{test} effect")
    close(g["effect2"], e2, 1e-12, f"{test} effect2")
    c.close()


def test_effect_sizes_mixed(napg, cohort):
    c = ctx_for(napg, cohort)
    cont, cat, bins = cohort["cont"], cohort["cat"], cohort["cat"][:6]
    for test, va, vb, bar in (("pearson", cont, None, 2e-6), ("anova", cat, cont, 4e-6), ("ttest", bins, cont, 1e-5),
                              ("chi2", cat, None, 1e-12)):
        g = c.run(test, va, vb, out="numpy", effects=True, precision="mixed")
        e1, e2 = oracle_effects(test, cohort, va, vb)
        close(g["effect"], e1, bar, f"mixed {test} effect")
        close(g["effect2"], e2, bar, f"mixed {test} effect2")
    c.close()


def test_effect_sizes_cross_block_context_and_device_outputs(napg, cohort):
    rng = np.random.default_rng(42)
    c = ctx_for(napg, cohort)
    cont, cat = cohort["cont"], cohort["cat"]
    A, B = cont[:15], cont[10:]
    g = c.run("pearson", A, B, out="numpy", effects=True)
    e1, _ = oracle_effects("pearson", cohort, A, B)
    close(g["effect"], e1, 1e-12, "pearson A x B r^2")
    Ca, Cb = cat[:5], cat[3:]
    g = c.run("chi2", Ca, Cb, out="numpy", effects=True)
    e1, e2 = oracle_effects("chi2", cohort, Ca, Cb)
    close(g["effect"], e1, 1e-12, "chi2 A x B phi")
    close(g["effect2"], e2, 1e-12, "chi2 A x B V")
    mask = (rng.random(cohort["X"].shape[1]) < 0.4).astype(np.uint8)
    gd = c.run("kruskal", cat[6:], cont, mask=mask, out="cuda", effects=True)
    gh = c.run("kruskal", cat[6:], cont, mask=mask, out="numpy", effects=True)
    assert np.array_equal(gd["effect"].cpu().numpy(), gh["effect"], equal_nan=True)
    e1, _ = O.effects("kruskal", cohort["X"].astype(np.float64), NAN, cohort["vtype"], cohort["nlev"], cat[6:], cont,
                      ctx=mask)
    close(gh["effect"], e1, 1e-12, "kruskal in a context")
    # no effect outputs asked: the statistics are unchanged
    plain = c.run("kruskal", cat[6:], cont, mask=mask, out="numpy")
    for k in ("stat", "p", "n"):
        assert np.array_equal(plain[k], gh[k], equal_nan=True)
    c.close()


@pytest.mark.parametrize("method", ["bonferroni", "bh", "by"])
def test_adjust_matches_oracle_bit_for_bit(napg, cohort, method):
    c = ctx_for(napg, cohort)
    # a symmetric matrix (diagonal, constant and sparse columns give NaN) and a
    # categorical x continuous one
    g = c.run("pearson", cohort["cont"], out="numpy")
    adj = c.adjust(g["p"], method, symmetric=True)
    assert np.array_equal(adj, O.adjust(g["p"], method, True), equal_nan=True)
    gk = c.run("kruskal", cohort["cat"][6:], cohort["cont"], out="cuda")
    adj_dev = c.adjust(gk["p"], method, symmetric=False)
    pk = gk["p"].cpu().numpy()
    assert np.array_equal(adj_dev.cpu().numpy(), O.adjust(pk, method, False), equal_nan=True)
    c.close()


def test_adjust_ties_nans_and_size(napg):
    rng = np.random.default_rng(43)
    c = napg.Context(0)
    F = 700
    A = np.round(rng.random((F, F)) ** 4, 3)          # many ties
    P = np.triu(A, 1) + np.triu(A, 1).T
    P[rng.random((F, F)) < 0.05] = np.nan
    P = np.where(np.isnan(P) | np.isnan(P.T), np.nan, P)
    for method in ("bonferroni", "bh", "by"):
        got = c.adjust(P, method, symmetric=True)
        assert np.array_equal(got, O.adjust(P, method, True), equal_nan=True), method
        assert np.all(np.isnan(np.diag(got)))
    flat = rng.random((3, 5000))
    flat[0, :10] = np.nan
    for method in ("bonferroni", "bh", "by"):
        assert np.array_equal(c.adjust(flat, method), O.adjust(flat, method, False), equal_nan=True)
    with pytest.raises(napg.NapgError):
        c.adjust(np.zeros((3, 4)), "bh", symmetric=True)
    with pytest.raises(napg.NapgError):
        c.adjust(np.zeros((3, 4)), 7)
    empty = np.full((4, 4), np.nan)
    assert np.all(np.isnan(c.adjust(empty, "bh", symmetric=True)))
    c.close()
