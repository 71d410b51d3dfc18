"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle,
element by element, on seeded synthetic cohorts that span several tiles and a
ragged tail, with deletion patterns, contexts and the degenerate cases the
tests define (Sec. 3.5). Counts, tables and rank sums must be bit-exact.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_00448_gb300 import synth
from tests._parity import compare, oracle_run

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




def with_degenerate_columns(coh, rng):
    """Append a constant column, an all-missing column, a one-observation column
    and an exactly linear copy (r = 1) to the continuous block."""
    X = coh["X"]
    S = X.shape[1]
    extra = np.full((4, S), np.nan, X.dtype)
    extra[0, rng.random(S) < 0.8] = 3.25
    extra[2, int(rng.integers(0, S))] = 1.0
    src = X[0].copy()
    extra[3] = 2.0 * src + 7.0
    Fc = len(coh["cont"])
    Xn = np.concatenate([X[:Fc], extra, X[Fc:]])
    vtype = np.concatenate([coh["vtype"][:Fc], np.zeros(4, np.uint8), coh["vtype"][Fc:]])
    nlev = np.concatenate([coh["nlev"][:Fc], np.zeros(4, np.int32), coh["nlev"][Fc:]])
    out = dict(coh, X=Xn, vtype=vtype, nlev=nlev)
    out["cont"] = np.arange(Fc + 4, dtype=np.int32)
    out["cat"] = np.arange(Fc + 4, Fc + 4 + len(coh["cat"]), dtype=np.int32)
    return out


# ------------------------------------------------------------------ Pearson --

@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_pearson_parity(napg, dtype):
    rng = np.random.default_rng(1)
    coh = synth.small_cohort(101, n_cont=66, n_cat=0, S=1000 + 13, miss=0.25, dtype=dtype)
    coh = with_degenerate_columns(coh, rng)
    c = ctx_for(napg, coh)
    va = coh["cont"]
    g = c.run("pearson", va, out="numpy")
    compare("pearson", g, oracle_run("pearson", coh, va))
    # sample context, and a cross block A x B with overlap
    mask = (rng.random(coh["X"].shape[1]) < 0.6).astype(np.uint8)
    g = c.run("pearson", va, mask=mask, out="numpy")
    compare("pearson", g, oracle_run("pearson", coh, va, mask=mask))
    A, B = va[:30], va[20:]
    g = c.run("pearson", A, B, out="numpy")
    compare("pearson", g, oracle_run("pearson", coh, A, B))
    c.close()


def test_pearson_offsets_and_empty_context(napg):
    coh = synth.small_cohort(102, n_cont=40, n_cat=0, S=700, miss=0.3, offset=1e4)
    c = ctx_for(napg, coh)
    va = coh["cont"]
    compare("pearson", c.run("pearson", va, out="numpy"), oracle_run("pearson", coh, va))
    empty = np.zeros(700, np.uint8)
    g = c.run("pearson", va, mask=empty, out="numpy")
    assert (g["n"] == 0).all() and np.isnan(g["stat"]).all() and np.isnan(g["p"]).all()
    c.close()


def test_small_pearson_full(napg):
    coh = synth.small_pearson_cohort()
    c = ctx_for(napg, coh)
    va = coh["cont"]
    compare("pearson", c.run("pearson", va, out="numpy"), oracle_run("pearson", coh, va))
    c.close()


@pytest.mark.parametrize("S", [31, 33, 257, 1007])
def test_pearson_fp64_sample_split(napg, S):
    """Few variables: the plain FP64 moments split the sample axis over a cluster
    of CTAs (up to 8, at least one 32-sample word each); every split size agrees
    with the oracle, and repeated calls are bit-identical."""
    coh = synth.small_cohort(110 + S, n_cont=70, n_cat=0, S=S, miss=0.2, offset=50.0)
    c = ctx_for(napg, coh)
    for nv in (1, 2, 33, 70):
        va = coh["cont"][:nv]
        g = c.run("pearson", va, out="numpy")
        compare("pearson", g, oracle_run("pearson", coh, va))
        g2 = c.run("pearson", va, out="numpy")
        for k in ("stat", "p", "n"):
            assert np.array_equal(g[k], g2[k], equal_nan=True)
    c.close()


@pytest.mark.parametrize("levels", [(2, 4), (5, 16), (17, 64)])
def test_anova_fp64_level_counts(napg, levels):
    """The plain FP64 group sums at each level-count class (up to 4, 16, 64)."""
    coh = synth.small_cohort(120 + levels[1], n_cont=9, n_cat=6, S=2000 + 5, miss=0.2, lev_lo=levels[0],
                             lev_hi=levels[1])
    c = ctx_for(napg, coh)
    cats, conts = coh["cat"], coh["cont"]
    compare("anova", c.run("anova", cats, conts, out="numpy"), oracle_run("anova", coh, cats, conts))
    c.close()


# ----------------------------------------------------------------- Spearman --

def test_spearman_parity_and_rank_sums(napg):
    rng = np.random.default_rng(3)
    coh = synth.small_cohort(103, n_cont=45, n_cat=0, S=900 + 7, miss=0.3, ties=True)
    coh = with_degenerate_columns(coh, rng)
    c = ctx_for(napg, coh)
    va = coh["cont"]
    compare("spearman", c.run("spearman", va, out="numpy"), oracle_run("spearman", coh, va))
    mask = (rng.random(coh["X"].shape[1]) < 0.5).astype(np.uint8)
    compare("spearman", c.run("spearman", va, mask=mask, out="numpy"),
            oracle_run("spearman", coh, va, mask=mask))
    A, B = va[:10], va[5:30]
    compare("spearman", c.run("spearman", A, B, out="numpy"), oracle_run("spearman", coh, A, B))
    Xd = coh["X"].astype(np.float64)
    for i, j in [(0, 1), (3, 17), (5, 5), (10, 44), (2, 47)]:
        a, b = int(va[i]), int(va[j])
        got = c.debug_integers("spearman", a, b)
        ref = O.pair_ints("spearman", Xd, NAN, coh["vtype"], coh["nlev"], a, b)
        assert np.array_equal(got, ref), (i, j, got, ref)
    c.close()


# -------------------------------------------------------------- chi-squared --

@pytest.mark.parametrize("yates", [False, True])
def test_chi2_parity_and_tables(napg, yates):
    rng = np.random.default_rng(4)
    coh = synth.small_cohort(104, n_cont=0, n_cat=45, S=1200 + 5, miss=0.2, lev_lo=2, lev_hi=9, binary_cats=10)
    # a variable with a level that only occurs where most others are missing
    c = ctx_for(napg, coh)
    va = coh["cat"]
    compare("chi2", c.run("chi2", va, yates=yates, out="numpy"), oracle_run("chi2", coh, va, yates=int(yates)))
    mask = (rng.random(coh["X"].shape[1]) < 0.4).astype(np.uint8)
    compare("chi2", c.run("chi2", va, mask=mask, yates=yates, out="numpy"),
            oracle_run("chi2", coh, va, mask=mask, yates=int(yates)))
    Xd = coh["X"].astype(np.float64)
    for i, j in [(0, 1), (3, 17), (12, 12), (40, 44)]:
        a, b = int(va[i]), int(va[j])
        got = c.debug_integers("chi2", a, b)
        ref = O.pair_ints("chi2", Xd, NAN, coh["vtype"], coh["nlev"], a, b)
        assert np.array_equal(got, ref), (i, j)
    c.close()


def test_chi2_single_and_emptied_levels(napg):
    S = 64
    rng = np.random.default_rng(5)
    a = rng.integers(0, 3, S).astype(float)
    b = rng.integers(0, 2, S).astype(float)
    b[a == 2] = np.nan                    # level 2 of a emptied by deletion against b
    one = np.zeros(S)
    X = np.array([a, b, one])
    coh = {"X": X, "vtype": np.ones(3, np.uint8), "nlev": np.array([3, 2, 1], np.int32), "missing": NAN,
           "cat": np.arange(3, dtype=np.int32), "cont": np.zeros(0, np.int32)}
    c = ctx_for(napg, coh)
    compare("chi2", c.run("chi2", coh["cat"], out="numpy"), oracle_run("chi2", coh, coh["cat"]))
    c.close()


# --------------------------------------------------------- ANOVA / t-tests --

@pytest.mark.parametrize("welch", [True, False])
def test_anova_ttest_parity(napg, welch):
    rng = np.random.default_rng(6)
    coh = synth.small_cohort(105, n_cont=37, n_cat=20, S=1100 + 3, miss=0.2, lev_lo=2, lev_hi=7, binary_cats=8)
    coh = with_degenerate_columns(coh, rng)
    c = ctx_for(napg, coh)
    cats, conts = coh["cat"], coh["cont"]
    compare("anova", c.run("anova", cats, conts, out="numpy"), oracle_run("anova", coh, cats, conts))
    bins = cats[:8]
    compare("ttest", c.run("ttest", bins, conts, welch=welch, out="numpy"),
            oracle_run("ttest", coh, bins, conts, welch=int(welch)))
    mask = (rng.random(coh["X"].shape[1]) < 0.3).astype(np.uint8)
    compare("anova", c.run("anova", cats, conts, mask=mask, out="numpy"),
            oracle_run("anova", coh, cats, conts, mask=mask))
    compare("ttest", c.run("ttest", bins, conts, mask=mask, welch=welch, out="numpy"),
            oracle_run("ttest", coh, bins, conts, mask=mask, welch=int(welch)))
    c.close()


def test_anova_ttest_constant_groups(napg):
    lab = np.array([0, 0, 0, 1, 1, 1, 2, 2, 2, 0, 1, 2], float)
    X = np.array([lab, lab == 1,
                  [1, 1, 1, 2, 2, 2, 3, 3, 3, 1, 2, 3],
                  [4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4, 4],
                  [1, 2, 3, 4, 5, 6, np.nan, np.nan, np.nan, 1, 2, np.nan]], float)
    X[1] = X[1].astype(float)
    coh = {"X": X, "vtype": np.array([1, 1, 0, 0, 0], np.uint8), "nlev": np.array([3, 2, 0, 0, 0], np.int32),
           "missing": NAN}
    c = ctx_for(napg, coh)
    compare("anova", c.run("anova", [0], [2, 3, 4], out="numpy"), oracle_run("anova", coh, [0], [2, 3, 4]))
    for welch in (True, False):
        compare("ttest", c.run("ttest", [1], [2, 3, 4], welch=welch, out="numpy"),
                oracle_run("ttest", coh, [1], [2, 3, 4], welch=int(welch)))
    c.close()


# ---------------------------------------------------------- MWU / Kruskal --

def test_mwu_kruskal_parity_and_rank_sums(napg):
    rng = np.random.default_rng(7)
    coh = synth.small_cohort(106, n_cont=33, n_cat=14, S=1000 + 9, miss=0.25, ties=True, lev_lo=2, lev_hi=6,
                             binary_cats=6)
    c = ctx_for(napg, coh)
    cats, conts = coh["cat"], coh["cont"]
    bins = cats[:6]
    compare("mwu", c.run("mwu", bins, conts, mwu_mode="asymptotic", out="numpy"),
            oracle_run("mwu", coh, bins, conts, mwu_mode=2))
    compare("kruskal", c.run("kruskal", cats, conts, out="numpy"), oracle_run("kruskal", coh, cats, conts))
    mask = (rng.random(coh["X"].shape[1]) < 0.4).astype(np.uint8)
    compare("kruskal", c.run("kruskal", cats, conts, mask=mask, out="numpy"),
            oracle_run("kruskal", coh, cats, conts, mask=mask))
    Xd = coh["X"].astype(np.float64)
    for a_, j_ in [(0, 0), (3, 17), (10, 32)]:
        a, j = int(cats[a_]), int(conts[j_])
        for test in ("kruskal",) + (("mwu",) if a_ < 6 else ()):
            got = c.debug_integers(test, a, j)
            ref = O.pair_ints(test, Xd, NAN, coh["vtype"], coh["nlev"], a, j)
            assert np.array_equal(got, ref), (test, a_, j_, got, ref)
    c.close()


@pytest.mark.parametrize("levels", [(2, 2), (3, 4), (5, 8), (9, 20)])
def test_kruskal_level_classes(napg, levels):
    """Rank sums per level through each level-count class of the rank kernel (per
    level warp reductions up to 8 levels, the last level from the totals; lane
    grouping above), bit-exact, with the statistics against the oracle."""
    coh = synth.small_cohort(130 + levels[1], n_cont=7, n_cat=6, S=2000 + 7, miss=0.25, ties=True,
                             lev_lo=levels[0], lev_hi=levels[1])
    c = ctx_for(napg, coh)
    cats, conts = coh["cat"], coh["cont"]
    compare("kruskal", c.run("kruskal", cats, conts, out="numpy"), oracle_run("kruskal", coh, cats, conts))
    Xd = coh["X"].astype(np.float64)
    for a, j in ((cats[0], conts[0]), (cats[5], conts[6])):
        got = c.debug_integers("kruskal", int(a), int(j))
        ref = O.pair_ints("kruskal", Xd, NAN, coh["vtype"], coh["nlev"], int(a), int(j))
        assert np.array_equal(got, ref), (got, ref)
    c.close()


def test_rank_groups_wide_level_slots(napg):
    """60,007 samples: a lane's level totals may pass the 32-bit slot (more than
    2^24 / (2S + 1) words per warp at 256 threads), so the kernel keeps 64-bit
    slots; rank sums, counts and tie terms bit-exact for 2, 4 and 8 levels."""
    for levels in ((2, 2), (3, 4), (5, 8)):
        coh = synth.small_cohort(150 + levels[1], n_cont=3, n_cat=3, S=60_000 + 7, miss=0.2, ties=True,
                                 lev_lo=levels[0], lev_hi=levels[1])
        c = ctx_for(napg, coh)
        cats, conts = coh["cat"], coh["cont"]
        compare("kruskal", c.run("kruskal", cats, conts, out="numpy"), oracle_run("kruskal", coh, cats, conts))
        Xd = coh["X"].astype(np.float64)
        for a, j in ((cats[0], conts[0]), (cats[2], conts[1])):
            got = c.debug_integers("kruskal", int(a), int(j))
            ref = O.pair_ints("kruskal", Xd, NAN, coh["vtype"], coh["nlev"], int(a), int(j))
            assert np.array_equal(got, ref), (levels, got, ref)
        c.close()


def test_rank_groups_labels_from_cohort(napg):
    """150,000 samples: the sorted labels no longer fit beside the per-pair rank
    arrays in shared memory, so the walk reads them from the cohort."""
    coh = synth.small_cohort(140, n_cont=3, n_cat=3, S=150_000 + 3, miss=0.3, ties=True, lev_lo=2, lev_hi=6,
                             binary_cats=1)
    c = ctx_for(napg, coh)
    cats, conts = coh["cat"], coh["cont"]
    compare("kruskal", c.run("kruskal", cats, conts, out="numpy"), oracle_run("kruskal", coh, cats, conts))
    compare("mwu", c.run("mwu", cats[:1], conts, mwu_mode="asymptotic", out="numpy"),
            oracle_run("mwu", coh, cats[:1], conts, mwu_mode=2))
    Xd = coh["X"].astype(np.float64)
    got = c.debug_integers("kruskal", int(cats[2]), int(conts[1]))
    assert np.array_equal(got, O.pair_ints("kruskal", Xd, NAN, coh["vtype"], coh["nlev"], int(cats[2]), int(conts[1])))
    c.close()


def test_mwu_exact_mode(napg):
    """Small groups without ties: exact p by the product form vs the oracle's
    Mann-Whitney recurrence."""
    rng = np.random.default_rng(8)
    S = 400
    rows, vt, nl = [], [], []
    for k in range(6):
        lab = np.ones(S)
        lab[rng.choice(S, size=int(rng.integers(1, 8)), replace=False)] = 0.0
        rows.append(lab); vt.append(1); nl.append(2)
    for k in range(5):
        x = rng.permutation(S).astype(float) + 0.25
        x[rng.random(S) < 0.3] = np.nan
        rows.append(x); vt.append(0); nl.append(0)
    coh = {"X": np.array(rows), "vtype": np.array(vt, np.uint8), "nlev": np.array(nl, np.int32), "missing": NAN}
    c = ctx_for(napg, coh)
    A, B = list(range(6)), list(range(6, 11))
    compare("mwu", c.run("mwu", A, B, mwu_mode="auto", out="numpy"), oracle_run("mwu", coh, A, B, mwu_mode=0))
    c.close()


def test_mwu_forced_exact_within_and_beyond_its_range(napg):
    """Forced exact Mann-Whitney (Sec. 3.5.6): groups of 10-25 of 100 samples
    without ties give the oracle's exact p; groups of 70 and more (beyond the
    exact 128-bit range) give U exactly, p = NaN, and the call reports
    NAPG_E_UNSUPPORTED after writing its outputs."""
    rng = np.random.default_rng(18)

    def cohort(S, g_lo, g_hi, k):
        rows, vt, nl = [], [], []
        for _ in range(k):
            lab = np.ones(S)
            lab[rng.choice(S, size=int(rng.integers(g_lo, g_hi + 1)), replace=False)] = 0.0
            rows.append(lab); vt.append(1); nl.append(2)
        for _ in range(4):
            rows.append(rng.permutation(S).astype(float) + 0.5); vt.append(0); nl.append(0)
        return {"X": np.array(rows), "vtype": np.array(vt, np.uint8), "nlev": np.array(nl, np.int32), "missing": NAN}

    coh = cohort(100, 10, 25, 4)
    c = ctx_for(napg, coh)
    A, B = list(range(4)), list(range(4, 8))
    compare("mwu", c.run("mwu", A, B, mwu_mode="exact", out="numpy"), oracle_run("mwu", coh, A, B, mwu_mode=1))
    c.close()
    coh = cohort(300, 70, 120, 3)
    c = ctx_for(napg, coh)
    A, B = list(range(3)), list(range(3, 7))
    out = {"stat": np.full((3, 4), -1.0), "p": np.full((3, 4), -1.0), "n": np.full((3, 4), -1, np.int32)}
    with pytest.raises(napg.NapgError) as e:
        c.run("mwu", A, B, mwu_mode="exact", outputs=out)
    assert e.value.code == napg.E_UNSUPPORTED
    ref = oracle_run("mwu", coh, A, B, mwu_mode=1)
    assert np.array_equal(out["stat"], ref[0]) and np.array_equal(out["n"], ref[2])
    assert np.isnan(out["p"]).all()
    # the context stays usable: the asymptotic mode on the same pairs
    compare("mwu", c.run("mwu", A, B, mwu_mode="asymptotic", out="numpy"), oracle_run("mwu", coh, A, B, mwu_mode=2))
    c.close()


# -------------------------------------------------------------- errors --

def test_reloading_cohorts_reuses_buffers(napg):
    """One context, cohorts loaded one after another (smaller, then larger than
    the buffers it keeps, FP64 then FP32): every result matches the oracle."""
    c = napg.Context(0)
    for seed, nc, nk, S, dt in ((150, 30, 6, 2000 + 3, np.float64), (151, 12, 3, 700 + 1, np.float32),
                                (152, 40, 8, 3000 + 9, np.float32)):
        coh = synth.small_cohort(seed, n_cont=nc, n_cat=nk, S=S, miss=0.25, lev_lo=2, lev_hi=5, dtype=dt)
        c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
        cats, conts = coh["cat"], coh["cont"]
        compare("pearson", c.run("pearson", conts, out="numpy"), oracle_run("pearson", coh, conts))
        compare("kruskal", c.run("kruskal", cats, conts, out="numpy"), oracle_run("kruskal", coh, cats, conts))
        compare("chi2", c.run("chi2", cats, out="numpy"), oracle_run("chi2", coh, cats))
    c.close()


def test_paper_simulation_all_tests(napg):
    """The paper's simulated benchmark data (uniform values, c = 4 categorical and
    dichotomous features, exactly 10% missing per feature): every test against
    the oracle."""
    coh = synth.paper_simulation(60, 250)
    c = ctx_for(napg, coh)
    cont, cat, bins = coh["cont"], coh["cat"], coh["bins"]
    for test, va, vb, kw in (("pearson", cont, None, {}), ("spearman", cont, None, {}), ("chi2", cat, None, {}),
                             ("ttest", bins, cont, {}), ("mwu", bins, cont, {"mwu_mode": 2}),
                             ("anova", cat, cont, {}), ("kruskal", cat, cont, {})):
        opt = {"mwu_mode": "asymptotic"} if test == "mwu" else {}
        compare(test, c.run(test, va, vb, out="numpy", **opt), oracle_run(test, coh, va, vb, **kw))
    c.close()


def test_async_host_outputs(napg):
    """Host outputs with sync=False: several calls in flight (the staging sets
    alternate), outputs written once sync() returns, equal to synchronous runs;
    a correction queued behind them sees their results."""
    import torch
    coh = synth.small_cohort(160, n_cont=50, n_cat=10, S=1200 + 5, miss=0.2, lev_lo=2, lev_hi=5, binary_cats=3)
    c = ctx_for(napg, coh)
    cont, cat = coh["cont"], coh["cat"]
    jobs = [("pearson", cont, None), ("chi2", cat, None), ("kruskal", cat[3:], cont), ("pearson", cont[:20], None),
            ("anova", cat, cont)]
    ref = [c.run(t, a, b, out="numpy") for t, a, b in jobs]
    pin = lambda shape, dt: torch.empty(shape, dtype=dt).pin_memory().numpy()
    bufs = []
    for t, a, b in jobs:
        nb = len(a) if b is None else len(b)
        o = {"stat": pin((len(a), nb), torch.float64), "p": pin((len(a), nb), torch.float64),
             "n": pin((len(a), nb), torch.int32)}
        c.run(t, a, b, outputs=o, out="numpy", sync=False)
        bufs.append(o)
    c.sync()
    for r, o in zip(ref, bufs):
        for k in ("stat", "p", "n"):
            assert np.array_equal(r[k], o[k], equal_nan=True)
    # pageable outputs in flight, then a synchronous call and a correction
    o = {"stat": np.empty((50, 50)), "p": np.empty((50, 50)), "n": np.empty((50, 50), np.int32)}
    c.run("pearson", cont, outputs=o, out="numpy", sync=False)
    adj = c.adjust(ref[0]["p"], "bh", symmetric=True)
    c.sync()
    assert np.array_equal(o["p"], ref[0]["p"], equal_nan=True)
    assert np.array_equal(adj, O.adjust(ref[0]["p"], "bh", True), equal_nan=True)
    c.close()


def test_cohort_from_pinned_pageable_and_device_memory(napg):
    """The same cohort loaded from pageable host memory (copied), page-locked host
    memory (read by the validation kernel over the host link) and device memory
    gives identical results; bad values are caught on every path."""
    import torch
    coh = synth.small_cohort(161, n_cont=30, n_cat=8, S=2000 + 11, miss=0.2, lev_lo=2, lev_hi=5,
                             dtype=np.float32)
    outs = []
    for src in ("numpy", "pinned", "device"):
        X = coh["X"]
        if src == "pinned":
            X = torch.from_numpy(coh["X"]).pin_memory()
        elif src == "device":
            X = torch.from_numpy(coh["X"]).cuda()
        c = napg.Context(0)
        c.load_cohort(X, coh["vtype"], coh["nlev"], coh["missing"])
        outs.append([c.run(t, a, b, out="numpy") for t, a, b in (("pearson", coh["cont"], None),
                                                                  ("chi2", coh["cat"], None),
                                                                  ("kruskal", coh["cat"], coh["cont"]))])
        c.close()
    for o in outs[1:]:
        for r0, r1 in zip(outs[0], o):
            for k in ("stat", "p", "n"):
                assert np.array_equal(r0[k], r1[k], equal_nan=True)
    bad = coh["X"].copy()
    bad[coh["cat"][0], 5] = 7.5                    # not a label
    c = napg.Context(0)
    with pytest.raises(napg.NapgError) as e:
        c.load_cohort(torch.from_numpy(bad).pin_memory(), coh["vtype"], coh["nlev"], coh["missing"])
    assert e.value.code == napg.E_LABEL
    bad = coh["X"].copy()
    bad[coh["cont"][3], 9] = np.inf
    with pytest.raises(napg.NapgError) as e:
        c.load_cohort(torch.from_numpy(bad).pin_memory(), coh["vtype"], coh["nlev"], coh["missing"])
    assert e.value.code == napg.E_NONFINITE
    c.close()


def test_invalid_inputs_are_errors(napg):
    c = napg.Context(0)
    X = np.array([[0, 1, 3.0], [1.0, 2.0, 3.0]])
    with pytest.raises(napg.NapgError) as e:
        c.load_cohort(X, [1, 0], [3, 0])
    assert e.value.code == napg.E_LABEL
    with pytest.raises(napg.NapgError) as e:
        c.load_cohort(np.array([[0, 1, 2.0], [1.0, np.inf, 3.0]]), [1, 0], [3, 0])
    assert e.value.code == napg.E_NONFINITE
    c.load_cohort(np.array([[0, 1, 2.0, 1], [1.0, 5, 3.0, 2]]), [1, 0], [3, 0])
    with pytest.raises(napg.NapgError) as e:
        c.run("ttest", [0], [1])                      # 3 levels for a two-group test
    assert e.value.code == napg.E_ARG
    with pytest.raises(napg.NapgError) as e:
        c.run("pearson", [0])                          # categorical in a continuous test
    assert e.value.code == napg.E_ARG
    with pytest.raises(napg.NapgError) as e:
        c.run("anova", [0], [7])
    assert e.value.code == napg.E_ARG
    c.close()


def test_sentinel_and_samples_major(napg):
    coh = synth.small_cohort(107, n_cont=20, n_cat=4, S=500, miss=0.2, binary_cats=2)
    X = coh["X"].copy()
    X[np.isnan(X)] = -999.0
    c = napg.Context(0)
    c.load_cohort(np.ascontiguousarray(X.T), coh["vtype"], coh["nlev"], missing=-999.0, samples_major=True)
    va = coh["cont"]
    compare("pearson", c.run("pearson", va, out="numpy"), oracle_run("pearson", coh, va))
    compare("kruskal", c.run("kruskal", coh["cat"], va, out="numpy"), oracle_run("kruskal", coh, coh["cat"], va))
    c.close()


def test_rank_tests_many_samples(napg):
    """80,000 samples: the per-pair rank arrays no longer leave room for four
    256-thread blocks per SM, so each pair runs as one 1024-thread block; rank
    sums stay bit-exact and the statistics match the oracle."""
    rng = np.random.default_rng(17)
    coh = synth.small_cohort(111, n_cont=6, n_cat=4, S=80_000 + 13, miss=0.3, ties=True, lev_lo=2, lev_hi=5,
                             binary_cats=2)
    c = ctx_for(napg, coh)
    cats, conts = coh["cat"], coh["cont"]
    compare("spearman", c.run("spearman", conts, out="numpy"), oracle_run("spearman", coh, conts))
    mask = (rng.random(coh["X"].shape[1]) < 0.5).astype(np.uint8)
    compare("spearman", c.run("spearman", conts, mask=mask, out="numpy"),
            oracle_run("spearman", coh, conts, mask=mask))
    compare("kruskal", c.run("kruskal", cats, conts, out="numpy"), oracle_run("kruskal", coh, cats, conts))
    compare("mwu", c.run("mwu", cats[:2], conts, mwu_mode="asymptotic", out="numpy"),
            oracle_run("mwu", coh, cats[:2], conts, mwu_mode=2))
    Xd = coh["X"].astype(np.float64)
    for test, a, b in (("spearman", conts[0], conts[3]), ("kruskal", cats[3], conts[1]), ("mwu", cats[0], conts[5])):
        got = c.debug_integers(test, int(a), int(b))
        ref = O.pair_ints(test, Xd, NAN, coh["vtype"], coh["nlev"], int(a), int(b))
        assert np.array_equal(got, ref), (test, got, ref)
    c.close()
