"""GPU parity of the mixed-precision (tcgen05) form against the FP64 oracle.

Bars (Sec. 3.5 statistics, mixed form): counts exact; |dr| <= 1e-6 for Pearson;
F and t within 1e-6 on their effect-size scale (t/sqrt(t^2+n-2), sqrt(F/(F+n)):
the analogue of |dr|, since a relative bar is meaningless for statistics near
zero); contingency tables exact (so chi-squared equals the plain form bit for
bit). P-values: the device p-function applied to the
device statistic agrees with the oracle's p-function on that same statistic to
1e-12 relative; the end-to-end p difference is bounded by the statistic's
difference propagated through the p-value's slope.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_00448_gb300 import synth
from tests._parity import compare, oracle_run, p_function_agrees as _p_agrees, pair_dof

pytestmark = pytest.mark.gpu
NAN = float("nan")


@pytest.fixture(scope="module")
def napg():
    from paper_2505_00448_gb300 import napg as N
    return N




def p_function_agrees(test, g):
    """c14 (i) for the correlation tests: p_gpu == oracle p-function(stat_gpu, n)."""
    return _p_agrees(test, g, {"n": np.asarray(g["n"], dtype=np.float64)})


@pytest.mark.parametrize("offset,lognormal", [(0.0, False), (1e4, False), (0.0, True)])
def test_mixed_pearson(napg, offset, lognormal):
    coh = synth.small_cohort(201, n_cont=300, n_cat=0, S=3000 + 37, miss=0.25, dtype=np.float32, offset=offset,
                             lognormal=lognormal)
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    va = coh["cont"]
    g = c.run("pearson", va, out="numpy", precision="mixed")
    ref = oracle_run("pearson", coh, va)
    compare("pearson", g, ref, stat_tol=("abs", 1e-6))
    p_function_agrees("pearson", g)
    # the plain form on the same data for the record
    gp = c.run("pearson", va, out="numpy", precision="fp64")
    assert np.array_equal(gp["n"], g["n"])
    c.close()


@pytest.mark.parametrize("lognormal", [True, False])
def test_mixed_pearson_exact_copies(napg, lognormal):
    """Columns with exact copies and power-of-two multiples (r = 1 on every
    co-observed set; each copy has its own missing samples): the split x3 Sxy
    (the lo x lo product left out) and the centred-square planes still give r
    within the bar, on heavy-tailed (lognormal) and offset (1e4 sigma) columns."""
    rng = np.random.default_rng(31)
    base = synth.small_cohort(203, n_cont=40, n_cat=0, S=20_000 + 3, miss=0.0, dtype=np.float32,
                              offset=0.0 if lognormal else 1e4, lognormal=lognormal)
    src = base["X"]
    X = np.concatenate([src, src, 4.0 * src]).astype(np.float32)
    X[rng.random(X.shape) < 0.2] = np.nan
    F = X.shape[0]
    coh = {"X": X, "vtype": np.zeros(F, np.uint8), "nlev": np.zeros(F, np.int32), "missing": float("nan"),
           "cont": np.arange(F, dtype=np.int32), "cat": np.zeros(0, np.int32)}
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    va = coh["cont"]
    g = c.run("pearson", va, out="numpy", precision="mixed")
    ref = oracle_run("pearson", coh, va)
    compare("pearson", g, ref, stat_tol=("abs", 1e-6))
    k = np.arange(40)
    for off in (40, 80):
        assert np.abs(g["stat"][k, k + off] - 1.0).max() <= 1e-6
    c.close()


def test_mixed_pearson_context_and_ragged(napg):
    rng = np.random.default_rng(9)
    coh = synth.small_cohort(202, n_cont=131, n_cat=0, S=2000 + 5, miss=0.3, dtype=np.float32)
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    mask = (rng.random(coh["X"].shape[1]) < 0.55).astype(np.uint8)
    va = coh["cont"]
    compare("pearson", c.run("pearson", va, mask=mask, out="numpy", precision="mixed"),
            oracle_run("pearson", coh, va, mask=mask), stat_tol=("abs", 1e-6))
    c.close()


@pytest.mark.parametrize("dtype,S", [(np.float32, 60_000 + 17), (np.float64, 30_000 + 9)])
def test_mixed_rows_beyond_shared_memory(napg, dtype, S):
    """Rows too long to stage in shared memory (FP32 above ~56,000 samples, FP64
    above ~28,000): the plane builder reads them from the cohort, with unaligned
    row starts (S not a multiple of 4)."""
    coh = synth.small_cohort(209, n_cont=24, n_cat=6, S=S, miss=0.3, lev_lo=2, lev_hi=5, dtype=dtype, offset=50.0)
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    cats, conts = coh["cat"], coh["cont"]
    compare("pearson", c.run("pearson", conts, out="numpy", precision="mixed"), oracle_run("pearson", coh, conts),
            stat_tol=("abs", 1e-6))
    compare("anova", c.run("anova", cats, conts, out="numpy", precision="mixed"),
            oracle_run("anova", coh, cats, conts), stat_tol=("effect", 1e-6))
    c.close()


@pytest.mark.parametrize("welch", [True, False])
def test_mixed_anova_ttest(napg, welch):
    coh = synth.small_cohort(203, n_cont=150, n_cat=40, S=2500 + 11, miss=0.2, lev_lo=2, lev_hi=9, binary_cats=12,
                             dtype=np.float32, offset=100.0)
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    cats, conts = coh["cat"], coh["cont"]
    compare("anova", c.run("anova", cats, conts, out="numpy", precision="mixed"),
            oracle_run("anova", coh, cats, conts), stat_tol=("effect", 1e-6))
    bins = cats[:12]
    compare("ttest", c.run("ttest", bins, conts, out="numpy", precision="mixed", welch=welch),
            oracle_run("ttest", coh, bins, conts, welch=int(welch)), stat_tol=("effect", 1e-6))
    c.close()


@pytest.mark.parametrize("welch", [True, False])
def test_mixed_p_function_on_device_statistics(napg, welch):
    """c14 part (i) for F, t and chi-squared: each device p-value equals the
    oracle's p-function at the device's own statistic and degrees of freedom
    (F: k - 1 and n - k from the present levels and the exact n; Welch t: the
    device's Welch-Satterthwaite nu, returned as the t-test's second effect
    output; Student t: n - 2; chi-squared: (k_a - 1)(k_b - 1)), to 1e-12
    relative. Part (ii) is the end-to-end comparison against the oracle with the
    p-value's slope over the statistic's difference."""
    coh = synth.small_cohort(212, n_cont=120, n_cat=30, S=4000 + 13, miss=0.25, lev_lo=2, lev_hi=8, binary_cats=10,
                             dtype=np.float32, offset=30.0)
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    cats, conts = coh["cat"], coh["cont"]
    bins = cats[:10]
    ga = c.run("anova", cats, conts, out="numpy", precision="mixed")
    assert _p_agrees("anova", ga, pair_dof("anova", coh, cats, conts, ga["n"])) > 1000
    gt = c.run("ttest", bins, conts, out="numpy", precision="mixed", welch=welch, effects=True)
    dof = {"df": gt["effect2"]} if welch else {"df": gt["n"].astype(np.float64) - 2}
    fin = np.isfinite(gt["stat"])
    assert np.array_equal(np.isfinite(gt["effect2"]), fin)
    if not welch:
        assert np.array_equal(gt["effect2"][fin], gt["n"][fin] - 2.0)
    assert _p_agrees("ttest", gt, dof) > 1000
    ref_t = oracle_run("ttest", coh, bins, conts, welch=int(welch))
    compare("ttest", gt, ref_t, stat_tol=("effect", 1e-6))
    # the device's degrees of freedom against the oracle's (Welch nu moves with
    # the group variances: 1e-6 relative in the mixed form)
    okd = np.isfinite(ref_t.dof["df"]) & fin
    assert np.allclose(gt["effect2"][okd], ref_t.dof["df"][okd], rtol=1e-6, atol=0)
    gc = c.run("chi2", cats, out="numpy", precision="mixed")
    assert _p_agrees("chi2", gc, pair_dof("chi2", coh, cats, None, gc["n"])) > 300
    c.close()


def test_mixed_chi2_equals_plain(napg):
    coh = synth.small_cohort(204, n_cont=0, n_cat=70, S=3000 + 3, miss=0.2, lev_lo=2, lev_hi=10, binary_cats=10)
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    va = coh["cat"]
    gm = c.run("chi2", va, out="numpy", precision="mixed")
    gp = c.run("chi2", va, out="numpy", precision="fp64")
    for k in ("stat", "p", "n"):
        assert np.array_equal(gm[k], gp[k], equal_nan=True), k
    compare("chi2", gm, oracle_run("chi2", coh, va))
    c.close()


def test_mixed_counts_exact_beyond_2_16(napg):
    """All-observed one-hot columns over 70,000 samples: every count equals the
    exact integer (partial sums well past 2^16 stay exact in FP32)."""
    S = 70000
    rng = np.random.default_rng(10)
    X = np.stack([np.zeros(S), (rng.random(S) < 0.5).astype(float), rng.integers(0, 3, S).astype(float)])
    c = napg.Context(0)
    c.load_cohort(X, [1, 1, 1], [1, 2, 3])
    g = c.run("chi2", [0, 1, 2], out="numpy", precision="mixed")
    assert (g["n"] == S).all()
    T = c.debug_integers("chi2", 1, 2)
    ref = np.array([[np.sum((X[1] == a) & (X[2] == b)) for b in range(3)] for a in range(2)]).ravel()
    assert np.array_equal(T, ref)
    gm = c.run("chi2", [1, 2], out="numpy", precision="mixed")
    gp = c.run("chi2", [1, 2], out="numpy", precision="fp64")
    assert np.array_equal(gm["stat"], gp["stat"])
    c.close()


def test_plane_cache_reuse_and_invalidation(napg):
    """Planes built by one unmasked run are reused by the next run on the same
    variables; a masked run, another variable list and a new cohort rebuild them."""
    rng = np.random.default_rng(31)
    coh = synth.small_cohort(205, n_cont=150, n_cat=12, S=2500 + 3, miss=0.25, dtype=np.float32)
    coh2 = synth.small_cohort(206, n_cont=150, n_cat=12, S=2500 + 3, miss=0.25, dtype=np.float32)
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    va, cats = coh["cont"], coh["cat"]
    r1 = c.run("pearson", va, out="numpy", precision="mixed")
    c.trace(True)
    c.trace_read()
    g = c.run("anova", cats, va, out="numpy", precision="mixed")          # same continuous list: reused
    stages = c.trace_read().get("stages", {})
    assert "planes_f16" not in stages, stages
    c.trace(False)
    compare("anova", g, oracle_run("anova", coh, cats, va), stat_tol=("effect", 1e-6))
    r2 = c.run("pearson", va, out="numpy", precision="mixed")
    for k in ("stat", "p", "n"):
        assert np.array_equal(r1[k], r2[k], equal_nan=True)
    mask = (rng.random(coh["X"].shape[1]) < 0.6).astype(np.uint8)
    compare("pearson", c.run("pearson", va, mask=mask, out="numpy", precision="mixed"),
            oracle_run("pearson", coh, va, mask=mask), stat_tol=("abs", 1e-6))
    sub = va[::2]
    compare("pearson", c.run("pearson", sub, out="numpy", precision="mixed"), oracle_run("pearson", coh, sub),
            stat_tol=("abs", 1e-6))
    r3 = c.run("pearson", va, out="numpy", precision="mixed")
    for k in ("stat", "p", "n"):
        assert np.array_equal(r1[k], r3[k], equal_nan=True)
    c.load_cohort(coh2["X"], coh2["vtype"], coh2["nlev"], coh2["missing"])
    compare("pearson", c.run("pearson", va, out="numpy", precision="mixed"), oracle_run("pearson", coh2, va),
            stat_tol=("abs", 1e-6))
    c.close()


def test_autotuner_keeps_results_identical(napg):
    """Launch shapes picked by the autotuner change timing only: outputs with
    tuning off, on the tuning run and on a later run are bit-identical."""
    coh = synth.small_cohort(207, n_cont=140, n_cat=10, S=6000 + 5, miss=0.2, dtype=np.float32, ties=True)
    outs = []
    for tune_on in (False, True, True):
        c = outs_ctx = napg.Context(0)
        c.tune(tune_on)
        c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
        r = {}
        r["pearson"] = c.run("pearson", coh["cont"], out="numpy", precision="mixed")
        r["anova"] = c.run("anova", coh["cat"], coh["cont"], out="numpy", precision="mixed")
        bins = coh["cat"][coh["nlev"][coh["cat"]] == 2]
        r["ttest"] = c.run("ttest", bins, coh["cont"], out="numpy", precision="mixed")
        r["spearman"] = c.run("spearman", coh["cont"], out="numpy")
        r["kruskal"] = c.run("kruskal", coh["cat"], coh["cont"], out="numpy")
        if tune_on:
            again = c.run("pearson", coh["cont"], out="numpy", precision="mixed")
            for k in ("stat", "p", "n"):
                assert np.array_equal(again[k], r["pearson"][k], equal_nan=True)
            recs = c.tune_read()
            kinds = {x["kind"] for x in recs}
            # ANOVA: level rows x (count, sum) planes and observed rows x square
            # planes; the t-test: level rows x all five planes
            assert {"stacked_mask", "stacked_onehot", "stacked_onehot_counts_sums", "stacked_observed_squares",
                    "sxy_stage_samples", "spearman_threads", "rank_groups_threads"} <= kinds, recs
            assert all(len(x["ms"]) == TUNE_CANDIDATES.get(x["kind"], 2) and min(x["ms"]) > 0
                       for x in recs), recs
        else:
            assert c.tune_read() == []
        outs.append(r)
        c.close()
    for r in outs[1:]:
        for t in outs[0]:
            for k in ("stat", "p", "n"):
                assert np.array_equal(outs[0][t][k], r[t][k], equal_nan=True), (t, k)


TUNE_KINDS = ("stacked_mask", "stacked_onehot", "stacked_onehot_counts_sums", "stacked_observed_squares",
              "sxy_stage_samples", "spearman_threads", "rank_groups_threads")
TUNE_CANDIDATES = {"stacked_mask": 4, "stacked_onehot": 4, "stacked_onehot_counts_sums": 4,
                   "stacked_observed_squares": 4}      # the other kinds: 2


def test_autotuner_every_candidate_bit_identical(napg):
    """Every launch-shape candidate of every tunable kernel, pinned in turn,
    gives bit-identical outputs (the tuning run keeps whichever is fastest, so
    a wrong slower candidate would otherwise go unseen); the sizes span
    several tiles of each kernel and a ragged tail in every dimension."""
    # 8,997 samples: 141 K-blocks of 64 (odd, so two-K-block stages end on a
    # single one) with a ragged last block
    coh = synth.small_cohort(211, n_cont=300, n_cat=60, S=8960 + 37, miss=0.25, dtype=np.float32, ties=True,
                             binary_cats=8)
    bins = coh["cat"][coh["nlev"][coh["cat"]] == 2]
    outs = []
    for pin in (0, 1, 2, 3):
        c = napg.Context(0)
        for k in TUNE_KINDS:
            c.tune_pin(k, pin % TUNE_CANDIDATES.get(k, 2))
        c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
        r = {"pearson": c.run("pearson", coh["cont"], out="numpy", precision="mixed"),
             "anova": c.run("anova", coh["cat"], coh["cont"], out="numpy", precision="mixed"),
             "ttest": c.run("ttest", bins, coh["cont"], out="numpy", precision="mixed"),
             "spearman": c.run("spearman", coh["cont"], out="numpy"),
             "kruskal": c.run("kruskal", coh["cat"], coh["cont"], out="numpy"),
             "mwu": c.run("mwu", bins, coh["cont"], out="numpy")}
        assert c.tune_read() == []          # pinned kinds are never timed
        outs.append(r)
        c.close()
    assert len(bins) >= 2
    for r in outs[1:]:
        for t in outs[0]:
            for k in ("stat", "p", "n"):
                assert np.array_equal(outs[0][t][k], r[t][k], equal_nan=True), (t, k)
    # the pinned outputs are the library's: one of them matches the oracle
    compare("pearson", outs[1]["pearson"], oracle_run("pearson", coh, coh["cont"]), stat_tol=("abs", 1e-6))


def test_tune_pin_arguments(napg):
    c = napg.Context(0)
    with pytest.raises(napg.NapgError):
        c.tune_pin("no_such_kind", 0)
    with pytest.raises(napg.NapgError):
        c.tune_pin("stacked_mask", 4)
    c.tune_pin("stacked_mask", 1)
    c.tune_pin("stacked_mask", -1)
    c.close()


def test_autotuner_near_shapes_reuse_choice(napg):
    """A shape within a factor of 4 in rows of a recorded one (same K) takes the
    recorded choice without timing; a far shape is timed; results are those of
    the untuned run."""
    coh = synth.small_cohort(208, n_cont=200, n_cat=0, S=4000 + 7, miss=0.2, dtype=np.float32, ties=True)
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    ref = napg.Context(0)
    ref.tune(False)
    ref.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    cont = coh["cont"]
    for k, expect in ((100, 1), (130, 1), (60, 1), (20, 2)):
        g = c.run("spearman", cont[:k], out="numpy")
        r = ref.run("spearman", cont[:k], out="numpy")
        for f in ("stat", "p", "n"):
            assert np.array_equal(g[f], r[f], equal_nan=True)
        recs = [x for x in c.tune_read() if x["kind"] == "spearman_threads"]
        assert len(recs) == expect, (k, recs)
    c.close()
    ref.close()

