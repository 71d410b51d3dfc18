"""Parity at the workloads' full sizes, in the launch configuration the bench
times: every pair where the oracle can afford it (the 200 x 1,000 Pearson
cohort), otherwise random sampled pairs plus every pair of a 64-variable slice,
compared element by element with the oracle run on exactly those pairs."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_00448_gb300 import synth
from tests._parity import compare, oracle_run, oracle_run_pairs

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

MIXED_BAR = {"pearson": ("abs", 1e-6), "anova": ("effect", 1e-6), "ttest": ("effect", 1e-6), "chi2": None}


_COHORTS = {}


def cohort(name):
    """Each cohort generated once per session (the mixed and serving cohorts take tens of seconds)."""
    k = name
    if k not in _COHORTS:
        coh = getattr(synth, name)()
        coh["X64"] = coh["X"] if coh["X"].dtype == np.float64 else coh["X"].astype(np.float64)
        _COHORTS[k] = coh
    return _COHORTS[k]


@pytest.fixture(scope="module")
def napg():
    from paper_2505_00448_gb300 import napg as N
    return N


def sampled(test, coh, g, va, vb, rng, k, mask=None, bar=None, **kw):
    """k random pairs of the n_a x n_b output plus the first 64 x 64 block."""
    na = len(va)
    nb = na if vb is None else len(vb)
    ia = rng.integers(0, na, k)
    ib = rng.integers(0, nb, k)
    sa, sb = np.meshgrid(np.arange(min(64, na)), np.arange(min(64, nb)), indexing="ij")
    ia = np.concatenate([ia, sa.ravel()])
    ib = np.concatenate([ib, sb.ravel()])
    pa = np.asarray(va)[ia]
    pb = (np.asarray(va) if vb is None else np.asarray(vb))[ib]
    ref = oracle_run_pairs(test, coh, pa, pb, mask=mask, **kw)
    got = {k2: (v.cpu().numpy() if hasattr(v, "cpu") else np.asarray(v))[ia, ib] for k2, v in g.items()}
    compare(test, got, ref, stat_tol=bar)


def test_small_pearson_full(napg):
    coh = cohort("small_pearson_cohort")
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    va = coh["cont"]
    g = c.run("pearson", va, out="numpy")
    compare("pearson", g, oracle_run("pearson", coh, va))
    c.close()


def test_rank_cohort_full_size(napg):
    rng = np.random.default_rng(2)
    coh = cohort("rank_cohort")
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    cat, cont = coh["cat"], coh["cont"]
    bins, multi = cat[coh["nlev"][cat] == 2], cat[coh["nlev"][cat] >= 3]
    sampled("spearman", coh, c.run("spearman", cont, out="cuda"), cont, None, rng, 300)
    sampled("mwu", coh, c.run("mwu", bins, cont, out="cuda", mwu_mode="asymptotic"), bins, cont, rng, 300, mwu_mode=2)
    sampled("kruskal", coh, c.run("kruskal", multi, cont, out="cuda"), multi, cont, rng, 300)
    c.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_mixed_cohort_full_size(napg, precision):
    rng = np.random.default_rng(3)
    coh = cohort("mixed_cohort")
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    cat, cont = coh["cat"], coh["cont"]
    bins = cat[coh["nlev"][cat] == 2]
    bar = MIXED_BAR if precision == "mixed" else {}
    for test, va, vb in (("pearson", cont, None), ("anova", cat, cont), ("ttest", bins, cont), ("chi2", cat, None)):
        if precision == "fp64" and test == "pearson":
            va = cont[:1500]                    # the FP64 form of the full triangle takes seconds
        g = c.run(test, va, vb, out="cuda", precision=precision)
        sampled(test, coh, g, va, vb, rng, 200, bar=bar.get(test))
    c.close()


def test_context_batch_full_size(napg):
    rng = np.random.default_rng(4)
    coh = cohort("context_cohort")
    masks = coh["contexts"]
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    dm = c.torch.from_numpy(masks).to(c.torch.device("cuda", 0))
    mlist = [dm[k] for k in range(len(masks))]
    for test, va, bar in (("pearson", coh["cont"], ("abs", 1e-6)), ("chi2", coh["cat"], None)):
        g = c.run_batch(test, mlist, va, out="cuda", precision="mixed")
        for k in rng.choice(len(masks), size=3, replace=False):
            sampled(test, coh, g[k], va, None, rng, 100, mask=masks[k], bar=bar)
    c.close()


def test_serving_cohort_requests(napg):
    rng = np.random.default_rng(5)
    coh = cohort("serving_cohort")
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    S = coh["X"].shape[1]
    mask = (rng.random(S) < 0.5).astype(np.uint8)
    va = np.sort(rng.choice(coh["cont"], 600, replace=False))
    sampled("pearson", coh, c.run("pearson", va, mask=mask, out="cuda", precision="mixed"), va, None, rng, 200,
            mask=mask, bar=("abs", 1e-6))
    vs = va[:120]
    sampled("spearman", coh, c.run("spearman", vs, mask=mask, out="cuda"), vs, None, rng, 100, mask=mask)
    cats = np.sort(rng.choice(coh["cat"], 200, replace=False))
    sampled("chi2", coh, c.run("chi2", cats, mask=mask, out="cuda", precision="mixed"), cats, None, rng, 200,
            mask=mask)
    kw_cats = cats[np.asarray(coh["nlev"])[cats] >= 3][:40]
    sampled("kruskal", coh, c.run("kruskal", kw_cats, vs, mask=mask, out="cuda"), kw_cats, vs, rng, 100, mask=mask)
    c.close()
