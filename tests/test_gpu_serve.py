"""The serving loop on the resident cohort: concurrent requests (continuous
batching over slots and streams) give the same results as each request alone,
and as the oracle; admission by memory; busy rules while serving."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_00448_gb300 import synth
from tests._parity import compare, oracle_run

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def napg():
    from paper_2505_00448_gb300 import napg as N
    return N




def make_requests(coh, rng, count):
    S = coh["X"].shape[1]
    cont, cats = coh["cont"], coh["cat"]
    binary = np.array([v for v in cats if coh["nlev"][v] == 2], np.int32)
    multi = np.array([v for v in cats if coh["nlev"][v] > 2], np.int32)
    kinds = ["pearson", "spearman", "chi2", "kruskal", "anova", "ttest", "mwu"]
    reqs = []
    for q in range(count):
        test = kinds[q % len(kinds)]
        mask = None if q % 5 == 0 else (rng.random(S) < rng.uniform(0.05, 0.8)).astype(np.uint8)
        prec = "mixed" if q % 2 else "fp64"
        if test in ("pearson", "spearman"):
            va, vb = np.sort(rng.choice(cont, size=int(rng.integers(3, len(cont))), replace=False)), None
        elif test == "chi2":
            va, vb = np.sort(rng.choice(cats, size=int(rng.integers(2, len(cats))), replace=False)), None
        else:
            pool = binary if test in ("ttest", "mwu") else (multi if test == "kruskal" else cats)
            va = np.sort(rng.choice(pool, size=int(rng.integers(1, len(pool) + 1)), replace=False))
            vb = np.sort(rng.choice(cont, size=int(rng.integers(2, len(cont))), replace=False))
        opt = {"precision": prec}
        if test == "mwu":
            opt["mwu_mode"] = "asymptotic"
        reqs.append((test, va, vb, mask, opt))
    return reqs


def test_concurrent_requests_match_alone_and_oracle(napg):
    rng = np.random.default_rng(61)
    coh = synth.small_cohort(401, n_cont=60, n_cat=14, S=3000 + 11, miss=0.2, dtype=np.float32, binary_cats=6)
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    reqs = make_requests(coh, rng, 21)
    alone = [c.run(t, va, vb, mask=m, out="numpy", **o) for t, va, vb, m, o in reqs]
    c.serve_start(mem_budget=0, slots=4)
    tickets = [c.serve_submit(t, va, vb, mask=m, **o) for t, va, vb, m, o in reqs]
    got = []
    for tk in tickets:
        lat, st, out = c.serve_wait(tk)
        assert st == 0 and lat > 0
        got.append(out)
    c.serve_stop()
    for (t, va, vb, m, o), a, g in zip(reqs, alone, got):
        for k in ("stat", "p", "n"):
            assert np.array_equal(a[k], g[k], equal_nan=True), (t, k)
    # and against the oracle for a few of them
    for q in (0, 3, 8):
        t, va, vb, m, o = reqs[q]
        bar = ("abs", 1e-6) if (t == "pearson" and o["precision"] == "mixed") else None
        if t in ("anova", "ttest") and o["precision"] == "mixed":
            bar = ("effect", 1e-6)
        kw = {"mwu_mode": 2} if t == "mwu" else {}
        compare(t, got[q], oracle_run(t, coh, va, vb, mask=m, **kw), stat_tol=bar)
    c.close()


def test_admission_by_memory_and_busy_rules(napg):
    rng = np.random.default_rng(62)
    coh = synth.small_cohort(402, n_cont=40, n_cat=6, S=2000 + 1, miss=0.2, dtype=np.float32)
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    va = coh["cont"]
    ref = c.run("pearson", va, out="numpy")
    # a budget that holds about one request at a time: requests still all complete
    c.serve_start(mem_budget=3 << 20, slots=4)
    with pytest.raises(napg.NapgError) as e:
        c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    assert e.value.code == napg.E_BUSY
    with pytest.raises(napg.NapgError) as e:
        c.release_cache()
    assert e.value.code == napg.E_BUSY
    tickets = [c.serve_submit("pearson", va) for _ in range(6)]
    for tk in tickets:
        lat, st, out = c.serve_wait(tk)
        assert st == 0
        for k in ("stat", "p", "n"):
            assert np.array_equal(out[k], ref[k], equal_nan=True)
    # larger than the whole budget: refused at submission
    with pytest.raises(napg.NapgError) as e:
        c.serve_submit("spearman", np.concatenate([va] * 30))
    assert e.value.code == napg.E_UNSUPPORTED
    c.serve_stop()
    c.serve_stop()            # stopping twice is harmless
    c.close()
