"""Batched sample contexts (napg_run_batch): every context of a batch equals the
oracle on that context (Sec. 3.3: a sample context is a submatrix call), both
through the captured-graph path (device outputs) and the per-context loop (host
outputs); the graph is reused for a new batch of the same shape and rebuilt for
another."""
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




def ctx_masks(rng, S, sizes):
    """Masks selecting `sizes` random samples (None = every sample)."""
    out = []
    for k in sizes:
        if k is None:
            out.append(None)
            continue
        m = np.zeros(S, np.uint8)
        m[rng.choice(S, size=k, replace=False)] = 1
        out.append(m)
    return out


def host(r):
    return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in r.items()}


BARS = {"mixed": {"pearson": ("abs", 1e-6), "anova": ("effect", 1e-6), "ttest": ("effect", 1e-6)},
        "fp64": {}}


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_pearson_chi2_graph_and_loop(napg, precision):
    rng = np.random.default_rng(41)
    coh = synth.small_cohort(301, n_cont=90, n_cat=14, S=1500 + 21, miss=0.25, dtype=np.float32)
    S = coh["X"].shape[1]
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    sizes = [None, 700, 0, 5, 1200, 64, 333, 1]
    masks = ctx_masks(rng, S, sizes)
    for test, va in (("pearson", coh["cont"]), ("chi2", coh["cat"])):
        bar = BARS[precision].get(test)
        g = c.run_batch(test, masks, va, out="cuda", precision=precision)        # graph path
        h = c.run_batch(test, masks, va, out="numpy", precision=precision)       # per-context loop
        for k, m in enumerate(masks):
            ref = oracle_run(test, coh, va, mask=m)
            compare(test, host(g[k]), ref, stat_tol=bar)
            compare(test, h[k], ref, stat_tol=bar)
            assert np.array_equal(host(g[k])["n"], h[k]["n"])
    c.close()


def test_batch_graph_reuse_and_rebuild(napg):
    rng = np.random.default_rng(42)
    coh = synth.small_cohort(302, n_cont=70, n_cat=0, S=1200 + 7, miss=0.3, dtype=np.float32)
    S = coh["X"].shape[1]
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    va = coh["cont"]
    sizes = [500, 900, 31]
    dev = c.torch.device("cuda", 0)
    outs = [{"stat": c.torch.empty((70, 70), dtype=c.torch.float64, device=dev),
             "p": c.torch.empty((70, 70), dtype=c.torch.float64, device=dev),
             "n": c.torch.empty((70, 70), dtype=c.torch.int32, device=dev)} for _ in sizes]
    l0 = napg.kernel_launches()
    m1 = ctx_masks(rng, S, sizes)
    c.run_batch("pearson", m1, va, out="cuda", outputs=outs, precision="mixed")
    first = napg.kernel_launches() - l0
    for k, m in enumerate(m1):
        compare("pearson", host(outs[k]), oracle_run("pearson", coh, va, mask=m), stat_tol=("abs", 1e-6))
    # same sizes and buffers, new mask contents: the same graph runs again
    m2 = ctx_masks(rng, S, sizes)
    l1 = napg.kernel_launches()
    c.run_batch("pearson", m2, va, out="cuda", outputs=outs, precision="mixed")
    again = napg.kernel_launches() - l1
    assert 0 < again < first, (first, again)       # no sizing run this time
    for k, m in enumerate(m2):
        compare("pearson", host(outs[k]), oracle_run("pearson", coh, va, mask=m), stat_tol=("abs", 1e-6))
    # device masks, other sizes: rebuilt
    m3 = ctx_masks(rng, S, [100, 1100])
    dm = [c.torch.from_numpy(m).to(dev) for m in m3]
    g = c.run_batch("pearson", dm, va, out="cuda", precision="mixed")
    for k, m in enumerate(m3):
        compare("pearson", host(g[k]), oracle_run("pearson", coh, va, mask=m), stat_tol=("abs", 1e-6))
    c.close()


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_mixed_type_tests(napg, precision):
    rng = np.random.default_rng(43)
    coh = synth.small_cohort(303, n_cont=40, n_cat=10, S=1400 + 3, miss=0.2, dtype=np.float32, binary_cats=5)
    S = coh["X"].shape[1]
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    masks = ctx_masks(rng, S, [800, None, 150, 0])
    cont = coh["cont"]
    cats = coh["cat"]
    binary = np.array([v for v in cats if coh["nlev"][v] == 2], np.int32)
    for test, va in (("anova", cats), ("ttest", binary)):
        g = c.run_batch(test, masks, va, cont, out="cuda", precision=precision)
        for k, m in enumerate(masks):
            compare(test, host(g[k]), oracle_run(test, coh, va, cont, mask=m), stat_tol=BARS[precision].get(test))
    c.close()


def test_batch_rank_tests(napg):
    """Spearman, Mann-Whitney and Kruskal-Wallis per context: the presort is
    rebuilt inside the graph for every compacted context; rank sums exact."""
    rng = np.random.default_rng(44)
    coh = synth.small_cohort(304, n_cont=30, n_cat=8, S=1000 + 9, miss=0.2, ties=True, binary_cats=4)
    S = coh["X"].shape[1]
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    masks = ctx_masks(rng, S, [600, 37, None])
    cont, cats = coh["cont"], coh["cat"]
    binary = np.array([v for v in cats if coh["nlev"][v] == 2], np.int32)
    multi = np.array([v for v in cats if coh["nlev"][v] > 2], np.int32)
    g = c.run_batch("spearman", masks, cont, out="cuda")
    for k, m in enumerate(masks):
        compare("spearman", host(g[k]), oracle_run("spearman", coh, cont, mask=m))
    for test, va in (("mwu", binary), ("kruskal", multi)):
        g = c.run_batch(test, masks, va, cont, out="cuda", mwu_mode="asymptotic")
        for k, m in enumerate(masks):
            compare(test, host(g[k]), oracle_run(test, coh, va, cont, mask=m, mwu_mode=2))
    c.close()
