"""The seeded synthetic cohorts follow the recipes the benchmark and the parity
tests are described with: sizes, dtypes, missingness, level counts, ties,
context sizes and the paper's simulation (Sec. 4.1.1). Host only; the large
cohorts are checked at reduced variable counts where the generator takes them."""
import numpy as np

from paper_2505_00448_gb300 import synth


def _levels_present(X, cat, nlev):
    for v in cat:
        obs = X[v][~np.isnan(X[v])]
        assert np.all(obs == np.floor(obs)) and obs.min() >= 0 and obs.max() < nlev[v]
        assert len(np.unique(obs)) == nlev[v], f"variable {v}: a level is absent"


def test_seeded_and_repeatable():
    a, b = synth.small_pearson_cohort(), synth.small_pearson_cohort()
    assert np.array_equal(a["X"], b["X"], equal_nan=True)
    p, q = synth.paper_simulation(20, 250), synth.paper_simulation(20, 250)
    assert np.array_equal(p["X"], q["X"], equal_nan=True)
    assert not np.array_equal(synth.paper_simulation(20, 250, seed=1)["X"], p["X"], equal_nan=True)


def test_small_pearson_recipe():
    c = synth.small_pearson_cohort()
    X = c["X"]
    assert X.shape == (200, 1000) and X.dtype == np.float64
    assert np.all(c["vtype"] == 0)
    assert abs(np.isnan(X).mean() - 0.2) < 0.01
    mu = np.nanmean(X, axis=1)
    sd = np.nanstd(X, axis=1)
    assert np.all(np.abs(mu) < 100 + 5 * sd) and sd.min() > 0.05 and sd.max() < 15
    # the 5-factor model: columns share variance (mean |r| well above independent columns')
    Z = np.where(np.isnan(X), np.nan, (X - mu[:, None]) / sd[:, None])
    r = np.nanmean(Z[:20, None, :] * Z[None, :20, :], axis=2)
    assert np.mean(np.abs(r[np.triu_indices(20, 1)])) > 0.2


def test_rank_recipe():
    c = synth.rank_cohort()
    X, cont, cat, nlev = c["X"], c["cont"], c["cat"], c["nlev"]
    assert X.shape == (1200, 10_000) and len(cont) == 1000 and len(cat) == 200
    V = X[cont]
    obs = V[~np.isnan(V)]
    assert np.array_equal(np.round(obs * 10), obs * 10)          # one decimal: ties
    distinct = np.median([len(np.unique(r[~np.isnan(r)])) for r in V[:50]])
    assert 40 <= distinct <= 120
    # 30% MCAR plus a contiguous missing block in a tenth of the columns
    assert 0.30 < np.isnan(V).mean() < 0.34
    runs = 0
    for r in np.isnan(V):
        d = np.diff(np.concatenate([[0], r.astype(np.int8), [0]]))
        longest = (np.flatnonzero(d == -1) - np.flatnonzero(d == 1)).max()
        runs += longest >= 500
    assert runs >= 100
    assert nlev[cat].min() >= 2 and nlev[cat].max() <= 8
    assert abs(np.isnan(X[cat]).mean() - 0.1) < 0.005
    _levels_present(X, cat, nlev)


def test_mixed_recipe_scaled():
    c = synth.mixed_cohort(n_cont=60, n_cat=20, S=5_000)
    X, cont, cat, nlev = c["X"], c["cont"], c["cat"], c["nlev"]
    assert X.dtype == np.float32 and X.shape == (80, 5_000)
    g, ln = X[cont[:30]], X[cont[30:]]
    mu, sd = np.nanmean(g.astype(np.float64), axis=1), np.nanstd(g.astype(np.float64), axis=1)
    assert np.max(np.abs(mu) / sd) > 1_000                       # offsets up to 1e4 sigma
    assert np.nanmin(ln) > 0                                      # lognormal half
    rates = np.isnan(X[cont]).mean(axis=1)
    assert 0.15 < rates.mean() < 0.42 and rates.std() > 0.05     # Beta(2, 5) per column
    assert nlev[cat].min() >= 2 and nlev[cat].max() <= 10


def test_context_recipe():
    c = synth.context_cohort()
    X, masks = c["X"], c["contexts"]
    assert X.shape == (2_000, 20_000) and X.dtype == np.float32
    assert masks.shape == (256, 20_000) and masks.dtype == np.uint8
    sizes = masks.sum(axis=1)
    assert sizes.min() >= 500 and sizes.max() <= 20_000
    # log-uniform sizes: the median near sqrt(500 * 20,000)
    assert 1_500 < np.median(sizes) < 7_000
    assert abs(np.isnan(X).mean() - 0.25) < 0.005
    assert c["nlev"][c["cat"]].min() >= 2 and c["nlev"][c["cat"]].max() <= 6


def test_serving_recipe_scaled():
    c = synth.serving_cohort(n_cont=40, n_cat=10, S=20_000)
    X, cat, nlev = c["X"], c["cat"], c["nlev"]
    assert X.dtype == np.float32
    assert abs(np.isnan(X).mean() - 0.35) < 0.01
    assert nlev[cat].min() >= 2 and nlev[cat].max() <= 8


def test_paper_simulation_recipe():
    F, S = 30, 250
    c = synth.paper_simulation(F, S)
    X, vtype, nlev = c["X"], c["vtype"], c["nlev"]
    assert X.shape == (3 * F, S)
    # exactly 10% of every feature missing
    assert np.all(np.isnan(X).sum(axis=1) == round(0.1 * S))
    cont = X[:F]
    obs = cont[~np.isnan(cont)]
    assert obs.min() >= 0.0 and obs.max() < 1.0
    assert np.all(vtype[:F] == 0) and np.all(vtype[F:] == 1)
    assert np.all(nlev[F:2 * F] == 4) and np.all(nlev[2 * F:] == 2)
    _levels_present(X, np.arange(F, 3 * F), nlev)
