"""Seeded synthetic cohorts (variables x samples) for tests and benchmarks.

This module only draws inputs: it computes no statistic. Both the GPU path and
the CPU oracle consume what it returns.

A cohort is a dict with
  X      (F, S) float32 or float64, row-major, one row per variable;
         categorical labels are stored as floats 0.0 .. c-1 (Sec. 3.2);
  vtype  (F,) uint8, 0 continuous, 1 categorical;
  nlev   (F,) int32, level count c per categorical variable (0 for continuous);
  missing  the sentinel (NaN here);
  cont, cat  index arrays of the continuous / categorical variables.

The five workload recipes follow the synthetic stand-ins for the paper's
cohort data (the CHRIS cohort of Sec. 4.1.2 is not available; its mixed-type
shape with heavy missingness is reproduced at larger scale):
  1  200 continuous x 1,000 samples, FP64, 5-factor model, 20% MCAR.
  2  1,000 continuous (rounded to 1 decimal: heavy ties, 30% MCAR plus block
     losses) + 200 categorical (2-8 levels, Dirichlet(1), 10% MCAR), 10,000 samples.
  3  4,000 continuous FP32 (2,000 Gaussian with offsets up to 1e4 sigma,
     2,000 lognormal(0,1.5)) + 1,000 categorical (2-10 levels), 50,000 samples,
     per-column missing rate ~ Beta(2,5).
  4  1,600 continuous FP32 + 400 categorical (2-6 levels), 20,000 samples,
     25% MCAR, plus 256 sample contexts of uneven size (500-20,000).
  5  8,000 continuous FP32 + 2,000 categorical (2-8 levels), 100,000 samples,
     35% MCAR.
Seeds are PCG64(20250501 + config id).
"""
from __future__ import annotations

import numpy as np

BASE_SEED = 20250501


def rng_for(config_id: int, salt: int = 0) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(BASE_SEED + config_id + 1000 * salt))


def factor_scores(rng, n_vars, n_samples, n_factors=5, dtype=np.float64, chunk=512):
    """Standardised rows of L Z + e with L ~ N(0,1)^{n_vars x k}, Z ~ N(0,1)^{k x S}."""
    L = rng.standard_normal((n_vars, n_factors))
    Z = rng.standard_normal((n_factors, n_samples))
    out = np.empty((n_vars, n_samples), dtype)
    for r0 in range(0, n_vars, chunk):
        r1 = min(n_vars, r0 + chunk)
        z = L[r0:r1] @ Z + rng.standard_normal((r1 - r0, n_samples))
        z -= z.mean(axis=1, keepdims=True)
        z /= z.std(axis=1, keepdims=True)
        out[r0:r1] = z
    return out


def categorical_rows(rng, n_vars, n_samples, lev_lo, lev_hi, dtype=np.float64):
    """Labels with c ~ U{lev_lo..lev_hi}, level probabilities Dirichlet(1_c);
    every level is forced to appear at least once in its row (Sec. 4.1.1)."""
    nlev = rng.integers(lev_lo, lev_hi + 1, size=n_vars).astype(np.int32)
    out = np.empty((n_vars, n_samples), dtype)
    for v in range(n_vars):
        c = int(nlev[v])
        p = rng.dirichlet(np.ones(c))
        lab = rng.choice(c, size=n_samples, p=p)
        pos = rng.choice(n_samples, size=c, replace=False)
        lab[pos] = np.arange(c)
        out[v] = lab
    return out, nlev


def apply_mcar(rng, X, rate, protect_levels=None):
    """Set entries to NaN independently with probability `rate` (scalar or per row)."""
    rate = np.broadcast_to(np.asarray(rate, dtype=np.float64).reshape(-1, 1), (X.shape[0], 1))
    for r0 in range(0, X.shape[0], 256):
        r1 = min(X.shape[0], r0 + 256)
        m = rng.random((r1 - r0, X.shape[1])) < rate[r0:r1]
        X[r0:r1][m] = np.nan
    return X


def assemble(cont_X, cat_X, cat_nlev, dtype):
    Fc = 0 if cont_X is None else cont_X.shape[0]
    Fg = 0 if cat_X is None else cat_X.shape[0]
    S = (cont_X if cont_X is not None else cat_X).shape[1]
    X = np.empty((Fc + Fg, S), dtype)
    if Fc:
        X[:Fc] = cont_X
    if Fg:
        X[Fc:] = cat_X
    vtype = np.zeros(Fc + Fg, np.uint8)
    vtype[Fc:] = 1
    nlev = np.zeros(Fc + Fg, np.int32)
    if Fg:
        nlev[Fc:] = cat_nlev
    return {"X": X, "vtype": vtype, "nlev": nlev, "missing": float("nan"),
            "cont": np.arange(Fc, dtype=np.int32), "cat": np.arange(Fc, Fc + Fg, dtype=np.int32)}


def small_pearson_cohort():
    """200 continuous x 1,000 samples, FP64, 20% MCAR."""
    rng = rng_for(1)
    z = factor_scores(rng, 200, 1000)
    sigma = rng.uniform(0.1, 10.0, size=(200, 1))
    mu = rng.uniform(-100.0, 100.0, size=(200, 1))
    X = mu + sigma * z
    apply_mcar(rng, X, 0.2)
    return assemble(X, None, None, np.float64)


def rank_cohort(n_cont=1000, n_cat=200, S=10_000):
    """Rank-test cohort: tied continuous columns with block losses + categoricals."""
    rng = rng_for(2)
    z = np.round(factor_scores(rng, n_cont, S), 1)
    apply_mcar(rng, z, 0.3)
    blocks = rng.choice(n_cont, size=max(1, n_cont // 10), replace=False)
    for v in blocks:
        length = int(round(rng.uniform(0.05, 0.30) * S))
        start = int(rng.integers(0, S - length + 1))
        z[v, start:start + length] = np.nan
    cat, nlev = categorical_rows(rng, n_cat, S, 2, 8)
    apply_mcar(rng, cat, 0.1)
    return assemble(z, cat, nlev, np.float64)


def mixed_cohort(n_cont=4000, n_cat=1000, S=50_000):
    """Mixed-type FP32 cohort with large offsets and heavy tails."""
    rng = rng_for(3)
    half = n_cont // 2
    z = factor_scores(rng, n_cont, S, dtype=np.float64)
    X = np.empty((n_cont, S), np.float32)
    sigma = rng.uniform(0.1, 10.0, size=(half, 1))
    mu = sigma * rng.uniform(-1e4, 1e4, size=(half, 1))
    X[:half] = (mu + sigma * z[:half]).astype(np.float32)
    X[half:] = np.exp(1.5 * z[half:]).astype(np.float32)
    del z
    rates = rng.beta(2.0, 5.0, size=n_cont)
    apply_mcar(rng, X, rates)
    cat, nlev = categorical_rows(rng, n_cat, S, 2, 10, dtype=np.float32)
    apply_mcar(rng, cat, rng.beta(2.0, 5.0, size=n_cat))
    return assemble(X, cat, nlev, np.float32)


def context_cohort(n_cont=1600, n_cat=400, S=20_000, n_ctx=256):
    """Cohort plus n_ctx sample contexts (uint8 masks) of uneven size."""
    rng = rng_for(4)
    z = factor_scores(rng, n_cont, S)
    sigma = rng.uniform(0.1, 10.0, size=(n_cont, 1))
    mu = rng.uniform(-100.0, 100.0, size=(n_cont, 1))
    X = (mu + sigma * z).astype(np.float32)
    apply_mcar(rng, X, 0.25)
    cat, nlev = categorical_rows(rng, n_cat, S, 2, 6, dtype=np.float32)
    apply_mcar(rng, cat, 0.25)
    coh = assemble(X, cat, nlev, np.float32)
    sizes = np.rint(np.exp(rng.uniform(np.log(500), np.log(S), size=n_ctx))).astype(np.int64)
    masks = np.zeros((n_ctx, S), np.uint8)
    for k in range(n_ctx):
        score = rng.random(S)
        masks[k, np.argsort(score, kind="stable")[:sizes[k]]] = 1
    coh["contexts"] = masks
    return coh


def serving_cohort(n_cont=8000, n_cat=2000, S=100_000):
    """Serving cohort, 35% MCAR."""
    rng = rng_for(5)
    X = np.empty((n_cont + n_cat, S), np.float32)
    for r0 in range(0, n_cont, 1000):
        r1 = min(n_cont, r0 + 1000)
        z = factor_scores(rng, r1 - r0, S)
        sigma = rng.uniform(0.1, 10.0, size=(r1 - r0, 1))
        mu = rng.uniform(-100.0, 100.0, size=(r1 - r0, 1))
        X[r0:r1] = (mu + sigma * z).astype(np.float32)
    cat, nlev = categorical_rows(rng, n_cat, S, 2, 8, dtype=np.float32)
    X[n_cont:] = cat
    apply_mcar(rng, X, 0.35)
    vtype = np.zeros(n_cont + n_cat, np.uint8)
    vtype[n_cont:] = 1
    lev = np.zeros(n_cont + n_cat, np.int32)
    lev[n_cont:] = nlev
    return {"X": X, "vtype": vtype, "nlev": lev, "missing": float("nan"),
            "cont": np.arange(n_cont, dtype=np.int32),
            "cat": np.arange(n_cont, n_cont + n_cat, dtype=np.int32)}


def small_cohort(seed, n_cont=12, n_cat=6, S=300, miss=0.2, lev_lo=2, lev_hi=5, ties=False,
                 dtype=np.float64, offset=0.0, lognormal=False, binary_cats=0):
    """A small mixed cohort for parity tests: factor-model continuous columns
    (optionally rounded to force ties, shifted by `offset`, or lognormal) and
    Dirichlet categoricals; `binary_cats` of the categoricals have exactly 2 levels."""
    rng = np.random.Generator(np.random.PCG64(BASE_SEED + 7919 * (seed + 1)))
    cont = None
    if n_cont:
        z = factor_scores(rng, n_cont, S)
        if lognormal:
            cont = np.exp(1.5 * z)
        else:
            sigma = rng.uniform(0.1, 10.0, size=(n_cont, 1))
            cont = offset * sigma + sigma * z
        if ties:
            cont = np.round(cont, 0 if not lognormal else 1)
        apply_mcar(rng, cont, miss)
    cat = nlev = None
    if n_cat:
        cat, nlev = categorical_rows(rng, n_cat, S, lev_lo, lev_hi)
        if binary_cats:
            b, bl = categorical_rows(rng, binary_cats, S, 2, 2)
            cat = np.concatenate([b, cat[binary_cats:]]) if binary_cats < n_cat else b
            nlev = np.concatenate([bl, nlev[binary_cats:]]) if binary_cats < n_cat else bl
        apply_mcar(rng, cat, miss)
    return assemble(cont, cat, nlev, dtype)


def poisson_requests(rng, n_req, rate_per_s, n_samples, cont_ids, cat_ids, tests=("pearson", "spearman", "chi2", "kruskal"),
                     frac_lo=0.05, frac_hi=0.8, vars_lo=50, vars_hi=2000):
    """Serving workload: Poisson arrival times and per-request (test, sample mask, variables)."""
    gaps = rng.exponential(1.0 / rate_per_s, size=n_req)
    t = np.cumsum(gaps)
    reqs = []
    for k in range(n_req):
        test = tests[int(rng.integers(0, len(tests)))]
        frac = rng.uniform(frac_lo, frac_hi)
        mask = (rng.random(n_samples) < frac).astype(np.uint8)
        nv = int(rng.integers(vars_lo, vars_hi + 1))
        if test in ("pearson", "spearman"):
            va = np.sort(rng.choice(cont_ids, size=min(nv, len(cont_ids)), replace=False)).astype(np.int32)
            vb = None
        elif test == "chi2":
            va = np.sort(rng.choice(cat_ids, size=min(nv, len(cat_ids)), replace=False)).astype(np.int32)
            vb = None
        else:
            h = max(1, nv // 2)
            va = np.sort(rng.choice(cat_ids, size=min(h, len(cat_ids)), replace=False)).astype(np.int32)
            vb = np.sort(rng.choice(cont_ids, size=min(nv - h, len(cont_ids)), replace=False)).astype(np.int32)
        reqs.append({"t": float(t[k]), "test": test, "mask": mask, "vars_a": va, "vars_b": vb})
    return reqs


def paper_simulation(F, S, c=4, miss=0.1, seed=0):
    """The paper's simulated benchmark data (Sec. 4.1.1): F continuous features
    with values uniform on [0, 1], F categorical features with labels in
    {0..c-1} and F dichotomous features (labels {0, 1}), S samples; in every
    feature exactly round(miss S) samples are missing (NaN) at random positions,
    and every category of a categorical or dichotomous feature appears at least
    once among its observed samples (reading: the categories are forced after
    the missing positions are drawn). Rows: [continuous | categorical |
    dichotomous]."""
    rng = rng_for(100 + seed, salt=F * 10007 + S)
    k = int(round(miss * S))
    cont = rng.random((F, S))
    labs = []
    for levels in (c, 2):
        out = np.empty((F, S))
        for v in range(F):
            lab = rng.integers(0, levels, S).astype(float)
            miss_pos = rng.choice(S, k, replace=False)
            keep = np.setdiff1d(np.arange(S), miss_pos)
            force = rng.choice(keep, levels, replace=False)
            lab[force] = np.arange(levels)
            lab[miss_pos] = np.nan
            out[v] = lab
        labs.append(out)
    for v in range(F):
        cont[v, rng.choice(S, k, replace=False)] = np.nan
    X = np.concatenate([cont, labs[0], labs[1]])
    vtype = np.concatenate([np.zeros(F, np.uint8), np.ones(2 * F, np.uint8)])
    nlev = np.concatenate([np.zeros(F, np.int32), np.full(F, c, np.int32), np.full(F, 2, np.int32)])
    return {"X": X, "vtype": vtype, "nlev": nlev, "missing": float("nan"),
            "cont": np.arange(F, dtype=np.int32), "cat": np.arange(F, 2 * F, dtype=np.int32),
            "bins": np.arange(2 * F, 3 * F, dtype=np.int32)}

