"""Comparison helpers shared by the GPU parity tests (test infrastructure)."""
import math

import numpy as np

from oracle import oracle as O

# |delta| bars (the plain FP64 path): correlation coefficients absolute; the other
# statistics ("rel") absolute up to 1 and relative above it, since F or t near 0
# carries the cancellation of its mean differences; counts and U exact.
STAT_TOL = {"pearson": ("abs", 1e-12), "spearman": ("abs", 1e-12), "chi2": ("rel", 1e-12),
            "anova": ("rel", 1e-12), "ttest": ("rel", 1e-12), "mwu": ("exact", 0.0),
            "kruskal": ("rel", 1e-12)}
P_REL = 1e-12


class Ref(tuple):
    """The oracle's (stat, p, n) with the degrees of freedom of each pair's
    p-value beside it (`dof`: a dict of arrays, see pair_dof)."""
    dof = None


def present_levels(coh, v, mask=None):
    """Levels of categorical variable v observed within the sample context
    (before pairwise deletion): the categories of the call."""
    x = np.asarray(coh["X"][v], dtype=np.float64)
    miss = coh["missing"]
    obs = ~np.isnan(x) if (isinstance(miss, float) and math.isnan(miss)) else (x != miss)
    if mask is not None:
        obs &= np.asarray(mask).astype(bool)
    return len(np.unique(x[obs]))


def pair_dof(test, coh, va, vb, n, mask=None, welch=1):
    """Degrees of freedom of each pair's p-value, from the data and the exact
    co-observed counts n: F (k - 1, n - k) with k the present levels, Student t
    n - 2, Welch t the oracle's Welch-Satterthwaite value, chi-squared
    (k_a - 1)(k_b - 1), Kruskal-Wallis k - 1; for the correlation tests the
    p-function's argument is n itself."""
    n = np.asarray(n, dtype=np.float64)
    if test in ("pearson", "spearman"):
        return {"n": n}
    if test == "anova":
        k = np.array([present_levels(coh, a, mask) for a in va], dtype=np.float64)[:, None]
        return {"d1": np.broadcast_to(k - 1, n.shape), "d2": n - k}
    if test == "kruskal":
        k = np.array([present_levels(coh, a, mask) for a in va], dtype=np.float64)[:, None]
        return {"df": np.broadcast_to(k - 1, n.shape).copy()}
    if test == "chi2":
        kb_vars = va if vb is None else vb
        ka = np.array([present_levels(coh, a, mask) for a in va], dtype=np.float64)[:, None]
        kb = np.array([present_levels(coh, b, mask) for b in kb_vars], dtype=np.float64)[None, :]
        return {"df": (ka - 1) * (kb - 1)}
    if test == "ttest":
        if not welch:
            return {"df": n - 2}
        _, nu = O.effects("ttest", np.asarray(coh["X"], dtype=np.float64), coh["missing"], coh["vtype"], coh["nlev"],
                          va, vb, ctx=mask, welch=1)
        return {"df": nu}
    return None


def _welch_nu(x, y, obs_x, obs_y, mask=None):
    """Welch-Satterthwaite degrees of freedom of one pair (two-pass FP64)."""
    keep = obs_x & obs_y
    if mask is not None:
        keep &= np.asarray(mask).astype(bool)
    lab, v = x[keep], y[keep]
    g0, g1 = v[lab == 0], v[lab == 1]
    if len(g0) < 2 or len(g1) < 2:
        return math.nan
    a0, a1 = np.var(g0, ddof=1) / len(g0), np.var(g1, ddof=1) / len(g1)
    den = a0 * a0 / (len(g0) - 1) + a1 * a1 / (len(g1) - 1)
    return (a0 + a1) ** 2 / den if den > 0 else math.nan


def pairs_dof(test, coh, pa, pb, n, mask=None, welch=1):
    """pair_dof for a list of pairs (pa[k], pb[k])."""
    n = np.asarray(n, dtype=np.float64)
    if test in ("pearson", "spearman"):
        return {"n": n}
    lev = {}

    def k_of(v):
        if v not in lev:
            lev[v] = present_levels(coh, v, mask)
        return lev[v]
    if test in ("anova", "kruskal"):
        k = np.array([k_of(a) for a in pa], dtype=np.float64)
        return {"d1": k - 1, "d2": n - k} if test == "anova" else {"df": k - 1}
    if test == "chi2":
        return {"df": np.array([(k_of(a) - 1) * (k_of(b) - 1) for a, b in zip(pa, pb)], dtype=np.float64)}
    if test == "ttest":
        if not welch:
            return {"df": n - 2}
        X = np.asarray(coh["X"], dtype=np.float64)
        miss = coh["missing"]
        isnan_m = isinstance(miss, float) and math.isnan(miss)
        obs = lambda v: ~np.isnan(X[v]) if isnan_m else X[v] != miss
        return {"df": np.array([_welch_nu(X[a], X[b], obs(a), obs(b), mask) for a, b in zip(pa, pb)])}
    return None


def oracle_run_pairs(test, coh, pa, pb, mask=None, **kw):
    """The oracle on listed pairs, with their degrees of freedom attached."""
    X = coh["X64"] if "X64" in coh else np.asarray(coh["X"], dtype=np.float64)
    s, p, n = O.run_pairs(test, X, coh["missing"], coh["vtype"], coh["nlev"], pa, pb, ctx=mask, validate=False, **kw)
    r = Ref((s, p, n))
    r.dof = pairs_dof(test, coh, pa, pb, n, mask=mask, welch=kw.get("welch", 1))
    return r


def oracle_run(test, coh, va, vb=None, mask=None, **kw):
    """The oracle on a cohort dict, with the pairs' degrees of freedom attached."""
    s, p, n = O.run(test, np.asarray(coh["X"], dtype=np.float64), coh["missing"], coh["vtype"], coh["nlev"], va, vb,
                    ctx=mask, **kw)
    r = Ref((s, p, n))
    r.dof = pair_dof(test, coh, va, vb, n, mask=mask, welch=kw.get("welch", 1))
    return r


def p_of(test, s, dof, idx=None):
    """The oracle's p-function of `test` at statistics s (the dof entries taken at
    the same positions `idx` when given)."""
    pick = (lambda a: np.asarray(a)[idx]) if idx is not None else np.asarray
    if test in ("pearson", "spearman"):
        return O.corr_p(s, pick(dof["n"]))
    if test == "anova":
        return O.f_sf(s, pick(dof["d1"]), pick(dof["d2"]))
    if test == "ttest":
        return O.t_p2(s, pick(dof["df"]))
    if test in ("chi2", "kruskal"):
        return O.chi2_sf(s, pick(dof["df"]))
    raise NotImplementedError(test)


def p_function_agrees(test, g, dof, rel=1e-12):
    """c14 part (i): the device p-value equals the oracle's p-function applied to
    the device's own statistic and degrees of freedom, to `rel` relative."""
    s, p = np.asarray(g["stat"]), np.asarray(g["p"])
    ok = np.isfinite(s) & np.isfinite(p) & (p > 1e-300)
    for v in dof.values():
        ok &= np.isfinite(np.asarray(v, dtype=np.float64))
    idx = np.nonzero(ok)
    ref = p_of(test, s[idx], dof, idx)
    err = np.abs(p[idx] - ref) / ref
    assert err.max(initial=0) <= rel, f"{test}: device p vs oracle p-function, max rel {err.max()}"
    return int(ok.sum())


def compare(test, gpu, ref, stat_tol=None, p_rel=P_REL, check_p=True):
    """Element-by-element: n bit-exact, NaN patterns equal, stat within its bar,
    p within p_rel relative plus the statistic's propagated difference."""
    gs, gp, gn = [np.asarray(gpu[k]) for k in ("stat", "p", "n")]
    rs, rp, rn = ref
    assert gn.shape == rn.shape
    bad_n = np.argwhere(gn != rn)
    assert bad_n.size == 0, f"n differs at {bad_n[:5].tolist()}: gpu {gn[tuple(bad_n[0])]} oracle {rn[tuple(bad_n[0])]}"
    nan_g, nan_r = np.isnan(gs), np.isnan(rs)
    bad = np.argwhere(nan_g != nan_r)
    assert bad.size == 0, f"stat NaN pattern differs at {bad[:5].tolist()}: gpu {gs[tuple(bad[0])]} oracle {rs[tuple(bad[0])]}"
    kind, tol = stat_tol or STAT_TOL[test]
    if kind == "effect":
        # judge F and t on their effect-size (correlation) scale, the analogue of
        # |dr| for Pearson: t -> t / sqrt(t^2 + n - 2), F -> sqrt(F / (F + n))
        nn = rn.astype(np.float64)
        if test == "ttest":
            tr = lambda v: v / np.sqrt(v * v + np.maximum(nn - 2, 1))
        else:
            tr = lambda v: np.sqrt(np.maximum(v, 0) / (np.maximum(v, 0) + nn))
        with np.errstate(invalid="ignore", divide="ignore"):
            gs_e, rs_e = tr(gs), tr(rs)
        fin_e = np.isfinite(rs_e) & np.isfinite(rs)
        de = np.abs(gs_e[fin_e] - rs_e[fin_e])
        assert de.max(initial=0) <= tol, f"max effect-scale difference {de.max()} > {tol}"
        kind = "none"
    ok = ~nan_r
    inf_r = np.isinf(rs)
    assert np.array_equal(gs[inf_r], rs[inf_r]), "infinite statistics differ"
    fin = ok & ~inf_r
    d = np.abs(gs[fin] - rs[fin])
    if kind == "abs":
        assert d.max(initial=0) <= tol, f"max |dstat| {d.max()} > {tol}"
    elif kind == "rel":
        r = d / np.maximum(np.abs(rs[fin]), 1.0)
        worst = r.max(initial=0)
        assert worst <= tol, f"max rel dstat {worst} > {tol} at {np.argwhere(fin)[np.argmax(r)].tolist()}"
    elif kind == "exact":
        assert np.array_equal(gs[fin], rs[fin]), "statistic not bit-exact"
    if not check_p:
        return
    pn_g, pn_r = np.isnan(gp), np.isnan(rp)
    badp = np.argwhere(pn_g != pn_r)
    assert badp.size == 0, f"p NaN pattern differs at {badp[:5].tolist()}: gpu {gp[tuple(badp[0])]} oracle {rp[tuple(badp[0])]}"
    ok = ~pn_r
    # conditioning: p moves with the statistic; allow the propagated difference
    dstat = np.zeros_like(rs)
    dstat[fin] = np.abs(gs[fin] - rs[fin])
    tiny = (rp < 1e-300) & ok
    assert (gp[tiny] < 1e-290).all(), "oracle p underflows but GPU p does not"
    chk = ok & ~tiny
    dp = np.abs(gp[chk] - rp[chk])
    allow = p_rel * rp[chk] + 1e-300
    moved = dstat[chk] > 0
    if moved.any():
        # the p-value's change over the statistic's difference: the oracle's own
        # p-function evaluated around the oracle statistic (a finite difference)
        dof = getattr(ref, "dof", None)
        if test in ("pearson", "spearman") and dof is None:
            dof = {"n": rn}
        assert dof is not None, f"{test}: the statistic moved; degrees of freedom are needed for the p-value bound"
        idx = tuple(a[moved] for a in np.nonzero(chk))
        slope = np.zeros(dp.shape)
        slope[moved] = _slope_bound(test, rs[idx], dstat[idx], dof, idx)
        allow = allow + slope
    worst = np.argmax(dp - allow) if dp.size else 0
    assert (dp <= allow).all(), f"p differs beyond bound: gpu {gp[chk][worst]} oracle {rp[chk][worst]}"


def _slope_bound(test, s, ds, dof, idx):
    """Upper bound of |p(s') - p(s)| for |s' - s| <= ds: the range of the
    oracle's p-function of the test over [s - h, s + h], h = 4 ds (at least
    1e-15), clipped to the statistic's domain (|r| <= 1; F, chi-squared, H >= 0;
    t through 0, where the two-sided p is 1)."""
    h = np.maximum(4 * ds, 1e-15)
    lo, hi = s - h, s + h
    if test in ("pearson", "spearman"):
        lo, hi = np.maximum(lo, -1.0), np.minimum(hi, 1.0)
        n = np.asarray(dof["n"])[idx]
        ok = n > 2
        out = np.zeros_like(s)
        if ok.any():
            pl = O.corr_p(lo[ok], n[ok])
            ph = O.corr_p(hi[ok], n[ok])
            p0 = O.corr_p(np.where((lo[ok] < 0) & (hi[ok] > 0), 0.0, s[ok]), n[ok])
            out[ok] = np.maximum.reduce([pl, ph, p0]) - np.minimum.reduce([pl, ph, p0])
        return out + 1e-300
    if test in ("anova", "chi2", "kruskal"):
        lo = np.maximum(lo, 0.0)
    pl = p_of(test, lo, dof, idx)
    ph = p_of(test, hi, dof, idx)
    if test == "ttest":
        p0 = p_of(test, np.where((lo < 0) & (hi > 0), 0.0, s), dof, idx)
        return np.maximum.reduce([pl, ph, p0]) - np.minimum.reduce([pl, ph, p0]) + 1e-300
    return np.abs(pl - ph) + 1e-300
