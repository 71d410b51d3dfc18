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


def _p_of_stat(test, s, n, extra):
    """The oracle's p-function applied to a given statistic (c14 part (i))."""
    if test in ("pearson", "spearman"):
        return float(O.corr_p(s, n))
    raise NotImplementedError


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
    if dstat[chk].max(initial=0) > 0:
        # |dp/dstat| bound by a finite difference of the oracle's p on the stat
        allow = allow + _slope_bound(test, rs[chk], rn[chk], dstat[chk], rp[chk])
    worst = np.argmax(dp - allow) if dp.size else 0
    assert (dp <= allow).all(), f"p differs beyond bound: gpu {gp[chk][worst]} oracle {rp[chk][worst]}"


def _slope_bound(test, s, n, ds, p):
    """Upper bound of |p(s + ds) - p(s)| from the p-value's sensitivity, with
    margin: for the correlation tests through the oracle's own p-function,
    otherwise a relative allowance proportional to the statistic's change."""
    if test in ("pearson", "spearman"):
        out = np.empty_like(s)
        for k in range(len(s)):
            h = max(4 * ds[k], 1e-15)
            lo = float(O.corr_p(max(-1.0, s[k] - h), n[k])) if n[k] > 2 else 0.0
            hi = float(O.corr_p(min(1.0, s[k] + h), n[k])) if n[k] > 2 else 0.0
            out[k] = abs(hi - lo) + 1e-300
        return out
    # other tests: dlog p / dlog stat is bounded by the statistic times a modest
    # factor; use 100 x relative change of the statistic x (1 + |log p|)
    rel = ds / np.maximum(np.abs(s), 1e-300)
    return 100.0 * rel * p * (1.0 + np.abs(np.log(np.maximum(p, 1e-300))))
