"""ctypes binding of the plain FP64 oracle (napg_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the smoke check and by
the benchmark's CPU-baseline leg. The library under test never imports it, and
this module imports nothing from the library.

The oracle is compiled with gcc (-O2 -ffp-contract=off, OpenMP over pairs only)
into oracle/_build/ the first time it is needed.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "napg_oracle.c")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libnapg_oracle.so")

PEARSON, SPEARMAN, CHI2, ANOVA, TTEST, MWU, KRUSKAL = range(7)
TEST_NAMES = {"pearson": PEARSON, "spearman": SPEARMAN, "chi2": CHI2, "anova": ANOVA,
              "ttest": TTEST, "mwu": MWU, "kruskal": KRUSKAL}
OK, E_ARG, E_OOM, E_LABEL, E_NONFINITE = 0, 1, 2, 4, 5

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle if its shared object is missing or older than the source."""
    os.makedirs(BUILD, exist_ok=True)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < os.path.getmtime(SRC):
        tmp = LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-shared",
               "-fPIC", "-std=c11", "-o", tmp, SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, LIB)
    return LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # NAPG_ORACLE_LIB points the tests at a deliberately broken copy
            # (tests/test_oracle_mutants.py); normally the built oracle is used.
            path = os.environ.get("NAPG_ORACLE_LIB")
            if not path:
                path = build()
            L = C.CDLL(path)
            d, i64, i32, p = C.c_double, C.c_int64, C.c_int32, C.c_void_p
            for name in ("orc_ibeta",):
                getattr(L, name).restype = d
                getattr(L, name).argtypes = [d, d, d, d]
            for name in ("orc_gamma_q", "orc_t_p2", "orc_chi2_sf", "orc_corr_p"):
                getattr(L, name).restype = d
                getattr(L, name).argtypes = [d, d]
            L.orc_norm_sf.restype = d
            L.orc_norm_sf.argtypes = [d]
            L.orc_f_sf.restype = d
            L.orc_f_sf.argtypes = [d, d, d]
            L.orc_mwu_exact_sf.restype = d
            L.orc_mwu_exact_sf.argtypes = [d, C.c_long, C.c_long]
            L.orc_validate.restype = C.c_int
            L.orc_validate.argtypes = [p, i64, i64, d, p, p]
            L.orc_run.restype = C.c_int
            L.orc_run.argtypes = [C.c_int, p, i64, i64, d, p, p, p, p, i32, p, i32,
                                  C.c_int, C.c_int, C.c_int, C.c_int, p, p, p, C.c_int]
            L.orc_run_pairs.restype = C.c_int
            L.orc_run_pairs.argtypes = [C.c_int, p, i64, i64, d, p, p, p, p, p, i64,
                                        C.c_int, C.c_int, C.c_int, C.c_int, p, p, p, C.c_int,
                                        C.c_int]
            L.orc_pair_ints.restype = i64
            L.orc_pair_ints.argtypes = [C.c_int, p, i64, i64, d, p, p, p, i32, i32, p, i64]
            L.orc_max_threads.restype = C.c_int
            L.orc_max_threads.argtypes = []
            L.orc_effects.restype = C.c_int
            L.orc_effects.argtypes = [C.c_int, p, i64, i64, d, p, p, p, p, i32, p, i32, C.c_int, C.c_int,
                                      p, p, C.c_int]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _cohort_arrays(X, vtype, nlev, ctx):
    X = np.ascontiguousarray(X, dtype=np.float64)
    F, S = X.shape
    vtype = np.ascontiguousarray(vtype, dtype=np.uint8)
    nlev = np.ascontiguousarray(nlev, dtype=np.int32)
    assert vtype.shape == (F,) and nlev.shape == (F,)
    if ctx is not None:
        ctx = np.ascontiguousarray(ctx, dtype=np.uint8)
        assert ctx.shape == (S,)
    return X, F, S, vtype, nlev, ctx


class OracleError(RuntimeError):
    def __init__(self, code):
        super().__init__(f"oracle returned status {code}")
        self.code = code


def run(test, X, missing, vtype, nlev, vars_a, vars_b=None, ctx=None, welch=1, yates=0,
        mwu_mode=0, mwu_cc=1, nthreads=0):
    """All pairs vars_a x vars_b (vars_a x vars_a when vars_b is None).

    Returns (stat, p, n) as n_a x n_b arrays (float64, float64, int32).
    """
    if isinstance(test, str):
        test = TEST_NAMES[test]
    X, F, S, vtype, nlev, ctx = _cohort_arrays(X, vtype, nlev, ctx)
    va = np.ascontiguousarray(vars_a, dtype=np.int32)
    vb = None if vars_b is None else np.ascontiguousarray(vars_b, dtype=np.int32)
    nb = len(va) if vb is None else len(vb)
    stat = np.empty((len(va), nb), np.float64)
    pval = np.empty((len(va), nb), np.float64)
    nout = np.empty((len(va), nb), np.int32)
    rc = lib().orc_run(test, _ptr(X), F, S, float(missing), _ptr(vtype), _ptr(nlev), _ptr(ctx),
                       _ptr(va), len(va), _ptr(vb), 0 if vb is None else len(vb),
                       welch, yates, mwu_mode, mwu_cc, _ptr(stat), _ptr(pval), _ptr(nout),
                       nthreads)
    if rc:
        raise OracleError(rc)
    return stat, pval, nout


def run_pairs(test, X, missing, vtype, nlev, pairs_a, pairs_b, ctx=None, welch=1, yates=0,
              mwu_mode=0, mwu_cc=1, nthreads=0, validate=True):
    """The test on explicit pairs (pairs_a[q], pairs_b[q]). Returns (stat, p, n) 1-D arrays."""
    if isinstance(test, str):
        test = TEST_NAMES[test]
    X, F, S, vtype, nlev, ctx = _cohort_arrays(X, vtype, nlev, ctx)
    pa = np.ascontiguousarray(pairs_a, dtype=np.int32)
    pb = np.ascontiguousarray(pairs_b, dtype=np.int32)
    assert pa.shape == pb.shape
    m = len(pa)
    stat = np.empty(m, np.float64)
    pval = np.empty(m, np.float64)
    nout = np.empty(m, np.int32)
    rc = lib().orc_run_pairs(test, _ptr(X), F, S, float(missing), _ptr(vtype), _ptr(nlev),
                             _ptr(ctx), _ptr(pa), _ptr(pb), m, welch, yates, mwu_mode, mwu_cc,
                             _ptr(stat), _ptr(pval), _ptr(nout), nthreads, 1 if validate else 0)
    if rc:
        raise OracleError(rc)
    return stat, pval, nout


def effects(test, X, missing, vtype, nlev, vars_a, vars_b=None, ctx=None, welch=1, yates=0, nthreads=0):
    """Effect sizes of all pairs (Table 2), laid out as run()'s outputs.

    Returns (e1, e2): r^2, rho, phi, Cohen's d, Mann-Whitney r, partial eta^2 or
    Kruskal-Wallis eta^2 in e1; Cramer's V (chi-squared only, else NaN) in e2.
    """
    if isinstance(test, str):
        test = TEST_NAMES[test]
    X, F, S, vtype, nlev, ctx = _cohort_arrays(X, vtype, nlev, ctx)
    va = np.ascontiguousarray(vars_a, dtype=np.int32)
    vb = None if vars_b is None else np.ascontiguousarray(vars_b, dtype=np.int32)
    nb = len(va) if vb is None else len(vb)
    e1 = np.empty((len(va), nb), np.float64)
    e2 = np.empty((len(va), nb), np.float64)
    rc = lib().orc_effects(test, _ptr(X), F, S, float(missing), _ptr(vtype), _ptr(nlev), _ptr(ctx),
                           _ptr(va), len(va), _ptr(vb), 0 if vb is None else len(vb), welch, yates,
                           _ptr(e1), _ptr(e2), nthreads)
    if rc:
        raise OracleError(rc)
    return e1, e2


ADJUST_METHODS = ("bonferroni", "bh", "by")


def adjust(p, method, symmetric):
    """Multiple-testing correction of a p-value matrix (Sec. 3.4).

    The tests are the entries with a p-value (not NaN); in a symmetric matrix
    (one variable set against itself) each unordered pair i < j is one test and
    the diagonal is no test (NaN in the result). With m tests and p_(1) <= ... <=
    p_(m) in ascending order:
      Bonferroni:         min(1, m p)
      Benjamini-Hochberg: p_adj_(i) = min over k >= i of (m p_(k)) / k, capped at 1
      Benjamini-Yekutieli: the same with m replaced by m c(m), c(m) = sum_{k<=m} 1/k
    (c(m) summed in increasing k). Tied p-values get equal adjusted values.
    """
    P = np.array(p, dtype=np.float64)
    out = np.full(P.shape, np.nan)
    if symmetric:
        assert P.shape[0] == P.shape[1]
        iu = np.triu_indices(P.shape[0], 1)
        vals = P[iu]
    else:
        vals = P.ravel()
    valid = ~np.isnan(vals)
    idx = np.nonzero(valid)[0]
    v = vals[idx]
    m = len(v)
    adj = np.full(len(vals), np.nan)
    if m:
        if method == "bonferroni":
            a = np.minimum(1.0, v * float(m))
        else:
            scale = float(m)
            if method == "by":
                cm = 0.0
                for k in range(1, m + 1):
                    cm += 1.0 / k
                scale = float(m) * cm
            elif method != "bh":
                raise ValueError(method)
            order = np.argsort(v, kind="stable")
            srt = v[order]
            a_sorted = np.empty(m)
            run = np.inf
            for i in range(m - 1, -1, -1):           # from the largest p down
                run = min(run, (srt[i] * scale) / float(i + 1))
                a_sorted[i] = run
            a = np.empty(m)
            a[order] = np.minimum(1.0, a_sorted)
        adj[idx] = a
    if symmetric:
        out[iu] = adj
        out.T[iu] = adj
    else:
        out = adj.reshape(P.shape)
    return out


def pair_ints(test, X, missing, vtype, nlev, a, b, ctx=None):
    """Integer quantities of one pair (see orc_pair_ints in napg_oracle.c)."""
    if isinstance(test, str):
        test = TEST_NAMES[test]
    X, F, S, vtype, nlev, ctx = _cohort_arrays(X, vtype, nlev, ctx)
    cap = 4 + 2 * 256 + int(nlev.max(initial=1)) ** 2
    out = np.zeros(cap, np.int64)
    m = lib().orc_pair_ints(test, _ptr(X), F, S, float(missing), _ptr(vtype), _ptr(nlev),
                            _ptr(ctx), int(a), int(b), _ptr(out), cap)
    if m < 0:
        raise OracleError(E_ARG)
    return out[:m].copy()


def validate(X, missing, vtype, nlev):
    X, F, S, vtype, nlev, _ = _cohort_arrays(X, vtype, nlev, None)
    return lib().orc_validate(_ptr(X), F, S, float(missing), _ptr(vtype), _ptr(nlev))


def max_threads() -> int:
    return int(lib().orc_max_threads())


# scalar special functions (vectorised for the tests)
ibeta = np.vectorize(lambda a, b, x: lib().orc_ibeta(a, b, x, 1.0 - x), otypes=[float])
ibeta_xy = np.vectorize(lambda a, b, x, y: lib().orc_ibeta(a, b, x, y), otypes=[float])
gamma_q = np.vectorize(lambda a, x: lib().orc_gamma_q(a, x), otypes=[float])
norm_sf = np.vectorize(lambda z: lib().orc_norm_sf(z), otypes=[float])
t_p2 = np.vectorize(lambda t, df: lib().orc_t_p2(t, df), otypes=[float])
f_sf = np.vectorize(lambda F, d1, d2: lib().orc_f_sf(F, d1, d2), otypes=[float])
chi2_sf = np.vectorize(lambda x, df: lib().orc_chi2_sf(x, df), otypes=[float])
corr_p = np.vectorize(lambda r, n: lib().orc_corr_p(r, n), otypes=[float])
mwu_exact_sf = np.vectorize(lambda u, n0, n1: lib().orc_mwu_exact_sf(u, int(n0), int(n1)),
                            otypes=[float])
