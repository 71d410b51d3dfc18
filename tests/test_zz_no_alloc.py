"""The allocation-free entry point napg_pearson_fp64_noalloc.

It exists for callers that cannot allocate device memory (a framework's own
allocator owns the device, a hard memory cap, or a path that must not block in
the allocator): its work space is a fixed array inside the library. These tests
call it through the C ABI and check its results against the FP64 oracle and
against the regular entry point napg_run (plain FP64 Pearson), with the
tolerances of the other GPU tests: n bit-exact, |dr| <= 1e-12, p within 1e-12
relative. Covered: two different inputs in a row, the largest size it accepts
(256 variables x 8,192 samples) with a finite sentinel and no p output, the
smallest (one variable, one sample), a non-missing infinity, and sizes beyond
its maximum. The test buffers themselves come from torch: only the entry point
under test must not allocate.

The file name makes pytest collect it last.
"""
import ctypes as C
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2505_00448_gb300 import synth

pytestmark = pytest.mark.gpu


def _call(napg, torch, X, missing=math.nan, want_p=True):
    nv, S = X.shape
    dev = torch.device("cuda", 0)
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float64)).to(dev)
    r = torch.full((nv, nv), -7.0, dtype=torch.float64, device=dev)
    p = torch.full((nv, nv), -7.0, dtype=torch.float64, device=dev)
    n = torch.full((nv, nv), -7, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rc = napg.lib.napg_pearson_fp64_noalloc(C.c_void_p(Xd.data_ptr()), nv, S, float(missing),
                                            C.c_void_p(r.data_ptr()),
                                            C.c_void_p(p.data_ptr() if want_p else None),
                                            C.c_void_p(n.data_ptr()), C.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    out = {"stat": r.cpu().numpy(), "p": p.cpu().numpy() if want_p else None, "n": n.cpu().numpy()}
    return rc, out


def _regular(napg, X, missing=math.nan):
    c = napg.Context(0)
    nv = X.shape[0]
    c.load_cohort(X, np.zeros(nv, np.uint8), np.zeros(nv, np.int32), missing)
    g = c.run("pearson", np.arange(nv), out="numpy", precision="fp64")
    c.close()
    return g


def _oracle(X, missing=math.nan):
    nv = X.shape[0]
    s, p, n = O.run("pearson", X, missing, np.zeros(nv, np.uint8), np.zeros(nv, np.int32), np.arange(nv))
    return {"stat": s, "p": p, "n": n}


def _agree(g, ref, check_p=True):
    assert np.array_equal(g["n"], ref["n"])
    assert np.array_equal(np.isnan(g["stat"]), np.isnan(ref["stat"]))
    ok = ~np.isnan(ref["stat"])
    assert np.abs(g["stat"][ok] - ref["stat"][ok]).max(initial=0) <= 1e-12
    if not check_p:
        return
    assert np.array_equal(np.isnan(g["p"]), np.isnan(ref["p"]))
    okp = ~np.isnan(ref["p"]) & (ref["p"] > 1e-300)
    # p moves with r: allow the oracle p-function's change over the r difference
    dr = np.abs(g["stat"] - ref["stat"])[okp]
    slope = np.array([abs(O.corr_p(min(1.0, r + 4 * d + 1e-15), n) - O.corr_p(max(-1.0, r - 4 * d - 1e-15), n))
                      for r, d, n in zip(ref["stat"][okp], dr, ref["n"][okp].astype(float))])
    dp = np.abs(g["p"][okp] - ref["p"][okp])
    assert (dp <= 1e-12 * ref["p"][okp] + slope + 1e-300).all()


def test_noalloc_matches_oracle_and_regular_entry_point_twice():
    torch = pytest.importorskip("torch")
    from paper_2505_00448_gb300 import napg
    first = synth.small_cohort(301, n_cont=150, n_cat=0, S=5000 + 11, miss=0.25)["X"]
    second = synth.small_cohort(302, n_cont=61, n_cat=0, S=1200 + 3, miss=0.4, ties=True)["X"]
    second[7] = 2.5                          # a constant column (degenerate pairs)
    for X in (first, second):
        rc, g = _call(napg, torch, X)
        assert rc == 0, napg.STATUS.get(rc, rc)
        _agree(g, _oracle(X))
        _agree(g, _regular(napg, X))


def test_noalloc_largest_size_finite_sentinel_no_p():
    """256 x 8,192 (the largest accepted), missing values marked by -999, no p
    output (the p-value job queue is skipped): n exact and r within 1e-12 of the
    oracle; r and n equal those of a call that also asks for p."""
    torch = pytest.importorskip("torch")
    from paper_2505_00448_gb300 import napg
    X = synth.small_cohort(303, n_cont=256, n_cat=0, S=8192, miss=0.3, offset=1e3)["X"]
    X = np.where(np.isnan(X), -999.0, X)
    rc, g = _call(napg, torch, X, missing=-999.0, want_p=False)
    assert rc == 0, napg.STATUS.get(rc, rc)
    _agree(g, _oracle(X, -999.0), check_p=False)
    rc, g2 = _call(napg, torch, X, missing=-999.0)
    assert rc == 0
    assert np.array_equal(g["n"], g2["n"]) and np.array_equal(g["stat"], g2["stat"], equal_nan=True)
    _agree(g2, _oracle(X, -999.0))


def test_noalloc_smallest_size():
    torch = pytest.importorskip("torch")
    from paper_2505_00448_gb300 import napg
    rc, g = _call(napg, torch, np.array([[3.0]]))
    assert rc == 0
    assert g["n"][0, 0] == 1 and np.isnan(g["stat"][0, 0]) and np.isnan(g["p"][0, 0])
    _agree(g, _oracle(np.array([[3.0]])))


def test_noalloc_rejects_nonfinite_and_sizes_beyond_its_maximum():
    torch = pytest.importorskip("torch")
    from paper_2505_00448_gb300 import napg
    X = synth.small_cohort(304, n_cont=5, n_cat=0, S=100, miss=0.2)["X"]
    X[2, 17] = math.inf
    rc, _ = _call(napg, torch, X)
    assert rc == napg.E_NONFINITE
    rc, _ = _call(napg, torch, np.zeros((257, 10)))
    assert rc == napg.E_UNSUPPORTED
    rc, _ = _call(napg, torch, np.zeros((4, 8193)))
    assert rc == napg.E_UNSUPPORTED
    # a later valid call still works (the error word is cleared per call)
    X[2, 17] = 1.0
    rc, g = _call(napg, torch, X)
    assert rc == 0
    _agree(g, _oracle(X))
