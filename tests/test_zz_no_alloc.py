"""The allocation-free entry point napg_pearson_fp64_noalloc.

It exists for callers that cannot allocate device memory (a framework's own
allocator owns the device, a hard memory cap, or a path that must not block in
the allocator): its work space is a fixed array inside the library. This test
calls it through the C ABI on two different inputs in a row and checks each
result against the regular entry point napg_run (plain FP64 Pearson) with the
tolerances of the other GPU tests. The test buffers themselves come from torch:
only the entry point under test must not allocate.

The file name makes pytest collect it last.
"""
import ctypes as C
import math

import numpy as np
import pytest

from paper_2505_00448_gb300 import synth

pytestmark = pytest.mark.gpu


def _call(napg, torch, X):
    nv, S = X.shape
    dev = torch.device("cuda", 0)
    Xd = torch.from_numpy(np.ascontiguousarray(X, dtype=np.float64)).to(dev)
    r = torch.full((nv, nv), -7.0, dtype=torch.float64, device=dev)
    p = torch.full((nv, nv), -7.0, dtype=torch.float64, device=dev)
    n = torch.full((nv, nv), -7, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    rc = napg.lib.napg_pearson_fp64_noalloc(C.c_void_p(Xd.data_ptr()), nv, S, math.nan, C.c_void_p(r.data_ptr()),
                                            C.c_void_p(p.data_ptr()), C.c_void_p(n.data_ptr()),
                                            C.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return rc, {"stat": r.cpu().numpy(), "p": p.cpu().numpy(), "n": n.cpu().numpy()}


def _reference(napg, X):
    c = napg.Context(0)
    nv = X.shape[0]
    c.load_cohort(X, np.zeros(nv, np.uint8), np.zeros(nv, np.int32))
    g = c.run("pearson", np.arange(nv), out="numpy", precision="fp64")
    c.close()
    return g


def _agree(g, ref):
    assert np.array_equal(g["n"], ref["n"])
    assert np.array_equal(np.isnan(g["stat"]), np.isnan(ref["stat"]))
    assert np.array_equal(np.isnan(g["p"]), np.isnan(ref["p"]))
    ok = ~np.isnan(ref["stat"])
    assert np.abs(g["stat"][ok] - ref["stat"][ok]).max(initial=0) <= 1e-12
    okp = ~np.isnan(ref["p"]) & (ref["p"] > 1e-300)
    rel = np.abs(g["p"][okp] - ref["p"][okp]) / ref["p"][okp]
    assert rel.max(initial=0) <= 1e-12


def test_noalloc_matches_regular_entry_point_twice():
    torch = pytest.importorskip("torch")
    from paper_2505_00448_gb300 import napg
    first = synth.small_cohort(301, n_cont=150, n_cat=0, S=5000 + 11, miss=0.25)["X"]
    second = synth.small_cohort(302, n_cont=61, n_cat=0, S=1200 + 3, miss=0.4, ties=True)["X"]
    second[7] = 2.5                          # a constant column (degenerate pairs)
    for X in (first, second):
        rc, g = _call(napg, torch, X)
        assert rc == 0, napg.STATUS.get(rc, rc)
        _agree(g, _reference(napg, X))


def test_noalloc_rejects_sizes_beyond_its_maximum():
    torch = pytest.importorskip("torch")
    from paper_2505_00448_gb300 import napg
    rc, _ = _call(napg, torch, np.zeros((257, 10)))
    assert rc == napg.E_UNSUPPORTED
    rc, _ = _call(napg, torch, np.zeros((4, 8193)))
    assert rc == napg.E_UNSUPPORTED
