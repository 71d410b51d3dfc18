"""The split of one call over parts (napg_run_part, Sec. 3.5.1: the pairs are
independent): on one GPU, every part of a 2- and a 3-way split is run; each
part writes exactly the entries its rows own (the rest keep their sentinel),
and the stitched parts are bit-identical to one unsplit call, for every test,
in both precision forms where the test has two, with host and device outputs.
The cohort has more rows than one 256-row block in every variable list."""
import numpy as np
import pytest

from paper_2505_00448_gb300 import dist as D
from paper_2505_00448_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx_coh():
    from paper_2505_00448_gb300 import napg
    coh = synth.small_cohort(88, n_cont=600, n_cat=300, S=3000 + 5, miss=0.25, lev_lo=2, lev_hi=6, binary_cats=80,
                             dtype=np.float32, ties=True)
    c = napg.Context(0)
    c.load_cohort(coh["X"], coh["vtype"], coh["nlev"], coh["missing"])
    yield c, coh
    c.close()


def _cases(coh):
    cont, cat = coh["cont"], coh["cat"]
    bins = cat[:80]
    return [("pearson", cont, None, {"precision": "mixed"}), ("pearson", cont, None, {"precision": "fp64"}),
            ("spearman", cont, None, {}), ("chi2", cat, None, {"precision": "mixed"}),
            ("chi2", cat, None, {"precision": "fp64"}), ("anova", cat, cont[:120], {"precision": "mixed"}),
            ("ttest", bins, cont[:120], {"precision": "mixed"}), ("mwu", bins, cont[:60], {}),
            ("kruskal", cat, cont[:60], {}), ("pearson", cont[:300], cont[300:], {"precision": "mixed"})]


@pytest.mark.parametrize("k", range(10))
def test_parts_stitch_to_the_unsplit_call(ctx_coh, k):
    c, coh = ctx_coh
    test, va, vb, kw = _cases(coh)[k]
    full = c.run(test, va, vb, out="numpy", **kw)
    na = len(va)
    nb = na if vb is None else len(vb)
    sym = vb is None
    for nparts in (2, 3):
        parts = [c.run_part(test, va, vb, part=r, nparts=nparts, out="numpy", **kw) for r in range(nparts)]
        own = D.owner(na, nb, nparts, sym)
        for r, p in enumerate(parts):
            assert (p["n"][own != r] == -1).all(), f"part {r} wrote outside its rows"
            assert (p["n"][own == r] >= 0).all(), f"part {r} left an own entry unwritten"
        for f in ("stat", "p", "n"):
            got = D.stitch([p[f] for p in parts], na, nb, sym)
            assert np.array_equal(got, full[f], equal_nan=True), (test, kw, nparts, f)


def test_parts_device_outputs_in_place(ctx_coh):
    """Parts written in turn into the same device buffers give the unsplit call."""
    c, coh = ctx_coh
    torch = c.torch
    va = coh["cont"]
    full = c.run("pearson", va, out="numpy", precision="mixed")
    dev = torch.device("cuda", 0)
    n = len(va)
    outs = {"stat": torch.full((n, n), -5.0, dtype=torch.float64, device=dev),
            "p": torch.full((n, n), -5.0, dtype=torch.float64, device=dev),
            "n": torch.full((n, n), -5, dtype=torch.int32, device=dev)}
    for r in range(3):
        c.run_part("pearson", va, part=r, nparts=3, outputs=outs, precision="mixed")
    for f in ("stat", "p", "n"):
        assert np.array_equal(outs[f].cpu().numpy(), full[f], equal_nan=True), f


def test_part_arguments(ctx_coh):
    from paper_2505_00448_gb300 import napg
    c, coh = ctx_coh
    for part, nparts in ((2, 2), (-1, 2), (0, 0)):
        with pytest.raises(napg.NapgError) as e:
            c.run_part("pearson", coh["cont"][:10], part=part, nparts=nparts)
        assert e.value.code == napg.E_ARG
    # one part: the unsplit call
    a = c.run_part("pearson", coh["cont"][:50], part=0, nparts=1)
    b = c.run("pearson", coh["cont"][:50], out="numpy")
    for f in ("stat", "p", "n"):
        assert np.array_equal(a[f], b[f], equal_nan=True)
