"""The bench's per-stage roofline entries (host only): every traced stage of the
default and rank workloads gets its bound, algorithmic rate against the right
peak, fraction, and the committed DRAM traffic where one exists; the dominant
stage becomes the line's `roofline`. Stage times are made up: only the
arithmetic and the structure are checked."""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402
from paper_2505_00448_gb300 import synth  # noqa: E402

PEAKS = {"bf16_tflops_sustained": 1752.0, "hbm_gbs": 6678.5}
STAGES = ("prep", "planes_f16", "pearson_moments_tc", "finalize_pearson", "pvalues", "rescue", "planes_onehot",
          "groupsum_tc", "finalize_groups", "contingency_tc", "finalize_chi2", "pearson_moments_fp64",
          "groupsum_fp64", "spearman_rank", "rank_groups", "presort", "finalize_spearman", "finalize_rankgroups")


def _cohort_and_tests():
    coh = synth.small_cohort(3, n_cont=20, n_cat=8, S=1000, miss=0.2, lev_lo=2, lev_hi=5, binary_cats=3)
    cont, cat = coh["cont"], coh["cat"]
    bins = cat[coh["nlev"][cat] == 2]
    tests = [("pearson", cont, None), ("anova", cat, cont), ("ttest", bins, cont), ("chi2", cat, None),
             ("spearman", cont, None), ("mwu", bins, cont), ("kruskal", cat[coh["nlev"][cat] >= 3], cont)]
    return coh, tests


def test_every_modelled_stage_and_the_dominant_one():
    coh, tests = _cohort_and_tests()
    steps = 4
    stage_ms = {name: {"ms": 0.5 * steps * (k + 1), "launches": 2 * steps} for k, name in enumerate(STAGES)}
    ents = {e["kernel"]: e for e in bench.stage_rooflines(stage_ms, steps, coh, tests, PEAKS)}
    S = coh["X"].shape[1]
    for name in ("pearson_moments_tc", "groupsum_tc", "contingency_tc"):
        e = ents[name]
        # the contingency tables run as E4M3 MMAs: twice the bf16 figure
        assert e["bound"] == "tensor" and e["unit"] == "TFLOP/s"
        assert e["peak"] == (2 * 1752.0 if name == "contingency_tc" else 1752.0)
        assert e["issued_tflops"] >= e["achieved"] > 0          # the split issues more than the algorithm needs
        assert abs(e["frac"] - e["achieved"] / e["peak"]) < 1e-12
    for name in ("spearman_rank", "rank_groups"):
        e = ents[name]
        # the byte model's effective rate, labelled as such: the rank kernels are
        # bound by instruction issue (their working set stays in L2)
        assert e["bound"] == "alu" and e["unit"] == "GB/s of the byte model" and e["peak"] == 6678.5
        assert "instruction issue" in e["peak_source"]
    # the byte model of the Spearman stage: 16.25 S bytes per unordered pair (diagonal included)
    n = len(coh["cont"])
    secs = stage_ms["spearman_rank"]["ms"] / steps / 1000.0
    assert abs(ents["spearman_rank"]["achieved"] - 16.25 * S * n * (n + 1) / 2 / secs / 1e9) < 1e-9
    for name in ("pearson_moments_fp64", "groupsum_fp64"):
        assert ents[name]["bound"] == "alu" and ents[name]["unit"] == "GFLOP/s"
    assert ents["pvalues"]["unit"] == "M p-values/s" and ents["pvalues"]["frac"] is None
    for e in ents.values():
        assert e["launches_per_step"] == 2
    # traffic: the committed per-stage DRAM bytes where the profiles have them
    traffic = json.load(open(os.path.join(ROOT, "profiles", "traffic.json")))
    for name, e in ents.items():
        assert e["traffic"] == traffic.get(name)
    dom = bench.kernel_roofline(stage_ms, steps, coh, tests, PEAKS)
    assert dom["kernel"] == max(stage_ms, key=lambda k: stage_ms[k]["ms"])
    assert isinstance(dom["stages"], list) and len(dom["stages"]) == len(ents)
    json.dumps(dom)                                              # the bench line must serialise


def test_fallback_peaks_are_labelled():
    coh, tests = _cohort_and_tests()
    stage_ms = {"pearson_moments_tc": {"ms": 1.0, "launches": 1}, "spearman_rank": {"ms": 1.0, "launches": 1}}
    ents = {e["kernel"]: e for e in bench.stage_rooflines(stage_ms, 1, coh, tests, {})}
    assert ents["pearson_moments_tc"]["peak"] == 1700.0 and "fallback" in ents["pearson_moments_tc"]["peak_source"]
    assert ents["spearman_rank"]["peak"] == 6800.0 and "fallback" in ents["spearman_rank"]["peak_source"]
    assert bench.kernel_roofline({}, 1, coh, tests, {}) is None
    assert np.isfinite(ents["spearman_rank"]["frac"])
