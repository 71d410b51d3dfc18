"""bench.py keeps every workload entry point and its command-line contract (host only)."""
import importlib
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_workloads_and_arguments():
    sys.path.insert(0, ROOT)
    bench = importlib.import_module("bench")
    for fn in ("main", "batch_main", "serve_main", "make_workload", "oracle_sample", "sampled_accuracy",
               "stage_rooflines", "kernel_roofline", "serve_requests"):
        assert callable(getattr(bench, fn)), fn
    src = open(os.path.join(ROOT, "bench.py")).read()
    for flag in ("--gpus", "--steps", "--warmup", "--impl", "--workload", "--precision"):
        assert flag in src
    assert bench.pair_count("pearson", list(range(5)), None) == 10
    assert bench.pair_count("anova", list(range(3)), list(range(7))) == 21
