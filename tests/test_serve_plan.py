"""The serving loop's admission policy (host logic, no GPU): first-fit in
arrival order under the memory budget, a slot keeps the memory it holds, and a
request that has waited 200 ms is not overtaken."""
import numpy as np
import pytest


@pytest.fixture(scope="module")
def napg():
    from paper_2505_00448_gb300 import build
    build.build()
    from paper_2505_00448_gb300 import napg as N
    return N


def test_in_order_when_everything_fits(napg):
    a = napg.serve_plan([10, 20, 30, 40], [0, 0, 0, 0], [0, 0, 0], [0, 0, 0], budget=1000)
    assert a.tolist() == [0, 1, 2]


def test_smaller_request_overtakes_a_young_head(napg):
    a = napg.serve_plan([60, 50, 10], [5.0, 1.0, 0.5], [0, 0], [0, 0], budget=100)
    assert a.tolist() == [0, 2]


def test_old_head_is_not_overtaken(napg):
    a = napg.serve_plan([60, 50, 10], [400.0, 300.0, 0.5], [0, 0], [0, 0], budget=100)
    assert a.tolist() == [0, -1]


def test_busy_slot_memory_counts(napg):
    a = napg.serve_plan([30, 10], [1.0, 1.0], [80, 0], [1, 0], budget=100)
    assert a.tolist() == [-1, 1]


def test_idle_slot_keeps_what_it_holds(napg):
    # slot 1 holds 50 from an earlier request: a 20-byte request needs max(50, 20)
    assert napg.serve_plan([20], [0.0], [40, 50], [1, 0], budget=90).tolist() == [-1, 0]
    assert napg.serve_plan([20], [0.0], [41, 50], [1, 0], budget=90).tolist() == [-1, -1]


def test_nothing_fits_and_empty_queue(napg):
    assert napg.serve_plan([500], [0.0], [0, 0], [0, 0], budget=100).tolist() == [-1, -1]
    assert napg.serve_plan([], [], [0, 0], [0, 0], budget=100).tolist() == [-1, -1]


def test_every_admitted_plan_respects_the_budget(napg):
    rng = np.random.default_rng(5)
    for _ in range(200):
        nq, ns = int(rng.integers(0, 12)), int(rng.integers(1, 6))
        est = rng.integers(1, 60, nq)
        age = rng.uniform(0, 400, nq)
        mem = rng.integers(0, 40, ns)
        busy = rng.integers(0, 2, ns)
        budget = int(rng.integers(40, 200))
        a = napg.serve_plan(est, age, mem, busy, budget)
        held = mem.astype(np.int64).copy()
        used = set()
        for k in range(ns):
            if a[k] >= 0:
                assert not busy[k] and a[k] not in used
                used.add(int(a[k]))
                held[k] = max(held[k], est[a[k]])
        if used:
            assert held.sum() <= budget
