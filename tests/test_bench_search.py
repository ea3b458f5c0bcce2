"""The serving search of bench.py (the largest load scale alpha whose run meets
the p99 bound) on synthetic feasibility functions: a bound above the start,
a feasible band (a fixed batch size also misses at low rates), a bound below
the start, and no feasible rate at all."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _runner(feasible):
    def run_at(alpha):
        return feasible(alpha), {"p99_ms": 50.0 if feasible(alpha) else 150.0, "alpha": alpha}
    return run_at


def test_monotone_bound_above_start():
    limit = 37.3
    a, res, runs = bench.alpha_search(_runner(lambda x: x <= limit), start=4.0, iters=6)
    # doubling 4, 8, 16, 32 pass and 64 misses; six halvings of [32, 64]
    assert [r["alpha"] for r in runs[:5]] == [4.0, 8.0, 16.0, 32.0, 64.0]
    assert a <= limit < a + 32.0 / 2 ** 6
    assert res["alpha"] == a
    assert all(r["met"] == (r["alpha"] <= limit) for r in runs)


def test_band_reaches_its_upper_edge():
    a, _, runs = bench.alpha_search(_runner(lambda x: 10.0 <= x <= 20.0), start=4.0, iters=5)
    # 4 and 8 miss below the band; 16 passes, 32 misses; bisection of [16, 32]
    assert [r["met"] for r in runs[:4]] == [False, False, True, False]
    assert 20.0 - 16.0 / 2 ** 5 < a <= 20.0


def test_bound_below_start_is_found_by_halving():
    a, _, runs = bench.alpha_search(_runner(lambda x: x <= 3.0), start=16.0, iters=4)
    alphas = [r["alpha"] for r in runs]
    # four misses from the start upwards, then halving 8, 4, 2, then [2, 4]
    assert alphas[:4] == [16.0, 32.0, 64.0, 128.0]
    assert alphas[4:7] == [8.0, 4.0, 2.0]
    assert 3.0 - 2.0 / 2 ** 4 < a <= 3.0


def test_nothing_feasible_gives_none():
    a, res, runs = bench.alpha_search(_runner(lambda x: False), start=4.0, iters=3)
    assert a is None and res is None
    assert not any(r["met"] for r in runs)
    assert min(r["alpha"] for r in runs) >= 4.0 / 64.0
