"""Host logic of the autotuner (paper_2002_01334_gb300/autotune.py): the candidate with
the smallest median time wins, the first on a tie, and every candidate is measured `repeats`
times.  The CUDA timing harness itself needs a GPU."""
import itertools

import pytest

from paper_2002_01334_gb300 import autotune


def test_choose_takes_the_smallest_median():
    noise = itertools.cycle([0.0, 30.0, -0.5])  # one outlier per three repeats
    cost = {32: 20.0, 64: 14.0, 128: 11.0, 256: 12.5, 512: 18.0}
    calls = []

    def measure(s):
        calls.append(s)
        return cost[s] + next(noise)

    best, table = autotune.choose(autotune.CANDIDATES, measure, repeats=3)
    assert best == 128 and set(table) == set(autotune.CANDIDATES)
    assert all(calls.count(c) == 3 for c in autotune.CANDIDATES)
    assert table[128] == 11.0  # the median ignores the outlier


def test_choose_breaks_ties_by_order_and_rejects_empty():
    best, _ = autotune.choose((64, 128), lambda s: 5.0, repeats=1)
    assert best == 64
    with pytest.raises(ValueError):
        autotune.choose((), lambda s: 1.0)


def test_search_is_coordinate_descent_over_the_parameters_in_order():
    # a separable cost: leaf 64 and react_levels 3 are best; every setting timed once per repeat
    cost = {32: 9.0, 64: 4.0, 128: 5.0, 256: 7.0, 512: 8.0}
    extra = {2: 3.0, 3: 1.0, 4: 2.0, 6: 2.5}
    calls = []

    def measure(s):
        calls.append(tuple(sorted(s.items())))
        return cost[s["max_per_leaf"]] + extra[s["react_levels"]]

    best, rows = autotune.search(autotune.SPACE, measure, start=autotune.DEFAULTS, repeats=2)
    assert best == {"max_per_leaf": 64, "react_levels": 3}
    # leaf sizes at the default react_levels, then react_levels at leaf 64 (64, 4 already timed)
    assert [r[0] for r in rows] == [{"max_per_leaf": c, "react_levels": 4} for c in (32, 64, 128, 256, 512)] + \
        [{"max_per_leaf": 64, "react_levels": r} for r in (2, 3, 6)]
    assert len(calls) == 2 * len(rows)
    assert rows[1][1] == 6.0


def test_search_ties_keep_the_first_candidate():
    best, _ = autotune.search((("a", (3, 1, 2)), ("b", (5, 4))), lambda s: 1.0, repeats=1)
    assert best == {"a": 3, "b": 5}


def test_search_skips_settings_that_cannot_run():
    # leaf 32 runs out of memory (None): it is recorded and never chosen
    cost = {32: None, 64: 4.0, 128: 3.0, 256: 5.0, 512: 6.0}
    best, rows = autotune.search((("max_per_leaf", (32, 64, 128, 256, 512)),),
                                 lambda s: cost[s["max_per_leaf"]], repeats=2)
    assert best == {"max_per_leaf": 128}
    assert rows[0] == [{"max_per_leaf": 32}, None]
