"""Host logic of the leaf-size autotuner (paper_2002_01334_gb300/autotune.py): the candidate with
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
