"""CPU pins of the oracle's adaptive dual trees and lists (oracle/adaptive.py).

Coverage, by brute force: every (target, source) pair of points lies in exactly one listed box
pair (U, V at one level, W or X), the property that makes the FMM sum each interaction once.
The lists match their classical characterisations.  For a uniform tree they equal the uniform
lists of the C oracle, which the GPU's lists match bit for bit."""
import numpy as np
import pytest

import oracle
from oracle import adaptive as A
from paper_2002_01334_gb300 import inputs


def _group(n, seed, l=1, a=1):
    w = inputs.workload("three_layer", n=n, seed=seed)
    md = oracle.Medium(**w["medium"])
    root = oracle.tree_root(md, w["xyz"], w["layer"], l, a)
    return w, md, root


def _coverage(T, S, L, nt, ns):
    cnt = np.zeros((nt, ns), np.int32)
    for kind in ("U", "V", "W", "X"):
        for (bt, bs) in L[kind]:
            cnt[np.ix_(T.points(*bt), S.points(*bs))] += 1
    return cnt


@pytest.mark.parametrize("n,s,seed", [(300, 4, 1), (900, 16, 2), (600, 1, 3)])
@pytest.mark.parametrize("swap", [False, True])
def test_every_pair_is_covered_exactly_once(n, s, seed, swap):
    """The image tree is the denser one here, so the lists have W pairs; with the roles of the
    two trees swapped (images as targets) they have X pairs instead."""
    w, md, root = _group(n, seed)
    T, S, (tsrc, ssrc, _) = A.group_trees(md, w["xyz"], w["layer"], 1, 1, root, s)
    if swap:
        T, S, tsrc, ssrc = S, T, ssrc, tsrc
    L = A.dual_lists(T, S)
    cnt = _coverage(T, S, L, len(tsrc), len(ssrc))
    assert cnt.min() == 1 and cnt.max() == 1
    assert all(len(L[k]) > 0 for k in ("U", "V", "X" if swap else "W"))


def test_free_space_tree_covers_every_pair_including_self():
    w = inputs.workload("three_layer", n=800, seed=4)
    md = oracle.Medium(**w["medium"])
    root = oracle.tree_root(md, w["xyz"], w["layer"], 1, 1)
    tk, _, _ = oracle.tree_keys(md, w["xyz"], w["layer"], 1, 1, A.DMAX, root, 0)
    T = A.Tree(tk, 6)
    L = A.dual_lists(T, T)
    cnt = _coverage(T, T, L, len(tk), len(tk))
    assert cnt.min() == 1 and cnt.max() == 1


def test_lists_match_their_classical_characterisations():
    w, md, root = _group(1500, 5)
    T, S, _ = A.group_trees(md, w["xyz"], w["layer"], 1, 1, root, 5)
    L = A.dual_lists(T, S)
    par = lambda b: (b[0] - 1, b[1] >> 3)
    for (bt, bs) in L["V"]:
        assert bt[0] == bs[0] and not A.adjacent(*bt, *bs) and A.adjacent(*par(bt), *par(bs))
    for (bt, bs) in L["U"]:
        assert T.is_leaf(*bt) and S.is_leaf(*bs) and A.adjacent(*bt, *bs)
    for (bt, bs) in L["W"]:
        assert T.is_leaf(*bt) and bs[0] > bt[0] and not A.adjacent(*bt, *bs) and A.adjacent(*bt, *par(bs))
    for (bt, bs) in L["X"]:
        assert S.is_leaf(*bs) and bt[0] > bs[0] and not A.adjacent(*bt, *bs) and A.adjacent(*par(bt), *bs)
    # leaves hold at most s points unless at the finest level
    for (lev, key) in T.leaves:
        assert len(T.points(lev, key)) <= 5 or lev == A.DMAX


@pytest.mark.parametrize("D", [3, 4])
def test_uniform_tree_lists_equal_the_uniform_oracle_lists(D):
    w, md, root = _group(2000, 6)
    T, S, _ = A.group_trees(md, w["xyz"], w["layer"], 1, 1, root, 0, uniform=D)
    L = A.dual_lists(T, S)
    assert not L["W"] and not L["X"]
    tk, _, _ = oracle.tree_keys(md, w["xyz"], w["layer"], 1, 1, D, root, 0)
    sk, _, _ = oracle.tree_keys(md, w["xyz"], w["layer"], 1, 1, D, root, 1)
    for lev in range(2, D + 1):
        tb, sb = oracle.level_boxes(tk, D, lev), oracle.level_boxes(sk, D, lev)
        assert list(tb) == T.boxes[lev] and list(sb) == S.boxes[lev]
        for kind, name in ((0, "V"), (1, "U")):
            if kind == 1 and lev != D:
                continue
            off, idx = oracle.lists(tb, sb, lev, kind)
            ref = {(int(tb[t]), int(sb[j])) for t in range(len(tb)) for j in idx[off[t]:off[t + 1]]}
            got = {(bt[1], bs[1]) for (bt, bs) in L[name] if bt[0] == lev}
            assert got == ref, (lev, name)


@pytest.mark.parametrize("n,s,seed", [(300, 4, 1), (900, 16, 2)])
@pytest.mark.parametrize("swap", [False, True])
def test_two_box_lists_cover_every_pair_exactly_once(n, s, seed, swap):
    """With a separation of two boxes (the GPU's default, reading R22) the dual traversal still
    partitions every (target, source) pair: each lies in exactly one U, V, W or X box pair."""
    w, md, root = _group(n, seed)
    T, S, (tsrc, ssrc, _) = A.group_trees(md, w["xyz"], w["layer"], 1, 1, root, s)
    if swap:
        T, S, tsrc, ssrc = S, T, ssrc, tsrc
    L = A.dual_lists(T, S, ws=2)
    cnt = _coverage(T, S, L, len(tsrc), len(ssrc))
    assert cnt.min() == 1 and cnt.max() == 1
    assert all(len(L[k]) > 0 for k in ("U", "V", "X" if swap else "W"))


def test_two_box_near_rule():
    """adjacent(..., ws): at one level, indices within ws in every coordinate; across levels, the
    coarser cube grown by ws - 1 of its sides meets the finer one; ws = 1 is closed-cube contact."""
    key = lambda x, y, z: sum(((x >> k) & 1) << (3 * k + 2) | ((y >> k) & 1) << (3 * k + 1) | ((z >> k) & 1) << (3 * k)
                             for k in range(A.DMAX))
    for d in range(-4, 5):
        for ws in (1, 2):
            assert A.adjacent(4, key(8, 8, 8), 4, key(8 + d, 8, 8), ws) == (abs(d) <= ws)
            assert A.adjacent(4, key(8, 8, 8), 4, key(8 + d, 8 - d, 8 + d), ws) == (abs(d) <= ws)
    # level-3 box [4, 5) and level-5 boxes (units of 1/4 of it): grown by one side it spans [12, 24)
    for v in range(8, 28):
        near = 12 - 1 <= v <= 24  # closed cubes: the fine box [v, v + 1] meets [12, 24]
        assert A.adjacent(3, key(4, 4, 4), 5, key(v, 16, 16), 2) == near, v
        assert A.adjacent(5, key(v, 16, 16), 3, key(4, 4, 4), 2) == near, v
        assert A.adjacent(3, key(4, 4, 4), 5, key(v, 16, 16), 1) == (15 <= v <= 20), v


@pytest.mark.parametrize("D", [3, 4])
def test_uniform_tree_two_box_lists_equal_the_uniform_oracle_lists(D):
    w, md, root = _group(2000, 6)
    T, S, _ = A.group_trees(md, w["xyz"], w["layer"], 1, 1, root, 0, uniform=D)
    L = A.dual_lists(T, S, ws=2)
    assert not L["W"] and not L["X"]
    tk, _, _ = oracle.tree_keys(md, w["xyz"], w["layer"], 1, 1, D, root, 0)
    sk, _, _ = oracle.tree_keys(md, w["xyz"], w["layer"], 1, 1, D, root, 1)
    for lev in range(2, D + 1):
        tb, sb = oracle.level_boxes(tk, D, lev), oracle.level_boxes(sk, D, lev)
        for kind, name in ((0, "V"), (1, "U")):
            if kind == 1 and lev != D:
                continue
            off, idx = oracle.lists(tb, sb, lev, kind, ws=2)
            ref = {(int(tb[t]), int(sb[j])) for t in range(len(tb)) for j in idx[off[t]:off[t + 1]]}
            got = {(bt[1], bs[1]) for (bt, bs) in L[name] if bt[0] == lev}
            assert got == ref, (lev, name)
