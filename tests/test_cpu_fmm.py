"""CPU pins of the oracle's FMM (oracle/fmm.py), free space and reaction components, on uniform
and adaptive trees: with every expansion truncated at p and nothing else approximated, it must
converge geometrically in p to the direct sum (Sec. 3.1 and 3.4 expansions), for potential and
field.  Its pieces are checked on their own too (the near-field rule and the reaction M2L
operators against the oracle's adaptive quadratures).  It is the reference against which a GPU
FMM of the same trees and order can be compared to rounding."""
import numpy as np
import pytest

pytest.importorskip("scipy")

import oracle  # noqa: E402
from oracle import fmm  # noqa: E402
from paper_2002_01334_gb300 import inputs  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def w600():
    w = inputs.workload("three_layer", n=600, seed=31)
    md = oracle.Medium(**w["medium"])
    return w, md, oracle.direct(md, w["q"], w["xyz"], w["layer"], parts=1)


@pytest.mark.parametrize("D", [3, 4])
def test_free_fmm_converges_in_p_to_the_direct_sum(w600, D):
    w, md, ref = w600
    ep, ef = [], []
    for p in (2, 4, 6):
        phi, fld = fmm.free_fmm(md, w["q"], w["xyz"], w["layer"], p, D)
        ep.append(rel(phi, ref[0]))
        ef.append(rel(fld, ref[1]))
    assert ep[0] > 4 * ep[1] > 16 * ep[2] and ef[0] > 4 * ef[1] > 16 * ef[2], (ep, ef)
    assert ep[2] < 2e-4 and ef[2] < 1e-3, (ep, ef)


def test_free_fmm_at_depth_2_is_the_direct_sum(w600):
    """At depth 2 every pair of these charges is in the near lists (they fill one layer's cube,
    a small part of the group's root), so the FMM reduces to its exact near field."""
    w, md, ref = w600
    phi, fld = fmm.free_fmm(md, w["q"], w["xyz"], w["layer"], 2, 2)
    assert rel(phi, ref[0]) < 1e-13 and rel(fld, ref[1]) < 1e-13


def test_component_rule_matches_the_adaptive_pair_integral():
    """The near-field sum of oracle/fmm.py (a fixed composite rule per component) equals the
    oracle's adaptive quadrature of each pair, potential and field."""
    w = inputs.workload("four_layer", n=400, seed=3)
    md = oracle.Medium(**w["medium"])
    rng = np.random.default_rng(0)
    for (l, lp, a, b) in [(1, 1, 1, 1), (1, 2, 2, 2), (0, 3, 1, 2), (3, 0, 2, 1)]:
        T = w["xyz"][w["layer"] == l][:2]
        S = w["xyz"][w["layer"] == lp][:25]
        qs = rng.uniform(-1, 1, len(S))
        dmin = fmm._heights(md, l, a, T[:, 2]).min() + fmm._source_heights(md, lp, b, S[:, 2]).min()
        R = fmm.ComponentRule(md, l, lp, a, b, dmin, 1.5)
        for r in T:
            phi, f = R.sum_at(md, r, S, qs)
            ref = [oracle.green_react_ab(md, l, r, lp, s, a, b) for s in S]
            rphi = sum(qj * g for qj, (g, _) in zip(qs, ref))
            rf = sum(qj * gf for qj, (_, gf) in zip(qs, ref))
            assert abs(phi - rphi) <= 1e-12 * abs(rphi) and np.abs(f - rf).max() <= 1e-12 * np.abs(rf).max()


def test_reaction_m2l_shared_rule_matches_direct_quadrature():
    """The reaction M2L operators of oracle/fmm.py (one node set per component and level, the
    azimuth as phases) equal direct quadrature of eq. metoleimage2 (oracle/expansions.py)."""
    from oracle import expansions as E
    md = oracle.Medium([0.0, -1.2], [1.0, 8.6, 20.5], [1.2, 0.5, 2.1])
    h = 0.25
    M = np.random.default_rng(1).normal(size=25) + 1j * np.random.default_rng(2).normal(size=25)
    for (l, lp, a, b) in [(1, 1, 1, 1), (1, 2, 2, 2), (0, 2, 1, 2)]:
        dI = md.d[l] if a == 1 else md.d[l - 1]
        sg = 1 if a == 1 else -1
        R = fmm.ReactionM2L(md, l, lp, a, b, 4, h, np.sqrt(18) * h)
        for (dx, dy, kt, ks) in [(2, 1, 0, 0), (-3, -3, 2, 0)]:
            rct = np.array([0.1 + dx * h, 0.2 + dy * h, dI + sg * (kt + 0.5) * h])
            rcs = np.array([0.1, 0.2, dI - sg * (ks + 0.5) * h])
            ref = E.reaction_m2l(md, l, lp, a, b, rct, rcs, 4, 4) @ M
            assert np.abs(R.apply(rct, rcs, M) - ref).max() <= 1e-10 * np.abs(ref).max()


def test_reaction_fmm_converges_in_p_to_the_direct_sum():
    """Algorithm 1 for every component (oracle/fmm.py): geometric convergence in p of the
    reaction part to the oracle's direct sum, potential and field."""
    w = inputs.workload("three_layer", n=300, seed=21)
    md = oracle.Medium(**w["medium"])
    ref = oracle.direct(md, w["q"], w["xyz"], w["layer"], parts=2)
    ep, ef = [], []
    for p in (2, 4):
        phi, fld = fmm.react_fmm(md, w["q"], w["xyz"], w["layer"], p, 3)
        ep.append(rel(phi, ref[0]))
        ef.append(rel(fld, ref[1]))
    assert ep[0] > 8 * ep[1] and ef[0] > 5 * ef[1] and ep[1] < 3e-3 and ef[1] < 2e-2, (ep, ef)


def test_paper_accuracy_table_is_the_oracle_fmm_and_decays_in_p():
    """tests/golden/paper_accuracy_e2.json (make_paper_accuracy.py: the oracle's CPU FMM on the
    paper's irregular-body workload against the direct sum, per layer, the paper's Err_2 and
    Err_max) is reproduced for p = 2, and every layer's Err_2 falls at least 3x per two orders."""
    import json
    import os
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_accuracy_e2.json")) as f:
        fx = json.load(f)
    rows = fx["rows"]
    for k in range(3):
        e = [r["phi"][k]["err2"] for r in rows]
        assert all(e[i] > 3 * e[i + 1] for i in range(len(e) - 1)), (k, e)
    w = inputs.workload("paper_irregular")
    md = oracle.Medium(**w["medium"])
    ref_phi, _ = oracle.direct(md, w["q"], w["xyz"], w["layer"])
    phi, _ = fmm.fmm(md, w["q"], w["xyz"], w["layer"], rows[0]["p"], fx["depth"])
    for k in range(3):
        s = w["layer"] == k
        e2 = np.linalg.norm(phi[s] - ref_phi[s]) / np.linalg.norm(ref_phi[s])
        assert abs(e2 - rows[0]["phi"][k]["err2"]) <= 1e-9 * e2


def test_adaptive_free_fmm_converges_in_p_to_the_direct_sum():
    """The free-space FMM on adaptive trees (oracle/adaptive.py lists: V by M2L, U/W/X direct)
    on the paper's irregular bodies, where the leaves sit at several levels and W/X pairs occur,
    converges geometrically in p to the direct sum."""
    from oracle import adaptive as A
    w = inputs.workload("paper_irregular", n=1200)
    md = oracle.Medium(**w["medium"])
    root = oracle.tree_root(md, w["xyz"], w["layer"], 2, 2)
    keys, _, _ = oracle.tree_keys(md, w["xyz"], w["layer"], 2, 2, A.DMAX, root, 0)
    Ls = A.dual_lists(A.Tree(keys, 16), A.Tree(keys, 16))
    assert Ls["W"] and Ls["X"]
    ref = oracle.direct(md, w["q"], w["xyz"], w["layer"], parts=1)
    ep, ef = [], []
    for p in (2, 4, 6):
        phi, fld = fmm.free_fmm_adaptive(md, w["q"], w["xyz"], w["layer"], p, 16)
        ep.append(rel(phi, ref[0]))
        ef.append(rel(fld, ref[1]))
    assert ep[0] > 4 * ep[1] > 16 * ep[2] and ef[0] > 3 * ef[1] > 9 * ef[2] and ep[2] < 3e-4, (ep, ef)


def test_adaptive_two_box_free_fmm_is_more_accurate_at_the_same_order():
    """On adaptive trees too, lists with a separation of two boxes (reading R22) cut the truncation
    error at a given p by more than an order of magnitude (paper's bodies, p = 4: 4.3e-4 -> 2.4e-5
    in the potential), with every pair still summed once."""
    w = inputs.workload("paper_irregular", n=1200)
    md = oracle.Medium(**w["medium"])
    ref = oracle.direct(md, w["q"], w["xyz"], w["layer"], parts=1)
    e = {}
    for ws in (1, 2):
        phi, fld = fmm.free_fmm_adaptive(md, w["q"], w["xyz"], w["layer"], 4, 16, ws=ws)
        e[ws] = (rel(phi, ref[0]), rel(fld, ref[1]))
    assert e[2][0] < e[1][0] / 10 and e[2][1] < e[1][1] / 10 and e[2][0] < 1e-4, e


def test_adaptive_free_fmm_with_m2p_and_p2l():
    """The W and X pairs of adaptive lists by expansions (Sec. 3.5's lists for boxes of different
    sizes): M2P evaluates the finer source box's multipole expansion at the target leaf's points,
    P2L expands the coarser source leaf's charges about the target box's centre.  With two-box
    lists on the paper's bodies the error equals that of the direct W/X sums to 5 % and falls
    geometrically in p (2.4e-5 at p = 4)."""
    from oracle import adaptive as A
    w = inputs.workload("paper_irregular", n=1200)
    md = oracle.Medium(**w["medium"])
    root = oracle.tree_root(md, w["xyz"], w["layer"], 2, 2)
    keys, _, _ = oracle.tree_keys(md, w["xyz"], w["layer"], 2, 2, A.DMAX, root, 0)
    Ls = A.dual_lists(A.Tree(keys, 16), A.Tree(keys, 16), ws=2)
    assert Ls["W"] and Ls["X"]
    ref = oracle.direct(md, w["q"], w["xyz"], w["layer"], parts=1)
    e = {}
    for p, wx in ((2, "expansion"), (4, "expansion"), (4, "direct")):
        phi, fld = fmm.free_fmm_adaptive(md, w["q"], w["xyz"], w["layer"], p, 16, ws=2, wx=wx)
        e[(p, wx)] = (rel(phi, ref[0]), rel(fld, ref[1]))
    assert e[(2, "expansion")][0] > 10 * e[(4, "expansion")][0], e
    for k in (0, 1):
        assert abs(e[(4, "expansion")][k] - e[(4, "direct")][k]) <= 0.05 * e[(4, "direct")][k], e


def test_adaptive_reaction_fmm_converges_in_p_to_the_direct_sum():
    """The reaction part on adaptive dual trees (V by M2L with T, U/W/X by the component
    integral) converges in p to the direct sum on the paper's bodies."""
    w = inputs.workload("paper_irregular", n=300)
    md = oracle.Medium(**w["medium"])
    ref = oracle.direct(md, w["q"], w["xyz"], w["layer"], parts=2)
    ep, ef = [], []
    for p in (2, 4):
        phi, fld = fmm.react_fmm_adaptive(md, w["q"], w["xyz"], w["layer"], p, 8)
        ep.append(rel(phi, ref[0]))
        ef.append(rel(fld, ref[1]))
    assert ep[0] > 5 * ep[1] and ef[0] > 3 * ef[1] and ep[1] < 1e-2, (ep, ef)


def test_adaptive_two_box_reaction_fmm():
    """The reaction part on adaptive dual trees with two-box lists (reading R22): at p = 4 on the
    paper's bodies (300 charges, at most 8 per leaf) the error against the direct sum is 5.2e-4
    (potential) and 3.0e-3 (field), against 4.9e-3 and 2.0e-2 with one-box lists
    (test_adaptive_reaction_fmm_converges_in_p_to_the_direct_sum)."""
    w = inputs.workload("paper_irregular", n=300)
    md = oracle.Medium(**w["medium"])
    ref = oracle.direct(md, w["q"], w["xyz"], w["layer"], parts=2)
    phi, fld = fmm.react_fmm_adaptive(md, w["q"], w["xyz"], w["layer"], 4, 8, ws=2)
    assert rel(phi, ref[0]) < 1e-3 and rel(fld, ref[1]) < 6e-3, (rel(phi, ref[0]), rel(fld, ref[1]))


def test_two_box_separation_is_more_accurate_at_the_same_order(w600):
    """With far pairs at least two boxes apart (near field 5^3 boxes) the truncation error at a
    given p falls by more than an order of magnitude against the one-box rule."""
    w, md, ref = w600
    e1 = rel(fmm.free_fmm(md, w["q"], w["xyz"], w["layer"], 4, 4, ws=1)[0], ref[0])
    e2 = rel(fmm.free_fmm(md, w["q"], w["xyz"], w["layer"], 4, 4, ws=2)[0], ref[0])
    assert e2 < e1 / 10, (e1, e2)
