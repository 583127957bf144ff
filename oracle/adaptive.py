"""Adaptive dual trees and their interaction lists -- TEST INFRASTRUCTURE ONLY.

Plain Python restatement of the adaptive tree of one target group and its lists, for parity of a
GPU tree builder and for the coverage pin in tests/.  Only tests/ may import it; it shares no
code with the CUDA path.

Trees (Sec. 3.5: the root box of a component is bisected by its interface and the tree is built by
bisection): the target tree holds the group's targets, the source tree its sources (the same
charges for a free-space FMM, the polarization images for a reaction component).  Both live on
the group's root cube.  Every point has a cell at the finest depth Dmax, taken from the oracle's
key rule (oracle.tree_keys).  A box of either tree is split while it holds more than s of that
tree's points and its level is below Dmax; only non-empty boxes exist.

Lists, from the dual traversal that starts at the pair (target root, source root).  A pair (B, C)
of a target box and a source box, not adjacent (closed cubes disjoint), is far; an adjacent pair is
refined: both boxes when both have children, else the one that has.  Far pairs are
    V  same level                 (multipole-to-local),
    W  B a leaf, C finer than B   (multipole at B's targets; direct in a first version),
    X  C a leaf, B finer than C   (C's sources into B's local expansion; direct at first),
and an adjacent pair of two leaves is U (direct).  With a separation of ws boxes, "adjacent"
is "near": the coarser box grown by ws - 1 of its sides meets the finer one (ws = 1: the closed
cubes meet; at one level, indices within ws).  Every (target, source) pair of points then lies
in exactly one listed box pair: the traversal partitions B x C at every refinement.  For a tree of
uniform depth the lists are the uniform ones: V at every level is the same-level boxes whose
parents are adjacent but which are not, and U at the leaf level the adjacent leaves.
"""
import numpy as np

from . import tree_keys

DMAX = 21


def _decode(key):
    """Box coordinates (ix, iy, iz) of a Morton key (x in the highest of each bit triple)."""
    x = y = z = 0
    for k in range(DMAX):
        z |= ((key >> (3 * k)) & 1) << k
        y |= ((key >> (3 * k + 1)) & 1) << k
        x |= ((key >> (3 * k + 2)) & 1) << k
    return x, y, z


def adjacent(la, ka, lb, kb, ws=1):
    """Whether box (la, ka) and box (lb, kb) are near for a separation of ws boxes (levels may
    differ): the closed cube of the coarser box, grown by ws - 1 of its own sides in every
    direction, intersects the closed cube of the finer one.  ws = 1: the closed cubes intersect;
    for two boxes of one level: their indices differ by at most ws in every coordinate (the near
    rule of the uniform lists, Sec. 3.5 reading R22)."""
    ax, ay, az = _decode(ka)
    bx, by, bz = _decode(kb)
    L = max(la, lb)
    sa, sb = 1 << (L - la), 1 << (L - lb)
    ga = (ws - 1) * sa if la <= lb else 0  # the growth of the coarser cube, in units of level L
    gb = (ws - 1) * sb if lb < la else 0
    for u, v in ((ax, bx), (ay, by), (az, bz)):
        # [u sa - ga, (u + 1) sa + ga] and [v sb - gb, (v + 1) sb + gb] in units of level L
        if (u + 1) * sa + ga < v * sb - gb or (v + 1) * sb + gb < u * sa - ga:
            return False
    return True


class Tree:
    """Adaptive tree over points with depth-DMAX keys: split while count > s and level < dmax
    (or, with uniform set, split every box down to exactly level uniform)."""

    def __init__(self, keys, s, dmax=DMAX, uniform=None):
        self.keys = np.asarray(keys, np.uint64)
        self.order = np.argsort(self.keys, kind="stable")
        self.sk = self.keys[self.order]
        self.children = {}   # (level, key) -> list of child keys (level + 1)
        self.leaves = set()
        self.boxes = {0: [0]} if len(self.keys) else {}
        stack = [(0, 0)] if len(self.keys) else []
        while stack:
            lev, key = stack.pop()
            lo, hi = self.range(lev, key)
            split = (hi - lo > s and lev < dmax) if uniform is None else lev < uniform
            if not split:
                self.leaves.add((lev, key))
                continue
            ch = sorted({int(k) >> (3 * (DMAX - lev - 1)) for k in self.sk[lo:hi]})
            self.children[(lev, key)] = ch
            self.boxes.setdefault(lev + 1, []).extend(ch)
            stack.extend((lev + 1, c) for c in ch)
        for lev in self.boxes:
            self.boxes[lev] = sorted(set(self.boxes[lev]))

    def range(self, lev, key):
        """[lo, hi) of the sorted points inside box (lev, key)."""
        sh = 3 * (DMAX - lev)
        lo = np.searchsorted(self.sk, np.uint64(key << sh), "left")
        hi = np.searchsorted(self.sk, np.uint64(((key + 1) << sh) - 1), "right")
        return int(lo), int(hi)

    def points(self, lev, key):
        """Indices (into the input order) of the points in box (lev, key)."""
        lo, hi = self.range(lev, key)
        return self.order[lo:hi]

    def is_leaf(self, lev, key):
        return (lev, key) in self.leaves


def dual_lists(T, S, ws=1):
    """The lists of the dual traversal of target tree T and source tree S for a separation of ws
    boxes (adjacent(..., ws) decides near): a dict with keys 'V', 'U', 'W', 'X', each a sorted
    list of ((lt, kt), (ls, ks)) box pairs."""
    out = {"V": [], "U": [], "W": [], "X": []}
    if not T.boxes or not S.boxes:
        return out
    stack = [((0, 0), (0, 0))]
    while stack:
        (lt, kt), (ls, ks) = stack.pop()
        if not adjacent(lt, kt, ls, ks, ws):
            kind = "V" if lt == ls else ("W" if ls > lt else "X")
            out[kind].append(((lt, kt), (ls, ks)))
            continue
        tl, sl = T.is_leaf(lt, kt), S.is_leaf(ls, ks)
        if tl and sl:
            out["U"].append(((lt, kt), (ls, ks)))
        elif tl:
            stack.extend(((lt, kt), (ls + 1, c)) for c in S.children[(ls, ks)])
        elif sl:
            stack.extend(((lt + 1, c), (ls, ks)) for c in T.children[(lt, kt)])
        else:
            stack.extend(((lt + 1, a), (ls + 1, b)) for a in T.children[(lt, kt)] for b in S.children[(ls, ks)])
    for k in out:
        out[k].sort()
    return out


def group_trees(md, xyz, layer, l, a, root, s, uniform=None):
    """Target tree (the group's charges) and source tree (its images) of reaction group (l, a),
    with the point indices (charge index, image type) of the sources."""
    tk, tsrc, _ = tree_keys(md, xyz, layer, l, a, DMAX, root, 0)
    sk, ssrc, styp = tree_keys(md, xyz, layer, l, a, DMAX, root, 1)
    return Tree(tk, s, uniform=uniform), Tree(sk, s, uniform=uniform), (tsrc, ssrc, styp)
