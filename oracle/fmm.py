"""A plain CPU FMM for the free-space part -- TEST INFRASTRUCTURE ONLY.

The free-space Yukawa FMM of every layer (Sec. 3.1; Algorithm 2, first loop) on the uniform tree
of the layer's target group, written step by step from the paper's expansions and translations
(oracle/expansions.py, each pinned against the closed-form kernel):

  tree   the group's root cube (the C oracle's root rule), keys at depth D, boxes per level;
  P2M    M_nm = sum_j q_j 4 pi i_n(lam r_j) conj Y_n^m about each leaf centre (eq. melecoeffree);
  M2M    from level D up to level 2 (eq. metome, Thm. 2);
  M2L    at levels 2..D over the far lists: same-level boxes whose parents are adjacent but which
         are not (eq. metole, Thm. 3 with reading R20);
  L2L    from level 2 down to D (eq. metome);
  L2P    phi = c sum L_nm i_n(lam r) Y_n^m (eq. freespace3dlocexp) and the field from the LE
         shifted onto the target (its n <= 1 coefficients, exact);
  P2P    the near lists at level D, closed form, j != i;
with c = lam / (2 pi^2 eps) (k_0(lam r) = (pi/2) e^{-lam r} / (lam r)).  Every expansion is
truncated at degree p and nothing else is approximated, so its result is the FMM's own value at
that order and tree; against the direct sum it differs by the truncation error only.  Slow:
meant for a few thousand charges.  Only tests/ may import it; it shares no code with the CUDA
path.
"""
import math

import numpy as np
from scipy import special

from . import level_boxes, lists, tree_keys, tree_root
from . import expansions as E


def _decode(key):
    x = y = z = 0
    for k in range(21):
        z |= ((key >> (3 * k)) & 1) << k
        y |= ((key >> (3 * k + 1)) & 1) << k
        x |= ((key >> (3 * k + 2)) & 1) << k
    return x, y, z


class _Box:
    def __init__(self, root, lev):
        H = root[3]
        self.size = 2.0 * H / (1 << lev)
        self.x0 = np.array([root[0] - H, root[1] - H, root[2] - H])

    def centre(self, key):
        return self.x0 + (np.array(_decode(int(key)), float) + 0.5) * self.size


def _radial_rows(lam, R, p):
    """i_n(lam R) for the rows (n, m) of _nm(p), points along the second axis."""
    nrow = np.array([n for n, _ in E._nm(p)])
    return special.spherical_in(np.arange(p + 1)[:, None], lam * np.asarray(R)[None, :])[nrow]


def _me_of_points(lam, pts, q, c, p):
    """sum_j q_j 4 pi i_n(lam r_j) conj Y_n^m of the points about c (P2M)."""
    R, T, P = E.sph(pts - c)
    return 4 * math.pi * (_radial_rows(lam, R, p) * np.conj(E.ylm_all(p, T, P))) @ q


def _le_at_points(lam, L, c, pts, p):
    """sum L_nm i_n(lam r) Y_n^m about c at the points, and the gradient of that sum at each point
    from the LE shifted onto the point (Thm. 2): only its n <= 1 coefficients enter."""
    R, T, P = E.sph(pts - c)
    val = (L[:, None] * _radial_rows(lam, R, p) * E.ylm_all(p, T, P)).sum(0)
    grad = np.zeros((len(pts), 3))
    a0 = math.sqrt(3.0 / (4 * math.pi))
    a1 = math.sqrt(3.0 / (8 * math.pi))
    for i, r in enumerate(pts):
        Ls = E.free_shat(lam, r - c, p, 1).T @ L  # coefficients (0,0), (1,-1), (1,0), (1,1) about r
        # i_1(lam s) Y_1^m(s) = (lam / 3) s Y_1^m + O(s^3); s Y_1^0 = a0 z, s Y_1^{+-1} = -+a1 (x +- i y)
        g = (lam / 3.0) * np.array([(-Ls[3] + Ls[1]) * a1, (-1j * Ls[3] - 1j * Ls[1]) * a1, Ls[2] * a0])
        grad[i] = g.real
    return val.real, grad


def free_fmm(md, q, xyz, layer, p, D):
    """Free-space part of phi and field (field = -grad phi) of every charge by the FMM above, with
    every group tree at uniform depth D >= 2.  Returns (phi[n], field[n, 3])."""
    q = np.asarray(q, float)
    xyz = np.asarray(xyz, float).reshape(-1, 3)
    layer = np.asarray(layer, np.int32)
    n = len(q)
    phi = np.zeros(n)
    field = np.zeros((n, 3))
    for l in range(md.L + 1):
        if not np.any(layer == l):
            continue
        a = 1 if l < md.L else 2
        lam, eps = md.lam[l], md.eps[l]
        cfac = lam / (2 * math.pi ** 2 * eps)
        root = tree_root(md, xyz, layer, l, a)
        keys, src, _ = tree_keys(md, xyz, layer, l, a, D, root, 0)
        boxes = {lev: level_boxes(keys, D, lev) for lev in range(2, D + 1)}
        geo = {lev: _Box(root, lev) for lev in range(2, D + 1)}
        leaf_of = np.searchsorted(boxes[D], keys)
        members = [src[leaf_of == b] for b in range(len(boxes[D]))]
        # upward pass
        M = {D: np.array([_me_of_points(lam, xyz[mem], q[mem], geo[D].centre(k), p)
                          for k, mem in zip(boxes[D], members)])}
        for lev in range(D - 1, 1, -1):
            Mp = np.zeros((len(boxes[lev]), (p + 1) ** 2), complex)
            par = np.searchsorted(boxes[lev], boxes[lev + 1] >> np.uint64(3))
            ops = {}
            for ci, ck in enumerate(boxes[lev + 1]):
                off = tuple(geo[lev + 1].centre(ck) - geo[lev].centre(boxes[lev][par[ci]]))
                if off not in ops:
                    ops[off] = np.conj(E.free_shat(lam, np.array(off), p, p))  # b = child - parent
                Mp[par[ci]] += ops[off] @ M[lev + 1][ci]
            M[lev] = Mp
        # far field
        L = {lev: np.zeros((len(boxes[lev]), (p + 1) ** 2), complex) for lev in range(2, D + 1)}
        for lev in range(2, D + 1):
            off, idx = lists(boxes[lev], boxes[lev], lev, 0)
            ops = {}
            for t in range(len(boxes[lev])):
                ct = geo[lev].centre(boxes[lev][t])
                for s in idx[off[t]:off[t + 1]]:
                    b = ct - geo[lev].centre(boxes[lev][s])
                    kb = tuple(np.round(b / geo[lev].size).astype(int))
                    if kb not in ops:
                        ops[kb] = E.free_s(lam, b, p, p).T
                    L[lev][t] += ops[kb] @ M[lev][s]
        # downward pass
        for lev in range(2, D):
            par = np.searchsorted(boxes[lev], boxes[lev + 1] >> np.uint64(3))
            ops = {}
            for ci, ck in enumerate(boxes[lev + 1]):
                d = geo[lev + 1].centre(ck) - geo[lev].centre(boxes[lev][par[ci]])
                kd = tuple(np.sign(d).astype(int))
                if kd not in ops:
                    ops[kd] = E.free_shat(lam, d, p, p).T
                L[lev + 1][ci] += ops[kd] @ L[lev][par[ci]]
        # leaves: local expansion and near field
        uoff, uidx = lists(boxes[D], boxes[D], D, 1)
        for b, mem in enumerate(members):
            pts = xyz[mem]
            v, g = _le_at_points(lam, L[D][b], geo[D].centre(boxes[D][b]), pts, p)
            phi[mem] += cfac * v
            field[mem] -= cfac * g
            near = np.concatenate([members[s] for s in uidx[uoff[b]:uoff[b + 1]]])
            for i in mem:
                js = near[near != i]
                d = xyz[i] - xyz[js]
                r = np.sqrt((d * d).sum(1))
                e = q[js] * np.exp(-lam * r) / (4 * math.pi * eps * r)
                phi[i] += e.sum()
                field[i] += ((e * (1 + lam * r) / (r * r))[:, None] * d).sum(0)
    return phi, field
