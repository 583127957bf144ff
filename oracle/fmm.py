"""A plain CPU FMM, free-space and reaction parts -- TEST INFRASTRUCTURE ONLY.

free_fmm: the free-space Yukawa FMM of every layer (Sec. 3.1; Algorithm 2, first loop) on the uniform tree
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
with c = lam / (2 pi^2 eps) (k_0(lam r) = (pi/2) e^{-lam r} / (lam r)).
react_fmm: Algorithm 1 for every reaction component on the same group trees (images as sources,
one ME per source type, M2L by T of eqs. metoleimage1-2 on a shared quadrature node set per
component and level, near field by the component integral).
free_fmm_adaptive, react_fmm_adaptive: both parts on adaptive trees (oracle/adaptive.py), V by
M2L and U/W/X pairs directly.  Every expansion is
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
from .adaptive import _decode


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


def _lists_ws(tb, sb, lev, kind, ws):
    """Uniform-tree lists with separation ws boxes (oracle.lists): near (kind 1) = source boxes
    within ws boxes in every coordinate; far (kind 0) = source boxes farther than ws whose parents
    are within ws of the target's parent.  CSR over the target boxes: (off, idx)."""
    return lists(tb, sb, lev, kind, ws)


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


def free_fmm(md, q, xyz, layer, p, D, ws=1):
    """Free-space part of phi and field (field = -grad phi) of every charge by the FMM above, with
    every group tree at uniform depth D >= 2 and separation ws boxes (1: the GPU's lists).
    Returns (phi[n], field[n, 3])."""
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
            off, idx = _lists_ws(boxes[lev], boxes[lev], lev, 0, ws)
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
        uoff, uidx = _lists_ws(boxes[D], boxes[D], D, 1, ws)
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


# ------------------------------------------------------------------------------------------
# Reaction components (Sec. 3.3-3.4, Algorithm 1 for every component, Algorithm 2)

def _heights(md, l, a, z):
    """The target's distance to the interface of its side: z - d_l (a = 1), d_{l-1} - z (a = 2)."""
    return z - md.d[l] if a == 1 else md.d[l - 1] - z


def _source_heights(md, lp, b, z):
    """The source's distance in the exponent of eq. zexponential: z' - d_l' (b = 1), d_{l'-1} - z' (b = 2)."""
    return z - md.d[lp] if b == 1 else md.d[lp - 1] - z


class ComponentRule:
    """Composite 16-point Gauss-Legendre rule in lambda_rho for one component u^{ab}_{l l'}, with
    its layer densities at the nodes: panels of width min(2/dmin, pi/rhomax, (lmin + x)/2) up to
    x = 60/dmin, for pairs whose exponent distances sum to at least dmin and whose horizontal
    distances are at most rhomax (the integrand then decays below e^-60 of its size at 0)."""

    def __init__(self, md, l, lp, a, b, dmin, rhomax):
        from . import sigma
        self.l, self.lp, self.a, self.b = l, lp, a, b
        gx, gw = np.polynomial.legendre.leggauss(16)
        lmin = min(md.lam[l], md.lam[lp])
        wmax = 2.0 / dmin
        if rhomax > 0:
            wmax = min(wmax, math.pi / rhomax)
        xs, ws, x = [], [], 0.0
        X = 60.0 / dmin
        while x < X:
            dw = min(wmax, 0.5 * (lmin + x), X - x)
            xs.append(x + 0.5 * dw * (gx + 1.0))
            ws.append(0.5 * dw * gw)
            x += dw
        self.x = np.concatenate(xs)
        self.w = np.concatenate(ws)
        self.lz = np.sqrt(md.lam[l] ** 2 + self.x ** 2)
        self.lzp = np.sqrt(md.lam[lp] ** 2 + self.x ** 2)
        self.sig = np.array([sigma(md, v, l, lp, a, b) for v in self.x])

    def sum_at(self, md, r, src, q):
        """sum_j q_j u^{ab}_{l l'}(r, r'_j) and its -grad_r, r one target, src[j] source positions
        (eq. generalcomponents after the alpha integral: (1/4 pi) int lr J0(lr rho) e^{-lz h -
        lz' h'} sigma / lz d lr)."""
        ht = _heights(md, self.l, self.a, r[2])
        hs = _source_heights(md, self.lp, self.b, src[:, 2])
        dx, dy = r[0] - src[:, 0], r[1] - src[:, 1]
        rho = np.hypot(dx, dy)
        X = self.x[:, None]
        e = (self.w * self.x * self.sig / self.lz / (4 * math.pi))[:, None] * np.exp(
            -self.lz[:, None] * ht - self.lzp[:, None] * hs[None, :])
        j0 = special.j0(X * rho[None, :])
        # J1(x rho) / rho, with its limit x / 2 at rho = 0
        j1r = np.where(rho[None, :] > 0, special.j1(X * rho[None, :]) / np.where(rho > 0, rho, 1.0)[None, :], 0.5 * X)
        phi = (e * j0).sum(0) @ q
        fr = (e * X * j1r).sum(0)
        fz = (e * j0 * self.lz[:, None]).sum(0) * (1.0 if self.a == 1 else -1.0)
        return phi, np.array([(q * fr * dx).sum(), (q * fr * dy).sum(), (q * fz).sum()])


class ReactionM2L:
    """M2L operators T of one component u^{ab}_{l l'} at one tree level (eqs. metoleimage1,
    metoleimage2), by a composite Gauss-Legendre rule in lambda_rho shared by the level's classes.
    A class is the horizontal offset rho (along +x) and the heights zt, zs of the target and source
    centres above/below the interface; another azimuth phi multiplies entry (nm, nu mu) by
    e^{i (mu - m) phi}.  Rule: panels of width min(2/dmin, pi/rhomax, (lmin + x)/2) up to
    x = (70 + 2p)/dmin, dmin the smallest zt + zs of the level, rhomax its largest rho."""

    def __init__(self, md, l, lp, a, b, p, dmin, rhomax):
        from . import sigma
        self.md, self.l, self.lp, self.a, self.b, self.p = md, l, lp, a, b, p
        gx, gw = np.polynomial.legendre.leggauss(16)
        lam, lamp = md.lam[l], md.lam[lp]
        wmax = 2.0 / dmin
        if rhomax > 0:
            wmax = min(wmax, math.pi / rhomax)
        xs, ws, x = [], [], 0.0
        X = (70.0 + 2 * p) / dmin
        while x < X:
            dw = min(wmax, 0.5 * (min(lam, lamp) + x), X - x)
            xs.append(x + 0.5 * dw * (gx + 1.0))
            ws.append(0.5 * dw * gw)
            x += dw
        self.x = np.concatenate(xs)
        w = np.concatenate(ws)
        self.lz = np.sqrt(lam ** 2 + self.x ** 2)
        self.lzp = np.sqrt(lamp ** 2 + self.x ** 2)
        sig = np.array([sigma(md, v, l, lp, a, b) for v in self.x])
        self.base = w * self.x / self.lz * sig
        self.pt = np.array([E.phat_all(p, v / lam) for v in self.lz])    # [nodes, K]
        self.ps = np.array([E.phat_all(p, v / lamp) for v in self.lzp])
        idx = E._nm(p)
        self.k = np.array([[mu - m for _, mu in idx] for _, m in idx])
        n_ = np.array([n for n, _ in idx])[:, None]
        m_ = np.array([m for _, m in idx])[:, None]
        nu_ = np.array([n for n, _ in idx])[None, :]
        mu_ = np.array([m for _, m in idx])[None, :]
        self.sgn = ((-1.0) ** n_ * np.ones_like(nu_)) if a == 1 else (-1.0) ** (m_ + nu_ + mu_)
        self.cache = {}

    def T(self, rho, zt, zs):
        """The operator at azimuth 0 for horizontal offset rho and heights zt, zs (cached)."""
        key = (round(rho, 12), round(zt, 12), round(zs, 12))
        if key not in self.cache:
            e = self.base * np.exp(-self.lz * zt - self.lzp * zs)
            p = self.p
            J = special.jv(np.arange(-2 * p, 2 * p + 1)[None, :], self.x[:, None] * rho)  # [nodes, 4p + 1]
            m_row = np.array([m for _, m in E._nm(p)])
            mu_col = m_row
            T = np.zeros(self.k.shape, complex)
            for mv in range(-p, p + 1):
                rows = m_row == mv
                # entry (nm, nu mu) integrates e pt ps J_{mu - m}: one product per target order m
                T[rows] = (self.pt[:, rows] * e[:, None]).T @ (self.ps * J[:, mu_col - mv + 2 * p])
            self.cache[key] = self.sgn * (1j) ** self.k * T
        return self.cache[key]

    def apply(self, rct, rcs, M):
        """L += T(rct, rcs) M for the target centre rct and polarization centre rcs."""
        d = rct - rcs
        rho, ph = math.hypot(d[0], d[1]), math.atan2(d[1], d[0])
        dI = self.md.d[self.l] if self.a == 1 else self.md.d[self.l - 1]
        zt, zs = (rct[2] - dI, dI - rcs[2]) if self.a == 1 else (dI - rct[2], rcs[2] - dI)
        return (np.exp(1j * self.k * ph) * self.T(rho, zt, zs)) @ M


def react_fmm(md, q, xyz, layer, p, D, ws=1):
    """Reaction part of phi and field of every charge: Algorithm 1 for every component, on the
    uniform trees (depth D) of each target group (l, a).  Targets are the layer's charges; sources
    are the polarization images (eq. eqpolarizedsource) of every charge, one ME per source type
    (l', b) about each image box centre (eq. melayerupgoingimage, with lam_l'), shifted upward with
    lam_l' (eq. metome), translated by T (eqs. metoleimage1-2) over the far lists at levels 2..D,
    shifted down and evaluated with lam_l (eqs. metome, lelayerimage); the near lists at level D
    are summed directly by the component integral (eq. generalcomponents), the charge's own image
    included.  Returns (phi[n], field[n, 3])."""
    from . import image_z
    q = np.asarray(q, float)
    xyz = np.asarray(xyz, float).reshape(-1, 3)
    layer = np.asarray(layer, np.int32)
    n = len(q)
    phi = np.zeros(n)
    field = np.zeros((n, 3))
    Lm = md.L
    K = (p + 1) ** 2
    for l in range(Lm + 1):
        if not np.any(layer == l):
            continue
        lam = md.lam[l]
        for a in (1, 2):
            if (a == 1 and l == Lm) or (a == 2 and l == 0):
                continue
            root = tree_root(md, xyz, layer, l, a)
            tk, tsrc, _ = tree_keys(md, xyz, layer, l, a, D, root, 0)
            ik, isrc, ityp = tree_keys(md, xyz, layer, l, a, D, root, 1)
            if len(ik) == 0:
                continue
            ipos = xyz[isrc].copy()
            for j in range(len(ik)):
                lp, b = divmod(int(ityp[j]), 2)
                ipos[j, 2] = image_z(md, l, a, lp, b + 1, xyz[isrc[j], 2])
            types = sorted(set(int(t) for t in ityp))
            tb = {lev: level_boxes(tk, D, lev) for lev in range(2, D + 1)}
            ib = {lev: level_boxes(ik, D, lev) for lev in range(2, D + 1)}
            geo = {lev: _Box(root, lev) for lev in range(2, D + 1)}
            ileaf = np.searchsorted(ib[D], ik)
            tleaf = np.searchsorted(tb[D], tk)
            # upward pass on the image tree, one expansion per source type
            M = {D: np.zeros((len(ib[D]), len(types), K), complex)}
            for bi in range(len(ib[D])):
                c = geo[D].centre(ib[D][bi])
                for ti, t in enumerate(types):
                    sel = np.nonzero((ileaf == bi) & (ityp == t))[0]
                    if len(sel):
                        M[D][bi, ti] = _me_of_points(md.lam[t // 2], ipos[sel], q[isrc[sel]], c, p)
            for lev in range(D - 1, 1, -1):
                M[lev] = np.zeros((len(ib[lev]), len(types), K), complex)
                par = np.searchsorted(ib[lev], ib[lev + 1] >> np.uint64(3))
                ops = {}
                for ci, ck in enumerate(ib[lev + 1]):
                    off = geo[lev + 1].centre(ck) - geo[lev].centre(ib[lev][par[ci]])
                    for ti, t in enumerate(types):
                        key = (tuple(np.sign(off).astype(int)), t // 2)
                        if key not in ops:
                            ops[key] = np.conj(E.free_shat(md.lam[t // 2], off, p, p))  # b = child - parent
                        M[lev][par[ci], ti] += ops[key] @ M[lev + 1][ci, ti]
            # far field
            L = {lev: np.zeros((len(tb[lev]), K), complex) for lev in range(2, D + 1)}
            for lev in range(2, D + 1):
                off, idx = _lists_ws(tb[lev], ib[lev], lev, 0, ws)
                if len(idx) == 0:
                    continue
                h = geo[lev].size
                rmax = math.sqrt(2.0) * (2 * ws + 1) * h
                ops = {t: ReactionM2L(md, l, t // 2, a, t % 2 + 1, p, h, rmax) for t in types}
                for t_ in range(len(tb[lev])):
                    ct = geo[lev].centre(tb[lev][t_])
                    for s in idx[off[t_]:off[t_ + 1]]:
                        cs = geo[lev].centre(ib[lev][s])
                        for ti, t in enumerate(types):
                            if np.any(M[lev][s, ti]):
                                L[lev][t_] += ops[t].apply(ct, cs, M[lev][s, ti])
            for lev in range(2, D):
                par = np.searchsorted(tb[lev], tb[lev + 1] >> np.uint64(3))
                ops = {}
                for ci, ck in enumerate(tb[lev + 1]):
                    d = geo[lev + 1].centre(ck) - geo[lev].centre(tb[lev][par[ci]])
                    kd = tuple(np.sign(d).astype(int))
                    if kd not in ops:
                        ops[kd] = E.free_shat(lam, d, p, p).T
                    L[lev + 1][ci] += ops[kd] @ L[lev][par[ci]]
            # leaves: local expansion and near field
            uoff, uidx = _lists_ws(tb[D], ib[D], D, 1, ws)
            hD = geo[D].size
            rules = {}
            tz = xyz[tsrc, 2]
            for t in types:
                lp, b = t // 2, t % 2 + 1
                ht = _heights(md, l, a, tz).min()
                hs = _source_heights(md, lp, b, xyz[isrc[ityp == t], 2]).min()
                rules[t] = ComponentRule(md, l, lp, a, b, ht + hs, math.sqrt(2.0) * (ws + 1) * hD * 1.000001)
            for bt in range(len(tb[D])):
                mem = tsrc[tleaf == bt]
                v, g = _le_at_points(lam, L[D][bt], geo[D].centre(tb[D][bt]), xyz[mem], p)
                phi[mem] += v
                field[mem] -= g
                near = np.isin(ileaf, uidx[uoff[bt]:uoff[bt + 1]])
                for t in types:
                    sel = np.nonzero(near & (ityp == t))[0]
                    if not len(sel):
                        continue
                    srcs = xyz[isrc[sel]]
                    qs = q[isrc[sel]]
                    for i in mem:
                        ph, f = rules[t].sum_at(md, xyz[i], srcs, qs)
                        phi[i] += ph
                        field[i] += f
    return phi, field


def fmm(md, q, xyz, layer, p, D, ws=1):
    """phi and field of every charge (free part + reaction part), the sum of free_fmm and react_fmm."""
    a, fa = free_fmm(md, q, xyz, layer, p, D, ws)
    b, fb = react_fmm(md, q, xyz, layer, p, D, ws)
    return a + b, fa + fb


def _m2p(lam, M, c, pts, p):
    """Value and gradient at each point of the ME M (degree p) about c: the ME translated (Thm. 3)
    into a degree-1 LE about the point itself, whose n <= 1 coefficients give both exactly."""
    val = np.zeros(len(pts))
    grad = np.zeros((len(pts), 3))
    for i, r in enumerate(pts):
        Lr = E.free_m2l(lam, M, c, r, p, 1)
        v, g = _le_at_points(lam, Lr, r, r[None, :], 1)
        val[i], grad[i] = v[0], g[0]
    return val, grad


def _p2l(lam, pts, q, c, p):
    """LE about c (degree p) of the point sources (eq. melecoeffree, conjugate reading):
    sum_j q_j 4 pi k_n(lam |r_j - c|) conj Y_n^m of r_j - c."""
    R, T, P = E.sph(pts - c)
    rows = np.array([special.spherical_kn(n, lam * R) for n, _ in E._nm(p)])
    return 4 * math.pi * (rows * np.conj(E.ylm_all(p, T, P))) @ q


def free_fmm_adaptive(md, q, xyz, layer, p, s, ws=1, wx="direct"):
    """Free-space part of phi and field on adaptive trees: each layer's tree (the group root of the
    uniform case, keys at depth 21) split while a box holds more than s charges
    (oracle/adaptive.py).  Lists from the dual traversal of the tree with itself for a separation of
    ws boxes.  wx = "direct": W and X pairs summed directly; wx = "expansion": a W pair (target
    leaf B, finer source box C) by C's multipole expansion evaluated at B's targets (M2P), an X
    pair (target box B, coarser source leaf C) by C's charges expanded about B's centre and added
    to B's local expansion before it is shifted down (P2L); boxes above level 2 keep the direct
    sum.  V pairs by M2L
    (Thm. 3), U, W and X pairs summed directly (closed form, j != i).  Expansions exist for the
    boxes of level >= 2: P2M at leaves, M2M to parents, L2L to children, L2P at target leaves.
    Returns (phi[n], field[n, 3])."""
    from . import adaptive as A
    q = np.asarray(q, float)
    xyz = np.asarray(xyz, float).reshape(-1, 3)
    layer = np.asarray(layer, np.int32)
    n = len(q)
    phi = np.zeros(n)
    field = np.zeros((n, 3))
    K = (p + 1) ** 2
    for l in range(md.L + 1):
        if not np.any(layer == l):
            continue
        a = 1 if l < md.L else 2
        lam, eps = md.lam[l], md.eps[l]
        cfac = lam / (2 * math.pi ** 2 * eps)
        root = tree_root(md, xyz, layer, l, a)
        keys, src, _ = tree_keys(md, xyz, layer, l, a, A.DMAX, root, 0)
        T = A.Tree(keys, s)
        lists_ = A.dual_lists(T, T, ws)
        H = root[3]
        x0 = np.array([root[0] - H, root[1] - H, root[2] - H])

        def centre(lev, key):
            return x0 + (np.array(_decode(int(key)), float) + 0.5) * (2.0 * H / (1 << lev))

        def pts(lev, key):
            return src[T.points(lev, key)]

        levels = sorted(T.boxes)
        M = {}
        for lev in reversed(levels):
            if lev < 2:
                break
            for key in T.boxes[lev]:
                c = centre(lev, key)
                if T.is_leaf(lev, key):
                    mem = pts(lev, key)
                    M[(lev, key)] = _me_of_points(lam, xyz[mem], q[mem], c, p)
                else:
                    acc = np.zeros(K, complex)
                    for ch in T.children[(lev, key)]:
                        acc += np.conj(E.free_shat(lam, centre(lev + 1, ch) - c, p, p)) @ M[(lev + 1, ch)]
                    M[(lev, key)] = acc
        L = {}
        ops = {}
        for (bt, bs) in lists_["V"]:
            b = centre(*bt) - centre(*bs)
            kb = (bt[0],) + tuple(np.round(b / (2.0 * H / (1 << bt[0]))).astype(int))
            if kb not in ops:
                ops[kb] = E.free_s(lam, b, p, p).T
            L[bt] = L.get(bt, np.zeros(K, complex)) + ops[kb] @ M[bs]
        # the pairs summed directly: U, and W / X unless expanded
        direct = list(lists_["U"])
        if wx == "expansion":
            for (bt, bs) in lists_["X"]:
                if bt[0] < 2:
                    direct.append((bt, bs))
                    continue
                sm = pts(*bs)
                L[bt] = L.get(bt, np.zeros(K, complex)) + _p2l(lam, xyz[sm], q[sm], centre(*bt), p)
            for (bt, bs) in lists_["W"]:
                if bs not in M:
                    direct.append((bt, bs))
                    continue
                tm = pts(*bt)
                v, g = _m2p(lam, M[bs], centre(*bs), xyz[tm], p)
                phi[tm] += cfac * v
                field[tm] -= cfac * g
        else:
            direct += lists_["W"] + lists_["X"]
        for lev in levels:
            if lev < 2:
                continue
            for key in T.boxes[lev]:
                if (lev, key) not in L or T.is_leaf(lev, key):
                    continue
                c = centre(lev, key)
                for ch in T.children[(lev, key)]:
                    L[(lev + 1, ch)] = L.get((lev + 1, ch), np.zeros(K, complex)) + \
                        E.free_shat(lam, centre(lev + 1, ch) - c, p, p).T @ L[(lev, key)]
        for (lev, key) in T.leaves:
            if (lev, key) in L:
                mem = pts(lev, key)
                v, g = _le_at_points(lam, L[(lev, key)], centre(lev, key), xyz[mem], p)
                phi[mem] += cfac * v
                field[mem] -= cfac * g
        for (bt, bs) in direct:
            tm, sm = pts(*bt), pts(*bs)
            for i in tm:
                js = sm[sm != i]
                d = xyz[i] - xyz[js]
                r = np.sqrt((d * d).sum(1))
                e = q[js] * np.exp(-lam * r) / (4 * math.pi * eps * r)
                phi[i] += e.sum()
                field[i] += ((e * (1 + lam * r) / (r * r))[:, None] * d).sum(0)
    return phi, field


def react_fmm_adaptive(md, q, xyz, layer, p, s, ws=1):
    """Reaction part of phi and field on adaptive dual trees (oracle/adaptive.py): per target
    group (l, a) the target tree of its charges and the source tree of its images, each split
    while a box holds more than s of its points, lists for a separation of ws boxes.  V pairs by M2L (T of eqs. metoleimage1-2, one
    ME per source type), U, W and X pairs by the component integral directly; expansions for the
    boxes of level >= 2 (P2M at image leaves, M2M with lam_l', L2L and L2P with lam_l).
    Returns (phi[n], field[n, 3])."""
    from . import adaptive as A
    from . import image_z
    q = np.asarray(q, float)
    xyz = np.asarray(xyz, float).reshape(-1, 3)
    layer = np.asarray(layer, np.int32)
    n = len(q)
    phi = np.zeros(n)
    field = np.zeros((n, 3))
    K = (p + 1) ** 2
    for l in range(md.L + 1):
        if not np.any(layer == l):
            continue
        lam = md.lam[l]
        for a in (1, 2):
            if (a == 1 and l == md.L) or (a == 2 and l == 0):
                continue
            root = tree_root(md, xyz, layer, l, a)
            T, S, (tsrc, isrc, ityp) = A.group_trees(md, xyz, layer, l, a, root, s)
            if not S.boxes or not T.boxes:
                continue
            H = root[3]
            x0 = np.array([root[0] - H, root[1] - H, root[2] - H])

            def centre(lev, key):
                return x0 + (np.array(_decode(int(key)), float) + 0.5) * (2.0 * H / (1 << lev))

            ipos = xyz[isrc].copy()
            for j in range(len(isrc)):
                lp, b = divmod(int(ityp[j]), 2)
                ipos[j, 2] = image_z(md, l, a, lp, b + 1, xyz[isrc[j], 2])
            types = sorted(set(int(t) for t in ityp))
            Ls = A.dual_lists(T, S, ws)
            # upward pass on the image tree, one expansion per source type
            M = {}
            for lev in sorted(S.boxes, reverse=True):
                if lev < 2:
                    break
                for key in S.boxes[lev]:
                    c = centre(lev, key)
                    Mb = np.zeros((len(types), K), complex)
                    if S.is_leaf(lev, key):
                        sel = S.points(lev, key)
                        for ti, t in enumerate(types):
                            st = sel[ityp[sel] == t]
                            if len(st):
                                Mb[ti] = _me_of_points(md.lam[t // 2], ipos[st], q[isrc[st]], c, p)
                    else:
                        for ch in S.children[(lev, key)]:
                            off = centre(lev + 1, ch) - c
                            for ti, t in enumerate(types):
                                Mb[ti] += np.conj(E.free_shat(md.lam[t // 2], off, p, p)) @ M[(lev + 1, ch)][ti]
                    M[(lev, key)] = Mb
            # far field
            L = {}
            ops = {}
            for (bt, bs) in Ls["V"]:
                lev = bt[0]
                h = 2.0 * H / (1 << lev)
                for ti, t in enumerate(types):
                    if not np.any(M[bs][ti]):
                        continue
                    if (lev, t) not in ops:
                        # V pairs lie within (2 ws + 1) boxes in x and y: rho <= (2 ws + 1) sqrt(2) h
                        ops[(lev, t)] = ReactionM2L(md, l, t // 2, a, t % 2 + 1, p, h,
                                                   (2 * ws + 1) * math.sqrt(2.0) * h)
                    L[bt] = L.get(bt, np.zeros(K, complex)) + ops[(lev, t)].apply(centre(*bt), centre(*bs), M[bs][ti])
            for lev in sorted(T.boxes):
                if lev < 2:
                    continue
                for key in T.boxes[lev]:
                    if (lev, key) not in L or T.is_leaf(lev, key):
                        continue
                    c = centre(lev, key)
                    for ch in T.children[(lev, key)]:
                        L[(lev + 1, ch)] = L.get((lev + 1, ch), np.zeros(K, complex)) + \
                            E.free_shat(lam, centre(lev + 1, ch) - c, p, p).T @ L[(lev, key)]
            for (lev, key) in T.leaves:
                if (lev, key) in L:
                    mem = tsrc[T.points(lev, key)]
                    v, g = _le_at_points(lam, L[(lev, key)], centre(lev, key), xyz[mem], p)
                    phi[mem] += v
                    field[mem] -= g
            # direct pairs
            rules = {}
            for t in types:
                lp, b = t // 2, t % 2 + 1
                ht = _heights(md, l, a, xyz[tsrc, 2]).min()
                hs = _source_heights(md, lp, b, xyz[isrc[ityp == t], 2]).min()
                rules[t] = ComponentRule(md, l, lp, a, b, ht + hs, 2.0 * math.sqrt(2.0) * H)
            for kind in ("U", "W", "X"):
                for (bt, bs) in Ls[kind]:
                    tm = tsrc[T.points(*bt)]
                    sm = S.points(*bs)
                    for t in types:
                        st = sm[ityp[sm] == t]
                        if not len(st):
                            continue
                        srcs, qs = xyz[isrc[st]], q[isrc[st]]
                        for i in tm:
                            ph, f = rules[t].sum_at(md, xyz[i], srcs, qs)
                            phi[i] += ph
                            field[i] += f
    return phi, field
