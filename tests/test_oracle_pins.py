"""Pins of the oracle against what the paper and the mathematics fix (no GPU needed).

Each test names the pin it is and the passage it follows.  The oracle is test
infrastructure; these tests make sure a plausible mistake in it (a dropped term, a wrong
sign or index, a transposed operand) fails somewhere.

Parity status of the oracle's functions:
  layer_response  pinned: paper's printed 3-layer densities (Sec. 2.1), homogeneous medium,
                  two half-spaces closed form.
  green_react     pinned: homogeneous medium (P6), two half-spaces images (P7), reciprocity (P8),
                  finite differences of the field; each component agrees with a second,
                  independent quadrature (scipy) and with the limit of its truncated ME/LE
                  (tests/test_expansion_pins.py).
  direct          pinned: equals the sum of green_react / closed forms; reciprocity of the
                  assembled potential.
  S_table         pinned: Sommerfeld identity closed forms for K=1,d=0 and K=2,d=1 in a
                  homogeneous medium; Bessel three-term recurrence invariant; zero for rho=0,d>0.
  image_z         pinned: the paper's printed example coordinates (Sec. 3.4).
  tree/lists      pinned: brute force over integer box coordinates.
"""
import json
import os

import numpy as np
import pytest

import oracle
from paper_2002_01334_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def paper_sigma3(lr, d, eps, lam):
    """The 3-layer reaction densities as printed in Sec. 2.1 (eqs. densitythreelayer1-3), with
    d_0 = 0, exp(-d_1 lz_1) read literally (d_1 < 0), sigma_10^11's "lambda_1 lambda_1z" read as
    eps_1 lambda_1z and sigma_11^21's "+eps_0 lambda_0z" read as "-eps_0 lambda_0z"."""
    e0, e1, e2 = eps
    l0, l1, l2 = np.sqrt(np.asarray(lam) ** 2 + lr * lr)
    d1 = d[1]
    ch, sh, ex = np.cosh(-d1 * l1), np.sinh(-d1 * l1), np.exp(-d1 * l1)
    kap = e1 * l1 * (e0 * l0 + e2 * l2) * ch + (e1 ** 2 * l1 ** 2 + e0 * e2 * l0 * l2) * sh
    S = {}
    S[(0, 0, 1, 1)] = (e1 * l1 * (e0 * l0 - e2 * l2) * ch - (e1 ** 2 * l1 ** 2 - e0 * e2 * l0 * l2) * sh) / (e0 * kap)
    S[(1, 0, 1, 1)] = e0 * l1 * (e1 * l1 - e2 * l2) / (e0 * kap)
    S[(1, 0, 2, 1)] = e0 * l1 * (e1 * l1 + e2 * l2) * ex / (e0 * kap)
    S[(2, 0, 2, 1)] = 2 * e0 * e1 * l1 * l2 / (e0 * kap)
    S[(0, 1, 1, 1)] = e1 * l0 * (e1 * l1 - e2 * l2) / (e1 * kap)
    S[(0, 1, 1, 2)] = e1 * l0 * (e1 * l1 + e2 * l2) * ex / (e1 * kap)
    S[(1, 1, 1, 1)] = (e1 * l1 - e2 * l2) * (e1 * l1 + e0 * l0) * ex / (2 * e1 * kap)
    S[(1, 1, 1, 2)] = (e1 * l1 - e2 * l2) * (e1 * l1 - e0 * l0) / (2 * e1 * kap)
    S[(1, 1, 2, 1)] = (e1 * l1 - e2 * l2) * (e1 * l1 - e0 * l0) / (2 * e1 * kap)
    S[(1, 1, 2, 2)] = (e1 * l1 + e2 * l2) * (e1 * l1 - e0 * l0) * ex / (2 * e1 * kap)
    S[(2, 1, 2, 1)] = e1 * l2 * (e0 * l0 + e1 * l1) * ex / (e1 * kap)
    S[(2, 1, 2, 2)] = e1 * l2 * (e1 * l1 - e0 * l0) / (e1 * kap)
    S[(0, 2, 1, 2)] = 2 * e1 * l1 * e2 * l0 / (e2 * kap)
    S[(1, 2, 2, 2)] = e2 * l1 * (e1 * l1 - e0 * l0) / (e2 * kap)
    S[(1, 2, 1, 2)] = e2 * l1 * (e0 * l0 + e1 * l1) * ex / (e2 * kap)
    S[(2, 2, 2, 2)] = (e1 * l1 * (e2 * l2 - e0 * l0) * ch - (e1 ** 2 * l1 ** 2 - e0 * e2 * l0 * l2) * sh) / (e2 * kap)
    return S


@pytest.mark.parametrize("medium", ["three_layer", "paper_three_layer"])
@pytest.mark.parametrize("lr", [0.0, 0.37, 1.9, 7.5])
def test_P1_three_layer_densities_match_paper(medium, lr):
    m = inputs.MEDIA[medium]
    md = oracle.Medium(**m)
    for (l, lp, a, b), v in paper_sigma3(lr, m["d"], m["eps"], m["lam"]).items():
        got = oracle.sigma(md, lr, l, lp, a, b)
        assert abs(got - v) <= 1e-13 * max(1.0, abs(v)), (l, lp, a, b, got, v)


def test_P1_printed_sigma11_21_sign_is_a_typo():
    """Reciprocity fixes sigma_11^21 = sigma_11^12; the printed '+eps_0 lambda_0z' breaks it."""
    m = inputs.MEDIA["three_layer"]
    md = oracle.Medium(**m)
    lr = 0.8
    l0, l1, l2 = np.sqrt(np.asarray(m["lam"]) ** 2 + lr * lr)
    e0, e1, e2 = m["eps"]
    printed = paper_sigma3(lr, m["d"], m["eps"], m["lam"])[(1, 1, 2, 1)] / (e1 * l1 - e0 * l0) * (e1 * l1 + e0 * l0)
    assert abs(oracle.sigma(md, lr, 1, 1, 2, 1) - printed) > 1e-3
    assert abs(oracle.sigma(md, lr, 1, 1, 2, 1) - oracle.sigma(md, lr, 1, 1, 1, 2)) < 1e-15


def free(r, rp, lam, eps):
    R = np.linalg.norm(np.subtract(r, rp))
    phi = np.exp(-lam * R) / (4 * np.pi * eps * R)
    field = phi * (1 + lam * R) / R ** 2 * np.subtract(r, rp)
    return phi, field


def test_P6_homogeneous_medium():
    """All layers share eps, lambda: same-layer reaction vanishes, cross-layer reaction is the
    whole free-space kernel (Sec. 2.1 eq. layeredGreensfun)."""
    md = oracle.Medium([0.0, -1.0], [3.0, 3.0, 3.0], [0.7, 0.7, 0.7])
    r = np.array([0.1, 0.2, -0.4])
    for rp, lp in [([0.3, -0.1, -0.7], 1), ([0.0, 0.1, 0.6], 0), ([-0.2, 0.4, -1.5], 2)]:
        g, f = oracle.green_react(md, 1, r, lp, rp)
        if lp == 1:
            assert abs(g) < 1e-14 and np.abs(f).max() < 1e-13
        else:
            g0, f0 = free(r, rp, 0.7, 3.0)
            assert abs(g - g0) < 1e-12 * abs(g0)
            assert np.abs(f - f0).max() < 1e-11 * np.abs(f0).max()


@pytest.mark.parametrize("lam", [0.7, 1e-8])
def test_P7_two_half_spaces_image_charge(lam):
    """Two half-spaces with equal lambda: reflected part R e^{-lam r*}/(4 pi eps0 r*) at the
    mirror image, R = (eps0-eps1)/(eps0+eps1); transmitted 2 e^{-lam r}/(4 pi (eps0+eps1) r)."""
    e0, e1 = 2.0, 7.0
    md = oracle.Medium([0.0], [e0, e1], [lam, lam])
    rp = np.array([0.1, -0.2, 0.35])
    for r in ([0.4, 0.3, 0.6], [-0.3, 0.1, 0.15]):
        mirror = rp * [1, 1, -1]
        g, f = oracle.green_react(md, 0, r, 0, rp)
        g0, f0 = free(r, mirror, lam, e0)
        Rc = (e0 - e1) / (e0 + e1)
        assert abs(g - Rc * g0) < 1e-11 * abs(g0)
        assert np.abs(f - Rc * f0).max() < 1e-10 * np.abs(f0).max()
    r = np.array([0.2, -0.5, -0.45])
    g, f = oracle.green_react(md, 1, r, 0, rp)
    g0, f0 = free(r, rp, lam, 1.0)
    assert abs(g - 2 * g0 / (e0 + e1)) < 1e-11 * abs(g0)
    assert np.abs(f - 2 * f0 / (e0 + e1)).max() < 1e-10 * np.abs(f0).max()


def test_P7_unequal_lambda_limit_to_laplace():
    """lambda_0 != lambda_1 -> 0 tends to the Laplace image formula."""
    e0, e1 = 1.0, 4.0
    rp = np.array([0.0, 0.0, 0.3])
    r = np.array([0.2, 0.1, 0.5])
    Rlap = (e0 - e1) / (e0 + e1) / (4 * np.pi * e0 * np.linalg.norm(r - rp * [1, 1, -1]))
    errs = []
    for s in (1e-2, 1e-3, 1e-4):
        md = oracle.Medium([0.0], [e0, e1], [s, 2 * s])
        g, _ = oracle.green_react(md, 0, r, 0, rp)
        errs.append(abs(g - Rlap))
    assert errs[2] < errs[1] < errs[0] and errs[2] < 1e-4 * abs(Rlap)


@pytest.mark.parametrize("medium", ["three_layer", "four_layer"])
def test_P8_reciprocity(medium):
    m = inputs.MEDIA[medium]
    md = oracle.Medium(**m)
    rng = np.random.default_rng(5)
    boxes = inputs.THREE_LAYER_BOXES if medium == "three_layer" else inputs.FOUR_LAYER_BOXES
    for _ in range(6):
        l, lp = rng.integers(0, md.L + 1, 2)
        r = np.r_[rng.uniform(-0.5, 0.5, 2), rng.uniform(*boxes[l])]
        rp = np.r_[rng.uniform(-0.5, 0.5, 2), rng.uniform(*boxes[lp])]
        g1, _ = oracle.green_react(md, l, r, lp, rp)
        g2, _ = oracle.green_react(md, lp, rp, l, r)
        assert abs(g1 - g2) < 1e-12 * max(abs(g1), 1e-6), (l, lp, g1, g2)


def test_field_is_minus_gradient():
    md = oracle.Medium(**inputs.MEDIA["four_layer"])
    r = np.array([0.1, -0.2, -1.3])
    rp = np.array([-0.3, 0.25, -0.6])
    g, f = oracle.green_react(md, 2, r, 1, rp)
    h = 1e-5
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        gp, _ = oracle.green_react(md, 2, r + e, 1, rp)
        gm, _ = oracle.green_react(md, 2, r - e, 1, rp)
        assert abs(-(gp - gm) / (2 * h) - f[k]) < 1e-8 * np.abs(f).max()


def _scipy_component(md, l, r, lp, rp, a, b):
    """u^{ab}_{l l'}(r, r') and -grad_r of eq. generalcomponents (Sec. 2.2) after the alpha
    integral, by scipy's QUADPACK on [0, X]: (1/4 pi) int lr J0(lr rho) e^{-lz h - lz' h'}
    sigma / lz d lr, with h, h' the exponents' distances of eq. zexponential."""
    from scipy import integrate, special
    d = md.d
    h = r[2] - d[l] if a == 1 else d[l - 1] - r[2]
    hp = rp[2] - d[lp] if b == 1 else d[lp - 1] - rp[2]
    dx, dy = r[0] - rp[0], r[1] - rp[1]
    rho = np.hypot(dx, dy)
    X = 80.0 / (h + hp)
    pts = list(np.arange(np.pi / rho, X, np.pi / rho)) if rho > 0 else None

    def g(lr, k):
        lz = np.hypot(md.lam[l], lr)
        lzp = np.hypot(md.lam[lp], lr)
        e = np.exp(-lz * h - lzp * hp) * oracle.sigma(md, lr, l, lp, a, b) / lz / (4 * np.pi)
        if k == 0:
            return lr * special.j0(lr * rho) * e
        if k == 1:  # -d/dx and -d/dy share lr^2 J1(lr rho) / rho
            return lr * lr * (special.j1(lr * rho) / rho if rho > 0 else 0.5 * lr) * e
        return lr * special.j0(lr * rho) * e * lz * (1.0 if a == 1 else -1.0)

    v = [integrate.quad(g, 0.0, X, args=(k,), points=pts, limit=4000, epsabs=0.0, epsrel=1e-13)[0]
         for k in range(3)]
    return v[0], np.array([dx * v[1], dy * v[1], v[2]])


@pytest.mark.parametrize("medium", ["three_layer", "four_layer"])
def test_green_react_ab_agrees_with_a_second_quadrature(medium):
    """Two independent quadratures of the same component integral (the oracle's adaptive
    Gauss-Kronrod in C, scipy's QUADPACK here) agree for every component type."""
    m = inputs.MEDIA[medium]
    md = oracle.Medium(m["d"], m["eps"], m["lam"])
    rng = np.random.default_rng(11)
    L = md.L
    mids = [md.d[0] + 0.6] + [0.5 * (md.d[k - 1] + md.d[k]) for k in range(1, L)] + [md.d[L - 1] - 0.6]
    for l in range(L + 1):
        for lp in range(L + 1):
            for a in ((1,) if l == 0 else (2,) if l == L else (1, 2)):
                for b in ((1,) if lp == 0 else (2,) if lp == L else (1, 2)):
                    r = np.array([*rng.uniform(-0.4, 0.4, 2), mids[l] + rng.uniform(-0.1, 0.1)])
                    rp = np.array([*rng.uniform(-0.4, 0.4, 2), mids[lp] + rng.uniform(-0.1, 0.1)])
                    u, f = oracle.green_react_ab(md, l, r, lp, rp, a, b)
                    us, fs = _scipy_component(md, l, r, lp, rp, a, b)
                    assert abs(u - us) <= 1e-11 * abs(us), (l, lp, a, b, u, us)
                    assert np.abs(f - fs).max() <= 1e-10 * np.abs(fs).max(), (l, lp, a, b, f, fs)


def test_direct_matches_pairwise_definition():
    """The batched fixed-rule direct sum equals the per-pair adaptive definition."""
    w = inputs.workload("three_layer", n=30, seed=11)
    md = oracle.Medium(**w["medium"])
    phi, field = oracle.direct(md, w["q"], w["xyz"], w["layer"])
    for i in (0, 7, 29):
        acc = 0.0
        fac = np.zeros(3)
        for j in range(30):
            g, f = oracle.green_react(md, w["layer"][i], w["xyz"][i], w["layer"][j], w["xyz"][j])
            acc += w["q"][j] * g
            fac += w["q"][j] * f
            if j != i and w["layer"][j] == w["layer"][i]:
                lam, eps = md.lam[w["layer"][i]], md.eps[w["layer"][i]]
                g0, f0 = free(w["xyz"][i], w["xyz"][j], lam, eps)
                acc += w["q"][j] * g0
                fac += w["q"][j] * f0
        assert abs(phi[i] - acc) < 1e-11 * np.abs(phi).max()
        assert np.abs(field[i] - fac).max() < 1e-10 * np.abs(field).max()


def test_direct_reciprocity_of_assembled_potential():
    """sum_i q'_i phi_i[q] = sum_i q_i phi_i[q'] (symmetric Green's function)."""
    w = inputs.workload("four_layer", n=40, seed=3)
    md = oracle.Medium(**w["medium"])
    q2 = inputs.uniform(99, 40) - 0.5
    p1, _ = oracle.direct(md, w["q"], w["xyz"], w["layer"])
    p2, _ = oracle.direct(md, q2, w["xyz"], w["layer"])
    a, b = np.dot(q2, p1), np.dot(w["q"], p2)
    assert abs(a - b) < 1e-12 * max(abs(a), abs(b))


def test_S_table_closed_forms_homogeneous():
    """Homogeneous 2-half-space medium, cross-layer component (l=1 target, l'=0 source, a=2, b=1):
    sigma = 1/eps, so S^1 S_{1 0,00} = e^{-lam R}/(eps R) (Sommerfeld identity, Sec. 3.2) and
    S^2 S_{2 1,00} = h^2/sqrt(6) (rho/R)(1+lam R) e^{-lam R}/(eps R^2)."""
    lam, eps = 0.6, 2.5
    md = oracle.Medium([0.0], [eps, eps], [lam, lam])
    h, rho, zt, zs = 0.7, 1.3, 0.4, 0.5
    S = oracle.S_table(md, 1, 0, 2, 1, h, rho, zt, zs, 3)
    R = np.hypot(rho, zt + zs)
    v10 = h * np.exp(-lam * R) / (eps * R)
    v21 = h * h / np.sqrt(6.0) * (rho / R) * (1 + lam * R) * np.exp(-lam * R) / (eps * R * R)
    assert abs(S[1, 0, 0, 0] - v10) < 1e-12 * abs(v10)
    assert abs(S[2, 1, 0, 0] - v21) < 1e-12 * abs(v21)


def test_S_table_bessel_recurrence_and_rho_zero():
    """The definition obeys the three-term recurrence of Sec. 3.5 (eq. recurrence1) exactly,
    and vanishes for rho = 0, d > 0."""
    md = oracle.Medium(**inputs.MEDIA["three_layer"])
    h = 0.3
    Kmax = 9
    S = oracle.S_table(md, 1, 2, 1, 2, h, 2.2 * h, 1.5 * h, 0.5 * h, Kmax)
    a = lambda n: np.sqrt(n * (n + 1.0))
    rho = 2.2 * h
    worst = 0.0
    for d in range(1, Kmax - 1):
        for K in range(d + 2, Kmax + 1):
            rhs = 2 * d / a(K + d) * (h / rho) * S[K - 1, d] - a(K - d) / a(K + d) * S[K, d - 1]
            scale = np.abs(S[K]).max()
            worst = max(worst, np.abs(S[K, d + 1] - rhs).max() / scale)
    assert worst < 1e-10
    S0 = oracle.S_table(md, 1, 2, 1, 2, h, 0.0, 1.5 * h, 0.5 * h, 5)
    assert np.abs(S0[:, 1:]).max() == 0.0 and np.abs(S0[3, 0]).max() > 0


def test_image_coordinates_match_paper_example():
    g = json.load(open(os.path.join(GOLD, "paper_me_example.json")))
    md = oracle.Medium(g["d"], g["eps"], g["lam"])
    zp = g["source"][2]
    assert abs(oracle.image_z(md, 1, 1, 1, 1, zp) - g["image_11"][2]) < 1e-14
    assert abs(oracle.image_z(md, 1, 2, 1, 2, zp) - g["image_22"][2]) < 1e-14
    for key in ("11", "22"):
        dist = np.linalg.norm(np.subtract(g["image_" + key], g["center_" + key]))
        assert abs(dist - g["image_center_distance"]) < 5e-5


def test_images_across_interface_from_targets():
    """Images of group (l, a) lie beyond the interface from the targets (Sec. 3.3, Remark 1)."""
    m = inputs.MEDIA["four_layer"]
    md = oracle.Medium(**m)
    rng = np.random.default_rng(2)
    for _ in range(50):
        l = int(rng.integers(0, 4))
        lp = int(rng.integers(0, 4))
        zp = rng.uniform(*inputs.FOUR_LAYER_BOXES[lp])
        for a in (1, 2):
            if (a == 1 and l == 3) or (a == 2 and l == 0):
                continue
            for b in (1, 2):
                if (b == 1 and lp == 3) or (b == 2 and lp == 0):
                    continue
                zi = oracle.image_z(md, l, a, lp, b, zp)
                if a == 1:
                    assert zi < m["d"][l]
                else:
                    assert zi > m["d"][l - 1]


def brute_lists(tcoords, scoords, lev, kind, ws=1):
    sset = {tuple(c): i for i, c in enumerate(scoords)}
    R = 2 * ws + 1
    out = []
    for t in tcoords:
        row = []
        for dx in range(-R, R + 1):
            for dy in range(-R, R + 1):
                for dz in range(-R, R + 1):
                    s = (t[0] + dx, t[1] + dy, t[2] + dz)
                    if s not in sset:
                        continue
                    cheb = max(abs(dx), abs(dy), abs(dz))
                    if kind == 1:
                        ok = cheb <= ws
                    else:
                        ok = cheb > ws and all(abs((s[k] >> 1) - (t[k] >> 1)) <= ws for k in range(3))
                    if ok:
                        row.append(sset[s])
        out.append(row)
    return out


def coords_of(boxes):
    out = []
    for key in boxes:
        key = int(key)
        x = y = z = 0
        for k in range(21):
            z |= ((key >> (3 * k)) & 1) << k
            y |= ((key >> (3 * k + 1)) & 1) << k
            x |= ((key >> (3 * k + 2)) & 1) << k
        out.append((x, y, z))
    return out


def test_tree_keys_and_lists_brute_force():
    w = inputs.workload("three_layer", n=600, seed=7)
    md = oracle.Medium(**w["medium"])
    l, a, D = 1, 2, 4
    root = oracle.tree_root(md, w["xyz"], w["layer"], l, a)
    assert root[2] == md.d[0]
    tk, tsrc, _ = oracle.tree_keys(md, w["xyz"], w["layer"], l, a, D, root, 0)
    ik, isrc, ityp = oracle.tree_keys(md, w["xyz"], w["layer"], l, a, D, root, 1)
    assert len(tk) == 200 and len(ik) == 200 + 2 * 200 + 200
    # keys from an independent float computation of the cells
    H = root[3]
    for k, j in zip(tk[:50], tsrc[:50]):
        c = [int(np.floor((w["xyz"][j][t] - (root[t] - H)) * ((1 << D) / (2 * H)))) for t in range(3)]
        assert int(k) == int(oracle.morton(*c))
    # targets below, images above the bisecting interface: z-cells on either side of 2^(D-1)
    tz = [c[2] for c in coords_of(tk)]
    iz = [c[2] for c in coords_of(ik)]
    assert max(tz) < (1 << (D - 1)) <= min(iz)
    for ws in (1, 2):
        for lev in (2, 3, 4):
            tb = oracle.level_boxes(tk, D, lev)
            sb = oracle.level_boxes(ik, D, lev)
            for kind in (0, 1):
                off, idx = oracle.lists(tb, sb, lev, kind, ws)
                ref = brute_lists(coords_of(tb), coords_of(sb), lev, kind, ws)
                got = [list(idx[off[t]:off[t + 1]]) for t in range(len(tb))]
                assert got == ref


@pytest.mark.parametrize("ws", [1, 2])
def test_lists_cover_every_leaf_pair_once(ws):
    """With separation ws, every (target leaf, source leaf) pair of a uniform tree is handled exactly
    once: by the near list at the leaf level, or by the far list of exactly one pair of ancestors
    (the partition property the FMM's correctness rests on).  Brute force over random boxes."""
    rng = np.random.default_rng(11 + ws)
    D = 4
    n = 1 << D
    tc = {tuple(c) for c in rng.integers(0, n, size=(150, 3)).tolist()}
    sc = {tuple(c) for c in rng.integers(0, n, size=(150, 3)).tolist()}
    key = lambda c, lev: int(oracle.morton(c[0] >> (D - lev), c[1] >> (D - lev), c[2] >> (D - lev)))
    boxes = {}
    for lev in range(2, D + 1):
        boxes[lev] = (np.array(sorted({key(c, lev) for c in tc}), np.uint64),
                      np.array(sorted({key(c, lev) for c in sc}), np.uint64))
    hits = {}
    for lev in range(2, D + 1):
        tb, sb = boxes[lev]
        kinds = (0, 1) if lev == D else (0,)
        for kind in kinds:
            off, idx = oracle.lists(tb, sb, lev, kind, ws)
            for t in range(len(tb)):
                for s in idx[off[t]:off[t + 1]]:
                    hits.setdefault((lev, int(tb[t]), int(sb[s])), 0)
                    hits[(lev, int(tb[t]), int(sb[s]))] += 1
    assert max(hits.values()) == 1
    for t in tc:
        for s in sc:
            cover = sum((lev, key(t, lev), key(s, lev)) in hits for lev in range(2, D + 1))
            assert cover == 1, (t, s, cover)


def test_sommerfeld_recurrences_where_each_holds():
    """Sec. 3.5: the forward recurrence (eq. recurrence1) from exact columns d = 0, 1 and the
    backward recurrence (eq. backwardrecurrence1) from the exact top row and column d = 0,
    against direct quadrature of every entry (oracle.S_table), relative to each row's largest
    entry the operators use.  Backward holds for small rho/S, forward for large; forward at
    rho = S loses everything by K = 21, although the paper states it stable for rho >= S."""
    from oracle import expansions as E
    md = oracle.Medium([0.0, -1.2], [1.0, 2.0, 5.0], [0.5, 1.0, 0.8])
    h, K = 0.3, 21

    def errs(r2, kt, ks):
        r = np.sqrt(r2)
        D = oracle.S_table(md, 1, 1, 1, 2, h, r * h, (kt + 0.5) * h, (ks + 0.5) * h, K)
        F, B = E.forward_recurrence(D, r), E.backward_recurrence(D, r)
        ef = eb = 0.0
        for n in range(2, K + 1):
            used = [d for d in range(n + 1) if (n - d) % 2 == 1]
            rm = np.abs(D[n, used]).max()
            uf, ub = [d for d in used if d >= 2], [d for d in used if d >= 1]
            ef = max(ef, np.abs(F[n, uf] - D[n, uf]).max(initial=0) / rm)
            eb = max(eb, np.abs(B[n, ub] - D[n, ub]).max(initial=0) / rm)
        return ef, eb

    for r2, kt, ks in [(1, 1, 1), (2, 0, 1), (0.09, 0, 0)]:
        ef, eb = errs(r2, kt, ks)
        assert eb < 1e-12, (r2, eb)
    assert errs(1, 1, 1)[0] > 1e-2
    for r2, kt, ks in [(13, 0, 0), (18, 1, 1)]:
        ef, eb = errs(r2, kt, ks)
        assert ef < 1e-9, (r2, ef)
