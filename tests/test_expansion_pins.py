"""CPU pins: the truncated expansions of Sec. 3 converge in p to the oracle's direct values.

The expansions (oracle/expansions.py) and the oracle's direct reaction components
(oracle.green_react_ab, adaptive quadrature of the alpha-integrated Sommerfeld integral of
Sec. 2.2) are independent routes to the same numbers.  So agreement pins both: the oracle's
u^{ab} against the limit of the paper's ME/LE/M2L (Sec. 3.4), and the expansion formulas (their
signs, the Legendre continuation of Prop. 1-2, the Bessel alpha-integrals) against the
closed-form kernel and the oracle.  The ME case is the paper's single-source example of Sec. 3.4
(three-layer medium eps = (1, 8.6, 20.5), lambda = (1.2, 0.5, 2.1), d = (0, -1.2)), which the
paper shows only as a figure; tests/golden/me_convergence_e1.json holds the table.
"""
import json
import math
import os

import numpy as np
import pytest

pytest.importorskip("scipy")

from scipy import special  # noqa: E402

import oracle  # noqa: E402
from oracle import expansions as E  # noqa: E402

HERE = os.path.dirname(os.path.abspath(__file__))

# Sec. 3.4 example: source r' in the middle layer, two components, two ME centres, three targets
E1_MEDIUM = dict(d=[0.0, -1.2], eps=[1.0, 8.6, 20.5], lam=[1.2, 0.5, 2.1])
E1_SOURCE = np.array([0.625, 0.5, -0.1])
E1_CENTRES = {(1, 1): np.array([0.6, 0.6, -2.4]), (2, 2): np.array([0.6, 0.6, 0.2])}
E1_TARGETS = [np.array([0.5, 0.625, z]) for z in (-0.1, -0.6, -1.1)]


def e1_medium():
    return oracle.Medium(**E1_MEDIUM)


def image(md, l, a, lp, b, rp):
    return np.array([rp[0], rp[1], oracle.image_z(md, l, a, lp, b, rp[2])])


def test_spherical_harmonics_match_scipy():
    """Y_n^m of Sec. 3.1 (with its (-1)^m in front) equals scipy's Condon-Shortley harmonics."""
    if not hasattr(special, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    rng = np.random.default_rng(3)
    th = rng.uniform(0, math.pi, 7)
    ph = rng.uniform(-math.pi, math.pi, 7)
    for n in range(11):
        for m in range(-n, n + 1):
            assert np.abs(E.ylm(n, m, th, ph) - special.sph_harm_y(n, m, th, ph)).max() < 1e-13


def test_phat_all_equals_phat():
    for x in (-0.7, 0.0, 0.31, 1.0, 1.7, 23.0):
        v = E.phat_all(9, x)
        w = np.array([E.phat(n, m, x) for n, m in E._nm(9)])
        assert np.abs(v - w).max() <= 1e-13 * max(1.0, np.abs(w).max())


@pytest.mark.parametrize("lam,lr,alpha", [(0.5, 0.3, 0.7), (1.3, 4.0, 2.1), (0.8, 12.0, -1.0)])
def test_prop2_plane_wave_series_with_the_branch_of_prop1(lam, lr, alpha):
    """Prop. 2: e^{Lambda.r} = sum conj(B_n^m(r)) phat_n^m(lz/lam) e^{i m alpha} for
    lz/lam > 1, with the square-root branch of Prop. 1."""
    r = np.array([0.21, -0.17, 0.26])
    exact = E.plane_wave(lam, lr, alpha, r)
    s = E.plane_wave_series(lam, lr, alpha, r, 40)
    assert abs(s[-1] - exact) < 1e-12 * abs(exact)


def test_prop2_fails_with_the_other_branch(monkeypatch):
    """Planted mistake: the opposite square-root branch for x > 1 breaks Prop. 2."""
    orig = E.phat

    def flipped(n, m, x):
        v = orig(n, m, x)
        return np.where(np.asarray(x) > 1.0, v * (-1.0) ** abs(m), v)

    monkeypatch.setattr(E, "phat", flipped)
    r = np.array([0.21, -0.17, 0.26])
    exact = E.plane_wave(1.3, 4.0, 2.1, r)
    s = E.plane_wave_series(1.3, 4.0, 2.1, r, 40)
    assert abs(s[-1] - exact) > 1e-3 * abs(exact)


def test_free_space_addition_theorem_me_and_le():
    """Thm. 1 and the free-space ME/LE of Sec. 3.1 converge to k_0(lambda|r - r'|) at the rate
    (inner radius / outer radius)^{p+1}."""
    lam = 0.9
    r1 = np.array([0.1, -0.2, 0.15])
    b = np.array([0.6, 0.3, -0.7])
    ex = E.k0(lam, np.linalg.norm(r1 + b))
    s = E.addition_k0(lam, r1, b, 24)
    rate = np.linalg.norm(r1) / np.linalg.norm(b)
    err = np.abs(s - ex) / ex
    assert err[-1] < 1e-13 and all(err[p] <= 4 * rate ** (p + 1) + 1e-15 for p in range(25))

    rs, rc, r = np.array([0.55, 0.45, 0.5]), np.array([0.5, 0.5, 0.5]), np.array([-0.2, 0.9, 0.1])
    ex = E.k0(lam, np.linalg.norm(r - rs))
    rate = np.linalg.norm(rs - rc) / np.linalg.norm(r - rc)
    for s in (E.free_me(lam, rs, rc, r, 20), E.free_le(lam, r, rc, rs, 20)):
        err = np.abs(s - ex) / ex
        assert err[-1] < 1e-14 and all(err[p] <= 4 * rate ** (p + 1) + 1e-15 for p in range(21))


def test_image_coordinates_of_the_me_example():
    """The polarization coordinates the Sec. 3.4 example prints, and its source-centre distance."""
    md = e1_medium()
    assert np.allclose(image(md, 1, 1, 1, 1, E1_SOURCE), [0.625, 0.5, -2.3], atol=1e-15)
    assert np.allclose(image(md, 1, 2, 1, 2, E1_SOURCE), [0.625, 0.5, 0.1], atol=1e-15)
    for ab, rc in E1_CENTRES.items():
        assert abs(np.linalg.norm(image(md, 1, ab[0], 1, ab[1], E1_SOURCE) - rc) - 0.1436) < 1e-4


@pytest.mark.parametrize("ab", [(1, 1), (2, 2)])
def test_reaction_me_converges_to_the_oracle_component(ab):
    """Sec. 3.4 example: the ME (eqs. melayerupgoingimage, mebasis) of u~^{ab}_{11} about the
    polarization centre converges to the oracle's u^{ab}_{11} at the reference rate
    (|r'_ab - r_c| / |r - r_c|)^{p+1} (the rate the paper plots, read with the ratio inverted)."""
    md = e1_medium()
    a, b = ab
    rc = E1_CENTRES[ab]
    rimg = image(md, 1, a, 1, b, E1_SOURCE)
    for r in E1_TARGETS:
        u, _ = oracle.green_react_ab(md, 1, r, 1, E1_SOURCE, a, b)
        s = E.reaction_me(md, 1, 1, a, b, r, rimg, rc, 24)
        err = np.abs(s - u) / abs(u)
        rate = np.linalg.norm(rimg - rc) / np.linalg.norm(r - rc)
        assert all(err[p] <= 4 * rate ** (p + 1) + 2e-15 for p in range(25)), (r, err)
        assert err[-1] < max(1e-14, 10 * rate ** 25), (r, err[-1])


@pytest.mark.parametrize("ab", [(1, 1), (1, 2), (2, 1), (2, 2)])
def test_reaction_le_and_m2l_converge_to_the_oracle_component(ab):
    """LE (eqs. lelayerimage, lecoeffimage) about a target centre, and M2L (eqs. metoleimage1,
    metoleimage2) from an ME centre: the LE sum converges to u^{ab}; T.M with nu <= P converges
    to the LE coefficients of eq. lecoeffimage as P grows, and M2L + LE reaches u^{ab}."""
    md = e1_medium()
    a, b = ab
    rimg = image(md, 1, a, 1, b, E1_SOURCE)
    rcs = rimg + np.array([-0.03, 0.08, 0.06 if a == 1 else -0.06])
    r = np.array([0.5, 0.625, -0.6])
    rct = r + np.array([0.07, -0.05, 0.04])
    u, _ = oracle.green_react_ab(md, 1, r, 1, E1_SOURCE, a, b)
    s = E.reaction_le(md, 1, 1, a, b, r, rimg, rct, 18)
    assert abs(s[-1] - u) < 1e-13 * abs(u)
    p = 10
    Ld = E.reaction_le_coeffs(md, 1, 1, a, b, rimg, rct, p)
    cerr = []
    for P in (4, 8, 12):
        L = E.reaction_m2l(md, 1, 1, a, b, rct, rcs, p, P) @ E.me_coeffs(md.lam[1], rimg, rcs, P)
        cerr.append(np.abs(L - Ld).max() / np.abs(Ld).max())
    assert cerr[0] > 10 * cerr[1] > 100 * cerr[2], cerr
    v = E.le_eval(md.lam[1], L, rct, r, p)[-1]
    assert abs(v - u) < 1e-9 * abs(u)


def test_reaction_me_catches_planted_sign_errors(monkeypatch):
    """Planted mistakes in the expansion (the Prop. 1 branch; the 2b sign (-1)^{n+m} of eq.
    mebasis) move the ME away from the oracle's component."""
    md = e1_medium()
    r = E1_TARGETS[1]
    u, _ = oracle.green_react_ab(md, 1, r, 1, E1_SOURCE, 2, 2)
    rimg = image(md, 1, 2, 1, 2, E1_SOURCE)
    good = E.reaction_me(md, 1, 1, 2, 2, r, rimg, E1_CENTRES[(2, 2)], 16)[-1]
    assert abs(good - u) < 1e-12 * abs(u)
    orig = E.phat_all
    _, am, _ = E._phat_table(16)
    monkeypatch.setattr(E, "phat_all", lambda p, x: orig(p, x) * ((-1.0) ** am if x > 1 else 1.0))
    bad = E.reaction_me(md, 1, 1, 2, 2, r, rimg, E1_CENTRES[(2, 2)], 16)[-1]
    assert abs(bad - u) > 1e-3 * abs(u)
    monkeypatch.setattr(E, "phat_all", orig)
    monkeypatch.setattr(E, "_me_sign", lambda a, n, m: 1.0)
    bad = E.reaction_me(md, 1, 1, 2, 2, r, rimg, E1_CENTRES[(2, 2)], 16)[-1]
    assert abs(bad - u) > 1e-3 * abs(u)


def test_me_convergence_fixture_matches_the_oracle():
    """tests/golden/me_convergence_e1.json (written by make_me_convergence.py from oracle/ only)
    is what the oracle and the expansions give now."""
    with open(os.path.join(HERE, "golden", "me_convergence_e1.json")) as f:
        fx = json.load(f)
    md = oracle.Medium(**fx["medium"])
    for row in fx["rows"]:
        a, b = row["component"]
        rimg = image(md, 1, a, 1, b, np.array(fx["source"]))
        u, _ = oracle.green_react_ab(md, 1, np.array(row["target"]), 1, np.array(fx["source"]), a, b)
        assert abs(u - row["u"]) <= 1e-14 * abs(u)
        s = E.reaction_me(md, 1, 1, a, b, row["target"], rimg, np.array(row["centre"]), fx["pmax"])
        err = np.abs(s - u) / abs(u)
        assert np.abs(err - np.array(row["rel_err"])).max() < 1e-13


@pytest.mark.parametrize("n,m,nu,mu,lam,lamp", [(3, 1, 2, -2, 0.5, 1.2), (7, -4, 6, 3, 0.8, 0.8),
                                                (10, 0, 9, 9, 2.1, 0.5), (10, 7, 10, -10, 1.0, 0.3)])
def test_legendre_product_as_polynomial_in_lambda_rho(n, m, nu, mu, lam, lamp):
    """Sec. 3.5: phat_n^m(lz/lam) phat_nu^mu(lz'/lam') = sum_s C^s lr^{|m|+|mu|+2s}
    (lam/lz)^i (lam'/lz')^j with i, j the parities of n + |m|, nu + |mu|."""
    i, j, C = E.legendre_product_coeffs(n, m, nu, mu, lam, lamp)
    assert (i, j) == ((n + abs(m)) % 2, (nu + abs(mu)) % 2)
    for lr in (0.01, 0.7, 3.3, 12.0):
        lz, lzp = math.hypot(lam, lr), math.hypot(lamp, lr)
        ex = E.phat(n, m, lz / lam) * E.phat(nu, mu, lzp / lamp)
        v = sum(Cs * lr ** (abs(m) + abs(mu) + 2 * s) for s, Cs in enumerate(C)) * (lam / lz) ** i * (lamp / lzp) ** j
        assert abs(v - ex) <= 1e-10 * abs(ex)


@pytest.mark.parametrize("ab", [(1, 1), (1, 2), (2, 1), (2, 2)])
def test_m2l_table_route_matches_direct_quadrature(ab):
    """The M2L operator by the table route of Sec. 3.5 (eqs. coefintable, metoletableform with the
    oracle's S-tables of eq. M2Ltable, reading the garbled symbol in C~ as a factorial) equals the
    operator by direct quadrature of eq. metoleimage2, entry by entry."""
    md = e1_medium()
    a, b = ab
    rimg = image(md, 1, a, 1, b, E1_SOURCE)
    rcs = rimg + np.array([-0.03, 0.08, 0.06 if a == 1 else -0.06])
    rct = np.array([0.57, 0.575, -0.56])
    Td = E.reaction_m2l(md, 1, 1, a, b, rct, rcs, 6, 6)
    Tt = E.reaction_m2l_tables(md, 1, 1, a, b, rct, rcs, 6, 6)
    assert np.all(np.abs(Tt - Td) <= 1e-11 * np.abs(Td) + 1e-300)


@pytest.mark.parametrize("ab", [(1, 1), (1, 2), (2, 1), (2, 2)])
def test_m2l_operator_is_real_at_zero_azimuth(ab):
    """With the horizontal offset along +x the reaction M2L operator is real: the i^{mu-m} of
    the Bessel identity cancels the (-i)^{|m|+|mu|} of the Legendre branch (Prop. 1).  This is
    what lets an operator class be stored as two real matrices (for Re and Im of the source
    coefficients) with the azimuth applied as phases."""
    md = e1_medium()
    a, b = ab
    dI = md.d[1] if a == 1 else md.d[0]
    h = 0.25
    rct = np.array([0.8, 0.1, dI + (1.5 * h if a == 1 else -1.5 * h)])
    rcs = np.array([0.3, 0.1, dI + (-0.5 * h if a == 1 else 0.5 * h)])
    T = E.reaction_m2l(md, 1, 1, a, b, rct, rcs, 4, 4)
    assert np.abs(T.imag).max() <= 1e-14 * np.abs(T).max()
    # rotating the offset by phi multiplies entry (nm, nu mu) by e^{i (mu - m) phi}
    c, s = np.cos(0.7), np.sin(0.7)
    rct2 = rcs + np.array([0.5 * c, 0.5 * s, rct[2] - rcs[2]])
    T2 = E.reaction_m2l(md, 1, 1, a, b, rct2, rcs, 4, 4)
    ti, si = E._nm(4), E._nm(4)
    ph = np.exp(1j * 0.7 * np.array([[mu - m for _, mu in si] for _, m in ti]))
    assert np.abs(T2 - ph * T).max() <= 1e-12 * np.abs(T).max()


# ---- free-space translations (Sec. 3.1, Thm. 2-3, eqs. metole and metome) ----------------

FREE_LAM = 0.8
R1 = np.array([0.12, -0.05, 0.09])
BVEC = np.array([0.7, 0.4, -0.9])


def test_gaunt_coefficients_match_sympy():
    wigner = pytest.importorskip("sympy.physics.wigner")
    G = E.gaunt_all(6)
    for (n, m, nu, mu, q) in [(2, 1, 3, -2, 3), (4, -3, 2, 2, 4), (6, 0, 6, 5, 8), (5, 5, 6, -6, 1), (3, 0, 3, 0, 6)]:
        # int Y_n^m Y_nu^mu conj(Y_q^{m+mu}) = (-1)^{m+mu} int Y_n^m Y_nu^mu Y_q^{-m-mu}
        ex = (-1) ** (m + mu) * float(wigner.gaunt(n, nu, q, m, mu, -m - mu))
        assert abs(G[n * n + n + m, nu * nu + nu + mu, q] - ex) < 1e-14


def _basis(P, lam, r):
    R, T, Ph = E.sph(r)
    return np.array([special.spherical_in(nu, lam * R) * E.ylm(nu, mu, T, Ph) for nu, mu in E._nm(P)])


def test_thm2_regular_translation_is_exact():
    """Thm. 2 (eq. spmhat3d) as printed: i_n Y_n^m(r1 + b) = sum Shat i_nu Y_nu^mu(r1); the
    series in nu is finite (nu <= n + q ranges are cut by the Gaunt selection rules)."""
    Sh = E.free_shat(FREE_LAM, BVEC, 4, 12)
    R2, T2, P2 = E.sph(R1 + BVEC)
    bas = _basis(12, FREE_LAM, R1)
    for x, (n, m) in enumerate(E._nm(4)):
        ex = special.spherical_in(n, FREE_LAM * R2) * E.ylm(n, m, T2, P2)
        assert abs(Sh[x] @ bas - ex) <= 1e-13 * abs(ex)


def test_thm3_singular_translation_and_its_printed_prefactor():
    """Thm. 3 (eq. singularseparation): k_n Y_n^m(r1 + b) = sum S i_nu Y_nu^mu(r1) for |r1| < |b|,
    converging in nu.  The identity holds with the prefactor 4 pi (-1)^{m+nu}; the printed
    2 pi^2 (-1)^{m+nu+1} gives the series times -pi/2 (a misprint: k appears on both sides, so no
    normalization of k can account for it)."""
    R2, T2, P2 = E.sph(R1 + BVEC)
    errs = []
    for P in (6, 12):
        S = E.free_s(FREE_LAM, BVEC, 3, P)
        bas = _basis(P, FREE_LAM, R1)
        err = 0.0
        for x, (n, m) in enumerate(E._nm(3)):
            ex = special.spherical_kn(n, FREE_LAM * R2) * E.ylm(n, m, T2, P2)
            err = max(err, abs(S[x] @ bas - ex) / abs(ex))
        errs.append(err)
    assert errs[1] < 1e-9 and errs[0] > 100 * errs[1], errs
    Sp = E.free_s(FREE_LAM, BVEC, 3, 12, printed_prefactor=True)
    bas = _basis(12, FREE_LAM, R1)
    ratio = (Sp[5] @ bas) / (E.free_s(FREE_LAM, BVEC, 3, 12)[5] @ bas)
    assert abs(ratio - (-math.pi / 2)) < 1e-12


def test_free_m2m_m2l_l2l_reproduce_the_kernel():
    """ME about a source centre, shifted (M2M, eq. metome), translated (M2L, eq. metole with the
    Thm. 3 operator), shifted again (L2L, eq. metome) and evaluated (eq. freespace3dlocexp):
    converges to k_0(lam |r - r'|) as p grows."""
    rs = np.array([0.05, 0.02, -0.04])
    rcs, rcs2 = np.zeros(3), np.array([0.1, -0.1, 0.1])
    rct = np.array([0.9, -0.3, 0.5])
    rct2 = rct + np.array([0.03, 0.0, -0.02])
    r = rct + np.array([0.06, 0.05, -0.07])
    ex = E.k0(FREE_LAM, np.linalg.norm(r - rs))
    errs = []
    for p in (4, 8):
        M = E.free_me_coeffs(FREE_LAM, rs, rcs, p)
        M2 = E.free_m2m(FREE_LAM, M, rcs, rcs2, p)
        L = E.free_m2l(FREE_LAM, M2, rcs2, rct, p, p)
        L2 = E.free_l2l(FREE_LAM, L, rct, rct2, p)
        errs.append(abs(E.le_eval(FREE_LAM, L2, rct2, r, p)[-1] - ex) / ex)
        # M2M alone keeps the potential (within the shifted ME's truncation)
        assert abs(E.free_me_eval(FREE_LAM, M2, rcs2, r, p) - ex) / ex < 10 * 0.2 ** (p + 1)
    assert errs[1] < 1e-8 and errs[0] > 100 * errs[1], errs
