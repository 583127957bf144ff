"""Truncated expansions of Sec. 3 in FP64 -- TEST INFRASTRUCTURE ONLY.

Plain numpy/scipy restatement of the multipole and local expansions of Wang, Zhang & Cai
(arXiv 2002.01334), used by tests/ to check that the expansions the FMM truncates converge in p
to the oracle's direct values: the free-space Yukawa kernel in closed form, and the reaction
components u^{ab} of oracle.green_react_ab.  Only tests/ may import it; the product path never
does, and it shares no code with the CUDA path.

Contents (each cites the passage it follows):
  phat, ylm            normalized associated Legendre functions and spherical harmonics
                       (Sec. 3.1), continued to arguments x > 1 with the square-root branch of
                       Prop. 1 (eq. branch): sqrt(1 - x^2) = -i sqrt(x^2 - 1) for x > 1;
                       phat_all, ylm_all evaluate every order at once (same definition).
  phat_ratio_t_coeffs  phat_n^m / phat_m^m as a polynomial in t = x^2 - 1 (exact rationals).
  addition_k0          the zeroth-order addition theorem (Thm. 1, eq. sphbessel00).
  free_me, free_le     free-space ME and LE (Sec. 3.1, eqs. freespace3dmulexp,
                       freespace3dlocexp, melecoeffree).
  plane_wave_series    the extended modified Funk-Hecke expansion (Prop. 2).
  reaction_me          ME of a reaction component about an equivalent polarization centre
                       (Sec. 3.4, eqs. melayerupgoingimage and mebasis).
  reaction_le          LE of a reaction component about a target centre (Sec. 3.4, eqs.
                       lelayerimage and lecoeffimage).
  reaction_m2l         the M2L operator T of a reaction component (Sec. 3.4, eqs. metoleimage1
                       and metoleimage2), by direct quadrature.
  gaunt_all, free_shat, free_s, free_m2m, free_m2l, free_l2l
                       the free-space translations of Sec. 3.1 (Thm. 2-3, eqs. metome, metole);
                       the printed prefactor of Thm. 3 is off by -pi/2 (see free_s).
  legendre_product_coeffs, reaction_m2l_tables
                       the same operator by the table route of Sec. 3.5: products of two
                       Legendre functions as polynomials in lambda_rho (exact rational
                       coefficients), contracted with the Sommerfeld-type integrals S_{N M, ij}
                       of eq. M2Ltable (eqs. uniformintegral, coefintable, metoletableform).

The alpha-integrals of the Sommerfeld-type integrals are done in closed form with the Bessel
identity of Sec. 3.5 (J_n as an integral over the circle): for a horizontal offset with polar
coordinates (d, phi),
    int_0^{2 pi} exp(i lr d cos(alpha - phi)) exp(i k alpha) d alpha = 2 pi i^k exp(i k phi) J_k(lr d).
The remaining lambda_rho integral is scipy's adaptive vector quadrature (quad_vec) on
[0, inf), with the layer densities sigma from the oracle's transmission-condition solver.

Readings: the LE coefficient of the free-space kernel is taken as 4 pi k_n conj(Y_n^m) (the
addition theorem gives the conjugate; the printed Y_n^{-m} differs from it by (-1)^m under the
stated normalization), and the second row of the ME expansion of a 2b component uses the 2b
source offset (the printed 1b superscript is a typo).
"""
import functools
import math
from fractions import Fraction

import numpy as np
from numpy.polynomial import legendre as npleg
from scipy import integrate, special

from . import S_table, layer_response


# ------------------------------------------------------------------------------------------
# Spherical harmonics (Sec. 3.1)

def sph(v):
    """Spherical coordinates (r, theta, phi) of the vectors v[..., 3]."""
    v = np.asarray(v, float)
    r = np.sqrt((v * v).sum(-1))
    theta = np.arccos(np.clip(np.where(r > 0, v[..., 2] / np.where(r > 0, r, 1.0), 1.0), -1.0, 1.0))
    phi = np.arctan2(v[..., 1], v[..., 0])
    return r, theta, phi


def _norm(n, m):
    return math.sqrt((2 * n + 1) / (4 * math.pi) * math.factorial(n - m) / math.factorial(n + m))


def phat(n, m, x):
    """Normalized associated Legendre function P^m_n(x) of Sec. 3.1 (complex array).

    For m >= 0 it is (-1)^m N_nm (1 - x^2)^{m/2} d^m/dx^m P_n(x), so that
    Y_n^m = phat(cos theta) e^{i m phi}; for m < 0, phat_n^{-m} = (-1)^m phat_n^m, which gives
    Y_n^{-m} = (-1)^m conj(Y_n^m).  Outside [-1, 1] the square root takes the branch of Prop. 1:
    -i sqrt(x^2 - 1) for x > 1 and +i sqrt(x^2 - 1) for x < -1.
    """
    x = np.asarray(x, float)
    am = abs(m)
    if am > n:
        return np.zeros(x.shape, complex)
    der = npleg.legval(x, _legder(n, am))
    ax = np.abs(x)
    s = np.where(ax <= 1.0, np.sqrt(np.clip(1.0 - x * x, 0.0, None)) + 0j,
                 np.where(x > 0, -1j, 1j) * np.sqrt(np.clip(x * x - 1.0, 0.0, None)))
    val = (-1.0) ** am * _norm(n, am) * s ** am * der
    return val * (-1.0) ** am if m < 0 else val


def _nm(p):
    return [(n, m) for n in range(p + 1) for m in range(-n, n + 1)]


@functools.lru_cache(maxsize=None)
def _legder(n, am):
    """Legendre-basis coefficients of d^am/dx^am P_n."""
    c = np.eye(n + 1)[n]
    return npleg.legder(c, am) if am > 0 else c


@functools.lru_cache(maxsize=None)
def _phat_table(p):
    """Per (n, m) of _nm(p): Legendre-basis coefficients of d^{|m|}/dx^{|m|} P_n, |m|, and the
    constant factor of phat (normalization and signs)."""
    idx = _nm(p)
    D = np.zeros((p + 1, len(idx)))
    for j, (n, m) in enumerate(idx):
        c = _legder(n, abs(m))
        D[:len(c), j] = c
    am = np.array([abs(m) for _, m in idx])
    fac = np.array([(-1.0) ** abs(m) * _norm(n, abs(m)) * ((-1.0) ** abs(m) if m < 0 else 1.0) for n, m in idx])
    return D, am, fac


def phat_all(p, x):
    """phat_n^m(x) for every (n, m) of _nm(p) at one real x: the same definition as phat,
    evaluated for all orders at once."""
    D, am, fac = _phat_table(p)
    if abs(x) <= 1.0:
        s = math.sqrt(max(0.0, 1.0 - x * x)) + 0j
    else:
        s = (-1j if x > 0 else 1j) * math.sqrt(x * x - 1.0)
    return fac * s ** am * npleg.legval(x, D)


def ylm_all(p, theta, phi):
    """Y_n^m(theta, phi) for every (n, m) of _nm(p) at arrays of angles: rows in _nm(p) order
    (the same definition as ylm, all orders at once; |cos theta| <= 1)."""
    D, am, fac = _phat_table(p)
    x = np.cos(np.asarray(theta, float))
    s = np.sqrt(np.clip(1.0 - x * x, 0.0, None))
    ms = np.array([m for _, m in _nm(p)])
    leg = npleg.legval(x, D)  # [K, ...]
    sh = (-1,) + (1,) * x.ndim
    return (fac.reshape(sh) * s[None] ** am.reshape(sh) * leg
            * np.exp(1j * ms.reshape(sh) * np.asarray(phi, float)[None]))


def ylm(n, m, theta, phi):
    """Y_n^m(theta, phi) = phat_n^m(cos theta) e^{i m phi} (Sec. 3.1)."""
    return phat(n, m, np.cos(theta)) * np.exp(1j * m * np.asarray(phi, float))


# ------------------------------------------------------------------------------------------
# Free space (Sec. 3.1)

def k0(lam, r):
    """k_0(lambda r) = (pi / 2) e^{-lambda r} / (lambda r), the free-space kernel of Sec. 3.1."""
    return 0.5 * math.pi * math.exp(-lam * r) / (lam * r)


def addition_k0(lam, r1, b, p):
    """Partial sums over n <= 0..p of the addition theorem (Thm. 1, first case r1 < b):
    k_0(lam |r1 + b|) = 4 pi sum (-1)^n k_n(lam b) conj Y_n^m(b) i_n(lam r1) Y_n^m(r1)."""
    R1, T1, P1 = sph(r1)
    B, TB, PB = sph(b)
    terms = np.zeros(p + 1, complex)
    for n, m in _nm(p):
        terms[n] += (4 * math.pi * (-1) ** n * special.spherical_kn(n, lam * B) * np.conj(ylm(n, m, TB, PB))
                     * special.spherical_in(n, lam * R1) * ylm(n, m, T1, P1))
    return np.cumsum(terms).real


def free_me(lam, rsrc, rc, r, p):
    """Partial sums over n <= 0..p of the free-space ME about the source centre rc
    (eqs. freespace3dmulexp, melecoeffree): M_nm = 4 pi i_n(lam r's) conj Y_n^m(theta's, phi's),
    k_0 ~ sum M_nm k_n(lam r_s) Y_n^m(theta_s, phi_s)."""
    Rs_, Ts_, Ps_ = sph(np.asarray(rsrc, float) - rc)
    Rs, Ts, Ps = sph(np.asarray(r, float) - rc)
    terms = np.zeros(p + 1, complex)
    for n, m in _nm(p):
        M = 4 * math.pi * special.spherical_in(n, lam * Rs_) * np.conj(ylm(n, m, Ts_, Ps_))
        terms[n] += M * special.spherical_kn(n, lam * Rs) * ylm(n, m, Ts, Ps)
    return np.cumsum(terms).real


def free_le(lam, rsrc, rc, r, p):
    """Partial sums over n <= 0..p of the free-space LE about the target centre rc
    (eqs. freespace3dlocexp, melecoeffree with the conjugate reading):
    L_nm = 4 pi k_n(lam r't) conj Y_n^m(theta't, phi't), k_0 ~ sum L_nm i_n(lam r_t) Y_n^m."""
    Rt_, Tt_, Pt_ = sph(np.asarray(rsrc, float) - rc)
    Rt, Tt, Pt = sph(np.asarray(r, float) - rc)
    terms = np.zeros(p + 1, complex)
    for n, m in _nm(p):
        L = 4 * math.pi * special.spherical_kn(n, lam * Rt_) * np.conj(ylm(n, m, Tt_, Pt_))
        terms[n] += L * special.spherical_in(n, lam * Rt) * ylm(n, m, Tt, Pt)
    return np.cumsum(terms).real


def plane_wave_series(lam, lr, alpha, r, p):
    """Partial sums over n <= 0..p of Prop. 2 for the complex vector
    Lambda = (i lr cos alpha, i lr sin alpha, -sqrt(lam^2 + lr^2)):
    e^{Lambda . r} ~ sum conj(B_n^m(r)) phat_n^m(lz / lam) e^{i m alpha},
    B_n^m(r) = 4 pi (-1)^n i_n(lam |r|) Y_n^m(r)."""
    R, T, P = sph(r)
    w = math.sqrt(lam * lam + lr * lr) / lam
    terms = np.zeros(p + 1, complex)
    for n, m in _nm(p):
        B = 4 * math.pi * (-1) ** n * special.spherical_in(n, lam * R) * ylm(n, m, T, P)
        terms[n] += np.conj(B) * phat(n, m, w) * np.exp(1j * m * alpha)
    return np.cumsum(terms)


def plane_wave(lam, lr, alpha, r):
    """e^{Lambda . r} for the vector Lambda of Prop. 2, directly."""
    lz = math.sqrt(lam * lam + lr * lr)
    return np.exp(1j * lr * (math.cos(alpha) * r[0] + math.sin(alpha) * r[1]) - lz * r[2])


# ------------------------------------------------------------------------------------------
# Reaction components (Sec. 3.3-3.4)

class _Comp:
    """One reaction component u^{ab}_{l l'}: its layers, interfaces and densities (Sec. 2.2)."""

    def __init__(self, md, l, lp, a, b):
        self.md, self.l, self.lp, self.a, self.b = md, l, lp, a, b
        self.lam, self.lamp = md.lam[l], md.lam[lp]
        # interface the polarization sources sit against: d_l for a = 1, d_{l-1} for a = 2
        self.dI = md.d[l] if a == 1 else md.d[l - 1]

    def sigma(self, lr):
        s1, s2 = layer_response(self.md, lr, self.lp, self.b)
        return s1[self.l] if self.a == 1 else s2[self.l]

    def zfactor(self, lr, zt, zs):
        """exp of the z-part of E^+ (a = 1) or E^- (a = 2) (eq. mekernelimage) for a target at
        height zt and a polarization point (or centre) at height zs; and lz, lz'."""
        lz = math.sqrt(self.lam ** 2 + lr * lr)
        lzp = math.sqrt(self.lamp ** 2 + lr * lr)
        if self.a == 1:
            e = -lz * (zt - self.dI) - lzp * (self.dI - zs)
        else:
            e = -lz * (self.dI - zt) - lzp * (zs - self.dI)
        return math.exp(e), lz, lzp


def _quad(f, tol):
    """int_0^inf f(lr) d lr of a vector-valued f by scipy's adaptive quadrature."""
    val, _ = integrate.quad_vec(f, 0.0, np.inf, epsabs=0.0, epsrel=tol, norm="max", limit=20000)
    return val


def _polar(dx, dy):
    return math.hypot(dx, dy), math.atan2(dy, dx)


def _me_sign(a, n, m):
    """The sign of F~^{ab}_nm in eq. mebasis: (-1)^{n+m} for 2b components, 1 for 1b."""
    return (-1.0) ** (n + m) if a == 2 else 1.0


def reaction_me(md, l, lp, a, b, r, rimg, rc, p, tol=1e-13):
    """Partial sums over n <= 0..p of the ME of u~^{ab}_{l l'}(r, r'_ab) about the polarization
    centre rc (eq. melayerupgoingimage): sum M_nm F~_nm(r, rc), with
    M_nm = 4 pi i_n(lam_l' r_s) conj Y_n^m(theta_s, phi_s) of r'_ab - rc and F~ from eq. mebasis,
    whose alpha-integral is (2 pi) i^m e^{i m phi_d} J_m(lr d) for (d, phi_d) the polar form of
    the horizontal offset r - rc.  2b components carry the extra (-1)^{n+m} of eq. mebasis."""
    c = _Comp(md, l, lp, a, b)
    r = np.asarray(r, float)
    rc = np.asarray(rc, float)
    Rs, Ts, Ps = sph(np.asarray(rimg, float) - rc)
    d, phd = _polar(r[0] - rc[0], r[1] - rc[1])
    idx = _nm(p)
    M = np.array([4 * math.pi * special.spherical_in(n, c.lamp * Rs) * np.conj(ylm(n, m, Ts, Ps)) for n, m in idx])
    pre = np.array([(1j) ** m * np.exp(1j * m * phd) / (4 * math.pi) * _me_sign(a, n, m) for n, m in idx])
    ms = np.array([m for _, m in idx])

    def f(lr):
        ez, lz, lzp = c.zfactor(lr, r[2], rc[2])
        base = lr / lz * ez * c.sigma(lr)
        ph = phat_all(p, lzp / c.lamp)
        return (M * pre * base * ph * special.jv(ms, lr * d)).view(float)

    terms = _quad(f, tol).view(complex)
    out = np.zeros(p + 1, complex)
    for (n, _), t in zip(idx, terms):
        out[n] += t
    return np.cumsum(out).real


def reaction_le_coeffs(md, l, lp, a, b, rimg, rct, p, tol=1e-13):
    """LE coefficients L_nm of u~^{ab}_{l l'}(., r'_ab) about the target centre rct (eq.
    lecoeffimage), n <= p, in the order (n, m = -n..n).  The alpha-integral of e^{-i m alpha}
    against the horizontal offset rct - r'_ab (polar form (d, phi_d)) is 2 pi i^m e^{-i m phi_d}
    J_m(lr d); the prefactor is (-1)^n for 1b and (-1)^m for 2b components."""
    c = _Comp(md, l, lp, a, b)
    rimg = np.asarray(rimg, float)
    rct = np.asarray(rct, float)
    d, phd = _polar(rct[0] - rimg[0], rct[1] - rimg[1])
    idx = _nm(p)
    pre = np.array([(1j) ** m * np.exp(-1j * m * phd) * ((-1.0) ** n if a == 1 else (-1.0) ** m) for n, m in idx])
    ms = np.array([m for _, m in idx])

    def f(lr):
        ez, lz, lzp = c.zfactor(lr, rct[2], rimg[2])
        base = lr / lz * ez * c.sigma(lr)
        ph = phat_all(p, lz / c.lam)
        return (pre * base * ph * special.jv(ms, lr * d)).view(float)

    return _quad(f, tol).view(complex)


def le_eval(lam, L, rct, r, p):
    """Partial sums over n <= 0..p of sum L_nm i_n(lam r_t) Y_n^m(theta_t, phi_t) (eq.
    lelayerimage) with (r_t, theta_t, phi_t) the spherical coordinates of r - rct."""
    Rt, Tt, Pt = sph(np.asarray(r, float) - rct)
    out = np.zeros(p + 1, complex)
    for (n, m), Lnm in zip(_nm(p), L):
        out[n] += Lnm * special.spherical_in(n, lam * Rt) * ylm(n, m, Tt, Pt)
    return np.cumsum(out).real


def reaction_le(md, l, lp, a, b, r, rimg, rct, p, tol=1e-13):
    """Partial sums over n <= 0..p of the LE of u~^{ab}_{l l'}(r, r'_ab) about rct."""
    L = reaction_le_coeffs(md, l, lp, a, b, rimg, rct, p, tol)
    return le_eval(md.lam[l], L, rct, r, p)


def me_coeffs(lamp, rimg, rc, P):
    """M_nm = 4 pi i_n(lam' r_s) conj Y_n^m(theta_s, phi_s) of r'_ab - rc, n <= P (eq.
    melayerupgoingimage)."""
    Rs, Ts, Ps = sph(np.asarray(rimg, float) - rc)
    return np.array([4 * math.pi * special.spherical_in(n, lamp * Rs) * np.conj(ylm(n, m, Ts, Ps))
                     for n, m in _nm(P)])


def reaction_m2l(md, l, lp, a, b, rct, rcs, p, P, tol=1e-13):
    """M2L operator T_{nm, nu mu} (n <= p, nu <= P) from the polarization centre rcs to the
    target centre rct (eqs. metoleimage1, metoleimage2).  The alpha-integral of
    e^{i(mu - m) alpha} against the horizontal offset rct - rcs (polar form (d, phi_d)) is
    2 pi i^{mu-m} e^{i(mu-m) phi_d} J_{mu-m}(lr d); the sign is (-1)^n for 1b and
    (-1)^{m + nu + mu} for 2b components.  Returns T as a complex [(p+1)^2, (P+1)^2] matrix."""
    c = _Comp(md, l, lp, a, b)
    rct = np.asarray(rct, float)
    rcs = np.asarray(rcs, float)
    d, phd = _polar(rct[0] - rcs[0], rct[1] - rcs[1])
    ti, si = _nm(p), _nm(P)
    k = np.array([[mu - m for nu, mu in si] for n, m in ti])
    sgn = np.array([[(-1.0) ** n if a == 1 else (-1.0) ** (m + nu + mu) for nu, mu in si] for n, m in ti])
    pre = sgn * (1j) ** k * np.exp(1j * k * phd)

    def f(lr):
        ez, lz, lzp = c.zfactor(lr, rct[2], rcs[2])
        base = lr / lz * ez * c.sigma(lr)
        pt = phat_all(p, lz / c.lam)
        ps = phat_all(P, lzp / c.lamp)
        return (pre * base * np.outer(pt, ps) * special.jv(k, lr * d)).ravel().view(float)

    return _quad(f, tol).view(complex).reshape(len(ti), len(si))


# ------------------------------------------------------------------------------------------
# The table form of the reaction M2L (Sec. 3.5): Legendre products as polynomials in lambda_rho
# and Sommerfeld-type integrals S_{N M, ij} (eqs. uniformintegral, coefintable, M2Ltable,
# metoletableform)

def _legendre_power(n):
    """Exact power-basis coefficients of the Legendre polynomial P_n (index = power of x)."""
    c = [Fraction(0)] * (n + 1)
    for k in range(n // 2 + 1):
        c[n - 2 * k] = Fraction((-1) ** k * math.comb(n, k) * math.comb(2 * n - 2 * k, n), 2 ** n)
    return c


@functools.lru_cache(maxsize=None)
def _phat_t_poly(n, m):
    """phat_n^m(x) at x = lz/lam (lz = sqrt(lam^2 + lr^2)) written as
    (-1)^m c_nm (-i)^|m| (lr/lam)^|m| (lam/lz)^i sum_u e_u (lr/lam)^{2u},
    with i = (n + |m|) mod 2 and exact rationals e_u.  With x^2 = 1 + t, t = (lr/lam)^2:
    d^|m| P_n / dx^|m| has the parity of n - |m|; for odd parity one factor x is taken out as
    x = x^2 / x = (1 + t) (lam/lz), and x^{2q} = (1 + t)^q is expanded binomially.
    Returns (i, e) with e a tuple of Fractions."""
    am = abs(m)
    c = _legendre_power(n)
    for _ in range(am):  # differentiate |m| times
        c = [c[k + 1] * (k + 1) for k in range(len(c) - 1)] or [Fraction(0)]
    i = (n + am) % 2
    # multiply by x when odd so that only even powers remain
    if i:
        c = [Fraction(0)] + c
    e = [Fraction(0)] * (len(c) // 2 + 1)
    for k in range(0, len(c), 2):
        q = k // 2
        for u in range(q + 1):
            e[u] += c[k] * math.comb(q, u)
    while len(e) > 1 and e[-1] == 0:
        e.pop()
    return i, tuple(e)


def _phat_lr_coeffs(n, m, lam):
    """Complex g_u with phat_n^m(lz/lam) = (lam/lz)^i lr^|m| sum_u g_u lr^{2u}; returns (i, g)."""
    am = abs(m)
    i, e = _phat_t_poly(n, m)
    sign = (-1.0) ** am * ((-1.0) ** am if m < 0 else 1.0)
    pre = sign * _norm(n, am) * (-1j) ** am / lam ** am
    return i, np.array([pre * float(eu) / lam ** (2 * u) for u, eu in enumerate(e)])


def legendre_product_coeffs(n, m, nu, mu, lam, lamp):
    """C^s of Sec. 3.5: phat_n^m(lz/lam) phat_nu^mu(lz'/lam') =
    sum_s C^s lr^{|m| + |mu| + 2s} (lam/lz)^i (lam'/lz')^j; returns (i, j, C)."""
    i, g = _phat_lr_coeffs(n, m, lam)
    j, gp = _phat_lr_coeffs(nu, mu, lamp)
    return i, j, np.convolve(g, gp)


def reaction_m2l_tables(md, l, lp, a, b, rct, rcs, p, P, tol=1e-13):
    """M2L operator T (n <= p, nu <= P) by the table route of Sec. 3.5: T = sign e^{i(mu-m)phi}
    I_{nm,nu mu} (eq. coefintable), I = i^{mu-m} sum_s C~^s S_{N, mu-m, ij} (eq. metoletableform)
    with N = |m| + |mu| + 2s + 1 and C~^s = sqrt((N + mu - m)! (N - mu + m)!) C^s, the tables S
    by the oracle's direct quadrature (orc_S_table, unscaled), and S_{N,-M} = (-1)^M S_{N,M}."""
    c = _Comp(md, l, lp, a, b)
    rct = np.asarray(rct, float)
    rcs = np.asarray(rcs, float)
    d, phd = _polar(rct[0] - rcs[0], rct[1] - rcs[1])
    if a == 1:
        zt, zs = rct[2] - c.dI, c.dI - rcs[2]
    else:
        zt, zs = c.dI - rct[2], rcs[2] - c.dI
    S = S_table(md, l, lp, a, b, 1.0, d, zt, zs, p + P + 3, tol)
    ti, si = _nm(p), _nm(P)
    T = np.zeros((len(ti), len(si)), complex)
    for x, (n, m) in enumerate(ti):
        for y, (nu, mu) in enumerate(si):
            i, j, C = legendre_product_coeffs(n, m, nu, mu, c.lam, c.lamp)
            M = mu - m
            acc = 0j
            for s, Cs in enumerate(C):
                N = abs(m) + abs(mu) + 2 * s + 1
                Ct = math.sqrt(math.factorial(N + M) * math.factorial(N - M)) * Cs
                acc += Ct * S[N, abs(M), i, j] * ((-1.0) ** abs(M) if M < 0 else 1.0)
            sgn = (-1.0) ** n if a == 1 else (-1.0) ** (nu + m + mu)
            T[x, y] = sgn * np.exp(1j * M * phd) * (1j) ** M * acc
    return T


def phat_ratio_t_coeffs(n, m):
    """phat_n^m(x) / phat_m^m(x) = x^{-i} sum_k c_k t^k with t = x^2 - 1 and i = (n - m) mod 2,
    0 <= m <= n (Sec. 3.1 normalization; the ratio is a polynomial in x, free of the square-root
    branch).  From the definition: the ratio is N_nm d^m P_n / (N_mm d^m P_m) with d^m P_m the
    constant (2m)! / (2^m m!), expanded exactly as in _phat_t_poly.  Returns (i, c) floats."""
    i, e = _phat_t_poly(n, m)
    scale = _norm(n, m) / (_norm(m, m) * math.factorial(2 * m) / (2 ** m * math.factorial(m)))
    return i, [float(ek) * scale for ek in e]


# ------------------------------------------------------------------------------------------
# Free-space translations (Sec. 3.1, Thm. 2-3, eqs. metole and metome)

@functools.lru_cache(maxsize=None)
def gaunt_all(p):
    """G[f(n,m), f(nu,mu), q] = int Y_n^m Y_nu^mu conj(Y_q^{m+mu}) over the unit sphere for
    n, nu <= p and q <= 2p (f(n, m) = n^2 + n + m), by a product rule exact for these
    band-limited integrands: Gauss-Legendre in cos(theta) (2p + 2 nodes, degree <= 4p) times
    the trapezoid rule in phi (4p + 2 points, frequencies |k| <= 4p).  This is the Gaunt
    coefficient G(n, m; nu, mu; q) of Thm. 2-3 under the reading of it that makes Thm. 2 hold."""
    nt, nph = 2 * p + 2, 4 * p + 2
    x, w = np.polynomial.legendre.leggauss(nt)
    th = np.arccos(x)
    ph = 2 * math.pi * np.arange(nph) / nph
    TH, PH = np.meshgrid(th, ph, indexing="ij")
    W = (w[:, None] * np.full(nph, 2 * math.pi / nph)[None, :]).ravel()
    Y = {(n, m): ylm(n, m, TH, PH).ravel() for n in range(2 * p + 1) for m in range(-n, n + 1)}
    NF = (p + 1) ** 2
    G = np.zeros((NF, NF, 2 * p + 1))
    for n, m in _nm(p):
        for nu, mu in _nm(p):
            a = W * Y[(n, m)] * Y[(nu, mu)]
            for q in range(abs(n - nu), n + nu + 1):
                if abs(m + mu) <= q and (n + nu + q) % 2 == 0:
                    G[n * n + n + m, nu * nu + nu + mu, q] = (a * np.conj(Y[(q, m + mu)])).sum().real
    return G


def _gf(G, n, m, nu, mu, q):
    return G[n * n + n + m, nu * nu + nu + mu, q]


def _translation(lam, b, p, P, kind):
    """sum_q c_q f_q(lam |b|) conj Y_q^{mu-m}(b) G(n, m; nu, -mu; q) for all (n, m) <= p,
    (nu, mu) <= P, with f = i (kind "i", Thm. 2 with its sign (-1)^{nu-n+m+q} in c_q) or k
    (kind "k", Thm. 3, c_q = 1).  Vectorized over the entries; conj Y_q^k is taken as 0 for
    |k| > q, where the Gaunt coefficient vanishes."""
    Bn, TB, PB = sph(b)
    G = gaunt_all(max(p, P))
    f = special.spherical_in if kind == "i" else special.spherical_kn
    qmax = p + P
    ti, si = _nm(p), _nm(P)
    n = np.array([a for a, _ in ti])[:, None]
    m = np.array([c for _, c in ti])[:, None]
    nu = np.array([a for a, _ in si])[None, :]
    mu = np.array([c for _, c in si])[None, :]
    fo = (n * n + n + m) * np.ones_like(nu)
    fi = (nu * nu + nu - mu) * np.ones_like(n)
    k = mu - m
    yb = phat_all(qmax, math.cos(TB)) * np.exp(1j * np.array([kk for _, kk in _nm(qmax)]) * PB)
    out = np.zeros((len(ti), len(si)), complex)
    for q in range(qmax + 1):
        ok = np.abs(k) <= q
        ang = np.where(ok, np.conj(yb[q * q + q + np.clip(k, -q, q)]), 0.0)
        g = G[fo, fi, q] if q < G.shape[2] else np.zeros(k.shape)
        c = (-1.0) ** (nu - n + m + q) if kind == "i" else 1.0
        out += c * f(q, lam * Bn) * ang * g
    return out


def free_shat(lam, b, p, P):
    """Shat_{n nu}^{m mu}(b) of Thm. 2 (eq. spmhat3d), n <= p, nu <= P, as a complex matrix
    [(n, m), (nu, mu)]: i_n Y_n^m(r1 + b) = sum Shat i_nu Y_nu^mu(r1).  Entry by entry,
    4 pi sum_q (-1)^{nu-n+m+q} i_q(lam b) conj Y_q^{mu-m}(b) G(n, m; nu, -mu; q)."""
    return 4 * math.pi * _translation(lam, b, p, P, "i")


def free_s(lam, b, p, P, printed_prefactor=False):
    """S_{n nu}^{m mu}(b) of Thm. 3 (eq. singularseparation), n <= p, nu <= P:
    k_n Y_n^m(r1 + b) = sum S i_nu Y_nu^mu(r1) for |r1| < |b|.  Entry by entry,
    4 pi (-1)^{m+nu} sum_q k_q(lam b) conj Y_q^{mu-m}(b) G(n, m; nu, -mu; q).  The printed
    prefactor 2 pi^2 (-1)^{m+nu+1} is off by the factor -pi/2 (with the Gaunt coefficient of
    Thm. 2 and any normalization of k, which appears on both sides); printed_prefactor=True
    uses the printed constant."""
    ti, si = _nm(p), _nm(P)
    m = np.array([c for _, c in ti])[:, None]
    nu = np.array([a for a, _ in si])[None, :]
    pref = 2 * math.pi ** 2 * (-1.0) ** (m + nu + 1) if printed_prefactor else 4 * math.pi * (-1.0) ** (m + nu)
    return pref * _translation(lam, b, p, P, "k")


def free_me_coeffs(lam, rsrc, rc, p):
    """M_nm = 4 pi i_n(lam r's) conj Y_n^m(theta's, phi's) of one unit source (eq. melecoeffree)."""
    R, T, P = sph(np.asarray(rsrc, float) - rc)
    return np.array([4 * math.pi * special.spherical_in(n, lam * R) * np.conj(ylm(n, m, T, P)) for n, m in _nm(p)])


def free_me_eval(lam, M, rc, r, p):
    """sum M_nm k_n(lam r_s) Y_n^m(theta_s, phi_s) about rc (eq. freespace3dmulexp)."""
    R, T, P = sph(np.asarray(r, float) - rc)
    return sum(Mnm * special.spherical_kn(n, lam * R) * ylm(n, m, T, P) for (n, m), Mnm in zip(_nm(p), M)).real


def free_m2l(lam, M, rcs, rct, p, P):
    """LE coefficients about rct (degree <= P) of the ME M (degree <= p) about rcs (eq. metole,
    with Thm. 3 applied to each k_n Y_n^m of the ME): L_{nu mu} = sum_{nm} M_nm S_{n nu}^{m mu}(b),
    b = rct - rcs."""
    return free_s(lam, np.asarray(rct, float) - rcs, p, P).T @ M


def free_m2m(lam, M, rcs, rcs_new, p):
    """ME about rcs shifted to rcs_new (eq. metome): M~_nm = sum conj(Shat_{n nu}^{m mu}(rcs - rcs_new)) M_{nu mu}."""
    return np.conj(free_shat(lam, np.asarray(rcs, float) - rcs_new, p, p)) @ M


def free_l2l(lam, L, rct, rct_new, p):
    """LE about rct shifted to rct_new (eq. metome): L~_nm = sum Shat_{nu n}^{mu m}(rct_new - rct) L_{nu mu}."""
    return free_shat(lam, np.asarray(rct_new, float) - rct, p, p).T @ L


# ------------------------------------------------------------------------------------------
# Recurrences of the scaled Sommerfeld-type integrals (Sec. 3.5, eqs. recurrence1 and
# backwardrecurrence1), on arrays S[n, m, i, j] = S^n S_{nm,ij} (as oracle.S_table returns)

def _a(n):
    return math.sqrt(n * (n + 1.0))


def forward_recurrence(S0, rho_over_S):
    """Fill m >= 2 from the columns m = 0, 1 of S0 by eq. recurrence1:
    S^n S_{n,m+1} = (2m / a_{n+m}) (S/rho) S^{n-1} S_{n-1,m} - (a_{n-m} / a_{n+m}) S^n S_{n,m-1}."""
    S = np.array(S0, float)
    S[:, 2:] = 0.0
    K = S.shape[0] - 1
    if rho_over_S == 0:  # S_{nm}(0, z, z') = 0 for m > 0 (Sec. 3.5)
        return S
    for m in range(1, K):
        for n in range(m + 1, K + 1):
            S[n, m + 1] = (2 * m / _a(n + m)) / rho_over_S * S[n - 1, m] - (_a(n - m) / _a(n + m)) * S[n, m - 1]
    return S


def backward_recurrence(S0, rho_over_S):
    """Fill the rows n < K (columns m >= 1) from the top row n = K and the column m = 0 of S0 by
    eq. backwardrecurrence1, the forward recurrence solved for its lower-order term:
    S^{n-1} S_{n-1,m} = (a_{n+m} / 2m) (rho/S) S^n S_{n,m+1} + (a_{n-m} / 2m) (rho/S) S^n S_{n,m-1}.
    The column m = 0 below the top row is not produced by the recurrence (its 2m vanishes) and is
    taken from S0, like the top row."""
    S = np.array(S0, float)
    K = S.shape[0] - 1
    S[:K, 1:] = 0.0
    for n in range(K, 1, -1):
        for m in range(1, n):
            S[n - 1, m] = (_a(n + m) / (2 * m)) * rho_over_S * S[n, m + 1] + \
                (_a(n - m) / (2 * m)) * rho_over_S * S[n, m - 1]
    return S
