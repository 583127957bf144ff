"""CPU tests of the host-side tables that lpbfmm_create builds and uploads (lpbfmm_host_table:
host code of the library, no device).  Each table is compared with an independent computation:
Gaunt coefficients with sympy's exact Gaunt integrals (Sec. 3.1, Thm. 2-3), the Legendre-product
polynomials with the oracle's exact rational expansion of the definition (Sec. 3.5), the
direction table with scipy's harmonics, the factorial norms with exact integers."""
import math
from decimal import Context, Decimal

import numpy as np
import pytest

from paper_2002_01334_gb300 import build as B
from paper_2002_01334_gb300 import lpbfmm as F


@pytest.fixture(scope="module", autouse=True)
def built():
    B.build()


def f(n, m):
    return n * n + n + m


def h(n, m):
    return n * (n + 1) // 2 + m


def test_host_table_argument_checks():
    L = F.lib()
    import ctypes as C
    n = C.c_int64()
    assert L.lpbfmm_host_table(0, 8, None, 0, None) == 1
    assert L.lpbfmm_host_table(0, 1, None, 0, C.byref(n)) == 3
    assert L.lpbfmm_host_table(0, 17, None, 0, C.byref(n)) == 3
    assert L.lpbfmm_host_table(9, 8, None, 0, C.byref(n)) == 1
    assert L.lpbfmm_host_table(3, 8, None, 0, C.byref(n)) == 0 and n.value == 36 * 36
    buf = (C.c_double * 10)()
    assert L.lpbfmm_host_table(3, 8, buf, 10, C.byref(n)) == 1


@pytest.mark.parametrize("p", [2, 3])
def test_gaunt_table_equals_exact_gaunt_integrals(p):
    wigner = pytest.importorskip("sympy.physics.wigner")
    G = F.host_table(F.TABLE_GAUNT, p).reshape((p + 1) ** 2, (p + 1) ** 2, 2 * p + 1)
    for n in range(p + 1):
        for a in range(-n, n + 1):
            for nu in range(p + 1):
                for g in range(-nu, nu + 1):
                    for q in range(2 * p + 1):
                        v = G[f(n, a), f(nu, g), q]
                        if abs(g - a) > q or (n + nu + q) % 2:
                            assert v == 0.0
                            continue
                        # conj(Y_nu^g) = (-1)^g Y_nu^{-g}
                        ex = (-1) ** g * float(wigner.gaunt(n, q, nu, a, g - a, -g))
                        assert abs(v - ex) <= 1e-14, (n, a, nu, g, q, v, ex)


def test_gaunt_table_spot_checks_at_p10():
    wigner = pytest.importorskip("sympy.physics.wigner")
    p = 10
    G = F.host_table(F.TABLE_GAUNT, p).reshape((p + 1) ** 2, (p + 1) ** 2, 2 * p + 1)
    rng = np.random.default_rng(5)
    checked = 0
    while checked < 60:
        n, nu = rng.integers(0, p + 1, 2)
        a, g = rng.integers(-n, n + 1), rng.integers(-nu, nu + 1)
        q = rng.integers(abs(n - nu), n + nu + 1)
        if (n + nu + q) % 2 or abs(g - a) > q:
            continue
        ex = (-1) ** int(g) * float(wigner.gaunt(int(n), int(q), int(nu), int(a), int(g - a), int(-g)))
        assert abs(G[f(n, a), f(nu, g), q] - ex) <= 1e-14
        checked += 1


@pytest.mark.parametrize("p", [4, 10, 16])
def test_tpoly_table_equals_exact_legendre_ratio(p):
    E = pytest.importorskip("oracle.expansions")
    tpk = p // 2 + 2
    c = F.host_table(F.TABLE_TPOLY, p).reshape(-1, tpk)
    assert c.shape[0] == (p + 1) * (p + 2) // 2
    for n in range(p + 1):
        for m in range(n + 1):
            i, ex = E.phat_ratio_t_coeffs(n, m)
            assert i == (n - m) % 2 and len(ex) <= tpk
            ex = np.array(ex + [0.0] * (tpk - len(ex)))
            assert np.abs(c[h(n, m)] - ex).max() <= 1e-13 * np.abs(ex).max(), (n, m, c[h(n, m)], ex)
            for x in (1.3, 4.0):  # the ratio itself, against the direct definition
                v = sum(ck * (x * x - 1) ** k for k, ck in enumerate(c[h(n, m)])) / x ** i
                d = E.phat(n, m, x) / E.phat(m, m, x)
                assert abs(v - d) <= 1e-12 * abs(d), (n, m, x)


@pytest.mark.parametrize("p", [4, 16])
def test_phat_dir_table_equals_scipy_harmonics(p):
    special = pytest.importorskip("scipy.special")
    if not hasattr(special, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    qmax = 2 * p
    # every distinct dx^2 + dy^2 for |dx|, |dy| <= 5 (the far offsets of two-box separation)
    rho2 = sorted({dx * dx + dy * dy for dx in range(6) for dy in range(6)})
    assert len(rho2) == 20
    nd = 11 * len(rho2) + 2
    P = F.host_table(F.TABLE_PHAT_DIR, p).reshape(nd, -1)
    for d in range(nd):
        if d < nd - 2:
            ri, dz = d // 11, d % 11 - 5
            bn = math.sqrt(rho2[ri] + dz * dz)
            x = -dz / bn if bn > 0 else 1.0
        else:
            x = (-1.0 if d == nd - 2 else 1.0) / math.sqrt(3.0)
        th = math.acos(x)
        for q in range(qmax + 1):
            for k in range(q + 1):
                ex = special.sph_harm_y(q, k, th, 0.0).real
                assert abs(P[d, h(q, k)] - ex) <= 1e-12 * max(1.0, abs(ex)), (d, q, k)


def test_sfac_table_equals_exact_factorials():
    s = F.host_table(F.TABLE_SFAC, 8).reshape(36, 36)
    for K in range(36):
        for d in range(36):
            if d > K:
                assert s[K, d] == 0.0
            else:
                # exact to 30 digits: the table rounds once, so it is within an ulp of the value
                ex = Decimal(math.factorial(K + d) * math.factorial(K - d)).sqrt(Context(prec=40))
                assert abs(Decimal(s[K, d]) - ex) <= Decimal(2.3e-16) * ex, (K, d)
