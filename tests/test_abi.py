"""The C-ABI library loads and exports every entry point declared in include/lpbfmm.h; host-side
argument checks return their documented codes (no GPU computation is issued)."""
import ctypes as C
import os
import re

import pytest

from paper_2002_01334_gb300 import build as B
from paper_2002_01334_gb300 import lpbfmm as F

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    B.build()
    return F.lib()


def declared():
    txt = open(os.path.join(ROOT, "include", "lpbfmm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lpbfmm_[a-z_]+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(L):
    names = declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n


def test_default_opts_and_strerror(L):
    o = F.Opts()
    L.lpbfmm_default_opts(C.byref(o))
    assert (o.precision, o.max_per_leaf, o.uniform_depth, o.separation, o.react_levels) == (0, 128, 0, 0, 4)
    assert L.lpbfmm_strerror(0) == b"ok"
    assert L.lpbfmm_strerror(4) == b"charge on an interface"


def _create(L, d, eps, lam, p, tol=1e-14):
    h = C.c_void_p()
    arr = lambda v: (C.c_double * len(v))(*v)
    return L.lpbfmm_create(len(d), arr(d), arr(eps), arr(lam), p, tol, None, C.byref(h))


def test_create_rejects_bad_media_and_orders(L):
    assert _create(L, [0.0, 0.5], [1, 2, 3], [1, 1, 1], 8) == 2   # not descending
    assert _create(L, [0.0], [1, -2], [1, 1], 8) == 2             # eps <= 0
    assert _create(L, [0.0], [1, 2], [1, 0.0], 8) == 2            # lambda <= 0 (Sec. 1 requires lambda > 0)
    assert _create(L, [0.0], [1, 2], [1, 1], 1) == 3              # p below range
    assert _create(L, [0.0], [1, 2], [1, 1], 17) == 3             # p above range
    assert _create(L, [0.0], [1, 2], [1, 1], 8, tol=0.5) == 1     # tol out of range
    assert L.lpbfmm_eval(None, 0, None, None, None, None, None) == 1
