"""Oracle for the layered-media screened-Coulomb FMM -- TEST INFRASTRUCTURE ONLY.

Plain FP64 CPU implementation (oracle.c) of what the GPU path computes, written from
Wang, Zhang & Cai, arXiv 2002.01334.  Only tests/, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path never does.

Parity status of each function is stated in tests/test_oracle_pins.py, which pins it
against closed forms, the paper's printed formulas, invariants and brute force.  Submodules:
``expansions`` restates the truncated expansions and translations of Sec. 3 (numpy/scipy;
tests/test_expansion_pins.py checks that they converge in p to this package's direct values),
``adaptive`` the adaptive dual trees and their lists (tests/test_adaptive_tree.py), and ``fmm``
a plain CPU FMM, free-space and reaction parts, built from them (tests/test_cpu_fmm.py).
"""
import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None
MAXL = 9


def build(force=False):
    """Compile oracle.c into oracle/_build/liboracle.so (gcc, OpenMP, no FMA contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    tmp = _SO + ".tmp%d" % os.getpid()
    subprocess.check_call(["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-shared", "-fPIC",
                           "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_SO)
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int)
        lp = C.POINTER(C.c_int64)
        up = C.POINTER(C.c_uint64)
        L.orc_layer_response.argtypes = [C.c_void_p, C.c_double, C.c_int, C.c_int, dp, dp]
        L.orc_green_react.argtypes = [C.c_void_p, C.c_int, dp, C.c_int, dp, C.c_double, dp, dp]
        L.orc_green_react_ab.argtypes = [C.c_void_p, C.c_int, dp, C.c_int, dp, C.c_int, C.c_int, C.c_double, dp, dp]
        L.orc_direct.argtypes = [C.c_void_p, C.c_int64, dp, dp, ip, C.c_int64, lp, C.c_int, C.c_int, dp, dp]
        L.orc_S_table.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                  C.c_double, C.c_double, C.c_int, C.c_double, dp]
        L.orc_image_z.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double]
        L.orc_image_z.restype = C.c_double
        L.orc_layer_of.argtypes = [C.c_void_p, C.c_double]
        L.orc_tree_root.argtypes = [C.c_void_p, C.c_int64, dp, ip, C.c_int, C.c_int, dp]
        L.orc_tree_keys.argtypes = [C.c_void_p, C.c_int64, dp, ip, C.c_int, C.c_int, C.c_int, dp, C.c_int,
                                    up, lp, ip]
        L.orc_tree_keys.restype = C.c_int64
        L.orc_level_boxes.argtypes = [up, C.c_int64, C.c_int, C.c_int, up]
        L.orc_level_boxes.restype = C.c_int64
        L.orc_lists.argtypes = [up, C.c_int64, up, C.c_int64, C.c_int, C.c_int, C.c_int, lp, lp]
        L.orc_lists.restype = C.c_int64
        L.orc_morton.argtypes = [C.c_int, C.c_int, C.c_int]
        L.orc_morton.restype = C.c_uint64
        L.orc_num_threads.restype = C.c_int
        _lib = L
    return _lib


class _Medium(C.Structure):
    _fields_ = [("L", C.c_int), ("d", C.c_double * MAXL), ("eps", C.c_double * MAXL),
                ("lam", C.c_double * MAXL)]


def _p(a, t=C.c_double):
    return a.ctypes.data_as(C.POINTER(t))


class Medium:
    """Layered medium: interfaces d[0] > ... > d[L-1], eps[0..L], lam[0..L] (Sec. 2.1)."""

    def __init__(self, d, eps, lam):
        self.d = np.asarray(d, float)
        self.eps = np.asarray(eps, float)
        self.lam = np.asarray(lam, float)
        self.L = len(self.d)
        assert len(self.eps) == self.L + 1 and len(self.lam) == self.L + 1
        m = _Medium()
        m.L = self.L
        for i, v in enumerate(self.d):
            m.d[i] = v
        for i in range(self.L + 1):
            m.eps[i] = self.eps[i]
            m.lam[i] = self.lam[i]
        self._m = m

    @property
    def ptr(self):
        return C.byref(self._m)

    def layer_of(self, z):
        return lib().orc_layer_of(self.ptr, float(z))


def layer_response(md, lr, lp, b):
    """sigma^{1b}_{k,lp}, sigma^{2b}_{k,lp} for k = 0..L at lambda_rho = lr."""
    s1 = np.zeros(md.L + 1)
    s2 = np.zeros(md.L + 1)
    rc = lib().orc_layer_response(md.ptr, float(lr), int(lp), int(b), _p(s1), _p(s2))
    if rc:
        raise ValueError("layer_response rc=%d" % rc)
    return s1, s2


def sigma(md, lr, l, lp, a, b):
    s1, s2 = layer_response(md, lr, lp, b)
    return s1[l] if a == 1 else s2[l]


def green_react(md, l, r, lp, rp, tol=1e-14):
    """(G^R_{l lp}(r, rp), -grad_r G^R) by adaptive quadrature."""
    r = np.ascontiguousarray(r, float)
    rp = np.ascontiguousarray(rp, float)
    phi = np.zeros(1)
    f = np.zeros(3)
    rc = lib().orc_green_react(md.ptr, int(l), _p(r), int(lp), _p(rp), float(tol), _p(phi), _p(f))
    if rc:
        raise ValueError("green_react rc=%d" % rc)
    return phi[0], f


def green_react_ab(md, l, r, lp, rp, a, b, tol=1e-14):
    """One reaction component u^{ab}_{l lp}(r, rp) and its -grad_r (Sec. 2.2)."""
    r = np.ascontiguousarray(r, float)
    rp = np.ascontiguousarray(rp, float)
    phi = np.zeros(1)
    f = np.zeros(3)
    rc = lib().orc_green_react_ab(md.ptr, int(l), _p(r), int(lp), _p(rp), int(a), int(b), float(tol), _p(phi), _p(f))
    if rc:
        raise ValueError("green_react_ab rc=%d" % rc)
    return phi[0], f


def direct(md, q, xyz, layer, targets=None, parts=3, nodes=16):
    """Direct O(N^2) potential and field at the targets (all if None); parts: 1 free, 2 reaction."""
    q = np.ascontiguousarray(q, float)
    xyz = np.ascontiguousarray(xyz, float).reshape(-1, 3)
    layer = np.ascontiguousarray(layer, np.int32)
    n = len(q)
    if targets is None:
        tidx = None
        nt = n
    else:
        tidx = np.ascontiguousarray(targets, np.int64)
        nt = len(tidx)
    phi = np.zeros(nt)
    field = np.zeros((nt, 3))
    rc = lib().orc_direct(md.ptr, n, _p(q), _p(xyz), _p(layer, C.c_int), nt,
                          None if tidx is None else _p(tidx, C.c_int64), int(parts), int(nodes),
                          _p(phi), _p(field))
    if rc:
        raise ValueError("direct rc=%d" % rc)
    return phi, field


def S_table(md, l, lp, a, b, h, rho, zt, zs, Kmax, tol=1e-13):
    """Scaled Sommerfeld integrals h^K S_{K d, ij}; returns array [K, d, i, j] (d <= K)."""
    out = np.zeros((Kmax + 1) * (Kmax + 1) * 4)
    rc = lib().orc_S_table(md.ptr, l, lp, a, b, float(h), float(rho), float(zt), float(zs), Kmax,
                           float(tol), _p(out))
    if rc:
        raise ValueError("S_table rc=%d" % rc)
    return out.reshape(Kmax + 1, Kmax + 1, 2, 2)


def image_z(md, l, a, lp, b, zp):
    return lib().orc_image_z(md.ptr, l, a, lp, b, float(zp))


def tree_root(md, xyz, layer, l, a):
    xyz = np.ascontiguousarray(xyz, float).reshape(-1, 3)
    layer = np.ascontiguousarray(layer, np.int32)
    out = np.zeros(4)
    lib().orc_tree_root(md.ptr, len(layer), _p(xyz), _p(layer, C.c_int), l, a, _p(out))
    return out


def tree_keys(md, xyz, layer, l, a, D, root, kind):
    """Morton keys at depth D of the group's targets (kind 0) or images (kind 1), unsorted,
    with the source charge index and image type (2*l' + b - 1) of each point."""
    xyz = np.ascontiguousarray(xyz, float).reshape(-1, 3)
    layer = np.ascontiguousarray(layer, np.int32)
    n = len(layer)
    keys = np.zeros(2 * n + 1, np.uint64)
    src = np.zeros(2 * n + 1, np.int64)
    typ = np.zeros(2 * n + 1, np.int32)
    root = np.ascontiguousarray(root, float)
    c = lib().orc_tree_keys(md.ptr, n, _p(xyz), _p(layer, C.c_int), l, a, D, _p(root), kind,
                            _p(keys, C.c_uint64), _p(src, C.c_int64), _p(typ, C.c_int))
    return keys[:c], src[:c], typ[:c]


def level_boxes(keys, D, lev):
    keys = np.ascontiguousarray(keys, np.uint64)
    out = np.zeros(max(1, len(keys)), np.uint64)
    c = lib().orc_level_boxes(_p(keys, C.c_uint64), len(keys), D, lev, _p(out, C.c_uint64))
    return out[:c]


def lists(tboxes, sboxes, lev, kind, ws=1):
    """CSR interaction lists (kind 0 far/V, kind 1 near/U) at level lev, separation ws boxes."""
    tb = np.ascontiguousarray(tboxes, np.uint64)
    sb = np.ascontiguousarray(sboxes, np.uint64)
    off = np.zeros(len(tb) + 1, np.int64)
    tot = lib().orc_lists(_p(tb, C.c_uint64), len(tb), _p(sb, C.c_uint64), len(sb), lev, kind, int(ws),
                          _p(off, C.c_int64), None)
    idx = np.zeros(max(1, tot), np.int64)
    lib().orc_lists(_p(tb, C.c_uint64), len(tb), _p(sb, C.c_uint64), len(sb), lev, kind, int(ws),
                    _p(off, C.c_int64), _p(idx, C.c_int64))
    return off, idx[:tot]


def morton(ix, iy, iz):
    return lib().orc_morton(ix, iy, iz)


def num_threads():
    return lib().orc_num_threads()
