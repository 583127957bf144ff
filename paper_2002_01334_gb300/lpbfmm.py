"""Thin Python binding of liblpbfmm.so (ctypes; argument marshalling only).

Every step of the computation runs in the library's CUDA kernels; this module only passes
device pointers of torch tensors.  If the library has not been built it raises: there is no
CPU fallback.  Build with ``python -m paper_2002_01334_gb300.build``.
"""
import ctypes as C
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "liblpbfmm.so")
_lib = None

FP64 = 0
MIXED = 1
ERR_OOM = 7
STATUS = {
    0: "ok", 1: "invalid argument", 2: "invalid medium", 3: "truncation order out of range",
    4: "charge on an interface", 5: "layer_id does not match z", 6: "non-finite input",
    7: "out of device memory", 8: "CUDA error", 9: "device wait timed out", 10: "unsupported size",
}


class LpbfmmError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        super().__init__("%s: %s (code %d)" % (where, STATUS.get(code, "unknown"), code))


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("max_per_leaf", C.c_int), ("uniform_depth", C.c_int),
                ("separation", C.c_int), ("react_levels", C.c_int), ("stream", C.c_void_p)]


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("liblpbfmm.so is not built (expected at %s); run "
                               "`python -m paper_2002_01334_gb300.build`" % LIB_PATH)
        L = C.CDLL(LIB_PATH)
        vp, dp, i64 = C.c_void_p, C.POINTER(C.c_double), C.c_int64
        L.lpbfmm_default_opts.argtypes = [C.POINTER(Opts)]
        L.lpbfmm_create.argtypes = [C.c_int, dp, dp, dp, C.c_int, C.c_double, C.POINTER(Opts), C.POINTER(vp)]
        L.lpbfmm_eval.argtypes = [vp, i64, vp, vp, vp, vp, vp]
        L.lpbfmm_eval_parts.argtypes = [vp, i64, vp, vp, vp, C.c_int, vp, vp]
        L.lpbfmm_eval_groups.argtypes = [vp, i64, vp, vp, vp, C.POINTER(C.c_int32), vp, vp]
        L.lpbfmm_adjoint.argtypes = [vp, i64, vp, vp, vp, vp, vp, vp]
        L.lpbfmm_eval_batched.argtypes = [C.c_int, C.POINTER(vp), C.POINTER(i64), vp, vp, vp, vp, vp]
        L.lpbfmm_debug_tree.argtypes = [vp, C.c_int, C.c_int, dp, C.POINTER(i64), C.POINTER(i64),
                                        C.POINTER(C.c_int), vp, vp, vp, vp, vp]
        L.lpbfmm_debug_adaptive_lists.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(i64), vp, i64]
        L.lpbfmm_debug_lists.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.POINTER(i64),
                                         C.POINTER(i64), vp, vp]
        L.lpbfmm_debug_stable.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                          C.c_double, C.c_double, C.c_int, dp]
        L.lpbfmm_stable_noalloc.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                            C.c_double, C.c_double, C.c_int, vp]
        L.lpbfmm_debug_array.argtypes = [vp, C.c_int, C.c_int, C.c_char_p, C.c_int, vp, i64, C.POINTER(i64)]
        L.lpbfmm_last_counts.argtypes = [vp, C.POINTER(i64)]
        L.lpbfmm_status.argtypes = [vp]
        L.lpbfmm_strerror.argtypes = [C.c_int]
        L.lpbfmm_strerror.restype = C.c_char_p
        L.lpbfmm_destroy.argtypes = [vp]
        L.lpbfmm_destroy.restype = None
        L.lpbfmm_last_profile.argtypes = [vp, C.c_int, C.POINTER(C.c_char_p), C.POINTER(C.c_float),
                                          C.POINTER(C.c_int)]
        L.lpbfmm_host_table.argtypes = [C.c_int, C.c_int, dp, i64, C.POINTER(i64)]
        L.lpbfmm_measure_peak.argtypes = [C.c_int, dp]
        _lib = L
    return _lib


def _check(rc, where):
    if rc:
        raise LpbfmmError(rc, where)


def _dptr(t, dtype):
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA %s tensor" % dtype)
    return C.c_void_p(t.data_ptr())


def _darr(vals):
    a = (C.c_double * len(vals))(*[float(v) for v in vals])
    return a


class Context:
    """One medium (interfaces d, eps, lambda per layer) and truncation order p (lpbfmm_create);
    separation = 1 (one-box) or 2 (two-box) interaction lists, 0 = the library default (2)."""

    def __init__(self, d, eps, lam, p, tol=1e-14, precision=FP64, max_per_leaf=128, uniform_depth=0,
                 stream=None, separation=0, react_levels=None):
        L = lib()
        o = Opts()
        L.lpbfmm_default_opts(C.byref(o))
        o.precision = int(precision)
        o.max_per_leaf = int(max_per_leaf)
        o.uniform_depth = int(uniform_depth or 0)
        o.separation = int(separation or 0)
        if react_levels is not None:
            o.react_levels = int(react_levels)
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream()
        o.stream = C.c_void_p(stream.cuda_stream if stream is not None else 0)
        self.stream = stream
        h = C.c_void_p()
        self.d, self.eps, self.lam, self.p = list(d), list(eps), list(lam), int(p)
        _check(L.lpbfmm_create(len(self.d), _darr(self.d), _darr(self.eps), _darr(self.lam), self.p, float(tol),
                               C.byref(o), C.byref(h)), "lpbfmm_create")
        self.h = h

    def status(self):
        """Read and clear the device status word (0, or an error code such as a timed-out
        device wait); synchronizes the context's stream."""
        return int(lib().lpbfmm_status(self.h))

    def close(self):
        if getattr(self, "h", None) and self.h.value:
            lib().lpbfmm_destroy(self.h)
            self.h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def eval(self, q, xyz, layer, field=True, parts=3, out=None):
        """phi[n] and field[n,3] (float64 CUDA tensors) for float64 q[n], xyz[n,3], int32 layer[n]."""
        n = q.shape[0]
        if out is None:
            phi = torch.empty(n, dtype=torch.float64, device=q.device)
            fld = torch.empty((n, 3), dtype=torch.float64, device=q.device) if field else None
        else:
            phi, fld = out
        rc = lib().lpbfmm_eval_parts(self.h, n, _dptr(q, torch.float64), _dptr(xyz, torch.float64),
                                     _dptr(layer, torch.int32), int(parts), _dptr(phi, torch.float64),
                                     _dptr(fld, torch.float64) if fld is not None else None)
        _check(rc, "lpbfmm_eval")
        return phi, fld

    def eval_groups(self, q, xyz, layer, mask, field=True):
        """lpbfmm_eval_groups: the parts of the evaluation that mask (2 (L + 1) ints, entry 2 l + a - 1
        for target group (l, a): bit 0 free-space, bit 1 reaction) selects."""
        n = q.shape[0]
        phi = torch.empty(n, dtype=torch.float64, device=q.device)
        fld = torch.empty((n, 3), dtype=torch.float64, device=q.device) if field else None
        m = (C.c_int32 * len(mask))(*[int(v) for v in mask])
        rc = lib().lpbfmm_eval_groups(self.h, n, _dptr(q, torch.float64), _dptr(xyz, torch.float64),
                                      _dptr(layer, torch.int32), m, _dptr(phi, torch.float64),
                                      _dptr(fld, torch.float64) if fld is not None else None)
        _check(rc, "lpbfmm_eval_groups")
        return phi, fld

    def adjoint(self, q, xyz, layer, g_phi):
        n = q.shape[0]
        gq = torch.empty(n, dtype=torch.float64, device=q.device)
        gx = torch.empty((n, 3), dtype=torch.float64, device=q.device)
        rc = lib().lpbfmm_adjoint(self.h, n, _dptr(q, torch.float64), _dptr(xyz, torch.float64),
                                  _dptr(layer, torch.int32), _dptr(g_phi, torch.float64),
                                  _dptr(gq, torch.float64), _dptr(gx, torch.float64))
        _check(rc, "lpbfmm_adjoint")
        return gq, gx

    def counts(self):
        out = (C.c_int64 * 8)()
        _check(lib().lpbfmm_last_counts(self.h, out), "lpbfmm_last_counts")
        keys = ["m2l_free", "m2l_react", "p2p_pairs", "near_react_pairs", "targets", "images", "boxes", "launches"]
        return dict(zip(keys, list(out)))

    def profile(self):
        cap = 64
        names = (C.c_char_p * cap)()
        ms = (C.c_float * cap)()
        lc = (C.c_int * cap)()
        k = lib().lpbfmm_last_profile(self.h, cap, names, ms, lc)
        return [(names[i].decode(), ms[i], lc[i]) for i in range(max(k, 0))]

    # ---- diagnostics used by the tests ------------------------------------------------------
    def debug_tree(self, l, a):
        import numpy as np
        root = (C.c_double * 4)()
        nt, ni, D = C.c_int64(), C.c_int64(), C.c_int()
        _check(lib().lpbfmm_debug_tree(self.h, l, a, root, C.byref(nt), C.byref(ni), C.byref(D), None, None,
                                       None, None, None), "lpbfmm_debug_tree")
        kt = np.zeros(nt.value, np.uint64)
        st = np.zeros(nt.value, np.int64)
        ki = np.zeros(ni.value, np.uint64)
        si = np.zeros(ni.value, np.int64)
        ti = np.zeros(ni.value, np.int32)
        p = lambda a: C.c_void_p(a.ctypes.data)
        _check(lib().lpbfmm_debug_tree(self.h, l, a, root, C.byref(nt), C.byref(ni), C.byref(D), p(kt), p(st),
                                       p(ki), p(si), p(ti)), "lpbfmm_debug_tree")
        return dict(root=list(root), depth=D.value, keys_t=kt, src_t=st, keys_i=ki, src_i=si, type_i=ti)

    def debug_lists(self, l, a, lev, kind, src):
        import numpy as np
        nb, ne = C.c_int64(), C.c_int64()
        _check(lib().lpbfmm_debug_lists(self.h, l, a, lev, kind, src, C.byref(nb), C.byref(ne), None, None),
               "lpbfmm_debug_lists")
        off = np.zeros(nb.value + 1, np.int64)
        idx = np.zeros(max(ne.value, 1), np.int64)
        _check(lib().lpbfmm_debug_lists(self.h, l, a, lev, kind, src, C.byref(nb), C.byref(ne),
                                        C.c_void_p(off.ctypes.data), C.c_void_p(idx.ctypes.data)),
               "lpbfmm_debug_lists")
        return off, idx[:ne.value]

    def debug_adaptive_lists(self, l, a, s, ws=1):
        """Adaptive dual-tree lists of group (l, a)'s free-space tree (lpbfmm_debug_adaptive_lists):
        {'V', 'U', 'W', 'X'} -> set of ((target level, key), (source level, key))."""
        import numpy as np
        n = C.c_int64()
        _check(lib().lpbfmm_debug_adaptive_lists(self.h, l, a, s, ws, C.byref(n), None, 0), "debug_adaptive_lists")
        rec = np.zeros((max(n.value, 1), 5), np.int64)
        _check(lib().lpbfmm_debug_adaptive_lists(self.h, l, a, s, ws, C.byref(n), C.c_void_p(rec.ctypes.data),
                                                 n.value), "debug_adaptive_lists")
        out = {k: set() for k in "VUWX"}
        for kind, lt, kt, ls, ks in rec[:n.value].tolist():
            out["VUWX"[kind]].add(((lt, kt), (ls, ks)))
        return out

    def debug_array(self, l, a, name, lev, dtype):
        import numpy as np
        nb = C.c_int64()
        _check(lib().lpbfmm_debug_array(self.h, l, a, name.encode(), lev, None, 0, C.byref(nb)), "debug_array")
        out = np.zeros(nb.value, np.uint8)
        _check(lib().lpbfmm_debug_array(self.h, l, a, name.encode(), lev, C.c_void_p(out.ctypes.data), nb.value,
                                        C.byref(nb)), "debug_array")
        return out.view(dtype)

    def debug_stable(self, l, a, lp, b, h, rho, zt, zs, Kmax):
        import numpy as np
        out = np.zeros((Kmax + 1) * (Kmax + 1) * 4)
        _check(lib().lpbfmm_debug_stable(self.h, l, a, lp, b, float(h), float(rho), float(zt), float(zs), Kmax,
                                         out.ctypes.data_as(C.POINTER(C.c_double))), "lpbfmm_debug_stable")
        return out.reshape(Kmax + 1, Kmax + 1, 2, 2)

    def stable_noalloc(self, l, a, lp, b, h, rho, zt, zs, Kmax, out):
        """lpbfmm_stable_noalloc into the CUDA float64 tensor out ((Kmax+1)^2*4 elements), on
        the context's stream; the table of debug_stable computed without any allocation."""
        if out.dtype != torch.float64 or not out.is_cuda or out.numel() != (Kmax + 1) * (Kmax + 1) * 4:
            raise ValueError("out must be a CUDA float64 tensor of (Kmax+1)^2*4 elements")
        _check(lib().lpbfmm_stable_noalloc(self.h, l, a, lp, b, float(h), float(rho), float(zt), float(zs), Kmax,
                                           C.c_void_p(out.data_ptr())), "lpbfmm_stable_noalloc")
        return out


TABLE_GAUNT, TABLE_TPOLY, TABLE_PHAT_DIR, TABLE_SFAC = 0, 1, 2, 3
PEAK_FP32_FMA, PEAK_FP64_FMA = 0, 1


def measure_peak(which):
    """lpbfmm_measure_peak: the current device's measured FMA peak (TFLOP/s) in FP32 or FP64."""
    v = C.c_double()
    _check(lib().lpbfmm_measure_peak(int(which), C.byref(v)), "lpbfmm_measure_peak")
    return v.value


def host_table(which, p):
    """lpbfmm_host_table: one host-side table of lpbfmm_create for order p, as a flat float64
    numpy array (computed on the host; no device needed)."""
    import numpy as np
    L = lib()
    n = C.c_int64()
    _check(L.lpbfmm_host_table(which, p, None, 0, C.byref(n)), "lpbfmm_host_table")
    out = np.zeros(n.value)
    _check(L.lpbfmm_host_table(which, p, out.ctypes.data_as(C.POINTER(C.c_double)), n.value, C.byref(n)),
           "lpbfmm_host_table")
    return out


def eval_batched(ctxs, offsets, q, xyz, layer, field=True):
    n = q.shape[0]
    phi = torch.empty(n, dtype=torch.float64, device=q.device)
    fld = torch.empty((n, 3), dtype=torch.float64, device=q.device) if field else None
    hs = (C.c_void_p * len(ctxs))(*[c.h.value for c in ctxs])
    offs = (C.c_int64 * len(offsets))(*[int(o) for o in offsets])
    rc = lib().lpbfmm_eval_batched(len(ctxs), hs, offs, _dptr(q, torch.float64), _dptr(xyz, torch.float64),
                                   _dptr(layer, torch.int32), _dptr(phi, torch.float64),
                                   _dptr(fld, torch.float64) if fld is not None else None)
    _check(rc, "lpbfmm_eval_batched")
    return phi, fld


class Potential(torch.autograd.Function):
    """phi = FMM potential of charges q at positions xyz; backward by the library's adjoint
    (reciprocity of the layered Green's function): grad_q = phi[g], grad_xyz = -(q field[g] + g field[q])."""

    @staticmethod
    def forward(ctx_, context, q, xyz, layer):
        phi, _ = context.eval(q.detach().contiguous(), xyz.detach().contiguous(), layer, field=False)
        ctx_.context = context
        ctx_.save_for_backward(q, xyz, layer)
        return phi

    @staticmethod
    def backward(ctx_, g):
        q, xyz, layer = ctx_.saved_tensors
        gq, gx = ctx_.context.adjoint(q.detach().contiguous(), xyz.detach().contiguous(), layer,
                                      g.detach().contiguous().to(torch.float64))
        return None, gq, gx, None


def potential(context, q, xyz, layer):
    return Potential.apply(context, q, xyz, layer)
