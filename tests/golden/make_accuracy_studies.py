"""Accuracy studies quoted in the design notes, rerun from the oracle alone (the oracle's CPU FMM
against its direct sum).  Run from the repository root:

    python tests/golden/make_accuracy_studies.py separation   # free part, one- and two-box, p = 4..14
    python tests/golden/make_accuracy_studies.py reaction     # reaction part at p = 10, 12, 14 (one-box)
    python tests/golden/make_accuracy_studies.py recurrence    # table-route T: forward-recurred vs exact tables

All use the three-layer test workload of the GPU tests (N = 3000, seed 21; N = 400 for the
recurrence study), uniform depth 4 (3), and the oracle's direct sum as reference.  Slow: minutes
to an hour each on one core.
"""
import math
import sys
import time

import numpy as np

import os

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import Medium, S_table, direct  # noqa: E402
from oracle import expansions as E  # noqa: E402
from oracle import fmm  # noqa: E402


def _workload(n, seed=21):
    from paper_2002_01334_gb300 import inputs
    return inputs.workload("three_layer", n=n, seed=seed)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def separation():
    w = _workload(3000)
    md = Medium(**w["medium"])
    ref = direct(md, w["q"], w["xyz"], w["layer"], parts=1)
    for ws, orders in ((1, (4, 6, 8, 10, 12, 14)), (2, (4, 6, 8, 10))):
        for p in orders:
            t = time.time()
            a, fa = fmm.free_fmm(md, w["q"], w["xyz"], w["layer"], p, 4, ws)
            print("free, separation %d, p=%2d: phi %.2e field %.2e (%.0f s)"
                  % (ws, p, _rel(a, ref[0]), _rel(fa, ref[1]), time.time() - t), flush=True)


def reaction():
    w = _workload(3000)
    md = Medium(**w["medium"])
    ref = direct(md, w["q"], w["xyz"], w["layer"], parts=2)
    for p in (10, 12, 14):
        t = time.time()
        a, fa = fmm.react_fmm(md, w["q"], w["xyz"], w["layer"], p, 4)
        print("reaction, p=%d: phi %.2e field %.2e (%.0f s)" % (p, _rel(a, ref[0]), _rel(fa, ref[1]), time.time() - t),
              flush=True)


class TableM2L:
    """Reaction M2L by the table route of Sec. 3.5 (eqs. coefintable, metoletableform), the tables
    by direct quadrature of every entry, or (recurrence="forward") their columns d = 0, 1 continued
    by eq. recurrence1.  Same interface as fmm.ReactionM2L."""

    def __init__(self, md, l, lp, a, b, p, h, recurrence=None):
        self.md, self.l, self.lp, self.a, self.b, self.p, self.h, self.rec = md, l, lp, a, b, p, h, recurrence
        idx = E._nm(p)
        lam, lamp = md.lam[l], md.lam[lp]
        self.terms = []
        for x, (n, m) in enumerate(idx):
            for y, (nu, mu) in enumerate(idx):
                i, j, Cs = E.legendre_product_coeffs(n, m, nu, mu, lam, lamp)
                M = mu - m
                Ns = np.array([abs(m) + abs(mu) + 2 * s + 1 for s in range(len(Cs))])
                Ct = np.array([math.sqrt(math.factorial(N + M) * math.factorial(N - M)) for N in Ns]) * Cs
                sg = (-1.0) ** n if a == 1 else (-1.0) ** (m + nu + mu)
                self.terms.append((x, y, i, j, M, Ns, Ct * sg * (1j) ** M * ((-1.0) ** abs(M) if M < 0 else 1.0)))
        self.k = np.array([[mu - m for _, mu in idx] for _, m in idx])
        self.K = len(idx)
        self.cache = {}

    def T(self, rho, zt, zs):
        rho = math.sqrt(round((rho / self.h) ** 2)) * self.h  # the class's exact rho^2 in box units
        key = (round(rho, 12), round(zt, 12), round(zs, 12))
        if key not in self.cache:
            h = self.h
            S = S_table(self.md, self.l, self.lp, self.a, self.b, h, rho, zt, zs, 2 * self.p + 3)
            if self.rec == "forward":
                S = E.forward_recurrence(S, rho / h)
            hp = h ** -np.arange(2 * self.p + 4, dtype=float)
            T = np.zeros((self.K, self.K), complex)
            for (x, y, i, j, M, Ns, Ct) in self.terms:
                T[x, y] = (Ct * S[Ns, abs(M), i, j] * hp[Ns]).sum()
            self.cache[key] = T
        return self.cache[key]

    def apply(self, rct, rcs, M):
        d = rct - rcs
        rho, ph = math.hypot(d[0], d[1]), math.atan2(d[1], d[0])
        dI = self.md.d[self.l] if self.a == 1 else self.md.d[self.l - 1]
        zt, zs = (rct[2] - dI, dI - rcs[2]) if self.a == 1 else (dI - rct[2], rcs[2] - dI)
        return (np.exp(1j * self.k * ph) * self.T(rho, zt, zs)) @ M


def recurrence():
    w = _workload(400)
    md = Medium(**w["medium"])
    ref = direct(md, w["q"], w["xyz"], w["layer"], parts=2)
    orig = fmm.ReactionM2L
    try:
        for p in (6, 10, 12, 14):
            out = {}
            for rec in (None, "forward"):
                fmm.ReactionM2L = lambda md_, l, lp, a, b, p_, h, rmax, rec=rec: TableM2L(md_, l, lp, a, b, p_, h, rec)
                out[rec] = fmm.react_fmm(md, w["q"], w["xyz"], w["layer"], p, 3)
            ex, fw = out[None], out["forward"]
            print("p=%d: exact tables vs direct %.2e / %.2e; recurred vs exact tables %.2e / %.2e"
                  % (p, _rel(ex[0], ref[0]), _rel(ex[1], ref[1]), _rel(fw[0], ex[0]), _rel(fw[1], ex[1])), flush=True)
    finally:
        fmm.ReactionM2L = orig


if __name__ == "__main__":
    {"separation": separation, "reaction": reaction, "recurrence": recurrence}[sys.argv[1]]()
