"""Write paper_accuracy_e2.json: the accuracy-against-p experiment of Sec. 4 on the paper's own
workload, computed by the oracle's CPU FMM.

Workload: the paper's three-layer medium (eps = (1, 8.6, 20.5), lambda = (1.2, 0.5, 2.1),
interfaces 0 and -1.2) with 912 + 640 + 1296 charges in its three irregular bodies (the seeded
generator's default seed).  FMM: oracle/fmm.py (free part + all reaction components) on uniform
trees of depth 4 for every group.  Reference: the oracle's direct sum.  Errors per layer, in the
paper's form: Err_2 = ||phi - phi_ref||_2 / ||phi_ref||_2 and Err_max = max|phi - phi_ref| /
max|phi_ref| over the charges of that layer; the same for the field (all three components).
The paper shows this experiment only as a figure.  Uses only oracle/ and the input generator;
several minutes on one core.  Run from the repository root:
    python tests/golden/make_paper_accuracy.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import fmm  # noqa: E402
from paper_2002_01334_gb300 import inputs  # noqa: E402

DEPTH = 4
ORDERS = [2, 4, 6, 8, 10]


def layer_errors(a, ref, layer):
    out = []
    for k in range(int(layer.max()) + 1):
        s = layer == k
        d, r = np.abs(a[s] - ref[s]), np.abs(ref[s])
        out.append({"layer": k, "err2": float(np.linalg.norm(d) / np.linalg.norm(r)), "errmax": float(d.max() / r.max())})
    return out


def main():
    w = inputs.workload("paper_irregular")
    md = oracle.Medium(**w["medium"])
    ref_phi, ref_fld = oracle.direct(md, w["q"], w["xyz"], w["layer"])
    rows = []
    for p in ORDERS:
        t0 = time.time()
        phi, fld = fmm.fmm(md, w["q"], w["xyz"], w["layer"], p, DEPTH)
        rows.append({"p": p, "phi": layer_errors(phi, ref_phi, w["layer"]),
                     "field": layer_errors(fld, ref_fld, w["layer"]),
                     "relL2_phi": float(np.linalg.norm(phi - ref_phi) / np.linalg.norm(ref_phi)),
                     "relL2_field": float(np.linalg.norm(fld - ref_fld) / np.linalg.norm(ref_fld)),
                     "seconds": time.time() - t0})
        print(p, "%.2e %.2e (%.0f s)" % (rows[-1]["relL2_phi"], rows[-1]["relL2_field"], rows[-1]["seconds"]), flush=True)
    out = {"what": "per-layer errors of the FMM against the direct sum on the paper's workload (Sec. 4)",
           "workload": "paper_irregular", "n": int(len(w["q"])), "counts": np.bincount(w["layer"]).tolist(),
           "depth": DEPTH, "rows": rows}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_accuracy_e2.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
