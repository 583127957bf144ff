"""Write me_convergence_e1.json: the single-source ME convergence example of Sec. 3.4.

Three-layer medium eps = (1, 8.6, 20.5), lambda = (1.2, 0.5, 2.1), interfaces d = (0, -1.2);
source r' = (0.625, 0.5, -0.1) in the middle layer; components u~^{11}_{11} and u~^{22}_{11}
with ME centres (0.6, 0.6, -2.4) and (0.6, 0.6, 0.2); targets (0.5, 0.625, z) for
z = -0.1, -0.6, -1.1.  For each (component, target) it stores the oracle's direct component
value u and the relative error of the ME truncated at p = 0..pmax, with the reference rate
(|r'_ab - r_c| / |r - r_c|)^{p+1}.  The paper shows these curves as a figure only.

Uses only oracle/ (direct component by adaptive quadrature; ME by oracle/expansions.py).
Run from the repository root:  python tests/golden/make_me_convergence.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import expansions as E  # noqa: E402

MEDIUM = dict(d=[0.0, -1.2], eps=[1.0, 8.6, 20.5], lam=[1.2, 0.5, 2.1])
SOURCE = [0.625, 0.5, -0.1]
CENTRES = {(1, 1): [0.6, 0.6, -2.4], (2, 2): [0.6, 0.6, 0.2]}
TARGETS = [[0.5, 0.625, -0.1], [0.5, 0.625, -0.6], [0.5, 0.625, -1.1]]
PMAX = 24


def main():
    md = oracle.Medium(**MEDIUM)
    rows = []
    for (a, b), rc in CENTRES.items():
        rimg = np.array([SOURCE[0], SOURCE[1], oracle.image_z(md, 1, a, 1, b, SOURCE[2])])
        for r in TARGETS:
            u, _ = oracle.green_react_ab(md, 1, np.array(r), 1, np.array(SOURCE), a, b)
            s = E.reaction_me(md, 1, 1, a, b, r, rimg, np.array(rc), PMAX)
            err = np.abs(s - u) / abs(u)
            rate = float(np.linalg.norm(rimg - rc) / np.linalg.norm(np.array(r) - rc))
            rows.append({"component": [a, b], "target": r, "centre": rc, "image": rimg.tolist(),
                         "u": float(u), "rate": rate,
                         "rel_err": [float(e) for e in err],
                         "reference": [rate ** (p + 1) for p in range(PMAX + 1)]})
    out = {"what": "relative error of the reaction-component ME truncated at p (Sec. 3.4 example)",
           "medium": MEDIUM, "source": SOURCE, "pmax": PMAX, "rows": rows}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "me_convergence_e1.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    for row in rows:
        print(row["component"], row["target"][2], " ".join("%.1e" % e for e in row["rel_err"][::4]))


if __name__ == "__main__":
    main()
