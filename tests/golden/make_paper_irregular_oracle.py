"""Writes paper_irregular_oracle.json: the oracle's potential and field (FP64 direct sum,
Sec. 2.2 eq. potential1) at every 8th charge of the paper's irregular-body three-layer workload
(Sec. 4; inputs.workload("paper_irregular") with its default seed and counts).  Calls only the
oracle and the input generator.  Run: python tests/golden/make_paper_irregular_oracle.py"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2002_01334_gb300 import inputs  # noqa: E402

STRIDE = 8


def main():
    oracle.build()
    w = inputs.workload("paper_irregular")
    md = oracle.Medium(**w["medium"])
    tg = np.arange(0, len(w["q"]), STRIDE)
    phi, fld = oracle.direct(md, w["q"], w["xyz"], w["layer"], targets=tg)
    out = {
        "source": "oracle.direct (FP64 direct sum) on inputs.workload('paper_irregular'), every %d-th charge"
                  % STRIDE,
        "paper": "Sec. 4, three-layer example with irregular bodies; Sec. 2.2 eq. potential1",
        "medium": w["medium"], "counts": list(inputs.PAPER_COUNTS), "seed": inputs.BASE_SEED + 5,
        "targets": tg.tolist(), "phi": [float(v) for v in phi],
        "field": [[float(v) for v in row] for row in fld],
    }
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_irregular_oracle.json"), "w") as f:
        json.dump(out, f, separators=(",", ":"))


if __name__ == "__main__":
    main()
