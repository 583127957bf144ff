"""Write three_layer_1M_oracle.json: the oracle's potential and field at 1002 sampled targets of the
benchmark workload (three-layer medium, N = 1,000,000, the seeded generator's default seed).

Targets: 334 per layer, drawn without replacement by numpy's PCG64 seeded with 2002013342, in
ascending order.  Values: the oracle's direct sum (free part over the target's layer, reaction
part over all charges), FP64.  Uses only oracle/ and the input generator; about 30 core-seconds
per target (an hour on 8 cores).  Progress is kept in a sibling file ending in .partial, so an
interrupted run resumes where it stopped.  Run from the repository root:
    python tests/golden/make_three_layer_1M_oracle.py
"""
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from paper_2002_01334_gb300 import inputs  # noqa: E402

N = 1000000
SEED = inputs.BASE_SEED + 2
PER_LAYER = 334
CHUNK = 48


def sample_targets(layer, per_layer, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(int(layer.max()) + 1):
        idx = np.nonzero(layer == k)[0]
        out.extend(rng.choice(idx, size=per_layer, replace=False).tolist())
    return sorted(int(i) for i in out)


def main():
    w = inputs.workload("three_layer", n=N, seed=SEED)
    md = oracle.Medium(**w["medium"])
    tg = sample_targets(w["layer"], PER_LAYER, SEED)
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "three_layer_1M_oracle.json")
    part = path + ".partial"
    done = {"phi": [], "field": [], "seconds": 0.0}
    if os.path.exists(part):
        with open(part) as f:
            done = json.load(f)
    while len(done["phi"]) < len(tg):
        k0 = len(done["phi"])
        sel = np.array(tg[k0:k0 + CHUNK])
        t0 = time.time()
        phi, field = oracle.direct(md, w["q"], w["xyz"], w["layer"], targets=sel)
        done["phi"].extend(phi.tolist())
        done["field"].extend(field.tolist())
        done["seconds"] += time.time() - t0
        with open(part + ".tmp", "w") as f:
            json.dump(done, f)
        os.replace(part + ".tmp", part)
        print("%d / %d targets (%.0f s)" % (len(done["phi"]), len(tg), done["seconds"]), flush=True)
    out = {"what": "oracle phi and field at sampled targets of the three-layer N = 1M workload",
           "workload": "three_layer", "n": N, "seed": SEED, "per_layer": PER_LAYER,
           "targets": tg, "phi": done["phi"], "field": done["field"],
           "oracle_seconds": done["seconds"], "oracle_threads": oracle.num_threads()}
    with open(path, "w") as f:
        json.dump(out, f)
        f.write("\n")
    os.remove(part)
    print("wrote %s (%d targets, %.0f s)" % (path, len(tg), out["oracle_seconds"]))


if __name__ == "__main__":
    main()
