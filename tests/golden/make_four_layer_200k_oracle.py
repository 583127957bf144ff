"""Write four_layer_200k_oracle.json: the oracle's potential and field at 100 sampled charges of
the differentiation workload (four-layer medium d = (0, -1, -2), eps = (1, 4, 2, 8),
lambda = (0.3, 1, 0.6, 1.5), N = 200,000 spread over all layers; the seeded generator's default
seed).  With E = 1/2 sum q phi, dE/dq_j = phi_j and the force on charge j is q_j field_j
(reciprocity of the layered Green's function), so these values check an adjoint at full size.

Charges: 25 per layer, drawn without replacement by numpy's PCG64 seeded with 2002013344, in
ascending order.  Uses only oracle/ and the input generator; about 2 minutes on 8 cores.  Run from
the repository root:  python tests/golden/make_four_layer_200k_oracle.py
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

N = 200000
SEED = inputs.BASE_SEED + 4
PER_LAYER = 25


def sample_targets(layer, per_layer, seed):
    rng = np.random.default_rng(seed)
    out = []
    for k in range(int(layer.max()) + 1):
        out.extend(rng.choice(np.nonzero(layer == k)[0], size=per_layer, replace=False).tolist())
    return sorted(int(i) for i in out)


def main():
    w = inputs.workload("four_layer", n=N, seed=SEED)
    md = oracle.Medium(**w["medium"])
    tg = sample_targets(w["layer"], PER_LAYER, SEED)
    t0 = time.time()
    phi, field = oracle.direct(md, w["q"], w["xyz"], w["layer"], targets=np.array(tg))
    out = {"what": "oracle phi and field at sampled charges of the four-layer N = 200k workload",
           "workload": "four_layer", "n": N, "seed": SEED, "per_layer": PER_LAYER, "targets": tg,
           "q": [float(w["q"][i]) for i in tg], "phi": phi.tolist(), "field": field.tolist(),
           "oracle_seconds": time.time() - t0, "oracle_threads": oracle.num_threads()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "four_layer_200k_oracle.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")
    print("wrote %s (%d targets, %.0f s)" % (path, len(tg), out["oracle_seconds"]))


if __name__ == "__main__":
    main()
