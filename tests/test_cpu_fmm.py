"""CPU pins of the oracle's free-space FMM (oracle/fmm.py): with every expansion truncated at p
and nothing else approximated, it must converge geometrically in p to the direct sum (Sec. 3.1
expansions, one-box separation), for potential and field, at several tree depths.  It is the
reference against which a GPU FMM of the same tree and order can be compared to rounding."""
import numpy as np
import pytest

pytest.importorskip("scipy")

import oracle  # noqa: E402
from oracle import fmm  # noqa: E402
from paper_2002_01334_gb300 import inputs  # noqa: E402


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def w600():
    w = inputs.workload("three_layer", n=600, seed=31)
    md = oracle.Medium(**w["medium"])
    return w, md, oracle.direct(md, w["q"], w["xyz"], w["layer"], parts=1)


@pytest.mark.parametrize("D", [3, 4])
def test_free_fmm_converges_in_p_to_the_direct_sum(w600, D):
    w, md, ref = w600
    ep, ef = [], []
    for p in (2, 4, 6):
        phi, fld = fmm.free_fmm(md, w["q"], w["xyz"], w["layer"], p, D)
        ep.append(rel(phi, ref[0]))
        ef.append(rel(fld, ref[1]))
    assert ep[0] > 4 * ep[1] > 16 * ep[2] and ef[0] > 4 * ef[1] > 16 * ef[2], (ep, ef)
    assert ep[2] < 2e-4 and ef[2] < 1e-3, (ep, ef)


def test_free_fmm_at_depth_2_is_the_direct_sum(w600):
    """At depth 2 every pair of these charges is in the near lists (they fill one layer's cube,
    a small part of the group's root), so the FMM reduces to its exact near field."""
    w, md, ref = w600
    phi, fld = fmm.free_fmm(md, w["q"], w["xyz"], w["layer"], 2, 2)
    assert rel(phi, ref[0]) < 1e-13 and rel(fld, ref[1]) < 1e-13
