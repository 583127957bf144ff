"""The no-allocation entry point lpbfmm_stable_noalloc against lpbfmm_debug_stable: the same
kernels on the same inputs, so the tables agree bit for bit, call after call, although the
fixed scratch array is reused.  Collected last; also passes alone in a fresh process."""
import numpy as np
import pytest
import torch

from paper_2002_01334_gb300 import inputs
from paper_2002_01334_gb300 import lpbfmm as F

pytestmark = pytest.mark.gpu

# (l, a, l', b, h, rho^2 / h^2, k_t, k_s, Kmax)
CASES = [(1, 1, 1, 2, 0.3, 18, 0, 0, 19),
         (0, 1, 1, 1, 0.85, 5, 1, 1, 23),
         (1, 1, 1, 2, 0.3, 18, 0, 0, 19)]


def args_of(c):
    l, a, lp, b, h, r2, kt, ks, K = c
    return (l, a, lp, b, h, np.sqrt(r2) * h, (kt + .5) * h, (ks + .5) * h, K)


@pytest.fixture(scope="module")
def ctx():
    m = inputs.MEDIA["three_layer"]
    c = F.Context(m["d"], m["eps"], m["lam"], 10)
    yield c
    c.close()


def test_noalloc_matches_allocating_entry_point_call_after_call(ctx):
    for c in CASES:
        K = c[-1]
        ref = ctx.debug_stable(*args_of(c))
        out = torch.full(((K + 1) ** 2 * 4,), float("nan"), dtype=torch.float64, device="cuda")
        ctx.stable_noalloc(*args_of(c), out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().reshape(K + 1, K + 1, 2, 2)
        assert np.array_equal(got, ref), c


def test_noalloc_rejects_sizes_beyond_its_scratch(ctx):
    K = 24
    out = torch.zeros((K + 1) ** 2 * 4, dtype=torch.float64, device="cuda")
    with pytest.raises(F.LpbfmmError) as e:
        ctx.stable_noalloc(*args_of((1, 1, 1, 2, 0.3, 18, 0, 0, K)), out)
    assert e.value.code == 10
