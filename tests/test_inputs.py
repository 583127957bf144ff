"""Seeded input generators (no GPU): the irregular bodies of the paper's three-layer example
(Sec. 4) and the box workloads keep their charges where the recipe puts them, reproducibly."""
import numpy as np

from paper_2002_01334_gb300 import inputs


def test_body_radius_closed_form():
    for a in (0.05, 0.1, 0.15):
        assert inputs.body_radius(a, 1.0) == 0.5  # poles: 35 - 30 + 3 = 8
        assert inputs.body_radius(a, -1.0) == 0.5
        # the minimum, at cos^2 = 3/7: 35 (9/49) - 30 (3/7) + 3 = -24/7
        assert np.isclose(inputs.body_radius(a, np.sqrt(3.0 / 7.0)), 0.5 - 10.0 * a / 7.0)
        assert np.isclose(inputs.body_radius(a, 0.0), 0.5 - a + 3.0 * a / 8.0)


def test_paper_irregular_workload_geometry():
    w = inputs.workload("paper_irregular")
    q, xyz, layer = w["q"], w["xyz"], w["layer"]
    assert w["medium"] == inputs.MEDIA["paper_three_layer"]
    assert [int((layer == k).sum()) for k in range(3)] == list(inputs.PAPER_COUNTS)
    assert np.all(np.abs(q) <= 1.0)
    d = w["medium"]["d"]
    for k, (a, zc) in enumerate(inputs.PAPER_BODIES):
        p = xyz[layer == k] - np.array([0.0, 0.0, zc])
        r = np.linalg.norm(p, axis=1)
        cos_t = np.where(r > 0, p[:, 2] / np.maximum(r, 1e-300), 1.0)
        assert np.all(r <= inputs.body_radius(a, cos_t) + 1e-15)
        z = xyz[layer == k, 2]
        lo = d[k] if k < len(d) else -np.inf
        hi = d[k - 1] if k > 0 else np.inf
        assert np.all((z > lo + 0.0999) & (z < hi - 0.0999))  # 0.1 from the interfaces
    assert len(set(layer[:3].tolist())) == 3  # interleaved, not sorted by layer


def test_generators_are_reproducible():
    a = inputs.workload("paper_irregular", seed=7)
    b = inputs.workload("paper_irregular", seed=7)
    c = inputs.workload("paper_irregular", seed=8)
    assert np.array_equal(a["xyz"], b["xyz"]) and np.array_equal(a["q"], b["q"])
    assert not np.array_equal(a["xyz"], c["xyz"])
    s = inputs.workload("paper_irregular", n=10000)
    assert len(s["q"]) == 10000
    t = inputs.workload("three_layer", n=3000, seed=3)
    for k, (lo, hi) in enumerate(inputs.THREE_LAYER_BOXES):
        z = t["xyz"][t["layer"] == k, 2]
        assert np.all((z >= lo) & (z <= hi))


def test_paper_irregular_oracle_fixture_matches_the_oracle():
    """The stored reference (tests/golden/make_paper_irregular_oracle.py) is reproduced by the
    oracle on the regenerated workload, so generator and fixture stay in step."""
    import json
    import os

    import oracle

    oracle.build()
    g = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_irregular_oracle.json")))
    w = inputs.workload("paper_irregular")
    md = oracle.Medium(**w["medium"])
    pick = [0, 101, 250, 355]
    tg = np.array([g["targets"][k] for k in pick])
    phi, fld = oracle.direct(md, w["q"], w["xyz"], w["layer"], targets=tg)
    assert np.allclose(phi, [g["phi"][k] for k in pick], rtol=1e-12, atol=0)
    assert np.allclose(fld, [g["field"][k] for k in pick], rtol=1e-12, atol=1e-15)


def test_benchmark_oracle_fixture_matches_the_oracle_and_the_bench_workload():
    """tests/golden/three_layer_1M_oracle.json (make_three_layer_1M_oracle.py, oracle only) is the
    sample the benchmark compares its FMM results with: same workload as the benchmark's rank 0,
    the stated target draw, and one stored target recomputed by the oracle."""
    import importlib.util
    import os

    import bench
    import oracle

    here = os.path.dirname(__file__)
    spec = importlib.util.spec_from_file_location("mk1m", os.path.join(here, "golden", "make_three_layer_1M_oracle.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    fx = bench.load_oracle_fixture(1000000, bench.rank_seed(0))
    assert fx is not None and fx["seed"] == mk.SEED and bench.load_oracle_fixture(999, mk.SEED) is None
    w = inputs.workload("three_layer", n=1000000, seed=bench.rank_seed(0))
    assert fx["targets"] == mk.sample_targets(w["layer"], fx["per_layer"], fx["seed"])
    assert len(fx["targets"]) == 1002 and len(set(fx["targets"])) == 1002
    oracle.build()
    md = oracle.Medium(**w["medium"])
    k = 9  # one stored target, recomputed (about 40 s of one core)
    phi, fld = oracle.direct(md, w["q"], w["xyz"], w["layer"], targets=np.array([fx["targets"][k]]))
    assert abs(phi[0] - fx["phi"][k]) <= 1e-12 * abs(phi[0])
    assert np.allclose(fld[0], fx["field"][k], rtol=1e-12, atol=1e-14)


def test_four_layer_200k_oracle_fixture_matches_the_oracle():
    """tests/golden/four_layer_200k_oracle.json (make_four_layer_200k_oracle.py, oracle only):
    the stated draw of 25 charges per layer and one stored charge recomputed by the oracle."""
    import importlib.util
    import json
    import os

    import oracle

    here = os.path.dirname(__file__)
    spec = importlib.util.spec_from_file_location("mk200k", os.path.join(here, "golden", "make_four_layer_200k_oracle.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    fx = json.load(open(os.path.join(here, "golden", "four_layer_200k_oracle.json")))
    w = inputs.workload("four_layer", n=fx["n"], seed=fx["seed"])
    assert fx["targets"] == mk.sample_targets(w["layer"], fx["per_layer"], fx["seed"])
    assert np.array_equal(np.array(fx["q"]), w["q"][fx["targets"]])
    oracle.build()
    md = oracle.Medium(**w["medium"])
    k = 57
    phi, fld = oracle.direct(md, w["q"], w["xyz"], w["layer"], targets=np.array([fx["targets"][k]]))
    assert abs(phi[0] - fx["phi"][k]) <= 1e-12 * abs(phi[0])
    assert np.allclose(fld[0], fx["field"][k], rtol=1e-12, atol=1e-14)


def test_batch_systems_follow_their_recipe():
    """The batching workload's generator: N log-uniform in [1e3, 6.4e4]; 2-4 layers with
    eps ~ U[1, 10], lambda ~ U[0.2, 2], finite thicknesses ~ U[0.5, 2], d_0 = 0; every charge of a
    system in one host layer, inside it by the stated margin, xy in the unit square."""
    import oracle
    systems = inputs.batch(nsys=40)
    assert len(systems) == 40
    for s in systems:
        md = s["medium"]
        d, eps, lam = np.asarray(md["d"]), np.asarray(md["eps"]), np.asarray(md["lam"])
        n = len(s["q"])
        assert 1000 <= n <= 64000 and 2 <= len(eps) <= 4 and len(d) == len(eps) - 1
        assert d[0] == 0.0 and np.all(np.diff(d) < 0) and np.all((-np.diff(d) >= 0.5) & (-np.diff(d) <= 2.0))
        assert np.all((eps >= 1) & (eps <= 10)) and np.all((lam >= 0.2) & (lam <= 2.0))
        assert len(np.unique(s["layer"])) == 1
        o = oracle.Medium(d, eps, lam)
        host = int(s["layer"][0])
        assert all(o.layer_of(z) == host for z in s["xyz"][:200, 2])
        assert np.all(np.abs(s["xyz"][:, :2]) <= 0.5) and np.all(np.abs(s["q"]) <= 1.0)
        zs = s["xyz"][:, 2]
        top = d[host - 1] if host > 0 else np.inf
        bot = d[host] if host < len(d) else -np.inf
        assert np.all(zs < top - 0.04) and np.all(zs > bot + 0.04)
