"""Multi-rank host logic on CPU with the gloo backend (world size 2).  bench.py: every rank
evaluates its own independent system (distinct seeds, no collective on the data path), the job
time is the slowest rank's, and throughput counts the targets of all ranks.  multigpu: one
evaluation split into disjoint units per rank plus one FP64 sum-reduce equals the one-rank result."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2002_01334_gb300 import inputs


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = inputs.workload("three_layer", n=64, seed=bench.rank_seed(rank))
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slower one
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        out[rank] = (ms, float(np.sum(w["q"])), bench.job_throughput(world, 64, 3, ms))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_distinct_systems():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as man:
        out = man.dict()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, out)) for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
            assert p.exitcode == 0
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0
    assert res[0][1] != res[1][1]  # independent systems per rank
    assert res[0][2] == pytest.approx(2 * 64 * 3 / 0.015)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(7.5, None, "cpu") == 7.5
    assert bench.job_throughput(1, 1000, 2, 1000.0) == 2000.0


def test_profiled_traffic_reads_a_summary(tmp_path):
    f = tmp_path / "t.md"
    f.write_text("text\ntraffic_bytes_per_eval k_x 42\n")
    assert bench.profiled_traffic("k_x", str(f)) == 42
    assert bench.profiled_traffic("k_x", str(tmp_path / "missing.md")) is None


def test_per_layer_errors_match_their_definition():
    ref = torch.tensor([1.0, -2.0, 4.0, 0.5, 3.0], dtype=torch.float64)
    a = ref + torch.tensor([0.1, 0.0, -0.2, 0.05, 0.0], dtype=torch.float64)
    layer = torch.tensor([0, 0, 1, 1, 2], dtype=torch.int32)
    e = bench.per_layer_errors(a, ref, layer, 4)
    assert e[0]["err2"] == pytest.approx(0.1 / np.sqrt(5.0))
    assert e[0]["errmax"] == pytest.approx(0.1 / 2.0)
    assert e[1]["err2"] == pytest.approx(np.sqrt(0.04 + 0.0025) / np.sqrt(16.25))
    assert e[2]["err2"] == 0.0 and e[3] is None


def test_oracle_fixture_errors_match_their_definition():
    fx = {"targets": [3, 9], "per_layer": 1, "seed": 5, "phi": [1.0, -2.0], "field": [[1, 0, 0], [0, 2, 0]]}
    got = bench.oracle_fixture_errors({"x": (np.array([1.1, -2.0]), np.array([[1, 0, 0], [0, 2, 0.2]]))}, fx,
                                      layers=[0, 1])
    assert got["targets"] == 2
    assert abs(got["x"]["relL2_phi"] - 0.1 / np.sqrt(5.0)) < 1e-15
    assert abs(got["x"]["relL2_field"] - 0.2 / np.sqrt(5.0)) < 1e-15
    assert got["x"]["errmax_phi_per_layer"] == pytest.approx([0.1, 0.0])
    assert got["x"]["errmax_field_per_layer"] == pytest.approx([0.0, 0.1])
    assert got["x"]["pass"] is False
    ok = bench.oracle_fixture_errors({"y": (np.array([1.0, -2.0]), np.array([[1, 0, 0], [0, 2, 1e-7]]))}, fx)
    assert ok["y"]["pass"] is True and "errmax_phi_per_layer" not in ok["y"]


def test_paper_workload_option_names_its_own_metric_and_config():
    assert bench.metric_of("three_layer") == bench.METRIC
    assert bench.metric_of("paper_irregular") != bench.METRIC
    c = bench.workload_config(2861288, 5, "mixed", "paper_irregular")
    assert c["eps"] == [1.0, 8.6, 20.5] and c["lambda"] == [1.2, 0.5, 2.1] and c["p"] == 5
    assert bench.workload_config(1000000, 10, "mixed")["eps"] == [1.0, 2.0, 5.0]
    # the stored oracle sample belongs to the three-layer workload only
    seed = bench.rank_seed(0)
    assert bench.load_oracle_fixture(1000000, seed) is not None
    assert bench.load_oracle_fixture(1000000, seed, "paper_irregular") is None


def test_clock_summary_reads_median_max_and_active_reasons():
    """The clock record of the timed region: median SM clock, maximum, and the throttle reasons
    seen active, from nvidia-smi's CSV lines (malformed lines are skipped)."""
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1980, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2040, 2070, 1200.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "garbage", "0, N/A, 2070, 1, 0, a, b, c, d"]
    s = c.summary()
    assert s["sm_mhz"] == 2040.0 and s["sm_max_mhz"] == 2070.0 and s["reasons"] == ["sw_power_cap"]
    assert s["samples"] == 3
    assert bench.ClockSampler(0).summary()["samples"] == 0


# ---------------------------------------------------------------------------------------------
# one evaluation split across ranks (paper_2002_01334_gb300.multigpu): disjoint units of work,
# one FP64 sum-reduce; checked with the oracle's direct sum as each rank's evaluator
# ---------------------------------------------------------------------------------------------
def test_assignment_is_a_balanced_partition():
    from paper_2002_01334_gb300 import multigpu as M
    costs = M.unit_costs([333334, 333333, 333333])
    assert len(costs) == 6
    for world in (1, 2, 3, 4, 8):
        plan = M.assign(costs, world)
        got = sorted(k for p in plan for k in p)
        assert got == list(range(6))  # every unit exactly once
        loads = [sum(costs[k] for k in p) for p in plan]
        # LPT: no rank above the optimum by more than the largest unit
        assert max(loads) <= sum(costs) / world + max(costs) + 1e-9
    assert M.assign(costs, 2) == M.assign(list(costs), 2)  # deterministic


def test_group_mask_of_units():
    from paper_2002_01334_gb300 import multigpu as M
    # units: (0, free) (0, react) (1, free) (1, react) (2, free) (2, react)
    assert M.group_mask([0], 3) == [1, 1, 0, 0, 0, 0]
    assert M.group_mask([3, 4], 3) == [0, 0, 2, 2, 1, 1]
    assert M.group_mask(range(6), 3) == [3] * 6


def _partition_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        from paper_2002_01334_gb300 import multigpu as M
        w = inputs.workload("three_layer", n=240, seed=77)
        md = oracle.Medium(**w["medium"])
        n, nl = len(w["q"]), 3

        def ev(mask):  # the oracle's direct sum of the selected units, standing in for the GPU
            phi, fld = np.zeros(n), np.zeros((n, 3))
            for l in range(nl):
                tg = np.nonzero(w["layer"] == l)[0]
                for bit in (1, 2):
                    if (mask[2 * l] | mask[2 * l + 1]) & bit:
                        p, f = oracle.direct(md, w["q"], w["xyz"], w["layer"], targets=tg, parts=bit)
                        phi[tg] += p
                        fld[tg] += f
            return torch.tensor(phi), torch.tensor(fld)

        def red(t):
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
        counts = np.bincount(w["layer"], minlength=nl).tolist()
        phi, fld = M.partitioned(ev, n, nl, M.unit_costs(counts), rank, world, red)
        out[rank] = (phi.numpy().copy(), fld.numpy().copy())
    finally:
        dist.destroy_process_group()


def test_partitioned_evaluation_equals_one_rank():
    """Two gloo ranks take disjoint units (layer, free or reaction part), evaluate them, and one
    FP64 sum-reduce gives both ranks the whole potential and field: equal to the one-rank direct
    sum to rounding, and identical on the two ranks."""
    import oracle
    world = 2
    port = _free_port()
    out = mp.Manager().dict()
    mp.spawn(_partition_main, args=(world, port, out), nprocs=world, join=True)
    w = inputs.workload("three_layer", n=240, seed=77)
    ref_phi, ref_fld = oracle.direct(oracle.Medium(**w["medium"]), w["q"], w["xyz"], w["layer"])
    for r in range(world):
        phi, fld = out[r]
        assert np.abs(phi - ref_phi).max() <= 1e-13 * np.abs(ref_phi).max()
        assert np.abs(fld - ref_fld).max() <= 1e-13 * np.abs(ref_fld).max()
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])
