"""Benchmark: targets/s (potential + field) of the layered-media screened-Coulomb FMM.

Workload (one step = one full evaluation, trees + tables + all passes): N = 1,000,000 charges
in the three-layer medium d = (0, -1.2), eps = (1, 2, 5), lambda = (0.5, 1, 0.8), split evenly
over three unit cubes (one per layer), q ~ U[-1, 1], p = 10, mixed precision.  Inputs are
resident in HBM; L2 is flushed (256 MB write) between timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload three_layer|paper_irregular] [--n N] [--p P]

--workload paper_irregular runs the same measurement on the paper's own charges (Sec. 4: three
irregular bodies in the medium eps = (1, 8.6, 20.5), lambda = (1.2, 0.5, 2.1)) under its own
metric name, for context beside the paper's CPU timings (potential only, p = 5, N up to
2,861,288); the default workload is the headline.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle (direct sum) on the host
cores on a bounded sample of the same workload.  With --gpus N > 1 (launched by
torch.distributed.run) every rank evaluates its own independent system of N charges (weak
scaling, no collective on the data path).
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "targets/sec (potential+field) N=1M 3-layer @relL2<=1e-6: mixed vs FP64 FMM"
# the paper's own workload (Sec. 4: charges in three irregular bodies, eps = (1, 8.6, 20.5),
# lambda = (1.2, 0.5, 2.1)), for context beside its CPU timings; not the headline metric
METRIC_PAPER = "targets/sec (potential+field) paper irregular-body 3-layer workload: mixed FMM"
# the batching form: 256 independent systems in random 2- to 4-layer media, one batched call
METRIC_BATCH = "targets/sec (potential+field) 256 independent systems N=1e3..6.4e4, p=8: batched mixed FMM"


def metric_of(workload):
    return {"three_layer": METRIC, "paper_irregular": METRIC_PAPER, "batch": METRIC_BATCH}[workload]
N_DEFAULT = 1000000
P_DEFAULT = 10


def rank_seed(rank):
    """Seed of rank r's independent system (weak scaling: every rank evaluates its own N charges)."""
    from paper_2002_01334_gb300 import inputs
    return inputs.BASE_SEED + 2 + 1000 * rank


def max_over_ranks(ms, dist, device):
    """The slowest rank's time (ms); the job's time is that of its slowest rank."""
    if dist is None:
        return float(ms)
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, n, steps, ms):
    """Targets per second of the whole job: world ranks x n targets x steps in ms."""
    return world * n * steps / (ms / 1000.0)


def profiled_traffic(kernel, path=None):
    """DRAM bytes per evaluation of a kernel at the benchmark size, from the committed ncu summary
    (a line 'traffic_bytes_per_eval <kernel> <bytes>'), or None when none is recorded."""
    path = path or os.path.join(ROOT, "profiles", "traffic_three_layer_1M_p10.md")
    try:
        for line in open(path):
            f = line.split()
            if len(f) == 3 and f[0] == "traffic_bytes_per_eval" and f[1] == kernel:
                return int(f[2])
    except OSError:
        pass
    return None


def per_layer_errors(a, ref, layer, nlayers):
    """Per layer k: relative L2 error ||a - ref|| / ||ref|| and relative max error
    max|a - ref| / max|ref| over the targets in layer k (the paper's Err_2 / Err_max form)."""
    out = []
    for k in range(nlayers):
        sel = layer == k
        if not bool(sel.any()):
            out.append(None)
            continue
        d, r = (a[sel] - ref[sel]).abs(), ref[sel].abs()
        out.append({"layer": k, "err2": float(d.norm() / r.norm()), "errmax": float(d.max() / r.max())})
    return out


def load_oracle_fixture(n, seed, workload="three_layer", path=None):
    """The oracle's stored potential and field at sampled targets of this workload (a committed
    fixture written from the oracle alone), or None when none is stored for (workload, n, seed)."""
    path = path or os.path.join(ROOT, "tests", "golden", "three_layer_1M_oracle.json")
    try:
        with open(path) as f:
            fx = json.load(f)
    except (OSError, ValueError):
        return None
    ok = fx.get("workload") == workload and fx.get("n") == n and fx.get("seed") == seed
    return fx if ok else None


GATE = 1e-6  # relative L2 bound of the accuracy gate (potential and field)


def oracle_fixture_errors(sampled, fx, layers=None):
    """Errors against the oracle at the fixture's targets; sampled maps a name to (phi, field) host
    arrays at those targets, in the fixture's order.  Relative L2 over the sample, and with the
    targets' layers the paper's per-layer Err_max (max |a - ref| / max |ref|, field rows as vectors);
    "pass" when both relative L2 errors are within GATE."""
    ref_phi = np.asarray(fx["phi"], float)
    ref_fld = np.asarray(fx["field"], float)
    out = {"targets": len(fx["targets"]), "gate": GATE,
           "sample": "%d targets per layer, drawn without replacement (seed %d); oracle direct sum, FP64"
                     % (fx["per_layer"], fx["seed"])}
    for name, (ph, fl) in sampled.items():
        ph, fl = np.asarray(ph), np.asarray(fl)
        r = {"relL2_phi": float(np.linalg.norm(ph - ref_phi) / np.linalg.norm(ref_phi)),
             "relL2_field": float(np.linalg.norm(fl - ref_fld) / np.linalg.norm(ref_fld))}
        if layers is not None:
            lay = np.asarray(layers)
            em_p, em_f = [], []
            for k in np.unique(lay):
                s = lay == k
                em_p.append(float(np.abs(ph[s] - ref_phi[s]).max() / np.abs(ref_phi[s]).max()))
                em_f.append(float(np.linalg.norm(fl[s] - ref_fld[s], axis=1).max() /
                                  np.linalg.norm(ref_fld[s], axis=1).max()))
            r["errmax_phi_per_layer"] = em_p
            r["errmax_field_per_layer"] = em_f
        r["pass"] = bool(r["relL2_phi"] <= GATE and r["relL2_field"] <= GATE)
        out[name] = r
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="three_layer", choices=["three_layer", "paper_irregular", "batch"])
    ap.add_argument("--n", type=int, default=N_DEFAULT)
    ap.add_argument("--p", type=int, default=P_DEFAULT)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="skip the search of leaf size and reaction depth (use the library defaults)")
    return ap.parse_args()


def workload_config(n, p, precision, workload="three_layer"):
    if workload == "paper_irregular":
        return {"workload": "paper irregular-body three-layer screened Coulomb (Sec. 4), N=%d, p=%d" % (n, p),
                "n": n, "p": p, "layers": 3, "interfaces": [0.0, -1.2], "eps": [1.0, 8.6, 20.5],
                "lambda": [1.2, 0.5, 2.1],
                "charges": "q~U[-1,1], uniform in the bodies r(theta) = 0.5 - a + (a/8)(35 cos^4 - 30 cos^2 + 3), "
                           "a = 0.1, 0.15, 0.05, centres z = 0.6, -0.6, -1.8, counts in the ratio 912:640:1296",
                "precision": precision, "l2": "flushed between steps (256 MB write)",
                "tree": "automatic depth by mean leaf occupancy (library default 128; the autotune object gives "
                        "the setting timed)", "separation": "two-box interaction lists"}
    return {"workload": "three-layer screened Coulomb, N=%d, p=%d" % (n, p), "n": n, "p": p, "layers": 3,
            "interfaces": [0.0, -1.2], "eps": [1.0, 2.0, 5.0], "lambda": [0.5, 1.0, 0.8],
            "charges": "q~U[-1,1], uniform in three unit cubes (one per layer)", "precision": precision,
            "l2": "flushed between steps (256 MB write)",
            "tree": "automatic depth by mean leaf occupancy (library default 128; the autotune object gives the "
                    "setting timed)",
            "separation": "two-box interaction lists"}


# ---------------------------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "50"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------------------------
# CPU oracle baseline (bounded sample of the same workload, scaled to targets/s over all sources)
# ---------------------------------------------------------------------------------------------
CPU_SOURCE_STRIDE = 10  # the oracle's bounded sample: every 10th charge as a source


def oracle_sample(w, n_targets, source_stride):
    import oracle
    md = oracle.Medium(**w["medium"])
    n = len(w["q"])
    sel = np.arange(0, n, source_stride)
    q, xyz, layer = w["q"][sel], w["xyz"][sel], w["layer"][sel]
    tg = np.arange(n_targets) * (len(sel) // max(n_targets, 1))
    t0 = time.perf_counter()
    oracle.direct(md, q, xyz, layer, targets=tg)
    dt = time.perf_counter() - t0
    frac = len(sel) / n
    return n_targets * frac / dt, dt, {"kind": "oracle", "cores": oracle.num_threads(),
                                       "sample": "%d targets x %d of %d sources (every %d-th charge); "
                                                 "targets/s scaled by the source fraction %.4f"
                                                 % (n_targets, len(sel), n, source_stride, frac)}


def run_reference(args, rank, world):
    if rank != 0:
        return
    from paper_2002_01334_gb300 import inputs
    import oracle
    oracle.build()
    w = inputs.workload(args.workload, n=args.n)
    cores = oracle.num_threads()
    nt, stride = max(2, cores), CPU_SOURCE_STRIDE
    for _ in range(args.warmup):
        oracle_sample(w, nt, stride)
    vals, times = [], []
    for _ in range(args.steps):
        v, dt, info = oracle_sample(w, nt, stride)
        vals.append(v)
        times.append(dt)
    value = args.steps * nt * (args.n // stride) / args.n / sum(times)
    info["value"] = value
    line = {"impl": "reference", "metric": metric_of(args.workload), "value": value, "unit": "targets/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * sum(times) / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args.n, args.p, "mixed", args.workload), "cpu_baseline": info,
            "e2e": {"value": value, "unit": "targets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
def run_ours(args, rank, world, local_rank):
    import torch
    from paper_2002_01334_gb300 import build as B
    B.build()
    from paper_2002_01334_gb300 import autotune
    from paper_2002_01334_gb300 import inputs
    from paper_2002_01334_gb300 import lpbfmm as F

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = inputs.workload(args.workload, n=args.n, seed=rank_seed(rank))
    m = w["medium"]
    q = torch.tensor(w["q"], device=dev)
    x = torch.tensor(w["xyz"], device=dev)
    l = torch.tensor(w["layer"], dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)
    settings, tuned = dict(autotune.DEFAULTS), None
    if not args.no_autotune:
        measure, close = autotune.cuda_measure(m, args.p, F.MIXED, q, x, l, stream=stream)
        settings, rows = autotune.search(autotune.SPACE, measure, start=autotune.DEFAULTS, repeats=2)
        close()
        tuned = {"method": "coordinate descent over %s in order; median of 2 CUDA-event timings of one evaluation "
                           "per setting" % ", ".join(nm for nm, _ in autotune.SPACE),
                 "ms_by_setting": rows, "chosen": settings}
    ctx = F.Context(m["d"], m["eps"], m["lam"], args.p, precision=F.MIXED, stream=stream, **settings)
    n = args.n
    phi = torch.empty(n, dtype=torch.float64, device=dev)
    fld = torch.empty((n, 3), dtype=torch.float64, device=dev)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)  # 256 MB > L2

    def barrier():
        torch.cuda.synchronize(dev)
        if dist:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(args.warmup):
        ctx.eval(q, x, l, out=(phi, fld))
    torch.cuda.synchronize(dev)
    counts = ctx.counts()
    launches_per_step = counts["launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    phase_ms = {}  # per-phase CUDA-event intervals on the evaluation stream, summed over steps
    barrier()
    with ClockSampler(local_rank) as clk:
        for k in range(args.steps):
            flush.fill_(float(k))
            ev[k][0].record(stream)
            ctx.eval(q, x, l, out=(phi, fld))
            ev[k][1].record(stream)
            for nm, ms, _ in ctx.profile():
                phase_ms[nm] = phase_ms.get(nm, 0.0) + ms
        barrier()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), dist, dev)
    value = job_throughput(world, n, args.steps, total_ms)

    # end to end through the public call with host buffers (pinned), copies inside the timed region
    hq = torch.tensor(w["q"]).pin_memory()
    hx = torch.tensor(w["xyz"]).pin_memory()
    hl = torch.tensor(w["layer"], dtype=torch.int32).pin_memory()
    hphi = torch.empty(n, dtype=torch.float64).pin_memory()
    hfld = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    dq, dx, dl = torch.empty_like(q), torch.empty_like(x), torch.empty_like(l)
    e2e_steps = max(3, args.steps // 2)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        dq.copy_(hq, non_blocking=True)
        dx.copy_(hx, non_blocking=True)
        dl.copy_(hl, non_blocking=True)
        ctx.eval(dq, dx, dl, out=(phi, fld))
        hphi.copy_(phi, non_blocking=True)
        hfld.copy_(fld, non_blocking=True)
    e1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    e2e_val = job_throughput(world, n, e2e_steps, e2e_ms)

    # accuracy gate and the FP64 comparator (same tree rule, same inputs), untimed by the driver's clock
    accuracy, fp64_value = None, None
    if not args.no_fp64:
        ctx64 = F.Context(m["d"], m["eps"], m["lam"], args.p, precision=F.FP64, stream=stream, **settings)
        p64 = torch.empty_like(phi)
        f64 = torch.empty_like(fld)
        ctx64.eval(q, x, l, out=(p64, f64))
        torch.cuda.synchronize(dev)
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        ctx64.eval(q, x, l, out=(p64, f64))
        s1.record(stream)
        torch.cuda.synchronize(dev)
        fp64_value = n / (s0.elapsed_time(s1) / 1000.0)
        ctx.eval(q, x, l, out=(phi, fld))
        torch.cuda.synchronize(dev)
        accuracy = {"relL2_phi_mixed_vs_fp64": float(torch.linalg.norm(phi - p64) / torch.linalg.norm(p64)),
                    "relL2_field_mixed_vs_fp64": float(torch.linalg.norm(fld - f64) / torch.linalg.norm(f64)),
                    "gate": GATE,
                    "per_layer_phi": per_layer_errors(phi, p64, l, len(m["eps"]))}
        accuracy["pass"] = bool(accuracy["relL2_phi_mixed_vs_fp64"] <= GATE and
                                accuracy["relL2_field_mixed_vs_fp64"] <= GATE)
        ctx64.close()

    # both FMMs against the oracle's stored values at sampled targets (no oracle run here)
    vs_oracle = None
    if rank == 0:
        try:
            fx = load_oracle_fixture(n, rank_seed(rank), args.workload)
            if fx is not None:
                idx = torch.tensor(fx["targets"], dtype=torch.int64, device=dev)
                sampled = {"mixed": (phi[idx].cpu().numpy(), fld[idx].cpu().numpy())}
                if accuracy is not None:
                    sampled["fp64"] = (p64[idx].cpu().numpy(), f64[idx].cpu().numpy())
                vs_oracle = oracle_fixture_errors(sampled, fx, w["layer"][np.asarray(fx["targets"])])
        except Exception as e:  # a report only: never lose the measurement line over it
            vs_oracle = {"error": repr(e)}

    device_status = ctx.status()  # 0 unless a bounded device wait ran out during the run

    # rooflines of the heaviest kernels, from their CUDA-event intervals (per evaluation)
    K = (args.p + 1) * (args.p + 2) // 2
    R = 2 * K - (args.p + 1)  # real coordinates of an expansion
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    # FP32 / FP64: FMA chains timed on this device now (lpbfmm_measure_peak); TF32 tensor: the
    # measured bf16 burst x the nominal TF32 / BF16 ratio 1.1 / 2.25; HBM: the measured copy
    fp32_peak = F.measure_peak(F.PEAK_FP32_FMA)
    fp64_peak = F.measure_peak(F.PEAK_FP64_FMA)
    bf16 = peaks.get("bf16_tflops")
    tf32_peak = (bf16 if bf16 else 1900.0) * 1.1 / 2.25
    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    peak_info = {"fp32_fma_tflops": fp32_peak, "fp64_fma_tflops": fp64_peak, "tf32_tflops": tf32_peak,
                 "hbm_gbs": hbm_peak, "sms": torch.cuda.get_device_properties(dev).multi_processor_count,
                 "how": "fp32/fp64: measured FMA chains (lpbfmm_measure_peak); tf32: measured bf16 burst "
                        "(MEASURED_PEAKS.json) x 1.1/2.25; hbm: measured copy (MEASURED_PEAKS.json)" +
                        ("" if peaks.get("hbm_gbs") else " [fallback 6800 GB/s: file absent]")}
    per = lambda nm: phase_ms.get(nm, float("nan")) / args.steps

    traffic_of = profiled_traffic

    def roof(kernel, bound, flops, t, peak, unit_note):
        a = flops / (t / 1e3) / 1e12
        return {"kernel": kernel, "bound": bound, "achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
                "traffic": traffic_of(kernel.split()[0]), "ms_per_eval": t, "algorithmic_flops": flops,
                "flops_per_unit": unit_note}

    roofs = []
    if "p2p" in phase_ms:
        roofs.append(roof("k_p2p_free_f32 (free-space near field of every group, one launch)", "alu",
                          24.0 * counts["p2p_pairs"], per("p2p"), fp32_peak, "24 per pair (+2 SFU)"))
    if "m2l_tc" in phase_ms:
        tr = counts["m2l_free"] + counts["m2l_react"]
        roofs.append(roof("k_m2l_tc (free-space and reaction M2L, tcgen05 3xTF32)", "tensor", 2.0 * R * R * tr,
                          per("m2l_tc"), tf32_peak,
                          "2 R^2 = %d per translation (R = %d real coordinates)" % (2 * R * R, R)))
    if "m2l_simt" in phase_ms:
        roofs.append(roof("k_m2l_f32 (M2L, FP32 SIMT)", "alu", 4.0 * K * K * counts["m2l_react"], per("m2l_simt"),
                          fp32_peak, "4 K^2 per translation"))
    if "tree" in phase_ms:
        # the tree build streams the inputs once and writes every group's sorted point records:
        # 36 B per charge read, 44 B per target or image point written (key 8, index 4, x y z q 32)
        tb = 36.0 * n + 44.0 * (counts["targets"] + counts["images"])
        t = per("tree")
        a = tb / (t / 1e3) / 1e9
        roofs.append({"kernel": "tree build (validation, keys, radix sorts, boxes, lists)", "bound": "hbm",
                      "achieved": a, "peak": hbm_peak, "unit": "GB/s", "frac": a / hbm_peak, "traffic": None,
                      "ms_per_eval": t, "algorithmic_bytes": tb,
                      "bytes_per_unit": "36 per charge read + 44 per sorted target or image point written"})
    roof_main = max(roofs, key=lambda r: r["ms_per_eval"]) if roofs else None

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        oracle.build()
        v, dt, info = oracle_sample(w, max(2, oracle.num_threads()), CPU_SOURCE_STRIDE)
        info["value"] = v
        cpu = info

    if rank == 0:
        line = {"metric": metric_of(args.workload), "value": value, "unit": "targets/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
                "config": workload_config(n, args.p, "mixed", args.workload),
                "clocks": clk.summary(), "autotune": tuned,
                "e2e": {"value": e2e_val, "unit": "targets/s", "h2d_bytes_per_step": n * (8 + 24 + 4),
                        "d2h_bytes_per_step": n * (8 + 24)},
                "gpu_launches": launches_per_step * args.steps, "roofline": roof_main, "rooflines": roofs,
                "phases_ms_per_eval": {k: v / args.steps for k, v in phase_ms.items()}, "device_status": device_status,
                "cpu_baseline": cpu,
                "fp64_fmm_value": fp64_value, "accuracy": accuracy, "accuracy_vs_oracle": vs_oracle,
                "counts": counts, "peaks": peak_info}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_batch(args, rank, world, local_rank):
    """The batching form (one lpbfmm_eval_batched call per step over 256 systems, p = 8, mixed):
    targets of all systems per second.  Context measurement beside the headline workload."""
    import torch
    from paper_2002_01334_gb300 import build as B
    B.build()
    from paper_2002_01334_gb300 import autotune
    from paper_2002_01334_gb300 import inputs
    from paper_2002_01334_gb300 import lpbfmm as F
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    systems = inputs.batch(nsys=256, nmin=1000, nmax=64000, seed=inputs.BASE_SEED + 3 + 1000 * rank)
    stream = torch.cuda.current_stream(dev)
    offs = [0]
    for s in systems:
        offs.append(offs[-1] + len(s["q"]))
    n = offs[-1]
    q = torch.tensor(np.concatenate([s["q"] for s in systems]), device=dev)
    x = torch.tensor(np.concatenate([s["xyz"] for s in systems]), device=dev)
    l = torch.tensor(np.concatenate([s["layer"] for s in systems]), dtype=torch.int32, device=dev)
    settings, tuned = dict(autotune.DEFAULTS), None
    if not args.no_autotune:
        measure, close = autotune.batch_measure(systems, 8, F.MIXED, offs, q, x, l, stream=stream)
        settings, rows = autotune.search(autotune.SPACE, measure, start=autotune.DEFAULTS, repeats=2)
        close()
        tuned = {"method": "coordinate descent over %s in order (one setting for every system); median of 2 "
                           "CUDA-event timings of one batched evaluation per setting"
                           % ", ".join(nm for nm, _ in autotune.SPACE),
                 "ms_by_setting": rows, "chosen": settings}
    ctxs = [F.Context(s["medium"]["d"], s["medium"]["eps"], s["medium"]["lam"], 8, precision=F.MIXED, stream=stream,
                      **settings) for s in systems]
    for _ in range(args.warmup):
        F.eval_batched(ctxs, offs, q, x, l)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local_rank) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            F.eval_batched(ctxs, offs, q, x, l)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1)
    value = n * args.steps / (ms / 1e3)
    launches = sum(c.counts()["launches"] for c in ctxs)  # per step: every context's kernels + grouped ones
    if rank == 0:
        print(json.dumps({"metric": METRIC_BATCH, "value": value, "unit": "targets/s", "n_gpus": world,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
                          "data": "synthetic",
                          "config": {"workload": "256 systems, N log-uniform in [1000, 64000] (total %d), p = 8, "
                                                 "random 2-4 layer media" % n, "systems": 256, "n": n, "p": 8,
                                     "precision": "mixed", "separation": "two-box interaction lists",
                                     "tree": "automatic depth, <=%d mean targets per leaf, reaction trees up to %d "
                                             "levels deeper%s" % (settings["max_per_leaf"], settings["react_levels"],
                                                                  " (autotuned)" if tuned else ""),
                                     "l2": "not flushed: the inputs (%d MB) and each step's work space exceed the "
                                           "129 MB L2" % (n * 36 // 10**6)},
                          "gpu_launches": launches * args.steps, "autotune": tuned, "clocks": clk.summary()}),
              flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.workload == "batch":
        run_batch(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
