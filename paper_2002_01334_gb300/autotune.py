"""Choice of the leaf-size target by measurement.

The FMM's cost splits between the near field (grows with the charges per leaf) and the
translations (grow with the number of boxes).  Which balance is fastest depends on the workload
and the GPU, so the target mean occupancy of the leaves (``max_per_leaf``, from which every
target group's depth follows) is picked by timing candidate values on the workload itself.
The search is host logic (``choose``); the timing of one candidate (``cuda_measure``) runs the
library's evaluation through the public binding, with CUDA events on the evaluation stream.
"""
import statistics

CANDIDATES = (32, 64, 128, 256, 512)


def choose(candidates, measure, repeats=3):
    """Time every candidate with measure(c) -> milliseconds, `repeats` times each, and return
    (best, table): the candidate with the smallest median, the first one on a tie, and the
    medians by candidate."""
    if not candidates:
        raise ValueError("no candidates")
    table = {}
    for c in candidates:
        table[c] = statistics.median(measure(c) for _ in range(max(1, repeats)))
    best = min(candidates, key=lambda c: (table[c], candidates.index(c)))
    return best, table


def cuda_measure(medium, p, precision, q, xyz, layer, stream=None, warmup=1):
    """(measure, close): measure(max_per_leaf) -> ms of one evaluation of these device arrays by a
    context with that leaf target (created once per candidate and warmed up), timed with CUDA
    events; close() releases the candidates' contexts."""
    import torch

    from . import lpbfmm as F

    contexts = {}

    def measure(s):
        if s not in contexts:
            ctx = F.Context(medium["d"], medium["eps"], medium["lam"], p, precision=precision,
                            max_per_leaf=s, stream=stream)
            for _ in range(warmup):
                ctx.eval(q, xyz, layer)
            contexts[s] = ctx
        ctx = contexts[s]
        st = stream if stream is not None else torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        ctx.eval(q, xyz, layer)
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    def close():
        for ctx in contexts.values():
            ctx.close()
        contexts.clear()

    return measure, close
