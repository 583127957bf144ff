"""Choice of the evaluation's shape parameters by measurement.

The FMM's cost splits between the near field and the translations, and where the balance lies
depends on the workload and the GPU.  Two parameters set it:

* ``max_per_leaf``: the mean target occupancy of the free-space leaves, from which every target
  group's depth follows.  It is the tile shape of the near-field kernel (the targets a warp pair
  holds and the sources of a leaf's near list that stream past them) and the number of target
  boxes, hence of 128-row tiles, of the tensor-core M2L;
* ``react_levels``: how far below the free-space depth the reaction trees may go to separate
  targets from images (Sec. 3.5, Remark 1), trading direct Sommerfeld quadrature for reaction M2L
  on more boxes.

The tensor-core tile itself is fixed by the MMA shape (128 target rows, 32-column K-chunks).
The search is host logic (``search``, coordinate descent over the parameters in order); timing one
setting (``cuda_measure``, ``batch_measure``) runs the library through the public binding, with
CUDA events on the evaluation stream.
"""
import statistics

CANDIDATES = (32, 64, 128, 256, 512)
SPACE = (("max_per_leaf", (32, 64, 128, 256, 512)), ("react_levels", (2, 3, 4, 6)))
DEFAULTS = {"max_per_leaf": 128, "react_levels": 4}


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


def search(space, measure, start=None, repeats=2):
    """Coordinate descent: for each (name, candidates) of space in order, time every candidate with
    the other parameters at their best so far (measure(settings dict) -> ms, or None when the
    setting cannot run, e.g. out of device memory; each distinct setting timed once, `repeats`
    times) and keep the fastest.  Returns (best settings, rows), rows being [settings, median ms
    or None] for every setting tried, in order."""
    best = dict(start or {})
    for name, cands in space:
        best.setdefault(name, cands[0])
    seen = {}
    rows = []

    def timed(settings):
        key = tuple(sorted(settings.items()))
        if key not in seen:
            ts = []
            for _ in range(max(1, repeats)):
                t = measure(dict(settings))
                if t is None:
                    ts = None
                    break
                ts.append(t)
            seen[key] = statistics.median(ts) if ts else None
            rows.append([dict(settings), seen[key]])
        return seen[key]

    inf = float("inf")
    for name, cands in space:
        if not cands:
            raise ValueError("no candidates for %s" % name)
        ms = {c: timed(dict(best, **{name: c})) for c in cands}
        best[name] = min(cands, key=lambda c: (inf if ms[c] is None else ms[c], cands.index(c)))
    return best, rows


def cuda_measure(medium, p, precision, q, xyz, layer, stream=None, warmup=1):
    """(measure, close): measure(settings) -> ms of one evaluation of these device arrays by a
    context created with those options (max_per_leaf, react_levels; created when the setting
    changes, the previous setting's context released first, and warmed up), timed with CUDA
    events; close() releases the context.  An int stands for {"max_per_leaf": int}."""
    import torch

    from . import lpbfmm as F

    contexts = {}  # the current setting's context only (the search times one setting at a time)

    def measure(s):
        s = {"max_per_leaf": s} if isinstance(s, int) else dict(s)
        key = tuple(sorted(s.items()))
        try:
            if key not in contexts:
                close()
                ctx = F.Context(medium["d"], medium["eps"], medium["lam"], p, precision=precision, stream=stream,
                                **s)
                contexts[key] = ctx
                for _ in range(warmup):
                    ctx.eval(q, xyz, layer)
            ctx = contexts[key]
            st = stream if stream is not None else torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            ctx.eval(q, xyz, layer)
            e1.record(st)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)
        except F.LpbfmmError as e:
            if e.code != F.ERR_OOM:
                raise
            close()
            return None

    def close():
        for ctx in contexts.values():
            ctx.close()
        contexts.clear()

    return measure, close


def batch_measure(systems, p, precision, offsets, q, xyz, layer, stream=None, warmup=1):
    """(measure, close) for lpbfmm_eval_batched: measure(settings) -> ms of one batched evaluation
    of all systems, every context created with those options (one setting's contexts alive at a
    time)."""
    import torch

    from . import lpbfmm as F

    sets = {}  # the current setting's contexts only (the search times one setting at a time)

    def measure(s):
        s = dict(s)
        key = tuple(sorted(s.items()))
        try:
            if key not in sets:
                close()
                sets[key] = []
                for x in systems:
                    sets[key].append(F.Context(x["medium"]["d"], x["medium"]["eps"], x["medium"]["lam"], p,
                                               precision=precision, stream=stream, **s))
                for _ in range(warmup):
                    F.eval_batched(sets[key], offsets, q, xyz, layer)
            ctxs = sets[key]
            st = stream if stream is not None else torch.cuda.current_stream()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record(st)
            F.eval_batched(ctxs, offsets, q, xyz, layer)
            e1.record(st)
            torch.cuda.synchronize()
            return e0.elapsed_time(e1)
        except F.LpbfmmError as e:
            if e.code != F.ERR_OOM:
                raise
            close()
            return None

    def close():
        for ctxs in sets.values():
            for c in ctxs:
                c.close()
        sets.clear()

    return measure, close
