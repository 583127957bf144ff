"""One evaluation split across GPUs, one process per GPU (torch.distributed, NCCL on GPUs).

The potential is a sum of independent parts (Sec. 2.2, eq. freereactioncomponents): for every
layer l, the free-space FMM of its charges and the reaction components of its targets.  Sec. 4
remarks that the components can be computed in parallel.  A unit of work here is (layer, part);
ranks take disjoint sets of units, balanced by an estimated cost, evaluate them with
lpbfmm_eval_groups (the units as a group mask), and one sum-reduce of the FP64 partial results
(potential and field, 4 N doubles) gives every rank the whole result, equal to the one-rank
evaluation up to rounding: FP64 rounding of the summation order in FP64 mode; in the mixed mode
a layer's free and reaction local expansions are added in FP32 before their evaluation when one
rank holds both, so a split that separates them differs by that FP32 rounding.  Only the
assignment and the mask are computed here; every step of the evaluation runs in the library's
kernels.
"""
FREE, REACT = 0, 1


def units(nlayers):
    """The units of work of a medium with nlayers layers: (layer, part)."""
    return [(l, part) for l in range(nlayers) for part in (FREE, REACT)]


def unit_costs(layer_counts, react_weight=0.5):
    """Estimated cost of every unit: proportional to the layer's charges, the reaction part of a
    layer weighted by react_weight (its share of one layer's work measured on the three-layer
    workload: the reaction far field sits in a slab at the interfaces, Sec. 3.5, Remark 1)."""
    out = []
    for l, part in units(len(layer_counts)):
        out.append(float(layer_counts[l]) * (1.0 if part == FREE else react_weight))
    return out


def assign(costs, world):
    """Longest-processing-time assignment of units to ranks: units by decreasing cost (ties by
    index), each to the rank with the least total so far (ties to the lowest rank).  Returns one
    sorted list of unit indices per rank; deterministic, so every rank computes the same plan."""
    order = sorted(range(len(costs)), key=lambda k: (-costs[k], k))
    load = [0.0] * world
    plan = [[] for _ in range(world)]
    for k in order:
        r = min(range(world), key=lambda i: (load[i], i))
        plan[r].append(k)
        load[r] += costs[k]
    return [sorted(p) for p in plan]


def group_mask(unit_ids, nlayers):
    """lpbfmm_eval_groups mask (2 (L + 1) ints, entry 2 l + a - 1) of a set of units: the free
    part of layer l on both of its groups (the library takes it from the group that carries it),
    the reaction part of layer l on both sides."""
    all_units = units(nlayers)
    mask = [0] * (2 * nlayers)
    for k in unit_ids:
        l, part = all_units[k]
        bit = 1 if part == FREE else 2
        mask[2 * l] |= bit
        mask[2 * l + 1] |= bit
    return mask


def partitioned(evaluate_mask, n, nlayers, costs, rank, world, all_reduce):
    """This rank's share of one evaluation and the sum over ranks.  evaluate_mask(mask) returns the
    rank's partial (phi[n], field[n, 3]) as float64 tensors; all_reduce(t) sums a float64 tensor
    over the ranks in place.  Returns the whole (phi, field) on every rank."""
    import torch
    mine = assign(costs, world)[rank]
    phi, field = evaluate_mask(group_mask(mine, nlayers))
    buf = torch.cat([phi.reshape(-1), field.reshape(-1)])
    all_reduce(buf)
    return buf[:n], buf[n:].reshape(n, 3)


def evaluate(ctx, q, xyz, layer, rank, world, group=None):
    """lpbfmm on this rank's units of one system, reduced over the process group (NCCL): the whole
    potential and field on every rank."""
    import torch
    import torch.distributed as dist
    nl = len(ctx.eps)
    counts = torch.bincount(layer.to(torch.int64), minlength=nl).tolist()

    def ev(mask):
        return ctx.eval_groups(q, xyz, layer, mask)

    def red(t):
        dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return partitioned(ev, q.shape[0], nl, unit_costs(counts), rank, world, red)
