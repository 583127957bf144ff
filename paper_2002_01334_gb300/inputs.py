"""Seeded synthetic inputs: charges, positions and layered media.

This module holds only random-number generation and geometry of the synthetic workloads;
none of the method's arithmetic.  Both the oracle tests and the GPU tests draw inputs from
here.  The generator is SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), doubles from the top
53 bits, U[a, b] = a + (b - a) u.  Draw order: charges q first, then positions (x, y, z)
charge by charge.

Workloads (the media and boxes of the screened-Coulomb layered-media benchmarks):
  three_layer_small  d=(0,-1.2), eps=(1,2,5), lambda=(0.5,1,0.8); N=1000 in the middle layer
                     cube [-0.5,0.5]^2 x [-1.1,-0.1]; p=8; uniform depth 2.
  three_layer        same medium; N split evenly over three unit cubes, one per layer
                     (z in [0.1,1.1], [-1.1,-0.1], [-2.3,-1.3]); p=10.
  four_layer         d=(0,-1,-2), eps=(1,4,2,8), lambda=(0.3,1,0.6,1.5); N split evenly over
                     four cubes 0.05 from the interfaces; p=8.
  batch              many independent systems with random media (2-4 layers).
"""
import numpy as np

_M1 = np.uint64(0x9E3779B97F4A7C15)
_M2 = np.uint64(0xBF58476D1CE4E5B9)
_M3 = np.uint64(0x94D049BB133111EB)
BASE_SEED = 2002013340


def splitmix64(seed, count, start=0):
    """count outputs of SplitMix64 seeded with `seed`, starting at output index `start`."""
    with np.errstate(over="ignore"):
        i = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = np.uint64(seed) + i * _M1
        z = (z ^ (z >> np.uint64(30))) * _M2
        z = (z ^ (z >> np.uint64(27))) * _M3
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed, count, start=0):
    """doubles in [0, 1) from the top 53 bits."""
    return (splitmix64(seed, count, start) >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


class Stream:
    """Sequential draws from one seed."""

    def __init__(self, seed):
        self.seed = seed
        self.pos = 0

    def u(self, count, lo=0.0, hi=1.0):
        v = uniform(self.seed, count, self.pos)
        self.pos += count
        return lo + (hi - lo) * v


MEDIA = {
    "three_layer": dict(d=[0.0, -1.2], eps=[1.0, 2.0, 5.0], lam=[0.5, 1.0, 0.8]),
    "four_layer": dict(d=[0.0, -1.0, -2.0], eps=[1.0, 4.0, 2.0, 8.0], lam=[0.3, 1.0, 0.6, 1.5]),
    # the paper's own test medium (Sec. 4): eps=(1, 8.6, 20.5), lambda=(1.2, 0.5, 2.1)
    "paper_three_layer": dict(d=[0.0, -1.2], eps=[1.0, 8.6, 20.5], lam=[1.2, 0.5, 2.1]),
}

THREE_LAYER_BOXES = [(0.1, 1.1), (-1.1, -0.1), (-2.3, -1.3)]
FOUR_LAYER_BOXES = [(0.05, 1.05), (-0.95, -0.05), (-1.95, -1.05), (-3.05, -2.05)]


def charges_in_boxes(seed, counts, zboxes, xy=(-0.5, 0.5), interleave=True):
    """q ~ U[-1,1] and positions uniform in [xy]^2 x zboxes[k] for counts[k] charges of layer k.

    With interleave, charge i belongs to the layer given by a round-robin over the layers that
    still need charges, so the input is not sorted by layer."""
    n = int(sum(counts))
    s = Stream(seed)
    q = s.u(n, -1.0, 1.0)
    raw = s.u(3 * n).reshape(n, 3)
    nl = len(counts)
    labels = np.repeat(np.arange(nl, dtype=np.int32), counts)
    if interleave:
        # charge j of layer k sits at rank j*nl + k: a round-robin over the layers
        rank = np.concatenate([np.arange(c, dtype=np.int64) * nl + k for k, c in enumerate(counts)])
        layer = labels[np.argsort(rank, kind="stable")]
    else:
        layer = labels
    xyz = np.empty((n, 3))
    xyz[:, 0] = xy[0] + (xy[1] - xy[0]) * raw[:, 0]
    xyz[:, 1] = xy[0] + (xy[1] - xy[0]) * raw[:, 1]
    lo = np.array([zboxes[k][0] for k in layer])
    hi = np.array([zboxes[k][1] for k in layer])
    xyz[:, 2] = lo + (hi - lo) * raw[:, 2]
    return q, xyz, layer


# The irregular bodies of the paper's three-layer example (Sec. 4): around a centre on the z axis
# the surface is r(theta) = 0.5 - a + (a/8)(35 cos^4 theta - 30 cos^2 theta + 3), with
# (a, centre z) below for layers 0, 1, 2; 912 + 640 + 1296 charges in the accuracy test.
PAPER_BODIES = [(0.10, 0.6), (0.15, -0.6), (0.05, -1.8)]
PAPER_COUNTS = (912, 640, 1296)


def body_radius(a, cos_t):
    """Radius of the body surface in the direction with cos(theta) = cos_t."""
    c2 = cos_t * cos_t
    return 0.5 - a + (a / 8.0) * (35.0 * c2 * c2 - 30.0 * c2 + 3.0)


def charges_in_bodies(seed, counts, bodies=PAPER_BODIES, batch=4096):
    """q ~ U[-1,1]; the charges of layer k are uniform points of the cube
    [-0.5,0.5]^2 x [zc-0.5, zc+0.5] kept when inside body k (the body fits in that cube), drawn in
    batches until counts[k] are kept.  Layers are interleaved round-robin like charges_in_boxes."""
    n = int(sum(counts))
    s = Stream(seed)
    q = s.u(n, -1.0, 1.0)
    per = []
    for (a, zc), cnt in zip(bodies, counts):
        kept = np.empty((0, 3))
        while len(kept) < cnt:
            raw = s.u(3 * batch).reshape(batch, 3) - 0.5
            r = np.sqrt((raw * raw).sum(axis=1))
            cos_t = np.where(r > 0, raw[:, 2] / np.where(r > 0, r, 1.0), 1.0)
            inside = r <= body_radius(a, cos_t)
            kept = np.concatenate([kept, raw[inside]])
        pts = kept[:cnt].copy()
        pts[:, 2] += zc
        per.append(pts)
    nl = len(counts)
    labels = np.repeat(np.arange(nl, dtype=np.int32), counts)
    rank = np.concatenate([np.arange(c, dtype=np.int64) * nl + k for k, c in enumerate(counts)])
    order = np.argsort(rank, kind="stable")
    return q, np.concatenate(per)[order], labels[order]


def even_split(n, nl):
    base = n // nl
    return [base + (1 if k < n - base * nl else 0) for k in range(nl)]


def workload(name, n=None, seed=None):
    """Returns dict(medium=..., q, xyz, layer, p, depth (None = automatic))."""
    if name == "three_layer_small":
        n = 1000 if n is None else n
        seed = BASE_SEED + 0 if seed is None else seed
        q, xyz, layer = charges_in_boxes(seed, [0, n, 0], THREE_LAYER_BOXES)
        return dict(medium=MEDIA["three_layer"], q=q, xyz=xyz, layer=layer, p=8, depth=2)
    if name == "three_layer":
        n = 100000 if n is None else n
        seed = BASE_SEED + (1 if n <= 100000 else 2) if seed is None else seed
        q, xyz, layer = charges_in_boxes(seed, even_split(n, 3), THREE_LAYER_BOXES)
        return dict(medium=MEDIA["three_layer"], q=q, xyz=xyz, layer=layer, p=10, depth=None)
    if name == "four_layer":
        n = 200000 if n is None else n
        seed = BASE_SEED + 4 if seed is None else seed
        q, xyz, layer = charges_in_boxes(seed, even_split(n, 4), FOUR_LAYER_BOXES)
        return dict(medium=MEDIA["four_layer"], q=q, xyz=xyz, layer=layer, p=8, depth=None)
    if name == "paper_irregular":
        # the paper's accuracy-test workload; n scales the three counts in proportion
        counts = list(PAPER_COUNTS)
        if n is not None:
            tot = sum(PAPER_COUNTS)
            counts = [int(round(n * c / tot)) for c in PAPER_COUNTS]
            counts[-1] = n - sum(counts[:-1])
        seed = BASE_SEED + 5 if seed is None else seed
        q, xyz, layer = charges_in_bodies(seed, counts)
        return dict(medium=MEDIA["paper_three_layer"], q=q, xyz=xyz, layer=layer, p=10, depth=None)
    raise KeyError(name)


def random_medium(stream, nlayers_choices=(2, 3, 4)):
    """Random medium: layer count U{2,3,4}, d_0 = 0, finite thicknesses U[0.5,2],
    eps ~ U[1,10], lambda ~ U[0.2,2] per layer."""
    nl = int(nlayers_choices[min(len(nlayers_choices) - 1, int(stream.u(1)[0] * len(nlayers_choices)))])
    L = nl - 1
    d = [0.0]
    for _ in range(L - 1):
        d.append(d[-1] - float(stream.u(1, 0.5, 2.0)[0]))
    eps = list(stream.u(nl, 1.0, 10.0))
    lam = list(stream.u(nl, 0.2, 2.0))
    return dict(d=d, eps=eps, lam=lam)


def batch(nsys=256, nmin=1000, nmax=64000, seed=BASE_SEED + 3, delta=0.05):
    """Independent systems: N log-uniform in [nmin, nmax], random medium, all charges of a system
    in one random host layer, xy in [-0.5,0.5]^2, z-range min(1, t - 2 delta) tall centred in a
    finite layer, or a unit-tall range delta away from the interface of the top/bottom layer."""
    s = Stream(seed)
    systems = []
    for k in range(nsys):
        n = int(round(np.exp(s.u(1, np.log(nmin), np.log(nmax))[0])))
        md = random_medium(s)
        nl = len(md["eps"])
        host = min(nl - 1, int(s.u(1)[0] * nl))
        d = md["d"]
        if host == 0:
            zlo, zhi = d[0] + delta, d[0] + delta + 1.0
        elif host == nl - 1:
            zlo, zhi = d[-1] - delta - 1.0, d[-1] - delta
        else:
            top, bot = d[host - 1], d[host]
            t = top - bot
            hgt = min(1.0, t - 2 * delta)
            mid = 0.5 * (top + bot)
            zlo, zhi = mid - 0.5 * hgt, mid + 0.5 * hgt
        counts = [0] * nl
        counts[host] = n
        boxes = [(zlo, zhi)] * nl
        q, xyz, layer = charges_in_boxes(int(s.u(1)[0] * 2**52), counts, boxes)
        systems.append(dict(medium=md, q=q, xyz=xyz, layer=layer, p=8, depth=None))
    return systems
