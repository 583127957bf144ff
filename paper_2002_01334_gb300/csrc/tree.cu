// Input validation, per-group octrees (Morton keys + radix sort) and interaction lists.
// Tree rule (Sec. 3.5, before Algorithm 1): the root cube of target group (l, a) is bisected by its interface
// (d_l for a = 1, d_{l-1} for a = 2), so every box of level >= 1 has its centre on the
// side of the points it holds; all trees here have uniform depth D.
#include "internal.h"
#include "prims.cuh"

namespace lpb {

// ---------------------------------------------------------------------------------------
// scan / sort wrappers
// ---------------------------------------------------------------------------------------
void scan_u32(Ctx &c, const uint32_t *in, uint32_t *out, int64_t n, uint32_t *d_total) {
  if (n <= 8192) {  // one launch, one chunk
    k_scan_one<<<1, 1024, 0, c.stream>>>(in, out, n, d_total);
    LPB_LAUNCH();
    c.launches++;
    return;
  }
  const int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
  uint32_t *sums = c.arena.get<uint32_t>(tiles + 1);
  if (n > 0) {
    k_scan_tiles<<<(unsigned)tiles, SCAN_THREADS, 0, c.stream>>>(in, out, sums, n);
    LPB_LAUNCH();
  }
  k_scan_sums<<<1, 1024, 0, c.stream>>>(sums, tiles, d_total);
  LPB_LAUNCH();
  if (tiles > 1) {
    k_scan_add<<<(unsigned)tiles, SCAN_THREADS, 0, c.stream>>>(out, sums, n);
    LPB_LAUNCH();
  }
  c.launches += 2 + (tiles > 1) + (n > 0 ? 0 : -1);
}

// stable sort by key bits [lo, bits): lower bits must not matter for the order (zero, or a
// field equal within a run that the caller does not need sorted)
void radix_sort(Ctx &c, uint64_t *&keys, uint32_t *&vals, int64_t n, int bits, int lo) {
  if (n <= 1) return;
  const int nblocks = (int)((n + RS_TILE - 1) / RS_TILE);
  uint64_t *k2 = c.arena.get<uint64_t>(n);
  uint32_t *v2 = c.arena.get<uint32_t>(n);
  uint32_t *hist = c.arena.get<uint32_t>((size_t)256 * nblocks);
  uint32_t *offs = c.arena.get<uint32_t>((size_t)256 * nblocks);
  for (int shift = lo; shift < bits; shift += 8) {
    k_radix_hist<<<nblocks, RS_THREADS, 0, c.stream>>>(keys, n, shift, hist, nblocks);
    LPB_LAUNCH();
    scan_u32(c, hist, offs, (int64_t)256 * nblocks, nullptr);
    k_radix_scatter<<<nblocks, RS_THREADS, 0, c.stream>>>(keys, vals, k2, v2, n, shift, offs, nblocks);
    LPB_LAUNCH();
    c.launches += 2;
    uint64_t *tk = keys; keys = k2; k2 = tk;
    uint32_t *tv = vals; vals = v2; v2 = tv;
  }
}

// ---------------------------------------------------------------------------------------
// validation: finite, off the interfaces, layer_id consistent with z; counts and extents
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ord_of(double v) {
  unsigned long long u = (unsigned long long)__double_as_longlong(v);
  return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ unsigned long long wmin(unsigned long long v) {
  for (int o = 16; o; o >>= 1) { unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o); v = w < v ? w : v; }
  return v;
}
__device__ __forceinline__ unsigned long long wmax(unsigned long long v) {
  for (int o = 16; o; o >>= 1) { unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o); v = w > v ? w : v; }
  return v;
}

// Grid-stride validation: every thread keeps its own extremes (order-preserving integers of
// the FP64 coordinates) and per-layer counts; they are reduced per warp by shuffles, per block
// in shared memory, and merged into the global statistics with one atomic per block and field.
constexpr int VAL_THREADS = 256;
__global__ void __launch_bounds__(VAL_THREADS) k_validate(int64_t n, const double *q, const double *xyz,
                                                          const int32_t *layer, Medium md, double thr, Stats *st) {
  const unsigned long long HI = ~0ull, LO = 0ull;
  unsigned long long xlo = HI, xhi = LO, ylo = HI, yhi = LO, zlo[MAXLAYER], zhi[MAXLAYER];
  unsigned cnt[MAXLAYER];
#pragma unroll
  for (int k = 0; k < MAXLAYER; ++k) {
    zlo[k] = HI;
    zhi[k] = LO;
    cnt[k] = 0;
  }
  int code_seen = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    const double qq = q[i];
    const int lay = layer[i];
    int code = 0;
    if (!isfinite(x) || !isfinite(y) || !isfinite(z) || !isfinite(qq)) {
      code = LPBFMM_ERR_NONFINITE;
    } else {
      int l = 0;
      while (l < md.L && z < md.d[l]) ++l;
      for (int k = 0; k < md.L; ++k)
        if (fabs(z - md.d[k]) < thr) code = LPBFMM_ERR_ON_INTERFACE;
      if (!code && l != lay) code = LPBFMM_ERR_LAYER_MISMATCH;
    }
    if (code) {
      if (!code_seen) atomicCAS(&st->status, 0, code);
      code_seen = 1;
      continue;
    }
    const unsigned long long ox = ord_of(x), oy = ord_of(y), oz = ord_of(z);
    xlo = min(xlo, ox); xhi = max(xhi, ox);
    ylo = min(ylo, oy); yhi = max(yhi, oy);
#pragma unroll
    for (int k = 0; k < MAXLAYER; ++k)
      if (k == lay) {
        zlo[k] = min(zlo[k], oz);
        zhi[k] = max(zhi[k], oz);
        ++cnt[k];
      }
  }
  __shared__ unsigned long long red[VAL_THREADS / 32][4 + 3 * MAXLAYER];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  unsigned long long v[4 + 3 * MAXLAYER];
  v[0] = wmin(xlo); v[1] = wmax(xhi); v[2] = wmin(ylo); v[3] = wmax(yhi);
#pragma unroll
  for (int k = 0; k < MAXLAYER; ++k) {
    v[4 + k] = wmin(zlo[k]);
    v[4 + MAXLAYER + k] = wmax(zhi[k]);
    unsigned c = cnt[k];
#pragma unroll
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    v[4 + 2 * MAXLAYER + k] = c;
  }
  if (lane == 0)
    for (int f = 0; f < 4 + 3 * MAXLAYER; ++f) red[warp][f] = v[f];
  __syncthreads();
  if (threadIdx.x < 4 + 3 * MAXLAYER) {
    const int f = threadIdx.x;
    const bool is_min = f == 0 || f == 2 || (f >= 4 && f < 4 + MAXLAYER);
    const bool is_cnt = f >= 4 + 2 * MAXLAYER;
    unsigned long long a = is_min ? HI : LO;
    for (int w2 = 0; w2 < nw; ++w2) {
      const unsigned long long b = red[w2][f];
      a = is_cnt ? a + b : (is_min ? min(a, b) : max(a, b));
    }
    unsigned long long *dst = f == 0 ? &st->xlo : f == 1 ? &st->xhi : f == 2 ? &st->ylo : f == 3 ? &st->yhi
                            : f < 4 + MAXLAYER ? &st->zlo[f - 4]
                            : f < 4 + 2 * MAXLAYER ? &st->zhi[f - 4 - MAXLAYER]
                            : &st->cnt[f - 4 - 2 * MAXLAYER];
    if (is_cnt) { if (a) atomicAdd(dst, a); }
    else if (is_min) { if (a != HI) atomicMin(dst, a); }
    else if (a != LO) atomicMax(dst, a);
  }
}

void launch_validate(Ctx &c, int64_t n, const double *q, const double *xyz, const int32_t *layer, Stats *st) {
  double scale = 1.0;
  for (int k = 0; k < c.md.L; ++k) scale = fmax(scale, fabs(c.md.d[k]));
  const double thr = 1e-12 * scale;
  const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n + VAL_THREADS - 1) / VAL_THREADS, 152 * 4));
  k_validate<<<blocks, VAL_THREADS, 0, c.stream>>>(n, q, xyz, layer, c.md, thr, st);
  LPB_LAUNCH();
  c.launches++;
}

__global__ void k_flag_layer(int64_t n, const int32_t *layer, int lay, uint32_t *f) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) f[i] = layer[i] == lay ? 1u : 0u;
}
void layer_rank(Ctx &c, int64_t n, const int32_t *layer, int lay, uint32_t *rank) {
  uint32_t *f = c.arena.get<uint32_t>(n);
  k_flag_layer<<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>(n, layer, lay, f);
  LPB_LAUNCH();
  c.launches++;
  scan_u32(c, f, rank, n, nullptr);
}

// ---------------------------------------------------------------------------------------
// points and Morton keys
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x3ffu;  // 10 bits
  x = (x | (x << 16)) & 0x30000ffull;
  x = (x | (x << 8)) & 0x300f00full;
  x = (x | (x << 4)) & 0x30c30c3ull;
  x = (x | (x << 2)) & 0x9249249ull;
  return x;
}
__device__ __forceinline__ uint32_t compact3(uint64_t x) {
  x &= 0x9249249ull;
  x = (x ^ (x >> 2)) & 0x30c30c3ull;
  x = (x ^ (x >> 4)) & 0x300f00full;
  x = (x ^ (x >> 8)) & 0x30000ffull;
  x = (x ^ (x >> 16)) & 0x3ffull;
  return (uint32_t)x;
}
// cell index i = floor((x - x0) * s) clamped to [0, 2^DMAX - 1]; rounded ops, no contraction
__device__ __forceinline__ uint32_t cell_of(double x, double x0, double s) {
  double t = floor(__dmul_rn(__dsub_rn(x, x0), s));
  t = fmin(fmax(t, 0.0), double((1 << DMAX) - 1));
  return (uint32_t)t;
}
__device__ __forceinline__ uint64_t morton_of(double x, double y, double z, const double *o, double s) {
  return (spread3(cell_of(x, o[0], s)) << 2) | (spread3(cell_of(y, o[1], s)) << 1) | spread3(cell_of(z, o[2], s));
}

struct RankPtrs {
  uint32_t *r[MAXLAYER];
};
struct GroupGeom {
  double o[3];  // lower corner of the root cube
  double s;     // 2^DMAX / (2H)
  int l, a;
  int64_t type_off[2 * MAXLAYER];
};

__global__ void k_make_targets(int64_t n, const double *xyz, const int32_t *layer, RankPtrs rk, GroupGeom gg,
                               uint64_t *key, uint32_t *src) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n || layer[i] != gg.l) return;
  const uint32_t pos = rk.r[gg.l][i];
  key[pos] = morton_of(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], gg.o, gg.s) << 4;
  src[pos] = (uint32_t)i;
}

__global__ void k_make_images(int64_t n, const double *xyz, const int32_t *layer, Medium md, RankPtrs rk,
                              GroupGeom gg, int D, uint64_t *key, uint32_t *src) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int lp = layer[i];
  for (int b = 1; b <= 2; ++b) {
    if ((b == 1 && lp == md.L) || (b == 2 && lp == 0)) continue;
    const int t = type_index(lp, b);
    const int64_t pos = gg.type_off[t] + rk.r[lp][i];
    const double zi = image_z(md, gg.l, gg.a, lp, b, xyz[3 * i + 2]);
    key[pos] = ((morton_of(xyz[3 * i], xyz[3 * i + 1], zi, gg.o, gg.s) >> (3 * (DMAX - D))) << 4) | (uint64_t)t;
    src[pos] = (uint32_t)i;
  }
}

__global__ void k_gather_points(int64_t np, const uint64_t *key, const uint32_t *src, const double *q,
                                const double *xyz, Medium md, int l, int a, int images, double *x, double *y,
                                double *z, double *qq, const int32_t *layer) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  const uint32_t i = src[k];
  x[k] = xyz[3 * i];
  y[k] = xyz[3 * i + 1];
  if (images) {
    int lp, b;
    type_decode((int)(key[k] & 15ull), lp, b);
    z[k] = image_z(md, l, a, lp, b, xyz[3 * i + 2]);
  } else {
    z[k] = xyz[3 * i + 2];
  }
  qq[k] = q[i];
}

static GroupGeom group_geom(Ctx &c, const Group &g, const int64_t *cnt) {
  GroupGeom gg;
  const double H = g.root[3];
  gg.o[0] = g.root[0] - H;
  gg.o[1] = g.root[1] - H;
  gg.o[2] = g.root[2] - H;
  gg.s = double(1 << DMAX) / (2.0 * H);
  gg.l = g.l;
  gg.a = g.a;
  int64_t off = 0;
  for (int t = 0; t < 2 * c.md.L; ++t) {
    int lp, b;
    type_decode(t, lp, b);
    gg.type_off[t] = off;
    off += cnt[lp];
  }
  return gg;
}

static void gather(Ctx &c, Group &g, PointSet &P, int images, const double *q, const double *xyz,
                   const int32_t *layer) {
  P.x = c.arena.get<double>(P.np);
  P.y = c.arena.get<double>(P.np);
  P.z = c.arena.get<double>(P.np);
  P.q = c.arena.get<double>(P.np);
  if (P.np) {
    k_gather_points<<<(unsigned)((P.np + 255) / 256), 256, 0, c.stream>>>(P.np, P.key, P.src, q, xyz, c.md, g.l,
                                                                          g.a, images, P.x, P.y, P.z, P.q, layer);
    LPB_LAUNCH();
    c.launches++;
  }
}

// targets of the group, sorted by their depth-DMAX Morton keys (every coarser key is a prefix)
void build_group_targets(Ctx &c, Group &g, int64_t n, const double *q, const double *xyz, const int32_t *layer,
                         uint32_t *const *rank, const int64_t *cnt) {
  GroupGeom gg = group_geom(c, g, cnt);
  RankPtrs rk;
  for (int k = 0; k <= c.md.L; ++k) rk.r[k] = rank[k];
  g.T.np = cnt[g.l];
  g.T.key = c.arena.get<uint64_t>(g.T.np);
  g.T.src = c.arena.get<uint32_t>(g.T.np);
  k_make_targets<<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>(n, xyz, layer, rk, gg, g.T.key, g.T.src);
  LPB_LAUNCH();
  c.launches++;
  radix_sort(c, g.T.key, g.T.src, g.T.np, DMAX * 3 + 4, 4);  // target keys: low 4 bits are zero
  gather(c, g, g.T, 0, q, xyz, layer);
}

// images of the group, sorted by (depth-D leaf key, type, input order): every (leaf box,
// type) pair is one contiguous run
void build_group_images(Ctx &c, Group &g, int64_t n, const double *q, const double *xyz, const int32_t *layer,
                        uint32_t *const *rank, const int64_t *cnt) {
  GroupGeom gg = group_geom(c, g, cnt);
  RankPtrs rk;
  for (int k = 0; k <= c.md.L; ++k) rk.r[k] = rank[k];
  int64_t tot = 0;
  for (int t = 0; t < 2 * c.md.L; ++t) {
    int lp, b;
    type_decode(t, lp, b);
    tot += cnt[lp];
  }
  g.I.np = tot;
  g.I.key = c.arena.get<uint64_t>(g.I.np);
  g.I.src = c.arena.get<uint32_t>(g.I.np);
  k_make_images<<<(unsigned)((n + 255) / 256), 256, 0, c.stream>>>(n, xyz, layer, c.md, rk, gg, g.D, g.I.key,
                                                                   g.I.src);
  LPB_LAUNCH();
  c.launches++;
  radix_sort(c, g.I.key, g.I.src, g.I.np, g.D * 3 + 4, 0);
  gather(c, g, g.I, 1, q, xyz, layer);
}

// number of non-empty target boxes at every level 2..DMAX (automatic depth rule)
__global__ void k_count_levels(int64_t np, const uint64_t *key, uint32_t *cnt) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (int l = 2; l <= DMAX; ++l) {
    bool f = false;
    if (k < np) {
      const int sh = 4 + 3 * (DMAX - l);
      f = (k == 0) || ((key[k] >> sh) != (key[k - 1] >> sh));
    }
    const unsigned b = __popc(__ballot_sync(0xffffffffu, f));
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(&cnt[l], b);
  }
}
void count_levels(Ctx &c, Group &g, uint32_t *d_counts) {
  if (!g.T.np) return;
  k_count_levels<<<(unsigned)((g.T.np + 255) / 256), 256, 0, c.stream>>>(g.T.np, g.T.key, d_counts);
  LPB_LAUNCH();
  c.launches++;
}

// ---------------------------------------------------------------------------------------
// boxes per level
// ---------------------------------------------------------------------------------------
__global__ void k_leaf_flags(int64_t np, const uint64_t *key, int sh, uint32_t *f) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < np) f[k] = (k == 0 || (key[k] >> sh) != (key[k - 1] >> sh)) ? 1u : 0u;
}
__global__ void k_seg_flags(int64_t np, const uint64_t *key, int sh, uint32_t *f) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= np) return;
  const uint64_t a = ((key[k] >> 4) >> sh << 4) | (key[k] & 15ull);
  const uint64_t b = k ? (((key[k - 1] >> 4) >> sh << 4) | (key[k - 1] & 15ull)) : 0ull;
  f[k] = (k == 0 || a != b) ? 1u : 0u;
}
// flagged item k starts box idx[k]
__global__ void k_leaf_boxes(int64_t np, const uint64_t *key, int sh, const uint32_t *f, const uint32_t *idx,
                             uint64_t *bkey, uint32_t *bstart) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < np && f[k]) {
    bkey[idx[k]] = key[k] >> sh;
    bstart[idx[k]] = (uint32_t)k;
  }
}
__global__ void k_counts_from_starts(const uint32_t *d_n, const uint32_t *start, uint32_t total, uint32_t *cnt,
                                     int64_t cap) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t n = *d_n;
  if (b < n && b < cap) cnt[b] = ((b + 1 < n) ? start[b + 1] : total) - start[b];
}
__global__ void k_seg_fill(int64_t np, const uint64_t *key, const uint32_t *f, const uint32_t *sidx,
                           const uint32_t *bf, const uint32_t *bidx, uint32_t *sstart, uint32_t *sbox,
                           uint32_t *stype) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < np && f[k]) {
    const uint32_t s = sidx[k];
    sstart[s] = (uint32_t)k;
    sbox[s] = bidx[k] + bf[k] - 1u;
    stype[s] = (uint32_t)(key[k] & 15ull);
  }
}
// parents of level l+1 boxes
__global__ void k_parent_flags(const uint32_t *d_n, const uint64_t *ckey, uint32_t *f, int64_t cap) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t n = *d_n;
  if (j < n && j < cap) f[j] = (j == 0 || (ckey[j] >> 3) != (ckey[j - 1] >> 3)) ? 1u : 0u;
  else if (j < cap) f[j] = 0u;
}
__global__ void k_parent_fill(const uint32_t *d_n, const uint64_t *ckey, const uint32_t *f, const uint32_t *idx,
                              uint32_t *cparent, uint64_t *pkey, uint32_t *pstart, int64_t cap) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t n = *d_n;
  if (j >= n || j >= cap) return;
  const uint32_t pid = idx[j] + f[j] - 1u;
  cparent[j] = pid;
  if (f[j]) {
    pkey[pid] = ckey[j] >> 3;
    pstart[pid] = (uint32_t)j;
  }
}

static int64_t level_cap(int64_t np, int l) {
  int64_t c = 1;
  for (int k = 0; k < l && c < np; ++k) c *= 8;
  return c < np ? c : np;
}

static void build_levels(Ctx &c, PointSet &P, int D, bool images) {
  const int64_t np = P.np;
  const unsigned pb = (unsigned)((np + 255) / 256);
  for (int l = 0; l <= DMAX; ++l) P.lev[l] = Level();
  if (!np) return;
  // targets carry depth-DMAX keys, images depth-D keys (both shifted by 4 type bits)
  const int sh = images ? 4 : 4 + 3 * (DMAX - D);
  uint32_t *f = c.arena.get<uint32_t>(np), *idx = c.arena.get<uint32_t>(np);
  Level &Lf = P.lev[D];
  const int64_t capD = level_cap(np, D);
  Lf.key = c.arena.get<uint64_t>(capD);
  Lf.start = c.arena.get<uint32_t>(capD);
  Lf.count = c.arena.get<uint32_t>(capD);
  Lf.d_n = c.arena.get<uint32_t>(1);
  k_leaf_flags<<<pb, 256, 0, c.stream>>>(np, P.key, sh, f);
  LPB_LAUNCH();
  scan_u32(c, f, idx, np, Lf.d_n);
  k_leaf_boxes<<<pb, 256, 0, c.stream>>>(np, P.key, sh, f, idx, Lf.key, Lf.start);
  LPB_LAUNCH();
  k_counts_from_starts<<<(unsigned)((capD + 255) / 256), 256, 0, c.stream>>>(Lf.d_n, Lf.start, (uint32_t)np,
                                                                              Lf.count, capD);
  LPB_LAUNCH();
  c.launches += 3;
  if (images) {
    uint32_t *sf = c.arena.get<uint32_t>(np), *sidx = c.arena.get<uint32_t>(np);
    P.seg_start = c.arena.get<uint32_t>(np);
    P.seg_count = c.arena.get<uint32_t>(np);
    P.seg_box = c.arena.get<uint32_t>(np);
    P.seg_type = c.arena.get<uint32_t>(np);
    P.d_nseg = c.arena.get<uint32_t>(1);
    k_seg_flags<<<pb, 256, 0, c.stream>>>(np, P.key, 0, sf);
    LPB_LAUNCH();
    scan_u32(c, sf, sidx, np, P.d_nseg);
    k_seg_fill<<<pb, 256, 0, c.stream>>>(np, P.key, sf, sidx, f, idx, P.seg_start, P.seg_box, P.seg_type);
    LPB_LAUNCH();
    k_counts_from_starts<<<pb, 256, 0, c.stream>>>(P.d_nseg, P.seg_start, (uint32_t)np, P.seg_count, np);
    LPB_LAUNCH();
    c.launches += 3;
  }
  for (int l = D - 1; l >= 2; --l) {
    Level &C = P.lev[l + 1], &Pa = P.lev[l];
    const int64_t ccap = level_cap(np, l + 1), pcap = level_cap(np, l);
    uint32_t *cf = c.arena.get<uint32_t>(ccap), *cidx = c.arena.get<uint32_t>(ccap);
    Pa.key = c.arena.get<uint64_t>(pcap);
    Pa.start = c.arena.get<uint32_t>(pcap);
    Pa.count = c.arena.get<uint32_t>(pcap);
    Pa.d_n = c.arena.get<uint32_t>(1);
    C.parent = c.arena.get<uint32_t>(ccap);
    const unsigned cb = (unsigned)((ccap + 255) / 256);
    k_parent_flags<<<cb, 256, 0, c.stream>>>(C.d_n, C.key, cf, ccap);
    LPB_LAUNCH();
    scan_u32(c, cf, cidx, ccap, Pa.d_n);
    k_parent_fill<<<cb, 256, 0, c.stream>>>(C.d_n, C.key, cf, cidx, C.parent, Pa.key, Pa.start, ccap);
    LPB_LAUNCH();
    k_counts_from_starts<<<(unsigned)((pcap + 255) / 256), 256, 0, c.stream>>>(Pa.d_n, Pa.start, 0u, Pa.count,
                                                                                pcap);
    LPB_LAUNCH();
    c.launches += 3;
  }
}

__global__ void k_fix_last_count(const uint32_t *d_nc, const uint32_t *d_np, const uint32_t *pstart,
                                 uint32_t *pcount) {
  // the last parent's count is (number of children) - start
  const uint32_t np = *d_np;
  if (np) pcount[np - 1] = *d_nc - pstart[np - 1];
}

// points of every box of a coarser target level: its first child's first point, up to the next
// box's first point (points are sorted by key, so a box's points are one contiguous run)
__global__ void k_point_ranges(const uint32_t *d_n, const uint32_t *start, const uint32_t *cpstart, uint32_t np,
                               uint32_t *pstart, uint32_t *pcount, int64_t cap) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t n = *d_n;
  if (b >= n || b >= cap) return;
  const uint32_t s = cpstart[start[b]];
  pstart[b] = s;
  pcount[b] = ((b + 1 < n) ? cpstart[start[b + 1]] : np) - s;
}

void build_group_boxes(Ctx &c, Group &g) {
  build_levels(c, g.T, g.D, false);
  build_levels(c, g.I, g.D, true);
  if (g.T.np) {
    g.T.lev[g.D].pstart = g.T.lev[g.D].start;
    g.T.lev[g.D].pcount = g.T.lev[g.D].count;
    for (int l = g.D - 1; l >= 2; --l) {
      Level &P = g.T.lev[l];
      const int64_t cap = level_cap(g.T.np, l);
      P.pstart = c.arena.get<uint32_t>(cap);
      P.pcount = c.arena.get<uint32_t>(cap);
      k_point_ranges<<<(unsigned)((cap + 255) / 256), 256, 0, c.stream>>>(P.d_n, P.start, g.T.lev[l + 1].pstart,
                                                                         (uint32_t)g.T.np, P.pstart, P.pcount, cap);
      LPB_LAUNCH();
      c.launches++;
    }
  }
  for (int which = 0; which < 2; ++which) {
    PointSet &P = which ? g.I : g.T;
    if (!P.np) continue;
    for (int l = g.D - 1; l >= 2; --l) {
      k_fix_last_count<<<1, 1, 0, c.stream>>>(P.lev[l + 1].d_n, P.lev[l].d_n, P.lev[l].start, P.lev[l].count);
      LPB_LAUNCH();
      c.launches++;
    }
  }
}

// ---------------------------------------------------------------------------------------
// interaction lists with separation ws.  Far list (multipole-to-local, V): source boxes at
// offset d with |d|_inf > ws whose parent lies within ws of the target's parent.  Near list
// (U): |d|_inf <= ws.  Dense layout: [target box][offset slot] -> source box index or -1, with
// the slots of WS_MAX (offsets of a smaller ws leave the outer slots at -1).
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ int64_t find_key(const uint64_t *keys, int64_t n, uint64_t k) {
  int64_t lo = 0, hi = n - 1;
  while (lo <= hi) {
    const int64_t m = (lo + hi) >> 1;
    const uint64_t v = keys[m];
    if (v == k) return m;
    if (v < k) lo = m + 1; else hi = m - 1;
  }
  return -1;
}

// dense box index of a level: grid[Morton key] = box index or -1 (levels up to GRID_LEV_MAX)
constexpr int GRID_LEV_MAX = 8;
__global__ void k_grid_fill(const uint64_t *key, const uint32_t *d_n, int32_t *grid, int64_t cap) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b < *d_n && b < cap) grid[key[b]] = (int32_t)b;
}
static const int32_t *level_grid(Ctx &c, const Level &L, int lev, int64_t np) {
  if (lev > GRID_LEV_MAX || !L.n) return nullptr;
  const size_t cells = (size_t)1 << (3 * lev);
  int32_t *grid = c.arena.get<int32_t>(cells);
  LPB_CUDA(cudaMemsetAsync(grid, 0xff, sizeof(int32_t) * cells, c.stream));
  const int64_t cap = level_cap(np, lev);
  k_grid_fill<<<(unsigned)((cap + 255) / 256), 256, 0, c.stream>>>(L.key, L.d_n, grid, cap);
  LPB_LAUNCH();
  c.launches++;
  return grid;
}

// far = 1: V list over NOFF slots; far = 0: near list over NNEAR slots
// react: reaction list (targets vs images): also records the classes in use
// sgrid: dense box index of the source level (nullptr: binary search in skey)
__global__ void k_lists(const uint64_t *tkey, const uint32_t *d_nt, const uint64_t *skey, const uint32_t *d_ns,
                        const int32_t *sgrid, int lev, int far, int react, int a, int ws, int32_t *out,
                        uint8_t *used) {
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int nslot = far ? NOFF : NNEAR;
  const int64_t t = gid / nslot;
  const int o = (int)(gid % nslot);
  const int64_t nt = *d_nt;
  if (t >= nt) return;
  int dx, dy, dz;
  if (far) off_decode(o, dx, dy, dz);
  else near_decode(o, dx, dy, dz);
  const uint64_t k = tkey[t];
  const int ix = compact3(k >> 2), iy = compact3(k >> 1), iz = compact3(k);
  const int jx = ix + dx, jy = iy + dy, jz = iz + dz, nc = 1 << lev;
  int32_t res = -1;
  const int cheb = cheb3(dx, dy, dz);
  bool ok = jx >= 0 && jy >= 0 && jz >= 0 && jx < nc && jy < nc && jz < nc;
  if (far) {
    ok = ok && cheb > ws && abs((jx >> 1) - (ix >> 1)) <= ws && abs((jy >> 1) - (iy >> 1)) <= ws &&
         abs((jz >> 1) - (iz >> 1)) <= ws;
  } else {
    ok = ok && cheb <= ws;
  }
  const int64_t ns = *d_ns;
  if (ok && ns > 0) {
    const uint64_t sk = (spread3(jx) << 2) | (spread3(jy) << 1) | spread3(jz);
    const int64_t s = sgrid ? (int64_t)sgrid[sk] : find_key(skey, ns, sk);
    if (s >= 0) {
      res = (int32_t)s;
      if (react && far && used) {
        const int half = 1 << (lev - 1);
        const int kt = (a == 1) ? iz - half : half - 1 - iz;
        const int ks = (a == 1) ? half - 1 - jz : jz - half;
        const int kk = kk_index(kt, ks);
        if (kk >= 0) used[rho_index(dx, dy) * NKK + kk] = 1;
      }
    }
  }
  out[t * nslot + o] = res;
}

// reaction target rows: boxes at k_t = 0 .. 2 ws box layers from the interface, per row
__global__ void k_rows(const uint64_t *tkey, const uint32_t *d_nt, int lev, int a, int nkt, int32_t *rows,
                       uint32_t *nrows, int32_t *ktrow, int64_t cap) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= *d_nt) return;
  const int iz = compact3(tkey[t]);
  const int half = 1 << (lev - 1);
  const int kt = (a == 1) ? iz - half : half - 1 - iz;
  ktrow[t] = kt;
  if (kt >= 0 && kt < nkt) {
    const uint32_t pos = atomicAdd(&nrows[kt], 1u);
    rows[kt * cap + pos] = (int32_t)t;
  }
}

void build_group_lists(Ctx &c, Group &g, int parts) {
  const int ws = c.ws, nkt = 2 * c.ws + 1;
  for (int l = 2; l <= g.D; ++l) {
    const Level &T = g.T.lev[l];
    const Level &I = g.I.lev[l];
    const int64_t nt = T.n;
    if (!nt) continue;
    const unsigned fb = (unsigned)((nt * NOFF + 255) / 256);
    if (g.is_free && (parts & 1) && l <= g.Df) {
      g.vfree[l] = c.arena.get<int32_t>(nt * NOFF);
      const int32_t *tg = level_grid(c, T, l, g.T.np);
      k_lists<<<fb, 256, 0, c.stream>>>(T.key, T.d_n, T.key, T.d_n, tg, l, 1, 0, g.a, ws, g.vfree[l], nullptr);
      LPB_LAUNCH();
      c.launches++;
    }
    if ((parts & 2) && I.n) {
      g.vreact[l] = c.arena.get<int32_t>(nt * NOFF);
      g.used[l] = c.arena.get<uint8_t>(NREACT_CLS);
      LPB_CUDA(cudaMemsetAsync(g.used[l], 0, NREACT_CLS, c.stream));
      const int32_t *ig = level_grid(c, I, l, g.I.np);
      k_lists<<<fb, 256, 0, c.stream>>>(T.key, T.d_n, I.key, I.d_n, ig, l, 1, 1, g.a, ws, g.vreact[l], g.used[l]);
      LPB_LAUNCH();
      g.rows[l] = c.arena.get<int32_t>((size_t)NKT * nt);
      g.nrows[l] = c.arena.get<uint32_t>(NKT);
      g.ktrow[l] = c.arena.get<int32_t>(nt);
      LPB_CUDA(cudaMemsetAsync(g.nrows[l], 0, NKT * sizeof(uint32_t), c.stream));
      k_rows<<<(unsigned)((nt + 255) / 256), 256, 0, c.stream>>>(T.key, T.d_n, l, g.a, nkt, g.rows[l], g.nrows[l],
                                                                 g.ktrow[l], nt);
      LPB_LAUNCH();
      c.launches += 2;
    }
  }
  const int Df = g.Df;
  const int64_t ntf = g.T.lev[Df].n;
  if (g.is_free && (parts & 1) && ntf) {
    g.ufree = c.arena.get<int32_t>(ntf * NNEAR);
    k_lists<<<(unsigned)((ntf * NNEAR + 255) / 256), 256, 0, c.stream>>>(
        g.T.lev[Df].key, g.T.lev[Df].d_n, g.T.lev[Df].key, g.T.lev[Df].d_n, nullptr, Df, 0, 0, g.a, ws, g.ufree,
        nullptr);
    LPB_LAUNCH();
    c.launches++;
  }
  const int D = g.D;
  const int64_t nt = g.T.lev[D].n;
  if (!nt) return;
  const unsigned nb = (unsigned)((nt * NNEAR + 255) / 256);
  if ((parts & 2) && g.I.lev[D].n) {
    g.ureact = c.arena.get<int32_t>(nt * NNEAR);
    k_lists<<<nb, 256, 0, c.stream>>>(g.T.lev[D].key, g.T.lev[D].d_n, g.I.lev[D].key, g.I.lev[D].d_n, nullptr, D, 0,
                                      1, g.a, ws, g.ureact, nullptr);
    LPB_LAUNCH();
    c.launches++;
  }
}

}  // namespace lpb

namespace lpb {

// ---------------------------------------------------------------------------------------
// Adaptive dual-tree lists of a group's free-space target tree with itself (Sec. 3.5 builds the
// method on the adaptive FMM framework; diagnostic for now, the evaluation uses uniform trees).
// A box of level l >= 3 exists in the adaptive tree when its parent exists and holds more than s
// targets (every box of level 2 exists); a box is a leaf when it holds at most s or l = D.  The
// dual traversal starts from every pair of level-2 boxes and runs level-synchronously over
// frontiers of box pairs: a pair that is not near (separation ws: the coarser box grown by ws - 1
// of its sides meets the finer one) is V (same level), W (target leaf, finer source) or X (source
// leaf, finer target); a near pair of two leaves is U; any other near pair is replaced by its
// child pairs (both boxes refined when both have children, else the one that has).
// ---------------------------------------------------------------------------------------
struct APair {
  uint32_t bt, bs;  // box indices in their levels
  int32_t lt, ls;   // levels
};
struct ALevel {
  const uint64_t *key;
  const uint32_t *start, *count, *pcount, *parent;
  const uint8_t *flag;  // bit 0: the box exists in the adaptive tree; bit 1: it is a leaf
  uint32_t n;
};

__global__ void k_adapt_flags(int l, int D, int s, ALevel cur, const uint8_t *pflag, uint8_t *flag) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= cur.n) return;
  bool present = true;
  if (l > 2) {
    const uint8_t pf = pflag[cur.parent[b]];
    present = (pf & 1) && !(pf & 2);
  }
  const bool leaf = present && (cur.pcount[b] <= (uint32_t)s || l == D);
  flag[b] = (uint8_t)((present ? 1 : 0) | (leaf ? 2 : 0));
}

__global__ void k_adapt_init(uint32_t n2, APair *pairs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (int64_t)n2 * n2) return;
  pairs[i] = APair{(uint32_t)(i / n2), (uint32_t)(i % n2), 2, 2};
}

// boxes (la, ka) and (lb, kb) near for separation ws (integer geometry at the finer level)
__device__ bool adapt_near(int la, uint64_t ka, int lb, uint64_t kb, int ws) {
  const int L = max(la, lb);
  const int64_t sa = (int64_t)1 << (L - la), sb = (int64_t)1 << (L - lb);
  const int64_t ga = la <= lb ? (ws - 1) * sa : 0, gb = lb < la ? (ws - 1) * sb : 0;
  for (int d = 0; d < 3; ++d) {
    const int64_t u = compact3(ka >> (2 - d)), v = compact3(kb >> (2 - d));
    if ((u + 1) * sa + ga < v * sb - gb || (v + 1) * sb + gb < u * sa - ga) return false;
  }
  return true;
}

// classify every frontier pair; nchild[i] = its child pairs (0 when classified).  Records of
// 5 int64: kind (0 V, 1 U, 2 W, 3 X), lt, key t, ls, key s; at most one per pair
__global__ void k_adapt_step(const APair *pairs, uint32_t np, const ALevel *lv, int ws, uint32_t *nchild,
                             int64_t *rec, uint32_t *nrec) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const APair P = pairs[i];
  const ALevel &T = lv[P.lt], &S = lv[P.ls];
  if (P.bt >= T.n || P.bs >= S.n) {  // cannot happen for pairs built below; checked all the same
    nchild[i] = 0;
    return;
  }
  const uint64_t kt = T.key[P.bt], ks = S.key[P.bs];
  const bool tl = T.flag[P.bt] & 2, sl = S.flag[P.bs] & 2;
  int kind = -1;
  uint32_t nc = 0;
  if (!adapt_near(P.lt, kt, P.ls, ks, ws)) kind = P.lt == P.ls ? 0 : (P.ls > P.lt ? 2 : 3);
  else if (tl && sl) kind = 1;
  else nc = (tl ? 1u : T.count[P.bt]) * (sl ? 1u : S.count[P.bs]);
  nchild[i] = nc;
  if (kind >= 0) {
    const uint32_t r = atomicAdd(nrec, 1u);
    if (r < np) {
      int64_t *o = rec + (size_t)r * 5;
      o[0] = kind; o[1] = P.lt; o[2] = (int64_t)kt; o[3] = P.ls; o[4] = (int64_t)ks;
    }
  }
}

__global__ void k_adapt_children(const APair *pairs, uint32_t np, const ALevel *lv, const uint32_t *nchild,
                                 const uint32_t *off, APair *next, uint32_t cap) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np || !nchild[i]) return;
  const APair P = pairs[i];
  const ALevel &T = lv[P.lt], &S = lv[P.ls];
  const bool tl = T.flag[P.bt] & 2, sl = S.flag[P.bs] & 2;
  const uint32_t nt = tl ? 1u : T.count[P.bt], ns = sl ? 1u : S.count[P.bs];
  for (uint32_t a = 0; a < nt; ++a)
    for (uint32_t b = 0; b < ns; ++b) {
      const uint64_t o = (uint64_t)off[i] + (uint64_t)a * ns + b;
      if (o >= cap) continue;
      next[o] = APair{tl ? P.bt : T.start[P.bt] + a, sl ? P.bs : S.start[P.bs] + b, tl ? P.lt : P.lt + 1,
                      sl ? P.ls : P.ls + 1};
    }
}

void adaptive_lists(Ctx &c, Group &g, int s, int ws, std::vector<int64_t> &rec) {
  rec.clear();
  PointSet &P = g.T;
  const int D = g.Df;
  if (!P.np || D < 2) return;
  // flags, top down
  std::vector<ALevel> hl(DMAX + 1);
  for (int l = 2; l <= D; ++l) {
    const Level &L = P.lev[l];
    uint8_t *f = c.arena.get<uint8_t>((size_t)std::max<int64_t>(L.n, 1));
    hl[l] = ALevel{L.key, L.start, L.count, L.pcount, L.parent, f, (uint32_t)L.n};
    if (L.n)
      k_adapt_flags<<<(unsigned)((L.n + 255) / 256), 256, 0, c.stream>>>(l, D, s, hl[l], l > 2 ? hl[l - 1].flag : nullptr,
                                                                         f);
    LPB_LAUNCH();
  }
  ALevel *dl = c.arena.get<ALevel>(DMAX + 1);
  LPB_CUDA(cudaMemcpyAsync(dl, hl.data(), sizeof(ALevel) * (DMAX + 1), cudaMemcpyHostToDevice, c.stream));
  const uint32_t n2 = (uint32_t)P.lev[2].n;
  uint64_t F = (uint64_t)n2 * n2;
  constexpr uint64_t FMAX = (uint64_t)1 << 26;  // frontier pairs this diagnostic handles
  if (F > FMAX) throw StatusError{LPBFMM_ERR_UNSUPPORTED};
  APair *pairs = c.arena.get<APair>((size_t)std::max<uint64_t>(F, 1));
  if (F) k_adapt_init<<<(unsigned)((F + 255) / 256), 256, 0, c.stream>>>(n2, pairs);
  LPB_LAUNCH();
  uint32_t *hp = (uint32_t *)c.h_pinned;
  for (int step = 0; F > 0; ++step) {
    if (step > 4 * DMAX) throw StatusError{LPBFMM_ERR_UNSUPPORTED};
    uint32_t *nchild = c.arena.get<uint32_t>(F), *off = c.arena.get<uint32_t>(F), *d2 = c.arena.get<uint32_t>(2);
    int64_t *drec = c.arena.get<int64_t>((size_t)F * 5);
    LPB_CUDA(cudaMemsetAsync(d2, 0, 2 * sizeof(uint32_t), c.stream));
    k_adapt_step<<<(unsigned)((F + 255) / 256), 256, 0, c.stream>>>(pairs, (uint32_t)F, dl, ws, nchild, drec, d2);
    LPB_LAUNCH();
    scan_u32(c, nchild, off, (int64_t)F, d2 + 1);
    LPB_CUDA(cudaMemcpyAsync(hp, d2, 2 * sizeof(uint32_t), cudaMemcpyDeviceToHost, c.stream));
    LPB_CUDA(cudaStreamSynchronize(c.stream));
    const uint32_t nr = std::min<uint64_t>(hp[0], F), nnext = hp[1];
    const size_t base = rec.size();
    rec.resize(base + (size_t)nr * 5);
    if (nr) LPB_CUDA(cudaMemcpy(rec.data() + base, drec, sizeof(int64_t) * nr * 5, cudaMemcpyDeviceToHost));
    if (nnext > FMAX) throw StatusError{LPBFMM_ERR_UNSUPPORTED};
    APair *next = nnext ? c.arena.get<APair>(nnext) : nullptr;
    if (nnext)
      k_adapt_children<<<(unsigned)((F + 255) / 256), 256, 0, c.stream>>>(pairs, (uint32_t)F, dl, nchild, off, next,
                                                                         nnext);
    LPB_LAUNCH();
    pairs = next;
    F = nnext;
  }
  LPB_CUDA(cudaStreamSynchronize(c.stream));
}

}  // namespace lpb
