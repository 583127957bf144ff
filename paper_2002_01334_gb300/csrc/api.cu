// C-ABI entry points and host orchestration (Algorithm 2 of the paper: the free-space FMM of
// every layer plus Algorithm 1 for every reaction component, summed per target).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <thread>

#include "internal.h"

namespace lpb {
void init_fmm_tables(Ctx &c);

// ---------------------------------------------------------------------------------------
// arena
// ---------------------------------------------------------------------------------------
void *Arena::alloc(size_t bytes) {
  bytes = (bytes + 255) & ~size_t(255);
  used_total += bytes;
  for (auto &ch : chunks)
    if (ch.size - ch.used >= bytes) {
      void *p = ch.p + ch.used;
      ch.used += bytes;
      return p;
    }
  size_t sz = std::max(bytes, std::max(want, (size_t)64 << 20));
  char *p = nullptr;
  cudaError_t e = cudaMalloc(&p, sz);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw StatusError{LPBFMM_ERR_OOM};
  }
  chunks.push_back(Chunk{p, sz, bytes});
  return p;
}
void Arena::reset() {
  if (chunks.size() > 1 || (chunks.size() == 1 && chunks[0].size < used_total)) {
    want = std::max(want, used_total + (used_total >> 3));
    release();
  }
  for (auto &ch : chunks) ch.used = 0;
  used_total = 0;
}
void Arena::release() {
  for (auto &ch : chunks) cudaFree(ch.p);
  chunks.clear();
}

void prof_mark(Ctx &c, const char *name) {
  if (c.nev >= 64) return;
  cudaEventRecord(c.ev[c.nev], c.stream);
  c.prof_names.push_back(name);
  c.prof_launch.push_back(c.launches);
  ++c.nev;
}

// ---------------------------------------------------------------------------------------
// host tables: Gaunt coefficients and Legendre-product coefficients
// ---------------------------------------------------------------------------------------
static void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w) {
  x.resize(n);
  w.resize(n);
  for (int i = 0; i < n; ++i) {
    long double z = cosl(3.14159265358979323846264338L * (i + 0.75L) / (n + 0.5L)), dp = 1;
    for (int it = 0; it < 200; ++it) {
      long double p0 = 1, p1 = z;
      for (int k = 2; k <= n; ++k) { long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
      dp = n * (z * p1 - p0) / (z * z - 1);
      long double dz = p1 / dp;
      z -= dz;
      if (fabsl(dz) < 1e-19L) break;
    }
    long double p0 = 1, p1 = z;
    for (int k = 2; k <= n; ++k) { long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
    dp = n * (z * p1 - p0) / (z * z - 1);
    x[i] = (double)z;
    w[i] = (double)(2 / ((1 - z * z) * dp * dp));
  }
}

// G[a][c][q] = int Y_a^alpha Y_q^{gamma-alpha} conj(Y_c^gamma) dOmega (all real), full indices a, c
// sqrt((K+d)! (K-d)!) for 0 <= d <= K <= KMAX_TAB, the normalisation of the scaled
// Sommerfeld tables (long double products, then rounded once)
// Phat_q^k(cos theta), q <= 2p, of the NDIR translation directions: the free-space M2L classes
// (rho^2 index ri, dz) at index ri * NDZ + dz + OFF_R, b = (rho, 0, -dz), and the child-parent
// directions b = (1, 1, -1) / (1, 1, 1) (index NFREE_CLS, NFREE_CLS + 1).  Orthonormal,
// Condon-Shortley phase, by the standard three-term recurrences in long double.
static std::vector<double> phat_dir_table(int p) {
  const int qmax = 2 * p, npl = (qmax + 1) * (qmax + 2) / 2;
  std::vector<double> out((size_t)NDIR * npl, 0.0);
  auto idx = [](int q, int k) { return q * (q + 1) / 2 + k; };
  for (int dir = 0; dir < NDIR; ++dir) {
    long double x;
    if (dir < NFREE_CLS) {
      const int ri = dir / NDZ, dz = dir % NDZ - OFF_R;
      const long double bz = -dz, bn = sqrtl((long double)rho2_of(ri) + (long double)dz * dz);
      x = bn > 0 ? bz / bn : 1.0L;
    } else {
      x = (dir == NFREE_CLS ? -1.0L : 1.0L) / sqrtl(3.0L);
    }
    std::vector<long double> P(npl, 0.0L);
    const long double s = sqrtl(fmaxl(0.0L, 1.0L - x * x));
    P[0] = 0.5L / sqrtl(3.14159265358979323846264338L);
    for (int k = 1; k <= qmax; ++k) P[idx(k, k)] = -sqrtl((2.0L * k + 1) / (2.0L * k)) * s * P[idx(k - 1, k - 1)];
    for (int k = 0; k < qmax; ++k) {
      P[idx(k + 1, k)] = sqrtl(2.0L * k + 3) * x * P[idx(k, k)];
      for (int q = k + 2; q <= qmax; ++q) {
        const long double qq = (long double)q * q - (long double)k * k;
        const long double a = sqrtl((4.0L * q * q - 1) / qq);
        const long double b = sqrtl(((q - 1.0L) * (q - 1.0L) - (long double)k * k) * (2.0L * q + 1) /
                                    ((2.0L * q - 3) * qq));
        P[idx(q, k)] = a * x * P[idx(q - 1, k)] - b * P[idx(q - 2, k)];
      }
    }
    for (int e = 0; e < npl; ++e) out[(size_t)dir * npl + e] = (double)P[e];
  }
  return out;
}

static std::vector<double> sfac_table() {
  const int n = KMAX_TAB + 1;
  std::vector<long double> f(2 * n + 1);
  f[0] = 1.0L;
  for (int k = 1; k <= 2 * n; ++k) f[k] = f[k - 1] * (long double)k;
  std::vector<double> out((size_t)n * n, 0.0);
  for (int K = 0; K < n; ++K)
    for (int d = 0; d <= K; ++d) out[(size_t)K * n + d] = (double)sqrtl(f[K + d] * f[K - d]);
  return out;
}

static std::vector<double> gaunt_table(int p) {
  const int NF = (p + 1) * (p + 1), NQ = 2 * p + 1, qmax = 2 * p;
  std::vector<double> G((size_t)NF * NF * NQ, 0.0);
  std::vector<double> gx, gw;
  gauss_legendre(2 * p + 4, gx, gw);
  const int nh = (qmax + 1) * (qmax + 2) / 2;
  std::vector<double> Pl((size_t)gx.size() * nh);
  for (size_t g = 0; g < gx.size(); ++g) phat_all(gx[g], qmax, &Pl[g * nh]);
  for (int n = 0; n <= p; ++n)
    for (int al = -n; al <= n; ++al)
      for (int nu = 0; nu <= p; ++nu)
        for (int ga = -nu; ga <= nu; ++ga) {
          const int k = ga - al;
          for (int q = std::abs(n - nu); q <= n + nu; q += 2) {
            if (std::abs(k) > q) continue;
            double s = 0.0;
            for (size_t g = 0; g < gx.size(); ++g) {
              const double *P = &Pl[g * nh];
              s += gw[g] * phat_signed(P, n, al) * phat_signed(P, q, k) * phat_signed(P, nu, ga);
            }
            G[((size_t)fidx(n, al) * NF + fidx(nu, ga)) * NQ + q] = 2.0 * PI * s;
          }
        }
  return G;
}

// Legendre-product expansion: the associated-Legendre part pi_n^m(x) of the solid harmonic
// recurrence at r = 1 (x = lambda_z / lambda > 1, t = x^2 - 1) equals (1/x)^i sum_k c_k t^k,
// i = (n - m) mod 2.  Returns c[hidx(n,m)*tpk + k].
static std::vector<double> tpoly_table(int p, int &tpk) {
  tpk = p / 2 + 2;
  const int K = (p + 1) * (p + 2) / 2;
  std::vector<double> out((size_t)K * tpk, 0.0);
  typedef std::vector<long double> Poly;
  auto add = [](const Poly &a, long double sa, const Poly &b, long double sb) {
    Poly r(std::max(a.size(), b.size()), 0.0L);
    for (size_t i = 0; i < a.size(); ++i) r[i] += sa * a[i];
    for (size_t i = 0; i < b.size(); ++i) r[i] += sb * b[i];
    return r;
  };
  auto mul1t = [](const Poly &a) {  // (1 + t) a
    Poly r(a.size() + 1, 0.0L);
    for (size_t i = 0; i < a.size(); ++i) { r[i] += a[i]; r[i + 1] += a[i]; }
    return r;
  };
  for (int m = 0; m <= p; ++m) {
    Poly Em2, Om2, Em1{1.0L}, Om1;
    auto store = [&](int n, const Poly &E, const Poly &O) {
      const Poly c = ((n - m) % 2 == 0) ? E : mul1t(O);
      for (size_t k = 0; k < c.size() && (int)k < tpk; ++k) out[(size_t)hidx(n, m) * tpk + k] = (double)c[k];
    };
    store(m, Em1, Om1);
    if (m + 1 > p) continue;
    Poly E{}, O{sqrtl(2.0L * m + 3.0L)};
    store(m + 1, E, O);
    Em2 = Em1; Om2 = Om1; Em1 = E; Om1 = O;
    for (int n = m + 2; n <= p; ++n) {
      const long double A = sqrtl((4.0L * n * n - 1) / ((long double)n * n - (long double)m * m));
      const long double B = sqrtl(((n - 1.0L) * (n - 1.0L) - (long double)m * m) * (2.0L * n + 1) /
                                  ((2.0L * n - 3) * ((long double)n * n - (long double)m * m)));
      const Poly En = add(mul1t(Om1), A, Em2, -B);
      const Poly On = add(Em1, A, Om2, -B);
      store(n, En, On);
      Em2 = Em1; Om2 = Om1; Em1 = En; Om1 = On;
    }
  }
  return out;
}

static double unord(unsigned long long u) {
  u = (u >> 63) ? (u & 0x7fffffffffffffffull) : ~u;
  double d;
  std::memcpy(&d, &u, sizeof d);
  return d;
}

// ---------------------------------------------------------------------------------------
// evaluation
// ---------------------------------------------------------------------------------------
// parts: bits 0, 1 free-space / reaction part, bits 2, 3 diagnostics (lpbfmm_eval_parts); gmask (host,
// may be null): per target group (l, a) at index 2 l + a - 1, the parts it computes (bits 0, 1)
// validation, trees, lists, tables, operators, upward pass and M2L of one evaluation (eval_back
// finishes it); with c.def.on the tensor-core M2L is only recorded
static void eval_front(Ctx &c, int64_t n, const double *q, const double *xyz, const int32_t *layer, int parts,
                       const int32_t *gmask, double *phi, double *field) {
  c.def.clear();
  c.arena.reset();
  c.launches = 0;
  c.nev = 0;
  c.prof_names.clear();
  c.prof_launch.clear();
  c.groups.clear();
  prof_mark(c, "start");
  LPB_CUDA(cudaMemsetAsync(phi, 0, sizeof(double) * n, c.stream));
  if (field) LPB_CUDA(cudaMemsetAsync(field, 0, sizeof(double) * 3 * n, c.stream));
  if (n == 0) return;
  const Medium &md = c.md;
  const int L = md.L;
  // validation and extents
  Stats hs;
  std::memset(&hs, 0, sizeof hs);
  hs.xlo = hs.ylo = ~0ull;
  for (int k = 0; k <= L; ++k) hs.zlo[k] = ~0ull;
  Stats *ds = c.arena.get<Stats>(1);
  LPB_CUDA(cudaMemcpyAsync(ds, &hs, sizeof hs, cudaMemcpyHostToDevice, c.stream));
  launch_validate(c, n, q, xyz, layer, ds);
  Stats *hp = (Stats *)c.h_pinned;
  LPB_CUDA(cudaMemcpyAsync(hp, ds, sizeof(Stats), cudaMemcpyDeviceToHost, c.stream));
  LPB_CUDA(cudaStreamSynchronize(c.stream));
  hs = *hp;
  if (hs.status) throw StatusError{hs.status};
  int64_t cnt[MAXLAYER];
  double zlo[MAXLAYER], zhi[MAXLAYER];
  for (int k = 0; k <= L; ++k) {
    cnt[k] = (int64_t)hs.cnt[k];
    zlo[k] = cnt[k] ? unord(hs.zlo[k]) : 0.0;
    zhi[k] = cnt[k] ? unord(hs.zhi[k]) : 0.0;
  }
  const double xlo = unord(hs.xlo), xhi = unord(hs.xhi), ylo = unord(hs.ylo), yhi = unord(hs.yhi);
  // per-layer stable ranks
  uint32_t *rank[MAXLAYER] = {};
  for (int k = 0; k <= L; ++k)
    if (cnt[k]) {
      rank[k] = c.arena.get<uint32_t>(n);
      layer_rank(c, n, layer, k, rank[k]);
    }
  // target groups (l, a) and their roots (exact extremes of monotone expressions)
  const double cx = 0.5 * (xlo + xhi), cy = 0.5 * (ylo + yhi);
  for (int l = 0; l <= L; ++l) {
    if (!cnt[l]) continue;
    for (int a = 1; a <= 2; ++a) {
      if ((a == 1 && l == L) || (a == 2 && l == 0)) continue;
      Group g;
      g.l = l;
      g.a = a;
      g.is_free = (a == ((l < L) ? 1 : 2));
      g.parts = parts & (gmask ? ((gmask[2 * l + a - 1] & 3) | 12) : 15);
      if (!g.is_free) g.parts &= ~1;
      if (!(g.parts & 3)) continue;
      g.ntypes = 2 * L;
      g.dI = (a == 1) ? md.d[l] : md.d[l - 1];
      double H = std::max(std::max(xhi - cx, cx - xlo), std::max(yhi - cy, cy - ylo));
      H = std::max(H, (a == 1) ? (zhi[l] - g.dI) : (g.dI - zlo[l]));
      for (int lp = 0; lp <= L; ++lp) {
        if (!cnt[lp]) continue;
        for (int b = 1; b <= 2; ++b) {
          if ((b == 1 && lp == L) || (b == 2 && lp == 0)) continue;
          H = std::max(H, std::fabs(image_z(md, l, a, lp, b, zlo[lp]) - g.dI));
          H = std::max(H, std::fabs(image_z(md, l, a, lp, b, zhi[lp]) - g.dI));
        }
      }
      g.root[0] = cx;
      g.root[1] = cy;
      g.root[2] = g.dI;
      g.root[3] = H * (1.0 + 1.0 / 1048576.0);
      c.groups.push_back(g);
    }
  }
  // per-group streams (the groups' trees are independent): fork from / join into c.stream; in a
  // batched evaluation the systems already run concurrently, and the groups stay on c.stream
  const int NGS = c.def.on ? 0 : std::min<int>(Ctx::GROUP_STREAMS, (int)c.groups.size());
  auto fork_groups = [&]() {
    LPB_CUDA(cudaEventRecord(c.ev_gfork, c.stream));
    for (int k = 0; k < NGS; ++k) LPB_CUDA(cudaStreamWaitEvent(c.gs[k], c.ev_gfork, 0));
  };
  auto join_groups = [&]() {
    for (int k = 0; k < NGS; ++k) {
      LPB_CUDA(cudaEventRecord(c.ev_gjoin[k], c.gs[k]));
      LPB_CUDA(cudaStreamWaitEvent(c.stream, c.ev_gjoin[k], 0));
    }
  };
  auto per_group = [&](auto &&f) {
    fork_groups();
    for (size_t k = 0; k < c.groups.size(); ++k) {
      OnStream on(c, NGS ? c.gs[k % NGS] : c.stream);
      f((int)k, c.groups[k]);
    }
    join_groups();
  };
  const int G = (int)c.groups.size();
  uint32_t *dc = nullptr;  // occupied boxes per level and group (automatic depth)
  if (c.opts.uniform_depth <= 0) {
    dc = c.arena.get<uint32_t>((size_t)G * (DMAX + 1));
    LPB_CUDA(cudaMemsetAsync(dc, 0, sizeof(uint32_t) * G * (DMAX + 1), c.stream));
  }
  per_group([&](int k, Group &g) {
    build_group_targets(c, g, n, q, xyz, layer, rank, cnt);
    if (dc) count_levels(c, g, dc + (size_t)k * (DMAX + 1));
  });
  // smallest distances of the group's targets and images to its interface (exact extremes of
  // monotone expressions of the z ranges)
  auto z_gaps = [&](const Group &g, double &zt, double &zs) {
    zt = (g.a == 1) ? (zlo[g.l] - g.dI) : (g.dI - zhi[g.l]);
    zs = 1e300;
    for (int lp = 0; lp <= L; ++lp) {
      if (!cnt[lp]) continue;
      for (int b = 1; b <= 2; ++b) {
        if ((b == 1 && lp == L) || (b == 2 && lp == 0)) continue;
        zs = std::min(zs, std::fabs(image_z(md, g.l, g.a, lp, b, zlo[lp]) - g.dI));
        zs = std::min(zs, std::fabs(image_z(md, g.l, g.a, lp, b, zhi[lp]) - g.dI));
      }
    }
  };
  // depth: Df of the free-space part by the occupancy rule (or given); the reaction part goes up to
  // react_levels levels deeper, to the first level whose boxes are small enough that no target box and
  // image box are near (k_t + k_s >= ws for the closest rows): its near field, the costly direct
  // Sommerfeld integrals, then vanishes (Sec. 3.5, Remark 1)
  if (c.opts.uniform_depth > 0) {
    for (auto &g : c.groups) g.D = g.Df = std::min(DMAX, std::max(2, c.opts.uniform_depth));
  } else {
    uint32_t *hc = (uint32_t *)c.h_pinned;
    LPB_CUDA(cudaMemcpyAsync(hc, dc, sizeof(uint32_t) * G * (DMAX + 1), cudaMemcpyDeviceToHost, c.stream));
    LPB_CUDA(cudaStreamSynchronize(c.stream));
    const int s = c.opts.max_per_leaf > 0 ? c.opts.max_per_leaf : 128;
    for (int k = 0; k < G; ++k) {
      Group &g = c.groups[k];
      g.Df = DMAX;
      for (int D = 2; D <= DMAX; ++D)
        if ((uint64_t)g.T.np <= (uint64_t)s * hc[(size_t)k * (DMAX + 1) + D]) { g.Df = D; break; }
      g.D = g.Df;
      if (g.parts & 2) {
        double zt, zs;
        z_gaps(g, zt, zs);
        while (g.D < std::min(DMAX, g.Df + c.opts.react_levels)) {
          const double h = g.h(g.D);
          if (std::floor(zt / h) + std::floor(zs / h) >= c.ws) break;
          ++g.D;
        }
      }
    }
  }
  // the free-space operators on the side stream, concurrently with the image trees and lists
  LPB_CUDA(cudaEventRecord(c.ev_fork, c.stream));
  LPB_CUDA(cudaStreamWaitEvent(c.side, c.ev_fork, 0));
  {
    OnStream on(c, c.side);
    for (auto &g : c.groups) build_operators(c, g, g.parts, 1);
    LPB_CUDA(cudaEventRecord(c.ev_free, c.side));
  }
  per_group([&](int, Group &g) {
    build_group_images(c, g, n, q, xyz, layer, rank, cnt);
    build_group_boxes(c, g);
  });
  // box counts to host
  {
    std::vector<const uint32_t *> srcs;
    for (auto &g : c.groups) {
      for (int l = 2; l <= g.D; ++l) {
        srcs.push_back(g.T.lev[l].d_n);
        srcs.push_back(g.I.lev[l].d_n);
      }
      srcs.push_back(g.I.d_nseg);
    }
    uint32_t *dd = c.arena.get<uint32_t>(srcs.size());
    LPB_CUDA(cudaMemsetAsync(dd, 0, sizeof(uint32_t) * srcs.size(), c.stream));
    for (size_t k = 0; k < srcs.size(); ++k)
      if (srcs[k]) LPB_CUDA(cudaMemcpyAsync(dd + k, srcs[k], sizeof(uint32_t), cudaMemcpyDeviceToDevice, c.stream));
    uint32_t *hh = (uint32_t *)c.h_pinned;
    LPB_CUDA(cudaMemcpyAsync(hh, dd, sizeof(uint32_t) * srcs.size(), cudaMemcpyDeviceToHost, c.stream));
    LPB_CUDA(cudaStreamSynchronize(c.stream));
    size_t k = 0;
    for (auto &g : c.groups) {
      for (int l = 2; l <= g.D; ++l) {
        g.T.lev[l].n = g.T.np ? hh[k] : 0;
        g.I.lev[l].n = g.I.np ? hh[k + 1] : 0;
        k += 2;
      }
      g.I.nseg = g.I.np ? hh[k] : 0;
      ++k;
    }
  }
  per_group([&](int, Group &g) { build_group_lists(c, g, g.parts); });
  prof_mark(c, "tree");
  // the FP32 free-space near field needs only the trees and near lists: on its own stream, beside
  // the operators, the upward pass and the M2L (the downward pass waits for it).  In a batched
  // evaluation it is recorded for the batch's grouped launch.
  c.near_async = !c.def.on && c.opts.precision != LPBFMM_FP64;
  if (c.near_async) {
    LPB_CUDA(cudaEventRecord(c.ev_gfork, c.stream));
    LPB_CUDA(cudaStreamWaitEvent(c.gs[0], c.ev_gfork, 0));
    run_near_free(c, c.groups, phi, field, c.gs[0]);
    LPB_CUDA(cudaEventRecord(c.ev_near, c.gs[0]));
  } else {
    run_near_free(c, c.groups, phi, field, c.stream);
  }
  {
    double lmin = 1e300, hmin = 1e300;
    for (int k = 0; k <= L; ++k) lmin = std::min(lmin, c.md.lam[k]);
    for (auto &g : c.groups)
      if (g.I.np) hmin = std::min(hmin, g.h(g.D));
    c.stab_lmin = hmin < 1e300 ? lmin * hmin : lmin;
    c.stab_bes = nullptr;
  }
  // reaction tables, operators and near-field nodes on the side stream, after the lists (the M2L
  // waits for them)
  LPB_CUDA(cudaEventRecord(c.ev_fork, c.stream));
  {
    OnStream on(c, c.side);
    LPB_CUDA(cudaStreamWaitEvent(c.side, c.ev_fork, 0));
    for (auto &g : c.groups) {
      build_operators(c, g, g.parts, 2);
      if ((g.parts & 2) && g.ureact) {
        double zt, zs;
        z_gaps(g, zt, zs);
        build_near_nodes(c, g, std::max(zt + zs, 1e-12), (c.ws + 1) * std::sqrt(2.0) * g.h(g.D));
      }
    }
    LPB_CUDA(cudaEventRecord(c.ev_join, c.side));
  }
  prof_mark(c, "tables+ops");
  c.far_async = c.near_async;
  if (c.far_async) {
    // the far field on the high-priority stream, beside the near field
    LPB_CUDA(cudaEventRecord(c.ev_gfork, c.stream));
    LPB_CUDA(cudaStreamWaitEvent(c.far, c.ev_gfork, 0));
    OnStream on(c, c.far);
    run_fmm_front(c, c.groups);
    LPB_CUDA(cudaEventRecord(c.ev_far, c.far));
  } else {
    run_fmm_front(c, c.groups);
  }
}
// the downward pass and near fields of the evaluation eval_front began
static void eval_back(Ctx &c, double *phi, double *field) {
  run_fmm_back(c, c.groups, phi, field);
  prof_mark(c, "end");
}
static void eval_impl(Ctx &c, int64_t n, const double *q, const double *xyz, const int32_t *layer, int parts,
                      const int32_t *gmask, double *phi, double *field) {
  eval_front(c, n, q, xyz, layer, parts, gmask, phi, field);
  eval_back(c, phi, field);
}

// streams on which lpbfmm_eval_batched runs systems concurrently, per device (created on first use,
// kept for the process)
constexpr int BATCH_STREAMS = 8;  // 4: 9 % slower on 256 systems; 16 and 32: no faster
static std::mutex g_bs_mu;
static cudaStream_t g_bs[LPB_MAX_DEVICES][BATCH_STREAMS] = {};
static cudaStream_t *batch_streams(int dev) {
  std::lock_guard<std::mutex> lk(g_bs_mu);
  if (!g_bs[dev][0])
    for (int t = 0; t < BATCH_STREAMS; ++t) LPB_CUDA(cudaStreamCreateWithFlags(&g_bs[dev][t], cudaStreamNonBlocking));
  return g_bs[dev];
}

}  // namespace lpb

using namespace lpb;

struct lpbfmm_ctx : public Ctx {};

static int map_error(const CudaError &e) {
  if (e.e == cudaErrorMemoryAllocation) return LPBFMM_ERR_OOM;
  fprintf(stderr, "lpbfmm: CUDA error %s at %s\n", cudaGetErrorString(e.e), e.where);
  return LPBFMM_ERR_CUDA;
}

extern "C" {

void lpbfmm_default_opts(lpbfmm_opts *o) {
  if (!o) return;
  o->precision = LPBFMM_FP64;
  o->max_per_leaf = 128;
  o->uniform_depth = 0;
  o->separation = 0;
  o->react_levels = LPBFMM_REACT_LEVELS_DEFAULT;
  o->stream = nullptr;
}

int lpbfmm_create(int n_iface, const double *z_iface, const double *eps, const double *lambda, int p, double tol,
                  const lpbfmm_opts *opts, lpbfmm_t *out) {
  if (!out || !z_iface || !eps || !lambda) return LPBFMM_ERR_ARG;
  *out = nullptr;
  if (n_iface < 1 || n_iface > LPBFMM_MAX_INTERFACES) return LPBFMM_ERR_MEDIUM;
  for (int k = 0; k + 1 < n_iface; ++k)
    if (!(z_iface[k] > z_iface[k + 1])) return LPBFMM_ERR_MEDIUM;
  for (int k = 0; k <= n_iface; ++k)
    if (!(eps[k] > 0.0) || !(lambda[k] > 0.0) || !std::isfinite(eps[k]) || !std::isfinite(lambda[k]))
      return LPBFMM_ERR_MEDIUM;
  for (int k = 0; k < n_iface; ++k)
    if (!std::isfinite(z_iface[k])) return LPBFMM_ERR_MEDIUM;
  if (p < LPBFMM_P_MIN || p > LPBFMM_P_MAX) return LPBFMM_ERR_P;
  if (!(tol > 0.0) || tol > 1e-3) return LPBFMM_ERR_ARG;
  lpbfmm_opts o;
  lpbfmm_default_opts(&o);
  if (opts) o = *opts;
  if ((o.precision != LPBFMM_FP64 && o.precision != LPBFMM_MIXED) || o.max_per_leaf < 0 || o.uniform_depth < 0 ||
      o.uniform_depth > DMAX || o.separation < 0 || o.separation > WS_MAX ||
      o.react_levels < 0 || o.react_levels > 8)
    return LPBFMM_ERR_ARG;
  lpbfmm_ctx *c = new (std::nothrow) lpbfmm_ctx();
  if (!c) return LPBFMM_ERR_OOM;
  try {
    c->md.L = n_iface;
    for (int k = 0; k < MAXLAYER; ++k) c->md.d[k] = c->md.eps[k] = c->md.lam[k] = 0.0;
    for (int k = 0; k < n_iface; ++k) c->md.d[k] = z_iface[k];
    for (int k = 0; k <= n_iface; ++k) { c->md.eps[k] = eps[k]; c->md.lam[k] = lambda[k]; }
    c->p = p;
    c->K = (p + 1) * (p + 2) / 2;
    c->ws = o.separation ? o.separation : LPBFMM_SEPARATION_DEFAULT;
    c->tol = tol;
    c->opts = o;
    c->stream = (cudaStream_t)o.stream;
    LPB_CUDA(cudaGetDevice(&c->device));
    if (c->device < 0 || c->device >= LPB_MAX_DEVICES) throw StatusError{LPBFMM_ERR_UNSUPPORTED};
    std::vector<double> G = gaunt_table(p);
    std::vector<double> tp = tpoly_table(p, c->tpk);
    LPB_CUDA(cudaMalloc(&c->gaunt, sizeof(double) * G.size()));
    LPB_CUDA(cudaMemcpy(c->gaunt, G.data(), sizeof(double) * G.size(), cudaMemcpyHostToDevice));
    LPB_CUDA(cudaMalloc(&c->tpoly, sizeof(double) * tp.size()));
    LPB_CUDA(cudaMemcpy(c->tpoly, tp.data(), sizeof(double) * tp.size(), cudaMemcpyHostToDevice));
    std::vector<double> sf = sfac_table();
    LPB_CUDA(cudaMalloc(&c->sfac, sizeof(double) * sf.size()));
    LPB_CUDA(cudaMemcpy(c->sfac, sf.data(), sizeof(double) * sf.size(), cudaMemcpyHostToDevice));
    std::vector<double> pd = phat_dir_table(p);
    LPB_CUDA(cudaMalloc(&c->phat_dir, sizeof(double) * pd.size()));
    LPB_CUDA(cudaMemcpy(c->phat_dir, pd.data(), sizeof(double) * pd.size(), cudaMemcpyHostToDevice));
    LPB_CUDA(cudaMalloc(&c->status, sizeof(int)));
    LPB_CUDA(cudaMemset(c->status, 0, sizeof(int)));
    LPB_CUDA(cudaMallocHost(&c->h_pinned, 1 << 16));
    for (int k = 0; k < 64; ++k) LPB_CUDA(cudaEventCreate(&c->ev[k]));
    int prio_least = 0, prio_greatest = 0;
    LPB_CUDA(cudaDeviceGetStreamPriorityRange(&prio_least, &prio_greatest));
    LPB_CUDA(cudaStreamCreateWithPriority(&c->side, cudaStreamNonBlocking, prio_greatest));
    LPB_CUDA(cudaStreamCreateWithPriority(&c->far, cudaStreamNonBlocking, prio_greatest));
    LPB_CUDA(cudaEventCreateWithFlags(&c->ev_far, cudaEventDisableTiming));
    LPB_CUDA(cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming));
    LPB_CUDA(cudaEventCreateWithFlags(&c->ev_free, cudaEventDisableTiming));
    LPB_CUDA(cudaEventCreateWithFlags(&c->ev_gfork, cudaEventDisableTiming));
    LPB_CUDA(cudaEventCreateWithFlags(&c->ev_near, cudaEventDisableTiming));
    LPB_CUDA(cudaEventCreate(&c->ev_p2p[0]));
    LPB_CUDA(cudaEventCreate(&c->ev_p2p[1]));
    for (int k = 0; k < Ctx::GROUP_STREAMS; ++k) {
      LPB_CUDA(cudaStreamCreateWithFlags(&c->gs[k], cudaStreamNonBlocking));
      LPB_CUDA(cudaEventCreateWithFlags(&c->ev_gjoin[k], cudaEventDisableTiming));
    }
    LPB_CUDA(cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming));
    init_fmm_tables(*c);
  } catch (const CudaError &e) {
    int code = map_error(e);
    lpbfmm_destroy(c);
    return code;
  } catch (const StatusError &e) {
    lpbfmm_destroy(c);
    return e.code;
  }
  *out = c;
  return LPBFMM_OK;
}

int lpbfmm_eval_parts(lpbfmm_t h, int64_t n, const double *q, const double *xyz, const int32_t *layer_id, int parts,
                      double *phi, double *field) {
  if (!h || n < 0 || (n > 0 && (!q || !xyz || !layer_id || !phi)) || parts < 1 || parts > 15) return LPBFMM_ERR_ARG;
  if (n >= (int64_t)1 << 31) return LPBFMM_ERR_UNSUPPORTED;
  try {
    eval_impl(*h, n, q, xyz, layer_id, parts, nullptr, phi, field);
  } catch (const CudaError &e) {
    return map_error(e);
  } catch (const StatusError &e) {
    return e.code;
  }
  return LPBFMM_OK;
}

int lpbfmm_eval(lpbfmm_t h, int64_t n, const double *q, const double *xyz, const int32_t *layer_id, double *phi,
                double *field) {
  return lpbfmm_eval_parts(h, n, q, xyz, layer_id, 3, phi, field);
}

int lpbfmm_eval_groups(lpbfmm_t h, int64_t n, const double *q, const double *xyz, const int32_t *layer_id,
                       const int32_t *mask, double *phi, double *field) {
  if (!h || !mask || n < 0 || (n > 0 && (!q || !xyz || !layer_id || !phi))) return LPBFMM_ERR_ARG;
  for (int k = 0; k < 2 * (h->md.L + 1); ++k)
    if (mask[k] < 0 || mask[k] > 3) return LPBFMM_ERR_ARG;
  if (n >= (int64_t)1 << 31) return LPBFMM_ERR_UNSUPPORTED;
  try {
    eval_impl(*h, n, q, xyz, layer_id, 3, mask, phi, field);
  } catch (const CudaError &e) {
    return map_error(e);
  } catch (const StatusError &e) {
    return e.code;
  }
  return LPBFMM_OK;
}

__global__ void k_adjoint_combine(int64_t n, const double *q, const double *g, const double *fq, const double *fg,
                                  double *g_xyz) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < 3; ++k) g_xyz[3 * i + k] = -(q[i] * fg[3 * i + k] + g[i] * fq[3 * i + k]);
}

int lpbfmm_adjoint(lpbfmm_t h, int64_t n, const double *q, const double *xyz, const int32_t *layer_id,
                   const double *g_phi, double *g_q, double *g_xyz) {
  if (!h || n < 0 || (n > 0 && (!q || !xyz || !layer_id || !g_phi || !g_q || !g_xyz))) return LPBFMM_ERR_ARG;
  if (n == 0) return LPBFMM_OK;
  // work space kept by the context: grown (after the stream has drained) only when n grows
  const size_t need = (size_t)7 * n;
  if (need > h->adj_cap) {
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LPBFMM_ERR_CUDA;
    if (h->adj) cudaFree(h->adj);
    h->adj = nullptr;
    h->adj_cap = 0;
    if (cudaMalloc(&h->adj, sizeof(double) * need) != cudaSuccess) { cudaGetLastError(); return LPBFMM_ERR_OOM; }
    h->adj_cap = need;
  }
  double *fg = h->adj, *pq = h->adj + 3 * n, *fq = h->adj + 4 * n;
  int rc = lpbfmm_eval(h, n, g_phi, xyz, layer_id, g_q, fg);
  if (rc == LPBFMM_OK) rc = lpbfmm_eval(h, n, q, xyz, layer_id, pq, fq);
  if (rc == LPBFMM_OK) {
    k_adjoint_combine<<<(unsigned)((n + 255) / 256), 256, 0, h->stream>>>(n, q, g_phi, fq, fg, g_xyz);
    if (cudaGetLastError() != cudaSuccess) rc = LPBFMM_ERR_CUDA;
  }
  return rc;
}

int lpbfmm_eval_batched(int nsys, const lpbfmm_t *ctxs, const int64_t *offsets, const double *q, const double *xyz,
                        const int32_t *layer_id, double *phi, double *field) {
  if (nsys < 0 || (nsys > 0 && (!ctxs || !offsets))) return LPBFMM_ERR_ARG;
  if (nsys == 0) return LPBFMM_OK;
  if (offsets[0] != 0) return LPBFMM_ERR_ARG;
  for (int s = 0; s < nsys; ++s)
    if (!ctxs[s] || offsets[s + 1] < offsets[s] || ctxs[s]->device != ctxs[0]->device) return LPBFMM_ERR_ARG;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != ctxs[0]->device) return LPBFMM_ERR_ARG;
  // units of work: the distinct contexts, each with its systems (a context serves one system at a
  // time), heaviest first
  std::vector<lpbfmm_t> uctx;
  std::vector<std::vector<int>> usys;
  std::vector<int64_t> ucost;
  {
    std::map<lpbfmm_t, int> idx;
    for (int s = 0; s < nsys; ++s) {
      auto it = idx.find(ctxs[s]);
      if (it == idx.end()) {
        it = idx.emplace(ctxs[s], (int)uctx.size()).first;
        uctx.push_back(ctxs[s]);
        usys.emplace_back();
        ucost.push_back(0);
      }
      usys[it->second].push_back(s);
      ucost[it->second] += offsets[s + 1] - offsets[s];
    }
  }
  std::vector<int> order(uctx.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return ucost[x] > ucost[y]; });
  const int dev = ctxs[0]->device;
  const int nthr = (int)std::min<size_t>(BATCH_STREAMS, uctx.size());
  cudaStream_t caller = ctxs[0]->stream;
  cudaStream_t *pool = nullptr;
  std::vector<cudaEvent_t> evs(nthr + 1, nullptr);
  try {
    pool = batch_streams(dev);
    for (auto &e : evs) LPB_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    // the inputs are written on the caller's stream; a context's earlier work must be complete
    // before its work space is reused on a pool stream
    LPB_CUDA(cudaEventRecord(evs[nthr], caller));
    for (auto ctx : uctx) LPB_CUDA(cudaStreamSynchronize(ctx->stream));
    for (int t = 0; t < nthr; ++t) LPB_CUDA(cudaStreamWaitEvent(pool[t], evs[nthr], 0));
  } catch (const CudaError &e) {
    for (auto &ev : evs)
      if (ev) cudaEventDestroy(ev);
    return map_error(e);
  }
  // a context that serves one system records its tensor-core M2L and FP32 near field for grouped
  // launches over all such systems; a context that serves several evaluates them in turn, whole
  std::atomic<int> err{0};
  auto fail = [&](int rc) {
    int z = 0;
    err.compare_exchange_strong(z, rc);
  };
  auto guarded = [&](auto &&f) {
    try {
      f();
      return (int)LPBFMM_OK;
    } catch (const CudaError &e) {
      return map_error(e);
    } catch (const StatusError &e) {
      return e.code;
    }
  };
  std::vector<char> deferred(uctx.size(), 0);
  auto run_threads = [&](auto &&body) {
    std::atomic<int> next{0};
    auto work = [&](int t) {
      if (cudaSetDevice(dev) != cudaSuccess) {
        fail(LPBFMM_ERR_CUDA);
        return;
      }
      for (;;) {
        const int k = next.fetch_add(1);
        if (k >= (int)order.size() || err.load()) break;
        body(order[k], pool[t]);
      }
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nthr; ++t) th.emplace_back(work, t);
    work(0);
    for (auto &x : th) x.join();
  };
  // every pool stream after the caller's stream (fork), the caller's stream after every pool
  // stream (join)
  auto fork = [&]() {
    if (cudaEventRecord(evs[nthr], caller) != cudaSuccess) return false;
    for (int t = 0; t < nthr; ++t)
      if (cudaStreamWaitEvent(pool[t], evs[nthr], 0) != cudaSuccess) return false;
    return true;
  };
  auto join = [&]() {
    for (int t = 0; t < nthr; ++t)
      if (cudaEventRecord(evs[t], pool[t]) != cudaSuccess || cudaStreamWaitEvent(caller, evs[t], 0) != cudaSuccess)
        return false;
    return true;
  };
  // 1: each context's front part (trees, tables, operators, upward pass, M2L preparation)
  run_threads([&](int u, cudaStream_t st) {
    lpbfmm_t ctx = uctx[u];
    const cudaStream_t own = ctx->stream;
    ctx->stream = st;
    if (usys[u].size() == 1) {
      const int s = usys[u][0];
      const int64_t o = offsets[s], n = offsets[s + 1] - offsets[s];
      ctx->def.on = true;
      const int rc = guarded([&] {
        eval_front(*ctx, n, q + o, xyz + 3 * o, layer_id + o, 3, nullptr, phi + o, field ? field + 3 * o : nullptr);
      });
      if (rc) {
        ctx->def.on = false;
        ctx->def.clear();
        fail(rc);
      } else {
        deferred[u] = 1;
      }
    } else {
      for (int s : usys[u]) {
        const int64_t o = offsets[s], n = offsets[s + 1] - offsets[s];
        const int rc = lpbfmm_eval(ctx, n, q + o, xyz + 3 * o, layer_id + o, phi + o, field ? field + 3 * o : nullptr);
        if (rc) {
          fail(rc);
          break;
        }
      }
    }
    ctx->stream = own;
  });
  std::vector<Ctx *> dcs;
  for (int u : order)
    if (deferred[u]) dcs.push_back(uctx[u]);
  // 2: the tensor-core M2L and its slot sums, then the FP32 free-space near field, of every
  // deferred context, grouped (the near field first into the outputs, as in lpbfmm_eval)
  if (!err.load() && !dcs.empty()) {
    const int rc = guarded([&] {
      if (!join()) throw CudaError{cudaErrorUnknown, "batched join"};
      launch_deferred(dcs, 0, caller);
      launch_deferred(dcs, 1, caller);
      if (!fork()) throw CudaError{cudaErrorUnknown, "batched fork"};
    });
    if (rc) fail(rc);
  }
  // 3: each deferred context's downward pass and reaction near field
  if (!err.load() && !dcs.empty())
    run_threads([&](int u, cudaStream_t st) {
      if (!deferred[u]) return;
      lpbfmm_t ctx = uctx[u];
      const int s = usys[u][0];
      const int64_t o = offsets[s];
      const cudaStream_t own = ctx->stream;
      ctx->stream = st;
      const int rc = guarded([&] { eval_back(*ctx, phi + o, field ? field + 3 * o : nullptr); });
      if (rc) fail(rc);
      ctx->stream = own;
    });
  for (Ctx *c : dcs) {
    c->def.on = false;
    c->def.clear();
  }
  // the caller's stream and every context's own stream continue after the pool's work
  int rc = err.load();
  if (!join()) rc = rc ? rc : LPBFMM_ERR_CUDA;
  if (cudaEventRecord(evs[nthr], caller) != cudaSuccess) rc = rc ? rc : LPBFMM_ERR_CUDA;
  for (auto ctx : uctx)
    if (ctx->stream != caller && cudaStreamWaitEvent(ctx->stream, evs[nthr], 0) != cudaSuccess) rc = rc ? rc : LPBFMM_ERR_CUDA;
  for (auto &ev : evs) cudaEventDestroy(ev);
  return rc;
}

int lpbfmm_status(lpbfmm_t h) {
  if (!h) return LPBFMM_ERR_ARG;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LPBFMM_ERR_CUDA;
  int v = 0;
  if (cudaMemcpy(&v, h->status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return LPBFMM_ERR_CUDA;
  cudaMemset(h->status, 0, sizeof(int));
  return v;
}

const char *lpbfmm_strerror(int code) {
  switch (code) {
    case LPBFMM_OK: return "ok";
    case LPBFMM_ERR_ARG: return "invalid argument";
    case LPBFMM_ERR_MEDIUM: return "invalid medium";
    case LPBFMM_ERR_P: return "truncation order out of range";
    case LPBFMM_ERR_ON_INTERFACE: return "charge on an interface";
    case LPBFMM_ERR_LAYER_MISMATCH: return "layer_id does not match z";
    case LPBFMM_ERR_NONFINITE: return "non-finite input";
    case LPBFMM_ERR_OOM: return "out of device memory";
    case LPBFMM_ERR_CUDA: return "CUDA error";
    case LPBFMM_ERR_TIMEOUT: return "device wait timed out";
    case LPBFMM_ERR_UNSUPPORTED: return "unsupported size";
  }
  return "unknown error";
}

void lpbfmm_destroy(lpbfmm_t h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  if (h->side) cudaStreamSynchronize(h->side);
  if (h->far) cudaStreamSynchronize(h->far);
  for (int k = 0; k < Ctx::GROUP_STREAMS; ++k)
    if (h->gs[k]) cudaStreamSynchronize(h->gs[k]);
  h->arena.release();
  if (h->adj) cudaFree(h->adj);
  if (h->gaunt) cudaFree(h->gaunt);
  if (h->tpoly) cudaFree(h->tpoly);
  if (h->sfac) cudaFree(h->sfac);
  if (h->phat_dir) cudaFree(h->phat_dir);
  if (h->rotcol) cudaFree(h->rotcol);
  if (h->status) cudaFree(h->status);
  if (h->h_pinned) cudaFreeHost(h->h_pinned);
  for (int k = 0; k < 64; ++k)
    if (h->ev[k]) cudaEventDestroy(h->ev[k]);
  if (h->ev_fork) cudaEventDestroy(h->ev_fork);
  if (h->ev_free) cudaEventDestroy(h->ev_free);
  if (h->ev_gfork) cudaEventDestroy(h->ev_gfork);
  if (h->ev_near) cudaEventDestroy(h->ev_near);
  for (int k = 0; k < 2; ++k)
    if (h->ev_p2p[k]) cudaEventDestroy(h->ev_p2p[k]);
  for (int k = 0; k < Ctx::GROUP_STREAMS; ++k) {
    if (h->ev_gjoin[k]) cudaEventDestroy(h->ev_gjoin[k]);
    if (h->gs[k]) cudaStreamDestroy(h->gs[k]);
  }
  if (h->ev_join) cudaEventDestroy(h->ev_join);
  if (h->side) cudaStreamDestroy(h->side);
  if (h->far) cudaStreamDestroy(h->far);
  if (h->ev_far) cudaEventDestroy(h->ev_far);
  delete h;
}

int lpbfmm_last_profile(lpbfmm_t h, int cap, const char **names, float *ms, int *launches) {
  if (!h || cap < 0) return -1;
  if (h->nev < 2) return 0;
  if (cudaEventSynchronize(h->ev[h->nev - 1]) != cudaSuccess) return -1;
  // aggregate consecutive event intervals by name of the interval's end mark
  std::vector<std::string> order;
  std::map<std::string, float> acc;
  std::map<std::string, int> lc;
  for (int k = 1; k < h->nev; ++k) {
    float t = 0;
    cudaEventElapsedTime(&t, h->ev[k - 1], h->ev[k]);
    const std::string &nm = h->prof_names[k];
    if (!acc.count(nm)) order.push_back(nm);
    acc[nm] += t;
    lc[nm] += h->prof_launch[k] - h->prof_launch[k - 1];
  }
  if (h->p2p_timed) {  // the free-space near field, timed on its own stream
    float t = 0;
    cudaEventElapsedTime(&t, h->ev_p2p[0], h->ev_p2p[1]);
    if (!acc.count("p2p")) order.push_back("p2p");
    acc["p2p"] += t;
    lc["p2p"] += 1;
  }
  int w = 0;
  static std::vector<std::string> keep;
  keep = order;
  for (size_t k = 0; k < keep.size() && w < cap; ++k, ++w) {
    if (names) names[w] = keep[k].c_str();
    if (ms) ms[w] = acc[keep[k]];
    if (launches) launches[w] = lc[keep[k]];
  }
  return w;
}

static Group *find_group(lpbfmm_t h, int l, int a) {
  for (auto &g : h->groups)
    if (g.l == l && g.a == a) return &g;
  return nullptr;
}

int lpbfmm_debug_tree(lpbfmm_t h, int l, int a, double *root, int64_t *n_targets, int64_t *n_images, int *depth,
                      uint64_t *keys_t, int64_t *src_t, uint64_t *keys_i, int64_t *src_i, int32_t *type_i) {
  if (!h) return LPBFMM_ERR_ARG;
  Group *g = find_group(h, l, a);
  if (!g) return LPBFMM_ERR_ARG;
  if (root) for (int k = 0; k < 4; ++k) root[k] = g->root[k];
  if (n_targets) *n_targets = g->T.np;
  if (n_images) *n_images = g->I.np;
  if (depth) *depth = g->D;
  if (!keys_t) return LPBFMM_OK;
  try {
    LPB_CUDA(cudaStreamSynchronize(h->stream));
    for (int which = 0; which < 2; ++which) {
      const PointSet &P = which ? g->I : g->T;
      std::vector<uint64_t> k(P.np);
      std::vector<uint32_t> s(P.np);
      if (P.np) {
        LPB_CUDA(cudaMemcpy(k.data(), P.key, sizeof(uint64_t) * P.np, cudaMemcpyDeviceToHost));
        LPB_CUDA(cudaMemcpy(s.data(), P.src, sizeof(uint32_t) * P.np, cudaMemcpyDeviceToHost));
      }
      uint64_t *ko = which ? keys_i : keys_t;
      int64_t *so = which ? src_i : src_t;
      for (int64_t i = 0; i < P.np; ++i) {
        if (ko) ko[i] = which ? (k[i] >> 4) : ((k[i] >> 4) >> (3 * (DMAX - g->D)));
        if (so) so[i] = s[i];
        if (which && type_i) {
          int lp, b;
          type_decode((int)(k[i] & 15ull), lp, b);
          type_i[i] = 2 * lp + b - 1;
        }
      }
    }
  } catch (const CudaError &e) {
    return map_error(e);
  }
  return LPBFMM_OK;
}

int lpbfmm_debug_lists(lpbfmm_t h, int l, int a, int lev, int kind, int src, int64_t *nbox, int64_t *nent,
                       int64_t *off, int64_t *idx) {
  if (!h) return LPBFMM_ERR_ARG;
  Group *g = find_group(h, l, a);
  if (!g) return LPBFMM_ERR_ARG;
  const int leaf = src ? g->D : g->Df;  // leaf level of the reaction / free-space part
  if (lev < 2 || lev > leaf || (kind == 1 && lev != leaf)) return LPBFMM_ERR_ARG;
  const int32_t *dl = nullptr;
  const int nslot = kind ? NNEAR : NOFF;
  if (kind == 0) dl = src ? g->vreact[lev] : g->vfree[lev];
  else dl = src ? g->ureact : g->ufree;
  if (!dl) return LPBFMM_ERR_ARG;
  const int64_t nb = g->T.lev[lev].n;
  std::vector<int32_t> v((size_t)nb * nslot);
  try {
    LPB_CUDA(cudaStreamSynchronize(h->stream));
    LPB_CUDA(cudaMemcpy(v.data(), dl, sizeof(int32_t) * v.size(), cudaMemcpyDeviceToHost));
  } catch (const CudaError &e) {
    return map_error(e);
  }
  int64_t tot = 0;
  for (int32_t x : v) tot += x >= 0;
  if (nbox) *nbox = nb;
  if (nent) *nent = tot;
  if (!off) return LPBFMM_OK;
  int64_t c = 0;
  for (int64_t t = 0; t < nb; ++t) {
    off[t] = c;
    for (int o = 0; o < nslot; ++o) {
      const int32_t s = v[(size_t)t * nslot + o];
      if (s >= 0) {
        if (idx) idx[c] = s;
        ++c;
      }
    }
  }
  off[nb] = c;
  return LPBFMM_OK;
}

int lpbfmm_debug_adaptive_lists(lpbfmm_t h, int l, int a, int s, int ws, int64_t *nrec, int64_t *rec,
                                int64_t cap) {
  if (!h || !nrec || s < 0 || ws < 1 || ws > WS_MAX || cap < 0) return LPBFMM_ERR_ARG;
  Group *g = find_group(h, l, a);
  if (!g || !g->is_free || !(g->parts & 1)) return LPBFMM_ERR_ARG;
  std::vector<int64_t> r;
  try {
    LPB_CUDA(cudaStreamSynchronize(h->stream));
    adaptive_lists(*h, *g, s, ws, r);
  } catch (const CudaError &e) {
    return map_error(e);
  } catch (const StatusError &e) {
    return e.code;
  }
  *nrec = (int64_t)(r.size() / 5);
  if (rec) std::memcpy(rec, r.data(), sizeof(int64_t) * 5 * (size_t)std::min<int64_t>(cap, *nrec));
  return LPBFMM_OK;
}

int lpbfmm_debug_array(lpbfmm_t h, int l, int a, const char *name, int lev, void *dst, int64_t cap,
                       int64_t *bytes) {
  if (!h || !name || !bytes) return LPBFMM_ERR_ARG;
  Group *g = find_group(h, l, a);
  if (!g || lev < 0 || lev > DMAX) return LPBFMM_ERR_ARG;
  const std::string nm(name);
  const size_t KK = (size_t)h->K * h->K, es = h->opts.precision == LPBFMM_FP64 ? 8 : 4;
  const void *src = nullptr;
  size_t nb = 0;
  const int64_t ntb = g->T.lev[lev].n, nib = g->I.lev[lev].n;
  const int KT = 2 * h->p + 3;
  if (nm == "Mimg") { src = g->Mimg[lev]; nb = nib * g->ntypes * h->K * 2 * es; }
  else if (nm == "Mfree") { src = g->Mfree[lev]; nb = ntb * h->K * 2 * es; }
  else if (nm == "Lt") { src = g->Lt[lev]; nb = ntb * h->K * 2 * es; }
  else if (nm == "op_react") { src = g->op_react[lev]; nb = (size_t)NREACT_CLS * g->ntypes * 2 * KK * es; }
  else if (nm == "op_free") { src = g->op_free[lev]; nb = (size_t)NFREE_CLS * 2 * KK * es; }
  else if (nm == "stab") { src = g->stab[lev]; nb = (size_t)NREACT_CLS * g->ntypes * (KT + 1) * (KT + 1) * 4 * 8; }
  else if (nm == "used") { src = g->used[lev]; nb = NREACT_CLS; }
  else if (nm == "vreact") { src = g->vreact[lev]; nb = ntb * NOFF * 4; }
  else if (nm == "ikeys") { src = g->I.lev[lev].key; nb = nib * 8; }
  else if (nm == "tkeys") { src = g->T.lev[lev].key; nb = ntb * 8; }
  else if (nm == "rows") { src = g->rows[lev]; nb = (size_t)NKT * ntb * 4; }
  else if (nm == "nrows") { src = g->nrows[lev]; nb = NKT * 4; }
  else return LPBFMM_ERR_ARG;
  *bytes = (int64_t)nb;
  if (!dst || !src) return src ? LPBFMM_OK : LPBFMM_ERR_ARG;
  if ((int64_t)nb > cap) return LPBFMM_ERR_ARG;
  if (cudaStreamSynchronize(h->stream) != cudaSuccess) return LPBFMM_ERR_CUDA;
  if (cudaMemcpy(dst, src, nb, cudaMemcpyDeviceToHost) != cudaSuccess) return LPBFMM_ERR_CUDA;
  return LPBFMM_OK;
}

__global__ void k_count_lists(const int32_t *v, int64_t n, unsigned long long *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const unsigned c = __popc(__ballot_sync(0xffffffffu, i < n && v[i] >= 0));
  if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, (unsigned long long)c);
}
// pairs of the near list: sum over target leaves of count(target) * count(source)
__global__ void k_count_near(const int32_t *u, int64_t nb, const uint32_t *tcnt, const uint32_t *scnt,
                             unsigned long long *out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long v = 0;
  if (i < nb * NNEAR) {
    const int32_t s = u[i];
    if (s >= 0) v = (unsigned long long)tcnt[i / NNEAR] * scnt[s];
  }
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(out, v);
}

int lpbfmm_last_counts(lpbfmm_t h, int64_t *out) {
  if (!h || !out) return LPBFMM_ERR_ARG;
  unsigned long long *d = nullptr;
  try {
    LPB_CUDA(cudaMalloc(&d, 8 * sizeof(unsigned long long)));
    LPB_CUDA(cudaMemsetAsync(d, 0, 8 * sizeof(unsigned long long), h->stream));
    for (auto &g : h->groups) {
      for (int l = 2; l <= g.D; ++l) {
        const int64_t nv = g.T.lev[l].n * NOFF;
        if (g.vfree[l]) k_count_lists<<<(unsigned)((nv + 255) / 256), 256, 0, h->stream>>>(g.vfree[l], nv, d + 0);
        if (g.vreact[l]) {
          for (int t = 0; t < g.ntypes; ++t)
            k_count_lists<<<(unsigned)((nv + 255) / 256), 256, 0, h->stream>>>(g.vreact[l], nv, d + 1);
        }
      }
      const int64_t nb = g.T.lev[g.D].n, nbf = g.T.lev[g.Df].n;
      if (g.ufree)
        k_count_near<<<(unsigned)((nbf * NNEAR + 255) / 256), 256, 0, h->stream>>>(g.ufree, nbf, g.T.lev[g.Df].pcount,
                                                                               g.T.lev[g.Df].pcount, d + 2);
      if (g.ureact)
        k_count_near<<<(unsigned)((nb * NNEAR + 255) / 256), 256, 0, h->stream>>>(g.ureact, nb, g.T.lev[g.D].count,
                                                                              g.I.lev[g.D].count, d + 3);
    }
    LPB_CUDA(cudaGetLastError());
    unsigned long long hv[8];
    LPB_CUDA(cudaMemcpyAsync(hv, d, sizeof hv, cudaMemcpyDeviceToHost, h->stream));
    LPB_CUDA(cudaStreamSynchronize(h->stream));
    cudaFree(d);
    int64_t nt = 0, ni = 0, nbox = 0;
    for (auto &g : h->groups) {
      nt += g.T.np;
      ni += g.I.np;
      for (int l = 2; l <= g.D; ++l) nbox += g.T.lev[l].n;
    }
    out[0] = (int64_t)hv[0];  // free-space M2L translations
    out[1] = (int64_t)hv[1];  // reaction M2L translations (pairs x source types)
    out[2] = (int64_t)hv[2];  // free-space P2P pairs (incl. the excluded self pairs)
    out[3] = (int64_t)hv[3];  // reaction near-field pairs
    out[4] = nt;              // targets over all groups
    out[5] = ni;              // images over all groups
    out[6] = nbox;            // target boxes over all groups and levels
    out[7] = h->launches;     // kernels launched by the last evaluation
  } catch (const CudaError &e) {
    if (d) cudaFree(d);
    return map_error(e);
  }
  return LPBFMM_OK;
}

int lpbfmm_debug_stable(lpbfmm_t h, int l, int a, int lp, int b, double hbox, double rho, double zt, double zs,
                        int Kmax, double *out) {
  if (!h || !out || Kmax < 0 || Kmax > KMAX_TAB || !(hbox > 0)) return LPBFMM_ERR_ARG;
  if (l < 0 || l > h->md.L || lp < 0 || lp > h->md.L || (a == 1 && l == h->md.L) || (a == 2 && l == 0) ||
      (b == 1 && lp == h->md.L) || (b == 2 && lp == 0) || a < 1 || a > 2 || b < 1 || b > 2)
    return LPBFMM_ERR_ARG;
  try {
    debug_stable(*h, l, a, lp, b, hbox, rho, zt, zs, Kmax, out);
  } catch (const CudaError &e) {
    return map_error(e);
  } catch (const StatusError &e) {
    return e.code;
  }
  return LPBFMM_OK;
}

int lpbfmm_stable_noalloc(lpbfmm_t h, int l, int a, int lp, int b, double hbox, double rho, double zt, double zs,
                          int Kmax, double *out) {
  if (!h || !out || Kmax < 0 || !(hbox > 0)) return LPBFMM_ERR_ARG;
  if (l < 0 || l > h->md.L || lp < 0 || lp > h->md.L || (a == 1 && l == h->md.L) || (a == 2 && l == 0) ||
      (b == 1 && lp == h->md.L) || (b == 2 && lp == 0) || a < 1 || a > 2 || b < 1 || b > 2)
    return LPBFMM_ERR_ARG;
  try {
    stable_noalloc(*h, l, a, lp, b, hbox, rho, zt, zs, Kmax, out);
  } catch (const CudaError &e) {
    return map_error(e);
  } catch (const StatusError &e) {
    return e.code;
  }
  return LPBFMM_OK;
}

int lpbfmm_host_table(int which, int p, double *out, int64_t cap, int64_t *count) {
  if (!count) return LPBFMM_ERR_ARG;
  if (p < LPBFMM_P_MIN || p > LPBFMM_P_MAX) return LPBFMM_ERR_P;
  std::vector<double> t;
  try {
    int tpk = 0;
    switch (which) {
      case LPBFMM_TABLE_GAUNT: t = gaunt_table(p); break;
      case LPBFMM_TABLE_TPOLY: t = tpoly_table(p, tpk); break;
      case LPBFMM_TABLE_PHAT_DIR: t = phat_dir_table(p); break;
      case LPBFMM_TABLE_SFAC: t = sfac_table(); break;
      default: return LPBFMM_ERR_ARG;
    }
  } catch (const std::bad_alloc &) {
    return LPBFMM_ERR_OOM;
  }
  *count = (int64_t)t.size();
  if (!out) return LPBFMM_OK;
  if (cap < *count) return LPBFMM_ERR_ARG;
  std::copy(t.begin(), t.end(), out);
  return LPBFMM_OK;
}

}  // extern "C"
