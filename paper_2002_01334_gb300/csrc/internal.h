// Internal declarations of the lpbfmm library (host orchestration + kernels).
#pragma once
#include <atomic>
#include <cuda_runtime.h>

#include <cstdint>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/lpbfmm.h"
#include "devmath.cuh"

namespace lpb {

constexpr int DMAX = 10;      // Morton keys are built at this depth (30 bits)

// Interaction lists of a uniform tree with a separation of ws boxes (1 <= ws <= WS_MAX): the near
// list holds the source boxes within ws boxes in every coordinate, the far (multipole-to-local)
// list the children of the parent's near boxes that are not near themselves, at offsets
// (dx, dy, dz) in [-(2 ws + 1), 2 ws + 1]^3.  Slots are laid out for WS_MAX whatever ws is.
constexpr int WS_MAX = 2;
constexpr int OFF_R = 2 * WS_MAX + 1;       // far offsets lie in [-OFF_R, OFF_R]^3
constexpr int OFF_D = 2 * OFF_R + 1;
constexpr int NOFF = OFF_D * OFF_D * OFF_D;  // far slots, index ((dx+R) D + (dy+R)) D + (dz+R)
constexpr int NSLICE = OFF_D;               // M2L work is split by dx
constexpr int SLICE_OFFS = OFF_D * OFF_D;   // offsets of one dx-slice
constexpr int NEAR_D = 2 * WS_MAX + 1;
constexpr int NNEAR = NEAR_D * NEAR_D * NEAR_D;  // near slots, index ((dx+W) E + (dy+W)) E + (dz+W)
constexpr int NRHO = 20;                    // distinct dx^2 + dy^2 for |dx|, |dy| <= OFF_R
constexpr int NDZ = OFF_D;
constexpr int NFREE_CLS = NRHO * NDZ;       // free-space M2L classes (rho^2, dz)
constexpr int NDIR = NFREE_CLS + 2;         // operator directions: the classes, then child -> parent
constexpr int NKT = 2 * WS_MAX + 1;         // reaction rows k_t (box distance to the interface)
constexpr int NKK = NKT * (NKT + 1) / 2;    // (k_t, k_s) with k_t + k_s < NKT
constexpr int NREACT_CLS = NRHO * NKK;      // reaction M2L classes (rho^2, k_t, k_s)

LPB_HD int rho2_of(int ri) {
  constexpr int t[NRHO] = {0, 1, 2, 4, 5, 8, 9, 10, 13, 16, 17, 18, 20, 25, 26, 29, 32, 34, 41, 50};
  return t[ri];
}
LPB_HD int rho_index(int dx, int dy) {
  const int r2 = dx * dx + dy * dy;
  for (int k = 0; k < NRHO; ++k)
    if (rho2_of(k) == r2) return k;
  return -1;
}
// (k_t, k_s) ordered by k_t + k_s, then k_t
LPB_HD int kk_index(int kt, int ks) {
  const int s = kt + ks;
  if (kt < 0 || ks < 0 || s >= NKT) return -1;
  return s * (s + 1) / 2 + kt;
}
LPB_HD void kk_decode(int kk, int &kt, int &ks) {
  int s = 0;
  while ((s + 1) * (s + 2) / 2 <= kk) ++s;
  kt = kk - s * (s + 1) / 2;
  ks = s - kt;
}
LPB_HD int off_index(int dx, int dy, int dz) { return ((dx + OFF_R) * OFF_D + (dy + OFF_R)) * OFF_D + dz + OFF_R; }
LPB_HD void off_decode(int o, int &dx, int &dy, int &dz) {
  dx = o / (OFF_D * OFF_D) - OFF_R;
  dy = (o / OFF_D) % OFF_D - OFF_R;
  dz = o % OFF_D - OFF_R;
}
LPB_HD void near_decode(int o, int &dx, int &dy, int &dz) {
  dx = o / (NEAR_D * NEAR_D) - WS_MAX;
  dy = (o / NEAR_D) % NEAR_D - WS_MAX;
  dz = o % NEAR_D - WS_MAX;
}
LPB_HD int cheb3(int dx, int dy, int dz) {
  const int ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
  return ax > ay ? (ax > az ? ax : az) : (ay > az ? ay : az);
}
// does some offset (dx, dy, dz) of the free-space class (rho^2 index ri, dz) lie in a far list of
// separation ws?
LPB_HD bool free_class_is_far(int ri, int dz, int ws) {
  for (int dx = -OFF_R; dx <= OFF_R; ++dx)
    for (int dy = -OFF_R; dy <= OFF_R; ++dy)
      if (dx * dx + dy * dy == rho2_of(ri) && cheb3(dx, dy, dz) > ws) return true;
  return false;
}

struct CudaError {
  cudaError_t e;
  const char *where;
};
#define LPB_CUDA(x)                                         \
  do {                                                      \
    cudaError_t _e = (x);                                   \
    if (_e != cudaSuccess) throw ::lpb::CudaError{_e, #x}; \
  } while (0)
#define LPB_LAUNCH() LPB_CUDA(cudaGetLastError())

// Per-device one-time set-up (constant memory, kernel attributes and the offset tables are
// per device).  LPB_MAX_DEVICES bounds the device ordinals a process may use.
constexpr int LPB_MAX_DEVICES = 64;
inline int current_device() {
  int d = 0;
  LPB_CUDA(cudaGetDevice(&d));
  return d;
}
// true until mark_done() has been called for the current device
inline bool not_done_on_device(const std::atomic<uint64_t> &mask) {
  return !(mask.load() & (1ull << (current_device() & (LPB_MAX_DEVICES - 1))));
}
inline void mark_done_on_device(std::atomic<uint64_t> &mask) {
  mask.fetch_or(1ull << (current_device() & (LPB_MAX_DEVICES - 1)));
}
// kernel attribute for the current device: set before the first launch on it (a race between
// host threads can only repeat the call)
#define LPB_ATTR_ONCE(kernel, bytes)                                                            \
  do {                                                                                          \
    static std::atomic<uint64_t> _m{0};                                                         \
    if (not_done_on_device(_m)) {                                                               \
      LPB_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(bytes))); \
      mark_done_on_device(_m);                                                                  \
    }                                                                                           \
  } while (0)

struct StatusError {
  int code;
};

// Stream-ordered bump allocator over device chunks, reset at the start of each evaluation.
struct Arena {
  struct Chunk {
    char *p;
    size_t size, used;
  };
  std::vector<Chunk> chunks;
  size_t want = 0, used_total = 0;
  void *alloc(size_t bytes);
  template <typename T>
  T *get(size_t n) {
    return (T *)alloc(sizeof(T) * (n ? n : 1));
  }
  void reset();
  void release();
};

struct Level {
  int64_t n = 0;
  uint64_t *key = nullptr;    // Morton key at this level (sorted)
  uint32_t *start = nullptr;  // first child box (finer level) or first point (leaf level)
  uint32_t *count = nullptr;  // number of children / points
  uint32_t *parent = nullptr; // parent box index in the coarser level (levels > 2)
  uint32_t *d_n = nullptr;    // device copy of n (written by the scan)
  uint32_t *pstart = nullptr, *pcount = nullptr;  // points of each box (target trees, every level)
};

struct PointSet {
  int64_t np = 0;
  uint64_t *key = nullptr;  // targets: morton30 << 4; images: (morton at depth D << 4) | type; sorted
  uint32_t *src = nullptr;  // input index
  double *x = nullptr, *y = nullptr, *z = nullptr, *q = nullptr;  // sorted (z = image z for images)
  Level lev[DMAX + 1];
  // leaf (box, type) segments (images)
  int64_t nseg = 0;
  uint32_t *seg_start = nullptr, *seg_count = nullptr, *seg_box = nullptr, *seg_type = nullptr;
  uint32_t *d_nseg = nullptr;
};

struct Group {
  // D: depth of the group's trees, the leaf level of the reaction part (images, their near field,
  // L2P of every target); Df <= D: leaf level of the free-space part (its P2M, near lists, P2P)
  int l = 0, a = 0, is_free = 0, D = 2, Df = 2, ntypes = 0;
  int parts = 3;  // what this group computes: bit 0 free-space part, bit 1 reaction part (+ bits 2, 3 as parts)
  double root[4] = {0, 0, 0, 0};  // cx, cy, cz (= interface), half-size
  double dI = 0;
  PointSet T, I;
  // lists (device), index [level]
  int32_t *vfree[DMAX + 1] = {};
  int32_t *vreact[DMAX + 1] = {};
  int32_t *ufree = nullptr, *ureact = nullptr;
  int32_t *rows[DMAX + 1] = {};  // reaction target boxes with k_t in [0, 2 ws]: NKT * ntb slots
  uint32_t *nrows[DMAX + 1] = {};  // [NKT]
  uint8_t *used[DMAX + 1] = {};  // reaction classes in use, NREACT_CLS per level
  int32_t *ktrow[DMAX + 1] = {};
  // expansions
  void *Mfree[DMAX + 1] = {}, *Mimg[DMAX + 1] = {}, *Lt[DMAX + 1] = {};
  // operators
  void *op_free[DMAX + 1] = {};        // [NFREE_CLS][2][K][K]
  void *op_react[DMAX + 1] = {};       // [NREACT_CLS][ntypes][2][K][K]
  void *op_m2m_t[DMAX + 1] = {};       // children at level -> parent, free sources: [2][2][K][K]
  void *op_m2m_i[DMAX + 1] = {};       // per image type: [ntypes][2][2][K][K]
  void *op_l2l[DMAX + 1] = {};         // parent (level-1) -> child at level: [2][2][K][K]
  double *stab[DMAX + 1] = {};         // reaction S-tables [NREACT_CLS][ntypes][(KT+1)^2*4]
  // reaction near-field quadrature nodes per type: [ntypes][nq][4]
  double *nodes = nullptr;
  int nq = 0;
  double h(int lev) const { return 2.0 * root[3] / double(1 << lev); }
};

// Job records of the grouped launches (one launch runs many jobs; a block finds its job by a
// binary search on the first work item of each job).
// Tensor-core M2L (k_m2l_tc): one (group, level, row class) of target boxes against one source tree.
struct TJob {
  const float *raw;         // source rows [nsb][ntypes][ldr], unrotated real coordinates
  const float *wimg;        // [ncls][ntypes] operator images (k_tc_pack_w)
  const float *rotcol;      // [NOFF][ldr] (cos, sin) of m phi per real column pair (make_rotcol)
  const int32_t *vlist;     // [ntb][NOFF]
  const int32_t *cls_of;    // [NOFF]
  const uint32_t *tmask;    // [nsb] source types with a nonzero row (nullptr: every type)
  const int32_t *tlist;     // target boxes (nullptr: octant or plain tiles over 0..ntb-1)
  const uint32_t *d_ntl;    // number of entries of tlist (device)
  float2 *L;                // partial sums [ntb][M2L_NSLOT][K]
  int64_t ntb, item0;
  int slot0, ntypes;
  const uint32_t *pstart, *pcount;  // octant tiles (nullptr: plain tiles of 128)
  const uint64_t *ckey;
  int64_t npar;
};
// Sum of a level's M2L partial slots into its local expansions (k_m2l_reduce).
struct RJob {
  const void *part;
  void *L;
  int64_t n;     // boxes x K
  int64_t e0;    // first element of this job in the flattened launch
};
// FP32 free-space near field of one target group's leaves (k_p2p_free_f32).
struct P2PJob {
  const uint32_t *d_nb;     // number of leaves (device)
  const uint64_t *bkey;     // leaf keys
  const uint32_t *bstart, *bcount;  // leaf point ranges
  const int32_t *ulist;     // [nb][NNEAR] near leaves or -1
  const float4 *h4, *l4;    // points as FP32 hi / lo offsets from their leaf centre, charge in h4.w
  const uint32_t *src;      // input index of each point
  double *phi, *field;      // outputs (input order)
  double scale;             // 1 / (4 pi eps)
  float hh, hl, lam;        // leaf side as FP32 hi + lo; screening
  int64_t block0;           // first block of this job in the launch
};

// launches of one evaluation held back for one grouped launch over several contexts
// (lpbfmm_eval_batched): the tensor-core M2L, its slot sums, the FP32 free-space near field
struct Deferred {
  bool on = false;
  int nc = 0;                       // column chunks of the tensor-core M2L (0: none recorded)
  std::vector<TJob> tc;             // item0 relative to this context
  std::vector<RJob> red;            // e0 relative to this context
  std::vector<P2PJob> p2p;          // block0 relative to this context
  int64_t tc_items = 0, red_elems = 0, p2p_blocks = 0;
  void clear() {
    nc = 0;
    tc.clear();
    red.clear();
    p2p.clear();
    tc_items = red_elems = p2p_blocks = 0;
  }
};

struct Ctx {
  Medium md;
  int p = 10, K = 66;
  int ws = 2;  // separation of the interaction lists (boxes)
  double tol = 1e-14;
  lpbfmm_opts opts;
  cudaStream_t stream = nullptr;
  int device = 0;
  // constant tables (device, FP64)
  double *gaunt = nullptr;   // [(p+1)^2 in][(p+1)^2 out][2p+1]
  double *tpoly = nullptr;   // [K][TPK] Legendre-product coefficients
  double *sfac = nullptr;    // [KMAX_TAB+1][KMAX_TAB+1]: sqrt((K+d)! (K-d)!) for d <= K
  double *phat_dir = nullptr;  // [NDIR][(2p+1)(2p+2)/2]: Phat_q^k(cos theta) of the operator directions
  float *rotcol = nullptr;     // tensor-core M2L: [NOFF][32 NC] (cos, sin) of m phi per real column pair
  // per evaluation: grading of the shared Sommerfeld node set and its Bessel columns
  double stab_lmin = 0.0;
  double *stab_bes = nullptr;
  int tpk = 0;
  double *adj = nullptr;     // adjoint work space (7 n doubles), grown on demand, kept
  size_t adj_cap = 0;
  int *status = nullptr;     // device status word
  int *h_status = nullptr;   // pinned
  void *h_pinned = nullptr;  // pinned staging
  Arena arena;
  std::vector<Group> groups;
  // profile of the last evaluation
  std::vector<std::string> prof_names;
  std::vector<float> prof_ms;
  std::vector<int> prof_launch;
  cudaEvent_t ev[64];
  int nev = 0;
  int launches = 0;
  Deferred def;
  // operators are built on a second stream: the free-space ones concurrently with the image
  // trees and lists (the upward pass waits for them, ev_free), the reaction ones concurrently
  // with the upward pass (the M2L waits for them, ev_join)
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_free = nullptr, ev_join = nullptr;
  // the target groups' trees and lists are independent: built on one stream per group
  // (group k on gs[k % GROUP_STREAMS]), forked from and joined into the evaluation stream
  static constexpr int GROUP_STREAMS = 4;
  cudaStream_t gs[GROUP_STREAMS] = {};
  cudaEvent_t ev_gfork = nullptr, ev_gjoin[GROUP_STREAMS] = {};
  // the FP32 free-space near field runs on gs[0] beside the upward pass and the M2L; the downward
  // pass (which also adds into the outputs) waits for ev_near.  ev_p2p[2] time its launch.
  cudaEvent_t ev_near = nullptr, ev_p2p[2] = {};
  bool near_async = false, p2p_timed = false;
  // beside it, the upward pass and the M2L run on a high-priority stream (far), so that their
  // blocks are scheduled ahead of the near field's; the downward pass waits for ev_far
  cudaStream_t far = nullptr;
  cudaEvent_t ev_far = nullptr;
  bool far_async = false;
};

// work of one scope on another stream of the context (restored on exit, also by an exception)
struct OnStream {
  Ctx &c;
  cudaStream_t saved;
  OnStream(Ctx &c_, cudaStream_t s) : c(c_), saved(c_.stream) { c.stream = s; }
  ~OnStream() { c.stream = saved; }
};

// tree.cu
struct Stats {
  int status;
  int pad;
  unsigned long long cnt[MAXLAYER];
  unsigned long long xlo, xhi, ylo, yhi;
  unsigned long long zlo[MAXLAYER], zhi[MAXLAYER];
};
void scan_u32(Ctx &c, const uint32_t *in, uint32_t *out, int64_t n, uint32_t *d_total);
void radix_sort(Ctx &c, uint64_t *&keys, uint32_t *&vals, int64_t n, int bits, int lo);
void launch_validate(Ctx &c, int64_t n, const double *q, const double *xyz, const int32_t *layer, Stats *st);
void build_group_targets(Ctx &c, Group &g, int64_t n, const double *q, const double *xyz, const int32_t *layer,
                         uint32_t *const *rank, const int64_t *cnt);
void build_group_images(Ctx &c, Group &g, int64_t n, const double *q, const double *xyz, const int32_t *layer,
                        uint32_t *const *rank, const int64_t *cnt);
void count_levels(Ctx &c, Group &g, uint32_t *d_counts);
void build_group_boxes(Ctx &c, Group &g);
void build_group_lists(Ctx &c, Group &g, int parts);
void layer_rank(Ctx &c, int64_t n, const int32_t *layer, int lay, uint32_t *rank);
// adaptive dual-tree lists of group g's free-space target tree with itself (diagnostic): records
// of 5 int64 (kind 0 V / 1 U / 2 W / 3 X, target level, target key, source level, source key)
void adaptive_lists(Ctx &c, Group &g, int s, int ws, std::vector<int64_t> &rec);

// ops.cu
// which: 1 the free-space operators (M2M, L2L, free M2L; need only the depths and roots),
// 2 the reaction tables and operators (need the interaction lists)
void build_operators(Ctx &c, Group &g, int parts, int which);
void build_near_nodes(Ctx &c, Group &g, double zeta_min, double rho_max);
void stable_noalloc(Ctx &c, int l, int a, int lp, int b, double h, double rho, double zt, double zs, int Kmax,
                    double *out);
void debug_stable(Ctx &c, int l, int a, int lp, int b, double h, double rho, double zt, double zs, int Kmax,
                  double *out);

// fmm.cu
// upward pass and M2L of every group (with c.def.on the tensor-core M2L and its slot sums are
// recorded in c.def instead of launched)
void run_fmm_front(Ctx &c, std::vector<Group> &groups);
// the FP32 free-space near field of every group (mixed precision): point splitting and one P2P
// launch on stream st, or, with c.def.on, the launch recorded in c.def for a grouped one
void run_near_free(Ctx &c, std::vector<Group> &groups, double *phi, double *field, cudaStream_t st);
// downward pass and the remaining near fields
void run_fmm_back(Ctx &c, std::vector<Group> &groups, double *phi, double *field);
// the recorded jobs of several contexts (all on the current device) as grouped launches on st:
// stage 0 the tensor-core M2L and the slot sums, stage 1 the free-space near field.  Timeouts of
// a grouped tensor-core launch are reported on the first context's status word.
void launch_deferred(const std::vector<Ctx *> &cs, int stage, cudaStream_t st);

// api.cu
void prof_mark(Ctx &c, const char *name);

}  // namespace lpb
