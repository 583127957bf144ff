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
constexpr int NOFF = 343;     // offsets (dx,dy,dz) in [-3,3]^3, index ((dx+3)*7+(dy+3))*7+(dz+3)
constexpr int NNEAR = 27;     // offsets in [-1,1]^3
constexpr int NHDIR = 49;     // horizontal directions (dx,dy) in [-3,3]^2
constexpr int NRHO = 10;      // distinct dx^2+dy^2 values {0,1,2,4,5,8,9,10,13,18}
constexpr int NFREE_CLS = NRHO * 7;       // free-space M2L classes (rho^2, dz)
constexpr int NKK = 6;                    // (k_t, k_s) with k_t + k_s <= 2
constexpr int NREACT_CLS = NRHO * NKK;    // reaction M2L classes (rho^2, k_t, k_s)

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
  int l = 0, a = 0, is_free = 0, D = 2, ntypes = 0;
  double root[4] = {0, 0, 0, 0};  // cx, cy, cz (= interface), half-size
  double dI = 0;
  PointSet T, I;
  // lists (device), index [level]
  int32_t *vfree[DMAX + 1] = {};
  int32_t *vreact[DMAX + 1] = {};
  int32_t *ufree = nullptr, *ureact = nullptr;
  int32_t *rows[DMAX + 1] = {};  // reaction target boxes with k_t in {0,1,2}: 3 * ntb slots
  uint32_t *nrows[DMAX + 1] = {};
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

struct Ctx {
  Medium md;
  int p = 10, K = 66;
  double tol = 1e-14;
  lpbfmm_opts opts;
  cudaStream_t stream = nullptr;
  int device = 0;
  // constant tables (device, FP64)
  double *gaunt = nullptr;   // [(p+1)^2 in][(p+1)^2 out][2p+1]
  double *tpoly = nullptr;   // [K][TPK] Legendre-product coefficients
  double *sfac = nullptr;    // [KMAX_TAB+1][KMAX_TAB+1]: sqrt((K+d)! (K-d)!) for d <= K
  double *phat_dir = nullptr;  // [72][(2p+1)(2p+2)/2]: Phat_q^k(cos theta) of the operator directions
  // per evaluation: grading of the shared Sommerfeld node set and its Bessel columns
  double stab_lmin = 0.0;
  double *stab_bes = nullptr;
  int tpk = 0;
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

// ops.cu
void build_operators(Ctx &c, Group &g, int parts);
void build_near_nodes(Ctx &c, Group &g, double zeta_min, double rho_max);
void stable_noalloc(Ctx &c, int l, int a, int lp, int b, double h, double rho, double zt, double zs, int Kmax,
                    double *out);
void debug_stable(Ctx &c, int l, int a, int lp, int b, double h, double rho, double zt, double zs, int Kmax,
                  double *out);

// fmm.cu
void run_fmm_all(Ctx &c, std::vector<Group> &groups, int parts, double *phi, double *field);

// api.cu
void prof_mark(Ctx &c, const char *name);

}  // namespace lpb
