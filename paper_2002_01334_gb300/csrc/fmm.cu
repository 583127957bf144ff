// FMM passes of one target group (Algorithm 1 for the reaction components of group (l, a),
// the free-space Yukawa FMM of layer l when the group carries it, Algorithm 2 around them):
// P2M, M2M, M2L (free + reaction), L2L, L2P with field, near-field P2P.
// Expansions use the half representation (m >= 0) and the scaling described in ops.cu:
//   M~_nm = sum_j q_j 4 pi itilde_n(lambda r_j) conj(R_n^m(r_j / h)),
//   phi(r) = sum_n [L~_n0 itilde_n R_n^0 + 2 Re sum_{m>0} L~_nm itilde_n R_n^m](r / h).
#include "internal.h"
#include "tc.cuh"

#include <algorithm>
#include <mutex>

namespace lpb {

// recurrence and gradient constants (index [n][m], n <= PMAX + 1)
struct Consts {
  double A[PMAX + 2][PMAX + 2], B[PMAX + 2][PMAX + 2];
  double sect[PMAX + 2], sub[PMAX + 2];
  double gz[PMAX + 2][PMAX + 2], ga[PMAX + 2][PMAX + 2], gb[PMAX + 2][PMAX + 2];
  int mof[KHALF_MAX];
};
__constant__ Consts cK;
// FP32 copies of the recurrence constants: the FP32 kernels read these directly (a conversion
// from FP64 runs on the FP64 pipe, ~2 lanes per clock per SM on this GPU)
struct ConstsF {
  float A[PMAX + 2][PMAX + 2], B[PMAX + 2][PMAX + 2];
  float sect[PMAX + 2], sub[PMAX + 2];
  float gz[PMAX + 2][PMAX + 2], ga[PMAX + 2][PMAX + 2], gb[PMAX + 2][PMAX + 2];
};
__constant__ ConstsF cKf;
template <typename T> struct CK;
template <> struct CK<float> {
  static __device__ __forceinline__ float A(int n, int m) { return cKf.A[n][m]; }
  static __device__ __forceinline__ float B(int n, int m) { return cKf.B[n][m]; }
  static __device__ __forceinline__ float sect(int m) { return cKf.sect[m]; }
  static __device__ __forceinline__ float sub(int m) { return cKf.sub[m]; }
  static __device__ __forceinline__ float gz(int n, int m) { return cKf.gz[n][m]; }
  static __device__ __forceinline__ float ga(int n, int m) { return cKf.ga[n][m]; }
  static __device__ __forceinline__ float gb(int n, int m) { return cKf.gb[n][m]; }
};
template <> struct CK<double> {
  static __device__ __forceinline__ double A(int n, int m) { return cK.A[n][m]; }
  static __device__ __forceinline__ double B(int n, int m) { return cK.B[n][m]; }
  static __device__ __forceinline__ double sect(int m) { return cK.sect[m]; }
  static __device__ __forceinline__ double sub(int m) { return cK.sub[m]; }
  static __device__ __forceinline__ double gz(int n, int m) { return cK.gz[n][m]; }
  static __device__ __forceinline__ double ga(int n, int m) { return cK.ga[n][m]; }
  static __device__ __forceinline__ double gb(int n, int m) { return cK.gb[n][m]; }
};

void upload_consts(cudaStream_t s) {
  static Consts h;
  for (int n = 0; n <= PMAX + 1; ++n)
    for (int m = 0; m <= PMAX + 1; ++m) {
      h.A[n][m] = h.B[n][m] = h.gz[n][m] = h.ga[n][m] = h.gb[n][m] = 0.0;
      if (m <= n && n >= m + 2) {
        h.A[n][m] = sqrt((4.0 * n * n - 1.0) / (double(n) * n - double(m) * m));
        h.B[n][m] = sqrt(((n - 1.0) * (n - 1.0) - double(m) * m) * (2.0 * n + 1.0) /
                         ((2.0 * n - 3.0) * (double(n) * n - double(m) * m)));
      }
      if (m <= n) {
        const double c1 = sqrt((2.0 * (n + 1) + 1.0) / (2.0 * (n + 1) - 1.0));
        h.gz[n][m] = c1 * sqrt(double(n + 1 + m) * (n + 1 - m));
        h.ga[n][m] = c1 * sqrt(double(n + 2 - m) * (n + 1 - m));
        h.gb[n][m] = c1 * sqrt(double(n + 2 + m) * (n + 1 + m));
      }
    }
  for (int m = 0; m <= PMAX + 1; ++m) {
    h.sect[m] = m ? -sqrt((2.0 * m + 1.0) / (2.0 * m)) : 1.0;
    h.sub[m] = sqrt(2.0 * m + 3.0);
  }
  for (int n = 0; n <= PMAX; ++n)
    for (int m = 0; m <= n; ++m) h.mof[hidx(n, m)] = m;
  LPB_CUDA(cudaMemcpyToSymbolAsync(cK, &h, sizeof(Consts), 0, cudaMemcpyHostToDevice, s));
  static ConstsF hf;
  for (int n = 0; n <= PMAX + 1; ++n) {
    for (int m = 0; m <= PMAX + 1; ++m) {
      hf.A[n][m] = (float)h.A[n][m];
      hf.B[n][m] = (float)h.B[n][m];
      hf.gz[n][m] = (float)h.gz[n][m];
      hf.ga[n][m] = (float)h.ga[n][m];
      hf.gb[n][m] = (float)h.gb[n][m];
    }
    hf.sect[n] = (float)h.sect[n];
    hf.sub[n] = (float)h.sub[n];
  }
  LPB_CUDA(cudaMemcpyToSymbolAsync(cKf, &hf, sizeof(ConstsF), 0, cudaMemcpyHostToDevice, s));
  LPB_CUDA(cudaStreamSynchronize(s));
}

template <typename T> struct C2;
template <> struct C2<float> { typedef float2 t; };
template <> struct C2<double> { typedef double2 t; };

struct Geo {
  double o[3];  // lower corner of the root cube
  double h;     // box size at the level
};

__device__ __forceinline__ uint32_t compact3_(uint64_t x) {
  x &= 0x9249249ull;
  x = (x ^ (x >> 2)) & 0x30c30c3ull;
  x = (x ^ (x >> 4)) & 0x300f00full;
  x = (x ^ (x >> 8)) & 0x30000ffull;
  x = (x ^ (x >> 16)) & 0x3ffull;
  return (uint32_t)x;
}
__device__ __forceinline__ void box_center(uint64_t key, const Geo &g, double &cx, double &cy, double &cz) {
  cx = g.o[0] + (compact3_(key >> 2) + 0.5) * g.h;
  cy = g.o[1] + (compact3_(key >> 1) + 0.5) * g.h;
  cz = g.o[2] + (compact3_(key) + 0.5) * g.h;
}

template <typename T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct LamTab {
  double v[2 * MAXLAYER];
};

// ---------------------------------------------------------------------------------------
// P2M: one warp per leaf (box, type) segment
// ---------------------------------------------------------------------------------------
template <typename T, int PT>
__global__ void k_p2m(const uint32_t *d_nseg, const uint32_t *seg_start, const uint32_t *seg_count,
                      const uint32_t *seg_box, const uint32_t *seg_type, int ntypes, const uint64_t *box_key,
                      const double *x, const double *y, const double *z, const double *q, Geo geo, LamTab lt,
                      int p, int K, typename C2<T>::t *M) {
  typedef typename C2<T>::t T2;
  __shared__ T2 acc[4][KHALF_MAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t seg = (int64_t)blockIdx.x * 4 + warp;
  if (seg >= *d_nseg) return;
  for (int e = lane; e < K; e += 32) acc[warp][e] = T2{0, 0};
  const uint32_t st = seg_start[seg], cnt = seg_count[seg];
  const uint32_t box = seg_box ? seg_box[seg] : (uint32_t)seg;
  const uint32_t type = seg_type ? seg_type[seg] : 0u;
  double cx, cy, cz;
  box_center(box_key[box], geo, cx, cy, cz);
  const double ih = 1.0 / geo.h;
  const T lh = (T)(lt.v[type] * geo.h);
  __syncwarp();
  for (uint32_t b0 = 0; b0 < cnt; b0 += 32) {
    const uint32_t j = b0 + lane;
    const bool valid = j < cnt;
    const uint32_t k = st + (valid ? j : 0);
    const T rx = (T)((x[k] - cx) * ih), ry = (T)((y[k] - cy) * ih), rz = (T)((z[k] - cz) * ih);
    const T qq = valid ? (T)(q[k] * 4.0 * PI) : T(0);
    const T r2 = rx * rx + ry * ry + rz * rz;
    T it[PT + 2];
    itilde_all<T, PT + 1>(lh * lh * r2, it);
    T2 Rmm = T2{(T)(0.5 / sqrt(PI)), T(0)};
#pragma unroll
    for (int m = 0; m <= PT; ++m) {
      if (m > p) break;
      if (m > 0) {
        const T s = CK<T>::sect(m);
        const T2 t = T2{Rmm.x * rx - Rmm.y * ry, Rmm.x * ry + Rmm.y * rx};
        Rmm = T2{s * t.x, s * t.y};
      }
      T2 p1 = T2{0, 0}, p2 = T2{0, 0};
#pragma unroll
      for (int n = m; n <= PT; ++n) {
        if (n > p) break;
        T2 R;
        if (n == m) R = Rmm;
        else if (n == m + 1) { const T s = CK<T>::sub(m) * rz; R = T2{s * p1.x, s * p1.y}; }
        else {
          const T a = CK<T>::A(n, m) * rz, b = CK<T>::B(n, m) * r2;
          R = T2{a * p1.x - b * p2.x, a * p1.y - b * p2.y};
        }
        p2 = p1;
        p1 = R;
        const T c = qq * it[n];
        const T vr = wsum(c * R.x), vi = wsum(-c * R.y);
        if (lane == 0) {
          T2 &A = acc[warp][hidx(n, m)];
          A.x += vr;
          A.y += vi;
        }
      }
    }
  }
  __syncwarp();
  T2 *out = M + ((size_t)box * ntypes + type) * K;
  for (int e = lane; e < K; e += 32) out[e] = acc[warp][e];
}

// ---------------------------------------------------------------------------------------
// M2M (children -> parent) and L2L (parent -> child): azimuth-factored dense operators
// ---------------------------------------------------------------------------------------
template <typename T>
__device__ __forceinline__ void rot_of_octant(uint64_t ckey, int m, const T *rot4, T &c, T &s) {
  const int oct = (int)(ckey & 7ull);
  const int dir = ((oct >> 2) & 1) * 2 + ((oct >> 1) & 1);
  c = rot4[(dir * (PMAX + 1) + m) * 2];
  s = rot4[(dir * (PMAX + 1) + m) * 2 + 1];
}

// One CTA per (parent, source type), one thread per output row.  All children's rotated
// multipoles are staged at once; a thread reads each operator row once per z-half (child octant
// bit cz) and applies it to the (at most four) children with that cz.
constexpr int M2M_THREADS = 96;  // >= K for p <= 12 handled in one pass; larger K loops
template <typename T>
__global__ void __launch_bounds__(M2M_THREADS) k_m2m(const uint32_t *d_np, const uint32_t *pstart,
                                                     const uint32_t *pcount, const uint64_t *ckey, int ntypes,
                                                     const typename C2<T>::t *Mc, typename C2<T>::t *Mp,
                                                     const T *ops, const T *rot4, int K) {
  typedef typename C2<T>::t T2;
  __shared__ T xr[8][KHALF_MAX], xi[8][KHALF_MAX];
  __shared__ int slot[2][4], nslot[2];
  __shared__ uint64_t ck_s[8];
  const uint32_t box = blockIdx.x, type = blockIdx.y;
  if (box >= *d_np) return;
  const size_t KK = (size_t)K * K;
  const uint32_t c0 = pstart[box], nc = min(pcount[box], 8u);
  if (threadIdx.x < nc) ck_s[threadIdx.x] = ckey[c0 + threadIdx.x];
  __syncthreads();
  if (threadIdx.x == 0) {
    nslot[0] = nslot[1] = 0;
    for (uint32_t c = 0; c < nc; ++c) {
      const int cz = (int)(ck_s[c] & 1ull);
      slot[cz][nslot[cz]++] = (int)c;
    }
  }
  for (uint32_t e = threadIdx.x; e < nc * (uint32_t)K; e += blockDim.x) {
    const int c = (int)(e / K), k = (int)(e % K);
    T cs, sn;
    rot_of_octant(ck_s[c], cK.mof[k], rot4, cs, sn);
    const T2 v = Mc[((size_t)(c0 + c) * ntypes + type) * K + k];
    xr[c][k] = cs * v.x - sn * v.y;
    xi[c][k] = sn * v.x + cs * v.y;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    const int m = cK.mof[i];
    T ar = 0, ai = 0;
    for (int cz = 0; cz < 2; ++cz) {
      const int ns = nslot[cz];
      if (ns == 0) continue;
      const T *P = ops + ((size_t)type * 2 + cz) * 2 * KK + (size_t)i * K, *Q = P + KK;
      T yr[4] = {0, 0, 0, 0}, yi[4] = {0, 0, 0, 0};
      int sl[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) sl[j] = j < ns ? slot[cz][j] : slot[cz][0];
#pragma unroll 2
      for (int k = 0; k < K; ++k) {
        const T pv = P[k], qv = Q[k];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          yr[j] += pv * xr[sl[j]][k];
          yi[j] += qv * xi[sl[j]][k];
        }
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        if (j >= ns) break;
        T cs, sn;
        rot_of_octant(ck_s[sl[j]], m, rot4, cs, sn);
        ar += cs * yr[j] + sn * yi[j];
        ai += cs * yi[j] - sn * yr[j];
      }
    }
    Mp[((size_t)box * ntypes + type) * K + i] = T2{ar, ai};
  }
}

template <typename T>
__global__ void k_l2l(const uint32_t *d_nc, const uint32_t *cparent, const uint64_t *ckey,
                      const typename C2<T>::t *Lp, typename C2<T>::t *Lc, const T *ops, const T *rot4, int K) {
  typedef typename C2<T>::t T2;
  __shared__ T xr[KHALF_MAX], xi[KHALF_MAX];
  const uint32_t c = blockIdx.x;
  if (c >= *d_nc) return;
  const uint64_t ck = ckey[c];
  const int cz = (int)(ck & 1ull);
  const size_t KK = (size_t)K * K;
  const T *P = ops + (size_t)cz * 2 * KK, *Q = P + KK;
  const uint32_t par = cparent[c];
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    T cs, sn;
    rot_of_octant(ck, cK.mof[e], rot4, cs, sn);
    const T2 v = Lp[(size_t)par * K + e];
    xr[e] = cs * v.x - sn * v.y;
    xi[e] = sn * v.x + cs * v.y;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < K; i += blockDim.x) {
    T yr = 0, yi = 0;
    for (int k = 0; k < K; ++k) {
      yr += P[(size_t)i * K + k] * xr[k];
      yi += Q[(size_t)i * K + k] * xi[k];
    }
    T cs, sn;
    rot_of_octant(ck, cK.mof[i], rot4, cs, sn);
    T2 &dst = Lc[(size_t)c * K + i];
    dst.x += cs * yr + sn * yi;
    dst.y += cs * yi - sn * yr;
  }
}

// ---------------------------------------------------------------------------------------
// M2L: one launch for every (group, level, free / reaction row) job.  A work item is
// (job, tile of target boxes, slice dx of the NOFF offsets).  For every offset of its slice
// the class operator (P, Q) and the phase-rotated multipoles of the tile's sources are staged
// in shared memory in K-chunks and multiplied as a small GEMM (rows = output coefficients,
// columns = target boxes); each target's partial local expansion of the slice is written to
// its own slot [box][slot] and the slots are summed in a fixed order (k_m2l_reduce), so the
// result does not depend on scheduling.  (FP64 mode and p > 10; the mixed mode uses k_m2l_tc.)
// ---------------------------------------------------------------------------------------
constexpr int M2L_KC = 32;
constexpr int M2L_NSLICE = NSLICE;  // offsets with dx = -OFF_R..OFF_R, SLICE_OFFS each

struct XJob {
  const int32_t *tlist;   // target box indices (nullptr: 0..ntb-1)
  const uint32_t *d_ntl;  // number of entries of tlist (device)
  int64_t ntb;
  const int32_t *vlist;   // [ntb][NOFF] source box or -1
  const int32_t *cls_of;  // [NOFF] operator class or -1
  const void *M;          // [nsb][ntypes][K]
  const void *ops;        // [ncls][ntypes][2][K][K]
  void *L;                // partial sums [ntb][M2L_NSLOT][K]: slot = slot0 + dx-slice
  int ntypes, slot0;
  int64_t item0;          // first work item of this job
  // octant tiles (free-space jobs at levels >= 3): tile = (octant, run of parents); its slot j
  // holds the child of parent j with that octant.  Boxes of one octant share their far offsets.
  const uint32_t *pstart; // parents' first child (nullptr: plain tiles over tlist / 0..ntb-1)
  const uint32_t *pcount;
  const uint64_t *ckey;   // keys of the target level
  int64_t npar;
};

__host__ __device__ __forceinline__ int64_t m2l_tiles(const XJob &J, int TT) {
  return J.pstart ? 8 * ((J.npar + TT - 1) / TT) : (J.ntb + TT - 1) / TT;
}

// target box of slot j of tile ti, or -1
__device__ __forceinline__ int m2l_target(const XJob &J, int64_t ti, int j, int TT, int64_t ntl) {
  if (J.pstart) {
    const int oct = (int)(ti & 7);
    const int64_t P = (ti >> 3) * TT + j;
    if (P >= J.npar) return -1;
    const uint32_t s0 = J.pstart[P], n = J.pcount[P];
    for (uint32_t k = 0; k < n; ++k)
      if ((int)(J.ckey[s0 + k] & 7ull) == oct) return (int)(s0 + k);
    return -1;
  }
  const int64_t t = ti * TT + j;
  return t < ntl ? (J.tlist ? J.tlist[t] : (int)t) : -1;
}
constexpr int M2L_NSLOT = 2 * M2L_NSLICE;  // free-space slices, then reaction slices

template <typename T, int TPT, int NR>
__global__ void __launch_bounds__(256) k_m2l(const XJob *jobs, int njobs, const T *rot, int K) {
  typedef typename C2<T>::t T2;
  constexpr int TT = 16 * TPT, KR = 16 * NR;
  extern __shared__ __align__(16) unsigned char smraw[];
  T *Pm = (T *)smraw;                 // [KR][KC]
  T *Qm = Pm + KR * M2L_KC;           // [KR][KC]
  T *Xr = Qm + KR * M2L_KC;           // [KC][TT]
  T *Xi = Xr + M2L_KC * TT;           // [KC][TT]
  int *sidx = (int *)(Xi + M2L_KC * TT);  // [TT]
  int *tid_ = sidx + TT;                  // [TT]
  // find the job of this item (jobs sorted by item0)
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].item0 <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const XJob J = jobs[lo];
  const int64_t local = (int64_t)blockIdx.x - J.item0;
  const int slice = (int)(local % M2L_NSLICE);
  const int64_t ti = local / M2L_NSLICE;
  const int64_t ntl = J.tlist ? (int64_t)*J.d_ntl : J.ntb;
  if (J.pstart ? (ti >> 3) * TT >= J.npar : ti * TT >= ntl) return;
  const T2 *M = (const T2 *)J.M;
  const T *ops = (const T *)J.ops;
  T2 *L = (T2 *)J.L;
  const int ntypes = J.ntypes;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  if (threadIdx.x < TT) tid_[threadIdx.x] = m2l_target(J, ti, threadIdx.x, TT, ntl);
  T Lr[NR][TPT], Li[NR][TPT];
#pragma unroll
  for (int r = 0; r < NR; ++r)
#pragma unroll
    for (int j = 0; j < TPT; ++j) Lr[r][j] = Li[r][j] = 0;
  const size_t KK = (size_t)K * K;
  bool any = false;
  __syncthreads();
  for (int o = slice * SLICE_OFFS; o < slice * SLICE_OFFS + SLICE_OFFS; ++o) {
    const int cls = J.cls_of[o];
    if (cls < 0) continue;
    int has = 0;
    if (threadIdx.x < TT) {
      const int t = tid_[threadIdx.x];
      const int s = (t >= 0) ? J.vlist[(size_t)t * NOFF + o] : -1;
      sidx[threadIdx.x] = s;
      has = s >= 0;
    }
    if (!__syncthreads_or(has)) continue;
    any = true;
    T Yr[NR][TPT], Yi[NR][TPT];
#pragma unroll
    for (int r = 0; r < NR; ++r)
#pragma unroll
      for (int j = 0; j < TPT; ++j) Yr[r][j] = Yi[r][j] = 0;
    const T *rc = rot + (size_t)o * (PMAX + 1) * 2;
    for (int tau = 0; tau < ntypes; ++tau) {
      const T *P = ops + ((size_t)cls * ntypes + tau) * 2 * KK, *Q = P + KK;
      for (int kc = 0; kc < K; kc += M2L_KC) {
        for (int e = threadIdx.x; e < KR * M2L_KC; e += blockDim.x) {
          const int r = e / M2L_KC, k = e % M2L_KC;
          const bool ok = r < K && kc + k < K;
          Pm[e] = ok ? P[(size_t)r * K + kc + k] : T(0);
          Qm[e] = ok ? Q[(size_t)r * K + kc + k] : T(0);
        }
        for (int e = threadIdx.x; e < M2L_KC * TT; e += blockDim.x) {
          const int k = e / TT, j = e % TT;
          const int s = sidx[j];
          T vr = 0, vi = 0;
          if (s >= 0 && kc + k < K) {
            const int m = cK.mof[kc + k];
            const T c = rc[2 * m], sn = rc[2 * m + 1];
            const T2 v = M[((size_t)s * ntypes + tau) * K + kc + k];
            vr = c * v.x - sn * v.y;
            vi = sn * v.x + c * v.y;
          }
          Xr[e] = vr;
          Xi[e] = vi;
        }
        __syncthreads();
#pragma unroll 4
        for (int k = 0; k < M2L_KC; ++k) {
          T xr[TPT], xi[TPT];
#pragma unroll
          for (int j = 0; j < TPT; ++j) {
            xr[j] = Xr[k * TT + tx + 16 * j];
            xi[j] = Xi[k * TT + tx + 16 * j];
          }
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            const T pv = Pm[(ty + 16 * r) * M2L_KC + k], qv = Qm[(ty + 16 * r) * M2L_KC + k];
#pragma unroll
            for (int j = 0; j < TPT; ++j) {
              Yr[r][j] += pv * xr[j];
              Yi[r][j] += qv * xi[j];
            }
          }
        }
        __syncthreads();
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int row = ty + 16 * r;
      if (row >= K) break;
      const int m = cK.mof[row];
      const T c = rc[2 * m], sn = rc[2 * m + 1];
#pragma unroll
      for (int j = 0; j < TPT; ++j) {
        Lr[r][j] += c * Yr[r][j] + sn * Yi[r][j];
        Li[r][j] += c * Yi[r][j] - sn * Yr[r][j];
      }
    }
  }
  if (!any) return;
#pragma unroll
  for (int j = 0; j < TPT; ++j) {
    const int t = tid_[tx + 16 * j];
    if (t < 0) continue;
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      const int row = ty + 16 * r;
      if (row >= K) break;
      L[((size_t)t * M2L_NSLOT + J.slot0 + slice) * K + row] = T2{Lr[r][j], Li[r][j]};
    }
  }
}

// FP32 multipole-to-local with asynchronous double-buffered staging.  A work item (job, tile of
// 96 target boxes, dx-slice) first lists its (offset, type) steps that have at least one source;
// every step copies the class operator (P, Q, K x K) and the tile's source multipoles into a
// shared-memory stage with cp.async while the previous step is multiplied.  After a stage lands
// the multipoles are rotated by e^{i mu phi} in place; the product is rotated by e^{-i m phi}
// into the register accumulators, which are written to the slice's partial slots at the end.
constexpr int F32_TPT = 6, F32_TT = 16 * F32_TPT, F32_NR = 5, F32_KR = 16 * F32_NR;
constexpr int F32_MAXSTEP = SLICE_OFFS * 2 * (MAXLAYER - 1);  // offsets x source types (2L, L <= 8)
constexpr int HASW = (SLICE_OFFS + 31) / 32;  // words of a per-slice offset mask

__device__ __forceinline__ void cp_async8(void *smem, const void *gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 8 : 0));
}
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, bool valid) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(valid ? 16 : 0));
}
__device__ __forceinline__ void cp_async4(void *smem, const void *gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

static size_t m2l_f32_smem(int K) {
  const size_t op = (size_t)2 * F32_KR * K * 4, xs = (size_t)F32_TT * (K + 1) * 8;
  return 2 * (op + xs) + sizeof(int) * (F32_TT + F32_MAXSTEP + 2 * F32_TT + F32_KR) + 2 * (PMAX + 1) * 8 * 2;
}

__global__ void __launch_bounds__(256, 1) k_m2l_f32(const XJob *jobs, int njobs, const float *rot, int K) {
  extern __shared__ __align__(16) unsigned char smraw[];
  const size_t opsz = (size_t)2 * F32_KR * K, xsz = (size_t)F32_TT * (K + 1) * 2;  // floats
  float *stage[2];
  stage[0] = (float *)smraw;
  stage[1] = stage[0] + opsz + xsz;
  int *tid_ = (int *)(stage[1] + opsz + xsz);
  int *steps = tid_ + F32_TT;                // (o << 4) | tau
  int *srcs = steps + F32_MAXSTEP;           // [2][TT] source box per stage
  int *mofs = srcs + 2 * F32_TT;              // [KR] m of each half-representation index
  float *rotc = (float *)(mofs + F32_KR);     // [2][PMAX+1][2]
  __shared__ int nsteps;
  __shared__ unsigned hasmask[HASW];
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].item0 <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const XJob J = jobs[lo];
  const int64_t local = (int64_t)blockIdx.x - J.item0;
  const int slice = (int)(local % M2L_NSLICE);
  const int64_t ti = local / M2L_NSLICE;
  const int64_t ntl = J.tlist ? (int64_t)*J.d_ntl : J.ntb;
  if (J.pstart ? (ti >> 3) * F32_TT >= J.npar : ti * F32_TT >= ntl) return;
  const float2 *M = (const float2 *)J.M;
  const float *ops = (const float *)J.ops;
  float2 *L = (float2 *)J.L;
  const int ntypes = J.ntypes;
  const size_t KK = (size_t)K * K;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  if (threadIdx.x < F32_TT) tid_[threadIdx.x] = m2l_target(J, ti, threadIdx.x, F32_TT, ntl);
  if (threadIdx.x < HASW) hasmask[threadIdx.x] = 0u;
  if (threadIdx.x < F32_KR) mofs[threadIdx.x] = threadIdx.x < K ? cK.mof[threadIdx.x] : 0;
  // zero the operator padding rows K..KR-1 of both stages once
  for (int s2 = 0; s2 < 2; ++s2)
    for (int e = threadIdx.x; e < 2 * (F32_KR - K) * K; e += blockDim.x) {
      const int half = e / ((F32_KR - K) * K), r = e % ((F32_KR - K) * K);
      stage[s2][half * F32_KR * K + K * K + r] = 0.0f;
    }
  __syncthreads();
  // offsets of the slice with at least one source in the tile
  if (threadIdx.x < F32_TT) {
    const int t = tid_[threadIdx.x];
    if (t >= 0)
      for (int k = 0; k < SLICE_OFFS; ++k) {
        const int o = slice * SLICE_OFFS + k;
        if (J.cls_of[o] >= 0 && J.vlist[(size_t)t * NOFF + o] >= 0) atomicOr(&hasmask[k >> 5], 1u << (k & 31));
      }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int n = 0;
    for (int k = 0; k < SLICE_OFFS; ++k)
      if (hasmask[k >> 5] & (1u << (k & 31)))
        for (int tau = 0; tau < ntypes; ++tau) steps[n++] = ((slice * SLICE_OFFS + k) << 4) | tau;
    nsteps = n;
  }
  __syncthreads();
  const int ns = nsteps;
  if (ns == 0) return;
  // --- staging helpers (explicit, see below)
  auto stage_step = [&](int st, int buf) {
    const int o = steps[st] >> 4, tau = steps[st] & 15;
    const int cls = J.cls_of[o];
    float *opP = stage[buf], *opQ = opP + F32_KR * K;
    float *xs = opP + opsz;
    const float *P = ops + ((size_t)cls * ntypes + tau) * 2 * KK, *Q = P + KK;
    if (KK & 1) {  // Q is only 4-byte aligned: 4-byte granules
      for (int e = threadIdx.x; e < (int)KK; e += blockDim.x) {
        cp_async4(opP + e, P + e);
        cp_async4(opQ + e, Q + e);
      }
    } else {
      const int halfKK = (int)(KK / 2);
      for (int e = threadIdx.x; e < halfKK; e += blockDim.x) {
        cp_async8(opP + 2 * e, P + 2 * e, true);
        cp_async8(opQ + 2 * e, Q + 2 * e, true);
      }
    }
    int *sb = srcs + buf * F32_TT;
    if (threadIdx.x < F32_TT) {
      const int t = tid_[threadIdx.x];
      sb[threadIdx.x] = t >= 0 ? J.vlist[(size_t)t * NOFF + o] : -1;
    }
    if (threadIdx.x < 2 * (PMAX + 1)) {
      float *rc = rotc + buf * 2 * (PMAX + 1);
      rc[threadIdx.x] = rot[(size_t)o * (PMAX + 1) * 2 + threadIdx.x];
    }
    __syncthreads();
    // multipoles: row j (K float2, padded to K+1) of source sb[j]; 8-byte granules
    for (int e = threadIdx.x; e < F32_TT * K; e += blockDim.x) {
      const int j = e / K, k = e % K;
      const int s = sb[j];
      const float2 *src = s >= 0 ? M + ((size_t)s * ntypes + tau) * K + k : M;
      cp_async8(xs + 2 * ((size_t)j * (K + 1) + k), src, s >= 0);
    }
    cp_commit();
  };
  float Lr[F32_NR][F32_TPT], Li[F32_NR][F32_TPT];
#pragma unroll
  for (int r = 0; r < F32_NR; ++r)
#pragma unroll
    for (int j = 0; j < F32_TPT; ++j) Lr[r][j] = Li[r][j] = 0.f;
  stage_step(0, 0);
  for (int st = 0; st < ns; ++st) {
    const int buf = st & 1;
    if (st + 1 < ns) {
      stage_step(st + 1, buf ^ 1);
      cp_wait1();
    } else {
      cp_wait0();
    }
    __syncthreads();
    float *opP = stage[buf], *opQ = opP + F32_KR * K;
    float *xs = opP + opsz;
    const float *rc = rotc + buf * 2 * (PMAX + 1);
    // rotate the staged multipoles by e^{i mu phi}
    for (int e = threadIdx.x; e < F32_TT * K; e += blockDim.x) {
      const int j = e / K, k = e % K;
      float2 *v = (float2 *)(xs + 2 * ((size_t)j * (K + 1) + k));
      const int m = mofs[k];
      const float c = rc[2 * m], sn = rc[2 * m + 1];
      const float2 a = *v;
      *v = make_float2(c * a.x - sn * a.y, sn * a.x + c * a.y);
    }
    __syncthreads();
    float Yr[F32_NR][F32_TPT], Yi[F32_NR][F32_TPT];
#pragma unroll
    for (int r = 0; r < F32_NR; ++r)
#pragma unroll
      for (int j = 0; j < F32_TPT; ++j) Yr[r][j] = Yi[r][j] = 0.f;
    const float2 *xv = (const float2 *)xs;
#pragma unroll 2
    for (int k = 0; k < K; ++k) {
      float2 x[F32_TPT];
#pragma unroll
      for (int j = 0; j < F32_TPT; ++j) x[j] = xv[(size_t)(tx + 16 * j) * (K + 1) + k];
#pragma unroll
      for (int r = 0; r < F32_NR; ++r) {
        const float pv = opP[(ty + 16 * r) * K + k], qv = opQ[(ty + 16 * r) * K + k];
#pragma unroll
        for (int j = 0; j < F32_TPT; ++j) {
          Yr[r][j] = fmaf(pv, x[j].x, Yr[r][j]);
          Yi[r][j] = fmaf(qv, x[j].y, Yi[r][j]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < F32_NR; ++r) {
      const int row = ty + 16 * r;
      const int m = mofs[row];
      const float c = rc[2 * m], sn = rc[2 * m + 1];
#pragma unroll
      for (int j = 0; j < F32_TPT; ++j) {
        Lr[r][j] += c * Yr[r][j] + sn * Yi[r][j];
        Li[r][j] += c * Yi[r][j] - sn * Yr[r][j];
      }
    }
    __syncthreads();  // the stage is refilled two steps later
  }
#pragma unroll
  for (int j = 0; j < F32_TPT; ++j) {
    const int t = tid_[tx + 16 * j];
    if (t < 0) continue;
#pragma unroll
    for (int r = 0; r < F32_NR; ++r) {
      const int row = ty + 16 * r;
      if (row >= K) break;
      L[((size_t)t * M2L_NSLOT + J.slot0 + slice) * K + row] = make_float2(Lr[r][j], Li[r][j]);
    }
  }
}

// L[box][k] += sum over the partial slots, in slot order (deterministic)
template <typename T>
__global__ void k_m2l_reduce(const RJob *jobs, int njobs, int K) {
  typedef typename C2<T>::t T2;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].e0 <= g) lo = mid; else hi = mid - 1;
  }
  const RJob J = jobs[lo];
  const int64_t e = g - J.e0;
  if (e < 0 || e >= J.n) return;
  const int64_t box = e / K, k = e % K;
  const T2 *P = (const T2 *)J.part + box * M2L_NSLOT * K + k;
  T sx = 0, sy = 0;
#pragma unroll
  for (int s = 0; s < M2L_NSLOT; ++s) {
    sx += P[(size_t)s * K].x;
    sy += P[(size_t)s * K].y;
  }
  T2 &d = ((T2 *)J.L)[e];
  d.x += sx;
  d.y += sy;
}

// ---------------------------------------------------------------------------------------
// L2P with field: one warp per leaf box
// ---------------------------------------------------------------------------------------
template <typename T, int PT>
__global__ void k_l2p(const uint32_t *d_nb, const uint64_t *bkey, const uint32_t *bstart, const uint32_t *bcount,
                      const double *x, const double *y, const double *z, const uint32_t *src, Geo geo, double lam,
                      int p, int K, const typename C2<T>::t *L, double *phi, double *field) {
  typedef typename C2<T>::t T2;
  __shared__ T2 Ls[4][KHALF_MAX];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t box = (int64_t)blockIdx.x * 4 + warp;
  if (box >= *d_nb) return;
  for (int e = lane; e < K; e += 32) Ls[warp][e] = L[(size_t)box * K + e];
  __syncwarp();
  double cx, cy, cz;
  box_center(bkey[box], geo, cx, cy, cz);
  const double ih = 1.0 / geo.h;
  const T lh = (T)(lam * geo.h);
  const uint32_t st = bstart[box], cnt = bcount[box];
  const T2 *Lw = Ls[warp];
  for (uint32_t j = lane; j < cnt; j += 32) {
    const uint32_t k = st + j;
    const T rx = (T)((x[k] - cx) * ih), ry = (T)((y[k] - cy) * ih), rz = (T)((z[k] - cz) * ih);
    const T r2 = rx * rx + ry * ry + rz * rz;
    T it[PT + 3];
    itilde_all<T, PT + 2>(lh * lh * r2, it);
    T ph = 0, S1 = 0, Gz = 0, Gpr = 0, Gpi = 0;
    T2 Rmm = T2{(T)(0.5 / sqrt(PI)), T(0)};
#pragma unroll
    for (int m = 0; m <= PT; ++m) {
      if (m > p) break;
      if (m > 0) {
        const T s = CK<T>::sect(m);
        const T2 t = T2{Rmm.x * rx - Rmm.y * ry, Rmm.x * ry + Rmm.y * rx};
        Rmm = T2{s * t.x, s * t.y};
      }
      const T wm = m ? T(2) : T(1);
      T2 p1 = T2{0, 0}, p2 = T2{0, 0};
#pragma unroll
      for (int n = m; n <= PT; ++n) {
        if (n > p) break;
        T2 R;
        if (n == m) R = Rmm;
        else if (n == m + 1) { const T s = CK<T>::sub(m) * rz; R = T2{s * p1.x, s * p1.y}; }
        else {
          const T a = CK<T>::A(n, m) * rz, b = CK<T>::B(n, m) * r2;
          R = T2{a * p1.x - b * p2.x, a * p1.y - b * p2.y};
        }
        p2 = p1;
        p1 = R;
        const T2 Lnm = Lw[hidx(n, m)];
        const T re = Lnm.x * R.x - Lnm.y * R.y;
        ph += wm * it[n] * re;
        S1 += wm * it[n + 1] / T(2 * n + 3) * re;
        if (n < p) {
          const T in1 = it[n + 1];
          const T2 Lz = Lw[hidx(n + 1, m)];
          Gz += wm * in1 * CK<T>::gz(n, m) * (Lz.x * R.x - Lz.y * R.y);
          if (m >= 1) {
            const T2 La = Lw[hidx(n + 1, m - 1)];
            const T ca = in1 * CK<T>::ga(n, m);
            Gpr += ca * (La.x * R.x - La.y * R.y);
            Gpi += ca * (La.x * R.y + La.y * R.x);
          }
          const T2 Lb = Lw[hidx(n + 1, m + 1)];
          const T cb = in1 * CK<T>::gb(n, m);
          // - conj(Lb R)
          Gpr -= cb * (Lb.x * R.x - Lb.y * R.y);
          Gpi += cb * (Lb.x * R.y + Lb.y * R.x);
        }
      }
    }
    const uint32_t i = src[k];
    phi[i] += (double)ph;
    if (field) {
      const double l2h = lam * lam * geo.h;  // lambda^2 r = lambda^2 h r_u
      field[3 * i] -= l2h * (double)rx * (double)S1 + (double)Gpr * ih;
      field[3 * i + 1] -= l2h * (double)ry * (double)S1 + (double)Gpi * ih;
      field[3 * i + 2] -= l2h * (double)rz * (double)S1 + (double)Gz * ih;
    }
  }
}

// ---------------------------------------------------------------------------------------
// free-space P2P over the near list (27 neighbours incl. the box itself).  One CTA of
// P2P_TPB threads per target leaf; the sources of all neighbours are streamed through shared
// memory in full tiles of P2P_SRC (position, charge) records; a thread holds up to two targets
// (t and t + P2P_TPB), chosen per warp, so each shared-memory record read serves two pairs.
// Pair math in T, per-tile partial sums in T, per-target accumulation in FP64.  The self pair
// (r = 0) is dropped by a select, so distinct charges at one point do not interact either.
// ---------------------------------------------------------------------------------------
constexpr int P2P_THREADS = 128;  // reaction near field
constexpr int P2P_TPB = 64, P2P_SRC = 128;

__device__ __forceinline__ float fexp(float x) { return __expf(x); }
__device__ __forceinline__ double fexp(double x) { return exp(x); }
__device__ __forceinline__ float frsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double frsqrt(double x) { return rsqrt(x); }

template <typename T>
struct alignas(4 * sizeof(T)) V4 {
  T x, y, z, w;
};

template <typename T, int NT, bool COMP>
__device__ __forceinline__ void p2p_free_tile(const V4<T> *__restrict__ sh, const V4<T> *__restrict__ sl, int nn,
                                              const T (&px)[2], const T (&py)[2], const T (&pz)[2],
                                              const T (&qx)[2], const T (&qy)[2], const T (&qz)[2], T lam,
                                              T (&fp)[2], T (&fx)[2], T (&fy)[2], T (&fz)[2]) {
#pragma unroll 2
  for (int j = 0; j < nn; ++j) {
    const V4<T> s = sh[j];
    V4<T> sL;
    if (COMP) sL = sl[j];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      T dx = px[t] - s.x, dy = py[t] - s.y, dz = pz[t] - s.z;
      if (COMP) {
        dx += qx[t] - sL.x;
        dy += qy[t] - sL.y;
        dz += qz[t] - sL.z;
      }
      const T r2 = dx * dx + dy * dy + dz * dz;
      const T ri = r2 > T(0) ? frsqrt(r2) : T(0);
      const T r = r2 * ri;
      const T e = s.w * fexp(-lam * r) * ri;
      fp[t] += e;
      const T f = e * (ri * ri) * (T(1) + lam * r);
      fx[t] += f * dx;
      fy[t] += f * dy;
      fz[t] += f * dz;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(P2P_TPB) k_p2p_free(const uint32_t *d_nb, const uint64_t *bkey,
                                                      const uint32_t *bstart, const uint32_t *bcount,
                                                      const int32_t *ulist, const double *x, const double *y,
                                                      const double *z, const double *q, const uint32_t *src,
                                                      Geo geo, double lam, double scale, double *phi,
                                                      double *field) {
  constexpr bool comp = sizeof(T) == 4;
  __shared__ V4<T> sh[P2P_SRC], sl[comp ? P2P_SRC : 1];
  __shared__ uint32_t nb_start[NNEAR], nb_pre[NNEAR + 1];
  const uint32_t box = blockIdx.x;
  if (box >= *d_nb) return;
  double cx, cy, cz;
  box_center(bkey[box], geo, cx, cy, cz);
  if (threadIdx.x == 0) {
    uint32_t acc = 0;
    for (int o = 0; o < NNEAR; ++o) {
      const int s = ulist[(size_t)box * NNEAR + o];
      nb_pre[o] = acc;
      nb_start[o] = s < 0 ? 0u : bstart[s];
      acc += s < 0 ? 0u : bcount[s];
    }
    nb_pre[NNEAR] = acc;
  }
  __syncthreads();
  const uint32_t stot = nb_pre[NNEAR];
  const uint32_t tst = bstart[box], tcnt = bcount[box];
  const T tl = (T)lam;
  const unsigned full = 0xffffffffu;
  for (uint32_t t0 = 0; t0 < tcnt; t0 += 2 * P2P_TPB) {
    T px[2], py[2], pz[2], qx[2], qy[2], qz[2];
    bool tv[2];
    uint32_t tk[2];
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      const uint32_t tj = t0 + threadIdx.x + t * P2P_TPB;
      tv[t] = tj < tcnt;
      tk[t] = tst + (tv[t] ? tj : 0);
      const double ox = x[tk[t]] - cx, oy = y[tk[t]] - cy, oz = z[tk[t]] - cz;
      px[t] = (T)ox;
      py[t] = (T)oy;
      pz[t] = (T)oz;
      qx[t] = comp ? (T)(ox - (double)px[t]) : T(0);
      qy[t] = comp ? (T)(oy - (double)py[t]) : T(0);
      qz[t] = comp ? (T)(oz - (double)pz[t]) : T(0);
    }
    const bool w2 = __any_sync(full, tv[1]), w1 = __any_sync(full, tv[0]);
    double aphi[2] = {0, 0}, ax[2] = {0, 0}, ay[2] = {0, 0}, az[2] = {0, 0};
    for (uint32_t s0 = 0; s0 < stot; s0 += P2P_SRC) {
      __syncthreads();
      for (uint32_t jj = threadIdx.x; jj < P2P_SRC; jj += P2P_TPB) {
        const uint32_t g = s0 + jj;
        if (g < stot) {
          int o = 0;
          while (nb_pre[o + 1] <= g) ++o;  // neighbour holding source g (empty ones skipped)
          const uint32_t k = nb_start[o] + (g - nb_pre[o]);
          const double ux = x[k] - cx, uy = y[k] - cy, uz = z[k] - cz;
          V4<T> h;
          h.x = (T)ux;
          h.y = (T)uy;
          h.z = (T)uz;
          h.w = (T)q[k];
          sh[jj] = h;
          if (comp) {
            V4<T> lo;
            lo.x = (T)(ux - (double)h.x);
            lo.y = (T)(uy - (double)h.y);
            lo.z = (T)(uz - (double)h.z);
            lo.w = T(0);
            sl[jj] = lo;
          }
        }
      }
      __syncthreads();
      const int nn = (int)min((uint32_t)P2P_SRC, stot - s0);
      T fp[2] = {0, 0}, fx[2] = {0, 0}, fy[2] = {0, 0}, fz[2] = {0, 0};
      if (w2) p2p_free_tile<T, 2, comp>(sh, sl, nn, px, py, pz, qx, qy, qz, tl, fp, fx, fy, fz);
      else if (w1) p2p_free_tile<T, 1, comp>(sh, sl, nn, px, py, pz, qx, qy, qz, tl, fp, fx, fy, fz);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        aphi[t] += (double)fp[t];
        ax[t] += (double)fx[t];
        ay[t] += (double)fy[t];
        az[t] += (double)fz[t];
      }
    }
#pragma unroll
    for (int t = 0; t < 2; ++t) {
      if (!tv[t]) continue;
      const uint32_t i = src[tk[t]];
      phi[i] += scale * aphi[t];
      if (field) {
        field[3 * i] += scale * ax[t];
        field[3 * i + 1] += scale * ay[t];
        field[3 * i + 2] += scale * az[t];
      }
    }
  }
}

// Mixed-precision P2P.  Every point of the target tree carries its offset from its own leaf
// centre as FP32 hi + lo pairs (k_split_points, once per evaluation).  For a neighbour whose
// centre lies delta * h away (delta in {-1,0,1}^3), the targets are moved into the
// neighbour's frame by an exact FP32 two-sum with h = hh + hl, so source records are plain
// copies: they are staged with cp.async, one neighbour chunk ahead of the one being summed.
// Per-chunk sums are folded into Kahan-compensated FP32 totals; no FP64 in the pair loop.
__global__ void k_split_points(const uint32_t *d_nb, const uint64_t *bkey, const uint32_t *bstart,
                               const uint32_t *bcount, const double *x, const double *y, const double *z,
                               const double *q, Geo geo, float4 *h4, float4 *l4) {
  const uint32_t box = blockIdx.x;
  if (box >= *d_nb) return;
  double cx, cy, cz;
  box_center(bkey[box], geo, cx, cy, cz);
  const uint32_t st = bstart[box], cnt = bcount[box];
  for (uint32_t j = threadIdx.x; j < cnt; j += blockDim.x) {
    const uint32_t k = st + j;
    const double ox = x[k] - cx, oy = y[k] - cy, oz = z[k] - cz;
    const float hx = (float)ox, hy = (float)oy, hz = (float)oz;
    h4[k] = make_float4(hx, hy, hz, (float)q[k]);
    l4[k] = make_float4((float)(ox - (double)hx), (float)(oy - (double)hy), (float)(oz - (double)hz), 0.f);
  }
}

__device__ __forceinline__ void two_sum_shift(float hi, float lo, float b, float bl, float &oh, float &ol) {
  // (hi + lo) + (b + bl) with b exact: oh + ol, the rounding error of hi + b kept in ol
  const float a = hi + b;
  const float bb = a - hi;
  const float e = (hi - (a - bb)) + (b - bb);
  oh = a;
  ol = (lo + bl) + e;
}

__device__ __forceinline__ void kahan_add(float &s, float &c, float v) {
  const float y = v - c;
  const float t = s + y;
  c = (t - s) - y;
  s = t;
}

// 2^x on the special-function unit (max. relative error about 2^-22)
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// 1/sqrt(x) on the special-function unit (max. relative error about 2^-22.9; subnormal inputs
// flushed to zero, which cannot occur for r^2 of distinct points at the FP32 offsets used here)
__device__ __forceinline__ float rsqrt_approx(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// e^{-lambda r} = 2^{(-lambda log2 e) r}; field factor (1 + lambda r) / r^2 = (1/r)(1/r + lambda).
// MODE by the source box's offset from the target leaf: P2P_SELF (the leaf itself: compensated
// coordinates, the r = 0 self pair dropped by a select), P2P_TOUCH (a box that touches the leaf:
// compensated coordinates, r > 0), P2P_APART (a box at least one box away: r >= h, so the FP32
// rounding of the plain differences, ~2^-23 of 3h, is below 1e-7 of r and the low parts are not
// used).
constexpr int P2P_APART = 0, P2P_TOUCH = 1, P2P_SELF = 2;
template <int NT, int MODE>
__device__ __forceinline__ void p2p_f32_chunk(const float4 *__restrict__ sh, const float4 *__restrict__ sl, int nn,
                                              const float (&px)[4], const float (&py)[4], const float (&pz)[4],
                                              const float (&qx)[4], const float (&qy)[4], const float (&qz)[4],
                                              float lam, float (&fp)[4], float (&fx)[4], float (&fy)[4],
                                              float (&fz)[4]) {
  const float nl2 = -lam * 1.44269504088896341f;
#pragma unroll 2
  for (int j = 0; j < nn; ++j) {
    const float4 s = sh[j];
    float4 sL = make_float4(0.f, 0.f, 0.f, 0.f);
    if (MODE != P2P_APART) sL = sl[j];
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      float dx, dy, dz;
      if (MODE == P2P_APART) {
        dx = px[t] - s.x;
        dy = py[t] - s.y;
        dz = pz[t] - s.z;
      } else {
        dx = (px[t] - s.x) + (qx[t] - sL.x);
        dy = (py[t] - s.y) + (qy[t] - sL.y);
        dz = (pz[t] - s.z) + (qz[t] - sL.z);
      }
      const float r2 = dx * dx + dy * dy + dz * dz;
      const float ri = (MODE == P2P_SELF) ? (r2 > 0.f ? rsqrt_approx(r2) : 0.f) : rsqrt_approx(r2);
      const float e = s.w * ex2_approx(nl2 * (r2 * ri)) * ri;
      fp[t] += e;
      const float f = e * ri * (ri + lam);
      fx[t] += f * dx;
      fy[t] += f * dy;
      fz[t] += f * dz;
    }
  }
}

// One warp per (target leaf, half) and no block-wide barriers: warp h of a leaf takes the
// targets 128 i + 64 h + lane + 32 t (t = 0, 1) and streams the sources of the leaf's near boxes
// through its own double-buffered chunks of P2P_WSRC records.  The near boxes are compacted to the
// non-empty ones first; a chunk is (near box k, offset within it), walked by a cursor.  Two warps
// per leaf and an 80-register budget keep 24 warps resident per SM.
constexpr int P2P_WARPS = 4, P2P_WSRC = 64;

struct P2PCursor {
  int k;
  uint32_t off;
};
__device__ __forceinline__ void p2p_next(P2PCursor &c, const uint32_t *nb_cnt) {
  c.off += P2P_WSRC;
  if (c.off >= nb_cnt[c.k]) {
    ++c.k;
    c.off = 0;
  }
}

template <int NT>
__device__ __forceinline__ void p2p_warp_pass(int lane, uint32_t t0, uint32_t tcnt, uint32_t tst,
                                              const float4 *__restrict__ h4, const float4 *__restrict__ l4,
                                              const uint32_t *src, float hh, float hl, float lam, double scale,
                                              double *phi, double *field, float4 (*sh)[P2P_WSRC],
                                              float4 (*sl)[P2P_WSRC], const uint32_t *nb_start,
                                              const uint32_t *nb_cnt, const int *nb_o, int nch) {
  float th[2][3], tl[2][3];
  uint32_t tk[2];
  bool tv[2];
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    const uint32_t tj = t0 + lane + 32 * t;
    tv[t] = t < NT && tj < tcnt;
    tk[t] = tst + (tv[t] ? tj : 0);
    const float4 a = h4[tk[t]], b = l4[tk[t]];
    th[t][0] = a.x; th[t][1] = a.y; th[t][2] = a.z;
    tl[t][0] = b.x; tl[t][1] = b.y; tl[t][2] = b.z;
  }
  auto mode_of = [&](int k) {
    int ddx, ddy, ddz;
    near_decode(nb_o[k], ddx, ddy, ddz);
    const int ch = cheb3(ddx, ddy, ddz);
    return ch == 0 ? P2P_SELF : (ch == 1 ? P2P_TOUCH : P2P_APART);
  };
  auto issue = [&](const P2PCursor &cc, int buf) {
    const uint32_t first = nb_start[cc.k] + cc.off;
    const int nn = (int)min((uint32_t)P2P_WSRC, nb_cnt[cc.k] - cc.off);
    if (mode_of(cc.k) == P2P_APART) {
      for (int j = lane; j < nn; j += 32) cp_async16(&sh[buf][j], &h4[first + j], true);
    } else {
      for (int e = lane; e < 2 * P2P_WSRC; e += 32) {
        const int j = e >> 1;
        if (j < nn) {
          if (e & 1) cp_async16(&sl[buf][j], &l4[first + j], true);
          else cp_async16(&sh[buf][j], &h4[first + j], true);
        }
      }
    }
    cp_commit();
  };
  float sp[2] = {0, 0}, cp[2] = {0, 0}, sx[2] = {0, 0}, cx[2] = {0, 0};
  float sy[2] = {0, 0}, cy[2] = {0, 0}, sz[2] = {0, 0}, cz[2] = {0, 0};
  P2PCursor ci{0, 0u}, cc{0, 0u};  // next chunk to issue, chunk being summed
  if (nch > 0) {
    issue(ci, 0);
    p2p_next(ci, nb_cnt);
  }
  for (int c = 0; c < nch; ++c) {
    const int buf = c & 1;
    if (c + 1 < nch) {
      issue(ci, buf ^ 1);
      p2p_next(ci, nb_cnt);
      cp_wait1();
    } else {
      cp_wait0();
    }
    __syncwarp();
    const int nn = (int)min((uint32_t)P2P_WSRC, nb_cnt[cc.k] - cc.off);
    int ddx, ddy, ddz;
    near_decode(nb_o[cc.k], ddx, ddy, ddz);
    const int mode = mode_of(cc.k);
    p2p_next(cc, nb_cnt);
    float px[4], py[4], pz[4], qx[4], qy[4], qz[4];
    const float dxh = -(float)ddx, dyh = -(float)ddy, dzh = -(float)ddz;
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      two_sum_shift(th[t][0], tl[t][0], dxh * hh, dxh * hl, px[t], qx[t]);
      two_sum_shift(th[t][1], tl[t][1], dyh * hh, dyh * hl, py[t], qy[t]);
      two_sum_shift(th[t][2], tl[t][2], dzh * hh, dzh * hl, pz[t], qz[t]);
    }
    float fp[4] = {0, 0, 0, 0}, fx[4] = {0, 0, 0, 0}, fy[4] = {0, 0, 0, 0}, fz[4] = {0, 0, 0, 0};
    if (mode == P2P_APART)
      p2p_f32_chunk<NT, P2P_APART>(sh[buf], sl[buf], nn, px, py, pz, qx, qy, qz, lam, fp, fx, fy, fz);
    else if (mode == P2P_TOUCH)
      p2p_f32_chunk<NT, P2P_TOUCH>(sh[buf], sl[buf], nn, px, py, pz, qx, qy, qz, lam, fp, fx, fy, fz);
    else
      p2p_f32_chunk<NT, P2P_SELF>(sh[buf], sl[buf], nn, px, py, pz, qx, qy, qz, lam, fp, fx, fy, fz);
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      kahan_add(sp[t], cp[t], fp[t]);
      kahan_add(sx[t], cx[t], fx[t]);
      kahan_add(sy[t], cy[t], fy[t]);
      kahan_add(sz[t], cz[t], fz[t]);
    }
    __syncwarp();  // buffer buf is refilled by the issue of chunk c + 2
  }
#pragma unroll
  for (int t = 0; t < NT; ++t) {
    if (!tv[t]) continue;
    const uint32_t i = src[tk[t]];
    phi[i] += scale * ((double)sp[t] - (double)cp[t]);
    if (field) {
      field[3 * i] += scale * ((double)sx[t] - (double)cx[t]);
      field[3 * i + 1] += scale * ((double)sy[t] - (double)cy[t]);
      field[3 * i + 2] += scale * ((double)sz[t] - (double)cz[t]);
    }
  }
}

__global__ void __launch_bounds__(32 * P2P_WARPS, 6) k_p2p_free_f32(const P2PJob *jobs, int njobs) {
  __shared__ __align__(16) float4 sh_[P2P_WARPS][2][P2P_WSRC], sl_[P2P_WARPS][2][P2P_WSRC];
  __shared__ uint32_t nb_start_[P2P_WARPS][NNEAR], nb_cnt_[P2P_WARPS][NNEAR];
  __shared__ int nb_o_[P2P_WARPS][NNEAR];
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].block0 <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const P2PJob &J = jobs[lo];
  const uint32_t *bstart = J.bstart, *bcount = J.bcount, *src = J.src;
  const int32_t *ulist = J.ulist;
  const float4 *h4 = J.h4, *l4 = J.l4;
  const float hh = J.hh, hl = J.hl, lam = J.lam;
  const double scale = J.scale;
  double *phi = J.phi, *field = J.field;
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t gw = (uint32_t)((int64_t)blockIdx.x - J.block0) * P2P_WARPS + w;
  const uint32_t box = gw >> 1, half = gw & 1;
  if (box >= *J.d_nb) return;
  const uint32_t tst = bstart[box], tcnt = bcount[box];
  if (64 * half >= tcnt) return;
  uint32_t *nb_start = nb_start_[w], *nb_cnt = nb_cnt_[w];
  int *nb_o = nb_o_[w];
  // compact the non-empty near boxes (slot order kept) and count their chunks
  int nnb = 0, nch = 0;
  for (int o0 = 0; o0 < NNEAR; o0 += 32) {
    const int o = o0 + lane;
    const int sb = o < NNEAR ? ulist[(size_t)box * NNEAR + o] : -1;
    const uint32_t cnt = sb >= 0 ? bcount[sb] : 0u;
    const unsigned m = __ballot_sync(0xffffffffu, cnt > 0);
    if (cnt > 0) {
      const int k = nnb + __popc(m & ((1u << lane) - 1u));
      nb_start[k] = bstart[sb];
      nb_cnt[k] = cnt;
      nb_o[k] = o;
    }
    nnb += __popc(m);
    int ch = (int)((cnt + P2P_WSRC - 1) / P2P_WSRC);
#pragma unroll
    for (int s2 = 16; s2; s2 >>= 1) ch += __shfl_xor_sync(0xffffffffu, ch, s2);
    nch += ch;
  }
  __syncwarp();
  for (uint32_t t0 = 64 * half; t0 < tcnt; t0 += 128) {
    if (tcnt - t0 > 32)
      p2p_warp_pass<2>(lane, t0, tcnt, tst, h4, l4, src, hh, hl, lam, scale, phi, field, sh_[w], sl_[w], nb_start,
                       nb_cnt, nb_o, nch);
    else
      p2p_warp_pass<1>(lane, t0, tcnt, tst, h4, l4, src, hh, hl, lam, scale, phi, field, sh_[w], sl_[w], nb_start,
                       nb_cnt, nb_o, nch);
  }
}

// ---------------------------------------------------------------------------------------
// reaction near field: target leaf box vs adjacent image leaf boxes across the interface,
// Sommerfeld integral by the precomputed node rule, truncated per pair at exp(-36)
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ float fj0(float x) { return j0f(x); }
__device__ __forceinline__ double fj0(double x) { return j0(x); }
__device__ __forceinline__ float fj1(float x) { return j1f(x); }
__device__ __forceinline__ double fj1(double x) { return j1(x); }

template <typename T>
__global__ void __launch_bounds__(P2P_THREADS) k_p2p_react(
    const uint32_t *d_nb, const uint64_t *tkey, const uint32_t *tstart, const uint32_t *tcount, const int32_t *ulist,
    const double *tx, const double *ty, const double *tz, const uint32_t *tsrc, const uint32_t *istart,
    const uint32_t *icount, const double *ix, const double *iy, const double *iz, const double *iq,
    const uint64_t *ikey, Geo geo, double dI, double sa, const double *nodes, int nq, double *phi, double *field) {
  __shared__ T sx[P2P_THREADS], sy[P2P_THREADS], szs[P2P_THREADS], sq[P2P_THREADS];
  __shared__ int st[P2P_THREADS];
  const uint32_t box = blockIdx.x;
  if (box >= *d_nb) return;
  bool any = false;
  for (int o = 0; o < NNEAR; ++o) any |= ulist[(size_t)box * NNEAR + o] >= 0;
  if (!any) return;
  double cx, cy, cz;
  box_center(tkey[box], geo, cx, cy, cz);
  const uint32_t tst = tstart[box], tcnt = tcount[box];
  for (uint32_t t0 = 0; t0 < tcnt; t0 += P2P_THREADS) {
    const uint32_t tj = t0 + threadIdx.x;
    const bool tv = tj < tcnt;
    const uint32_t tk = tst + (tv ? tj : 0);
    const T px = (T)(tx[tk] - cx), py = (T)(ty[tk] - cy);
    const T zt = (T)fabs(tz[tk] - dI);
    double aphi = 0, ax = 0, ay = 0, az = 0;
    for (int o = 0; o < NNEAR; ++o) {
      const int s = ulist[(size_t)box * NNEAR + o];
      if (s < 0) continue;
      const uint32_t sst = istart[s], scnt = icount[s];
      for (uint32_t s0 = 0; s0 < scnt; s0 += P2P_THREADS) {
        __syncthreads();
        if (s0 + threadIdx.x < scnt) {
          const uint32_t k = sst + s0 + threadIdx.x;
          sx[threadIdx.x] = (T)(ix[k] - cx);
          sy[threadIdx.x] = (T)(iy[k] - cy);
          szs[threadIdx.x] = (T)fabs(iz[k] - dI);
          sq[threadIdx.x] = (T)iq[k];
          st[threadIdx.x] = (int)(ikey[k] & 15ull);
        }
        __syncthreads();
        const uint32_t nn = min((uint32_t)P2P_THREADS, scnt - s0);
        if (!tv) continue;
        for (uint32_t jj = 0; jj < nn; ++jj) {
          const T dx = px - sx[jj], dy = py - sy[jj];
          const T rho = sqrt(dx * dx + dy * dy);
          const T zs = szs[jj];
          const T xcut = T(36) / (zt + zs);
          const double *nd = nodes + (size_t)st[jj] * nq * 4;
          T v = 0, vr = 0, vz = 0;
          for (int k = 0; k < nq; ++k) {
            const T lr = (T)nd[4 * k];
            if (lr > xcut) break;
            const T E = (T)nd[4 * k + 1] * fexp(-(T)nd[4 * k + 2] * zt - (T)nd[4 * k + 3] * zs);
            const T a = lr * rho;
            const T J0 = fj0(a);
            const T J1r = rho > T(0) ? fj1(a) / rho : T(0.5) * lr;
            v += E * J0;
            vr += E * lr * J1r;
            vz += E * J0 * (T)nd[4 * k + 2];
          }
          const T qq = sq[jj];
          aphi += (double)(qq * v);
          ax += (double)(qq * dx * vr);
          ay += (double)(qq * dy * vr);
          az += (double)(qq * vz);
        }
      }
    }
    if (tv) {
      const uint32_t i = tsrc[tk];
      phi[i] += aphi;
      if (field) {
        field[3 * i] += ax;
        field[3 * i + 1] += ay;
        field[3 * i + 2] += sa * az;
      }
    }
  }
}

// ---------------------------------------------------------------------------------------
// driver for one group
// ---------------------------------------------------------------------------------------
struct Tables {
  int32_t *cls_free, *cls_react;  // [NOFF], [2][NKT][NOFF]
  void *rot, *rot4;               // per precision
};
Tables g_tab_d[LPB_MAX_DEVICES], g_tab_f[LPB_MAX_DEVICES];  // per device
static std::atomic<uint64_t> g_tab_ready{0};

static void make_tables(Ctx &c) {
  if (!not_done_on_device(g_tab_ready)) return;
  // operator class of every offset that can appear in a far list (|d|_inf >= 2); which offsets
  // do appear is decided by the list builder for the context's separation
  std::vector<int32_t> cf(NOFF, -1), cr(2 * NKT * NOFF, -1);
  std::vector<double> rot(NOFF * (PMAX + 1) * 2), rot4(4 * (PMAX + 1) * 2);
  for (int o = 0; o < NOFF; ++o) {
    int dx, dy, dz;
    off_decode(o, dx, dy, dz);
    const int cheb = cheb3(dx, dy, dz);
    if (cheb >= 2) cf[o] = rho_index(dx, dy) * NDZ + dz + OFF_R;
    for (int a = 1; a <= 2; ++a)
      for (int kt = 0; kt < NKT; ++kt) {
        const int ks = (a == 1) ? -dz - 1 - kt : dz - 1 - kt;
        const int kk = kk_index(kt, ks);
        if (cheb < 2 || kk < 0) continue;
        cr[((a - 1) * NKT + kt) * NOFF + o] = rho_index(dx, dy) * NKK + kk;
      }
    const double ph = (dx == 0 && dy == 0) ? 0.0 : atan2(-(double)dy, -(double)dx);
    for (int m = 0; m <= PMAX; ++m) {
      rot[(o * (PMAX + 1) + m) * 2] = cos(m * ph);
      rot[(o * (PMAX + 1) + m) * 2 + 1] = sin(m * ph);
    }
  }
  for (int dir = 0; dir < 4; ++dir) {
    const int bx = dir >> 1, by = dir & 1;
    const double ph = atan2(2.0 * by - 1.0, 2.0 * bx - 1.0);
    for (int m = 0; m <= PMAX; ++m) {
      rot4[(dir * (PMAX + 1) + m) * 2] = cos(m * ph);
      rot4[(dir * (PMAX + 1) + m) * 2 + 1] = sin(m * ph);
    }
  }
  int32_t *dcf, *dcr;
  LPB_CUDA(cudaMalloc(&dcf, sizeof(int32_t) * NOFF));
  LPB_CUDA(cudaMalloc(&dcr, sizeof(int32_t) * 2 * NKT * NOFF));
  LPB_CUDA(cudaMemcpy(dcf, cf.data(), sizeof(int32_t) * NOFF, cudaMemcpyHostToDevice));
  LPB_CUDA(cudaMemcpy(dcr, cr.data(), sizeof(int32_t) * 2 * NKT * NOFF, cudaMemcpyHostToDevice));
  std::vector<float> rotf(rot.begin(), rot.end()), rot4f(rot4.begin(), rot4.end());
  void *rd, *r4d, *rf, *r4f;
  LPB_CUDA(cudaMalloc(&rd, sizeof(double) * rot.size()));
  LPB_CUDA(cudaMalloc(&r4d, sizeof(double) * rot4.size()));
  LPB_CUDA(cudaMalloc(&rf, sizeof(float) * rot.size()));
  LPB_CUDA(cudaMalloc(&r4f, sizeof(float) * rot4.size()));
  LPB_CUDA(cudaMemcpy(rd, rot.data(), sizeof(double) * rot.size(), cudaMemcpyHostToDevice));
  LPB_CUDA(cudaMemcpy(r4d, rot4.data(), sizeof(double) * rot4.size(), cudaMemcpyHostToDevice));
  LPB_CUDA(cudaMemcpy(rf, rotf.data(), sizeof(float) * rotf.size(), cudaMemcpyHostToDevice));
  LPB_CUDA(cudaMemcpy(r4f, rot4f.data(), sizeof(float) * rot4f.size(), cudaMemcpyHostToDevice));
  g_tab_d[c.device] = Tables{dcf, dcr, rd, r4d};
  g_tab_f[c.device] = Tables{dcf, dcr, rf, r4f};
  mark_done_on_device(g_tab_ready);
}

void upload_gl16();
void upload_an();
void make_rotcol(Ctx &c);
void init_fmm_tables(Ctx &c) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  upload_gl16();
  upload_an();
  make_tables(c);
  upload_consts(c.stream);
  make_rotcol(c);
}

template <typename T, int PT>
static void launch_p2m(Ctx &c, const uint32_t *d_nseg, int64_t nseg_cap, const uint32_t *sst, const uint32_t *scnt,
                       const uint32_t *sbox, const uint32_t *styp, int ntypes, const uint64_t *bkey,
                       const PointSet &P, Geo geo, const LamTab &lt, void *M) {
  typedef typename C2<T>::t T2;
  k_p2m<T, PT><<<(unsigned)((nseg_cap + 3) / 4), 128, 0, c.stream>>>(d_nseg, sst, scnt, sbox, styp, ntypes, bkey,
                                                                      P.x, P.y, P.z, P.q, geo, lt, c.p, c.K,
                                                                      (T2 *)M);
  LPB_LAUNCH();
  c.launches++;
}
template <typename T, int PT>
static void launch_l2p(Ctx &c, const Level &Lv, int64_t nb, const PointSet &P, Geo geo, double lam, const void *L,
                       double *phi, double *field) {
  typedef typename C2<T>::t T2;
  k_l2p<T, PT><<<(unsigned)((nb + 3) / 4), 128, 0, c.stream>>>(Lv.d_n, Lv.key, Lv.start, Lv.count, P.x, P.y, P.z,
                                                                P.src, geo, lam, c.p, c.K, (const T2 *)L, phi, field);
  LPB_LAUNCH();
  c.launches++;
}

// ---------------------------------------------------------------------------------------
// M2L on the tensor cores (tcgen05, TF32 with a three-product split), free space and reaction.
//
// Every translation of this library has the azimuth-factored form
//     X = e^{i mu phi} M,   Y_nm = sum P_{nm,nu mu} Re X_{nu mu} + i sum Q_{nm,nu mu} Im X_{nu mu},
//     L_nm += e^{-i m phi} Y_nm
// with real class operators P, Q that do not depend on the azimuth phi of the offset.  In real
// form (R = 2K - (p+1) coordinates: for m > 0 the pair (Re, Im) in adjacent columns, then the
// real parts of the m = 0 coefficients; the m = 0 imaginary parts vanish for real charges) the
// middle step is one real matrix W_c (P between real parts, Q between imaginary parts) per
// class c and source type.  A CTA owns 128 target boxes (an octant tile, or a run of a target
// list) and one dx-slice of the offsets.  For every (offset, source type) step it copies the
// unrotated source rows and W_c into shared memory with cp.async; before the MMAs each thread
// rotates its own row in place and splits it into TF32 hi + lo (the rotation couples only the
// adjacent Re, Im columns of one coefficient); it accumulates D = X W_c^T in a fresh TMEM accumulator
// as hi*hi + hi*lo + lo*hi, and folds D into FP32 registers after the rotation e^{-i m phi}:
// the tensor core's accumulation loses precision over long chains (measured), a dot product of
// 32 NC terms per step does not.
// ---------------------------------------------------------------------------------------
// real coordinate c -> half-representation index: >= 0 real part, <= -2 imaginary part of
// index (-code - 2), -1 padding
__host__ __device__ __forceinline__ int tc_remap(int c, int K, int p) {
  const int NI = K - (p + 1);  // coefficients with m > 0
  if (c < 2 * NI) {
    const int j = c >> 1;
    int n = 1;
    while ((n + 1) * n / 2 <= j) ++n;  // entries with m > 0 below degree n: n(n-1)/2
    const int h = n * (n + 1) / 2 + (j - n * (n - 1) / 2 + 1);
    return (c & 1) ? -h - 2 : h;
  }
  const int n = c - 2 * NI;
  return n <= p ? n * (n + 1) / 2 : -1;
}

// (cos m phi, sin m phi) of every far offset's azimuth phi for each real coordinate pair of the
// tensor-core layout: entry [o][c], [o][c + 1] for the (Re, Im) columns c, c + 1 of a coefficient
// of order m; (1, 0) for the columns of m = 0 real parts and padding, which no rotation changes.
// Per context (the layout depends on p); built once in lpbfmm_create.
void make_rotcol(Ctx &c) {
  const int R = 2 * c.K - (c.p + 1), NC = (R + 31) / 32, N = 32 * NC;
  if (NC > 4) return;  // only the tensor-core path (p <= 10) uses it
  const int NI2 = 2 * (c.K - (c.p + 1));
  std::vector<float> t((size_t)NOFF * N);
  for (int o = 0; o < NOFF; ++o) {
    int dx, dy, dz;
    off_decode(o, dx, dy, dz);
    const double ph = (dx == 0 && dy == 0) ? 0.0 : atan2(-(double)dy, -(double)dx);
    for (int col = 0; col < N; col += 2) {
      double cs = 1.0, sn = 0.0;
      if (col < NI2) {
        const int h = tc_remap(col, c.K, c.p);  // real part of half index h
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= h) ++n;
        const int m = h - n * (n + 1) / 2;
        cs = cos(m * ph);
        sn = sin(m * ph);
      }
      t[(size_t)o * N + col] = (float)cs;
      t[(size_t)o * N + col + 1] = (float)sn;
    }
  }
  LPB_CUDA(cudaMalloc(&c.rotcol, sizeof(float) * t.size()));
  LPB_CUDA(cudaMemcpy(c.rotcol, t.data(), sizeof(float) * t.size(), cudaMemcpyHostToDevice));
}

// W_c of every class and source type as the shared-memory image the MMA reads: per (class, type)
// a block of NC K-chunks, each [hi: ldr rows x 128 bytes][lo: ldr rows x 128 bytes] in the
// 128-byte swizzled K-major layout (tc::swz), so that one bulk copy moves a class's operator into
// shared memory.  Classes that used[] marks absent at this level are skipped.
__global__ void k_tc_pack_w(const float *ops, int ncls_types, int ntypes, const uint8_t *used, int K, int p, int ldr,
                            float *wimg) {
  __shared__ int code[256];
  const int ct = blockIdx.x;
  if (ct >= ncls_types || (used && !used[ct / ntypes])) return;
  for (int c = threadIdx.x; c < ldr; c += blockDim.x) code[c] = tc_remap(c, K, p);
  __syncthreads();
  const size_t KK = (size_t)K * K;
  const float *P = ops + (size_t)ct * 2 * KK, *Q = P + KK;
  const int total = ldr * ldr;
  unsigned char *blk = (unsigned char *)(wimg + (size_t)ct * 2 * ldr * ldr);
  const size_t tile = (size_t)ldr * 128;  // bytes of one hi (or lo) chunk tile
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < total; e += gridDim.y * blockDim.x) {
    const int r = e / ldr, k = e % ldr;
    const int ro = code[r], ko = code[k];
    float w = 0.f;
    if (ro >= 0 && ko >= 0) w = P[(size_t)ro * K + ko];
    else if (ro <= -2 && ko <= -2) w = Q[(size_t)(-ro - 2) * K + (-ko - 2)];
    const float h = tc::to_tf32(w);
    unsigned char *ch = blk + (size_t)(k >> 5) * 2 * tile;
    *(float *)(ch + tc::swz(r, k & 31)) = h;
    *(float *)(ch + tile + tc::swz(r, k & 31)) = tc::to_tf32(w - h);
  }
}

// unrotated source rows in real-coordinate order (FP32), ldr = 32 NC floats per (box, type); with
// tmask, bit tau of tmask[box] is set when the row of source type tau has a nonzero entry (a zero
// row adds nothing, so the M2L may skip that type for that box)
__global__ void k_tc_pack_raw(const float2 *M, int64_t nrows, int K, int p, int ldr, float *raw, int ntypes,
                              uint32_t *tmask) {
  const int64_t total = nrows * ldr;  // a multiple of 32: every warp is full and within one row
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e / ldr;
    const int code = tc_remap((int)(e % ldr), K, p);
    const float v = code >= 0 ? M[b * K + code].x : (code <= -2 ? M[b * K + (-code - 2)].y : 0.f);
    raw[e] = v;
    if (tmask) {
      const unsigned nz = __ballot_sync(0xffffffffu, v != 0.f);
      if ((threadIdx.x & 31) == 0 && nz) atomicOr(&tmask[b / ntypes], 1u << (int)(b % ntypes));
    }
  }
}

constexpr int TC_MAXSTEP = SLICE_OFFS * 2 * (MAXLAYER - 1);

constexpr int TC_ROWS = 128, TC_WORKERS = 256, TC_THREADS = TC_WORKERS + 32;
constexpr int TC_WAIT = 1 << 22;  // mbarrier polls before the kernel reports a timeout

__host__ __device__ constexpr int tc_nst(int NC) { return NC <= 5 ? 3 : 2; }
__host__ __device__ constexpr size_t tc_stage_bytes(int NC) { return (size_t)2 * (TC_ROWS + 32 * NC) * 128; }
static size_t tc_smem(int NC) { return tc_nst(NC) * tc_stage_bytes(NC) + 1024; }

__device__ __forceinline__ uint64_t to_global(const void *p) {
  uint64_t g;
  asm("cvta.to.global.u64 %0, %1;" : "=l"(g) : "l"(p));
  return g;
}
// one arrival that also announces tx bytes to come by bulk copies
__device__ __forceinline__ void mbar_expect_tx(uint64_t *mbar, uint32_t bytes) {
  asm volatile("{\n.reg .b64 st;\nmbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n" ::"r"(
                   tc::smem_u32(mbar)),
               "r"(bytes)
               : "memory");
}
// bulk copy of bytes (multiple of 16, both addresses 16-byte aligned) global -> shared, completing
// on mbar
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   tc::smem_u32(dst)),
               "l"(to_global(src)), "r"(bytes), "r"(tc::smem_u32(mbar))
               : "memory");
}

// x rounded to TF32 (10 stored significand bits), to nearest with ties away from zero, in integer
// arithmetic on the FP32 bits: the rounding of cvt.rna.tf32.f32 for the finite values here, on
// the integer pipes (the split of every staged source row runs once per step)
__device__ __forceinline__ float tf32i(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xffffe000u);
}
template <int NC>
__global__ void __launch_bounds__(TC_THREADS, 1) k_m2l_tc(const TJob *jobs, int njobs, int K, int p, int *status) {
  constexpr int N = 32 * NC, NST = tc_nst(NC);
  constexpr int TCOLS = 2 * N <= 32 ? 32 : (2 * N <= 64 ? 64 : (2 * N <= 128 ? 128 : 256));
  static_assert(2 * N <= 256, "two accumulators of N columns");
  constexpr size_t SA = (size_t)TC_ROWS * 128, SB = (size_t)N * 128;  // bytes of one A / B chunk tile
  extern __shared__ __align__(16) unsigned char tcsm[];  // base rounded up to 1024 below
  unsigned char *sbase = (unsigned char *)(((uintptr_t)tcsm + 1023) & ~(uintptr_t)1023);
  __shared__ int tid_[TC_ROWS];
  __shared__ int steps[TC_MAXSTEP];  // (offset << 4) | source type
  __shared__ int remap_s[N], mcol[N];  // coordinate -> half index code; m of that coefficient
  __shared__ int nsteps;
  __shared__ unsigned tmk[SLICE_OFFS];  // per offset of the slice: the source types some row needs
  // the rotation columns depend on the offset's azimuth only, i.e. on (dx, dy): a dx-slice needs
  // OFF_D rows of the table, kept here for the whole CTA
  __shared__ __align__(16) float rot_s[OFF_D * 128];
  // full[b]: the workers have staged buffer b (TC_WORKERS arrivals); empty[b]: its MMAs are done;
  // accbar[a]: a step's MMAs into accumulator a are done; foldbar[a]: the workers have read it
  // wfull[b]: the operator chunk of buffer b has landed (one bulk copy, issued by thread 0)
  __shared__ uint64_t full[NST], empty[NST], accbar[2], foldbar[2], wfull[NST];
  __shared__ uint32_t tbase;
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (jobs[mid].item0 <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const TJob &J = jobs[lo];
  // the fields the pipeline reads, in registers: the inline-assembly memory clobbers of the
  // barrier and copy instructions would otherwise make the compiler reload them from global
  // memory after every one
  const float *const Jraw = J.raw, *const Jwimg = J.wimg, *const Jrotcol = J.rotcol;
  const int32_t *const Jvlist = J.vlist, *const Jcls = J.cls_of;
  const int64_t local = (int64_t)blockIdx.x - J.item0;
  // slice-major: the CTAs resident at one time share a dx-slice, hence the operator classes of
  // its offsets, which then stay in L2 (a level's reaction operators alone exceed it)
  const int64_t ntiles = J.pstart ? 8 * ((J.npar + TC_ROWS - 1) / TC_ROWS) : (J.ntb + TC_ROWS - 1) / TC_ROWS;
  const int slice = (int)(local / ntiles);
  const int64_t ti = local % ntiles;
  const int64_t ntl = J.tlist ? (int64_t)*J.d_ntl : J.ntb;
  if (J.pstart ? (ti >> 3) * TC_ROWS >= J.npar : ti * TC_ROWS >= ntl) return;
  // worker thread (tid < TC_WORKERS) = (row, half): row = target slot and TMEM lane, half = which
  // 4 of a chunk's 8 units and which half of the accumulator columns it handles; the last warp
  // issues the MMAs (lane 0)
  const int tid = threadIdx.x, warp = tid >> 5, row = tid & (TC_ROWS - 1), hf = (tid >> 7) & 1;
  const bool worker = tid < TC_WORKERS;
  const int ntypes = J.ntypes;
  for (int c = tid; c < N; c += TC_THREADS) {
    const int code = tc_remap(c, K, p);
    remap_s[c] = code;
    mcol[c] = code == -1 ? 0 : cK.mof[code >= 0 ? code : -code - 2];
  }
  if (tid < TC_ROWS) {
    int t = -1;
    if (J.tlist) {
      const int64_t j = ti * TC_ROWS + tid;
      if (j < ntl) t = J.tlist[j];
    } else if (J.pstart) {
      const int oct = (int)(ti & 7);
      const int64_t P = (ti >> 3) * TC_ROWS + tid;
      if (P < J.npar) {
        const uint32_t s0 = J.pstart[P], n = J.pcount[P];
        for (uint32_t k = 0; k < n; ++k)
          if ((int)(J.ckey[s0 + k] & 7ull) == oct) t = (int)(s0 + k);
      }
    } else {
      const int64_t j = ti * TC_ROWS + tid;
      if (j < J.ntb) t = (int)j;
    }
    tid_[tid] = t;
  }
  for (int k = tid; k < SLICE_OFFS; k += TC_THREADS) tmk[k] = 0u;
  __syncthreads();
  if (tid < TC_ROWS) {
    const int t = tid_[tid];
    if (t >= 0)
      for (int k = 0; k < SLICE_OFFS; ++k) {
        const int o = slice * SLICE_OFFS + k;
        const int sb = J.cls_of[o] >= 0 ? J.vlist[(size_t)t * NOFF + o] : -1;
        if (sb >= 0) atomicOr(&tmk[k], J.tmask ? J.tmask[sb] : 0xffffffffu);
      }
  }
  __syncthreads();
  if (tid == 0) {
    int n = 0;
    for (int k = 0; k < SLICE_OFFS; ++k)
      for (int tau = 0; tau < ntypes; ++tau)
        if ((tmk[k] >> tau) & 1u) steps[n++] = ((slice * SLICE_OFFS + k) << 4) | tau;
    nsteps = n;
  }
  __syncthreads();
  const int ns = nsteps;
  if (ns == 0) return;
  if (warp == 0) tc::tmem_alloc(&tbase, TCOLS);
  if (tid == 0) {
    for (int b = 0; b < NST; ++b) {
      tc::mbar_init(&full[b], TC_WORKERS);
      tc::mbar_init(&empty[b], 1);
      tc::mbar_init(&wfull[b], 1);
    }
    for (int a = 0; a < 2; ++a) {
      tc::mbar_init(&accbar[a], 1);
      tc::mbar_init(&foldbar[a], TC_WORKERS);
    }
    tc::mbar_fence_init();
  }
  for (int e = tid; e < OFF_D * N; e += TC_THREADS) {
    const int dyi = e / N;
    rot_s[e] = Jrotcol[(size_t)off_index(slice - OFF_R, dyi - OFF_R, 0) * N + (e - dyi * N)];
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  // a warp reads the TMEM lanes of its quarter, 32 (warp % 4) .. + 31
  const uint32_t tmem = tbase, lanebase = (uint32_t)((warp & 3) * 32) << 16;
  const int S = ns * NC;  // stages: (step, K-chunk)
  const int myt = worker ? tid_[row] : -1;
  constexpr uint32_t IDESC = tc::idesc_tf32(TC_ROWS, N);
  constexpr int NH = N / 2;  // accumulator columns per thread
  float racc[NH];
#pragma unroll
  for (int j = 0; j < NH; ++j) racc[j] = 0.f;
  // fold the accumulator of step i into racc after the output rotation e^{-i m phi}
  auto fold = [&](int i) -> bool {
    const bool ok = tc::mbar_wait(&accbar[i & 1], (uint32_t)((i >> 1) & 1), TC_WAIT);
    if (ok) {
      tc::fence_after();
      const float4 *rr = (const float4 *)(rot_s + ((steps[i] >> 4) / OFF_D % OFF_D) * N + hf * NH);
      const uint32_t col = (uint32_t)((i & 1) * N + hf * NH);
#pragma unroll
      for (int c1 = 0; c1 < NH; c1 += 32) {
        uint32_t v[4][8];
#pragma unroll
        for (int q = 0; q < 4; ++q) tc::tmem_ld8_nw(tmem + lanebase + col + (uint32_t)(c1 + 8 * q), v[q]);
        tc::tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int c0 = c1 + 8 * q;
          const float4 ra = rr[c0 / 4], rb = rr[c0 / 4 + 1];
          const float cs[4] = {ra.x, ra.z, rb.x, rb.z}, sn[4] = {ra.y, ra.w, rb.y, rb.w};
#pragma unroll
          for (int j = 0; j < 8; j += 2) {
            const float vr = __uint_as_float(v[q][j]), vi = __uint_as_float(v[q][j + 1]);
            racc[c0 + j] += cs[j / 2] * vr + sn[j / 2] * vi;
            racc[c0 + j + 1] += cs[j / 2] * vi - sn[j / 2] * vr;
          }
        }
      }
      tc::fence_before();
    }
    return ok;
  };
  bool fail = false;
  int wl_last = -1;  // last stage whose operator chunk thread 0 requested
  if (worker) {
    int cur_o = -1, my_src = -1;
    // stage s is copied at iteration s and rotated / split at iteration s + 1; the MMA thread takes
    // it from there, so a buffer is refilled NST stages later, once its MMAs are done
    for (int s = 0; s < S + 1; ++s) {
      if (s < S) {
        const int b = s % NST;
        if (s >= NST && !tc::mbar_wait(&empty[b], (uint32_t)((s / NST - 1) & 1), TC_WAIT)) {
          fail = true;
          break;
        }
        const int o = steps[s / NC] >> 4, tau = steps[s / NC] & 15, kc = s % NC;
        if (o != cur_o) {
          cur_o = o;
          my_src = myt >= 0 ? Jvlist[(size_t)myt * NOFF + o] : -1;
        }
        unsigned char *st = sbase + (size_t)b * tc_stage_bytes(NC);
        unsigned char *Ah = st, *Bh = st + 2 * SA;
        if (tid == 0) {
          // the class operator's K-chunk (hi and lo tiles, one contiguous image) by one bulk copy
          const size_t ct = (size_t)Jcls[o] * ntypes + tau;
          const unsigned char *src = (const unsigned char *)(Jwimg + ct * 2 * N * N) + (size_t)kc * 2 * SB;
          mbar_expect_tx(&wfull[b], (uint32_t)(2 * SB));
          bulk_g2s(Bh, src, (uint32_t)(2 * SB), &wfull[b]);
          wl_last = s;
        }
        {
          // this thread's source row chunk, unrotated, into the A-hi slots (rotated next iteration)
          const bool v = my_src >= 0;
          const float *g = Jraw + ((size_t)(v ? my_src : 0) * ntypes + tau) * N + kc * 32;
#pragma unroll
          for (int u = hf * 4; u < hf * 4 + 4; ++u) cp_async16(Ah + tc::swz16(row, u), g + 4 * u, v);
        }
      }
      cp_commit();
      const int sc = s - 1;
      if (sc < 0) continue;
      asm volatile("cp.async.wait_group 1;\n" ::);
      const int si = sc / NC, kc = sc % NC;
      {
        // rotate this thread's half row by e^{i mu phi} and split it into TF32 hi (in place) + lo
        unsigned char *st = sbase + (size_t)(sc % NST) * tc_stage_bytes(NC);
        unsigned char *Ah = st, *Al = st + SA;
        const float4 *rr = (const float4 *)(rot_s + ((steps[si] >> 4) / OFF_D % OFF_D) * N + kc * 32);
#pragma unroll
        for (int uu = 0; uu < 4; ++uu) {
          const int u = hf * 4 + uu;
          float4 x = *(float4 *)(Ah + tc::swz16(row, u));
          const float4 r = rr[u];  // (cos, sin) of the unit's two column pairs
          const float xr0 = r.x * x.x - r.y * x.y, xi0 = r.y * x.x + r.x * x.y;
          const float xr1 = r.z * x.z - r.w * x.w, xi1 = r.w * x.z + r.z * x.w;
          x = make_float4(xr0, xi0, xr1, xi1);
          float4 h4v, l4v;
          h4v.x = tf32i(x.x);
          h4v.y = tf32i(x.y);
          h4v.z = tf32i(x.z);
          h4v.w = tf32i(x.w);
          l4v.x = tf32i(x.x - h4v.x);
          l4v.y = tf32i(x.y - h4v.y);
          l4v.z = tf32i(x.z - h4v.z);
          l4v.w = tf32i(x.w - h4v.w);
          *(float4 *)(Ah + tc::swz16(row, u)) = h4v;
          *(float4 *)(Al + tc::swz16(row, u)) = l4v;
        }
      }
      // this thread's copies (B part, its A row) and its stores are in place: hand over to the tensor core
      tc::fence_async_smem();
      tc::mbar_arrive(&full[sc % NST]);
      // step si is handed over in full: fold step si - 1 (its accumulator is reused by step si + 1)
      if (kc == NC - 1 && si >= 1) {
        if (!fold(si - 1)) {
          fail = true;
          break;
        }
        tc::mbar_arrive(&foldbar[(si - 1) & 1]);
      }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
    // no bulk copy may still be writing this CTA's shared memory when it exits
    if (tid == 0 && fail && wl_last >= 0)
      tc::mbar_wait(&wfull[wl_last % NST], (uint32_t)((wl_last / NST) & 1), TC_WAIT);
    if (!fail && !fold(ns - 1)) fail = true;
    if (!fail) {
      const int t = tid_[row];
      if (t >= 0) {
        float2 *Lrow = J.L + ((size_t)t * M2L_NSLOT + J.slot0 + slice) * K;
#pragma unroll
        for (int j = 0; j < NH; ++j) {
          const int code = remap_s[hf * NH + j];
          if (code >= 0) {
            Lrow[code].x = racc[j];
            if (mcol[hf * NH + j] == 0) Lrow[code].y = 0.f;
          } else if (code <= -2) {
            Lrow[-code - 2].y = racc[j];
          }
        }
      }
    }
  } else if (tid == TC_WORKERS) {
    // the MMA thread: stage after stage, once the workers have staged it; a step's first chunk
    // waits until the workers have read the accumulator two steps back
    int last = -1;
    for (int sc = 0; sc < S; ++sc) {
      const int b = sc % NST, si = sc / NC, kc = sc % NC;
      if (!tc::mbar_wait(&full[b], (uint32_t)((sc / NST) & 1), TC_WAIT) ||
          !tc::mbar_wait(&wfull[b], (uint32_t)((sc / NST) & 1), TC_WAIT)) {
        fail = true;
        break;
      }
      if (kc == 0 && si >= 2 && !tc::mbar_wait(&foldbar[si & 1], (uint32_t)(((si - 2) >> 1) & 1), TC_WAIT)) {
        fail = true;
        break;
      }
      tc::fence_after();
      unsigned char *st = sbase + (size_t)b * tc_stage_bytes(NC);
      const uint32_t ah = tc::smem_u32(st), al = ah + (uint32_t)SA, bh = ah + 2 * (uint32_t)SA,
                     bl = bh + (uint32_t)SB;
      const uint32_t dacc = tmem + (uint32_t)((si & 1) * N);
#pragma unroll
      for (int kk = 0; kk < 4; ++kk) {
        const uint32_t off = kk * 32;
        tc::mma_tf32(dacc, tc::sdesc(ah + off), tc::sdesc(bh + off), IDESC, (kc | kk) ? 1u : 0u);
        tc::mma_tf32(dacc, tc::sdesc(ah + off), tc::sdesc(bl + off), IDESC, 1u);
        tc::mma_tf32(dacc, tc::sdesc(al + off), tc::sdesc(bh + off), IDESC, 1u);
      }
      tc::commit(&empty[b]);
      if (kc == NC - 1) tc::commit(&accbar[si & 1]);
      last = sc;
    }
    // every MMA has completed once the last committed stage's barrier phase completes
    if (last >= 0) tc::mbar_wait(&empty[last % NST], (uint32_t)((last / NST) & 1), TC_WAIT);
  }
  if (fail) atomicExch(status, LPBFMM_ERR_TIMEOUT);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, TCOLS);
}

template <typename T, int TPT, int NR>
static void launch_m2l_t(Ctx &c, const std::vector<XJob> &jobs, int64_t items) {
  constexpr int TT = 16 * TPT, KR = 16 * NR;
  const size_t smem = sizeof(T) * (2 * KR * M2L_KC + 2 * M2L_KC * TT) + sizeof(int) * 2 * TT;
  LPB_ATTR_ONCE((k_m2l<T, TPT, NR>), smem);
  XJob *dj = c.arena.get<XJob>(jobs.size());
  LPB_CUDA(cudaMemcpyAsync(dj, jobs.data(), sizeof(XJob) * jobs.size(), cudaMemcpyHostToDevice, c.stream));
  const Tables &tb = sizeof(T) == 8 ? g_tab_d[c.device] : g_tab_f[c.device];
  k_m2l<T, TPT, NR><<<(unsigned)items, 256, smem, c.stream>>>(dj, (int)jobs.size(), (const T *)tb.rot, c.K);
  LPB_LAUNCH();
  c.launches++;
}

#define PT_DISPATCH(F, ...)                                   \
  do {                                                        \
    if (c.p <= 5) F<T, 5>(__VA_ARGS__);                       \
    else if (c.p <= 8) F<T, 8>(__VA_ARGS__);                  \
    else if (c.p <= 10) F<T, 10>(__VA_ARGS__);                \
    else if (c.p <= 12) F<T, 12>(__VA_ARGS__);                \
    else F<T, 16>(__VA_ARGS__);                               \
  } while (0)

template <typename T>
static Geo geo_at(const Group &g, int l) {
  Geo G;
  G.o[0] = g.root[0] - g.root[3];
  G.o[1] = g.root[1] - g.root[3];
  G.o[2] = g.root[2] - g.root[3];
  G.h = g.h(l);
  return G;
}

// P2M and M2M of one group; local expansions of every level zeroed
template <typename T>
static void upward_t(Ctx &c, Group &g, int parts) {
  typedef typename C2<T>::t T2;
  const int K = c.K, D = g.D, Df = g.Df;
  const Tables &tb = sizeof(T) == 8 ? g_tab_d[c.device] : g_tab_f[c.device];
  const bool dofree = g.is_free && (parts & 1);
  const bool doreact = (parts & 2) && g.I.np > 0;
  LamTab lt_t, lt_i;
  for (int k = 0; k < 2 * MAXLAYER; ++k) lt_t.v[k] = lt_i.v[k] = c.md.lam[g.l];
  for (int t = 0; t < g.ntypes; ++t) {
    int lp, b;
    type_decode(t, lp, b);
    lt_i.v[t] = c.md.lam[lp];
  }
  for (int l = 2; l <= D; ++l) {
    const int64_t ntb = g.T.lev[l].n, nib = g.I.lev[l].n;
    g.Lt[l] = c.arena.get<T2>(ntb * K);
    LPB_CUDA(cudaMemsetAsync(g.Lt[l], 0, sizeof(T2) * ntb * K, c.stream));
    if (dofree && l <= Df) g.Mfree[l] = c.arena.get<T2>(ntb * K);
    if (doreact) g.Mimg[l] = c.arena.get<T2>(nib * g.ntypes * K);
  }
  // free-space P2M at the free-space leaves (level Df; their point ranges)
  if (dofree)
    PT_DISPATCH(launch_p2m, c, g.T.lev[Df].d_n, g.T.lev[Df].n, g.T.lev[Df].pstart, g.T.lev[Df].pcount, nullptr,
                nullptr, 1, g.T.lev[Df].key, g.T, geo_at<T>(g, Df), lt_t, g.Mfree[Df]);
  if (doreact) {
    LPB_CUDA(cudaMemsetAsync(g.Mimg[D], 0, sizeof(T2) * g.I.lev[D].n * g.ntypes * K, c.stream));
    PT_DISPATCH(launch_p2m, c, g.I.d_nseg, g.I.nseg, g.I.seg_start, g.I.seg_count, g.I.seg_box, g.I.seg_type,
                g.ntypes, g.I.lev[D].key, g.I, geo_at<T>(g, D), lt_i, g.Mimg[D]);
  }
  for (int l = D; l >= 3; --l) {
    if (dofree && l <= Df && g.T.lev[l - 1].n) {
      k_m2m<T><<<dim3((unsigned)g.T.lev[l - 1].n, 1), M2M_THREADS, 0, c.stream>>>(
          g.T.lev[l - 1].d_n, g.T.lev[l - 1].start, g.T.lev[l - 1].count, g.T.lev[l].key, 1, (const T2 *)g.Mfree[l],
          (T2 *)g.Mfree[l - 1], (const T *)g.op_m2m_t[l], (const T *)tb.rot4, K);
      LPB_LAUNCH();
      c.launches++;
    }
    if (doreact && g.I.lev[l - 1].n) {
      k_m2m<T><<<dim3((unsigned)g.I.lev[l - 1].n, g.ntypes), M2M_THREADS, 0, c.stream>>>(
          g.I.lev[l - 1].d_n, g.I.lev[l - 1].start, g.I.lev[l - 1].count, g.I.lev[l].key, g.ntypes,
          (const T2 *)g.Mimg[l], (T2 *)g.Mimg[l - 1], (const T *)g.op_m2m_i[l], (const T *)tb.rot4, K);
      LPB_LAUNCH();
      c.launches++;
    }
  }
}

// every multipole-to-local translation of every group and level in one launch
template <typename T>
static void m2l_all_t(Ctx &c, std::vector<Group> &groups) {
  constexpr int TPT = sizeof(T) == 4 ? 4 : 2;
  constexpr int TT = 16 * TPT;
  const Tables &tb = sizeof(T) == 8 ? g_tab_d[c.device] : g_tab_f[c.device];
  std::vector<XJob> jobs;
  int64_t items = 0;
  typedef typename C2<T>::t T2;
  std::vector<RJob> rjobs;
  int64_t relem = 0;
  // tensor-core free-space path: mixed precision, 2K - (p+1) <= 128 real coordinates
  const int tc_nc = (2 * c.K - (c.p + 1) + 31) / 32;
  const bool use_tc = sizeof(T) == 4 && tc_nc <= 4;  // p <= 10
  std::vector<TJob> tjobs;
  int64_t titems = 0;
  auto add = [&](const int32_t *tlist, const uint32_t *d_ntl, int64_t ntb, const int32_t *vlist,
                 const int32_t *cls_of, const void *M, const void *ops, void *part, int ntypes, int slot0,
                 const Level *par, const Level *lev) {
    XJob j;
    j.tlist = tlist; j.d_ntl = d_ntl; j.ntb = ntb; j.vlist = vlist; j.cls_of = cls_of;
    j.M = M; j.ops = ops; j.L = part; j.ntypes = ntypes; j.slot0 = slot0; j.item0 = items;
    j.pstart = par ? par->start : nullptr;
    j.pcount = par ? par->count : nullptr;
    j.ckey = par ? lev->key : nullptr;
    j.npar = par ? par->n : 0;
    jobs.push_back(j);
    items += m2l_tiles(j, TT) * M2L_NSLICE;
  };
  for (auto &g : groups) {
    const int parts = g.parts;
    const bool react_far = (parts & 2) && g.I.np > 0 && !(parts & 8);
    for (int l = 2; l <= g.D; ++l) {
      const bool dofree = g.is_free && (parts & 1) && l <= g.Df;
      const int64_t ntb = g.T.lev[l].n;
      if (!ntb || !(dofree || (react_far && g.vreact[l]))) continue;
      T2 *part = c.arena.get<T2>((size_t)ntb * M2L_NSLOT * c.K);
      LPB_CUDA(cudaMemsetAsync(part, 0, sizeof(T2) * ntb * M2L_NSLOT * c.K, c.stream));
      RJob r;
      r.part = part; r.L = g.Lt[l]; r.n = ntb * c.K; r.e0 = relem;
      rjobs.push_back(r);
      relem += r.n;
      if (dofree && use_tc) {
        // tensor-core path: the level's class operators as TF32 hi/lo real matrices
        const int N = 32 * tc_nc;
        float *wimg = c.arena.get<float>((size_t)NFREE_CLS * 2 * N * N);
        k_tc_pack_w<<<dim3(NFREE_CLS, 4), 256, 0, c.stream>>>((const float *)g.op_free[l], NFREE_CLS, 1, nullptr,
                                                               c.K, c.p, N, wimg);
        LPB_LAUNCH();
        c.launches++;
        float *raw = c.arena.get<float>((size_t)ntb * N);
        k_tc_pack_raw<<<(unsigned)std::min<int64_t>(4096, (ntb * N + 255) / 256), 256, 0, c.stream>>>(
            (const float2 *)g.Mfree[l], ntb, c.K, c.p, N, raw, 1, nullptr);
        LPB_LAUNCH();
        c.launches++;
        TJob j;
        j.raw = raw; j.wimg = wimg; j.rotcol = c.rotcol;
        j.vlist = g.vfree[l]; j.cls_of = tb.cls_free; j.tmask = nullptr; j.tlist = nullptr; j.d_ntl = nullptr;
        j.L = (float2 *)part; j.ntb = ntb; j.item0 = titems; j.slot0 = 0; j.ntypes = 1;
        const Level *par = l >= 3 ? &g.T.lev[l - 1] : nullptr;
        j.pstart = par ? par->start : nullptr;
        j.pcount = par ? par->count : nullptr;
        j.ckey = par ? g.T.lev[l].key : nullptr;
        j.npar = par ? par->n : 0;
        const int64_t tiles = par ? 8 * ((j.npar + TC_ROWS - 1) / TC_ROWS) : (ntb + TC_ROWS - 1) / TC_ROWS;
        titems += tiles * M2L_NSLICE;
        tjobs.push_back(j);
      } else if (dofree) {
        add(nullptr, nullptr, ntb, g.vfree[l], tb.cls_free, g.Mfree[l], g.op_free[l], part, 1, 0,
            l >= 3 ? &g.T.lev[l - 1] : nullptr, &g.T.lev[l]);
      }
      if (react_far && g.vreact[l] && use_tc && g.ntypes <= 16) {
        // tensor-core reaction path: class operators per (class, source type)
        const int N = 32 * tc_nc;
        const int nct = NREACT_CLS * g.ntypes;
        float *wimg = c.arena.get<float>((size_t)nct * 2 * N * N);
        k_tc_pack_w<<<dim3(nct, 4), 256, 0, c.stream>>>((const float *)g.op_react[l], nct, g.ntypes, g.used[l], c.K,
                                                        c.p, N, wimg);
        LPB_LAUNCH();
        c.launches++;
        const int64_t nir = g.I.lev[l].n * g.ntypes;
        float *raw = c.arena.get<float>((size_t)nir * N);
        uint32_t *tmask = c.arena.get<uint32_t>((size_t)g.I.lev[l].n);
        LPB_CUDA(cudaMemsetAsync(tmask, 0, sizeof(uint32_t) * g.I.lev[l].n, c.stream));
        k_tc_pack_raw<<<(unsigned)std::min<int64_t>(4096, (nir * N + 255) / 256), 256, 0, c.stream>>>(
            (const float2 *)g.Mimg[l], nir, c.K, c.p, N, raw, g.ntypes, tmask);
        LPB_LAUNCH();
        c.launches++;
        for (int kt = 0; kt < 2 * c.ws + 1; ++kt) {
          TJob j;
          j.raw = raw; j.wimg = wimg; j.rotcol = c.rotcol;
          j.vlist = g.vreact[l]; j.cls_of = tb.cls_react + ((g.a - 1) * NKT + kt) * NOFF; j.tmask = tmask;
          j.tlist = g.rows[l] + (size_t)kt * ntb; j.d_ntl = g.nrows[l] + kt;
          j.L = (float2 *)part; j.ntb = ntb; j.item0 = titems; j.slot0 = M2L_NSLICE; j.ntypes = g.ntypes;
          j.pstart = nullptr; j.pcount = nullptr; j.ckey = nullptr; j.npar = 0;
          titems += ((ntb + TC_ROWS - 1) / TC_ROWS) * M2L_NSLICE;
          tjobs.push_back(j);
        }
      } else if (react_far && g.vreact[l]) {
        for (int kt = 0; kt < 2 * c.ws + 1; ++kt)
          add(g.rows[l] + (size_t)kt * ntb, g.nrows[l] + kt, ntb, g.vreact[l],
              tb.cls_react + ((g.a - 1) * NKT + kt) * NOFF, g.Mimg[l], g.op_react[l], part, g.ntypes, M2L_NSLICE,
              nullptr, nullptr);
      }
    }
  }
  if (jobs.empty() && tjobs.empty()) return;
  prof_mark(c, "m2l_prep");
  if (c.def.on && !tjobs.empty() && jobs.empty()) {
    // batched evaluation: the tensor-core M2L and the slot sums join a grouped launch
    c.def.nc = tc_nc;
    c.def.tc = tjobs;
    c.def.tc_items = titems;
    c.def.red = rjobs;
    c.def.red_elems = relem;
    return;
  }
  if (!tjobs.empty()) {
    TJob *dj = c.arena.get<TJob>(tjobs.size());
    LPB_CUDA(cudaMemcpyAsync(dj, tjobs.data(), sizeof(TJob) * tjobs.size(), cudaMemcpyHostToDevice, c.stream));
    switch (tc_nc) {
#define LPB_TC_CASE(NCV)                                                                                     \
  case NCV: {                                                                                                \
    LPB_ATTR_ONCE(k_m2l_tc<NCV>, tc_smem(NCV));                                                              \
    k_m2l_tc<NCV><<<(unsigned)titems, TC_THREADS, tc_smem(NCV), c.stream>>>(dj, (int)tjobs.size(), c.K, c.p, c.status); \
    break;                                                                                                   \
  }
      LPB_TC_CASE(1) LPB_TC_CASE(2) LPB_TC_CASE(3) LPB_TC_CASE(4)
#undef LPB_TC_CASE
    }
    LPB_LAUNCH();
    c.launches++;
    prof_mark(c, "m2l_tc");
  }
  auto launch_reduce = [&]() {
    RJob *dr = c.arena.get<RJob>(rjobs.size());
    LPB_CUDA(cudaMemcpyAsync(dr, rjobs.data(), sizeof(RJob) * rjobs.size(), cudaMemcpyHostToDevice, c.stream));
    k_m2l_reduce<T><<<(unsigned)((relem + 255) / 256), 256, 0, c.stream>>>(dr, (int)rjobs.size(), c.K);
    LPB_LAUNCH();
    c.launches++;
  };
  if (jobs.empty()) {
    launch_reduce();
    return;
  }
  if (sizeof(T) == 4 && c.K <= F32_KR) {
    // re-count items with the larger tile of the asynchronous FP32 kernel
    int64_t it = 0;
    for (auto &j : jobs) {
      j.item0 = it;
      it += m2l_tiles(j, F32_TT) * M2L_NSLICE;
    }
    const size_t smem = m2l_f32_smem(c.K);
    LPB_ATTR_ONCE(k_m2l_f32, m2l_f32_smem(F32_KR));  // the largest K of this kernel
    XJob *dj = c.arena.get<XJob>(jobs.size());
    LPB_CUDA(cudaMemcpyAsync(dj, jobs.data(), sizeof(XJob) * jobs.size(), cudaMemcpyHostToDevice, c.stream));
    k_m2l_f32<<<(unsigned)it, 256, smem, c.stream>>>(dj, (int)jobs.size(), (const float *)tb.rot, c.K);
    LPB_LAUNCH();
    c.launches++;
    prof_mark(c, "m2l_simt");
    launch_reduce();
    return;
  }
  if (c.K <= 80) launch_m2l_t<T, TPT, 5>(c, jobs, items);
  else if (c.K <= 128) launch_m2l_t<T, TPT, 8>(c, jobs, items);
  else launch_m2l_t<T, TPT, 10>(c, jobs, items);
  launch_reduce();
}

// L2L (adding the parent's shifted expansion), L2P and the near fields of one group
template <typename T>
static void downward_t(Ctx &c, Group &g, int parts, double *phi, double *field) {
  typedef typename C2<T>::t T2;
  const int K = c.K, D = g.D;
  const Tables &tb = sizeof(T) == 8 ? g_tab_d[c.device] : g_tab_f[c.device];
  const bool dofree = g.is_free && (parts & 1);
  const bool doreact = (parts & 2) && g.I.np > 0;
  const bool react_near = doreact && !(parts & 4);
  for (int l = 3; l <= D; ++l) {
    const int64_t ntb = g.T.lev[l].n;
    if (!ntb) continue;
    k_l2l<T><<<(unsigned)ntb, 128, 0, c.stream>>>(g.T.lev[l].d_n, g.T.lev[l].parent, g.T.lev[l].key,
                                                  (const T2 *)g.Lt[l - 1], (T2 *)g.Lt[l], (const T *)g.op_l2l[l],
                                                  (const T *)tb.rot4, K);
    LPB_LAUNCH();
    c.launches++;
  }
  PT_DISPATCH(launch_l2p, c, g.T.lev[D], g.T.lev[D].n, g.T, geo_at<T>(g, D), c.md.lam[g.l], g.Lt[D], phi, field);
  if (dofree && sizeof(T) == 8) {
    // the FP64 free-space near field at the free-space leaves (level Df); the FP32 one runs in
    // run_near_free, beside the far field
    const Level &Lf = g.T.lev[g.Df];
    k_p2p_free<T><<<(unsigned)Lf.n, P2P_TPB, 0, c.stream>>>(
        Lf.d_n, Lf.key, Lf.pstart, Lf.pcount, g.ufree, g.T.x, g.T.y, g.T.z, g.T.q, g.T.src, geo_at<T>(g, g.Df),
        c.md.lam[g.l], 1.0 / (4.0 * PI * c.md.eps[g.l]), phi, field);
    LPB_LAUNCH();
    c.launches++;
  }
  if (react_near && g.ureact && g.nodes) {
    k_p2p_react<T><<<(unsigned)g.T.lev[D].n, P2P_THREADS, 0, c.stream>>>(
        g.T.lev[D].d_n, g.T.lev[D].key, g.T.lev[D].start, g.T.lev[D].count, g.ureact, g.T.x, g.T.y, g.T.z, g.T.src,
        g.I.lev[D].start, g.I.lev[D].count, g.I.x, g.I.y, g.I.z, g.I.q, g.I.key, geo_at<T>(g, D), g.dI,
        g.a == 1 ? 1.0 : -1.0, g.nodes, g.nq, phi, field);
    LPB_LAUNCH();
    c.launches++;
  }
}

// one launch of the FP32 free-space near field over the jobs (block0 renumbered from 0)
static void launch_p2p(Ctx &c, const std::vector<P2PJob> &jobs, int64_t blocks, cudaStream_t st) {
  if (jobs.empty() || blocks <= 0) return;
  P2PJob *dj = c.arena.get<P2PJob>(jobs.size());
  LPB_CUDA(cudaMemcpyAsync(dj, jobs.data(), sizeof(P2PJob) * jobs.size(), cudaMemcpyHostToDevice, st));
  k_p2p_free_f32<<<(unsigned)blocks, 32 * P2P_WARPS, 0, st>>>(dj, (int)jobs.size());
  LPB_LAUNCH();
  c.launches++;
}

void run_fmm_front(Ctx &c, std::vector<Group> &groups) {
  c.def.nc = 0;
  c.def.tc.clear();
  c.def.red.clear();
  c.def.tc_items = c.def.red_elems = 0;
  const bool d = c.opts.precision == LPBFMM_FP64;
  // the free-space operators (side stream) are complete before the upward pass
  if (c.ev_free) LPB_CUDA(cudaStreamWaitEvent(c.stream, c.ev_free, 0));
  for (auto &g : groups) d ? upward_t<double>(c, g, g.parts) : upward_t<float>(c, g, g.parts);
  prof_mark(c, "upward");
  // the reaction tables and operators (side stream) are complete before any M2L
  if (c.ev_join) LPB_CUDA(cudaStreamWaitEvent(c.stream, c.ev_join, 0));
  d ? m2l_all_t<double>(c, groups) : m2l_all_t<float>(c, groups);
  prof_mark(c, "m2l");
}

void run_near_free(Ctx &c, std::vector<Group> &groups, double *phi, double *field, cudaStream_t st) {
  c.def.p2p.clear();
  c.def.p2p_blocks = 0;
  c.p2p_timed = false;
  if (c.opts.precision == LPBFMM_FP64) return;
  OnStream on(c, st);
  for (auto &g : groups) {
    if (!(g.is_free && (g.parts & 1))) continue;
    const Level &Lf = g.T.lev[g.Df];
    const unsigned nb = (unsigned)Lf.n;
    if (!nb) continue;
    const int64_t np = g.T.np;
    float4 *h4 = c.arena.get<float4>((size_t)np), *l4 = c.arena.get<float4>((size_t)np);
    k_split_points<<<nb, 64, 0, c.stream>>>(Lf.d_n, Lf.key, Lf.pstart, Lf.pcount, g.T.x, g.T.y, g.T.z, g.T.q,
                                             geo_at<float>(g, g.Df), h4, l4);
    LPB_LAUNCH();
    c.launches++;
    const double hD = g.h(g.Df);
    P2PJob j;
    j.d_nb = Lf.d_n; j.bkey = Lf.key; j.bstart = Lf.pstart; j.bcount = Lf.pcount; j.ulist = g.ufree;
    j.h4 = h4; j.l4 = l4; j.src = g.T.src; j.phi = phi; j.field = field;
    j.scale = 1.0 / (4.0 * PI * c.md.eps[g.l]);
    j.hh = (float)hD; j.hl = (float)(hD - (double)j.hh); j.lam = (float)c.md.lam[g.l];
    j.block0 = c.def.p2p_blocks;
    c.def.p2p.push_back(j);
    c.def.p2p_blocks += (2 * (int64_t)nb + P2P_WARPS - 1) / P2P_WARPS;
  }
  if (!c.def.on && !c.def.p2p.empty()) {
    LPB_CUDA(cudaEventRecord(c.ev_p2p[0], c.stream));
    launch_p2p(c, c.def.p2p, c.def.p2p_blocks, c.stream);
    LPB_CUDA(cudaEventRecord(c.ev_p2p[1], c.stream));
    c.p2p_timed = true;
    c.def.p2p.clear();
    c.def.p2p_blocks = 0;
  }
}

void run_fmm_back(Ctx &c, std::vector<Group> &groups, double *phi, double *field) {
  const bool d = c.opts.precision == LPBFMM_FP64;
  // the far field (its own stream) and the free-space near field, which adds into the same
  // outputs, are complete first
  if (c.far_async) LPB_CUDA(cudaStreamWaitEvent(c.stream, c.ev_far, 0));
  if (c.near_async) LPB_CUDA(cudaStreamWaitEvent(c.stream, c.ev_near, 0));
  for (auto &g : groups)
    d ? downward_t<double>(c, g, g.parts, phi, field) : downward_t<float>(c, g, g.parts, phi, field);
  prof_mark(c, "downward");
}

void launch_deferred(const std::vector<Ctx *> &cs, int stage, cudaStream_t st) {
  if (cs.empty()) return;
  Ctx &c0 = *cs[0];
  if (stage == 0) {
    // per truncation order (the kernels take K and p as arguments): one tensor-core M2L launch,
    // then one launch of the slot sums (FP32 partials: the tensor-core path runs in mixed mode)
    std::vector<int> orders;
    for (Ctx *c : cs)
      if (c->def.nc && std::find(orders.begin(), orders.end(), c->p) == orders.end()) orders.push_back(c->p);
    for (int p : orders) {
      std::vector<TJob> tj;
      std::vector<RJob> red;
      int64_t items = 0, relem = 0;
      Ctx *lead = nullptr;
      for (Ctx *c : cs) {
        if (!c->def.nc || c->p != p) continue;
        if (!lead) lead = c;
        for (TJob j : c->def.tc) {
          j.item0 += items;
          tj.push_back(j);
        }
        items += c->def.tc_items;
        for (RJob r : c->def.red) {
          r.e0 += relem;
          red.push_back(r);
        }
        relem += c->def.red_elems;
      }
      TJob *dj = c0.arena.get<TJob>(tj.size());
      LPB_CUDA(cudaMemcpyAsync(dj, tj.data(), sizeof(TJob) * tj.size(), cudaMemcpyHostToDevice, st));
      switch (lead->def.nc) {
#define LPB_TC_GROUP(NCV)                                                                                    \
  case NCV:                                                                                                 \
    LPB_ATTR_ONCE(k_m2l_tc<NCV>, tc_smem(NCV));                                                             \
    k_m2l_tc<NCV><<<(unsigned)items, TC_THREADS, tc_smem(NCV), st>>>(dj, (int)tj.size(), lead->K, p, c0.status); \
    break;
        LPB_TC_GROUP(1) LPB_TC_GROUP(2) LPB_TC_GROUP(3) LPB_TC_GROUP(4)
#undef LPB_TC_GROUP
      }
      LPB_LAUNCH();
      c0.launches++;
      if (!red.empty()) {
        RJob *dr = c0.arena.get<RJob>(red.size());
        LPB_CUDA(cudaMemcpyAsync(dr, red.data(), sizeof(RJob) * red.size(), cudaMemcpyHostToDevice, st));
        k_m2l_reduce<float><<<(unsigned)((relem + 255) / 256), 256, 0, st>>>(dr, (int)red.size(), lead->K);
        LPB_LAUNCH();
        c0.launches++;
      }
    }
  } else {
    std::vector<P2PJob> pj;
    int64_t blocks = 0;
    for (Ctx *c : cs) {
      for (P2PJob j : c->def.p2p) {
        j.block0 += blocks;
        pj.push_back(j);
      }
      blocks += c->def.p2p_blocks;
    }
    launch_p2p(c0, pj, blocks, st);
  }
}

}  // namespace lpb
