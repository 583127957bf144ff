// Translation operators, built on the device in FP64 for every evaluation.
//
// All translations have the azimuth-factored form (half representation m >= 0):
//   X'_{nu mu} = e^{i mu phi} X_{nu mu},  Y_{nm} = P Re X' + i Q Im X',  out_{nm} += e^{-i m phi} Y_{nm}
// with real P, Q of size K x K, K = (p+1)(p+2)/2.
//  * free-space M2M / L2L / M2L (Sec. 3.1, Theorems 1-3): Gaunt-coefficient sums over
//    i_q(lambda b) or k_q(lambda b) times Phat_q(cos theta_b);
//  * reaction M2L (Sec. 3.4 eq. metoleimage2, Sec. 3.5): the scaled Sommerfeld integrals
//    S^K S_{K d, ij} (eq. M2Ltable) by composite Gauss-Legendre quadrature for d = 0, 1,
//    the forward recurrence (eq. recurrence1) for d >= 2, and a Legendre-product expansion
//    of the two plane-wave factors (eq. metoletableform), in this library's own derivation.
// Scaling (Sec. 3.5, the rescaled expansions): with h the box size, multipole coefficients are stored as
// M~_n = M_n (2n+1)!!/(lambda h)^n and local ones as L~_n = c L_n (lambda h)^n/(2n+1)!!
// (c = lambda/(2 pi^2 eps) for the free-space part, 1 for reaction parts), so that
// phi = sum L~_nm itilde_n(lambda r) R_n^m(r/h) with R_n^m = r^n Y_n^m.
#include "internal.h"

#include <mutex>

namespace lpb {

struct OpDesc {
  int kind;     // 0 = M2L free, 1 = M2M, 2 = L2L
  int out_inv;  // 0: out scale x^n/(2n+1)!!, 1: (2n+1)!!/x^n
  int in_inv;
  int dir;      // direction of b: free M2L class (< NFREE_CLS), NFREE_CLS + cz for M2M / L2L (Ctx::phat_dir)
  double lam, bnorm, cosb, xout, xin, pref;
  int64_t dst;  // element offset of P (Q follows after K*K)
};

// half-representation index o = n(n+1)/2 + m -> (n, m), integer arithmetic only
__device__ __forceinline__ void hdecode(int o, int &n, int &m) {
  n = 0;
  while ((n + 1) * (n + 2) / 2 <= o) ++n;
  m = o - n * (n + 1) / 2;
}

// Per-descriptor radial factors, one thread each: f[q] = k_q or i_q (lambda |b|) and the
// output / input scalings so[n], si[n], stored as [NPREP] doubles per descriptor.  The angular
// factor Phat_q^k(cos theta_b) depends only on the direction of b and comes from Ctx::phat_dir.
constexpr int PREP_F = 0, PREP_SO = 2 * PMAX + 1, PREP_SI = PREP_SO + PMAX + 1, NPREP = PREP_SI + PMAX + 1;
constexpr int NPL_MAX = (2 * PMAX + 1) * (2 * PMAX + 2) / 2;

__global__ void k_ops_prep(const OpDesc *descs, int nd, int p, double *prep) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nd) return;
  const OpDesc d = descs[i];
  double *w = prep + (size_t)i * NPREP;
  const int qmax = 2 * p;
  const double x = d.lam * d.bnorm;
  if (d.kind == 0) kbessel_all(x, qmax, w + PREP_F);
  else ibessel_all(x, qmax, w + PREP_F);
  double a = 1.0, b = 1.0;  // x^n / (2n+1)!!
  for (int n = 0; n <= p; ++n) {
    if (n > 0) {
      a *= d.xout / (2.0 * n + 1.0);
      b *= d.xin / (2.0 * n + 1.0);
    }
    w[PREP_SO + n] = (d.out_inv ? 1.0 / a : a) * d.pref;
    w[PREP_SI + n] = d.in_inv ? 1.0 / b : b;
  }
}

constexpr int OPS_SPLIT = 4;  // CTAs per descriptor

template <typename T>
__global__ void k_build_ops(const OpDesc *descs, const double *prep, const double *phat_dir, int p, int K,
                            const double *gaunt, T *out) {
  const OpDesc d = descs[blockIdx.x];
  __shared__ double w[NPREP], Pl[NPL_MAX];
  const double *pw = prep + (size_t)blockIdx.x * NPREP;
  for (int e = threadIdx.x; e < NPREP; e += blockDim.x) w[e] = pw[e];
  const int npl = (2 * p + 1) * (2 * p + 2) / 2;
  const double *pd = phat_dir + (size_t)d.dir * npl;
  for (int e = threadIdx.x; e < npl; e += blockDim.x) Pl[e] = pd[e];
  __syncthreads();
  const double *f = w + PREP_F, *so = w + PREP_SO, *si = w + PREP_SI;
  const int NF = (p + 1) * (p + 1), NQ = 2 * p + 1;
  for (int e = blockIdx.y * blockDim.x + threadIdx.x; e < K * K; e += gridDim.y * blockDim.x) {
    const int o = e / K, i = e % K;
    int n, m, nu, mu;
    hdecode(o, n, m);
    hdecode(i, nu, mu);
    double r[2] = {0.0, 0.0};
    for (int sgn = 0; sgn < 2; ++sgn) {
      const int mus = sgn ? -mu : mu;
      if (sgn && mu == 0) break;
      double acc = 0.0;
      for (int q = abs(n - nu); q <= n + nu; q += 2) {
        if (d.kind == 2 || d.kind == 0) {
          const int k = m - mus;
          if (abs(k) > q) continue;
          acc += f[q] * phat_signed(Pl, q, k) * gaunt[((size_t)fidx(nu, mus) * NF + fidx(n, m)) * NQ + q];
        } else {
          const int k = mus - m;
          if (abs(k) > q) continue;
          acc += f[q] * phat_signed(Pl, q, k) * gaunt[((size_t)fidx(n, m) * NF + fidx(nu, mus)) * NQ + q];
        }
      }
      acc *= 4.0 * PI * so[n] * si[nu];
      if (d.kind == 0 && (n & 1)) acc = -acc;
      r[sgn] = acc;
    }
    double P, Q;
    if (mu == 0) { P = r[0]; Q = 0.0; }
    else {
      const double sg = (mu & 1) ? -1.0 : 1.0;
      P = r[0] + sg * r[1];
      Q = r[0] - sg * r[1];
    }
    out[d.dst + (size_t)o * K + i] = (T)P;
    out[d.dst + (size_t)K * K + (size_t)o * K + i] = (T)Q;
  }
}

// ---------------------------------------------------------------------------------------
// Reaction operators
// ---------------------------------------------------------------------------------------
struct RDesc {
  int l, a, lp, b, tau, ntypes, st, pad;
  int cls0, pad2;        // the table array holds classes cls0, cls0 + 1, ... (0: every class)
  double h, Lam, Lamp;
  const uint8_t *used;   // [NREACT_CLS]
  double *stab;          // [NREACT_CLS][ntypes][TS]
  float2 *coef;          // [K*K][NS] double-float (hi, lo) coefficients C_s
  int64_t dst;           // element offset of class 0, type tau in the op array
};


constexpr int MAXPANEL = 1024;

__device__ __forceinline__ int stab_index(int KT, int K, int d, int ij) { return ((K * (KT + 1)) + d) * 4 + ij; }

__device__ void make_panels(double umax, double wmax, double lmin, double *pu, double *pw, int *np) {
  int n = 0;
  double u = 0.0;
  while (u < umax && n < MAXPANEL) {
    double w = fmin(wmax, 0.5 * (lmin + u));
    if (u + w > umax) w = umax - u;
    pu[n] = u;
    pw[n] = w;
    u += w;
    ++n;
  }
  *np = n;
}

// Gauss-Legendre 16-point rule on [-1,1] (nodes by Newton iteration on the host)
__constant__ double c_glx[16], c_glw[16];
static std::atomic<uint64_t> g_gl_ready{0};
void upload_gl16() {
  if (!not_done_on_device(g_gl_ready)) return;
  double x[16], w[16];
  for (int i = 0; i < 16; ++i) {
    long double z = cosl(3.14159265358979323846264338L * (i + 0.75L) / 16.5L), dp = 1;
    for (int it = 0; it < 100; ++it) {
      long double p0 = 1, p1 = z;
      for (int k = 2; k <= 16; ++k) { long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
      dp = 16 * (z * p1 - p0) / (z * z - 1);
      const long double dz = p1 / dp;
      z -= dz;
      if (fabsl(dz) < 1e-19L) break;
    }
    long double p0 = 1, p1 = z;
    for (int k = 2; k <= 16; ++k) { long double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
    dp = 16 * (z * p1 - p0) / (z * z - 1);
    x[i] = (double)z;
    w[i] = (double)(2 / ((1 - z * z) * dp * dp));
  }
  LPB_CUDA(cudaMemcpyToSymbol(c_glx, x, sizeof x));
  LPB_CUDA(cudaMemcpyToSymbol(c_glw, w, sizeof w));
  mark_done_on_device(g_gl_ready);
}
__device__ __forceinline__ void gl16(double *x, double *w) {
  for (int i = 0; i < 16; ++i) { x[i] = c_glx[i]; w[i] = c_glw[i]; }
}

// Quadrature of S^K S_{K d, ij} for d = 0, 1, K = 0..KT on one composite Gauss-Legendre node
// set per (component, level) in u = lambda_rho h: panel width min(2/zeta_min, pi/rho_max),
// graded near u = 0 to resolve the branch points at u = +-i Lambda.  Node data (first kernel):
//   nd[q] = {u, w sigma / u_z, Lam / u_z, Lamp / u'_z, e^{-u_z (k+1/2)} (k < NKT),
//            e^{-u'_z (k+1/2)} (k < NKT), J0(u rho_r), J1(u rho_r) (r < NRHO)}
constexpr int ND_ET = 4, ND_ES = ND_ET + NKT, ND_J0 = ND_ES + NKT, ND_J1 = ND_J0 + NRHO;
constexpr int NDF = ND_J1 + NRHO;

// host: the u beyond which u^KT e^{-zeta u} has fallen by tol (and e^-3 more) below its peak
// at u = KT/zeta
static double node_umax(int KT, double zeta, double tol) {
  const double pk = fmax(KT / zeta, 1.0 / zeta);
  const double target = KT * log(pk) - zeta * pk + log(tol) - 3.0;
  double umax = pk;
  while (KT * log(umax) - zeta * umax > target) umax += 0.25 / zeta;
  return umax;
}

struct NDesc {
  double umax, wmax, lmin;
  double ucut[NKT];  // truncation point for zeta = k_t + k_s + 1 = 1 .. NKT
  int npan, nq;
  double *nodes;        // [nq][NDF]
  const double *bes;    // shared J0, J1 columns of this node set [nq][2 NRHO], or null (computed here)
};

// J0(u rho_r), J1(u rho_r) at the nodes of one node set, shared by every descriptor using it
__global__ void k_stab_bessel(NDesc N, double *bes) {
  __shared__ double pu[MAXPANEL], pw[MAXPANEL];
  __shared__ int npan;
  if (threadIdx.x == 0) make_panels(N.umax, N.wmax, N.lmin, pu, pw, &npan);
  __syncthreads();
  // one thread per (node, rho value): the node set is short, so a thread per node alone would
  // leave most of the GPU idle
  const int64_t total = (int64_t)N.nq * NRHO;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int j = (int)(e / NRHO), r = (int)(e % NRHO);
    double *o = bes + (size_t)j * 2 * NRHO;
    if (j >= npan * 16) {
      o[r] = 0.0;
      o[NRHO + r] = 0.0;
      continue;
    }
    const int pi_ = j >> 4, gi = 15 - (j & 15);  // ascending abscissae
    const double u = pu[pi_] + 0.5 * pw[pi_] * (c_glx[gi] + 1.0);
    const double x = u * sqrt((double)rho2_of(r));
    o[r] = j0(x);
    o[NRHO + r] = j1(x);
  }
}

__global__ void k_stab_nodes(const RDesc *descs, const NDesc *nds, Medium md) {
  const RDesc D = descs[blockIdx.y];
  const NDesc N = nds[blockIdx.y];
  __shared__ double pu[MAXPANEL], pw[MAXPANEL];
  __shared__ int npan;
  if (threadIdx.x == 0) make_panels(N.umax, N.wmax, N.lmin, pu, pw, &npan);
  __syncthreads();
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < N.nq; j += gridDim.x * blockDim.x) {
    double *o = N.nodes + (size_t)j * NDF;
    if (j >= npan * 16) {
      for (int k = 0; k < NDF; ++k) o[k] = 0.0;
      continue;
    }
    const int pi_ = j >> 4, gi = 15 - (j & 15);  // ascending abscissae
    const double u = pu[pi_] + 0.5 * pw[pi_] * (c_glx[gi] + 1.0);
    const double w = 0.5 * pw[pi_] * c_glw[gi];
    const double sg = layer_sigma(md, u / D.h, D.l, D.a, D.lp, D.b);
    const double uz = sqrt(D.Lam * D.Lam + u * u), uzp = sqrt(D.Lamp * D.Lamp + u * u);
    o[0] = u;
    o[1] = w * sg / uz;
    o[2] = D.Lam / uz;
    o[3] = D.Lamp / uzp;
    for (int k = 0; k < NKT; ++k) {
      o[ND_ET + k] = exp(-uz * (k + 0.5));
      o[ND_ES + k] = exp(-uzp * (k + 0.5));
    }
    if (N.bes) {
      const double *b = N.bes + (size_t)j * 2 * NRHO;
      for (int r = 0; r < 2 * NRHO; ++r) o[ND_J0 + r] = b[r];
    } else {
      for (int r = 0; r < NRHO; ++r) {
        const double x = u * sqrt((double)rho2_of(r));
        o[ND_J0 + r] = j0(x);
        o[ND_J1 + r] = j1(x);
      }
    }
  }
}

// One CTA per used class.  Per chunk of 256 nodes the power columns u^K (K = 0..KT) and the
// eight node values v_{d,ij} = w sigma/u_z (Lam/u_z)^i (Lamp/u'_z)^j Z_{kt,ks} J_d(u rho) are
// staged in shared memory; thread (d, i, j, K) accumulates sum_q u_q^K v_{d,ij}(q), a
// [KT+1 x Q] x [Q x 8] product in FP64, for the entries with K - d odd: the operators use
// only those, because K = 1 + |m| + |mu| + 2s and d = |mu - m| differ by an odd number.
constexpr int SQ_CHUNK = 256, SQ_LD = SQ_CHUNK + 1;
__global__ void k_stab_quad(const RDesc *descs, const NDesc *nds, int KT, const double *sfac) {
  const RDesc D = descs[blockIdx.y];
  const NDesc N = nds[blockIdx.y];
  const int cls = blockIdx.x;
  if (D.used && !D.used[cls]) return;
  extern __shared__ double sqsm[];
  double *Pw = sqsm;                          // [KT+1][SQ_LD] powers
  double *V = sqsm + (size_t)(KT + 1) * SQ_LD;  // [8][SQ_LD] node values
  const int ri = cls / NKK, kk = cls % NKK;
  int kt, ks;
  kk_decode(kk, kt, ks);
  const double ucut = N.ucut[kt + ks];
  // output of this thread: d, ij, K with K - d odd
  const int n0 = (KT + 1) / 2, n1 = KT / 2;  // K odd (d = 0): 1,3,..; K even >= 2 (d = 1): 2,4,..
  const int nout = 4 * (n0 + n1);
  int od = 0, oij = 0, oK = -1;
  if ((int)threadIdx.x < nout) {
    const int t = threadIdx.x;
    oij = t & 3;
    const int r = t >> 2;
    if (r < n0) { od = 0; oK = 2 * r + 1; } else { od = 1; oK = 2 * (r - n0) + 2; }
  }
  double acc = 0.0;
  for (int c0 = 0; c0 < N.nq; c0 += SQ_CHUNK) {
    const int q = c0 + threadIdx.x;
    double u = 0.0;
    if (q < N.nq) {
      const double *o = N.nodes + (size_t)q * NDF;
      u = o[0];
      const double base = o[1] * o[ND_ET + kt] * o[ND_ES + ks];
      const double j0v = o[ND_J0 + ri], j1v = o[ND_J1 + ri], fi = o[2], fj = o[3];
      const bool in = u <= ucut && u > 0.0;
      const double b0 = in ? base * j0v : 0.0, b1 = in ? base * j1v : 0.0;
      V[0 * SQ_LD + threadIdx.x] = b0;
      V[1 * SQ_LD + threadIdx.x] = b0 * fj;
      V[2 * SQ_LD + threadIdx.x] = b0 * fi;
      V[3 * SQ_LD + threadIdx.x] = b0 * fi * fj;
      V[4 * SQ_LD + threadIdx.x] = b1;
      V[5 * SQ_LD + threadIdx.x] = b1 * fj;
      V[6 * SQ_LD + threadIdx.x] = b1 * fi;
      V[7 * SQ_LD + threadIdx.x] = b1 * fi * fj;
    } else {
      for (int k = 0; k < 8; ++k) V[k * SQ_LD + threadIdx.x] = 0.0;
    }
    double pw = 1.0;
    for (int K = 0; K <= KT; ++K) {
      Pw[K * SQ_LD + threadIdx.x] = pw;
      pw *= u;
    }
    __syncthreads();
    if (oK >= 0) {
      const double *pr = Pw + oK * SQ_LD, *vr = V + (od * 4 + oij) * SQ_LD;
      const int nn = min(SQ_CHUNK, N.nq - c0);
      for (int j = 0; j < nn; ++j) acc = fma(pr[j], vr[j], acc);
    }
    __syncthreads();
    if (c0 + SQ_CHUNK < N.nq && N.nodes[(size_t)(c0 + SQ_CHUNK) * NDF] > ucut) break;
  }
  double *S = D.stab + ((size_t)(cls - D.cls0) * D.ntypes + D.tau) * (size_t)((KT + 1) * (KT + 1) * 4);
  if (oK >= 0) {
    const double nrm = 1.0 / sfac[oK * (KMAX_TAB + 1) + od];
    S[stab_index(KT, oK, od, oij)] = acc * nrm;
  }
  // entries with K - d even for d = 0, 1 are not used by the operators: zero
  for (int e = threadIdx.x; e < (KT + 1) * 2 * 4; e += blockDim.x) {
    const int K = e / 8, d = (e >> 2) & 1, ij = e & 3;
    if (((K - d) & 1) == 0 && K >= d) S[stab_index(KT, K, d, ij)] = 0.0;
  }
}
static size_t stab_quad_smem(int KT) { return sizeof(double) * (size_t)(KT + 1 + 8) * SQ_LD; }

// host: node set of one (component, level) covering every class (zeta >= 1, rho <= sqrt(50) h)
// number of panels of the graded rule (host mirror of make_panels)
static int count_panels(double umax, double wmax, double lmin) {
  int n = 0;
  double u = 0.0;
  while (u < umax && n < MAXPANEL) {
    double w = fmin(wmax, 0.5 * (lmin + u));
    if (u + w > umax) w = umax - u;
    u += w;
    ++n;
  }
  return n;
}

// Panel width 2 in u = lambda_rho h: with rho <= sqrt(50) the Bessel factor J_d(u rho) has
// derivatives bounded by rho^n, and the 16-point Gauss rule's error term on a width-2 panel,
// rho^32 2^33 (16!)^4 / (33 (32!)^3), is ~1e-18 of the integrand's scale (~1e-25 for
// rho <= sqrt(18)); the factors e^{-zeta u} (zeta <= NKT) are smoother still.  The panels are graded towards u = 0, where the
// branch points u = +-i Lambda of u_z sit.
static NDesc node_desc(int KT, double tol, double Lam, double Lamp) {
  NDesc N;
  N.umax = node_umax(KT, 1.0, tol);
  for (int z = 0; z < NKT; ++z) N.ucut[z] = node_umax(KT, z + 1.0, tol);
  N.wmax = 2.0;
  N.lmin = fmin(Lam, Lamp);
  N.npan = count_panels(N.umax, N.wmax, N.lmin);
  N.nq = N.npan * 16;
  N.nodes = nullptr;
  N.bes = nullptr;
  return N;
}

// a_n = sqrt(n (n+1)) and 1/a_n for n <= 2 KMAX_TAB + 1 (host, long double), for the recurrence
__constant__ double c_an[2 * KMAX_TAB + 2], c_ian[2 * KMAX_TAB + 2];
static std::atomic<uint64_t> g_an_ready{0};
void upload_an() {
  if (!not_done_on_device(g_an_ready)) return;
  double a[2 * KMAX_TAB + 2], ia[2 * KMAX_TAB + 2];
  for (int n = 0; n < 2 * KMAX_TAB + 2; ++n) {
    const long double v = sqrtl((long double)n * (n + 1));
    a[n] = (double)v;
    ia[n] = n ? (double)(1.0L / v) : 0.0;
  }
  LPB_CUDA(cudaMemcpyToSymbol(c_an, a, sizeof a));
  LPB_CUDA(cudaMemcpyToSymbol(c_ian, ia, sizeof ia));
  mark_done_on_device(g_an_ready);
}

// forward recurrence in d (Sec. 3.5 eq. recurrence1), one warp per class:
//   S_{K,d+1} = (2d / a_{K+d}) (1/rho) S_{K-1,d} - (a_{K-d} / a_{K+d}) S_{K,d-1}
__global__ void k_stab_recur(const RDesc *descs, int KT) {
  const RDesc D = descs[blockIdx.y];
  const int cls = blockIdx.x;
  if (D.used && !D.used[cls]) return;
  const int ri = cls / NKK;
  const double rh = sqrt((double)rho2_of(ri));
  const double irh = rh > 0.0 ? 1.0 / rh : 0.0;
  double *S = D.stab + ((size_t)(cls - D.cls0) * D.ntypes + D.tau) * (size_t)((KT + 1) * (KT + 1) * 4);
  const int lane = threadIdx.x;
  for (int d = 1; d < KT; ++d) {
    for (int e = lane; e < (KT + 1) * 4; e += 32) {
      const int K = e >> 2, ij = e & 3;
      if (K < d + 1) continue;
      double v = 0.0;
      if (rh > 0.0) {
        const double ia = c_ian[K + d];
        v = (2.0 * d * ia * irh) * S[stab_index(KT, K - 1, d, ij)] - (c_an[K - d] * ia) * S[stab_index(KT, K, d - 1, ij)];
      }
      S[stab_index(KT, K, d + 1, ij)] = v;
    }
    __syncwarp();
  }
}

// C_s(n,m,nu,mu) = sum_{k+k'=s} c^{nm}_k c^{nu mu}_{k'} Lam^{n-m-2k} Lamp^{nu-mu-2k'}
__global__ void k_react_coef(const RDesc *descs, const double *tpoly, int tpk, int p, int K) {
  const RDesc D = descs[blockIdx.y];
  __shared__ double pl[PMAX + 3], plp[PMAX + 3];  // Lam^e, Lamp^e for e = -1..p+1 at index e+1
  if (threadIdx.x == 0) {
    pl[0] = 1.0 / D.Lam;
    plp[0] = 1.0 / D.Lamp;
    pl[1] = plp[1] = 1.0;
    for (int e = 2; e <= p + 2; ++e) { pl[e] = pl[e - 1] * D.Lam; plp[e] = plp[e - 1] * D.Lamp; }
  }
  __syncthreads();
  const int NS = p + 2;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= K * K) return;
  const int o = e / K, i = e % K;
  int n, m, nu, mu;
  hdecode(o, n, m);
  hdecode(i, nu, mu);
  const int k1 = (n - m + 1) / 2, k2 = (nu - mu + 1) / 2;
  for (int s = 0; s < NS; ++s) {
    double acc = 0.0;
    for (int k = 0; k <= k1; ++k) {
      const int kp = s - k;
      if (kp < 0 || kp > k2) continue;
      acc += tpoly[o * tpk + k] * tpoly[i * tpk + kp] * pl[n - m - 2 * k + 1] * plp[nu - mu - 2 * kp + 1];
    }
    const float h = (float)acc;
    D.coef[(size_t)e * NS + s] = make_float2(h, (float)(acc - (double)h));
  }
}

// double-float arithmetic (value = hi + lo, two FP32 numbers; about 44 significant bits) on
// the FP32 pipes: exact products by FMA, sums by the two-sum of Knuth, then renormalised.
// The _rn intrinsics keep the compiler from contracting the error-free transformations.
__device__ __forceinline__ float2 df_split(double v) {
  const float h = (float)v;
  return make_float2(h, (float)(v - (double)h));
}
// hi + lo of (a.hi + a.lo) + (b.hi + b.lo) rounded to one FP32 number, without losing the low parts
// to cancellation between a and b
__device__ __forceinline__ float df_sum_f(float2 a, float2 b) {
  const float s = __fadd_rn(a.x, b.x);
  const float v = __fsub_rn(s, a.x);
  const float e = __fadd_rn(__fsub_rn(a.x, __fsub_rn(s, v)), __fsub_rn(b.x, v));
  return __fadd_rn(s, __fadd_rn(e, __fadd_rn(a.y, b.y)));
}
__device__ __forceinline__ void df_fma(float2 a, float2 b, float2 &acc) {
  const float p = __fmul_rn(a.x, b.x);
  float e = fmaf(a.x, b.x, -p);  // rounding error of p, exactly
  e = fmaf(a.x, b.y, e);
  e = fmaf(a.y, b.x, e);
  const float s = __fadd_rn(acc.x, p);
  const float v = __fsub_rn(s, acc.x);
  float t = __fadd_rn(__fsub_rn(acc.x, __fsub_rn(s, v)), __fsub_rn(p, v));
  t = __fadd_rn(t, __fadd_rn(acc.y, e));
  const float hi = __fadd_rn(s, t);
  acc = make_float2(hi, __fsub_rn(t, __fsub_rn(hi, s)));
}

// ASM_CC classes per CTA share each entry's decode and coefficient loads
constexpr int ASM_CC = 4;
template <typename T>
__global__ void k_react_assemble(const RDesc *descs, int p, int K, int KT, const double *sfac, T *out) {
  const RDesc D = descs[blockIdx.y];
  const int cls0 = blockIdx.x * ASM_CC;
  extern __shared__ double asm_sm[];
  const int TS = (KT + 1) * (KT + 1) * 4;
  float2 *Sf = (float2 *)asm_sm;  // [ASM_CC][TS]: sqrt((K+d)!(K-d)!) S^K S_{K d, ij}, double-float
  __shared__ double smm[PMAX + 1], rdf[PMAX + 1];
  __shared__ double fa[KHALF_MAX], fb[KHALF_MAX];  // prefactor A(o, i) = fa[o] fb[i]
  __shared__ float faf[KHALF_MAX], fbf[KHALF_MAX];  // the same in FP32 (FP32 operators, p <= 12)
  bool cuse[ASM_CC];
  bool any = false;
#pragma unroll
  for (int k = 0; k < ASM_CC; ++k) {
    const int cls = cls0 + k;
    cuse[k] = cls < NREACT_CLS && (!D.used || D.used[cls]);
    any |= cuse[k];
  }
  if (!any) return;
  for (int k = 0; k < ASM_CC; ++k) {
    if (!cuse[k]) continue;
    const double *S = D.stab + ((size_t)(cls0 + k - D.cls0) * D.ntypes + D.tau) * (size_t)TS;
    for (int e = threadIdx.x; e < TS; e += blockDim.x) {
      const int Kk = e / ((KT + 1) * 4), d = (e / 4) % (KT + 1);
      Sf[k * TS + e] = df_split((d <= Kk) ? sfac[Kk * (KMAX_TAB + 1) + d] * S[e] : 0.0);
    }
  }
  if (threadIdx.x == 0) {
    double sg = 1.0;
    smm[0] = 1.0;
    for (int m = 1; m <= p; ++m) { sg *= -sqrt((2.0 * m + 1.0) / (2.0 * m)); smm[m] = sg; }
    rdf[0] = 1.0;
    for (int n = 1; n <= p; ++n) rdf[n] = rdf[n - 1] / (2.0 * n + 1.0);  // 1/(2n+1)!!
  }
  __syncthreads();
  // fa[o] = smm(m) st^{n-m} / (2n+1)!!,  fb[i] = smm(mu) (-st)^{nu-mu} / ((2nu+1)!! 4 pi h)
  for (int e = threadIdx.x; e < K; e += blockDim.x) {
    int n, m;
    hdecode(e, n, m);
    const bool odd = (n - m) & 1;
    fa[e] = smm[m] * rdf[n] * (odd ? (double)D.st : 1.0);
    fb[e] = smm[m] * rdf[n] * (odd ? -(double)D.st : 1.0) * (0.25 / PI) / D.h;
    faf[e] = (float)fa[e];
    fbf[e] = (float)fb[e];
  }
  __syncthreads();
  // FP32 epilogue for FP32 operators while the prefactors stay well inside the FP32 range
  const bool f32_out = sizeof(T) == 4 && p <= 12;
  const int NS = p + 2;
  const size_t KK = (size_t)K * K;
  for (int e = threadIdx.x; e < K * K; e += blockDim.x) {
    const int o = e / K, i = e % K;
    int n, m, nu, mu;
    hdecode(o, n, m);
    hdecode(i, nu, mu);
    const int ij = 2 * ((n - m) & 1) + ((nu - mu) & 1);
    const int smax = (n - m + 1) / 2 + (nu - mu + 1) / 2;
    const float2 *cf = D.coef + (size_t)e * NS;
    const int dp = mu - m, dm = mu + m;  // |d| for +mu and -mu
    const int adp = dp < 0 ? -dp : dp;
    float2 ap[ASM_CC], am[ASM_CC];
#pragma unroll
    for (int k = 0; k < ASM_CC; ++k) ap[k] = am[k] = make_float2(0.f, 0.f);
    // the entry's coefficients, all loads in flight at once (smax <= p + 1 < PMAX + 2)
    float2 cv[PMAX + 2];
#pragma unroll
    for (int s = 0; s < PMAX + 2; ++s) cv[s] = s <= smax ? cf[s] : make_float2(0.f, 0.f);
#pragma unroll
    for (int s = 0; s < PMAX + 2; ++s) {
      const int Kk = 1 + m + mu + 2 * s;
      if (s > smax || Kk > KT) break;
      const float2 c = cv[s];
      const int ip = ((Kk * (KT + 1)) + adp) * 4 + ij, im = ((Kk * (KT + 1)) + dm) * 4 + ij;
#pragma unroll
      for (int k = 0; k < ASM_CC; ++k) {
        df_fma(c, Sf[k * TS + ip], ap[k]);
        df_fma(c, Sf[k * TS + im], am[k]);
      }
    }
    // signs: (-1)^|d| for d = mu - m < 0 and for d = -mu - m < 0; (-1)^mu of the -mu term
    const bool fp = dp < 0 && (adp & 1), fm = ((dm > 0 && (dm & 1)) != ((mu & 1) != 0));
#pragma unroll
    for (int k = 0; k < ASM_CC; ++k) {
      if (!cuse[k]) continue;
      const float2 Xd = fp ? make_float2(-ap[k].x, -ap[k].y) : ap[k];
      const float2 Yd = fm ? make_float2(-am[k].x, -am[k].y) : am[k];
      T *dP = out + D.dst + (size_t)(cls0 + k) * D.ntypes * 2 * KK + (size_t)D.tau * 2 * KK + (size_t)o * K + i;
      T *dQ = dP + KK;
      if (f32_out) {
        const float Af = faf[o] * fbf[i];
        if (mu == 0) {
          *dP = (T)(Af * df_sum_f(Xd, make_float2(0.f, 0.f)));
          *dQ = (T)0;
        } else {
          *dP = (T)(Af * df_sum_f(Xd, Yd));
          *dQ = (T)(Af * df_sum_f(Xd, make_float2(-Yd.x, -Yd.y)));
        }
      } else {
        const double A = fa[o] * fb[i];
        const double X = (double)Xd.x + (double)Xd.y, Y = (double)Yd.x + (double)Yd.y;
        *dP = (T)(mu == 0 ? A * X : A * (X + Y));
        *dQ = (T)(mu == 0 ? 0.0 : A * (X - Y));
      }
    }
  }
}
static size_t assemble_smem(int KT) { return ASM_CC * sizeof(double) * (size_t)(KT + 1) * (KT + 1) * 4; }

// near-field reaction quadrature nodes: W = w lr sigma / (4 pi lz_l), lz_l, lz_l'
__global__ void k_near_nodes(Medium md, int l, int a, int ntypes, double umax, double wmax, double lmin,
                             double *nodes, int nq) {
  __shared__ double pu[MAXPANEL], pw[MAXPANEL];
  __shared__ double gx[16], gw[16];
  __shared__ int npan;
  if (threadIdx.x == 0) {
    gl16(gx, gw);
    make_panels(umax, wmax, lmin, pu, pw, &npan);
  }
  __syncthreads();
  const int tau = blockIdx.y;
  int lp, b;
  type_decode(tau, lp, b);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < nq; j += gridDim.x * blockDim.x) {
    double *o = nodes + ((size_t)tau * nq + j) * 4;
    if (j >= npan * 16) { o[0] = o[1] = 0.0; o[2] = o[3] = 1.0; continue; }
    const int pi_ = j >> 4, gi = 15 - (j & 15);  // ascending abscissae
    const double lr = pu[pi_] + 0.5 * pw[pi_] * (gx[gi] + 1.0);
    const double w = 0.5 * pw[pi_] * gw[gi];
    const double lz = sqrt(md.lam[l] * md.lam[l] + lr * lr), lzp = sqrt(md.lam[lp] * md.lam[lp] + lr * lr);
    o[0] = lr;
    o[1] = w * lr * layer_sigma(md, lr, l, a, lp, b) / (4.0 * PI * lz);
    o[2] = lz;
    o[3] = lzp;
  }
}

template <typename T>
static void build_ops_t(Ctx &c, Group &g, int parts, int which) {
  const int p = c.p, K = c.K;
  const size_t KK = (size_t)K * K;
  const double lam_t = c.md.lam[g.l];
  if (which & 1) {
  std::vector<OpDesc> descs;
  size_t total = 0;
  auto add = [&](int kind, int out_inv, int in_inv, double lam, double bx, double by, double bz, double xout,
                 double xin, double pref, int dir, size_t offset_in_slot) {
    OpDesc d;
    d.kind = kind; d.out_inv = out_inv; d.in_inv = in_inv; d.dir = dir;
    d.lam = lam;
    d.bnorm = sqrt(bx * bx + by * by + bz * bz);
    d.cosb = bz / d.bnorm;
    d.xout = xout; d.xin = xin; d.pref = pref;
    d.dst = (int64_t)(total + offset_in_slot);
    descs.push_back(d);
      };
  // layout: per level a block with M2M (free + types), L2L, free M2L classes
  struct Blk { size_t m2m_t, m2m_i, l2l, fm2l; };
  std::vector<Blk> blk(DMAX + 1);
  for (int l = 2; l <= g.D; ++l) {
    const double h = g.h(l), hc = h, hp = 2.0 * h;
    Blk b{};
    // M2M: children at level l -> parents at l-1 (only l >= 3)
    const bool free_l = g.is_free && (parts & 1) && l <= g.Df;  // free-space part lives at levels <= Df
    if (l >= 3) {
      if (free_l) {
        b.m2m_t = total;
        for (int cz = 0; cz < 2; ++cz)
          add(1, 1, 0, lam_t, 0.5 * hc, 0.5 * hc, (cz ? 0.5 : -0.5) * hc, lam_t * hp, lam_t * hc, 1.0,
              NFREE_CLS + cz, (size_t)cz * 2 * KK);
        total += 4 * KK;
      }
      if (parts & 2) {
        b.m2m_i = total;
        for (int t = 0; t < g.ntypes; ++t) {
          int lp, bb;
          type_decode(t, lp, bb);
          const double la = c.md.lam[lp];
          for (int cz = 0; cz < 2; ++cz)
            add(1, 1, 0, la, 0.5 * hc, 0.5 * hc, (cz ? 0.5 : -0.5) * hc, la * hp, la * hc, 1.0, NFREE_CLS + cz,
                ((size_t)t * 2 + cz) * 2 * KK);
        }
        total += (size_t)g.ntypes * 4 * KK;
      }
      // L2L: parent (l-1) -> child at l
      b.l2l = total;
      for (int cz = 0; cz < 2; ++cz)
        add(2, 0, 1, lam_t, 0.5 * hc, 0.5 * hc, (cz ? 0.5 : -0.5) * hc, lam_t * hc, lam_t * hp, 1.0,
            NFREE_CLS + cz, (size_t)cz * 2 * KK);
      total += 4 * KK;
    }
    if (free_l) {
      b.fm2l = total;
      const double pref = lam_t / (2.0 * PI * PI * c.md.eps[g.l]);
      for (int ri = 0; ri < NRHO; ++ri)
        for (int dz = -OFF_R; dz <= OFF_R; ++dz) {
          const int cls = ri * NDZ + dz + OFF_R;
          if (!free_class_is_far(ri, dz, c.ws)) continue;
          // b = c_t - c_s = -(offset) h; azimuth factored out: b = (rho h, 0, -dz h)
          add(0, 0, 0, lam_t, sqrt((double)rho2_of(ri)) * h, 0.0, -dz * h, lam_t * h, lam_t * h, pref, cls,
              (size_t)cls * 2 * KK);
        }
      total += (size_t)NFREE_CLS * 2 * KK;
    }
    blk[l] = b;
  }
  T *ops = c.arena.get<T>(total);
  for (int l = 2; l <= g.D; ++l) {
    const bool free_l = g.is_free && (parts & 1) && l <= g.Df;
    g.op_m2m_t[l] = (l >= 3 && free_l) ? (void *)(ops + blk[l].m2m_t) : nullptr;
    g.op_m2m_i[l] = (l >= 3 && (parts & 2)) ? (void *)(ops + blk[l].m2m_i) : nullptr;
    g.op_l2l[l] = (l >= 3) ? (void *)(ops + blk[l].l2l) : nullptr;
    g.op_free[l] = free_l ? (void *)(ops + blk[l].fm2l) : nullptr;
  }
  if (!descs.empty()) {
    OpDesc *dd = c.arena.get<OpDesc>(descs.size());
    LPB_CUDA(cudaMemcpyAsync(dd, descs.data(), sizeof(OpDesc) * descs.size(), cudaMemcpyHostToDevice, c.stream));
    double *prep = c.arena.get<double>(descs.size() * NPREP);
    k_ops_prep<<<(unsigned)((descs.size() + 63) / 64), 64, 0, c.stream>>>(dd, (int)descs.size(), p, prep);
    LPB_LAUNCH();
    k_build_ops<T><<<dim3((unsigned)descs.size(), OPS_SPLIT), 256, 0, c.stream>>>(dd, prep, c.phat_dir, p, K,
                                                                                  c.gaunt, ops);
    LPB_LAUNCH();
    c.launches += 2;
  }
  }
  if (!(which & 2) || !(parts & 2) || !g.I.np) return;
  // reaction: one descriptor per (level, type)
  const int KT = 2 * p + 3, NS = p + 2;
  const size_t TS = (size_t)(KT + 1) * (KT + 1) * 4;
  std::vector<RDesc> rd;
  const int st = (g.a == 1) ? -1 : 1;
  for (int l = 2; l <= g.D; ++l) {
    if (!g.vreact[l]) continue;
    const double h = g.h(l);
    g.stab[l] = c.arena.get<double>((size_t)NREACT_CLS * g.ntypes * TS);
    g.op_react[l] = c.arena.get<T>((size_t)NREACT_CLS * g.ntypes * 2 * KK);
    float2 *coef = c.arena.get<float2>((size_t)g.ntypes * KK * NS);
    for (int t = 0; t < g.ntypes; ++t) {
      int lp, bb;
      type_decode(t, lp, bb);
      RDesc d;
      d.l = g.l; d.a = g.a; d.lp = lp; d.b = bb; d.tau = t; d.ntypes = g.ntypes; d.st = st; d.pad = l;
      d.cls0 = 0; d.pad2 = 0;
      d.h = h; d.Lam = c.md.lam[g.l] * h; d.Lamp = c.md.lam[lp] * h;
      d.used = g.used[l];
      d.stab = g.stab[l];
      d.coef = coef + (size_t)t * KK * NS;
      d.dst = 0;
      rd.push_back(d);
    }
  }
  if (!rd.empty()) {
    RDesc *dr = c.arena.get<RDesc>(rd.size());
    LPB_CUDA(cudaMemcpyAsync(dr, rd.data(), sizeof(RDesc) * rd.size(), cudaMemcpyHostToDevice, c.stream));
    const unsigned nd = (unsigned)rd.size();
    const double tol = fmax(c.tol, 1e-16);
    std::vector<NDesc> nv;
    int maxq = 0;
    // one node set for the whole evaluation (graded to the smallest Lambda of all reaction
    // groups), so the Bessel columns are evaluated once and shared
    if (!c.stab_bes) {
      const NDesc N0 = node_desc(KT, tol, c.stab_lmin, c.stab_lmin);
      c.stab_bes = c.arena.get<double>((size_t)N0.nq * 2 * NRHO);
      k_stab_bessel<<<(unsigned)(((int64_t)N0.nq * NRHO + 255) / 256), 256, 0, c.stream>>>(N0, c.stab_bes);
      LPB_LAUNCH();
      c.launches++;
    }
    for (auto &d : rd) {
      (void)d;
      NDesc N = node_desc(KT, tol, c.stab_lmin, c.stab_lmin);
      N.bes = c.stab_bes;
      N.nodes = c.arena.get<double>((size_t)N.nq * NDF);
      maxq = std::max(maxq, N.nq);
      nv.push_back(N);
    }
    NDesc *dn = c.arena.get<NDesc>(nv.size());
    LPB_CUDA(cudaMemcpyAsync(dn, nv.data(), sizeof(NDesc) * nv.size(), cudaMemcpyHostToDevice, c.stream));
    k_stab_nodes<<<dim3((unsigned)((maxq + 255) / 256), nd), 256, 0, c.stream>>>(dr, dn, c.md);
    LPB_LAUNCH();
    {
      const size_t sm = stab_quad_smem(KT);
      LPB_ATTR_ONCE(k_stab_quad, stab_quad_smem(KMAX_TAB));  // the largest table any order needs
      k_stab_quad<<<dim3(NREACT_CLS, nd), SQ_CHUNK, sm, c.stream>>>(dr, dn, KT, c.sfac);
      LPB_LAUNCH();
    }
    c.launches += 1;
    k_stab_recur<<<dim3(NREACT_CLS, nd), 32, 0, c.stream>>>(dr, KT);
    LPB_LAUNCH();
    k_react_coef<<<dim3((unsigned)((KK + 255) / 256), nd), 256, 0, c.stream>>>(dr, c.tpoly, c.tpk, p, K);
    LPB_LAUNCH();
    // assemble into each level's op array: descriptors grouped by level
    size_t first = 0;
    while (first < rd.size()) {
      const int l = rd[first].pad;
      size_t last = first;
      while (last < rd.size() && rd[last].pad == l) ++last;
      LPB_ATTR_ONCE(k_react_assemble<T>, assemble_smem(KMAX_TAB));
      k_react_assemble<T><<<dim3((NREACT_CLS + ASM_CC - 1) / ASM_CC, (unsigned)(last - first)), 256,
                            assemble_smem(KT), c.stream>>>(
          dr + first, p, K, KT, c.sfac, (T *)g.op_react[l]);
      LPB_LAUNCH();
      c.launches++;
      first = last;
    }
    c.launches += 3;
  }
}

void build_operators(Ctx &c, Group &g, int parts, int which) {
  if (c.opts.precision == LPBFMM_FP64) build_ops_t<double>(c, g, parts, which);
  else build_ops_t<float>(c, g, parts, which);
}

void build_near_nodes(Ctx &c, Group &g, double zeta_min, double rho_max) {
  const double lmin = fmin(c.md.lam[g.l], [&] {
    double m = 1e300;
    for (int k = 0; k <= c.md.L; ++k) m = fmin(m, c.md.lam[k]);
    return m;
  }());
  const double umax = 36.0 / zeta_min;
  const double wmax = fmin(2.0 / zeta_min, PI / fmax(rho_max, 1e-300));
  g.nq = count_panels(umax, wmax, lmin) * 16;
  g.nodes = c.arena.get<double>((size_t)g.ntypes * g.nq * 4);
  k_near_nodes<<<dim3((unsigned)((g.nq + 255) / 256), g.ntypes), 256, 0, c.stream>>>(c.md, g.l, g.a, g.ntypes, umax,
                                                                                     wmax, lmin, g.nodes, g.nq);
  LPB_LAUNCH();
  c.launches++;
}

// reaction class of a single-class table request: rho / h, zt / h - 1/2 and zs / h - 1/2 must be a
// class of the tables (rho^2 / h^2 one of the NRHO values, k_t + k_s < NKT)
static int class_of_request(double h, double rho, double zt, double zs) {
  const double r2 = (rho / h) * (rho / h);
  int ri = -1;
  for (int k = 0; k < NRHO; ++k)
    if (fabs(r2 - rho2_of(k)) < 1e-9) ri = k;
  const int kt = (int)llround(zt / h - 0.5), ks = (int)llround(zs / h - 0.5);
  const int kk = kk_index(kt, ks);
  if (ri < 0 || kk < 0 || fabs(zt / h - 0.5 - kt) > 1e-9 || fabs(zs / h - 0.5 - ks) > 1e-9)
    throw StatusError{LPBFMM_ERR_ARG};
  return ri * NKK + kk;
}

static RDesc one_class_desc(Ctx &c, int l, int a, int lp, int b, double h, int cls) {
  RDesc d;
  d.l = l; d.a = a; d.lp = lp; d.b = b; d.tau = 0; d.ntypes = 1; d.st = a == 1 ? -1 : 1; d.pad = 0;
  d.cls0 = cls; d.pad2 = 0;
  d.h = h; d.Lam = c.md.lam[l] * h; d.Lamp = c.md.lam[lp] * h;
  d.used = nullptr; d.stab = nullptr; d.coef = nullptr; d.dst = 0;
  return d;
}

void debug_stable(Ctx &c, int l, int a, int lp, int b, double h, double rho, double zt, double zs, int Kmax,
                  double *out) {
  // single class with the requested geometry: the quadrature + recurrence kernels of the FMM run
  // on a one-class descriptor whose table array holds that class alone
  const int cls = class_of_request(h, rho, zt, zs);
  const int KT = Kmax;
  const size_t TS = (size_t)(KT + 1) * (KT + 1) * 4;
  double *stab = nullptr;
  uint8_t *used = nullptr;
  RDesc *dr = nullptr;
  LPB_CUDA(cudaMalloc(&stab, sizeof(double) * TS));
  LPB_CUDA(cudaMalloc(&used, NREACT_CLS));
  LPB_CUDA(cudaMalloc(&dr, sizeof(RDesc)));
  LPB_CUDA(cudaMemsetAsync(stab, 0, sizeof(double) * TS, c.stream));
  std::vector<uint8_t> hu(NREACT_CLS, 0);
  hu[cls] = 1;
  LPB_CUDA(cudaMemcpyAsync(used, hu.data(), NREACT_CLS, cudaMemcpyHostToDevice, c.stream));
  RDesc d = one_class_desc(c, l, a, lp, b, h, cls);
  d.used = used;
  d.stab = stab;
  LPB_CUDA(cudaMemcpyAsync(dr, &d, sizeof(RDesc), cudaMemcpyHostToDevice, c.stream));
  const double tol = fmax(c.tol, 1e-16);
  NDesc N = node_desc(KT, tol, d.Lam, d.Lamp);
  NDesc *dn = nullptr;
  LPB_CUDA(cudaMalloc(&N.nodes, sizeof(double) * (size_t)N.nq * NDF));
  LPB_CUDA(cudaMalloc(&dn, sizeof(NDesc)));
  LPB_CUDA(cudaMemcpyAsync(dn, &N, sizeof(NDesc), cudaMemcpyHostToDevice, c.stream));
  k_stab_nodes<<<dim3((unsigned)((N.nq + 255) / 256), 1), 256, 0, c.stream>>>(dr, dn, c.md);
  LPB_LAUNCH();
  {
    const size_t sm = stab_quad_smem(KT);
    LPB_ATTR_ONCE(k_stab_quad, stab_quad_smem(KMAX_TAB));
    k_stab_quad<<<dim3(NREACT_CLS, 1), SQ_CHUNK, sm, c.stream>>>(dr, dn, KT, c.sfac);
    LPB_LAUNCH();
  }
  k_stab_recur<<<dim3(NREACT_CLS, 1), 32, 0, c.stream>>>(dr, KT);
  LPB_LAUNCH();
  std::vector<double> h_out(TS);
  LPB_CUDA(cudaMemcpyAsync(h_out.data(), stab, sizeof(double) * TS, cudaMemcpyDeviceToHost, c.stream));
  LPB_CUDA(cudaStreamSynchronize(c.stream));
  cudaFree(stab);
  cudaFree(used);
  cudaFree(dr);
  cudaFree(N.nodes);
  cudaFree(dn);
  // out[((K*(Kmax+1)) + d)*4 + ij] with ij = 2i + j
  for (size_t e = 0; e < TS; ++e) out[e] = h_out[e];
}


// ---------------------------------------------------------------------------------------
// Sommerfeld table of one class without any allocation.  Callers that cannot allocate: a
// host loop that has handed all free device memory to its own pool (cudaMalloc would fail),
// or one sharing the device with latency-critical streams (cudaMalloc and cudaFree may
// synchronize the whole device).  Every temporary lives in one fixed device array; its
// address is resolved per device with cudaGetSymbolAddress on the first call on that device.
// ---------------------------------------------------------------------------------------
constexpr size_t NA_TS = (size_t)(LPBFMM_NOALLOC_KMAX + 1) * (LPBFMM_NOALLOC_KMAX + 1) * 4;  // one class
constexpr size_t NA_NODES = (size_t)LPBFMM_NOALLOC_NQ * NDF;        // doubles
constexpr size_t NA_DESC = (sizeof(RDesc) + sizeof(NDesc) + NREACT_CLS + 7) / 8 + 8;
constexpr size_t NA_DOUBLES = NA_TS + NA_NODES + NA_DESC;           // ~1.8 MB in all
static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

static std::mutex g_noalloc_mu;
static double *g_noalloc_addr[LPB_MAX_DEVICES] = {};

// the scratch array's device address on the context's device (which must be current)
static double *noalloc_scratch(const Ctx &c) {
  int dev = -1;
  LPB_CUDA(cudaGetDevice(&dev));
  if (dev != c.device) throw StatusError{LPBFMM_ERR_ARG};
  std::lock_guard<std::mutex> lk(g_noalloc_mu);
  if (!g_noalloc_addr[c.device]) {
    void *p = nullptr;
    LPB_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
    g_noalloc_addr[c.device] = (double *)p;
  }
  return g_noalloc_addr[c.device];
}

// descriptors, class mask and the class's table are (re)initialised by one launch: the table
// entries the kernels do not write (d > K, and d >= 2 with K < d + 1) must read as zero
__global__ void k_noalloc_init(RDesc d, NDesc n, RDesc *rd, NDesc *nd, uint8_t *used, int cls, double *stab_cls,
                               int ts) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x, stride = gridDim.x * blockDim.x;
  if (t == 0) {
    *rd = d;
    *nd = n;
  }
  for (int e = t; e < NREACT_CLS; e += stride) used[e] = (e == cls) ? 1 : 0;
  for (int e = t; e < ts; e += stride) stab_cls[e] = 0.0;
}

void stable_noalloc(Ctx &c, int l, int a, int lp, int b, double h, double rho, double zt, double zs, int Kmax,
                    double *out) {
  if (Kmax > LPBFMM_NOALLOC_KMAX) throw StatusError{LPBFMM_ERR_UNSUPPORTED};
  const int cls = class_of_request(h, rho, zt, zs);
  const int KT = Kmax;
  const size_t TS = (size_t)(KT + 1) * (KT + 1) * 4;
  RDesc d = one_class_desc(c, l, a, lp, b, h, cls);
  NDesc N = node_desc(KT, fmax(c.tol, 1e-16), d.Lam, d.Lamp);
  if (N.nq > LPBFMM_NOALLOC_NQ) throw StatusError{LPBFMM_ERR_UNSUPPORTED};
  double *base = noalloc_scratch(c);
  double *stab = base, *nodes = base + NA_TS;
  RDesc *dr = (RDesc *)(nodes + NA_NODES);
  NDesc *dn = (NDesc *)((char *)dr + ((sizeof(RDesc) + 15) / 16) * 16);
  uint8_t *used = (uint8_t *)((char *)dn + ((sizeof(NDesc) + 15) / 16) * 16);
  d.used = used;
  d.stab = stab;
  N.nodes = nodes;
  k_noalloc_init<<<8, 256, 0, c.stream>>>(d, N, dr, dn, used, cls, stab, (int)TS);
  LPB_LAUNCH();
  k_stab_nodes<<<dim3((unsigned)((N.nq + 255) / 256), 1), 256, 0, c.stream>>>(dr, dn, c.md);
  LPB_LAUNCH();
  LPB_ATTR_ONCE(k_stab_quad, stab_quad_smem(KMAX_TAB));
  k_stab_quad<<<dim3(NREACT_CLS, 1), SQ_CHUNK, stab_quad_smem(KT), c.stream>>>(dr, dn, KT, c.sfac);
  LPB_LAUNCH();
  k_stab_recur<<<dim3(NREACT_CLS, 1), 32, 0, c.stream>>>(dr, KT);
  LPB_LAUNCH();
  LPB_CUDA(cudaMemcpyAsync(out, stab, sizeof(double) * TS, cudaMemcpyDeviceToDevice, c.stream));
}

}  // namespace lpb
