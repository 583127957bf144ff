// Device math for the layered-media screened-Coulomb FMM (Wang, Zhang & Cai, arXiv 2002.01334).
// Functions are __host__ __device__ so that the operator builders can also be unit-checked
// on a CPU; the library runs them on the GPU only.
#pragma once
#include <cmath>
#include <cstdint>

#ifdef __CUDACC__
#define LPB_HD __host__ __device__ __forceinline__
#else
#define LPB_HD inline
#endif

namespace lpb {

constexpr int PMAX = 16;                       // largest truncation order supported
constexpr int KHALF_MAX = (PMAX + 1) * (PMAX + 2) / 2;
constexpr int KMAX_TAB = 2 * PMAX + 3;         // largest S-table power (Sec. 3.5: n <= 2p+3)
constexpr int MAXLAYER = 9;
constexpr double PI = 3.14159265358979323846;

// index of (n, m) with 0 <= m <= n in the half representation
LPB_HD int hidx(int n, int m) { return n * (n + 1) / 2 + m; }
// index of (n, m) with -n <= m <= n in the full representation
LPB_HD int fidx(int n, int m) { return n * n + n + m; }

// (2n+1)!!
LPB_HD double dfact2(int n) {
  double r = 1.0;
  for (int k = 2 * n + 1; k > 1; k -= 2) r *= k;
  return r;
}

// Scaled modified spherical Bessel functions of the first kind,
//   it[n] = i_n(x) (2n+1)!! / x^n  (n = 0..nmax), x2 = x^2,
// from the power series of i_n at the two highest orders and the downward recurrence
//   it[n-1] = it[n] + x^2 it[n+1] / ((2n+1)(2n+3)),
// which only adds positive terms (stable for every x).
template <typename T>
LPB_HD T itilde_series(int n, T x2) {
  // sum_k (x^2/2)^k / (k! (2n+3)(2n+5)...(2n+2k+1))
  T s = T(1), t = T(1);
  for (int k = 1; k < 60; ++k) {
    t *= (x2 * T(0.5)) / (T(k) * T(2 * n + 2 * k + 1));
    s += t;
    if (t <= s * T(1e-17)) break;
  }
  return s;
}
template <typename T, int NMAX>
LPB_HD void itilde_all(T x2, T *it) {
  it[NMAX] = itilde_series<T>(NMAX, x2);
  it[NMAX - 1] = itilde_series<T>(NMAX - 1, x2);
#pragma unroll
  for (int n = NMAX - 1; n >= 1; --n) it[n - 1] = it[n] + x2 * it[n + 1] / T((2 * n + 1) * (2 * n + 3));
}

// Modified spherical Bessel functions with the paper's normalization (Sec. 3.1):
//   k_0(x) = (pi/2) e^{-x}/x,  k_{q+1} = k_{q-1} + (2q+1)/x k_q  (stable upward),
//   i_q(x) = x^q / (2q+1)!! * itilde_q(x).
LPB_HD void kbessel_all(double x, int qmax, double *k) {
  k[0] = 0.5 * PI * exp(-x) / x;
  if (qmax >= 1) k[1] = 0.5 * PI * exp(-x) * (1.0 + x) / (x * x);
  for (int q = 1; q < qmax; ++q) k[q + 1] = k[q - 1] + (2 * q + 1) / x * k[q];
}
LPB_HD void ibessel_all(double x, int qmax, double *iq) {
  // downward recurrence on scaled values, then rescale
  double top = itilde_series<double>(qmax, x * x);
  double top1 = (qmax >= 1) ? itilde_series<double>(qmax - 1, x * x) : top;
  iq[qmax] = top;
  if (qmax >= 1) iq[qmax - 1] = top1;
  for (int n = qmax - 1; n >= 1; --n) iq[n - 1] = iq[n] + x * x * iq[n + 1] / double((2 * n + 1) * (2 * n + 3));
  double xp = 1.0;
  for (int n = 0; n <= qmax; ++n) {
    iq[n] *= xp / dfact2(n);
    xp *= x;
  }
}

// Orthonormal associated Legendre functions with the Condon-Shortley phase,
//   Y_q^k(theta, phi) = Phat_q^k(cos theta) e^{i k phi},  k >= 0,
// stored P[q*(q+1)/2 + k] for q = 0..qmax (normalized three-term recurrences).
LPB_HD void phat_all(double x, int qmax, double *P) {
  const double s = sqrt(fmax(0.0, 1.0 - x * x));
  P[0] = 0.5 / sqrt(PI);
  for (int k = 1; k <= qmax; ++k) P[hidx(k, k)] = -sqrt((2.0 * k + 1.0) / (2.0 * k)) * s * P[hidx(k - 1, k - 1)];
  for (int k = 0; k < qmax; ++k) {
    P[hidx(k + 1, k)] = sqrt(2.0 * k + 3.0) * x * P[hidx(k, k)];
    for (int q = k + 2; q <= qmax; ++q) {
      const double a = sqrt((4.0 * q * q - 1.0) / (double(q) * q - double(k) * k));
      const double b = sqrt(((q - 1.0) * (q - 1.0) - double(k) * k) * (2.0 * q + 1.0) /
                            ((2.0 * q - 3.0) * (double(q) * q - double(k) * k)));
      P[hidx(q, k)] = a * x * P[hidx(q - 1, k)] - b * P[hidx(q - 2, k)];
    }
  }
}
// Phat_q^k for signed k (Phat_q^{-k} = (-1)^k Phat_q^k)
LPB_HD double phat_signed(const double *P, int q, int k) {
  if (k >= 0) return P[hidx(q, k)];
  return ((-k) & 1) ? -P[hidx(q, -k)] : P[hidx(q, -k)];
}

// ---------------------------------------------------------------------------------------
// Medium and layer response (Sec. 2.1).  Reaction part of the spectral Green's function in
// layer k: A_k e^{-lz_k (z-d_k)} + B_k e^{-lz_k (d_{k-1}-z)}; unit incident wave of the
// source layer l' at its bottom interface (b = 1) or top interface (b = 2) with amplitude
// 1/(2 eps' lz').  sigma^{1b}_{k l'} = 2 lz_k A_k, sigma^{2b}_{k l'} = 2 lz_k B_k.
// ---------------------------------------------------------------------------------------
struct Medium {
  int L;
  double d[MAXLAYER];
  double eps[MAXLAYER];
  double lam[MAXLAYER];
};

// Solves the 2L transmission equations by elimination with partial pivoting and returns the
// density of the requested target layer l and side a.
LPB_HD double layer_sigma(const Medium &md, double lr, int l, int a, int lp, int b) {
  const int L = md.L, n = 2 * L;
  double M[2 * (MAXLAYER - 1)][2 * (MAXLAYER - 1) + 1];  // augmented
  double lz[MAXLAYER], th[MAXLAYER];
  for (int k = 0; k <= L; ++k) lz[k] = sqrt(md.lam[k] * md.lam[k] + lr * lr);
  for (int k = 0; k <= L; ++k) th[k] = (k >= 1 && k < L) ? exp(-lz[k] * (md.d[k - 1] - md.d[k])) : 0.0;
  for (int r = 0; r < n; ++r)
    for (int c = 0; c <= n; ++c) M[r][c] = 0.0;
  // columns: A_k at k (k < L), B_k at L - 1 + k (k >= 1); rhs at column n
  for (int k = 0; k < L; ++k) {
    double *v = M[2 * k], *f = M[2 * k + 1];
    const double ea = md.eps[k] * lz[k], eb = md.eps[k + 1] * lz[k + 1];
    v[k] = 1.0;
    f[k] = -ea;
    if (k >= 1) { v[L - 1 + k] = th[k]; f[L - 1 + k] = ea * th[k]; }
    if (k + 1 < L) { v[k + 1] = -th[k + 1]; f[k + 1] = eb * th[k + 1]; }
    v[L + k] = -1.0;
    f[L + k] = -eb;
    if (b == 1 && lp == k) { v[n] = -0.5 / (md.eps[lp] * lz[lp]); f[n] = -0.5; }
    if (b == 2 && lp == k + 1) { v[n] = 0.5 / (md.eps[lp] * lz[lp]); f[n] = -0.5; }
  }
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(M[r][c]) > fabs(M[piv][c])) piv = r;
    if (piv != c)
      for (int k = c; k <= n; ++k) { double t = M[c][k]; M[c][k] = M[piv][k]; M[piv][k] = t; }
    const double inv = 1.0 / M[c][c];
    for (int r = c + 1; r < n; ++r) {
      const double f = M[r][c] * inv;
      if (f != 0.0)
        for (int k = c; k <= n; ++k) M[r][k] -= f * M[c][k];
    }
  }
  double x[2 * (MAXLAYER - 1)];
  for (int r = n - 1; r >= 0; --r) {
    double s = M[r][n];
    for (int k = r + 1; k < n; ++k) s -= M[r][k] * x[k];
    x[r] = s / M[r][r];
  }
  return (a == 1) ? 2.0 * lz[l] * x[l] : 2.0 * lz[l] * x[L - 1 + l];
}

// dense index of a source type (l', b): (l',1) -> 2l', (l',2) -> 2l'-1
LPB_HD int type_index(int lp, int b) { return b == 1 ? 2 * lp : 2 * lp - 1; }
LPB_HD void type_decode(int t, int &lp, int &b) {
  if (t & 1) { b = 2; lp = (t + 1) / 2; } else { b = 1; lp = t / 2; }
}

// image z of a source at zp in layer lp for target group (l, a), type b (Sec. 3.3)
LPB_HD double image_z(const Medium &md, int l, int a, int lp, int b, double zp) {
  if (a == 1) {
    const double dl = md.d[l];
    return (b == 1) ? dl - (zp - md.d[lp]) : dl - (md.d[lp - 1] - zp);
  }
  const double dl = md.d[l - 1];
  return (b == 1) ? dl + (zp - md.d[lp]) : dl + (md.d[lp - 1] - zp);
}

}  // namespace lpb
