/*
 * Oracle for the layered-media screened-Coulomb FMM: TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, FP64 CPU implementation of what the GPU path computes, written from
 * Wang, Zhang & Cai, "Fast Multipole Method for 3-D Linearized Poisson-Boltzmann
 * Equation in Layered Media" (arXiv 2002.01334).  Only tests/, __graft_entry__.smoke()
 * and bench.py's CPU-baseline leg may load it.  It shares no code with the CUDA path.
 *
 * Contents (each function cites the passage it follows):
 *   orc_layer_response   reaction densities sigma^{ab}_{l l'}(lambda_rho) from the
 *                        transmission conditions (Sec. 2.1, the interface conditions on
 *                        the densities; the paper gives only L=2 explicitly, so the general
 *                        L-layer densities are read as the solution of those conditions).
 *   orc_green_react      G^R_{l l'}(r,r') and grad_r by adaptive quadrature of the
 *                        alpha-integrated Sommerfeld integrals (Sec. 2.1, eqs.
 *                        greenfuncomponent / totaldensity).
 *   orc_direct           direct O(N^2) potential + field (Sec. 2.2, eq. potential1):
 *                        free-space e^{-lambda r}/(4 pi eps r) over j != i in the same
 *                        layer, reaction part over all j including j = i.
 *   orc_S_table          scaled Sommerfeld integrals S^K S_{K d, ij} by direct
 *                        quadrature of their definition (Sec. 3.5, eq. M2Ltable and its
 *                        scaled form), used to pin the table recurrence.
 *   orc_image_z          equivalent polarization coordinates (Sec. 3.3, eq.
 *                        eqpolarizedsource).
 *   orc_tree_*           uniform-depth octree and interaction lists of one target group
 *                        (root bisected by the interface, Sec. 3.5 tree rule), for the
 *                        bit-exact tree/list parity test.
 *
 * Parity: every function above is pinned by tests/test_oracle_pins.py except where noted
 * there; orc_green_react_ab is also the limit that the truncated reaction ME, LE and M2L of
 * Sec. 3.4 (expansions.py) must converge to, in tests/test_expansion_pins.py.
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no FMA contraction so that the
 * tree keys are the exact IEEE results of the stated formula).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXL 9 /* at most 8 interfaces, 9 layers */

typedef struct {
  int L;                 /* number of interfaces */
  double d[ORC_MAXL];    /* d[0] > d[1] > ... > d[L-1] */
  double eps[ORC_MAXL];  /* eps[0..L] */
  double lam[ORC_MAXL];  /* lambda[0..L] */
} orc_medium;

static const double ORC_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------------------ */
/* Layer response.  In layer k the reaction part of the spectral Green's function is    */
/*   u_k(z) = A_k exp(-lz_k (z - d_k)) + B_k exp(-lz_k (d_{k-1} - z)),                   */
/* with A_L and B_0 absent (decay at -inf / +inf).  A unit incident wave               */
/*   b = 1: exp(-lz' (d_l' - z)) / (2 eps' lz') hitting interface d_l' from above,       */
/*   b = 2: exp(-lz' (z - d_{l'-1})) / (2 eps' lz') hitting d_{l'-1} from below,         */
/* enforces continuity of u and eps du/dz at every interface.  The densities of the     */
/* paper are sigma^{1b}_{k l'} = 2 lz_k A_k and sigma^{2b}_{k l'} = 2 lz_k B_k, so that  */
/*   u^{ab}_{l l'} = (1/4 pi) int lr J0(lr rho) e^{-lz_l h_a} e^{-lz_l' h'_b} sigma / lz_l */
/* ------------------------------------------------------------------------------------ */
static int solve_dense(int n, double *M, double *rhs) {
  /* Gaussian elimination with partial pivoting, M row-major n x n */
  for (int c = 0; c < n; ++c) {
    int piv = c;
    double best = fabs(M[c * n + c]);
    for (int r = c + 1; r < n; ++r)
      if (fabs(M[r * n + c]) > best) { best = fabs(M[r * n + c]); piv = r; }
    if (best == 0.0) return -1;
    if (piv != c) {
      for (int k = 0; k < n; ++k) { double t = M[c * n + k]; M[c * n + k] = M[piv * n + k]; M[piv * n + k] = t; }
      double t = rhs[c]; rhs[c] = rhs[piv]; rhs[piv] = t;
    }
    for (int r = c + 1; r < n; ++r) {
      double f = M[r * n + c] / M[c * n + c];
      if (f == 0.0) continue;
      for (int k = c; k < n; ++k) M[r * n + k] -= f * M[c * n + k];
      rhs[r] -= f * rhs[c];
    }
  }
  for (int r = n - 1; r >= 0; --r) {
    double s = rhs[r];
    for (int k = r + 1; k < n; ++k) s -= M[r * n + k] * rhs[k];
    rhs[r] = s / M[r * n + r];
  }
  return 0;
}

int orc_layer_response(const orc_medium *md, double lr, int lp, int b, double *s1, double *s2) {
  const int L = md->L;
  const int n = 2 * L;
  double M[4 * ORC_MAXL * ORC_MAXL];
  double rhs[2 * ORC_MAXL];
  double lz[ORC_MAXL], t[ORC_MAXL];
  if (L < 1 || L > ORC_MAXL - 1) return -1;
  if ((b == 1 && lp == L) || (b == 2 && lp == 0)) return -1;
  for (int k = 0; k <= L; ++k) lz[k] = sqrt(md->lam[k] * md->lam[k] + lr * lr);
  for (int k = 0; k <= L; ++k) t[k] = (k >= 1 && k <= L - 1) ? md->d[k - 1] - md->d[k] : 0.0;
  memset(M, 0, sizeof(double) * n * n);
  memset(rhs, 0, sizeof(double) * n);
  /* unknown index: A_k -> k (k = 0..L-1); B_k -> L-1+k (k = 1..L) */
#define IA(k) (k)
#define IB(k) (L - 1 + (k))
  for (int k = 0; k < L; ++k) {
    const int r0 = 2 * k, r1 = 2 * k + 1;
    const double ek = exp(-lz[k] * t[k]);         /* used only when layer k has a top interface */
    const double ek1 = exp(-lz[k + 1] * t[k + 1]); /* used only when layer k+1 has a bottom one */
    /* value continuity: u_k(d_k) - u_{k+1}(d_k) = rhs */
    M[r0 * n + IA(k)] += 1.0;
    if (k >= 1) M[r0 * n + IB(k)] += ek;
    if (k + 1 <= L - 1) M[r0 * n + IA(k + 1)] -= ek1;
    M[r0 * n + IB(k + 1)] -= 1.0;
    /* flux continuity: eps_k u_k'(d_k) - eps_{k+1} u_{k+1}'(d_k) = rhs */
    M[r1 * n + IA(k)] += -md->eps[k] * lz[k];
    if (k >= 1) M[r1 * n + IB(k)] += md->eps[k] * lz[k] * ek;
    if (k + 1 <= L - 1) M[r1 * n + IA(k + 1)] -= -md->eps[k + 1] * lz[k + 1] * ek1;
    M[r1 * n + IB(k + 1)] -= md->eps[k + 1] * lz[k + 1];
    /* incident wave: value 1/(2 eps' lz'), flux +1/2 (upper side, b=1) or -1/2 (lower side, b=2) */
    if (b == 1 && lp == k) { rhs[r0] -= 1.0 / (2.0 * md->eps[lp] * lz[lp]); rhs[r1] -= 0.5; }
    if (b == 2 && lp == k + 1) { rhs[r0] += 1.0 / (2.0 * md->eps[lp] * lz[lp]); rhs[r1] -= 0.5; }
  }
  if (solve_dense(n, M, rhs)) return -2;
  for (int k = 0; k <= L; ++k) {
    s1[k] = (k <= L - 1) ? 2.0 * lz[k] * rhs[IA(k)] : 0.0;
    s2[k] = (k >= 1) ? 2.0 * lz[k] * rhs[IB(k)] : 0.0;
  }
#undef IA
#undef IB
  return 0;
}

/* layer of a z coordinate: 0 = top (z > d_0) ... L = bottom (z < d_{L-1}) */
int orc_layer_of(const orc_medium *md, double z) {
  int l = 0;
  while (l < md->L && z < md->d[l]) ++l;
  return l;
}

/* distance-like exponents of the two target waves and two source waves (Sec. 2.2 eq. zexponential) */
static int target_h(const orc_medium *md, int l, double z, double h[3]) {
  /* h[1] = z - d_l (a=1, needs l < L), h[2] = d_{l-1} - z (a=2, needs l > 0); returns mask */
  int mask = 0;
  if (l < md->L) { h[1] = z - md->d[l]; mask |= 2; }
  if (l > 0) { h[2] = md->d[l - 1] - z; mask |= 4; }
  return mask;
}
static int source_h(const orc_medium *md, int lp, double zp, double h[3]) {
  /* h[1] = z' - d_l' (b=1, l' < L), h[2] = d_{l'-1} - z' (b=2, l' > 0) */
  int mask = 0;
  if (lp < md->L) { h[1] = zp - md->d[lp]; mask |= 2; }
  if (lp > 0) { h[2] = md->d[lp - 1] - zp; mask |= 4; }
  return mask;
}

/* ------------------------------------------------------------------------------------ */
/* Gauss-Legendre nodes by Newton iteration on P_n (no tabulated constants).            */
/* ------------------------------------------------------------------------------------ */
#define GLN 16
static double GLX[GLN], GLW[GLN];
static int gl_ready = 0;
static void gl_init(void) {
  if (gl_ready) return;
  for (int i = 0; i < GLN; ++i) {
    double x = cos(ORC_PI * (i + 0.75) / (GLN + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= GLN; ++k) { double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
      double dp = GLN * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (fabs(dx) < 1e-16) {
        p0 = 1.0; p1 = x;
        for (int k = 2; k <= GLN; ++k) { double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
        dp = GLN * (x * p1 - p0) / (x * x - 1.0);
        break;
      }
    }
    double p0 = 1.0, p1 = x;
    for (int k = 2; k <= GLN; ++k) { double p2 = ((2 * k - 1) * x * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
    double dp = GLN * (x * p1 - p0) / (x * x - 1.0);
    GLX[i] = x;
    GLW[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
  gl_ready = 1;
}

/* vector-valued adaptive integration: compare one 16-point panel with two halves */
typedef void (*vfun)(double x, void *ctx, int nv, double *out);
static void gl_panel(vfun f, void *ctx, int nv, double a, double b, double *out) {
  double tmp[64];
  const double hw = 0.5 * (b - a), c = 0.5 * (a + b);
  for (int v = 0; v < nv; ++v) out[v] = 0.0;
  for (int i = 0; i < GLN; ++i) {
    f(c + hw * GLX[i], ctx, nv, tmp);
    for (int v = 0; v < nv; ++v) out[v] += GLW[i] * hw * tmp[v];
  }
}
static void adapt(vfun f, void *ctx, int nv, double a, double b, const double *whole, double tol, int depth,
                  double *out) {
  double l[64], r[64];
  const double m = 0.5 * (a + b);
  gl_panel(f, ctx, nv, a, m, l);
  gl_panel(f, ctx, nv, m, b, r);
  double err = 0.0;
  for (int v = 0; v < nv; ++v) err = fmax(err, fabs(l[v] + r[v] - whole[v]));
  if (err <= tol || depth >= 40) {
    for (int v = 0; v < nv; ++v) out[v] += l[v] + r[v];
    return;
  }
  adapt(f, ctx, nv, a, m, l, 0.5 * tol, depth + 1, out);
  adapt(f, ctx, nv, m, b, r, 0.5 * tol, depth + 1, out);
}
/* integrate over [0, xmax] in panels of width <= w, each refined adaptively */
static void integrate(vfun f, void *ctx, int nv, double xmax, double w, double lmin, double abstol, double *out) {
  gl_init();
  int np = 0;
  for (double x = 0.0; x < xmax; ++np) x += fmin(w, 0.5 * (lmin + x));
  for (int v = 0; v < nv; ++v) out[v] = 0.0;
  double x = 0.0;
  for (int k = 0; k < np; ++k) {
    double dw = fmin(w, 0.5 * (lmin + x));
    if (x + dw > xmax) dw = xmax - x;
    double whole[64];
    gl_panel(f, ctx, nv, x, x + dw, whole);
    adapt(f, ctx, nv, x, x + dw, whole, abstol / np, 0, out);
    x += dw;
  }
}

/* ------------------------------------------------------------------------------------ */
/* Reaction Green's function and its target gradient, adaptive quadrature (definition).  */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  const orc_medium *md;
  int l, lp, tmask, smask;
  double ht[3], hs[3], rho;
} gr_ctx;
static int gr_amask = 6, gr_bmask = 6; /* bits 1<<a, 1<<b of the components kept */

static void gr_integrand(double lr, void *vctx, int nv, double *out) {
  (void)nv;
  gr_ctx *c = (gr_ctx *)vctx;
  const orc_medium *md = c->md;
  double s1[ORC_MAXL], s2[ORC_MAXL];
  const double lz = sqrt(md->lam[c->l] * md->lam[c->l] + lr * lr);
  const double lzp = sqrt(md->lam[c->lp] * md->lam[c->lp] + lr * lr);
  double val = 0.0, dz = 0.0;
  for (int b = 1; b <= 2; ++b) {
    if (!(c->smask & (1 << b))) continue;
    orc_layer_response(md, lr, c->lp, b, s1, s2);
    const double es = exp(-lzp * c->hs[b]);
    for (int a = 1; a <= 2; ++a) {
      if (!(c->tmask & (1 << a))) continue;
      const double sg = (a == 1) ? s1[c->l] : s2[c->l];
      const double term = sg * exp(-lz * c->ht[a]) * es;
      val += term;
      dz += (a == 1 ? 1.0 : -1.0) * lz * term; /* -d/dz of e^{-lz h_a}: h_1 = z - d, h_2 = d - z */
    }
  }
  const double x = lr * c->rho;
  const double j0v = j0(x);
  /* J1(x)/rho with the rho -> 0 limit lr/2 */
  const double j1r = (c->rho > 0.0) ? j1(x) / c->rho : 0.5 * lr;
  const double g = lr / lz / (4.0 * ORC_PI);
  out[0] = g * val * j0v;
  out[1] = g * val * lr * j1r; /* field_x = (x - x') * out[1] */
  out[2] = g * dz * j0v;       /* field_z */
}

/* G^R_{l l'}(r, r') (potential) and field = -grad_r G^R.  tol: absolute tolerance scale
 * relative to 1/(4 pi Delta).  Returns 0 on success. */
int orc_green_react(const orc_medium *md, int l, const double *r, int lp, const double *rp, double tol,
                    double *phi, double *field) {
  gr_ctx c;
  c.md = md; c.l = l; c.lp = lp;
  c.tmask = target_h(md, l, r[2], c.ht) & gr_amask;
  c.smask = source_h(md, lp, rp[2], c.hs) & gr_bmask;
  const double dx = r[0] - rp[0], dy = r[1] - rp[1];
  c.rho = sqrt(dx * dx + dy * dy);
  double dmin = 1e300;
  for (int a = 1; a <= 2; ++a)
    for (int b = 1; b <= 2; ++b)
      if ((c.tmask & (1 << a)) && (c.smask & (1 << b))) dmin = fmin(dmin, c.ht[a] + c.hs[b]);
  if (dmin > 1e299) { *phi = 0.0; field[0] = field[1] = field[2] = 0.0; return 0; }
  if (!(dmin > 0.0)) return -1;
  const double xmax = 60.0 / dmin;
  double w = 2.0 / dmin;
  if (c.rho > 0.0) w = fmin(w, ORC_PI / c.rho);
  double out[3];
  integrate(gr_integrand, &c, 3, xmax, w, fmin(md->lam[l], md->lam[lp]), tol / (4.0 * ORC_PI * dmin * dmin), out);
  *phi = out[0];
  field[0] = dx * out[1];
  field[1] = dy * out[1];
  field[2] = out[2];
  return 0;
}

/* One reaction component u^{ab}_{l l'} (Sec. 2.2 eq. generalcomponents): a, b select the
 * target-side and source-side waves. */
int orc_green_react_ab(const orc_medium *md, int l, const double *r, int lp, const double *rp, int a, int b,
                       double tol, double *phi, double *field) {
  gr_amask = 1 << a;
  gr_bmask = 1 << b;
  const int rc = orc_green_react(md, l, r, lp, rp, tol, phi, field);
  gr_amask = gr_bmask = 6;
  return rc;
}

/* ------------------------------------------------------------------------------------ */
/* Direct sum (Sec. 2.2, eq. potential1 / totalinteraction) with a fixed composite rule   */
/* per (target, source layer), validated against orc_green_react by the pin tests.       */
/* parts: bit 0 = free-space part, bit 1 = reaction part.                                */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  int nq;
  double *x, *w;
} rule_t;

/* Composite 16-point rule on [0, xmax]: panel width min(wmax, (lmin + x)/2) so that the
 * panels near the origin resolve the branch points of lz = sqrt(lam^2 + lr^2) at lr = +-i lam. */
static void make_rule(double xmax, double wmax, double lmin, rule_t *R) {
  gl_init();
  int np = 0;
  for (double x = 0.0; x < xmax; ++np) x += fmin(wmax, 0.5 * (lmin + x));
  R->nq = np * GLN;
  R->x = (double *)malloc(sizeof(double) * R->nq);
  R->w = (double *)malloc(sizeof(double) * R->nq);
  double x = 0.0;
  for (int k = 0; k < np; ++k) {
    double dw = fmin(wmax, 0.5 * (lmin + x));
    if (x + dw > xmax) dw = xmax - x;
    for (int i = 0; i < GLN; ++i) {
      R->x[k * GLN + i] = x + 0.5 * dw * (GLX[i] + 1.0);
      R->w[k * GLN + i] = 0.5 * dw * GLW[i];
    }
    x += dw;
  }
}

int orc_direct(const orc_medium *md, int64_t n, const double *q, const double *xyz, const int *layer, int64_t nt,
               const int64_t *tidx, int parts, int nodes_per_unit, double *phi, double *field) {
  const int L = md->L;
  /* per-layer source lists and the extreme source exponents */
  int64_t *cnt = (int64_t *)calloc(L + 1, sizeof(int64_t));
  double hmin_s[ORC_MAXL][3];
  double xlo = 1e300, xhi = -1e300, ylo = 1e300, yhi = -1e300;
  for (int k = 0; k <= L; ++k) hmin_s[k][1] = hmin_s[k][2] = 1e300;
  for (int64_t j = 0; j < n; ++j) {
    const int lp = layer[j];
    cnt[lp]++;
    double hs[3];
    int sm = source_h(md, lp, xyz[3 * j + 2], hs);
    for (int b = 1; b <= 2; ++b)
      if (sm & (1 << b)) hmin_s[lp][b] = fmin(hmin_s[lp][b], hs[b]);
    xlo = fmin(xlo, xyz[3 * j]); xhi = fmax(xhi, xyz[3 * j]);
    ylo = fmin(ylo, xyz[3 * j + 1]); yhi = fmax(yhi, xyz[3 * j + 1]);
  }
  const double rhomax = sqrt((xhi - xlo) * (xhi - xlo) + (yhi - ylo) * (yhi - ylo));
  int status = 0;
  gl_init();
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t it = 0; it < nt; ++it) {
    const int64_t i = tidx ? tidx[it] : it;
    const int l = layer[i];
    const double *r = xyz + 3 * i;
    double acc = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
    if (parts & 1) {
      const double lam = md->lam[l], eps = md->eps[l];
      for (int64_t j = 0; j < n; ++j) {
        if (j == i || layer[j] != l) continue;
        const double dx = r[0] - xyz[3 * j], dy = r[1] - xyz[3 * j + 1], dz = r[2] - xyz[3 * j + 2];
        const double R = sqrt(dx * dx + dy * dy + dz * dz);
        const double e = exp(-lam * R) / (4.0 * ORC_PI * eps * R);
        acc += q[j] * e;
        const double f = q[j] * e * (1.0 + lam * R) / (R * R);
        ex += f * dx; ey += f * dy; ez += f * dz;
      }
    }
    if (parts & 2) {
      double ht[3];
      const int tm = target_h(md, l, r[2], ht);
      for (int lp = 0; lp <= L; ++lp) {
        if (!cnt[lp]) continue;
        double dmin = 1e300;
        for (int a = 1; a <= 2; ++a)
          for (int b = 1; b <= 2; ++b)
            if ((tm & (1 << a)) && hmin_s[lp][b] < 1e299) dmin = fmin(dmin, ht[a] + hmin_s[lp][b]);
        if (!(dmin > 0.0)) { status = -1; continue; }
        rule_t R;
        double w = 2.0 / dmin;
        if (rhomax > 0.0) w = fmin(w, ORC_PI / rhomax);
        make_rule(60.0 / dmin, w * 16.0 / (double)nodes_per_unit, fmin(md->lam[l], md->lam[lp]), &R);
        /* per-node target factors and densities */
        double *ft = (double *)malloc(sizeof(double) * R.nq * 8);
        for (int k = 0; k < R.nq; ++k) {
          const double lr = R.x[k];
          const double lz = sqrt(md->lam[l] * md->lam[l] + lr * lr);
          const double lzp = sqrt(md->lam[lp] * md->lam[lp] + lr * lr);
          double s1b[ORC_MAXL], s2b[ORC_MAXL];
          for (int b = 1; b <= 2; ++b) {
            double *slot = ft + 8 * k + 4 * (b - 1);
            slot[0] = slot[1] = slot[2] = 0.0;
            if (lp == (b == 1 ? L : 0)) continue;
            orc_layer_response(md, lr, lp, b, s1b, s2b);
            double v = 0.0, vz = 0.0;
            for (int a = 1; a <= 2; ++a) {
              if (!(tm & (1 << a))) continue;
              const double sg = (a == 1) ? s1b[l] : s2b[l];
              const double t = sg * exp(-lz * ht[a]);
              v += t;
              vz += (a == 1 ? 1.0 : -1.0) * lz * t;
            }
            const double g = R.w[k] * lr / lz / (4.0 * ORC_PI);
            slot[0] = g * v; slot[1] = g * vz; slot[2] = lzp;
          }
        }
        for (int64_t j = 0; j < n; ++j) {
          if (layer[j] != lp) continue;
          double hs[3];
          const int sm = source_h(md, lp, xyz[3 * j + 2], hs);
          const double dx = r[0] - xyz[3 * j], dy = r[1] - xyz[3 * j + 1];
          const double rho = sqrt(dx * dx + dy * dy);
          double sv = 0.0, sr = 0.0, sz = 0.0;
          /* this pair's integrand decays like exp(-lr * dpair): stop where it is below e^-36 */
          double dpair = 1e300;
          for (int a = 1; a <= 2; ++a)
            for (int b = 1; b <= 2; ++b)
              if ((tm & (1 << a)) && (sm & (1 << b))) dpair = fmin(dpair, ht[a] + hs[b]);
          const double xcut = 36.0 / dpair;
          for (int k = 0; k < R.nq; ++k) {
            const double lr = R.x[k];
            if (lr > xcut) break;
            double e = 0.0, ez2 = 0.0;
            for (int b = 1; b <= 2; ++b) {
              if (!(sm & (1 << b))) continue;
              const double *slot = ft + 8 * k + 4 * (b - 1);
              const double es = exp(-slot[2] * hs[b]);
              e += slot[0] * es;
              ez2 += slot[1] * es;
            }
            const double x = lr * rho;
            const double j0v = j0(x);
            const double j1r = rho > 0.0 ? j1(x) / rho : 0.5 * lr;
            sv += e * j0v;
            sr += e * lr * j1r;
            sz += ez2 * j0v;
          }
          acc += q[j] * sv;
          ex += q[j] * dx * sr;
          ey += q[j] * dy * sr;
          ez += q[j] * sz;
        }
        free(ft);
        free(R.x);
        free(R.w);
      }
    }
    phi[it] = acc;
    if (field) { field[3 * it] = ex; field[3 * it + 1] = ey; field[3 * it + 2] = ez; }
  }
  free(cnt);
  return status;
}

/* ------------------------------------------------------------------------------------ */
/* Scaled Sommerfeld integrals (Sec. 3.5, eq. M2Ltable, scaled by S^K with S = h):       */
/*   S^K S_{K d, ij} = h^K / sqrt((K+d)!(K-d)!) int lr^K J_d(lr rho) Z sigma / lz_l        */
/*                      (lam_l / lz_l)^i (lam_l' / lz_l')^j d lr,                         */
/* Z = exp(-lz_l zt - lz_l' zs), zt/zs = distances of target/source centre to the         */
/* interface of the component.  out[((K*(Kmax+1))+d)*4 + 2i + j], d = 0..K.               */
/* ------------------------------------------------------------------------------------ */
typedef struct {
  const orc_medium *md;
  int l, lp, a, b, K, d;
  double zt, zs, rho, h;
} st_ctx;
static void st_integrand(double lr, void *vctx, int nv, double *out) {
  (void)nv;
  st_ctx *c = (st_ctx *)vctx;
  const orc_medium *md = c->md;
  double s1[ORC_MAXL], s2[ORC_MAXL];
  orc_layer_response(md, lr, c->lp, c->b, s1, s2);
  const double sg = (c->a == 1) ? s1[c->l] : s2[c->l];
  const double lz = sqrt(md->lam[c->l] * md->lam[c->l] + lr * lr);
  const double lzp = sqrt(md->lam[c->lp] * md->lam[c->lp] + lr * lr);
  const double base = pow(lr * c->h, c->K) * jn(c->d, lr * c->rho) * exp(-lz * c->zt - lzp * c->zs) * sg / lz;
  out[0] = base;
  out[1] = base * md->lam[c->lp] / lzp;
  out[2] = base * md->lam[c->l] / lz;
  out[3] = base * md->lam[c->l] / lz * md->lam[c->lp] / lzp;
}
int orc_S_table(const orc_medium *md, int l, int lp, int a, int b, double h, double rho, double zt, double zs,
                int Kmax, double tol, double *out) {
  st_ctx c;
  c.md = md; c.l = l; c.lp = lp; c.a = a; c.b = b; c.zt = zt; c.zs = zs; c.rho = rho; c.h = h;
  const double dsum = zt + zs;
  if (!(dsum > 0.0)) return -1;
  for (int K = 0; K <= Kmax; ++K)
    for (int d = 0; d <= K; ++d) {
      c.K = K; c.d = d;
      /* lr^K e^{-lr dsum} peaks at K/dsum; integrate well past it */
      const double xmax = (K + 60.0 + 4.0 * sqrt((double)K + 1.0)) / dsum;
      double w = 2.0 / dsum;
      if (rho > 0.0) w = fmin(w, ORC_PI / rho);
      double v[4];
      const double peak = (K > 0) ? pow(h * K / dsum, K) * exp(-(double)K) : 1.0;
      integrate(st_integrand, &c, 4, xmax, w, fmin(md->lam[l], md->lam[lp]), tol * peak / dsum, v);
      const double nrm = 1.0 / sqrt(tgamma(K + d + 1.0) * tgamma(K - d + 1.0));
      /* ij order: (i,j) = (0,0),(0,1),(1,0),(1,1) -> out index 2i+j */
      for (int ij = 0; ij < 4; ++ij) out[((size_t)K * (Kmax + 1) + d) * 4 + ij] = v[ij] * nrm;
    }
  return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Equivalent polarization coordinates (Sec. 3.3, eq. eqpolarizedsource).                */
/* ------------------------------------------------------------------------------------ */
double orc_image_z(const orc_medium *md, int l, int a, int lp, int b, double zp) {
  const double dtop = (l > 0) ? md->d[l - 1] : 0.0, dbot = (l < md->L) ? md->d[l] : 0.0;
  const double sbot = (lp < md->L) ? md->d[lp] : 0.0, stop = (lp > 0) ? md->d[lp - 1] : 0.0;
  if (a == 1) return (b == 1) ? dbot - (zp - sbot) : dbot - (stop - zp);
  return (b == 1) ? dtop + (zp - sbot) : dtop + (stop - zp);
}

/* ------------------------------------------------------------------------------------ */
/* Uniform-depth octree of one target group g = (l, a) and its interaction lists.        */
/* Root: cube centred at (cx, cy, d_I) with d_I the interface of the group (d_l for a=1, */
/* d_{l-1} for a=2), half-size H = max over targets and images of max(|x-cx|, |y-cy|,    */
/* |z-d_I|) * (1 + 2^-20); cx, cy = midpoints of the x and y ranges of all charges.      */
/* Integer cell of a point at depth D: i = floor((x - (c - H)) * (2^D / (2H))), clamped. */
/* Morton key: bit k of ix -> bit 3k+2, iy -> 3k+1, iz -> 3k.                            */
/* ------------------------------------------------------------------------------------ */
static uint64_t spread3(uint64_t v) {
  uint64_t r = 0;
  for (int k = 0; k < 21; ++k) r |= ((v >> k) & 1ull) << (3 * k);
  return r;
}
uint64_t orc_morton(int ix, int iy, int iz) {
  return (spread3((uint64_t)ix) << 2) | (spread3((uint64_t)iy) << 1) | spread3((uint64_t)iz);
}
static int cell(double x, double x0, double s, int nmax) {
  double t = floor((x - x0) * s);
  if (t < 0.0) t = 0.0;
  if (t > (double)(nmax - 1)) t = (double)(nmax - 1);
  return (int)t;
}

/* root of group (l, a): out[0..3] = cx, cy, cz, H */
void orc_tree_root(const orc_medium *md, int64_t n, const double *xyz, const int *layer, int l, int a,
                   double *out) {
  const double dI = (a == 1) ? md->d[l] : md->d[l - 1];
  double xlo = 1e300, xhi = -1e300, ylo = 1e300, yhi = -1e300;
  for (int64_t j = 0; j < n; ++j) {
    xlo = fmin(xlo, xyz[3 * j]); xhi = fmax(xhi, xyz[3 * j]);
    ylo = fmin(ylo, xyz[3 * j + 1]); yhi = fmax(yhi, xyz[3 * j + 1]);
  }
  const double cx = 0.5 * (xlo + xhi), cy = 0.5 * (ylo + yhi);
  double H = 0.0;
  for (int64_t j = 0; j < n; ++j) {
    const double dx = fabs(xyz[3 * j] - cx), dy = fabs(xyz[3 * j + 1] - cy);
    H = fmax(H, fmax(dx, dy));
    const int lp = layer[j];
    if (lp == l) H = fmax(H, fabs(xyz[3 * j + 2] - dI));
    for (int b = 1; b <= 2; ++b) {
      if ((b == 1 && lp == md->L) || (b == 2 && lp == 0)) continue;
      H = fmax(H, fabs(orc_image_z(md, l, a, lp, b, xyz[3 * j + 2]) - dI));
    }
  }
  out[0] = cx; out[1] = cy; out[2] = dI; out[3] = H * (1.0 + 1.0 / 1048576.0);
}

/* Keys at depth D of the group's targets (kind 0) or images (kind 1: every valid (l',b) of
 * every charge, ordered by charge then b).  Returns the number of points written. */
int64_t orc_tree_keys(const orc_medium *md, int64_t n, const double *xyz, const int *layer, int l, int a, int D,
                      const double *root, int kind, uint64_t *keys, int64_t *src, int *type) {
  const double H = root[3];
  const double s = (double)(1 << D) / (2.0 * H);
  const double x0 = root[0] - H, y0 = root[1] - H, z0 = root[2] - H;
  const int nc = 1 << D;
  int64_t c = 0;
  for (int64_t j = 0; j < n; ++j) {
    const int lp = layer[j];
    if (kind == 0) {
      if (lp != l) continue;
      keys[c] = orc_morton(cell(xyz[3 * j], x0, s, nc), cell(xyz[3 * j + 1], y0, s, nc),
                           cell(xyz[3 * j + 2], z0, s, nc));
      if (src) src[c] = j;
      if (type) type[c] = 0;
      ++c;
    } else {
      for (int b = 1; b <= 2; ++b) {
        if ((b == 1 && lp == md->L) || (b == 2 && lp == 0)) continue;
        const double zi = orc_image_z(md, l, a, lp, b, xyz[3 * j + 2]);
        keys[c] = orc_morton(cell(xyz[3 * j], x0, s, nc), cell(xyz[3 * j + 1], y0, s, nc), cell(zi, z0, s, nc));
        if (src) src[c] = j;
        if (type) type[c] = 2 * lp + (b - 1);
        ++c;
      }
    }
  }
  return c;
}

static int cmp_u64(const void *x, const void *y) {
  const uint64_t a = *(const uint64_t *)x, b = *(const uint64_t *)y;
  return (a > b) - (a < b);
}
/* sorted unique keys of level lev (key >> 3(D-lev)); returns count */
int64_t orc_level_boxes(const uint64_t *keys, int64_t np, int D, int lev, uint64_t *boxes) {
  uint64_t *tmp = (uint64_t *)malloc(sizeof(uint64_t) * (np ? np : 1));
  for (int64_t i = 0; i < np; ++i) tmp[i] = keys[i] >> (3 * (D - lev));
  qsort(tmp, np, sizeof(uint64_t), cmp_u64);
  int64_t u = 0;
  for (int64_t i = 0; i < np; ++i)
    if (i == 0 || tmp[i] != tmp[i - 1]) boxes[u++] = tmp[i];
  free(tmp);
  return u;
}
static void unspread(uint64_t key, int *ix, int *iy, int *iz) {
  int x = 0, y = 0, z = 0;
  for (int k = 0; k < 21; ++k) {
    z |= (int)((key >> (3 * k)) & 1) << k;
    y |= (int)((key >> (3 * k + 1)) & 1) << k;
    x |= (int)((key >> (3 * k + 2)) & 1) << k;
  }
  *ix = x; *iy = y; *iz = z;
}
static int64_t find_box(const uint64_t *boxes, int64_t nb, uint64_t key) {
  int64_t lo = 0, hi = nb - 1;
  while (lo <= hi) {
    const int64_t m = (lo + hi) / 2;
    if (boxes[m] == key) return m;
    if (boxes[m] < key) lo = m + 1; else hi = m - 1;
  }
  return -1;
}
static int fdiv2(int v) { return v >= 0 ? v / 2 : -((-v + 1) / 2); }
/* Interaction lists at level lev between target boxes tb[0..nt) and source boxes sb[0..ns), for a
 * separation of ws boxes (ws = 1: one-box, ws = 2: two-box; the traditional FMM list rule that
 * Sec. 3.5 builds Algorithm 1 on, with the interaction list of a box made of the children of its
 * parent's neighbours that are not its own neighbours):
 * kind 0: far list (V): |d|_inf > ws and the parents are within ws of each other (|parent offset|_inf <= ws).
 * kind 1: near list (U): |d|_inf <= ws.
 * Offsets are visited dx outermost, then dy, then dz, each ascending from -(2 ws + 1) to 2 ws + 1.
 * off[nt+1] CSR offsets, idx[] source box indices.  Returns total entries. */
int64_t orc_lists(const uint64_t *tb, int64_t nt, const uint64_t *sb, int64_t ns, int lev, int kind, int ws,
                  int64_t *off, int64_t *idx) {
  int64_t c = 0;
  const int nc = 1 << lev, R = 2 * ws + 1;
  for (int64_t t = 0; t < nt; ++t) {
    off[t] = c;
    int ix, iy, iz;
    unspread(tb[t], &ix, &iy, &iz);
    for (int dx = -R; dx <= R; ++dx)
      for (int dy = -R; dy <= R; ++dy)
        for (int dz = -R; dz <= R; ++dz) {
          const int jx = ix + dx, jy = iy + dy, jz = iz + dz;
          if (jx < 0 || jy < 0 || jz < 0 || jx >= nc || jy >= nc || jz >= nc) continue;
          const int adist = abs(dx) > abs(dy) ? (abs(dx) > abs(dz) ? abs(dx) : abs(dz)) : (abs(dy) > abs(dz) ? abs(dy) : abs(dz));
          if (kind == 1) {
            if (adist > ws) continue;
          } else {
            if (adist <= ws) continue;
            if (abs(fdiv2(jx) - fdiv2(ix)) > ws || abs(fdiv2(jy) - fdiv2(iy)) > ws || abs(fdiv2(jz) - fdiv2(iz)) > ws)
              continue;
          }
          const int64_t s = find_box(sb, ns, orc_morton(jx, jy, jz));
          if (s < 0) continue;
          if (idx) idx[c] = s;
          ++c;
        }
  }
  off[nt] = c;
  return c;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
