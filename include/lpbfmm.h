/*
 * lpbfmm -- fast multipole evaluation of screened-Coulomb (linearized Poisson-Boltzmann)
 * potentials and fields of point charges in a layered medium, on one NVIDIA GB300 GPU.
 *
 * Method: Wang, Zhang & Cai, "Fast Multipole Method for 3-D Linearized Poisson-Boltzmann
 * Equation in Layered Media" (arXiv 2002.01334).  The potential at a charge in layer l is
 * the free-space Yukawa sum over the other charges of that layer plus the reaction
 * components carried by equivalent polarization sources (Sec. 2.2, eq. totalinteraction;
 * Sec. 3.3).  Each component is evaluated by an FMM whose multipole-to-local operators are
 * Sommerfeld-type integrals tabulated at run time (Sec. 3.4-3.5, Algorithms 1 and 2).
 *
 * Conventions (Sec. 2.1): L interfaces z = d_0 > d_1 > ... > d_{L-1}; layer 0 is z > d_0,
 * layer k is d_k < z < d_{k-1}, layer L is z < d_{L-1}.  Layer k has dielectric constant
 * eps_k > 0 and inverse Debye length lambda_k > 0.  The Green's function solves
 * eps_l (Laplacian - lambda_l^2) u = -delta with continuity of u and eps du/dz across the
 * interfaces, so the free-space part is exp(-lambda r) / (4 pi eps r).
 *
 * Every entry point returns an lpbfmm status code (0 = success).  Device pointers refer to
 * memory on the context's device; the caller owns all input and output arrays and the
 * library never frees them.  Work is issued on the context's stream and on streams the context
 * owns, forked from it and joined back into it, so the results are complete in the context's
 * stream order (lpbfmm_eval synchronizes the stream internally several times to size its work,
 * and returns without waiting for its last kernels).  A context lives on the device current at
 * lpbfmm_create (ordinal below 64); call its entry points with that device current.  Contexts on several
 * devices may coexist in one process; one context must not be used by two host threads at
 * once.
 */
#ifndef LPBFMM_H
#define LPBFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define LPBFMM_OK 0
#define LPBFMM_ERR_ARG 1            /* null pointer where one is required, n < 0, bad option  */
#define LPBFMM_ERR_MEDIUM 2         /* interfaces not strictly descending, eps <= 0, lambda <= 0,
                                       or more than LPBFMM_MAX_INTERFACES interfaces          */
#define LPBFMM_ERR_P 3              /* truncation order outside [LPBFMM_P_MIN, LPBFMM_P_MAX]   */
#define LPBFMM_ERR_ON_INTERFACE 4   /* a charge lies within 1e-12 (relative to the layer
                                       thickness scale) of an interface, where the Sommerfeld
                                       integrals do not converge (Sec. 3.5)                   */
#define LPBFMM_ERR_LAYER_MISMATCH 5 /* layer_id[i] differs from the layer containing z_i     */
#define LPBFMM_ERR_NONFINITE 6      /* NaN or Inf in q or xyz                                 */
#define LPBFMM_ERR_OOM 7            /* device allocation failed                               */
#define LPBFMM_ERR_CUDA 8           /* a CUDA call failed                                     */
#define LPBFMM_ERR_TIMEOUT 9        /* a bounded device wait expired                          */
#define LPBFMM_ERR_UNSUPPORTED 10   /* e.g. tree too deep for the input size                 */

#define LPBFMM_MAX_INTERFACES 8
#define LPBFMM_P_MIN 2
#define LPBFMM_P_MAX 16

/* precision modes */
#define LPBFMM_FP64 0  /* every step in FP64                                                  */
#define LPBFMM_MIXED 1 /* FP32 P2P, P2M/M2M/L2L/L2P; M2L on the tensor cores in 3xTF32 for
                          p <= 10 (FP32 otherwise); FP64 tables, operators and final sums  */

typedef struct lpbfmm_ctx *lpbfmm_t;

/* Separation of the interaction lists, in boxes (Sec. 3.5 builds Algorithm 1 on the traditional
 * FMM lists: a box's multipole-to-local list holds the children of its parent's near boxes that
 * are not near it, its near list the boxes within the separation).  1 = one-box: near boxes touch;
 * 2 = two-box: one box lies between a box and the nearest box of its far list, so every
 * expansion converges at a faster geometric rate at the same p (more M2L and near-field work). */
#define LPBFMM_SEPARATION_DEFAULT 2
#define LPBFMM_REACT_LEVELS_DEFAULT 4

typedef struct {
  int precision;     /* LPBFMM_FP64 or LPBFMM_MIXED                                        */
  int max_per_leaf;  /* automatic depth: the free-space part uses the smallest depth >= 2 whose
                        mean target occupancy of the non-empty leaves is <= max_per_leaf
                        (default 128); a group's reaction part goes up to react_levels
                        levels deeper, until no target box and image box are near (Sec. 3.5,
                        Remark 1)                                                            */
  int uniform_depth; /* > 0: use this tree depth for every target group and both parts;
                        0: automatic                                                         */
  int separation;    /* 1 or 2 boxes; 0 = LPBFMM_SEPARATION_DEFAULT                        */
  int react_levels;  /* automatic depth: how many levels below the free-space depth the
                        reaction part's tree may go to separate every target box from every
                        image box (0 .. 8; lpbfmm_default_opts sets
                        LPBFMM_REACT_LEVELS_DEFAULT).  Image pairs still near at that depth
                        are summed by direct Sommerfeld quadrature, whose cost grows with the
                        pairs and with the nodes that small target-image distances need      */
  void *stream;      /* cudaStream_t for all work; NULL = the legacy default stream          */
} lpbfmm_opts;

/* Fill *opts with the defaults (FP64, max_per_leaf 128, automatic depth, default separation,
 * react_levels LPBFMM_REACT_LEVELS_DEFAULT, default stream). */
void lpbfmm_default_opts(lpbfmm_opts *opts);

/*
 * Create a context for one medium and truncation order (Sec. 2.1 medium; Sec. 3.1 and 3.4
 * expansions truncated at degree p).  Host arrays: z_iface[n_iface] (strictly descending),
 * eps[n_iface+1] > 0, lambda[n_iface+1] > 0.  tol is the truncation tolerance of the
 * Sommerfeld integrals (Sec. 3.5: the integration range ends where the integrand has fallen
 * below a tolerance the user chooses), in (0, 1e-3].
 * The context allocates device tables for Gaunt coefficients and Legendre-product expansion
 * coefficients on the current device.  opts may be NULL (defaults).  On success *out holds a
 * new context that must be released with lpbfmm_destroy.
 */
int lpbfmm_create(int n_iface, const double *z_iface, const double *eps, const double *lambda, int p,
                  double tol, const lpbfmm_opts *opts, lpbfmm_t *out);

/*
 * Potential and field of n charges (Sec. 2.2 eq. potential1, Algorithm 2):
 *   phi_i = sum_{j != i, layer_j = layer_i} q_j exp(-lambda r_ij)/(4 pi eps r_ij)
 *         + sum_j q_j u^react_{layer_i layer_j}(r_i, r_j)      (reaction part includes j = i)
 *   field_i = -grad_{r_i} phi_i.
 * Device arrays: q[n] (FP64), xyz[n*3] (FP64, x y z per charge), layer_id[n] (int32, the layer
 * of each charge, 0 = top); outputs phi[n] (FP64) and field[n*3] (FP64, may be NULL).
 * Inputs are validated on the device (finite, off the interfaces, layer_id consistent with z);
 * on a data error phi/field are unspecified and the code is returned.  n = 0 is a no-op.
 */
int lpbfmm_eval(lpbfmm_t h, int64_t n, const double *q, const double *xyz, const int32_t *layer_id,
                double *phi, double *field);

/*
 * Same as lpbfmm_eval for a subset of the components, used to check the parts separately
 * (Sec. 2.2, eq. freereactioncomponents): bit 0 (1) the free-space part, bit 1 (2) the reaction
 * part; diagnostics: bit 2 (4) leaves out the reaction near field (direct interactions of
 * adjacent target / image leaves, Algorithm 1 last loop), bit 3 (8) leaves out the reaction
 * far field (multipole-to-local translations).  parts must be in [1, 15].
 */
int lpbfmm_eval_parts(lpbfmm_t h, int64_t n, const double *q, const double *xyz, const int32_t *layer_id,
                      int parts, double *phi, double *field);

/*
 * The part of lpbfmm_eval carried by chosen target groups, for splitting one evaluation across
 * devices or streams: the free-space FMM of every layer and the reaction components of every
 * (layer, interface side) are independent (Sec. 2.2 eq. freereactioncomponents; the paper's
 * Sec. 4 notes that the components can be computed in parallel), so the sum of the outputs over a
 * partition equals lpbfmm_eval's output: to FP64 rounding in FP64 mode; in the mixed mode a
 * group's free-space and reaction local expansions are added in FP32 before they are evaluated,
 * so a partition that separates them differs by that rounding (about 1e-7 relative).
 * mask is a host array of 2 (L + 1) ints, entry 2 l + a - 1 for target group (layer l, side a):
 * bit 0 = the free-space part of layer l (carried by group (l, 1), or (L, 2) for the bottom
 * layer; the bit is ignored on the other group), bit 1 = the reaction components of targets in
 * layer l whose polarization sources sit across interface d_l (a = 1) or d_{l-1} (a = 2); entries
 * of groups that do not exist (a = 1 for l = L, a = 2 for l = 0) are ignored.  Values outside
 * [0, 3] return LPBFMM_ERR_ARG.  Outputs as lpbfmm_eval (zero where no selected part contributes).
 */
int lpbfmm_eval_groups(lpbfmm_t h, int64_t n, const double *q, const double *xyz, const int32_t *layer_id,
                       const int32_t *mask, double *phi, double *field);

/*
 * Adjoint of phi with respect to q and positions for an upstream gradient g_phi[n] (device):
 *   g_q[j]   = sum_i g_phi[i] G(r_i, r_j)                  = phi[g_phi](r_j)
 *   g_xyz[j] = sum_i g_phi[i] d phi_i / d r_j = -(q_j field[g_phi](r_j) + g_phi[j] field[q](r_j))
 * using the reciprocity G_{l l'}(r, r') = G_{l' l}(r', r) of the layered Green's function (the
 * vector-Jacobian product of phi).  For E = 1/2 sum q_i phi_i: dE/dq = g_q with g_phi = q, and
 * dE/dr = g_xyz with g_phi = q / 2 (so the force on charge j is -g_xyz[j]).  Two evaluations
 * are run.  Device arrays; g_q[n], g_xyz[n*3] are outputs.  The context keeps a work space of
 * 7 n doubles between calls (allocated when n first exceeds its size); g_q and g_xyz are written
 * in stream order on the context's stream.
 */
int lpbfmm_adjoint(lpbfmm_t h, int64_t n, const double *q, const double *xyz, const int32_t *layer_id,
                   const double *g_phi, double *g_q, double *g_xyz);

/*
 * Batched evaluation of nsys independent systems, each with its own context (medium and
 * order): system s uses rows offsets[s] .. offsets[s+1]-1 of the concatenated device arrays.
 * offsets is a host array of nsys+1 non-decreasing entries with offsets[0] = 0.  All contexts live
 * on the current device.  The per-system parts (validation, trees, lists, tables, operators,
 * upward and downward passes) run concurrently, each distinct context on one of eight
 * library-owned streams driven by host threads, heaviest first.  For the contexts that serve one
 * system each, the two heaviest passes run grouped over all of them, on the stream of ctxs[0]:
 * one tensor-core M2L launch (and one launch of its slot sums) per truncation order, whose work
 * items span (system, target group, level, row class, far-list slice), and one launch of the FP32
 * free-space near field, whose blocks span (system, group, leaf).  A context that serves several
 * systems evaluates them in turn, whole.  Results equal lpbfmm_eval's bit for bit.  A timed-out
 * wait in a grouped launch is reported on the status word of the first such context (in batch
 * order, heaviest first).  The call returns when every system's host-side work is done, and the
 * stream of ctxs[0] (and every context's own stream) is ordered after all of it.  Not
 * stream-capturable.  The first error code any system returns is returned.
 */
int lpbfmm_eval_batched(int nsys, const lpbfmm_t *ctxs, const int64_t *offsets, const double *q,
                        const double *xyz, const int32_t *layer_id, double *phi, double *field);

/*
 * Diagnostics for the tests: after an lpbfmm_eval on h, copy out the tree of target group
 * (layer l, side a) at its depth D (Sec. 3.5: root cube bisected by interface d_l for a = 1,
 * d_{l-1} for a = 2).  root[4] = cx, cy, cz, half-size (host).  If keys is NULL only the
 * counts are returned: *n_targets, *n_images, *depth.  Otherwise keys_t[n_targets] and
 * keys_i[n_images] (host uint64) receive the depth-D Morton keys in sorted order, src_t and
 * src_i (host int64) the input index of each point, type_i (host int32) the image type
 * 2*l' + b - 1.  Returns LPBFMM_ERR_ARG if the group does not exist.
 */
int lpbfmm_debug_tree(lpbfmm_t h, int l, int a, double *root, int64_t *n_targets, int64_t *n_images,
                      int *depth, uint64_t *keys_t, int64_t *src_t, uint64_t *keys_i, int64_t *src_i,
                      int32_t *type_i);

/*
 * Diagnostics: after an lpbfmm_eval, the interaction lists of the adaptive dual tree of target
 * group (l, a)'s free-space tree with itself (Sec. 3.5 builds the method on the adaptive FMM
 * framework; built on the device by a level-synchronous traversal over frontiers of box pairs;
 * the evaluation itself uses uniform trees).  A box of level l >= 3 exists when its parent exists
 * and holds more than s targets (every box of level 2 exists); it is a leaf when it holds at most
 * s or sits at the group's free-space depth.  Two boxes are near for separation ws (1 or 2) when
 * the coarser one, grown by ws - 1 of its sides, meets the finer one.  Records of 5 int64 (host):
 * kind (0 = V: far, same level; 1 = U: near leaves; 2 = W: target leaf, finer far source box;
 * 3 = X: source leaf, finer far target box), target level, target box's Morton key at that level,
 * source level, source key; in no particular order.  *nrec receives their number; at most cap
 * are copied to rec (rec may be NULL).  The group must carry the free-space part.
 */
int lpbfmm_debug_adaptive_lists(lpbfmm_t h, int l, int a, int s, int ws, int64_t *nrec, int64_t *rec,
                                int64_t cap);

/*
 * Diagnostics: after an lpbfmm_eval, the interaction lists of group (l, a) at level lev:
 * kind 0 = far (multipole-to-local) list, kind 1 = near list at the leaf level; src 0 = the
 * group's free-space sources (its own targets; leaf level = the free-space depth), src 1 = its
 * images (leaf level = the tree depth of lpbfmm_debug_tree).  Host outputs in CSR form
 * over the level's target boxes (sorted by key): off[nbox+1], idx[off[nbox]] source box
 * indices, each row in ascending order of the offset (dx, dy, dz) with dx outermost.  With
 * off == NULL only *nbox and *nent are returned.
 */
int lpbfmm_debug_lists(lpbfmm_t h, int l, int a, int lev, int kind, int src, int64_t *nbox, int64_t *nent,
                       int64_t *off, int64_t *idx);

/*
 * Diagnostics: scaled Sommerfeld integrals of Sec. 3.5 (eq. M2Ltable scaled by S^K, S = h)
 *   out[((K*(Kmax+1)) + d)*4 + 2i + j] = h^K / sqrt((K+d)!(K-d)!)
 *        * int_0^inf lr^K J_d(lr rho) exp(-lz_l zt - lz_l' zs) sigma^{ab}_{l l'} / lz_l
 *          (lambda_l/lz_l)^i (lambda_l'/lz_l')^j d lr,         K = 0..Kmax, d = 0..K,
 * computed on the device the way the FMM computes them: quadrature for d = 0, 1 and the
 * forward recurrence in d (eq. recurrence1) for d >= 2.  Only the entries with K - d odd are
 * computed (the multipole-to-local operators use no others); the rest are 0.  zt, zs > 0 are the
 * distances of the target and source centres to the component's interface, zt = (k_t + 1/2) h and
 * zs = (k_s + 1/2) h with integers k_t, k_s >= 0, k_t + k_s <= 4; rho = ratio * h with ratio^2 in
 * {0,1,2,4,5,8,9,10,13,16,17,18,20,25,26,29,32,34,41,50}.  Other geometries return
 * LPBFMM_ERR_ARG.  out is a host array.
 */
int lpbfmm_debug_stable(lpbfmm_t h, int l, int a, int lp, int b, double hbox, double rho, double zt,
                        double zs, int Kmax, double *out);

/*
 * The table of lpbfmm_debug_stable for one class, computed without allocating: no cudaMalloc,
 * cudaFree or allocating library call.  The paper has no counterpart; this entry point serves
 * callers that cannot allocate, e.g. a loop that has given all free device memory to its own
 * pool, or one that must not suffer the device-wide synchronisation of cudaMalloc/cudaFree.
 *   out   device array of (Kmax+1)^2 * 4 doubles, same layout as lpbfmm_debug_stable; written
 *         on the context's stream (the call does not synchronize), owned by the caller.
 *   Kmax  at most LPBFMM_NOALLOC_KMAX; the class's quadrature may use at most
 *         LPBFMM_NOALLOC_NQ nodes.  Larger requests return LPBFMM_ERR_UNSUPPORTED.
 * Temporaries live in one fixed device array of about 1.8 MB per device, whose address is
 * looked up on the first call on each device: make that first call before any stream capture.
 * Calls that overlap in time on one device (other streams, other contexts) share that array
 * and race; serialize them.  The context's device must be current (LPBFMM_ERR_ARG otherwise).
 * Other errors as lpbfmm_debug_stable.
 */
#define LPBFMM_NOALLOC_KMAX 23   /* = 2p + 3 at p = 10 */
#define LPBFMM_NOALLOC_NQ 4096
int lpbfmm_stable_noalloc(lpbfmm_t h, int l, int a, int lp, int b, double hbox, double rho, double zt,
                          double zs, int Kmax, double *out);

/*
 * Diagnostics: after an lpbfmm_eval, copy an intermediate device array of group (l, a) at
 * level lev into the host buffer dst (capacity cap bytes); *bytes receives its size.  Names:
 * "Mimg", "Mfree", "Lt" (expansions, complex, working precision), "op_react", "op_free"
 * (translation operators), "stab" (FP64 Sommerfeld tables), "used" (uint8 reaction classes in
 * use), "vreact" (int32 far list), "ikeys", "tkeys" (uint64 box keys), "rows", "nrows".
 * With dst == NULL only *bytes is set.
 */
int lpbfmm_debug_array(lpbfmm_t h, int l, int a, const char *name, int lev, void *dst, int64_t cap,
                       int64_t *bytes);

/*
 * Work counts of the last lpbfmm_eval (host int64 out[8]): [0] free-space multipole-to-local
 * translations, [1] reaction translations (box pairs x source types), [2] free-space P2P pairs
 * (including the excluded self pairs), [3] reaction near-field pairs, [4] targets summed over
 * the target groups, [5] images summed over the groups, [6] target boxes over all groups and
 * levels, [7] kernels launched by the evaluation.  Synchronizes the context's stream.
 */
int lpbfmm_last_counts(lpbfmm_t h, int64_t *out);

/* Read and clear the device status word (synchronizes the context's stream). */
int lpbfmm_status(lpbfmm_t h);

/* Short description of a status code (static storage). */
const char *lpbfmm_strerror(int code);

/* Release the context's device memory. */
void lpbfmm_destroy(lpbfmm_t h);

/*
 * Per-phase device times (ms) of the last lpbfmm_eval, measured with CUDA events on the
 * context's stream, and the number of kernels it launched.  The mixed-precision free-space near
 * field ("p2p") runs on a stream of its own beside the operators, the upward pass and the M2L,
 * and is timed there; the operators run on another stream and show only as waits.  names[i] is
 * a static string.  Returns the number of phases written (at most cap).
 */
int lpbfmm_last_profile(lpbfmm_t h, int cap, const char **names, float *ms, int *launches);

/*
 * The host-side tables that lpbfmm_create computes for order p and uploads to the device, computed
 * here on the host alone: no context, no device, no CUDA call.  Intended for tests of the table
 * construction.  which selects the table; all entries are FP64.  Index helpers:
 * f(n, m) = n^2 + n + m (full, |m| <= n), h(n, m) = n(n+1)/2 + m (half, 0 <= m <= n).
 *   LPBFMM_TABLE_GAUNT     G[f(n,a)][f(nu,g)][q], n, nu <= p, q <= 2p: the integral over the unit
 *                          sphere of Y_n^a Y_q^{g-a} conj(Y_nu^g), the Gaunt coefficients of the
 *                          free-space translation theorems (Sec. 3.1, Thm. 2-3); Y_n^m as in
 *                          Sec. 3.1 (equal to the Condon-Shortley harmonics).  Zero where
 *                          |g - a| > q or n + nu + q is odd.
 *   LPBFMM_TABLE_TPOLY     c[h(n,m)][k], k < p/2 + 2 (row stride p/2 + 2): the ratio of normalized
 *                          Legendre functions phat_n^m(x) / phat_m^m(x) written as
 *                          x^{-i} sum_k c_k t^k with t = x^2 - 1, i = (n - m) mod 2.  These are the
 *                          Legendre-product expansions behind the reaction M2L operators of
 *                          Sec. 3.5 (eqs. metoletableform and the product formula before it).
 *   LPBFMM_TABLE_PHAT_DIR  P[dir][h(q,k)], q <= 2p: phat_q^k(cos theta) of the 222 translation
 *                          directions: dir = 11 ri + dz + 5 (ri indexes rho^2 in {0, 1, 2, 4, 5, 8,
 *                          9, 10, 13, 16, 17, 18, 20, 25, 26, 29, 32, 34, 41, 50}, dz in -5..5) with
 *                          cos theta = -dz / sqrt(rho^2 + dz^2) (1 when both vanish), and dir 220,
 *                          221 with cos theta = -1/sqrt(3), +1/sqrt(3) (child-to-parent shifts).
 *   LPBFMM_TABLE_SFAC      s[K][d], K, d < 36 (row stride 36): sqrt((K+d)! (K-d)!) for d <= K, else
 *                          0; the normalization of the Sommerfeld-type integrals (Sec. 3.5, eq.
 *                          M2Ltable).  Independent of p.
 * If out is NULL only *count (the number of doubles) is set; otherwise out must hold cap >= *count
 * doubles and receives the table.  Returns LPBFMM_ERR_ARG for a null count, an unknown table or a
 * short buffer, LPBFMM_ERR_P for p outside [LPBFMM_P_MIN, LPBFMM_P_MAX], LPBFMM_ERR_OOM if host
 * memory runs out.
 */
/*
 * Measured arithmetic peak of the current device for the rooflines of the library's SIMT kernels
 * (not part of the method): chains of fused multiply-adds, 8 independent chains per thread and 64
 * resident warps per SM, timed with CUDA events on a stream of its own after a warm-up.
 * which = LPBFMM_PEAK_FP32_FMA or LPBFMM_PEAK_FP64_FMA; *tflops receives 2 x FMAs per second / 1e12.
 * Runs for some tens of milliseconds; allocates 8 bytes of device memory.  LPBFMM_ERR_ARG for a
 * null pointer or an unknown which.
 */
#define LPBFMM_PEAK_FP32_FMA 0
#define LPBFMM_PEAK_FP64_FMA 1
int lpbfmm_measure_peak(int which, double *tflops);

#define LPBFMM_TABLE_GAUNT 0
#define LPBFMM_TABLE_TPOLY 1
#define LPBFMM_TABLE_PHAT_DIR 2
#define LPBFMM_TABLE_SFAC 3
int lpbfmm_host_table(int which, int p, double *out, int64_t cap, int64_t *count);

#ifdef __cplusplus
}
#endif
#endif
