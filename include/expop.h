/*
 * expop.h -- C ABI of the GB300 apply engine for the rational time-evolution
 * operator of Haut, Babb, Martinsson and Wingate:
 *
 *     exp(tau L) u  ~  R(tau L) u = sum_{m=-M..M} b_m (tau L - alpha_m)^{-1} u
 *
 * (Section 1.1 and eq. def_RM of Section 1.2), for a skew-Hermitian L.  Each
 * resolvent is reduced to one scalar elliptic solve (Section 2.1), discretised by
 * multidomain Chebyshev collocation (Section 2.2) and solved with precomputed
 * nested-dissection (HPS) solution operators (Section 2.3 and Section 1.3).
 *
 * Conventions shared by every call:
 *  - All functions return eo_status; they never print, abort or throw.  On error
 *    eo_last_error() returns a message for the calling thread.
 *  - Floating point data are IEEE FP64.  Complex numbers are interleaved
 *    (re, im) pairs.
 *  - A state is real, laid out [rhs][field][node] with the node order given by
 *    eo_grid_nodes.  Fields: EO_WAVE_DIRICHLET (u, v); EO_SW_WALLS (u, v, h).
 *  - Node order (the "public numbering"): the leaf square [x0,x1]x[y0,y1] is cut
 *    into nlx x nly leaves with p x p Chebyshev-Lobatto nodes each; the four corner
 *    nodes of every leaf are dropped (no equation references them).  Then
 *      interior nodes, leaf l = b*nlx + a, local (k, j), k,j = 1..p-2:
 *          id = l*q*q + (j-1)*q + (k-1),                       q = p - 2
 *      horizontal edge nodes, line e = 0..nly, leaf column a, k = 1..q:
 *          id = n_int + (e*nlx + a)*q + (k-1)
 *      vertical edge nodes, line e = 0..nlx, leaf row b, j = 1..q:
 *          id = n_int + n_h + (b*(nlx+1) + e)*q + (j-1)
 *    with n_int = nlx*nly*q*q and n_h = nlx*(nly+1)*q.
 *  - Handles are not thread-safe; distinct handles may be used concurrently.
 *  - "stream" arguments are cudaStream_t passed as void* (NULL = legacy default).
 */
#ifndef EXPOP_H
#define EXPOP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EO_OK = 0,
  EO_ERR_INVALID_ARG = 1, /* bad size, pointer or option                        */
  EO_ERR_FIT = 2,         /* no rational approximant meets delta for the request */
  EO_ERR_SINGULAR = 3,    /* a leaf, merge or root system is numerically singular */
  EO_ERR_OOM = 4,         /* device or host allocation failed                   */
  EO_ERR_BUDGET = 5,      /* operators would exceed opts.mem_budget_gb          */
  EO_ERR_CUDA = 6,        /* a CUDA runtime / cuBLAS call failed                */
  EO_ERR_TIMEOUT = 7,     /* a bounded device wait gave up                       */
  EO_ERR_UNSUPPORTED = 8  /* request outside what this build implements          */
} eo_status;

typedef enum {
  EO_WAVE_DIRICHLET = 0, /* u_t = v, v_t = div(c^2 grad u), u = 0 on the walls
                            (two-field form of Example 2, Section 2.1)          */
  EO_SW_WALLS = 1,       /* u_t = f v - g h_x, v_t = -f u - g h_y,
                            h_t = -H (u_x + v_y), no normal flow at the walls
                            (Example 1, Section 2.1, constant f, g, H)          */
  EO_WAVE_KAPPA = 2      /* u_tt = kappa Delta u in the three-field form of Example 2
                            (Section 2.1, eq. "forward oper, inhom"): state (w, z, v) =
                            (u_x, u_y, u_t), w_t = v_x, z_t = v_y, v_t = kappa (w_x + z_y),
                            on a periodic grid (Section 4.2); kappa > 0 at the nodes;
                            per-box operators.  Its resolvent is the elliptic solve
                            (Delta - alpha^2 / (tau^2 kappa)) v = alpha f_v / (tau^2 kappa)
                            + (d_x f_w + d_y f_z) / tau, then w = (tau v_x - f_w) / alpha,
                            z = (tau v_y - f_z) / alpha (eqs. "w and z eqns" to "v for
                            inhomog, inverse" with the data scaled by tau)        */
} eo_kind;

typedef enum {
  EO_PREC_FP64 = 0, /* operators stored and applied in FP64                         */
  EO_PREC_FP32 = 1, /* operators built in FP64, stored in FP32; block products in FP32,
                       vectors, pole sum and pre/post maps in FP64                   */
  EO_PREC_DF32 = 2  /* operators built in FP64, stored as FP32 (hi, lo) pairs (same
                       bytes as FP64, ~2^-48 relative); block products on the FP32
                       pipe with exact product splitting and compensated sums     */
} eo_precision;

typedef enum {
  EO_FIT_LINE = 0,  /* poles on one conjugate-closed line, residues by least squares,
                       eqs. RM_prop1 and RM_prop2 both enforced (see eo_fit)        */
  EO_FIT_GAUSS = 1  /* the paper's construction (Sections 3.1-3.2): shifted Gaussians
                       replaced by the Table 1 rational, two pole lines; meets
                       eq. RM_prop1 only (see eo_fit_gauss)                        */
} eo_fitter;

typedef struct eo_grid_s *eo_grid_t;
typedef struct eo_handle_s *eo_handle_t;
typedef struct eo_batch_s *eo_batch_t;

/* Options of eo_build_operator.  Zero-initialise and set what you need. */
typedef struct {
  int n_poles;         /* 2M+1 (odd) requested; the fitter then maximises the band
                          X it covers and tau = X / band.  0: tau is given and the
                          pole count is the smallest that covers tau * band.      */
  double band;         /* Lambda of eq. RM_prop1: largest |eigenvalue| resolved   */
  double tau;          /* time step (used when n_poles == 0)                      */
  double delta;        /* accuracy of eq. RM_prop1 (0: 1e-10)                     */
  double sw_f, sw_g, sw_H; /* shallow-water Coriolis, gravity, depth            */
  int precision;       /* eo_precision                                           */
  int shared_ops;      /* 1: one operator set per tree level (valid only for
                          constant coefficients; EO_SW_WALLS); 0: one per box     */
  int max_rhs;         /* largest n_rhs that eo_apply will be called with (>=1)   */
  double mem_budget_gb;/* cap on operator storage in GB (0: no cap)               */
  int fp64_top_levels; /* EO_PREC_FP32/DF32: this many top merge levels, and then also the
                          root wall solve, keep FP64 operators (0: all FP32)       */
  int use_graphs;      /* 1: eo_apply with n_steps >= 2 records a pair of steps as a
                          CUDA graph (per state pointer and n_rhs) and replays it;
                          the first such call must not itself be inside a capture */
  int dense_leaves;    /* 0: with shared_ops (constant coefficient), leaf solves use
                          the leaf's separable eigenbasis (fast diagonalisation, see
                          eo_leaf_basis), in FP32-pair arithmetic with EO_PREC_DF32
                          and FP64 otherwise; 1: the dense leaf solution operators
                          of Section 2.3 (always used for per-box operators and by
                          eo_apply_adjoint)                                      */
  int autotune;        /* 1: the first eo_apply (and the first with a new n_rhs) times
                          the candidate launch shapes of every merge level, the root
                          solve and the fast-diagonal leaf kernels on this handle's
                          operators and keeps the fastest (synchronises the stream
                          once; skipped inside a stream capture); 0: fixed shapes  */
  int sw_consistent;   /* EO_SW_WALLS with f != 0: 1 keeps the (tau f / alpha) Curl(G h)
                          term in the elliptic rows (G the recovered node gradient), the
                          exact elimination of (U, V) on this discretisation, so the
                          per-pole solves are resolvents of one discrete operator;
                          0: the elimination as the paper writes it (curl grad = 0).
                          1 uses dense leaf operators (no fast diagonalisation)     */
  int fitter;          /* eo_fitter (0: EO_FIT_LINE).  EO_FIT_GAUSS needs n_poles == 0
                          and tau > 0                                             */
  double gauss_h;      /* EO_FIT_GAUSS: Gaussian spacing h in x = theta / (2 pi)
                          (0: 0.18); smaller h, more poles, smaller aliasing error  */
  int root_dense;      /* EO_SW_WALLS on a square domain of square leaves: the wall
                          system commutes with the quarter turn of the domain, so it
                          splits into four Fourier blocks of a quarter of the wall
                          nodes each (4x fewer root bytes and flops; the build checks
                          the symmetry to 1e-9 and fails with EO_ERR_UNSUPPORTED if it
                          does not hold).  1: keep the dense wall inverse instead   */
  int merge_dense;     /* shared_ops without the consistent curl term: every box of a
                          level is symmetric under the reflections across and along its
                          merge interface, so the forward apply uses even/odd blocks
                          of the merge operators (Z in two, U and S in four; the build
                          checks the symmetry to 1e-9 and fails with
                          EO_ERR_UNSUPPORTED if it does not hold; the dense blocks stay
                          for eo_apply_adjoint).  1: dense merge blocks only        */
  int tensor_leaves;   /* 1: the leaf interior solves and the pole sum run on the tensor
                          cores (tcgen05.mma on bf16 slices, FP32 accumulation in TMEM):
                          the dense leaf operators [X | Y] of every pole are split at build
                          time into 6 bf16 slices of 7 bits per real part (41 bits), with
                          a power-of-two scale per row and block; per step and pole the
                          right-hand sides g = sum_k c_k s_k (formed in FP32 pairs) and the
                          edge values are split the same way per column and block; the
                          product levels i + j = 2, 3, 4 are summed exactly in FP32, the
                          deeper ones rounded (about 2^-40 of the leading level), and the
                          pole sum is kept in FP32 pairs.  Needs EO_PREC_DF32, dense leaves
                          (per-box operators, or opts.dense_leaves with shared ones) and
                          p <= 18; otherwise the build fails with EO_ERR_UNSUPPORTED.
                          Holds 24 bytes per entry of [X | Y] (rows padded to a multiple
                          of 128, columns to a multiple of 16) besides the dense
                          operators, which eo_apply_adjoint keeps using.  0: off     */
  int merge_fuse;      /* reflection-symmetric merge levels (opts.merge_dense = 0) of the
                          forward apply: 0 (default) runs one launch per level; k = 1 .. 4
                          runs levels 1 .. min(k, L - 1) in one launch per sweep (one block
                          per pole and box of the highest fused level, boundary data of the
                          levels below it in shared memory, the arithmetic of the per-level
                          kernels).  Fewer levels are fused where the shared memory of a
                          block (R right-hand sides) would exceed 200 KB, none where a level
                          is not symmetric.  On GB300 the per-level launches are faster for
                          the shallow-water workload (their FP32-pair products are
                          issue-bound and need the occupancy of many small blocks)      */
} eo_opts;

/* Leaf grid.  nlx, nly powers of two (>= 1), 4 <= p <= 24, x0 < x1, y0 < y1.
 * Errors: EO_ERR_INVALID_ARG.  The grid is owned by the library until
 * eo_grid_destroy; handles built from it keep their own copy. */
eo_status eo_grid_create(int nlx, int nly, int p, double x0, double x1, double y0,
                         double y1, eo_grid_t *out);
/* Periodic leaf grid: the square [x0,x1]x[y0,y1] with x1 identified with x0 and y1 with
 * y0, the setting of the examples of Section 4.
 * The seams x = x0 and y = y0 are interfaces between the last and the first leaf of each
 * row and column (flux continuity, Section 2.2); there is no domain boundary.  Public
 * numbering as above with nly horizontal and nlx vertical edge lines (line e = 0 is also
 * the top / right edge of the last leaf row / column): n_h = nlx*nly*q,
 *   vertical edge nodes: id = n_int + n_h + (b*nlx + e)*q + (j-1),  e = 0..nlx-1,
 * and seam nodes carry the coordinates x0 (vertical seam) and y0 (horizontal seam).
 * Built operators then have no walls: EO_SW_WALLS is rotating shallow water on the
 * torus, EO_WAVE_DIRICHLET the wave equation on the torus; the root solve is the
 * seam system of the root box merged with itself (half its boundary nodes).
 * eo_apply_adjoint is not built for periodic grids (EO_ERR_UNSUPPORTED), and merges
 * use the dense blocks (opts.merge_dense is implied).  Errors as eo_grid_create. */
eo_status eo_grid_create_periodic(int nlx, int nly, int p, double x0, double x1, double y0,
                                  double y1, eo_grid_t *out);
/* 1 for a periodic grid, 0 for a walled one. */
eo_status eo_grid_periodic(eo_grid_t grid, int *periodic);
/* Sizes: total nodes, interior nodes, edge nodes.  Any pointer may be NULL. */
eo_status eo_grid_info(eo_grid_t grid, int64_t *n_nodes, int64_t *n_interior,
                       int64_t *n_edge);
/* Coordinates of every node in the public order, into caller-owned HOST arrays
 * of n_nodes doubles. */
eo_status eo_grid_nodes(eo_grid_t grid, double *x, double *y);
eo_status eo_grid_destroy(eo_grid_t grid);

/* Build phase (Section 1.3): fit {alpha_m, b_m} (eqs. RM_prop1, RM_prop2), then
 * on the device, in FP64, for each distinct pole (the conjugate pairs of
 * eq. "conjugate, matrix inverses", Section 3.3): leaf collocation, leaf solution
 * operators, merge-level Schur complements, and for EO_SW_WALLS the root
 * oblique-boundary solve.  Operators stay resident in device memory until
 * eo_destroy.
 *   coeff: HOST array of n_nodes doubles with c^2 (EO_WAVE_DIRICHLET) or kappa
 *          (EO_WAVE_KAPPA) at the nodes, positive and finite; ignored (may be NULL)
 *          for EO_SW_WALLS.  EO_WAVE_KAPPA needs a periodic grid and per-box
 *          operators (shared_ops = 0) and does not take tensor_leaves
 *          (EO_ERR_UNSUPPORTED); the sw_* options do not apply to it.
 * Synchronous: returns when the operators are built.
 * Errors: EO_ERR_INVALID_ARG, EO_ERR_FIT, EO_ERR_SINGULAR, EO_ERR_OOM,
 *         EO_ERR_BUDGET, EO_ERR_CUDA, EO_ERR_UNSUPPORTED. */
eo_status eo_build_operator(eo_grid_t grid, eo_kind kind, const double *coeff,
                            const eo_opts *opts, void *stream, eo_handle_t *out);

/* Host-only: the rational approximant alone (eqs. RM_prop1, RM_prop2), without
 * building operators.  n_poles > 0: widest band for that odd pole count;
 * n_poles == 0: fewest poles covering band X (> 0).  Poles alpha_m = sigma + i s m
 * on one conjugate-closed line (m = -M..M); residues with b_{-m} = conj(b_m).
 *   cap: capacity (in poles) of alpha and b, each 2*cap doubles interleaved.
 *   n, X_out: pole count and band covered.  No device is touched.
 * Errors: EO_ERR_INVALID_ARG (cap too small: *n is still set), EO_ERR_FIT,
 *         EO_ERR_UNSUPPORTED. */
eo_status eo_fit(int n_poles, double X, double delta, int cap, double *alpha, double *b, int *n,
                 double *X_out);

/* Host-only: the paper's approximant (Sections 3.1-3.2) of e^z on z = i theta,
 * |theta| <= X.  With x = theta / (2 pi), e^{2 pi i x} = sum_{m=-M..M} c_m psi_h(x + m h),
 * psi_h(x) = (4 pi)^{-1/2} exp(-x^2 / (4 h^2)), c_m = exp(4 pi^2 h^2) exp(-2 pi i m h)
 * (Section 3.1), and every psi_h(x + m h) = psi_1(x/h + m) is replaced by the Table 1
 * rational psi_1(y) ~= Re sum_{j=-11..11} a_j / (i y + mu + i j) (Section 3.2; its even
 * part, which makes the result exactly conjugate-closed).  M is the smallest that
 * meets delta (0: 1e-10) on the band; h in (0, 0.5) (0: 0.18).  Output: two lines of
 * 2(M+11)+1 poles each, alpha = -2 pi h (mu + i n) (right half-plane) then its mirror
 * image 2 pi h (mu - i n), each line in order of increasing Im.  Unlike eo_fit, |R(iy)|
 * is NOT bounded by 1: it reaches about 1.44 near |y| = 2 pi M h, so repeated steps
 * amplify any content there unless filtered (EO_FN_FILTER).
 *   cap: capacity of alpha and b (poles, 2*cap doubles each); n, M: pole count and M.
 * Errors: EO_ERR_INVALID_ARG (cap too small: *n is still set), EO_ERR_FIT. */
eo_status eo_fit_gauss(double X, double h, double delta, int cap, double *alpha, double *b, int *n,
                       int *M);

/* The approximant in use: n poles alpha (2n doubles, interleaved), residues b
 * (2n doubles), the step tau and the band X = tau*Lambda it covers.  Pass
 * alpha = b = NULL to query n only.  Poles come as conjugate-closed lines, each
 * in order of increasing Im: one line m = -M..M (EO_FIT_LINE, n = 2M+1) or the
 * two lines of eo_fit_gauss (EO_FIT_GAUSS).  Operators exist for the poles with
 * Im >= 0 (eq. "conjugate, matrix inverses", Section 3.3). */
eo_status eo_get_poles(eo_handle_t h, double *alpha, double *b, int *n, double *tau,
                       double *X);

/* Host-only: the separable eigenbasis of a constant-coefficient leaf.  For p
 * Chebyshev-Lobatto points on an interval of length len and coefficient a > 0,
 * M = a (D D)_ii, the interior (q x q, q = p - 2) block of the squared scaled
 * differentiation matrix (the 1-D factor of the collocated div(a grad) of
 * Section 2.2), is factored as M = V diag(lam) Vinv with real lam in descending
 * order and unit-norm columns of V.  Caller-owned HOST arrays: lam (q doubles),
 * V and Vinv (q*q doubles, row-major).  The leaf solve of a pole is then
 * (V_y (x) V_x) diag(1 / (lx_a + ly_b - kappa^2)) (V_y (x) V_x)^{-1}.
 * Errors: EO_ERR_INVALID_ARG; EO_ERR_UNSUPPORTED if the factorisation fails
 * its residual checks. */
eo_status eo_leaf_basis(int p, double len, double a, double *lam, double *V, double *Vinv);

/* Bytes of device memory held for operators and for the apply workspace. */
eo_status eo_memory(eo_handle_t h, int64_t *operator_bytes, int64_t *workspace_bytes);

/* Apply phase: u <- R(tau L)^n_steps u for n_rhs states in DEVICE memory
 * (u_dev: [n_rhs][fields][n_nodes] FP64, caller-owned, updated in place).
 * Stream-ordered and asynchronous with respect to the host; n_rhs <= max_rhs.
 * With opts.use_graphs, repeated steps replay a recorded CUDA graph.
 * Each step runs two tree sweeps per distinct pole and the b_m-weighted sum.
 * Errors: EO_ERR_INVALID_ARG, EO_ERR_CUDA (launch errors only; asynchronous
 * faults surface at the caller's next synchronisation). */
eo_status eo_apply(eo_handle_t h, double *u_dev, int n_rhs, int n_steps, void *stream);

/* Adjoint of the step: y <- (G^T)^n_steps y, G the real linear map of one
 * eo_apply step (transpose for the Euclidean inner product of the state vector):
 * the forward sweeps run backwards with every stored block transposed
 * (conjugate-pole form of Section 3.3 kept).  Layout, stream and errors as
 * eo_apply.  The first call allocates seed buffers (P * max_rhs * n_interior
 * complex values, plus wall and field seeds for EO_SW_WALLS). */
eo_status eo_apply_adjoint(eo_handle_t h, double *y_dev, int n_rhs, int n_steps, void *stream);

/* Same as eo_apply for a state in HOST memory (pinned or pageable): copies in,
 * applies, copies back and synchronises the stream before returning. */
eo_status eo_apply_host(eo_handle_t h, double *u_host, int n_rhs, int n_steps,
                        void *stream);

/* One resolvent: x = (tau L - alpha_j)^{-1} u for the pole of index j in the
 * eo_get_poles order with Im(alpha_j) >= 0, for one state (n_rhs = 1).
 * u_dev: DEVICE [fields][n_nodes] FP64.  x_dev: DEVICE [fields][n_nodes]
 * complex (2 doubles each).  Asynchronous like eo_apply. */
eo_status eo_apply_resolvent(eo_handle_t h, int j, const double *u_dev, double *x_dev,
                             void *stream);

/* eo_apply_resolvent without any device allocation.  The paper has no
 * counterpart.  It exists for callers that cannot allocate device memory when
 * they call: host threads that must stay off the device allocator (cudaMalloc
 * takes process-wide locks and may synchronise the device), and programs that
 * hand all of the GPU's memory to their own pool, so that any other allocation
 * fails.  The caller passes the input and output; the scratch (the pole's K
 * weights and the real and imaginary staging of the result) comes from one
 * fixed 16 MiB array in device memory (a file-scope __device__ array of
 * 2 Mi doubles) that every GPU loading the library holds until the process
 * exits.  Problems needing more than 16 + 2 * fields * n_nodes doubles of it are
 * rejected with EO_ERR_INVALID_ARG.  The first call on a device looks the
 * array's device address up (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  Every call shares the array
 * and keeps the previous call's contents (each call rewrites the weights on the
 * device before reading them): calls whose work can overlap on the GPU race on
 * it, so order them on one stream.  Arguments and result as eo_apply_resolvent;
 * stream-ordered and asynchronous: x_dev holds the result once `stream` has
 * reached the end of the call's work.  No cudaMalloc, cudaFree or allocating
 * library routine is called. */
eo_status eo_apply_resolvent_noalloc(eo_handle_t h, int j, const double *u_dev, double *x_dev,
                                     void *stream);

/* Other functions of tau L on the SAME poles (dense output and phi-functions; the
 * solves are shared, only the pole-sum weights change).  Host-only fit of residues b
 * (n complex, interleaved, the eo_get_poles order, conjugate-symmetric) such that
 * sum_m b_m / (z - alpha_m) approximates, on the handle's band z = i x, |x| <= X:
 *   kind EO_FN_EXP (0):    exp(c z), 0 < c <= 1   (exp(c tau L): output inside the step)
 *   kind EO_FN_PHI1 (1):   phi1(z) = (exp(z) - 1) / z
 *   kind EO_FN_PHI2 (3):   phi2(z) = (exp(z) - 1 - z) / z^2 (both the phi-functions of
 *                          exponential integrators, Section 3.1)
 *   kind EO_FN_FILTER (2): EO_FIT_GAUSS only: the rational partition of unity
 *                          chi(x) = sum_{|m|<=M0} psi_h(x + m h), x = z / (2 pi i),
 *                          M0 = floor(c M), 0 < c <= 1 (the filter S of Section 3.3,
 *                          unreduced: its poles are the handle's own).
 * Line fits: narrow bands solve for every residue by least squares on the band; wide
 * bands take the central residues from the trapezoidal rule of the function's Cauchy
 * integral along the pole line and fit the outer pairs.  Gaussian-sum fits: the
 * Gaussian coefficients of the function (exp: closed form; phi1: quadrature over c;
 * filter: 1 for |m| <= M0) through the Table 1 rational.  err (may be NULL) receives
 * max |f(ix) - R(ix)| on the band.  Errors: EO_ERR_INVALID_ARG, EO_ERR_FIT,
 * EO_ERR_UNSUPPORTED (the filter on a line fit). */
#define EO_FN_EXP 0
#define EO_FN_PHI1 1
#define EO_FN_FILTER 2
#define EO_FN_PHI2 3
eo_status eo_fit_function(eo_handle_t h, int kind, double c, double *b, double *err);

/* out_dev[k] = f_k(tau L) u for n_out residue sets b_sets[k] (each n complex
 * interleaved, as from eo_fit_function or eo_get_poles) on the handle's poles: one
 * upward sweep and merge pass for all, then the leaf interiors, pole sums and
 * post-map once per set.  u_dev: DEVICE [fields][n_nodes] (one state);
 * out_dev: DEVICE [n_out][fields][n_nodes], not overlapping u_dev.  Synchronises the
 * stream before returning.  Errors: EO_ERR_INVALID_ARG, EO_ERR_CUDA. */
eo_status eo_apply_functions(eo_handle_t h, int n_out, const double *b_sets, const double *u_dev,
                             double *out_dev, void *stream);

/* The filter S(k0 Delta) of Section 3.3 (the variant applied after the conjugate-pole
 * step to damp only the highest wavenumbers), in place on n_rhs x n_fields real fields
 * u_dev (DEVICE [n_rhs][n_fields][n_nodes], fields of any state on the handle's grid).
 * Reading: for a rational Q(z) = sum_m s_m / (z - alpha_m) approximating an even window
 * chi on the imaginary axis, S(k0 Delta) := Q(i (-k0 Delta)^{1/2}), i.e. a mode of
 * wavenumber |k| is multiplied by about chi(sqrt(k0) |k| / 2 pi); since chi is even this
 * is sum_m s_m alpha_m (k0 Delta - alpha_m^2)^{-1}, one shifted-Laplacian solve per pole
 * (real part over the upper poles, weight 2 per pair).  h must be an EO_SW_WALLS handle
 * built with sw_f = 0: its solve (tau^2 g H Delta - alpha^2) w = alpha r is that one with
 * k0 = tau^2 g H, with the natural condition d_n w = 0 on walls (constants pass) and none
 * on a periodic grid.  s_set: n complex residues interleaved (eo_get_poles order), e.g.
 * eo_fit_function(h, EO_FN_FILTER, c, ...) on an EO_FIT_GAUSS handle, whose window keeps
 * sqrt(k0) |k| / 2 pi below about floor(c M) h.  The fields go through in groups of
 * max_rhs; the first call allocates two staging states of max_rhs x 3 x n_nodes doubles
 * in the handle.  Synchronises the stream.  Errors: EO_ERR_INVALID_ARG (null pointer,
 * n_fields or n_rhs < 1, non-finite residue), EO_ERR_UNSUPPORTED (not a shallow-water
 * handle with f = 0), EO_ERR_CUDA. */
eo_status eo_apply_laplacian_filter(eo_handle_t h, const double *s_set, double *u_dev, int n_fields,
                                    int n_rhs, void *stream);

/* Batches of independent instances (the paper has no counterpart).  n built handles -- any
 * grids, kinds, pole counts and precisions, each with its own DEVICE state u_dev[i]
 * ([n_rhs[i]][fields][n_nodes], caller-owned, 1 <= n_rhs[i] <= max_rhs) -- are advanced
 * together: eo_batch_create tunes every handle's launch shapes, then records one step pair
 * of every instance as parallel branches of one CUDA graph (so small instances run side by
 * side); eo_batch_apply(n_steps) replays it n_steps/2 times on `stream` (an odd last step
 * runs per instance).  The states and handles must stay alive and unchanged in address
 * until eo_batch_destroy; a handle may appear once; handles in a batch must not be used
 * concurrently elsewhere (they share their workspace with the graph).  Call
 * eo_batch_create outside any stream capture; it synchronises the device.
 * Errors: EO_ERR_INVALID_ARG, EO_ERR_CUDA. */
eo_status eo_batch_create(int n, const eo_handle_t *handles, double *const *u_dev, const int *n_rhs,
                          eo_batch_t *out);
eo_status eo_batch_apply(eo_batch_t batch, int n_steps, void *stream);
eo_status eo_batch_destroy(eo_batch_t batch);

/* Kernel tracing.  While on, every launch made by eo_apply / eo_apply_host /
 * eo_apply_resolvent is bracketed by CUDA events recorded on the launching stream.
 * eo_get_timing synchronises on those events and returns, per kernel class, the
 * number of launches and their summed device time in milliseconds since the
 * previous eo_get_timing (then resets).  Classes, in order: pre_map, up_leaf,
 * up_merge, root, down_merge, down_leaf, edge_sum, post_map.
 *   n_classes: in: capacity of the arrays; out: number of classes (8).
 *   names: array of n_classes C strings owned by the library (may be NULL). */
eo_status eo_set_timing(eo_handle_t h, int on);
eo_status eo_get_timing(eo_handle_t h, int *n_classes, const char **names, int64_t *launches,
                        double *ms);

/* Device status of the handle's kernels: every wait of the tensor-core kernels is
 * bounded; a wait that gave up sets a status word and the kernel returns.  This call
 * synchronises `stream`, reads the word, and returns EO_ERR_TIMEOUT (*flag = 1) if any
 * kernel of the handle gave up since the build, EO_OK (*flag = 0) otherwise. */
eo_status eo_device_status(eo_handle_t h, void *stream, int *flag);

/* Merge levels 1 .. *levels that eo_apply runs in one launch per sweep for n_rhs
 * right-hand sides (opts.merge_fuse; *levels = 0: one launch per level).  Host only, no device
 * work.  Errors: EO_ERR_INVALID_ARG (null argument, n_rhs outside [1, max_rhs]). */
eo_status eo_fused_levels(eo_handle_t h, int n_rhs, int *levels);

/* Release device memory.  Idempotent on NULL. */
eo_status eo_destroy(eo_handle_t h);

/* Message of the last error on this thread ("" if none).  Valid until the next
 * library call on the same thread. */
const char *eo_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* EXPOP_H */
