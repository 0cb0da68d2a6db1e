// Device-resident operator set and apply workspace of one built handle.
#pragma once

#include <cuda_runtime.h>

#include <complex>
#include <string>
#include <vector>

#include "engine.h"

namespace eo {

typedef double2 cd;   // complex FP64, interleaved (re, im)

#define EO_CUDA_TRY(expr)                                                        \
  do {                                                                           \
    cudaError_t e_ = (expr);                                                     \
    if (e_ != cudaSuccess)                                                       \
      return fail(EO_ERR_CUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// Raise a kernel's dynamic shared-memory cap (and prefer the full carveout) on the
// current device when `bytes` exceeds the 48 KB default.  The attribute is per
// device, so the record `cap` keeps one entry per device ordinal (< 64; larger
// ordinals set it on every call).
inline eo_status ensure_smem(const void* kern, size_t bytes, size_t* cap, size_t set_to) {
  if (bytes <= 48 * 1024) return EO_OK;
  int dev = 0;
  EO_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 64 && bytes <= cap[dev]) return EO_OK;
  const size_t v = set_to > bytes ? set_to : bytes;
  EO_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v));
  EO_CUDA_TRY(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  if (dev < 64) cap[dev] = v;
  return EO_OK;
}

// Launch shape chosen by the autotuner (0: the default heuristic).
struct Tuned {
  int nc = 0;   // columns per block
  int nt = 0;   // threads per block
  int rs = 1;   // row blocks per block product (root wall solve)
};

// One tree level as the kernels see it.
struct LevelDev {
  int nbox = 0, nbx = 0, nby = 0, nbd = 0, nseg = 0, n3 = 0, dir = -1;
  int nbx_child = 0;            // boxes per row one level below
  int* par_child = nullptr;     // [nbd]
  int* par_idx = nullptr;       // [nbd]
  int* a3 = nullptr;            // [n3]
  int* b3 = nullptr;            // [n3]
  int* bseg = nullptr;          // [nbox * nseg]
  int* iseg = nullptr;          // [nbox * n3/q]
  // operators (levels >= 1): [pole][box or 0][...], column-major blocks
  cd* ZU = nullptr;             // rows zu_rows = n3 (+ nbd unless Dirichlet root), cols n3: [-Z; U]
  int zu_rows = 0;
  cd* S = nullptr;              // n3 x nbd (absent at a Dirichlet root)
  int64_t zu_pstride = 0, zu_bstride = 0, s_pstride = 0, s_bstride = 0;
  cd* w3 = nullptr;             // workspace [pole][rhs][nbox][n3]
  const void* aZU = nullptr;    // operators the apply reads (FP64 above, or FP32 copies)
  const void* aS = nullptr;
  int fp32 = 0;                 // this level's blocks: 0 FP64, 1 FP32, 2 FP32 pairs
  Tuned up, down;               // autotuned launch shapes of the merge kernels
  // reflection-symmetric blocks of the forward apply (shared operators; the dense
  // ZU and S stay for the transposed sweeps): ZUs [pole][2][rh x n3/2], Ss
  // [pole][2][n3/2 x nbd/4], orbit maps of the box boundary
  int sym = 0, rh = 0;
  cd* ZUs = nullptr;
  cd* Ss = nullptr;
  int64_t zs_pstride = 0, ss_pstride = 0;
  int* orb = nullptr;           // [nbd]
  int* osg = nullptr;           // [nbd]
  int* mem = nullptr;           // [nbd] = [nbd/4][4]
  const void* aZUs = nullptr;
  const void* aSs = nullptr;
};

struct Handle {
  Grid g;
  Plan plan;
  eo_kind kind = EO_WAVE_DIRICHLET;
  eo_opts opts{};
  Fit fit;
  double tau = 0;
  int P = 0;                    // distinct poles (Im alpha >= 0)
  int K = 2;                    // pre-fields / accumulators per node
  int F = 2;                    // state fields
  int R = 1;                    // max rhs
  int shared = 0;
  std::vector<int> pole_index;  // distinct pole j -> index in the fit's order
  std::vector<std::complex<double>> alpha, cw;   // distinct poles and pole-sum weights
  // leaf operators: H (n_b x n_i), XY = [X | Y] (n_i x (n_i + n_b))
  cd* H = nullptr;
  cd* XY = nullptr;
  int64_t h_pstride = 0, h_bstride = 0, xy_pstride = 0, xy_bstride = 0;
  // root oblique solve (EO_SW_WALLS): Binv [pole][nroot x nroot], or on a square
  // domain the four Fourier blocks of the rotation-symmetric system [pole][4][c4 x c4]
  cd* Binv = nullptr;
  int nroot = 0;
  int c4 = 0;                   // nodes per side of the symmetric root (0: dense root)
  int* c4idx = nullptr;         // [4 * c4] wall index of side k, node s (counterclockwise)
  int* c4inv = nullptr;         // [nroot] inverse map
  int64_t binv_pstride = 0;     // Binv entries per pole
  int fp32 = 0;                 // leaf blocks: 0 FP64, 1 FP32, 2 FP32 pairs
  int root_fp32 = 0;            // root wall solve blocks, same code
  const void* aH = nullptr;     // operators the apply reads
  const void* aXY = nullptr;
  const void* aBinv = nullptr;
  std::vector<LevelDev> lv;
  // per-pole coefficient tables (device, complex): pre-map coefficients [P][K],
  // accumulation weights [P][K], wall rhs coefficients [P][4 sides][2],
  // flux multipliers nu [P][4 sides]
  cd* coef = nullptr;
  cd* wgt = nullptr;
  cd* bcoef = nullptr;
  cd* nu = nullptr;
  double C[4] = {0, 0, 0, 0};   // real constants of the post-map
  double Dx[24 * 24], Dy[24 * 24], Ex[22 * 22], Ey[22 * 22];   // scaled, row-major
  double* dDx = nullptr;        // device copies: Dx, Dy (p x p), Ex, Ey (q x q)
  // apply workspace
  cd* hA = nullptr;             // ping-pong particular fluxes [pole][rhs][box][nbd]
  cd* hB = nullptr;
  cd* E = nullptr;              // edge-node values [pole][rhs][n_edge]
  double* part = nullptr;       // interior partial sums [chunk][rhs][K][n_int]
  int nchunk = 1;
  double* eacc = nullptr;       // edge sums [rhs][K][n_edge]
  double* pre = nullptr;        // pre-map fields: wave A u [rhs][n_int]; SW div F, curl F [rhs][2][n_int]
  double* acoef = nullptr;      // wave: c^2 at every node (device)
  double* afull = nullptr;      // SW: accumulated fields at every node [rhs][K][n_nodes]
  double* ustate = nullptr;     // second state buffer [rhs][F][n_nodes]
  cd* gbar = nullptr;           // adjoint: seeds on the leaf sources [pole][rhs][leaf][q^2]
  double* abar = nullptr;       // adjoint (SW): seeds on the accumulated fields [rhs][3][n_nodes]
  cd* qbar = nullptr;           // adjoint (SW): transposed wall solve [pole][rhs][n_root]
  // fast-diagonalisation leaves (shared constant-coefficient operators)
  int fd = 0;
  int fd_pair = 0;              // leaf arithmetic: 0 FP64, 1 FP32 pairs (tables dc, wd then hold float4)
  int fd_ncol_up = 0, fd_ncol_down = 0;   // autotuned columns per block (0: default)
  double* fd_c = nullptr;       // leaf eigenbases and 1-D vectors (layout in fd.cu)
  cd* fd_dinv = nullptr;        // [P][q*q] 1 / (lx_a + ly_b - kappa_p^2), index b*q + a
  cd* fd_dc = nullptr;          // [P][K][q*q] coef[p][k] * dinv_p (FP64 or FP32-pair complex)
  cd* fd_wd = nullptr;          // workspace [P][K][q*q] pole-sum weight * dinv_p
  double* fd_gsum = nullptr;    // workspace [K][K][q*q] pole-summed particular part
  double* fd_ghat = nullptr;    // workspace [rhs][K][n_int] sources in the eigenbasis
  // tensor-core leaf down-solves (tc.cu): bf16 slices of [X | Y] per pole and operator
  // box with their row exponents, the sources as FP32 pairs, a device status word
  int tc = 0;                   // slices per value (0: off)
  int tc_nks = 0, tc_nke = 0;   // K steps of the X block and of the Y block
  void* tc_A = nullptr;
  int* tc_Aexp = nullptr;
  void* tc_B = nullptr;         // float2 [R][K][n_int]
  int* tc_status = nullptr;
  double* fstage = nullptr;     // S(k0 Delta): two staging states [max_rhs][3][n_nodes]
  // three-field wave form (EO_WAVE_KAPPA), run as shallow water with f = 0, g = -1,
  // H(x) = -kappa(x): per-node weight 1 / kappa on the shift and on the source of v
  int kappa_form = 0;
  double* hw = nullptr;         // 1 / kappa at every node (device)
  int64_t op_bytes = 0, ws_bytes = 0;
  Tuned root_tuned;             // autotuned launch shape of the root wall solve
  int tuned_R = 0;              // n_rhs the launch shapes were tuned for (0: not tuned)
  // recorded step pair (CUDA graph) for repeated applies
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t cap_st = nullptr;
  const double* graph_u = nullptr;
  int graph_R = 0;
  // tracing: events around launches, per kernel class
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<int> ev_class;      // one per recorded pair
  int ev_used = 0;                // pairs recorded
  eo_status trace_begin(cudaStream_t st);
  eo_status trace_end(int cls, cudaStream_t st);
  std::vector<void*> allocs;

  ~Handle();
  eo_status alloc(void** p, size_t bytes, bool op);
  void release(void* p, size_t bytes, bool op);
};

enum { TR_PRE = 0, TR_UP_LEAF, TR_UP_MERGE, TR_ROOT, TR_DOWN_MERGE, TR_DOWN_LEAF, TR_EDGE, TR_POST, TR_N };

// kappa^2 of the elliptic equation div grad w - kappa^2 w = s of distinct pole j
// (wave: (alpha/tau)^2; shallow water: (alpha^2 + (tau f)^2) / (tau^2 g H))
inline std::complex<double> kappa2(const Handle& h, int j) {
  const std::complex<double> al = h.alpha[j];
  if (h.kind == EO_WAVE_DIRICHLET) return (al / h.tau) * (al / h.tau);
  const double tf = h.tau * h.opts.sw_f;
  return (al * al + tf * tf) / (h.tau * h.tau * h.opts.sw_g * h.opts.sw_H);
}

eo_status build(Handle& h, const double* coeff, cudaStream_t st);
eo_status to_reduced(Handle& h, int prec, cudaStream_t st);
eo_status apply(Handle& h, double* u, int n_rhs, int n_steps, cudaStream_t st);
eo_status apply_resolvent(Handle& h, int j, const double* u, double* x, cudaStream_t st);
eo_status apply_adjoint(Handle& h, double* y, int n_rhs, int n_steps, cudaStream_t st);
eo_status apply_resolvent_noalloc(Handle& h, int j, const double* u, double* x, cudaStream_t st);
eo_status apply_functions(Handle& h, int n_out, const cd* wgts, const double* Cs, const double* u, double* out,
                          cudaStream_t st);
eo_status apply_laplacian_filter(Handle& h, const cd* wgts, const double* C, double* u, int ncol, cudaStream_t st);
void pole_weights(const Handle& h, const std::vector<std::complex<double>>& cw, std::vector<cd>& wgt, double C[4]);

// independent instances advanced together through one CUDA graph (apply.cu)
struct Batch {
  std::vector<Handle*> h;
  std::vector<double*> u;
  std::vector<int> R;
  std::vector<cudaStream_t> st;   // one branch stream per instance
  cudaStream_t st0 = nullptr;     // capture (fork/join) stream
  std::vector<cudaEvent_t> ev;    // per-instance join events, then the fork event
  cudaGraphExec_t exec = nullptr;
  ~Batch();
};
eo_status batch_build(Batch& b);
eo_status batch_apply(Batch& b, int n_steps, cudaStream_t st);

// fast-diagonalisation leaves (fd.cu)
eo_status fd_setup(Handle& h, const double* dAii0, const double* dAib, const double* dFbi, cudaStream_t st);
struct Sweep;
eo_status fd_up_leaf(Handle& h, const Sweep& s, int nleaf, cd* h0, cudaStream_t st);
eo_status fd_up_kernel(Handle& h, const Sweep& s, int nleaf, cd* h0, int ncol, cudaStream_t st);
eo_status fd_down_leaf(Handle& h, const Sweep& s, int nleaf, int ncol, int& nchunk, cudaStream_t st);
std::vector<int> fd_ncol_candidates(const Handle& h);

// tensor-core leaf down-solves (tc.cu)
bool tc_eligible(const Handle& h, std::string* why);
eo_status tc_build(Handle& h, cudaStream_t st);
eo_status tc_down_leaf(Handle& h, const Sweep& s, int& nchunk, cudaStream_t st);
eo_status tc_status(Handle& h, cudaStream_t st, int* out);
// merge levels 1 .. n fused into one launch per sweep for R right-hand sides (apply.cu)
int fused_levels(const Handle& h, int R);

}  // namespace eo
