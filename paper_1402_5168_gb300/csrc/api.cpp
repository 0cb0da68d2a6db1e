// C ABI of include/expop.h: argument checks, handle set-up (fit, pole tables,
// device allocations) and dispatch to the build and apply phases.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>

#include "handle.h"

namespace eo {
const char* last_error_cstr();
}

using namespace eo;
typedef std::complex<double> cx;

struct eo_grid_s {
  Grid g;
};
struct eo_handle_s {
  Handle h;
  double* host_stage = nullptr;   // device state used by eo_apply_host
};
struct eo_batch_s {
  Batch b;
};

namespace eo {

Handle::~Handle() {
  for (void* p : allocs) cudaFree(p);
  for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
  if (graph_exec) cudaGraphExecDestroy(graph_exec);
  if (cap_st) cudaStreamDestroy(cap_st);
}

eo_status Handle::alloc(void** p, size_t bytes, bool op) {
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(EO_ERR_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  allocs.push_back(*p);
  (op ? op_bytes : ws_bytes) += (int64_t)bytes;
  return EO_OK;
}

void Handle::release(void* p, size_t bytes, bool op) {
  for (size_t i = 0; i < allocs.size(); ++i)
    if (allocs[i] == p) {
      cudaFree(p);
      allocs.erase(allocs.begin() + i);
      (op ? op_bytes : ws_bytes) -= (int64_t)bytes;
      return;
    }
}

}  // namespace eo

namespace {

template <typename T>
eo_status upload(Handle& h, T** dst, const std::vector<T>& v, cudaStream_t st) {
  eo_status rc = h.alloc((void**)dst, sizeof(T) * std::max<size_t>(1, v.size()), false);
  if (rc) return rc;
  if (!v.empty())
    EO_CUDA_TRY(cudaMemcpyAsync(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st));
  return EO_OK;
}

}  // namespace

// Pole-sum weights [P][K] (device layout) and post-map constants for the pole
// weights cw (c_0 = b_0, c_j = 2 b_j of the conjugate-pole form, Section 3.3):
//   wave: V = Re sum c V_p, U = Re sum (c tau / alpha) V_p - C0 f_u, C0 = Re sum c / alpha;
//   shallow water: h = Re sum c h_p and the two velocity weights c (-alpha / D),
//   c (-tau f / D), D = alpha^2 + (tau f)^2, whose real sums C0, C1 scale the
//   input velocities in the post-map.
void eo::pole_weights(const Handle& h, const std::vector<cx>& cw, std::vector<cd>& wgt, double C[4]) {
  wgt.clear();
  C[0] = C[1] = C[2] = C[3] = 0.0;
  const double tau = h.tau;
  for (int j = 0; j < h.P; ++j) {
    const cx a = h.alpha[j], c = cw[j];
    if (h.kind == EO_WAVE_DIRICHLET) {
      const cx w0 = c, w1 = c * tau / a;
      wgt.push_back(make_double2(w0.real(), w0.imag()));
      wgt.push_back(make_double2(w1.real(), w1.imag()));
      C[0] += (c / a).real();
    } else {
      const double tf = tau * h.opts.sw_f;
      const cx D = a * a + tf * tf;
      const cx w0 = c, w1 = c * (-a / D), w2 = c * (-tf / D);
      for (cx v : {w0, w1, w2}) wgt.push_back(make_double2(v.real(), v.imag()));
      C[0] += w1.real();
      C[1] += w2.real();
    }
  }
}

namespace {

// Counterclockwise order of the root's wall nodes when the walled domain maps onto
// itself under a quarter turn about its centre (square domain, square leaves): side S
// in ascending x, then each side the quarter turn of the previous one.  idx[k * nq + s]
// is the wall index (S, E, N, W blocks of nq) of node s of side k.  False when any
// rotated node is missing or lands on another side.
bool root_c4_map(const Grid& g, const Level& rl, std::vector<int>& idx) {
  const int q = g.q, n = rl.nbd;
  if (rl.sx != rl.sy || n % 4 || std::abs(g.hx - g.hy) > 1e-14 * std::max(g.hx, g.hy)) return false;
  const int nq = n / 4;
  std::vector<double> X, Y;
  g.coords(X, Y);
  const double cx = 0.5 * (g.x0 + g.x1), cy = 0.5 * (g.y0 + g.y1);
  const double tol = 1e-10 * std::max(g.x1 - g.x0, g.y1 - g.y0);
  std::vector<double> bx(n), by(n);
  for (int i = 0; i < n; ++i) {
    const int64_t node = g.n_int + (int64_t)rl.bseg[i / q] * q + (i % q);
    bx[i] = X[node];
    by[i] = Y[node];
  }
  auto turn = [&](int j) {   // wall index of the quarter turn of node j, or -1
    const double rx = cx - (by[j] - cy), ry = cy + (bx[j] - cx);
    for (int i = 0; i < n; ++i)
      if (std::abs(bx[i] - rx) <= tol && std::abs(by[i] - ry) <= tol) return i;
    return -1;
  };
  idx.assign(4 * (size_t)nq, -1);
  for (int s = 0; s < nq; ++s) idx[s] = s;
  for (int k = 1; k < 4; ++k)
    for (int s = 0; s < nq; ++s) {
      const int i = turn(idx[(k - 1) * nq + s]);
      if (i < 0 || i / nq != k) return false;
      idx[k * nq + s] = i;
    }
  for (int s = 0; s < nq; ++s)
    if (turn(idx[3 * nq + s]) != idx[s]) return false;
  for (int s = 1; s < nq; ++s)
    if (!(bx[idx[s]] > bx[idx[s - 1]])) return false;
  return true;
}

// Reflection maps of the first box of merge level lv (all boxes of a level share one
// operator set, so box 0 stands for all).  Ra reflects across the interface line
// (it swaps the children and fixes every interface node), Rb along it (interface
// node t goes to n3 - 1 - t).  For the parent boundary: orbits {i, Ra i, Rb i, Ra Rb i}
// with the smallest index as representative, orb[i], osg[i] = +1 on {rep, Ra rep} and -1
// on {Rb rep, Ra Rb rep}, mem[4 r + g].  False when a reflected node is missing, an
// orbit has fewer than four members or the interface is not symmetric.
bool merge_sym_maps(const Grid& g, const Level& lv, bool need_par, const std::vector<double>& X,
                    const std::vector<double>& Y, std::vector<int>& orb, std::vector<int>& osg,
                    std::vector<int>& mem) {
  const int q = g.q, n3 = lv.n3, nbd = lv.nbd;
  if (n3 % 2 || (need_par && nbd % 4)) return false;
  const double xc = g.x0 + 0.5 * lv.sx * g.hx, yc = g.y0 + 0.5 * lv.sy * g.hy;
  const double tol = 1e-10 * std::max(g.x1 - g.x0, g.y1 - g.y0);
  auto refl = [&](int which, double x, double y, double& rx, double& ry) {   // 0: Ra, 1: Rb
    const bool flip_x = (lv.dir == 0) == (which == 0);
    rx = flip_x ? 2 * xc - x : x;
    ry = flip_x ? y : 2 * yc - y;
  };
  std::vector<double> ix(n3), iy(n3);
  for (int t = 0; t < n3; ++t) {
    const int64_t node = g.n_int + (int64_t)lv.iseg[t / q] * q + (t % q);
    ix[t] = X[node];
    iy[t] = Y[node];
  }
  for (int t = 0; t < n3; ++t) {
    double rx, ry;
    refl(0, ix[t], iy[t], rx, ry);
    if (std::abs(rx - ix[t]) > tol || std::abs(ry - iy[t]) > tol) return false;
    refl(1, ix[t], iy[t], rx, ry);
    if (std::abs(rx - ix[n3 - 1 - t]) > tol || std::abs(ry - iy[n3 - 1 - t]) > tol) return false;
  }
  orb.clear(); osg.clear(); mem.clear();
  if (!need_par) return true;
  std::vector<double> bx(nbd), by(nbd);
  for (int i = 0; i < nbd; ++i) {
    const int64_t node = g.n_int + (int64_t)lv.bseg[i / q] * q + (i % q);
    bx[i] = X[node];
    by[i] = Y[node];
  }
  auto image = [&](int which, int i) {
    double rx, ry;
    refl(which, bx[i], by[i], rx, ry);
    for (int j = 0; j < nbd; ++j)
      if (std::abs(bx[j] - rx) <= tol && std::abs(by[j] - ry) <= tol) return j;
    return -1;
  };
  std::vector<int> ra(nbd), rb(nbd);
  for (int i = 0; i < nbd; ++i) {
    ra[i] = image(0, i);
    rb[i] = image(1, i);
    if (ra[i] < 0 || rb[i] < 0) return false;
  }
  orb.assign(nbd, -1);
  osg.assign(nbd, 0);
  for (int i = 0; i < nbd; ++i) {
    if (orb[i] >= 0) continue;
    const int m4[4] = {i, ra[i], rb[i], ra[rb[i]]};
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b)
        if (m4[a] == m4[b]) return false;
    if (rb[ra[i]] != m4[3]) return false;
    const int r = (int)mem.size() / 4;
    for (int k = 0; k < 4; ++k) {
      if (orb[m4[k]] >= 0) return false;
      orb[m4[k]] = r;
      osg[m4[k]] = k < 2 ? 1 : -1;
      mem.push_back(m4[k]);
    }
  }
  return (int)mem.size() == nbd;
}

// Position in the distinct pole list of pole j (eo_get_poles order), or -1.
int distinct_of(const Handle& h, int j) {
  for (int d = 0; d < h.P; ++d)
    if (h.pole_index[d] == j) return d;
  return -1;
}

eo_status setup(Handle& h, const eo_opts& o, cudaStream_t st) {
  const Grid& g = h.g;
  const int p = g.p, q = g.q, ni = q * q, nb = 4 * q;
  const int nleaf = g.nlx * g.nly;
  // ---- approximant and time step
  const double delta = o.delta > 0 ? o.delta : 1e-10;
  if (!(o.band > 0)) return fail(EO_ERR_INVALID_ARG, "opts.band must be positive");
  eo_status rc;
  if (o.fitter != EO_FIT_LINE && o.fitter != EO_FIT_GAUSS) return fail(EO_ERR_INVALID_ARG, "unknown opts.fitter");
  if (o.merge_fuse < 0 || o.merge_fuse > 4) return fail(EO_ERR_INVALID_ARG, "opts.merge_fuse must be in 0 .. 4");
  if (o.fitter == EO_FIT_GAUSS) {
    if (o.n_poles > 0) return fail(EO_ERR_INVALID_ARG, "the Gaussian-sum fitter takes tau, not n_poles");
    if (!(o.tau > 0)) return fail(EO_ERR_INVALID_ARG, "opts.tau must be positive");
    if ((rc = fit_gauss(o.tau * o.band, o.gauss_h > 0 ? o.gauss_h : 0.18, delta, h.fit))) return rc;
    h.tau = o.tau;
  } else if (o.n_poles > 0) {
    if ((rc = fit_for_poles(o.n_poles, delta, h.fit))) return rc;
    h.tau = h.fit.X / o.band;
  } else {
    if (!(o.tau > 0)) return fail(EO_ERR_INVALID_ARG, "opts.tau must be positive when n_poles == 0");
    if ((rc = fit_for_band(o.tau * o.band, delta, 1 << 20, h.fit))) return rc;
    h.tau = o.tau;
  }
  // distinct poles of the conjugate-pole form: weight 1 on a real pole, 2 on a pair
  distinct_poles(h.fit, h.pole_index);
  h.P = (int)h.pole_index.size();
  h.alpha.resize(h.P);
  h.cw.resize(h.P);
  for (int j = 0; j < h.P; ++j) {
    const int i = h.pole_index[j];
    h.alpha[j] = cx(h.fit.are[i], h.fit.aim[i]);
    h.cw[j] = (h.fit.aim[i] == 0.0 ? 1.0 : 2.0) * cx(h.fit.bre[i], h.fit.bim[i]);
  }
  h.R = std::max(1, o.max_rhs);
  h.shared = o.shared_ops ? 1 : 0;
  // fast-diagonal leaves: shared operators (constant coefficient) and a leaf coupling
  // without the consistent curl term
  const bool curl = h.kind == EO_SW_WALLS && o.sw_consistent && o.sw_f != 0.0;
  h.fd = (h.shared && !o.dense_leaves && !curl) ? 1 : 0;
  h.fd_pair = (h.fd && o.precision == EO_PREC_DF32) ? 1 : 0;
  const double tau = h.tau;
  // ---- per-pole tables
  std::vector<cd> coef, wgt, bcoef, nu;
  double C[4] = {0, 0, 0, 0};
  if (h.kind == EO_WAVE_DIRICHLET) {
    h.K = 2; h.F = 2;
    // elliptic unknown V: (A - (alpha/tau)^2) V = (alpha/tau^2) f_v + (1/tau) A f_u,
    // U = (tau V - f_u) / alpha; sums: V = Re sum c V_p, U = Re sum (c tau/alpha) V_p - C0 f_u
    for (int j = 0; j < h.P; ++j) {
      const cx a = h.alpha[j];
      const cx c0 = a / (tau * tau), c1 = 1.0 / tau;
      coef.push_back(make_double2(c0.real(), c0.imag()));
      coef.push_back(make_double2(c1.real(), c1.imag()));
    }
  } else {
    h.K = 3; h.F = 3;
    const double f = o.sw_f, gg = o.sw_g, H = o.sw_H, tf = tau * f;
    if (!h.kappa_form && (!(gg > 0) || !(H > 0))) return fail(EO_ERR_INVALID_ARG, "sw_g and sw_H must be positive");
    for (int j = 0; j < h.P; ++j) {
      const cx a = h.alpha[j];
      const cx D = a * a + tf * tf;
      const cx c0 = D / (tau * tau * gg * H * a), c1 = -1.0 / (tau * gg), c2 = -f / (gg * a);
      for (cx v : {c0, c1, c2}) coef.push_back(make_double2(v.real(), v.imag()));
      // wall right-hand sides per side S, E, N, W: coefficients of (F1, F2)
      const cx xw0 = -a / (tau * gg), xw1 = -f / gg;       // x-walls: -(a F1 + tau f F2)/(tau g)
      const cx yw0 = f / gg, yw1 = -a / (tau * gg);         // y-walls: (tau f F1 - a F2)/(tau g)
      const cx sides[4][2] = {{yw0, yw1}, {xw0, xw1}, {yw0, yw1}, {xw0, xw1}};
      for (int sd = 0; sd < 4; ++sd)
        for (int t = 0; t < 2; ++t) bcoef.push_back(make_double2(sides[sd][t].real(), sides[sd][t].imag()));
      const double sg[4] = {-1.0, 1.0, 1.0, -1.0};
      for (int sd = 0; sd < 4; ++sd) nu.push_back(make_double2(sg[sd] * a.real(), sg[sd] * a.imag()));
    }
  }
  pole_weights(h, h.cw, wgt, C);
  std::memcpy(h.C, C, sizeof(C));
  // scaled differentiation matrices
  for (int i = 0; i < p * p; ++i) {
    h.Dx[i] = g.D[i] * 2.0 / g.hx;
    h.Dy[i] = g.D[i] * 2.0 / g.hy;
  }
  for (int i = 0; i < q * q; ++i) {
    h.Ex[i] = g.Ed[i] * 2.0 / g.hx;
    h.Ey[i] = g.Ed[i] * 2.0 / g.hy;
  }
  // ---- operator sizes and budget
  const Plan& plan = h.plan;
  const int L = plan.L();
  const int nlo = h.shared ? 1 : nleaf;
  const int64_t P = h.P;
  int64_t ops = P * nlo * ((int64_t)nb * ni + (int64_t)ni * (ni + nb));
  h.lv.resize(L + 1);
  std::vector<std::vector<int>> sym_orb(L + 1), sym_osg(L + 1), sym_mem(L + 1);
  std::vector<double> gx, gy;
  // (a periodic square's seam nodes carry the coordinates of lines x0, y0, so the
  // reflection maps of boxes that reach a seam are not found from them: periodic
  // grids keep the dense merge blocks)
  if (h.shared && !curl && !o.merge_dense && !g.periodic) g.coords(gx, gy);
  for (int l = 1; l <= L; ++l) {
    const Level& lv = plan.lv[l];
    LevelDev& ld = h.lv[l];
    const bool root = l == L;
    const bool need_par = !(root && h.kind == EO_WAVE_DIRICHLET && !g.periodic);
    const int nbo = h.shared ? 1 : lv.nbox;
    ld.zu_rows = lv.n3 + (need_par ? lv.nbd : 0);
    ld.zu_bstride = h.shared ? 0 : (int64_t)ld.zu_rows * lv.n3;
    ld.zu_pstride = (int64_t)nbo * ld.zu_rows * lv.n3;
    ops += P * ld.zu_pstride;
    if (need_par) {
      ld.s_bstride = h.shared ? 0 : (int64_t)lv.n3 * lv.nbd;
      ld.s_pstride = (int64_t)nbo * lv.n3 * lv.nbd;
      ops += P * ld.s_pstride;
    }
    // reflection-symmetric blocks (constant coefficient: shared operators, no curl term)
    if (!gx.empty() && merge_sym_maps(g, lv, need_par, gx, gy, sym_orb[l], sym_osg[l], sym_mem[l])) {
      const int n3h = lv.n3 / 2, nbq = need_par ? lv.nbd / 4 : 0;
      ld.sym = 1;
      ld.rh = n3h + nbq;
      ld.zs_pstride = 2LL * ld.rh * n3h;
      ld.ss_pstride = 2LL * n3h * nbq;
      ops += P * (ld.zs_pstride + ld.ss_pstride);
    }
  }
  std::vector<int> c4idx;
  if (g.periodic) {
    // seam system of the root box merged with itself: half of its boundary nodes
    h.nroot = plan.lv[L].nbd / 2;
    h.binv_pstride = (int64_t)h.nroot * h.nroot;
    ops += P * h.binv_pstride;
  } else if (h.kind == EO_SW_WALLS) {
    h.nroot = plan.lv[L].nbd;
    if (!o.root_dense && L >= 1 && root_c4_map(g, plan.lv[L], c4idx)) h.c4 = h.nroot / 4;
    h.binv_pstride = h.c4 ? 4LL * h.c4 * h.c4 : (int64_t)h.nroot * h.nroot;
    ops += P * h.binv_pstride;
  }
  const double op_gb = (double)ops * (o.precision == EO_PREC_FP32 ? sizeof(float2) : sizeof(cd)) / 1e9;
  if (o.mem_budget_gb > 0 && op_gb > o.mem_budget_gb)
    return fail(EO_ERR_BUDGET, "operators need " + std::to_string(op_gb) + " GB, over the budget");
  // ---- allocations: operators
  h.h_bstride = h.shared ? 0 : (int64_t)nb * ni;
  h.h_pstride = (int64_t)nlo * nb * ni;
  h.xy_bstride = h.shared ? 0 : (int64_t)ni * (ni + nb);
  h.xy_pstride = (int64_t)nlo * ni * (ni + nb);
  if ((rc = h.alloc((void**)&h.H, sizeof(cd) * P * h.h_pstride, true))) return rc;
  if ((rc = h.alloc((void**)&h.XY, sizeof(cd) * P * h.xy_pstride, true))) return rc;
  for (int l = 1; l <= L; ++l) {
    LevelDev& ld = h.lv[l];
    if ((rc = h.alloc((void**)&ld.ZU, sizeof(cd) * P * ld.zu_pstride, true))) return rc;
    if (ld.s_pstride && (rc = h.alloc((void**)&ld.S, sizeof(cd) * P * ld.s_pstride, true))) return rc;
    if (ld.sym) {
      if ((rc = h.alloc((void**)&ld.ZUs, sizeof(cd) * P * ld.zs_pstride, true))) return rc;
      if (ld.ss_pstride && (rc = h.alloc((void**)&ld.Ss, sizeof(cd) * P * ld.ss_pstride, true))) return rc;
      if (!sym_orb[l].empty()) {
        if ((rc = upload(h, &ld.orb, sym_orb[l], st))) return rc;
        if ((rc = upload(h, &ld.osg, sym_osg[l], st))) return rc;
        if ((rc = upload(h, &ld.mem, sym_mem[l], st))) return rc;
      }
    }
  }
  if ((h.kind == EO_SW_WALLS || g.periodic) &&
      (rc = h.alloc((void**)&h.Binv, sizeof(cd) * P * h.binv_pstride, true)))
    return rc;
  if (h.c4) {
    std::vector<int> inv(h.nroot, -1);
    for (int e = 0; e < 4 * h.c4; ++e) inv[c4idx[e]] = e;
    if ((rc = upload(h, &h.c4idx, c4idx, st))) return rc;
    if ((rc = upload(h, &h.c4inv, inv, st))) return rc;
  }
  // ---- index maps
  for (int l = 0; l <= L; ++l) {
    const Level& lv = plan.lv[l];
    LevelDev& ld = h.lv[l];
    ld.nbox = lv.nbox; ld.nbx = lv.nbx; ld.nby = lv.nby; ld.nbd = lv.nbd; ld.nseg = lv.nseg;
    ld.n3 = lv.n3; ld.dir = lv.dir;
    if ((rc = upload(h, &ld.bseg, lv.bseg, st))) return rc;
    if (l >= 1) {
      ld.nbx_child = plan.lv[l - 1].nbx;
      if ((rc = upload(h, &ld.par_child, lv.par_child, st))) return rc;
      if ((rc = upload(h, &ld.par_idx, lv.par_idx, st))) return rc;
      if ((rc = upload(h, &ld.a3, lv.a3, st))) return rc;
      if ((rc = upload(h, &ld.b3, lv.b3, st))) return rc;
      if ((rc = upload(h, &ld.iseg, lv.iseg, st))) return rc;
    }
  }
  if ((rc = upload(h, &h.coef, coef, st))) return rc;
  if ((rc = upload(h, &h.wgt, wgt, st))) return rc;
  if (h.kind == EO_SW_WALLS) {
    if ((rc = upload(h, &h.bcoef, bcoef, st))) return rc;
    if ((rc = upload(h, &h.nu, nu, st))) return rc;
  }
  if ((rc = h.alloc((void**)&h.dDx, sizeof(double) * (2 * p * p + 2 * q * q), false))) return rc;
  // ---- apply workspace
  const int64_t R = h.R;
  int64_t hmax = 0;
  for (int l = 0; l <= L; ++l) hmax = std::max<int64_t>(hmax, (int64_t)plan.lv[l].nbox * plan.lv[l].nbd);
  if ((rc = h.alloc((void**)&h.hA, sizeof(cd) * P * R * hmax, false))) return rc;
  if ((rc = h.alloc((void**)&h.hB, sizeof(cd) * P * R * hmax, false))) return rc;
  // finite contents for the launch-shape autotuner, which runs on this workspace
  EO_CUDA_TRY(cudaMemsetAsync(h.hA, 0, sizeof(cd) * P * R * hmax, st));
  EO_CUDA_TRY(cudaMemsetAsync(h.hB, 0, sizeof(cd) * P * R * hmax, st));
  if ((rc = h.alloc((void**)&h.E, sizeof(cd) * P * R * g.n_edge, false))) return rc;
  EO_CUDA_TRY(cudaMemsetAsync(h.E, 0, sizeof(cd) * P * R * g.n_edge, st));
  for (int l = 1; l <= L; ++l) {
    LevelDev& ld = h.lv[l];
    if ((rc = h.alloc((void**)&ld.w3, sizeof(cd) * P * R * ld.nbox * ld.n3, false))) return rc;
    EO_CUDA_TRY(cudaMemsetAsync(ld.w3, 0, sizeof(cd) * P * R * ld.nbox * ld.n3, st));
  }
  h.nchunk = (int)std::min<int64_t>(P, 64);
  if ((rc = h.alloc((void**)&h.part, sizeof(double) * h.nchunk * R * h.K * g.n_int, false))) return rc;
  if ((rc = h.alloc((void**)&h.eacc, sizeof(double) * R * h.K * g.n_edge, false))) return rc;
  if ((rc = h.alloc((void**)&h.ustate, sizeof(double) * R * h.F * g.n_nodes, false))) return rc;
  EO_CUDA_TRY(cudaMemsetAsync(h.ustate, 0, sizeof(double) * R * h.F * g.n_nodes, st));
  if ((rc = h.alloc((void**)&h.pre, sizeof(double) * R * 2 * g.n_int, false))) return rc;
  if (h.fd) {
    if ((rc = h.alloc((void**)&h.fd_c, sizeof(double) * (4 * ni + 10 * q), true))) return rc;
    if ((rc = h.alloc((void**)&h.fd_dinv, sizeof(cd) * P * ni, true))) return rc;
    if ((rc = h.alloc((void**)&h.fd_dc, sizeof(cd) * P * h.K * ni, true))) return rc;
    if ((rc = h.alloc((void**)&h.fd_wd, sizeof(cd) * P * h.K * ni, false))) return rc;
    if ((rc = h.alloc((void**)&h.fd_gsum, sizeof(double) * h.K * h.K * ni, false))) return rc;
    if ((rc = h.alloc((void**)&h.fd_ghat, sizeof(double) * R * h.K * g.n_int, false))) return rc;
    EO_CUDA_TRY(cudaMemsetAsync(h.fd_ghat, 0, sizeof(double) * R * h.K * g.n_int, st));
  }
  if (h.kind == EO_SW_WALLS) {
    if ((rc = h.alloc((void**)&h.afull, sizeof(double) * R * h.K * g.n_nodes, false))) return rc;
    if (h.kappa_form && (rc = h.alloc((void**)&h.hw, sizeof(double) * g.n_nodes, true))) return rc;
  } else {
    if ((rc = h.alloc((void**)&h.acoef, sizeof(double) * g.n_nodes, false))) return rc;
  }
  return EO_OK;
}

}  // namespace

extern "C" {

static eo_status grid_create(int nlx, int nly, int p, double x0, double x1, double y0, double y1, int periodic,
                             eo_grid_t* out) {
  if (!out) return fail(EO_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  eo_grid_s* gs = new (std::nothrow) eo_grid_s;
  if (!gs) return fail(EO_ERR_OOM, "host allocation failed");
  eo_status rc = make_grid(nlx, nly, p, x0, x1, y0, y1, gs->g, periodic);
  if (rc) { delete gs; return rc; }
  *out = gs;
  set_error("");
  return EO_OK;
}

eo_status eo_grid_create(int nlx, int nly, int p, double x0, double x1, double y0, double y1,
                         eo_grid_t* out) {
  return grid_create(nlx, nly, p, x0, x1, y0, y1, 0, out);
}

eo_status eo_grid_create_periodic(int nlx, int nly, int p, double x0, double x1, double y0, double y1,
                                  eo_grid_t* out) {
  return grid_create(nlx, nly, p, x0, x1, y0, y1, 1, out);
}

eo_status eo_grid_periodic(eo_grid_t grid, int* periodic) {
  if (!grid || !periodic) return fail(EO_ERR_INVALID_ARG, "null argument");
  *periodic = grid->g.periodic;
  return EO_OK;
}

eo_status eo_grid_info(eo_grid_t grid, int64_t* n_nodes, int64_t* n_interior, int64_t* n_edge) {
  if (!grid) return fail(EO_ERR_INVALID_ARG, "null grid");
  if (n_nodes) *n_nodes = grid->g.n_nodes;
  if (n_interior) *n_interior = grid->g.n_int;
  if (n_edge) *n_edge = grid->g.n_edge;
  return EO_OK;
}

eo_status eo_grid_nodes(eo_grid_t grid, double* x, double* y) {
  if (!grid || !x || !y) return fail(EO_ERR_INVALID_ARG, "null argument");
  std::vector<double> vx, vy;
  grid->g.coords(vx, vy);
  std::memcpy(x, vx.data(), sizeof(double) * vx.size());
  std::memcpy(y, vy.data(), sizeof(double) * vy.size());
  return EO_OK;
}

eo_status eo_grid_destroy(eo_grid_t grid) {
  delete grid;
  return EO_OK;
}

eo_status eo_build_operator(eo_grid_t grid, eo_kind kind, const double* coeff, const eo_opts* opts,
                            void* stream, eo_handle_t* out) {
  if (!grid || !opts || !out) return fail(EO_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (kind != EO_WAVE_DIRICHLET && kind != EO_SW_WALLS && kind != EO_WAVE_KAPPA)
    return fail(EO_ERR_INVALID_ARG, "unknown kind");
  const bool kap = kind == EO_WAVE_KAPPA;
  if (kap && !grid->g.periodic)
    return fail(EO_ERR_UNSUPPORTED, "EO_WAVE_KAPPA is built on periodic grids (eo_grid_create_periodic)");
  if (kap && opts->tensor_leaves) return fail(EO_ERR_UNSUPPORTED, "tensor_leaves: not built for EO_WAVE_KAPPA");
  if (kind != EO_SW_WALLS && !coeff) return fail(EO_ERR_INVALID_ARG, "wave kinds need their coefficient at the nodes");
  if (kind != EO_SW_WALLS && opts->shared_ops)
    return fail(EO_ERR_INVALID_ARG, "shared operators need constant coefficients (EO_SW_WALLS)");
  if (opts->precision != EO_PREC_FP64 && opts->precision != EO_PREC_FP32 && opts->precision != EO_PREC_DF32)
    return fail(EO_ERR_INVALID_ARG, "unknown precision");
  if (opts->max_rhs < 0) return fail(EO_ERR_INVALID_ARG, "max_rhs must be >= 1");
  if (kind != EO_SW_WALLS)
    for (int64_t i = 0; i < grid->g.n_nodes; ++i)
      if (!(coeff[i] > 0) || !std::isfinite(coeff[i]))
        return fail(EO_ERR_INVALID_ARG, kap ? "kappa must be positive and finite at every node"
                                            : "c^2 must be positive and finite at every node");
  eo_handle_s* hs = new (std::nothrow) eo_handle_s;
  if (!hs) return fail(EO_ERR_OOM, "host allocation failed");
  Handle& h = hs->h;
  h.g = grid->g;
  h.kind = kind;
  h.opts = *opts;
  if (kap) {
    // the three-field wave form is shallow water with f = 0, g = -1 and depth
    // H(x) = -kappa(x): the shift and the source of v carry 1 / (g H) = 1 / kappa per node
    h.kind = EO_SW_WALLS;
    h.kappa_form = 1;
    h.opts.sw_f = 0.0;
    h.opts.sw_g = -1.0;
    h.opts.sw_H = -1.0;
    h.opts.sw_consistent = 0;
  }
  make_plan(h.g, h.plan);
  cudaStream_t st = (cudaStream_t)stream;
  eo_status rc = setup(h, h.opts, st);
  if (!rc) rc = build(h, coeff, st);
  if (!rc && opts->tensor_leaves) {
    // split the FP64 leaf operators for the tensor cores before reduced copies replace them
    std::string why;
    if (!tc_eligible(h, &why)) rc = fail(EO_ERR_UNSUPPORTED, "tensor_leaves: " + why);
    else rc = tc_build(h, st);
  }
  if (!rc && opts->precision != EO_PREC_FP64) rc = to_reduced(h, opts->precision, st);
  if (rc) {
    delete hs;
    return rc;
  }
  *out = hs;
  set_error("");
  return EO_OK;
}

eo_status eo_fit_function(eo_handle_t hd, int kind, double c, double* b, double* err) {
  if (!hd || !b) return fail(EO_ERR_INVALID_ARG, "null argument");
  std::vector<cx> bv;
  double e = 0;
  eo_status rc = fit_function(hd->h.fit, kind, c, bv, e);
  if (rc) return rc;
  for (size_t i = 0; i < bv.size(); ++i) { b[2 * i] = bv[i].real(); b[2 * i + 1] = bv[i].imag(); }
  if (err) *err = e;
  set_error("");
  return EO_OK;
}

eo_status eo_apply_functions(eo_handle_t hd, int n_out, const double* b_sets, const double* u_dev, double* out_dev,
                             void* stream) {
  if (!hd || !b_sets || !u_dev || !out_dev) return fail(EO_ERR_INVALID_ARG, "null argument");
  if (n_out < 1) return fail(EO_ERR_INVALID_ARG, "n_out must be >= 1");
  Handle& h = hd->h;
  const int N = h.fit.N();
  std::vector<cd> wall;
  std::vector<double> Call(4 * (size_t)n_out);
  for (int k = 0; k < n_out; ++k) {
    const double* bk = b_sets + (size_t)2 * N * k;
    std::vector<cx> cw(h.P);
    for (int j = 0; j < h.P; ++j) {
      const int i = h.pole_index[j];
      if (!std::isfinite(bk[2 * i]) || !std::isfinite(bk[2 * i + 1])) return fail(EO_ERR_INVALID_ARG, "non-finite residue");
      cw[j] = (h.fit.aim[i] == 0.0 ? 1.0 : 2.0) * cx(bk[2 * i], bk[2 * i + 1]);
    }
    std::vector<cd> w;
    pole_weights(h, cw, w, &Call[4 * (size_t)k]);
    wall.insert(wall.end(), w.begin(), w.end());
  }
  cudaStream_t st = (cudaStream_t)stream;
  cd* dw = nullptr;
  EO_CUDA_TRY(cudaMallocAsync(&dw, sizeof(cd) * wall.size(), st));
  EO_CUDA_TRY(cudaMemcpyAsync(dw, wall.data(), sizeof(cd) * wall.size(), cudaMemcpyHostToDevice, st));
  eo_status rc = apply_functions(h, n_out, dw, Call.data(), u_dev, out_dev, st);
  cudaFreeAsync(dw, st);
  EO_CUDA_TRY(cudaStreamSynchronize(st));
  if (!rc) set_error("");
  return rc;
}

eo_status eo_apply_laplacian_filter(eo_handle_t hd, const double* s_set, double* u_dev, int n_fields, int n_rhs,
                                    void* stream) {
  if (!hd || !s_set || !u_dev) return fail(EO_ERR_INVALID_ARG, "null argument");
  if (n_fields < 1 || n_rhs < 1) return fail(EO_ERR_INVALID_ARG, "n_fields and n_rhs must be >= 1");
  Handle& h = hd->h;
  if (h.kind != EO_SW_WALLS || h.opts.sw_f != 0.0 || h.kappa_form)
    return fail(EO_ERR_UNSUPPORTED, "the Laplacian filter needs a shallow-water handle built with f = 0");
  std::vector<cx> cw(h.P);
  for (int j = 0; j < h.P; ++j) {
    const int i = h.pole_index[j];
    if (!std::isfinite(s_set[2 * i]) || !std::isfinite(s_set[2 * i + 1]))
      return fail(EO_ERR_INVALID_ARG, "non-finite residue");
    cw[j] = (h.fit.aim[i] == 0.0 ? 1.0 : 2.0) * cx(s_set[2 * i], s_set[2 * i + 1]);
  }
  std::vector<cd> w;
  double C[4];
  pole_weights(h, cw, w, C);
  cudaStream_t st = (cudaStream_t)stream;
  cd* dw = nullptr;
  EO_CUDA_TRY(cudaMallocAsync(&dw, sizeof(cd) * w.size(), st));
  eo_status rc = EO_OK;
  const cudaError_t e = cudaMemcpyAsync(dw, w.data(), sizeof(cd) * w.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) rc = fail(EO_ERR_CUDA, std::string("cudaMemcpyAsync: ") + cudaGetErrorString(e));
  if (!rc) rc = apply_laplacian_filter(h, dw, C, u_dev, n_fields * n_rhs, st);
  cudaFreeAsync(dw, st);
  const cudaError_t e2 = cudaStreamSynchronize(st);
  if (!rc && e2 != cudaSuccess) rc = fail(EO_ERR_CUDA, std::string("cudaStreamSynchronize: ") + cudaGetErrorString(e2));
  if (!rc) set_error("");
  return rc;
}

eo_status eo_batch_create(int n, const eo_handle_t* handles, double* const* u_dev, const int* n_rhs,
                          eo_batch_t* out) {
  if (!out) return fail(EO_ERR_INVALID_ARG, "null output pointer");
  *out = nullptr;
  if (n < 1 || !handles || !u_dev || !n_rhs) return fail(EO_ERR_INVALID_ARG, "empty batch or null array");
  eo_batch_s* bs = new (std::nothrow) eo_batch_s;
  if (!bs) return fail(EO_ERR_OOM, "host allocation failed");
  for (int i = 0; i < n; ++i) {
    if (!handles[i] || !u_dev[i]) { delete bs; return fail(EO_ERR_INVALID_ARG, "null handle or state"); }
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) { delete bs; return fail(EO_ERR_INVALID_ARG, "a handle appears twice"); }
    Handle& h = handles[i]->h;
    if (n_rhs[i] < 1 || n_rhs[i] > h.R) { delete bs; return fail(EO_ERR_INVALID_ARG, "n_rhs out of range"); }
    if (h.timing) { delete bs; return fail(EO_ERR_INVALID_ARG, "tracing is on for a batched handle"); }
    bs->b.h.push_back(&h);
    bs->b.u.push_back(u_dev[i]);
    bs->b.R.push_back(n_rhs[i]);
  }
  eo_status rc = batch_build(bs->b);
  if (rc) { delete bs; return rc; }
  *out = bs;
  set_error("");
  return EO_OK;
}

eo_status eo_batch_apply(eo_batch_t batch, int n_steps, void* stream) {
  if (!batch) return fail(EO_ERR_INVALID_ARG, "null batch");
  return batch_apply(batch->b, n_steps, (cudaStream_t)stream);
}

eo_status eo_batch_destroy(eo_batch_t batch) {
  delete batch;
  return EO_OK;
}

eo_status eo_fit(int n_poles, double X, double delta, int cap, double* alpha, double* b, int* n,
                 double* X_out) {
  if (!n || !X_out) return fail(EO_ERR_INVALID_ARG, "null argument");
  Fit f;
  const double d = delta > 0 ? delta : 1e-10;
  eo_status rc = n_poles > 0 ? fit_for_poles(n_poles, d, f) : fit_for_band(X, d, 1 << 20, f);
  if (rc) return rc;
  *n = f.N();
  *X_out = f.X;
  if (cap < f.N() || !alpha || !b) return fail(EO_ERR_INVALID_ARG, "output arrays too small");
  for (int i = 0; i < f.N(); ++i) {
    alpha[2 * i] = f.are[i]; alpha[2 * i + 1] = f.aim[i];
    b[2 * i] = f.bre[i]; b[2 * i + 1] = f.bim[i];
  }
  set_error("");
  return EO_OK;
}

eo_status eo_fit_gauss(double X, double h, double delta, int cap, double* alpha, double* b, int* n, int* M) {
  if (!n) return fail(EO_ERR_INVALID_ARG, "null argument");
  Fit f;
  eo_status rc = fit_gauss(X, h > 0 ? h : 0.18, delta > 0 ? delta : 1e-10, f);
  if (rc) return rc;
  *n = f.N();
  if (M) *M = f.gM;
  if (cap < f.N() || !alpha || !b) return fail(EO_ERR_INVALID_ARG, "output arrays too small");
  for (int i = 0; i < f.N(); ++i) {
    alpha[2 * i] = f.are[i]; alpha[2 * i + 1] = f.aim[i];
    b[2 * i] = f.bre[i]; b[2 * i + 1] = f.bim[i];
  }
  set_error("");
  return EO_OK;
}

eo_status eo_get_poles(eo_handle_t hd, double* alpha, double* b, int* n, double* tau, double* X) {
  if (!hd) return fail(EO_ERR_INVALID_ARG, "null handle");
  const Fit& f = hd->h.fit;
  if (n) *n = f.N();
  if (tau) *tau = hd->h.tau;
  if (X) *X = f.X;
  if (alpha)
    for (int i = 0; i < f.N(); ++i) { alpha[2 * i] = f.are[i]; alpha[2 * i + 1] = f.aim[i]; }
  if (b)
    for (int i = 0; i < f.N(); ++i) { b[2 * i] = f.bre[i]; b[2 * i + 1] = f.bim[i]; }
  return EO_OK;
}

eo_status eo_memory(eo_handle_t hd, int64_t* operator_bytes, int64_t* workspace_bytes) {
  if (!hd) return fail(EO_ERR_INVALID_ARG, "null handle");
  if (operator_bytes) *operator_bytes = hd->h.op_bytes;
  if (workspace_bytes) *workspace_bytes = hd->h.ws_bytes;
  return EO_OK;
}

eo_status eo_apply(eo_handle_t hd, double* u_dev, int n_rhs, int n_steps, void* stream) {
  if (!hd) return fail(EO_ERR_INVALID_ARG, "null handle");
  return apply(hd->h, u_dev, n_rhs, n_steps, (cudaStream_t)stream);
}

eo_status eo_device_status(eo_handle_t hd, void* stream, int* flag) {
  if (!hd || !flag) return fail(EO_ERR_INVALID_ARG, "null argument");
  eo_status rc = tc_status(hd->h, (cudaStream_t)stream, flag);
  if (rc) return rc;
  if (*flag) return fail(EO_ERR_TIMEOUT, "a bounded device wait gave up");
  set_error("");
  return EO_OK;
}

eo_status eo_fused_levels(eo_handle_t hd, int n_rhs, int* levels) {
  if (!hd || !levels) return fail(EO_ERR_INVALID_ARG, "null argument");
  if (n_rhs < 1 || n_rhs > hd->h.R) return fail(EO_ERR_INVALID_ARG, "n_rhs out of range [1, max_rhs]");
  *levels = fused_levels(hd->h, n_rhs);
  set_error("");
  return EO_OK;
}

eo_status eo_apply_adjoint(eo_handle_t hd, double* y_dev, int n_rhs, int n_steps, void* stream) {
  if (!hd) return fail(EO_ERR_INVALID_ARG, "null handle");
  if (hd->h.g.periodic) return fail(EO_ERR_UNSUPPORTED, "the transposed sweeps are built for walled grids only");
  return apply_adjoint(hd->h, y_dev, n_rhs, n_steps, (cudaStream_t)stream);
}

eo_status eo_apply_host(eo_handle_t hd, double* u_host, int n_rhs, int n_steps, void* stream) {
  if (!hd || !u_host) return fail(EO_ERR_INVALID_ARG, "null argument");
  Handle& h = hd->h;
  if (n_rhs < 1 || n_rhs > h.R) return fail(EO_ERR_INVALID_ARG, "n_rhs out of range [1, max_rhs]");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bytes = sizeof(double) * (size_t)n_rhs * h.F * h.g.n_nodes;
  if (!hd->host_stage) {
    eo_status rc = h.alloc((void**)&hd->host_stage, sizeof(double) * (size_t)h.R * h.F * h.g.n_nodes, false);
    if (rc) return rc;
  }
  EO_CUDA_TRY(cudaMemcpyAsync(hd->host_stage, u_host, bytes, cudaMemcpyHostToDevice, st));
  eo_status rc = apply(h, hd->host_stage, n_rhs, n_steps, st);
  if (rc) return rc;
  EO_CUDA_TRY(cudaMemcpyAsync(u_host, hd->host_stage, bytes, cudaMemcpyDeviceToHost, st));
  EO_CUDA_TRY(cudaStreamSynchronize(st));
  return EO_OK;
}

eo_status eo_apply_resolvent(eo_handle_t hd, int j, const double* u_dev, double* x_dev, void* stream) {
  if (!hd || !u_dev || !x_dev) return fail(EO_ERR_INVALID_ARG, "null argument");
  // j is an index of eo_get_poles' order; map to the distinct pole list (Im >= 0)
  const int d = distinct_of(hd->h, j);
  if (d < 0) return fail(EO_ERR_INVALID_ARG, "pole index must have Im(alpha) >= 0");
  return apply_resolvent(hd->h, d, u_dev, x_dev, (cudaStream_t)stream);
}

eo_status eo_set_timing(eo_handle_t hd, int on) {
  if (!hd) return fail(EO_ERR_INVALID_ARG, "null handle");
  hd->h.timing = on != 0;
  hd->h.ev_used = 0;
  return EO_OK;
}

eo_status eo_get_timing(eo_handle_t hd, int* n_classes, const char** names, int64_t* launches, double* ms) {
  static const char* kNames[TR_N] = {"pre_map", "up_leaf", "up_merge", "root", "down_merge", "down_leaf",
                                     "edge_sum", "post_map"};
  if (!hd || !n_classes) return fail(EO_ERR_INVALID_ARG, "null argument");
  const int cap = *n_classes;
  *n_classes = TR_N;
  if (cap < TR_N) return fail(EO_ERR_INVALID_ARG, "arrays need room for 8 classes");
  Handle& h = hd->h;
  for (int c = 0; c < TR_N; ++c) {
    if (names) names[c] = kNames[c];
    if (launches) launches[c] = 0;
    if (ms) ms[c] = 0.0;
  }
  for (int i = 0; i < h.ev_used; ++i) {
    EO_CUDA_TRY(cudaEventSynchronize(h.ev_pool[2 * i + 1]));
    float t = 0;
    EO_CUDA_TRY(cudaEventElapsedTime(&t, h.ev_pool[2 * i], h.ev_pool[2 * i + 1]));
    const int c = h.ev_class[i];
    if (launches) launches[c] += 1;
    if (ms) ms[c] += t;
  }
  h.ev_used = 0;
  return EO_OK;
}

eo_status eo_apply_resolvent_noalloc(eo_handle_t hd, int j, const double* u_dev, double* x_dev, void* stream) {
  if (!hd || !u_dev || !x_dev) return fail(EO_ERR_INVALID_ARG, "null argument");
  const int d = distinct_of(hd->h, j);
  if (d < 0) return fail(EO_ERR_INVALID_ARG, "pole index must have Im(alpha) >= 0");
  return apply_resolvent_noalloc(hd->h, d, u_dev, x_dev, (cudaStream_t)stream);
}

eo_status eo_destroy(eo_handle_t hd) {
  delete hd;
  return EO_OK;
}

const char* eo_last_error(void) { return last_error_cstr(); }

}  // extern "C"
