// Leaf grid, public node numbering and the nested-dissection tree plan
// (Section 2.2, Fig. 1; Section 2.3).
#include <cmath>
#include <sstream>

#include "engine.h"

namespace eo {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }
eo_status fail(eo_status st, const std::string& msg) {
  g_err = msg;
  return st;
}
const char* last_error_cstr() { return g_err.c_str(); }

// Differentiation matrix of the interpolating polynomial through nodes x
// (barycentric weights; diagonal from the rows of a constant summing to 0).
static std::vector<double> diffmat(const std::vector<double>& x) {
  const int n = (int)x.size();
  std::vector<double> w(n, 1.0), D((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (j != i) w[i] /= (x[i] - x[j]);
  for (int i = 0; i < n; ++i) {
    double s = 0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      D[(size_t)i * n + j] = (w[j] / w[i]) / (x[i] - x[j]);
      s += D[(size_t)i * n + j];
    }
    D[(size_t)i * n + i] = -s;
  }
  return D;
}

static bool pow2(int v) { return v >= 1 && (v & (v - 1)) == 0; }

eo_status make_grid(int nlx, int nly, int p, double x0, double x1, double y0, double y1,
                    Grid& g, int periodic) {
  if (!pow2(nlx) || !pow2(nly)) return fail(EO_ERR_INVALID_ARG, "nlx, nly must be powers of two");
  if (p < 4 || p > 24) return fail(EO_ERR_INVALID_ARG, "p must be in [4, 24]");
  if (!(x1 > x0) || !(y1 > y0)) return fail(EO_ERR_INVALID_ARG, "empty domain");
  if ((int64_t)nlx * nly > (1 << 16)) return fail(EO_ERR_INVALID_ARG, "too many leaves");
  g.nlx = nlx; g.nly = nly; g.p = p; g.q = p - 2;
  g.x0 = x0; g.x1 = x1; g.y0 = y0; g.y1 = y1;
  g.hx = (x1 - x0) / nlx;
  g.hy = (y1 - y0) / nly;
  g.xi.resize(p);
  for (int k = 0; k < p; ++k) g.xi[k] = -std::cos(M_PI * k / (p - 1));
  g.xi[0] = -1.0;
  g.xi[p - 1] = 1.0;
  g.D = diffmat(g.xi);
  std::vector<double> inner(g.xi.begin() + 1, g.xi.end() - 1);
  g.Ed = diffmat(inner);
  const int64_t q = g.q;
  g.n_int = (int64_t)nlx * nly * q * q;
  g.periodic = periodic ? 1 : 0;
  g.nhl = periodic ? nly : nly + 1;
  g.nvl = periodic ? nlx : nlx + 1;
  g.n_hseg = (int64_t)nlx * g.nhl;
  g.n_vseg = (int64_t)g.nvl * nly;
  g.n_seg = g.n_hseg + g.n_vseg;
  g.n_edge = g.n_seg * q;
  g.n_nodes = g.n_int + g.n_edge;
  return EO_OK;
}

int64_t Grid::node_id(int a, int b, int k, int j) const {
  const bool kin = k > 0 && k < p - 1, jin = j > 0 && j < p - 1;
  if (kin && jin) return ((int64_t)b * nlx + a) * q * q + (int64_t)(j - 1) * q + (k - 1);
  if (kin) return n_int + hseg(j == 0 ? b : b + 1, a) * q + (k - 1);
  if (jin) return n_int + vseg(b, k == 0 ? a : a + 1) * q + (j - 1);
  return -1;
}

void Grid::coords(std::vector<double>& x, std::vector<double>& y) const {
  x.assign(n_nodes, 0.0);
  y.assign(n_nodes, 0.0);
  for (int b = 0; b < nly; ++b)
    for (int a = 0; a < nlx; ++a)
      for (int j = 0; j < p; ++j)
        for (int k = 0; k < p; ++k) {
          int64_t id = node_id(a, b, k, j);
          if (id < 0) continue;
          // on a periodic square the seams x = x1, y = y1 are the lines x = x0, y = y0
          const bool seam_x = periodic && a == nlx - 1 && k == p - 1;
          const bool seam_y = periodic && b == nly - 1 && j == p - 1;
          x[id] = seam_x ? x0 : x0 + (a + 0.5 * (xi[k] + 1.0)) * hx;
          y[id] = seam_y ? y0 : y0 + (b + 0.5 * (xi[j] + 1.0)) * hy;
        }
}

// Boundary segments of a box [a0, a0+sx) x [b0, b0+sy) in S, E, N, W order.
static void box_segments(const Grid& g, int a0, int b0, int sx, int sy, int* out) {
  int t = 0;
  for (int a = a0; a < a0 + sx; ++a) out[t++] = (int)g.hseg(b0, a);          // S
  for (int b = b0; b < b0 + sy; ++b) out[t++] = (int)g.vseg(b, a0 + sx);     // E
  for (int a = a0; a < a0 + sx; ++a) out[t++] = (int)g.hseg(b0 + sy, a);     // N
  for (int b = b0; b < b0 + sy; ++b) out[t++] = (int)g.vseg(b, a0);          // W
}

void make_plan(const Grid& g, Plan& plan) {
  const int q = g.q;
  plan.lv.clear();
  Level l0;
  l0.sx = l0.sy = 1;
  l0.nbx = g.nlx; l0.nby = g.nly; l0.nbox = g.nlx * g.nly;
  l0.nseg = 4; l0.nbd = 4 * q;
  l0.bseg.resize((size_t)l0.nbox * 4);
  for (int b = 0; b < g.nly; ++b)
    for (int a = 0; a < g.nlx; ++a) box_segments(g, a, b, 1, 1, &l0.bseg[(size_t)(b * g.nlx + a) * 4]);
  plan.lv.push_back(l0);
  int next_dir = 0;
  while (plan.lv.back().nbox > 1) {
    const Level& c = plan.lv.back();
    int dir = next_dir;
    if (dir == 0 && c.nbx == 1) dir = 1;
    if (dir == 1 && c.nby == 1) dir = 0;
    next_dir = 1 - dir;
    Level l;
    l.dir = dir;
    l.sx = dir == 0 ? 2 * c.sx : c.sx;
    l.sy = dir == 1 ? 2 * c.sy : c.sy;
    l.nbx = g.nlx / l.sx; l.nby = g.nly / l.sy; l.nbox = l.nbx * l.nby;
    l.nseg = 2 * (l.sx + l.sy); l.nbd = l.nseg * q;
    const int sx = c.sx, sy = c.sy;     // child size
    // child boundary offsets: S [0, sx q), E [sx q, (sx+sy) q), N, W
    const int oS = 0, oE = sx * q, oN = (sx + sy) * q, oW = (2 * sx + sy) * q;
    auto push = [&](int child, int off, int len) {
      for (int t = 0; t < len; ++t) { l.par_child.push_back(child); l.par_idx.push_back(off + t); }
    };
    if (dir == 0) {   // alpha west, beta east; interface alpha.E = beta.W
      l.n3 = sy * q;
      for (int t = 0; t < l.n3; ++t) { l.a3.push_back(oE + t); l.b3.push_back(oW + t); }
      push(0, oS, sx * q); push(1, oS, sx * q);    // S
      push(1, oE, sy * q);                         // E
      push(0, oN, sx * q); push(1, oN, sx * q);    // N
      push(0, oW, sy * q);                         // W
    } else {          // alpha south, beta north; interface alpha.N = beta.S
      l.n3 = sx * q;
      for (int t = 0; t < l.n3; ++t) { l.a3.push_back(oN + t); l.b3.push_back(oS + t); }
      push(0, oS, sx * q);                         // S
      push(0, oE, sy * q); push(1, oE, sy * q);    // E
      push(1, oN, sx * q);                         // N
      push(0, oW, sy * q); push(1, oW, sy * q);    // W
    }
    l.bseg.resize((size_t)l.nbox * l.nseg);
    const int n3s = l.n3 / q;
    l.iseg.resize((size_t)l.nbox * n3s);
    for (int by = 0; by < l.nby; ++by)
      for (int bx = 0; bx < l.nbx; ++bx) {
        const int box = by * l.nbx + bx, a0 = bx * l.sx, b0 = by * l.sy;
        box_segments(g, a0, b0, l.sx, l.sy, &l.bseg[(size_t)box * l.nseg]);
        for (int t = 0; t < n3s; ++t)
          l.iseg[(size_t)box * n3s + t] =
              dir == 0 ? (int)g.vseg(b0 + t, a0 + sx) : (int)g.hseg(b0 + sy, a0 + t);
      }
    plan.lv.push_back(std::move(l));
  }
}

}  // namespace eo
