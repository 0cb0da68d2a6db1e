// Internal structures of the expop engine (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <complex>
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/expop.h"

namespace eo {

// Thread-local error message and a helper that records it.
void set_error(const std::string& msg);
eo_status fail(eo_status st, const std::string& msg);

// ---------------------------------------------------------------- leaf grid
struct Grid {
  int nlx = 0, nly = 0, p = 0, q = 0;
  double x0 = 0, x1 = 1, y0 = 0, y1 = 1, hx = 0, hy = 0;
  int64_t n_int = 0, n_hseg = 0, n_vseg = 0, n_seg = 0, n_edge = 0, n_nodes = 0;
  // periodic square (the setting of the paper's examples): the lines y = y1 and
  // x = x1 are the lines y = y0 and x = x0, so there are nhl = nly horizontal and
  // nvl = nlx vertical edge lines (walled square: nly + 1 and nlx + 1)
  int periodic = 0;
  int nhl = 0, nvl = 0;
  std::vector<double> xi;        // Chebyshev-Lobatto points on [-1, 1], ascending
  std::vector<double> D;         // p x p differentiation matrix on [-1,1], row-major D[i*p+j]
  std::vector<double> Ed;        // q x q differentiation matrix through the q inner points

  // global node id of local node (k, j) of leaf (a, b); -1 at a corner
  int64_t node_id(int a, int b, int k, int j) const;
  int64_t hseg(int e, int a) const { return (int64_t)(e % nhl) * nlx + a; }
  int64_t vseg(int b, int e) const { return n_hseg + (int64_t)b * nvl + (e % nvl); }
  void coords(std::vector<double>& x, std::vector<double>& y) const;
};

eo_status make_grid(int nlx, int nly, int p, double x0, double x1, double y0, double y1,
                    Grid& g, int periodic = 0);

// ---------------------------------------------------------------- tree plan
// Level 0: leaves.  Level l >= 1: boxes made by merging pairs of level-(l-1)
// boxes, alternating x and y merges.  Box boundary order: sides S, E, N, W,
// each a list of leaf-edge segments in ascending coordinate, q nodes per
// segment in ascending coordinate.
struct Level {
  int sx = 1, sy = 1;          // box size in leaves
  int nbx = 0, nby = 0, nbox = 0;
  int nseg = 0, nbd = 0;       // boundary segments / nodes per box
  int dir = -1;                // merge that made this level: 0 = x, 1 = y
  int n3 = 0;                  // interface nodes of that merge
  std::vector<int> par_child;  // [nbd] child (0 = alpha, 1 = beta) of each boundary node
  std::vector<int> par_idx;    // [nbd] index of the node in that child's boundary
  std::vector<int> a3, b3;     // [n3] interface node indices in alpha's / beta's boundary
  std::vector<int> bseg;       // [nbox * nseg] global segment ids of each box boundary
  std::vector<int> iseg;       // [nbox * n3/q] global segment ids of each interface
};

struct Plan {
  std::vector<Level> lv;       // lv[0] = leaves, lv.back() = root
  int L() const { return (int)lv.size() - 1; }
};

void make_plan(const Grid& g, Plan& plan);

// ---------------------------------------------------------------- fitter
// Poles and residues, as consecutive conjugate-closed vertical lines, each of
// odd length 2K+1 in order of increasing imaginary part (index K of a line is
// its real pole).  The line fit has one line (m = -M..M); the Gaussian-sum
// construction of Sections 3.1-3.2 has two (the right line, then its mirror).
struct Fit {
  std::vector<double> are, aim, bre, bim;
  std::vector<int> lines;                   // line lengths (empty: one line of N)
  double X = 0, sigma = 0, s = 0;
  int E = 0;                                // wide fits: outer pairs fitted by least squares (0: all)
  double gh = 0;                            // Gaussian-sum fit: spacing h (0: line fit)
  int gM = 0, gL = 0;                       // Gaussian-sum fit: M Gaussians per side, L of Table 1
  int N() const { return (int)are.size(); }
};

// Indices (into the fit's order) of the distinct poles of the conjugate-pole form
// (Section 3.3): per line its real pole, then the poles with Im > 0.
void distinct_poles(const Fit& f, std::vector<int>& idx);

// Residues on the poles of f for exp(c z) (kind 0), phi1(z) (kind 1) or, on a
// Gaussian-sum fit, the rational partition of unity keeping a fraction c of the
// Gaussians (kind 2); err = max |f(ix) - R(ix)| on [-X, X].
eo_status fit_function(const Fit& f, int kind, double c, std::vector<std::complex<double>>& b, double& err);

// The paper's approximant (Sections 3.1-3.2): e^{i theta} = e^{2 pi i x} as a
// sum of 2M+1 shifted Gaussians psi_h, each replaced by the Table 1 rational;
// M is the smallest meeting delta on [-X, X].  Two lines of 2(M+L)+1 poles.
eo_status fit_gauss(double X, double h, double delta, Fit& out);

// Widest band X for a given odd pole count; returns EO_ERR_FIT if none.
eo_status fit_for_poles(int n_poles, double delta, Fit& out);
// Smallest pole count covering band X (n_poles <= nmax).
eo_status fit_for_band(double X, double delta, int nmax, Fit& out);

// ---------------------------------------------------------------- leaf eigenbasis
// Real eigen-decomposition M = V diag(lam) Vinv (row-major n x n) of a matrix
// with real, distinct eigenvalues; EO_ERR_UNSUPPORTED otherwise.
eo_status real_eigen(int n, const std::vector<double>& M, std::vector<double>& lam, std::vector<double>& V,
                     std::vector<double>& Vinv);

}  // namespace eo
