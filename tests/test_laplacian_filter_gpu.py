"""The filter S(k0 Delta) of Section 3.3 on the GPU (eo_apply_laplacian_filter through a
shallow-water handle with f = 0; Python LaplacianFilter).

* Parity with the oracle's S(k0 Delta) (oracle/filter.py: shifted-Laplacian solves of
  the global sparse system), on walled and periodic grids, FP64 and FP32 pairs, three
  fields of two right-hand sides (six columns through groups of four and two), with the
  library's own poles and residues: relative L2 <= 1e-10 per field.
* The paper's use of it: the Gaussian-sum approximant with the conjugate-pole shortcut
  grows by about 1.44 per step on the modes at the peak of |R(i y)| (a periodic wave,
  tau chosen to put the top eigenvalue of the discrete operator there); the step
  followed by S(k0 Delta), with k0 chosen so that the window ends below those modes and
  keeps the smooth part of the data, stays bounded (from a random state whose edge values
  follow from its interior ones, as every state the step produces) and leaves a smooth
  state nearly unchanged.
* Handles without the right elliptic operator are refused.
"""
import numpy as np
import pytest

import workloads as W
from oracle import gauss, rational, sem
from oracle.filter import LaplacianFilter as OracleFilter
from oracle.reference import WaveLh
from oracle.resolvent import Problem
from tests.test_oracle_rational import load_table1

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MU, A = load_table1()


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("periodic,precision", [(False, "fp64"), (True, "fp64"), (False, "df32"), (True, "df32")])
def test_filter_matches_the_oracle(periodic, precision):
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(4, 4, 12, periodic=periodic)
    k0 = 0.36
    flt = eo.LaplacianFilter(g, k0, X=30.0, keep=0.9, precision=precision, max_rhs=4)
    x, y = g.nodes()
    rng = np.random.default_rng(17)
    fields = []
    for r in range(2):
        c, s, a = W.draw_gaussians(100 + r, 3, (0.06, 0.12), (0.2, 1.0), (0.2, 0.8))
        base = W.gaussian_sum(x, y, c, s, a)
        fields.append(np.stack([base, np.cos(2 * np.pi * 3 * x) * np.sin(2 * np.pi * y) + 0.1 * base,
                                0.05 * rng.standard_normal(g.n_nodes) + base]))
    U = np.stack(fields)                                   # [2 rhs][3 fields][n]
    u = torch.tensor(U, device="cuda")
    flt.apply(u)
    got = u.cpu().numpy()
    orc = OracleFilter(sem.Grid(4, 4, 12, periodic=periodic), flt.op.tau ** 2, flt.op.alpha, flt.s)
    worst = 0.0
    for r in range(2):
        for f in range(3):
            want = orc.apply(U[r, f])
            e = rel(got[r, f], want)
            worst = max(worst, e)
            assert e <= 1e-10, (r, f, e)
    print(f"S(k0 Delta) periodic={periodic} {precision}: worst field vs oracle {worst:.2e} "
          f"(M = {flt.M}, M0 = {flt.M0}, {flt.op.alpha.size} poles)")


def test_filter_stops_the_growth_of_the_conjugate_pole_step():
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(2, 2, 8, periodic=True)
    og = sem.Grid(2, 2, 8, periodic=True)
    lam = WaveLh(Problem(og, "wave", 1.0, c2=np.ones(og.n_nodes))).eig()[0]
    kmax = np.abs(lam.imag).max()
    X, H = 20.0, 0.18
    alpha, b, M = gauss.gauss_fit(X, H, MU, A)
    yy = np.linspace(0, 2 * np.pi * (M * H + 20), 200001)
    ypk = yy[np.argmax(np.abs(rational.R_eval(1j * yy, alpha, b)))]
    tau = ypk / kmax                                       # the top mode at the peak of |R|
    op = eo.Operator(g, eo.WAVE_DIRICHLET, band=X / tau, tau=tau, c2=np.ones(g.n_nodes), fitter="gauss")
    rho = np.abs(rational.R_eval(1j * tau * lam.imag, op.alpha, op.b)).max()
    assert rho > 1.3
    # window: flat below |k| = 0.5 X / tau (the data), zero above X / tau (where |R| may
    # exceed one); the filter's own window ends at about (M0 + 10) h in sqrt(k0) |k| / 2 pi
    probe = eo.LaplacianFilter(g, 1.0, X=30.0, keep=0.9)
    k_stop = X / tau / (2 * np.pi)
    k0 = ((probe.M0 + 10) * probe.h / k_stop) ** 2
    flt = eo.LaplacianFilter(g, k0, X=30.0, keep=0.9)
    flat = (flt.M0 - 10) * flt.h / np.sqrt(k0)
    # a random state on the discrete problem's own manifold (edge values from the interior
    # ones through the flux rows): there S(k0 Delta) and the step commute; an arbitrary
    # node vector carries edge components the two treat differently, and its filtered
    # trajectory shows a long non-normal transient (6.9x) although the spectral radius of
    # the filtered step is 1 + 1e-11 (oracle, dense matrices)
    rng = np.random.default_rng(7)
    lh = WaveLh(Problem(og, "wave", tau, c2=np.ones(og.n_nodes)))
    u0 = lh.lift(rng.standard_normal(lh.i.size), rng.standard_normal(lh.i.size))
    n0 = np.linalg.norm(u0)
    u = torch.tensor(u0, device="cuda")
    v = torch.tensor(u0, device="cuda")
    nu, nv = [], []
    for _ in range(40):
        op.apply(u, 1)
        nu.append(float(torch.linalg.vector_norm(u)))
        op.apply(v, 1)
        flt.apply(v)
        nv.append(float(torch.linalg.vector_norm(v)))
    print(f"conjugate-pole step: growth {nu[-1] / n0:.2e} over 40 steps (max |R| on the spectrum {rho:.4f}); "
          f"with S(k0 Delta) (k0 = {k0:.3e}, flat to |k|/2pi = {flat:.2f}, zero from {k_stop:.2f}): "
          f"|u_1| / |u_0| = {nv[0] / n0:.3f}, max_k |u_k| / |u_1| = {max(nv) / nv[0]:.3f}")
    assert nu[-1] > 1e4 * n0
    assert max(nv) <= 1.5 * nv[0]
    # a smooth state (content far below the window's edge) passes unchanged, to the
    # collocation error of the grid (4x4 leaves, p = 16: the 2x2, p = 8 grid above
    # resolves these modes only to ~1e-6)
    gf = eo.Grid(4, 4, 16, periodic=True)
    fine = eo.LaplacianFilter(gf, k0, X=30.0, keep=0.9)
    x, y = gf.nodes()
    sm = np.stack([np.cos(2 * np.pi * x) * np.sin(2 * np.pi * y), np.sin(2 * np.pi * (x + y))])
    assert np.hypot(1, 1) < flat
    w = torch.tensor(sm, device="cuda")
    fine.apply(w)
    e = rel(w.cpu().numpy(), sm)
    print(f"smooth state through S(k0 Delta) on 4x4/p16: rel change {e:.2e}")
    assert e <= 1e-8


def test_filter_refuses_other_handles():
    import paper_1402_5168_gb300 as eo
    from paper_1402_5168_gb300 import ExpopError
    g = eo.Grid(2, 2, 8)
    x, y = g.nodes()
    u = torch.zeros((3, g.n_nodes), dtype=torch.float64, device="cuda")
    sw = eo.Operator(g, eo.SW_WALLS, band=60.0, n_poles=21, f=10.0, shared_ops=True)
    with pytest.raises(ExpopError, match="f = 0"):
        sw.apply_laplacian_filter(sw.b, u)
    wave = eo.Operator(g, eo.WAVE_DIRICHLET, band=60.0, n_poles=21, c2=np.ones_like(x))
    with pytest.raises(ExpopError, match="f = 0"):
        wave.apply_laplacian_filter(wave.b, u[:2].contiguous())
