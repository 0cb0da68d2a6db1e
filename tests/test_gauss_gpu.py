"""The paper's own approximant (Sections 3.1-3.3) on the GPU path: operators
built on the two pole lines of the Gaussian-sum construction, the filter S on
the same poles, and the growth the paper reports for the unfiltered
approximant.  Poles and residues of the expected values come from the oracle's
own construction (``oracle/gauss.py``), checked equal to the library's first."""
import numpy as np
import pytest

import workloads as W
from oracle import gauss, rational, sem
from oracle.reference import WaveLh
from oracle.resolvent import Problem, Stepper
from tests.test_oracle_rational import load_table1

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

MU, A = load_table1()
H = 0.18


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def oracle_poles(X, op):
    alpha, b, M = gauss.gauss_fit(X, H, MU, A)
    assert alpha.size == op.alpha.size
    assert np.abs(op.alpha - alpha).max() <= 1e-14 * np.abs(alpha).max()
    assert np.abs(op.b - b).max() <= 1e-13 * np.abs(b).max()
    return alpha, b, M


def sw_case(eo, precision, dense):
    g = eo.Grid(2, 2, 8)
    x, y = g.nodes()
    X, tau = 24.0, 0.05
    op = eo.Operator(g, eo.SW_WALLS, band=X / tau, tau=tau, f=10.0, g=1.0, H=1.0, shared_ops=True,
                     precision=precision, dense_leaves=dense, fitter="gauss")
    c, s, a = W.draw_gaussians(11, 3, (0.1, 0.15), (0.1, 1.0), (0.3, 0.7))
    h = W.gaussian_sum(x, y, c, s, a)
    u0 = np.stack([0.3 * np.sin(np.pi * y) * x * (1 - x), -0.2 * np.sin(np.pi * x) * y * (1 - y), h])
    prob = Problem(sem.Grid(2, 2, 8), "sw", tau, f=10.0, g=1.0, H=1.0)
    return op, X, u0, prob


@pytest.mark.parametrize("precision,dense", [("fp64", False), ("fp64", True), ("df32", False)])
def test_shallow_water_step_on_the_two_pole_lines(precision, dense):
    import paper_1402_5168_gb300 as eo
    op, X, u0, prob = sw_case(eo, precision, dense)
    alpha, b, _ = oracle_poles(X, op)
    assert (alpha.real < 0).any() and (alpha.real > 0).any()      # both half-planes
    want = Stepper(prob, alpha, b).step(u0)
    u = torch.tensor(u0, device="cuda")
    op.apply(u, 1)
    e = rel(u.cpu().numpy(), want)
    print(f"SW gauss {precision} dense={dense}: rel L2 vs oracle {e:.2e}")
    assert e <= 1e-10


@pytest.fixture(scope="module")
def wave():
    # constant c: the discrete operator's eigenvalues are imaginary; tau puts the top
    # eigenvalue where the unfiltered |R(i y)| peaks (about 1.44, near y = 2 pi M h)
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(2, 2, 8)
    og = sem.Grid(2, 2, 8)
    lam = WaveLh(Problem(og, "wave", 1.0, c2=np.ones(og.n_nodes))).eig()[0]
    X = 20.0
    alpha, b, M = gauss.gauss_fit(X, H, MU, A)
    y = np.linspace(0, 2 * np.pi * (M * H + 20), 200001)
    ypk = y[np.argmax(np.abs(rational.R_eval(1j * y, alpha, b)))]
    tau = ypk / np.abs(lam.imag).max()
    op = eo.Operator(g, eo.WAVE_DIRICHLET, band=X / tau, tau=tau, c2=np.ones(g.n_nodes), fitter="gauss")
    prob = Problem(og, "wave", tau, c2=np.ones(og.n_nodes))
    rng = np.random.default_rng(7)
    u0 = rng.standard_normal((2, g.n_nodes))
    u0[:, prob.cls == 2] = 0.0
    return eo, op, prob, lam, u0, X


def test_wave_step_and_function_residues(wave):
    eo, op, prob, lam, u0, X = wave
    alpha, b, M = oracle_poles(X, op)
    u = torch.tensor(u0, device="cuda")
    op.apply(u, 1)
    e = rel(u.cpu().numpy(), Stepper(prob, alpha, b).step(u0))
    print(f"wave gauss step: rel L2 vs oracle {e:.2e}")
    assert e <= 1e-10
    # exp(c z), phi1, phi2 and the filter on the same poles: the library's residues are the
    # oracle's Gaussian coefficients composed through Table 1
    ae = gauss.even_table(A)
    for kind, c, coef in [("exp", 0.5, gauss.exp_coeffs(M, H, 0.5)), ("phi1", 1.0, gauss.phi1_coeffs(M, H)),
                          ("phi2", 1.0, gauss.phi2_coeffs(M, H)),
                          ("filter", 0.9, gauss.window_coeffs(M, int(np.floor(0.9 * M))))]:
        bl, err = op.fit_function(kind, c)
        bo = gauss.compose(coef, H, MU, ae)[1]
        print(f"{kind}: residue diff {np.abs(bl - bo).max() / np.abs(bo).max():.1e}, band error {err:.1e}")
        assert np.abs(bl - bo).max() <= 1e-12 * np.abs(bo).max()
        assert err <= 1e-10


def test_filtered_step_matches_the_oracle(wave):
    eo, op, prob, lam, u0, X = wave
    alpha, b, M = oracle_poles(X, op)
    bq = gauss.filter_residues(M, int(np.floor(0.9 * M)), H, MU, A)
    want = Stepper(prob, alpha, bq).step(Stepper(prob, alpha, b).step(u0))
    u = torch.tensor(u0, device="cuda")
    op.apply_filtered(u, 1, keep=0.9)
    e = rel(u.cpu().numpy(), want)
    print(f"filtered step: rel L2 vs oracle {e:.2e}")
    assert e <= 1e-10


def test_unfiltered_steps_grow_at_the_predicted_rate_and_the_filter_stops_it(wave):
    # Section 3.3: the Gaussian-sum approximant exceeds one in modulus near |x| = M h,
    # so repeated steps amplify the discrete operator's top modes at the rate
    # rho = max_k |R(i tau lambda_k)| (dense eigenvalues, oracle).  The dominant modes
    # come in conjugate pairs, so the norm oscillates step to step; the rate is taken
    # over 20 steps.  The filtered step S R has spectral radius 1 + O(delta): after the
    # first step (a random state is far from smooth; the eigenvectors' condition
    # number allows a transient) the norm stops growing.
    eo, op, prob, lam, u0, X = wave
    rho = np.abs(rational.R_eval(1j * op.tau * lam.imag, op.alpha, op.b)).max()
    assert rho > 1.3
    u = torch.tensor(u0, device="cuda")
    n0 = np.linalg.norm(u0)
    norms = []
    for _ in range(40):
        op.apply(u, 1)
        norms.append(float(torch.linalg.vector_norm(u)))
    rate = (norms[39] / norms[19]) ** (1 / 20)
    print(f"unfiltered: growth {norms[-1] / n0:.2e} over 40 steps, rate {rate:.4f}, predicted {rho:.4f}")
    assert norms[-1] > 1e4 * n0
    assert abs(rate - rho) <= 0.02 * rho
    v = torch.tensor(u0, device="cuda")
    fn = []
    for _ in range(40):
        op.apply_filtered(v, 1, keep=0.9)
        fn.append(float(torch.linalg.vector_norm(v)))
    print(f"filtered: |u_1| / |u_0| = {fn[0] / n0:.2f}, max_k |u_k| / |u_1| = {max(fn) / fn[0]:.3f}")
    assert max(fn) <= 1.5 * fn[0]
