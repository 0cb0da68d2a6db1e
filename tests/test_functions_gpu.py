"""Other functions of tau L on the same poles (dense output and phi1): the
residue fits against brute force on the band (oracle's R_eval), the shared-sweep
multi-output apply against the oracle's pole sums with the same residues, and
the semigroup property exp(tau L / 2)^2 = exp(tau L) to the approximation error."""
import numpy as np
import pytest

import workloads as W
from oracle import rational, sem
from oracle.resolvent import Problem, Stepper

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _phi(j, th):
    """phi_j(i theta), j = 1, 2: the closed form where it has no cancellation
    (|theta| >= 0.5, rounding below 1e-15) and the Taylor series sum_k z^k / (k + j)!
    (30 terms) inside, so that the reference is accurate well below the band errors."""
    z = 1j * np.asarray(th, dtype=np.float64)
    out = np.zeros(z.shape, dtype=np.complex128)
    small = np.abs(th) < 0.5
    zs = z[small]
    term = np.ones_like(zs)
    fact = float(np.prod(np.arange(1, j + 1)))
    acc = np.zeros_like(zs)
    for k in range(30):
        acc += term / fact
        term = term * zs
        fact *= k + j + 1
    out[small] = acc
    zb = z[~small]
    out[~small] = (np.exp(zb) - 1) / zb if j == 1 else (np.exp(zb) - 1 - zb) / zb ** 2
    return out


def phi1(th):
    return _phi(1, th)


def phi2(th):
    return _phi(2, th)


@pytest.fixture(scope="module")
def wave():
    import paper_1402_5168_gb300 as eo
    w = W.WAVE_4X4_P12
    g = eo.Grid(4, 4, 10)
    x, y = g.nodes()
    c = W.wave_c(w, x, y)
    op = eo.Operator(g, eo.WAVE_DIRICHLET, band=W.BAND[w.name], n_poles=21, c2=c * c)
    prob = Problem(sem.Grid(4, 4, 10), "wave", op.tau, c2=c * c)
    u0 = np.stack(W.initial_fields(w, x, y))
    return eo, g, op, prob, u0


@pytest.mark.parametrize("n_poles", [21, 301])
def test_function_residues_meet_their_band_error(n_poles):
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(2, 2, 8)
    op = eo.Operator(g, eo.SW_WALLS, band=60.0, n_poles=n_poles, f=10.0, g=1.0, H=1.0, shared_ops=True)
    th = np.linspace(-op.X, op.X, 20001)
    for kind, c, f in [("exp", 0.5, lambda t: np.exp(0.5j * t)), ("exp", 0.25, lambda t: np.exp(0.25j * t)),
                       ("exp", 1.0, lambda t: np.exp(1j * t)), ("phi1", 1.0, phi1), ("phi2", 1.0, phi2)]:
        b, err = op.fit_function(kind, c)
        assert np.array_equal(b[::-1], np.conj(b))
        brute = np.abs(f(th) - rational.R_eval(1j * th, op.alpha, b)).max()
        print(f"{n_poles} poles {kind} c={c}: reported {err:.2e}, brute force {brute:.2e}")
        assert brute <= 1.01 * err + 1e-14
        # exp(cz) to the step's own accuracy; phi1 on wide pole sets (trapezoidal
        # centre + fitted ends) reaches ~3e-8
        assert err <= (1e-8 if kind == "exp" or n_poles <= 101 else 1e-7)
        if kind == "phi2":
            # phi2 is not phi1: the residue sets differ on the band
            b1, _ = op.fit_function("phi1", 1.0)
            assert np.abs(rational.R_eval(1j * th, op.alpha, b1) - f(th)).max() > 1e-2


def test_shared_sweep_outputs_match_the_oracle(wave):
    eo, g, op, prob, u0 = wave
    sets = [op.fit_function("exp", 0.5)[0], op.b, op.fit_function("phi1")[0], op.fit_function("phi2")[0]]
    u = torch.tensor(u0, device="cuda")
    out = torch.zeros((4, 2, g.n_nodes), dtype=torch.float64, device="cuda")
    op.apply_functions(sets, u, out)
    got = out.cpu().numpy()
    for k, b in enumerate(sets):
        want = Stepper(prob, op.alpha, b).step(u0)
        e = rel(got[k], want)
        print(f"function {k}: rel L2 vs oracle {e:.3e}")
        assert e <= 1e-10
    # the original residues through this path equal the plain step
    v = torch.tensor(u0, device="cuda")
    op.apply(v, 1)
    assert rel(got[1], v.cpu().numpy()) < 1e-12


def test_half_steps_compose_to_a_step(wave):
    eo, g, op, prob, u0 = wave
    bh, err = op.fit_function("exp", 0.5)
    u = torch.tensor(u0, device="cuda")
    out = torch.zeros((1, 2, g.n_nodes), dtype=torch.float64, device="cuda")
    op.apply_functions([bh], u, out)
    mid = out[0].clone()
    op.apply_functions([bh], mid, out)
    v = torch.tensor(u0, device="cuda")
    op.apply(v, 1)
    e = rel(out[0].cpu().numpy(), v.cpu().numpy())
    print(f"exp(tau L/2)^2 vs exp(tau L): {e:.3e} (band errors {err:.1e})")
    assert e <= 1e-7
