"""GPU parity: the CUDA apply path (through the C ABI) against the FP64 oracle on
the same seeded inputs and the same poles (eo_get_poles), element by element.

Tolerances: one step from identical inputs must agree to relative L2 <= 1e-10
(the FP64 target).  Multi-step trajectories are compared too; both sides round
differently and the pole sum cancels terms larger than its result, so their
tolerance is wider and stated per test."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import rational, sem
from oracle.resolvent import Problem, Stepper

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def eo():
    import paper_1402_5168_gb300 as m
    return m


def wave_case(eo, w, nlx=None, nly=None, p=None, band=None, n_poles=None):
    nlx = nlx or w.nlx
    nly = nly or w.nly
    p = p or w.p
    g = eo.Grid(nlx, nly, p)
    x, y = g.nodes()
    c = W.wave_c(w, x, y)
    op = eo.Operator(g, eo.WAVE_DIRICHLET, band=band or W.BAND[w.name], n_poles=n_poles or w.n_poles,
                     c2=c * c)
    og = sem.Grid(nlx, nly, p)
    prob = Problem(og, "wave", op.tau, c2=c * c)
    u0 = np.stack(W.initial_fields(w, x, y))
    return g, op, prob, u0


def test_library_poles_meet_the_contract(eo):
    w = W.WAVE_4X4_P12
    g, op, prob, u0 = wave_case(eo, w)
    band, mod, tail = rational.check_contract(op.alpha, op.b, op.X, 1e-10)
    assert band <= 1e-10 and mod <= 1.0 + 1e-12 and tail < 1.0
    assert op.alpha.size == 21
    assert np.array_equal(op.alpha[::-1], np.conj(op.alpha))
    assert np.array_equal(op.b[::-1], np.conj(op.b))


@pytest.mark.parametrize("shape", [(4, 4, 12), (2, 8, 9), (8, 4, 6), (1, 1, 10)])
def test_wave_single_step_parity(eo, shape):
    w = W.WAVE_4X4_P12
    nlx, nly, p = shape
    g, op, prob, u0 = wave_case(eo, w, nlx, nly, p)
    st = Stepper(prob, op.alpha, op.b)
    want = st.step(u0)
    u = torch.tensor(u0, device="cuda")
    op.apply(u, 1)
    got = u.cpu().numpy()
    e = rel(got, want)
    # rounding floor of the problem itself: the oracle against itself with a
    # different sparse-LU column ordering (same system, different rounding)
    st2 = Stepper(prob, op.alpha, op.b)
    st2._lu = {i: spla.splu(prob.system(op.alpha[i]), permc_spec="MMD_AT_PLUS_A")
               for i in range(op.alpha.size)}
    floor = rel(st2.step(u0), want)
    print(f"wave {shape} one-step rel L2 {e:.3e} (oracle rounding floor {floor:.3e})")
    assert e <= max(1e-10, 2 * floor)


def test_wave_config0_trajectory(eo):
    # 4x4 leaves, p = 12, 21 poles, Gaussian bump: ten steps, compared at every step
    w = W.WAVE_4X4_P12
    g, op, prob, u0 = wave_case(eo, w)
    st = Stepper(prob, op.alpha, op.b)
    u = torch.tensor(u0, device="cuda")
    s = u0.copy()
    worst_step, worst_traj = 0.0, 0.0
    for k in range(w.steps):
        # single-step parity from the oracle's own state
        ug = torch.tensor(s, device="cuda")
        op.apply(ug, 1)
        s_next = st.step(s)
        worst_step = max(worst_step, rel(ug.cpu().numpy(), s_next))
        op.apply(u, 1)
        worst_traj = max(worst_traj, rel(u.cpu().numpy(), s_next))
        s = s_next
    print(f"config0: worst one-step {worst_step:.3e}, worst trajectory {worst_traj:.3e}")
    assert worst_step <= 1e-10
    assert worst_traj <= 1e-8


def test_multi_step_call_equals_repeated_calls(eo):
    w = W.WAVE_4X4_P12
    g, op, prob, u0 = wave_case(eo, w)
    a = torch.tensor(u0, device="cuda")
    b = torch.tensor(u0, device="cuda")
    op.apply(a, 3)
    for _ in range(3):
        op.apply(b, 1)
    assert torch.equal(a, b)


def test_host_entry_point_matches_device(eo):
    w = W.WAVE_4X4_P12
    g, op, prob, u0 = wave_case(eo, w)
    a = torch.tensor(u0, device="cuda")
    op.apply(a, 2)
    h = u0.copy()
    op.apply_host(h, 2)
    assert np.array_equal(h, a.cpu().numpy())


def test_wave_resolvent_parity(eo):
    w = W.WAVE_4X4_P12
    g, op, prob, u0 = wave_case(eo, w)
    st = Stepper(prob, op.alpha, op.b)
    M = (op.alpha.size - 1) // 2
    u = torch.tensor(u0, device="cuda")
    for j in (M, M + 3, 2 * M):
        x = torch.zeros((2, g.n_nodes), dtype=torch.complex128, device="cuda")
        op.resolvent(j, u, x)
        want = st.resolvent(j, u0)
        e = rel(x.cpu().numpy(), want)
        print(f"resolvent j={j} rel {e:.3e}")
        assert e <= 1e-10


def sw_case(eo, nl, p, shared, f=10.0, n_poles=21, band=60.0, seed=1000):
    g = eo.Grid(nl, nl, p)
    x, y = g.nodes()
    op = eo.Operator(g, eo.SW_WALLS, band=band, n_poles=n_poles, f=f, g=1.0, H=1.0, shared_ops=shared)
    og = sem.Grid(nl, nl, p)
    prob = Problem(og, "sw", op.tau, f=f, g=1.0, H=1.0)
    c, s, a = W.draw_gaussians(seed, 3, (0.1, 0.15), (0.1, 1.0), (0.3, 0.7))
    h = W.gaussian_sum(x, y, c, s, a)
    u0 = np.stack([0.3 * np.sin(np.pi * y) * x * (1 - x), -0.2 * np.sin(np.pi * x) * y * (1 - y), h])
    return g, op, prob, u0


@pytest.mark.parametrize("nl,p,shared", [(2, 10, False), (4, 8, True), (4, 8, False), (1, 9, False)])
def test_sw_single_step_parity(eo, nl, p, shared):
    g, op, prob, u0 = sw_case(eo, nl, p, shared)
    want = Stepper(prob, op.alpha, op.b).step(u0)
    u = torch.tensor(u0, device="cuda")
    op.apply(u, 1)
    e = rel(u.cpu().numpy(), want)
    print(f"sw {nl}x{nl} p{p} shared={shared} one-step rel L2 {e:.3e}")
    assert e <= 1e-10


def test_sw_shared_equals_per_box(eo):
    g, op1, prob, u0 = sw_case(eo, 4, 8, True)
    g2, op2, _, _ = sw_case(eo, 4, 8, False)
    a = torch.tensor(u0, device="cuda")
    b = torch.tensor(u0, device="cuda")
    op1.apply(a, 2)
    op2.apply(b, 2)
    assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-12


def test_multi_rhs_equals_single(eo):
    w = W.WAVE_4X4_P12
    g = eo.Grid(4, 4, 8)
    x, y = g.nodes()
    c = W.wave_c(w, x, y)
    op = eo.Operator(g, eo.WAVE_DIRICHLET, band=200.0, n_poles=21, c2=c * c, max_rhs=4)
    rng = np.random.default_rng(3)
    U = rng.standard_normal((4, 2, g.n_nodes))
    a = torch.tensor(U, device="cuda")
    op.apply(a, 2)
    for r in range(4):
        b = torch.tensor(U[r:r + 1].copy(), device="cuda")
        op.apply(b, 2)
        assert rel(a[r].cpu().numpy(), b[0].cpu().numpy()) < 1e-13


@pytest.mark.parametrize("n_steps", [2, 3, 5])
def test_graph_replay_matches_plain_steps(eo, n_steps):
    """Repeated steps replayed from a recorded CUDA graph give bit-identical
    states to the same steps launched one by one, on the default stream, for
    even and odd step counts and after the state buffer changes."""
    w = W.WAVE_4X4_P12
    g, _, prob, u0 = wave_case(eo, w)
    x, y = g.nodes()
    c = W.wave_c(w, x, y)
    # fixed launch shapes on both handles (autotuned shapes may differ between
    # handles and change the rounding)
    op_g = eo.Operator(g, eo.WAVE_DIRICHLET, band=W.BAND[w.name], n_poles=w.n_poles, c2=c * c,
                       autotune=False)
    op_p = eo.Operator(g, eo.WAVE_DIRICHLET, band=W.BAND[w.name], n_poles=w.n_poles, c2=c * c,
                       use_graphs=False, autotune=False)
    a = torch.tensor(u0, device="cuda")
    b = torch.tensor(u0, device="cuda")
    op_g.apply(a, n_steps)
    op_p.apply(b, n_steps)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    # a second buffer: the recorded graph must not keep writing the first one
    a2 = torch.tensor(u0, device="cuda")
    keep = a.clone()
    op_g.apply(a2, n_steps)
    torch.cuda.synchronize()
    assert torch.equal(a2, b) and torch.equal(a, keep)


def test_autotuned_launch_shapes_give_the_same_step(eo):
    """The autotuner only changes launch shapes (columns per block, k groups):
    the step it produces equals the heuristic shapes' step up to rounding."""
    g, op_t, prob, u0 = sw_case(eo, 4, 10, True)
    _, op_h, _, _ = sw_case(eo, 4, 10, True)
    x, y = g.nodes()
    op_h = eo.Operator(g, eo.SW_WALLS, band=60.0, n_poles=21, f=10.0, g=1.0, H=1.0, shared_ops=True,
                       autotune=False)
    a = torch.tensor(u0, device="cuda")
    b = torch.tensor(u0, device="cuda")
    op_t.apply(a, 2)
    op_h.apply(b, 2)
    assert rel(a.cpu().numpy(), b.cpu().numpy()) < 1e-12
