"""Adjoint of the step (eo_apply_adjoint): against the oracle's factor-by-factor
transpose (itself pinned to the transpose of the dense step matrix), the
dot-product identity <y, G u> = <G^T y, u> through the GPU forward and adjoint,
and central finite differences of a quadratic sensor misfit over several steps."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import sem
from oracle.resolvent import Problem, Stepper, adjoint_step

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def make(eo, shape, precision="fp64"):
    w = W.WAVE_4X4_P12
    nlx, nly, p = shape
    g = eo.Grid(nlx, nly, p)
    x, y = g.nodes()
    c = W.wave_c(w, x, y)
    op = eo.Operator(g, eo.WAVE_DIRICHLET, band=250.0, n_poles=21, c2=c * c, precision=precision)
    prob = Problem(sem.Grid(nlx, nly, p), "wave", op.tau, c2=c * c)
    return g, op, Stepper(prob, op.alpha, op.b)


@pytest.mark.parametrize("shape", [(4, 4, 12), (2, 4, 9), (1, 1, 8)])
def test_adjoint_matches_oracle(shape):
    import paper_1402_5168_gb300 as eo
    g, op, st = make(eo, shape)
    rng = np.random.default_rng(11)
    y = rng.standard_normal((2, g.n_nodes))
    want = adjoint_step(st, y)
    t = torch.tensor(y, device="cuda")
    op.apply_adjoint(t, 1)
    e = rel(t.cpu().numpy(), want)
    # rounding floor: the oracle against itself with another sparse-LU ordering
    st2 = Stepper(st.prob, op.alpha, op.b)
    st2._lu = {i: spla.splu(st.prob.system(op.alpha[i]), permc_spec="MMD_AT_PLUS_A")
               for i in range(op.alpha.size)}
    floor = rel(adjoint_step(st2, y), want)
    print(f"adjoint {shape}: rel L2 vs oracle {e:.3e} (oracle rounding floor {floor:.3e})")
    assert e <= max(1e-10, 2 * floor)


def test_dot_product_identity_gpu():
    import paper_1402_5168_gb300 as eo
    g, op, st = make(eo, (4, 4, 12))
    rng = np.random.default_rng(12)
    u = rng.standard_normal((2, g.n_nodes))
    y = rng.standard_normal((2, g.n_nodes))
    gu = torch.tensor(u, device="cuda")
    op.apply(gu, 3)
    gy = torch.tensor(y, device="cuda")
    op.apply_adjoint(gy, 3)
    lhs = float(np.sum(y * gu.cpu().numpy()))
    rhs = float(np.sum(gy.cpu().numpy() * u))
    print(f"<y, G^3 u> = {lhs:.15e}, <G^T^3 y, u> = {rhs:.15e}")
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + np.linalg.norm(y) * np.linalg.norm(u))


def test_gradient_matches_central_differences():
    # loss = 1/2 sum_n |S u_n - d_n|^2 over n = 1..N steps, S = sampling at seeded
    # interior sensors; gradient by the adjoint recursion, checked in random directions
    import paper_1402_5168_gb300 as eo
    g, op, st = make(eo, (4, 4, 12))
    rng = np.random.default_rng(13)
    N = 4
    sensors = rng.choice(g.n_interior, 64, replace=False)
    x, y = g.nodes()
    u0 = np.stack(W.initial_fields(W.WAVE_4X4_P12, x, y))
    d = [rng.standard_normal(64) * 0.01 for _ in range(N)]

    def loss(u):
        t = torch.tensor(u, device="cuda")
        val = 0.0
        for n in range(N):
            op.apply(t, 1)
            val += 0.5 * np.sum((t.cpu().numpy()[0][sensors] - d[n]) ** 2)
        return val

    # forward trajectory, then lambda_N = r_N, lambda_n = G^T lambda_{n+1} + r_n
    t = torch.tensor(u0, device="cuda")
    res = []
    for n in range(N):
        op.apply(t, 1)
        r = np.zeros((2, g.n_nodes))
        r[0][sensors] = t.cpu().numpy()[0][sensors] - d[n]
        res.append(r)
    lam = torch.tensor(res[N - 1], device="cuda")
    for n in range(N - 2, -1, -1):
        op.apply_adjoint(lam, 1)
        lam += torch.tensor(res[n], device="cuda")
    op.apply_adjoint(lam, 1)
    grad = lam.cpu().numpy()
    for k in range(5):
        dirn = rng.standard_normal(u0.shape)
        eps = 1e-3 * np.linalg.norm(u0) / np.linalg.norm(dirn)
        fd = (loss(u0 + eps * dirn) - loss(u0 - eps * dirn)) / (2 * eps)
        an = float(np.sum(grad * dirn))
        print(f"direction {k}: FD {fd:.12e} adjoint {an:.12e}")
        assert abs(fd - an) <= 1e-6 * abs(an) + 1e-12


def test_forward_unchanged_by_adjoint_calls():
    import paper_1402_5168_gb300 as eo
    g, op, st = make(eo, (4, 4, 10))
    rng = np.random.default_rng(14)
    u = rng.standard_normal((2, g.n_nodes))
    a = torch.tensor(u, device="cuda")
    op.apply(a, 1)
    y = torch.tensor(rng.standard_normal((2, g.n_nodes)), device="cuda")
    op.apply_adjoint(y, 2)
    b = torch.tensor(u, device="cuda")
    op.apply(b, 1)
    assert torch.equal(a, b)


def sw_op(eo, nl, p, shared, precision="fp64"):
    g = eo.Grid(nl, nl, p)
    op = eo.Operator(g, eo.SW_WALLS, band=60.0, n_poles=21, f=10.0, g=1.0, H=1.0, shared_ops=shared,
                     precision=precision)
    return g, op


def test_sw_adjoint_matches_dense_oracle_transpose():
    # 2x2 leaves, p = 6: the oracle's dense step matrix G (column by column), G^T y
    import paper_1402_5168_gb300 as eo
    from oracle.resolvent import step_matrix
    g, op = sw_op(eo, 2, 6, False)
    st = Stepper(Problem(sem.Grid(2, 2, 6), "sw", op.tau, f=10.0, g=1.0, H=1.0), op.alpha, op.b)
    G = step_matrix(st)
    rng = np.random.default_rng(31)
    y = rng.standard_normal((3, g.n_nodes))
    t = torch.tensor(y, device="cuda")
    op.apply_adjoint(t, 1)
    e = rel(t.cpu().numpy().ravel(), G.T @ y.ravel())
    print(f"sw adjoint vs dense oracle transpose: {e:.3e}")
    assert e <= 1e-10


@pytest.mark.parametrize("nl,p,shared,precision", [(4, 8, True, "fp64"), (4, 8, False, "fp64"),
                                                   (2, 10, True, "df32")])
def test_sw_dot_product_identity(nl, p, shared, precision):
    import paper_1402_5168_gb300 as eo
    g, op = sw_op(eo, nl, p, shared, precision)
    rng = np.random.default_rng(32)
    u = rng.standard_normal((3, g.n_nodes))
    y = rng.standard_normal((3, g.n_nodes))
    gu = torch.tensor(u, device="cuda")
    op.apply(gu, 2)
    gy = torch.tensor(y, device="cuda")
    op.apply_adjoint(gy, 2)
    lhs = float(np.sum(y * gu.cpu().numpy()))
    rhs = float(np.sum(gy.cpu().numpy() * u))
    print(f"sw {nl}x{nl}/p{p} shared={shared} {precision}: <y,G^2u> {lhs:.15e} <G^T^2y,u> {rhs:.15e}")
    assert abs(lhs - rhs) <= 1e-11 * (abs(lhs) + np.linalg.norm(y) * np.linalg.norm(u))
