"""GPU parity of the fast-diagonalisation leaf path (shared constant-coefficient
operators): the leaf solves through the separable eigenbasis against the FP64
oracle, against the dense leaf operators of the same build, across leaf shapes
(square and rectangular leaves, several p), several right-hand sides with a
ragged last column block, and single resolvents."""
import numpy as np
import pytest

import workloads as W
from oracle import sem
from oracle.resolvent import Problem, Stepper

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.fixture(scope="module")
def eo():
    import paper_1402_5168_gb300 as m
    return m


def case(eo, nlx, nly, p, dense=False, n_poles=21, band=60.0, f=10.0, max_rhs=1, seed=1000):
    g = eo.Grid(nlx, nly, p)
    x, y = g.nodes()
    op = eo.Operator(g, eo.SW_WALLS, band=band, n_poles=n_poles, f=f, g=1.0, H=1.0, shared_ops=True,
                     dense_leaves=dense, max_rhs=max_rhs)
    c, s, a = W.draw_gaussians(seed, 3, (0.1, 0.15), (0.1, 1.0), (0.3, 0.7))
    h = W.gaussian_sum(x, y, c, s, a)
    u0 = np.stack([0.3 * np.sin(np.pi * y) * x * (1 - x), -0.2 * np.sin(np.pi * x) * y * (1 - y), h])
    return g, op, u0


@pytest.mark.parametrize("nlx,nly,p", [(1, 1, 6), (2, 4, 10), (4, 4, 16), (8, 8, 12), (4, 2, 5)])
def test_fd_single_step_matches_oracle(eo, nlx, nly, p):
    g, op, u0 = case(eo, nlx, nly, p)
    prob = Problem(sem.Grid(nlx, nly, p), "sw", op.tau, f=10.0, g=1.0, H=1.0)
    want = Stepper(prob, op.alpha, op.b).step(u0)
    u = torch.tensor(u0, device="cuda")
    op.apply(u, 1)
    e = rel(u.cpu().numpy(), want)
    print(f"fd leaves {nlx}x{nly} p{p}: one-step rel L2 vs oracle {e:.3e}")
    assert e <= 1e-10


@pytest.mark.parametrize("nlx,nly,p", [(4, 4, 10), (2, 8, 16)])
def test_fd_equals_dense_leaf_operators(eo, nlx, nly, p):
    g, op_fd, u0 = case(eo, nlx, nly, p)
    _, op_dn, _ = case(eo, nlx, nly, p, dense=True)
    a = torch.tensor(u0, device="cuda")
    b = torch.tensor(u0, device="cuda")
    op_fd.apply(a, 3)
    op_dn.apply(b, 3)
    e = rel(a.cpu().numpy(), b.cpu().numpy())
    print(f"fd vs dense leaves {nlx}x{nly} p{p}, three steps: {e:.3e}")
    assert e <= 1e-12


def test_fd_many_poles_chunked(eo):
    """Enough poles that both leaf kernels split the poles into several chunks."""
    g, op_fd, u0 = case(eo, 4, 4, 8, n_poles=301, band=60.0)
    _, op_dn, _ = case(eo, 4, 4, 8, dense=True, n_poles=301, band=60.0)
    a = torch.tensor(u0, device="cuda")
    b = torch.tensor(u0, device="cuda")
    op_fd.apply(a, 1)
    op_dn.apply(b, 1)
    e = rel(a.cpu().numpy(), b.cpu().numpy())
    print(f"fd vs dense, 301 poles: {e:.3e}")
    assert e <= 1e-11


def test_fd_multi_rhs_ragged(eo):
    """3 right-hand sides on 2x2 leaves: 12 columns, not a multiple of the
    columns per block; each column must equal its single-rhs run."""
    g, op, u0 = case(eo, 2, 2, 12, max_rhs=3)
    rng = np.random.default_rng(5)
    U = np.stack([u0, rng.standard_normal(u0.shape), 0.5 * u0 + 0.1 * rng.standard_normal(u0.shape)])
    a = torch.tensor(U, device="cuda")
    op.apply(a, 2)
    for r in range(3):
        b = torch.tensor(U[r:r + 1].copy(), device="cuda")
        op.apply(b, 2)
        assert rel(a[r].cpu().numpy(), b[0].cpu().numpy()) < 1e-13


def test_fd_resolvents_match_oracle(eo):
    g, op, u0 = case(eo, 4, 4, 10)
    prob = Problem(sem.Grid(4, 4, 10), "sw", op.tau, f=10.0, g=1.0, H=1.0)
    st = Stepper(prob, op.alpha, op.b)
    u = torch.tensor(u0, device="cuda")
    M = (op.alpha.size - 1) // 2
    for j in (M, M + 3, 2 * M):
        xg = torch.zeros((3, g.n_nodes), dtype=torch.complex128, device="cuda")
        op.resolvent(j, u, xg)
        e = rel(xg.cpu().numpy(), st.resolvent(j, u0))
        print(f"fd resolvent j={j}: {e:.3e}")
        assert e <= 1e-10


@pytest.mark.parametrize("nlx,nly,p", [(4, 4, 10), (2, 4, 16)])
def test_fd_pair_arithmetic_matches_oracle(eo, nlx, nly, p):
    """FP32-pair leaf arithmetic (precision df32): FP64-class agreement with the
    oracle after one step and with the FP64 leaf path after four."""
    g = eo.Grid(nlx, nly, p)
    x, y = g.nodes()
    kw = dict(band=60.0, n_poles=21, f=10.0, g=1.0, H=1.0, shared_ops=True)
    op_pair = eo.Operator(g, eo.SW_WALLS, precision="df32", **kw)
    op_64 = eo.Operator(g, eo.SW_WALLS, precision="fp64", **kw)
    _, _, u0 = case(eo, nlx, nly, p)
    prob = Problem(sem.Grid(nlx, nly, p), "sw", op_64.tau, f=10.0, g=1.0, H=1.0)
    want = Stepper(prob, op_64.alpha, op_64.b).step(u0)
    a = torch.tensor(u0, device="cuda")
    op_pair.apply(a, 1)
    e1 = rel(a.cpu().numpy(), want)
    a = torch.tensor(u0, device="cuda")
    b = torch.tensor(u0, device="cuda")
    op_pair.apply(a, 4)
    op_64.apply(b, 4)
    e4 = rel(a.cpu().numpy(), b.cpu().numpy())
    print(f"fd pair leaves {nlx}x{nly} p{p}: one step vs oracle {e1:.3e}, four steps vs fp64 {e4:.3e}")
    assert e1 <= 1e-10 and e4 <= 1e-10
