"""Batches of independent instances (different grids, kinds, pole counts,
right-hand-side counts and precisions) advanced through one CUDA graph: every
instance's state equals, bit for bit, the same steps taken on its own."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def instances(eo):
    rng = np.random.default_rng(40)
    ops, states = [], []
    g1 = eo.Grid(2, 2, 8)
    x, y = g1.nodes()
    ops.append(eo.Operator(g1, eo.WAVE_DIRICHLET, band=100.0, n_poles=21, c2=1.0 + 0.3 * x * y))
    states.append(rng.standard_normal((2, g1.n_nodes)))
    g2 = eo.Grid(4, 4, 10)
    ops.append(eo.Operator(g2, eo.SW_WALLS, band=60.0, n_poles=41, f=10.0, g=1.0, H=1.0, shared_ops=True,
                           precision="df32", max_rhs=3))
    states.append(rng.standard_normal((3, 3, g2.n_nodes)))
    g3 = eo.Grid(4, 2, 12)
    x, y = g3.nodes()
    ops.append(eo.Operator(g3, eo.WAVE_DIRICHLET, band=200.0, n_poles=31, c2=1.0 + 0.1 * np.cos(x), max_rhs=2))
    states.append(rng.standard_normal((2, 2, g3.n_nodes)))
    return ops, states


@pytest.mark.parametrize("n_steps", [2, 5])
def test_batch_equals_separate_instances(n_steps):
    import paper_1402_5168_gb300 as eo
    ops, states = instances(eo)
    a = [torch.tensor(s, device="cuda") for s in states]
    b = [torch.tensor(s, device="cuda") for s in states]
    batch = eo.Batch(ops, a)
    batch.apply(n_steps)
    for op, u in zip(ops, b):
        for _ in range(n_steps):
            op.apply(u, 1)
    torch.cuda.synchronize()
    for x, y in zip(a, b):
        assert torch.equal(x, y)


def test_batch_rejects_a_repeated_handle():
    import paper_1402_5168_gb300 as eo
    ops, states = instances(eo)
    a = [torch.tensor(s, device="cuda") for s in states]
    with pytest.raises(eo.ExpopError):
        eo.Batch([ops[0], ops[0]], [a[0], a[0].clone()])
