"""torch.autograd wrappers (forward and adjoint steps of the library): the
gradient of G^n u0 and of a per-step sensor misfit with checkpointed
recomputation, against central finite differences (the losses are quadratic
in u0, so central differences are exact up to rounding) and across checkpoint
intervals."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def make_op(eo, kind="sw"):
    g = eo.Grid(2, 2, 10)
    if kind == "sw":
        op = eo.Operator(g, eo.SW_WALLS, band=60.0, n_poles=21, f=10.0, g=1.0, H=1.0, shared_ops=True)
    else:
        x, y = g.nodes()
        op = eo.Operator(g, eo.WAVE_DIRICHLET, band=120.0, n_poles=21, c2=1.0 + 0.2 * np.sin(3 * x) * y)
    return g, op


@pytest.mark.parametrize("kind", ["sw", "wave"])
def test_evolve_gradient_matches_central_differences(kind):
    import paper_1402_5168_gb300 as eo
    from paper_1402_5168_gb300.autograd import evolve
    g, op = make_op(eo, kind)
    F = op.fields
    rng = np.random.default_rng(30)
    u0 = torch.tensor(rng.standard_normal((F, g.n_nodes)), device="cuda", requires_grad=True)
    w = torch.tensor(rng.standard_normal((F, g.n_nodes)), device="cuda")
    loss = (evolve(op, u0, 3) * w).sum() ** 2
    loss.backward()
    for k in range(3):
        v = torch.tensor(rng.standard_normal((F, g.n_nodes)), device="cuda")
        eps = 1e-3
        with torch.no_grad():
            lp = (evolve(op, u0 + eps * v, 3) * w).sum() ** 2
            lm = (evolve(op, u0 - eps * v, 3) * w).sum() ** 2
        fd = float((lp - lm) / (2 * eps))
        an = float((u0.grad * v).sum())
        assert abs(fd - an) <= 1e-8 * abs(an) + 1e-10


def test_sensor_misfit_checkpointed_gradient():
    import paper_1402_5168_gb300 as eo
    from paper_1402_5168_gb300.autograd import sensor_misfit
    g, op = make_op(eo, "sw")
    rng = np.random.default_rng(31)
    n, ns = 7, 40
    idx = torch.tensor(rng.choice(g.n_nodes, ns, replace=False), device="cuda")
    data = torch.tensor(rng.standard_normal((n, ns)) * 0.1, device="cuda")
    u_np = rng.standard_normal((3, g.n_nodes))
    grads = []
    for every in (1, 3, 10):
        u0 = torch.tensor(u_np, device="cuda", requires_grad=True)
        loss = sensor_misfit(op, u0, n, 2, idx, data, checkpoint_every=every)
        loss.backward()
        grads.append(u0.grad.clone())
    for gk in grads[1:]:
        assert float(torch.linalg.vector_norm(gk - grads[0]) / torch.linalg.vector_norm(grads[0])) < 1e-12
    u0 = torch.tensor(u_np, device="cuda")
    for k in range(3):
        v = torch.tensor(rng.standard_normal((3, g.n_nodes)), device="cuda")
        eps = 1e-3
        lp = sensor_misfit(op, u0 + eps * v, n, 2, idx, data)
        lm = sensor_misfit(op, u0 - eps * v, n, 2, idx, data)
        fd = float((lp - lm) / (2 * eps))
        an = float((grads[0] * v).sum())
        print(f"sensor misfit direction {k}: FD {fd:.12e} adjoint {an:.12e}")
        assert abs(fd - an) <= 1e-7 * abs(an) + 1e-10
