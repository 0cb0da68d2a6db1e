"""The adjoint at configuration 4's stated size: rotating shallow water with walls on
32x32 leaves, p = 16, 61 poles; the misfit

    L(u0) = sum_{n=1..50} || h_n[sensors] - d_n ||^2

over 512 seeded sensor nodes, d_n from a second seeded draw stepped by the FP64
handle, its gradient through the checkpointed transposed sweeps (every 10 steps).
L is quadratic in u0, so central differences along a direction v are exact up to
rounding: (L(u0 + e v) - L(u0 - e v)) / 2e = grad . v, with e = 1e-3 ||u0|| and unit
v; 20 seeded directions, in FP64 and in FP32 pairs (each handle against its own
differences), and the FP32-pair gradient against the FP64 one.

The oracle's FP64 gradient, from the transpose of its dense step matrix (the
plainest definition of G^T), on a small grid with the same recipe (2x2 leaves,
p = 10, 61 poles, 50 steps, 64 sensors) against the library's.
"""
import time

import numpy as np
import pytest

import workloads as W
from oracle import sem
from oracle.resolvent import Problem, Stepper, step_matrix

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

CFG4 = W.SW_ADJOINT_32X32_P16


def build(eo, w, precision):
    pr = w.params
    g = eo.Grid(w.nlx, w.nly, w.p)
    op = eo.Operator(g, eo.SW_WALLS, band=W.BAND[CFG4.name], n_poles=w.n_poles, f=pr["f"], g=pr["g"], H=pr["H"],
                     shared_ops=True, precision=precision)
    return g, op


def problem_data(w, g, op, n_sensors, rng):
    x, y = g.nodes()
    u0 = np.stack(W.initial_fields(w, x, y, 0))
    ref = np.stack(W.initial_fields(w, x, y, 1))
    idx = np.sort(rng.choice(g.n_nodes, n_sensors, replace=False))
    d = []
    r = torch.tensor(ref, device="cuda")
    for _ in range(w.steps):
        op.apply(r, 1)
        d.append(r[2, torch.tensor(idx, device="cuda")].clone())
    return u0, idx, torch.stack(d)


def test_cfg4_gradient_at_stated_size():
    import paper_1402_5168_gb300 as eo
    from paper_1402_5168_gb300.autograd import sensor_misfit
    w = CFG4
    pr = w.params
    rng = np.random.default_rng(w.seed)
    g, op64 = build(eo, w, "fp64")
    assert op64.alpha.size == 61
    u0, idx_np, data = problem_data(w, g, op64, pr["n_sensors"], rng)
    idx = torch.tensor(idx_np, device="cuda")
    dirs = rng.standard_normal((pr["fd_directions"], 3, g.n_nodes))
    dirs /= np.linalg.norm(dirs.reshape(len(dirs), -1), axis=1)[:, None, None]
    eps = 1e-3 * float(np.linalg.norm(u0))
    grads = {}
    for prec, op in (("fp64", op64), ("df32", build(eo, w, "df32")[1])):
        ut = torch.tensor(u0, device="cuda", requires_grad=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        loss = sensor_misfit(op, ut, w.steps, 2, idx, data, checkpoint_every=pr["checkpoint_every"])
        loss.backward()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        gr = ut.grad.detach()
        grads[prec] = gr
        u0t = torch.tensor(u0, device="cuda")
        worst = 0.0
        with torch.no_grad():
            for k in range(len(dirs)):
                v = torch.tensor(dirs[k], device="cuda")
                lp = sensor_misfit(op, u0t + eps * v, w.steps, 2, idx, data)
                lm = sensor_misfit(op, u0t - eps * v, w.steps, 2, idx, data)
                fd = float((lp - lm) / (2 * eps))
                an = float((gr * v).sum())
                err = abs(fd - an) / max(abs(an), 1e-30)
                worst = max(worst, err)
                assert abs(fd - an) <= 1e-7 * abs(an) + 1e-9 * float(loss), (prec, k, fd, an)
        print(f"cfg4 {prec}: loss {float(loss):.6e}, gradient (50 forward + 50 transposed steps, "
              f"checkpoints every 10) in {dt:.2f} s, worst FD relative error over 20 directions {worst:.2e}")
    e = float(torch.linalg.vector_norm(grads["df32"] - grads["fp64"]) / torch.linalg.vector_norm(grads["fp64"]))
    print(f"cfg4: FP32-pair gradient vs FP64 gradient {e:.3e}")
    assert e <= 1e-7


def test_cfg4_recipe_small_grid_against_oracle_gradient():
    import paper_1402_5168_gb300 as eo
    from paper_1402_5168_gb300.autograd import sensor_misfit
    w = W.dataclasses.replace(CFG4, nlx=2, nly=2, p=10)
    rng = np.random.default_rng(w.seed + 1)
    g, op = build(eo, w, "fp64")
    u0, idx_np, data = problem_data(w, g, op, 64, rng)
    idx = torch.tensor(idx_np, device="cuda")
    ut = torch.tensor(u0, device="cuda", requires_grad=True)
    loss = sensor_misfit(op, ut, w.steps, 2, idx, data, checkpoint_every=10)
    loss.backward()
    got = ut.grad.detach().cpu().numpy()
    pr = w.params
    prob = Problem(sem.Grid(2, 2, 10), "sw", op.tau, f=pr["f"], g=pr["g"], H=pr["H"])
    G = step_matrix(Stepper(prob, op.alpha, op.b))
    n = g.n_nodes
    dn = data.cpu().numpy()
    # forward states and the backward recursion lam_t = G^T lam_{t+1} + 2 S^T r_t
    us = [u0.ravel()]
    for _ in range(w.steps):
        us.append(G @ us[-1])
    sel = 2 * n + idx_np
    lam = np.zeros(3 * n)
    for t in range(w.steps, 0, -1):
        seed = np.zeros(3 * n)
        seed[sel] = 2.0 * (us[t][sel] - dn[t - 1])
        lam = G.T @ (lam + seed)
    e = float(np.linalg.norm(got.ravel() - lam) / np.linalg.norm(lam))
    growth = float(np.linalg.norm(us[-1]) / np.linalg.norm(us[0]))
    print(f"cfg4 recipe on 2x2/p10, 50 steps, 64 sensors: library gradient vs oracle (dense G^T) {e:.3e}, "
          f"state norm growth over 50 steps {growth:.3f}")
    assert e <= 1e-9
