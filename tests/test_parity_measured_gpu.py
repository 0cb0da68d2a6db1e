"""Oracle parity of the configurations the benchmark times, in the precision it
times them in.

* The FP32-pair (df32) handle of the full shallow-water workload (16x16 leaves,
  p = 16, tau = 20 inertial periods, thousands of poles): sampled single
  resolvents the oracle can compute one by one.
* One full df32 step of rotating shallow water on a square 4x4-leaf, p = 16 grid
  with 301 poles, where every variant of the timed path is active at once: the
  fast-diagonal leaves over more than one pole chunk, the even/odd merge blocks
  (n3 up to 56), the four-block root wall solve, the q = 14 register leaf kernels.
* The batched wave path (per-box operators, c = clip(exp(GRF), 0.5, 2), p = 16,
  61 poles) with 9 right-hand sides, so that an 8-column block and a ragged
  1-column block both run, in FP64 and df32, compared column by column.

Tolerance: relative L2 <= 1e-10 per step or resolvent (the FP64 parity target),
for df32 as well (its operators carry ~2^-48 relative error); where two FP64
orderings of the oracle itself differ by more (the variable-coefficient case), twice
that rounding floor.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

import workloads as W
from oracle import sem
from oracle.resolvent import Problem, Stepper

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def test_full_size_df32_sampled_resolvents():
    import paper_1402_5168_gb300 as eo
    w = W.SW_16X16_P16
    pr = w.params
    g = eo.Grid(w.nlx, w.nly, w.p)
    op = eo.Operator(g, eo.SW_WALLS, band=W.BAND[w.name], tau=w.tau, f=pr["f"], g=pr["g"], H=pr["H"],
                     shared_ops=True, precision="df32")
    prob = Problem(sem.Grid(w.nlx, w.nly, w.p), "sw", op.tau, f=pr["f"], g=pr["g"], H=pr["H"])
    st = Stepper(prob, op.alpha, op.b)
    x, y = g.nodes()
    u0 = np.stack(W.initial_fields(w, x, y))
    u = torch.tensor(u0, device="cuda")
    M = (op.alpha.size - 1) // 2
    for j in (M, M + (M // 3), 2 * M):        # real pole, inside the band, outermost
        xg = torch.zeros((3, g.n_nodes), dtype=torch.complex128, device="cuda")
        op.resolvent(j, u, xg)
        want = st.resolvent(j, u0)
        e = rel(xg.cpu().numpy(), want)
        print(f"df32 resolvent j={j} alpha={op.alpha[j]:.3f} rel {e:.3e}")
        assert e <= 1e-10


@pytest.mark.parametrize("precision", ["df32", "fp64"])
def test_sw_4x4_p16_301_poles_full_step(precision):
    import paper_1402_5168_gb300 as eo
    w = W.dataclasses.replace(W.SW_16X16_P16, nlx=4, nly=4)
    pr = w.params
    g = eo.Grid(4, 4, 16)
    x, y = g.nodes()
    op = eo.Operator(g, eo.SW_WALLS, band=W.BAND[W.SW_16X16_P16.name], n_poles=301, f=pr["f"], g=pr["g"],
                     H=pr["H"], shared_ops=True, precision=precision)
    assert op.alpha.size == 301
    u0 = np.stack(W.initial_fields(w, x, y))
    u = torch.tensor(u0, device="cuda")
    op.apply(u, 1)
    torch.cuda.synchronize()
    prob = Problem(sem.Grid(4, 4, 16), "sw", op.tau, f=pr["f"], g=pr["g"], H=pr["H"])
    want = Stepper(prob, op.alpha, op.b).step(u0)
    e = rel(u.cpu().numpy(), want)
    print(f"sw 4x4/p16, 301 poles, {precision}: one step rel L2 vs oracle {e:.3e}")
    assert e <= 1e-10


@pytest.fixture(scope="module")
def grf_case():
    """The oracle's steps and rounding floors of the batched wave case, computed once
    for both precisions (the FP64 handle's poles and residues; the df32 handle is built
    from the same fit)."""
    import paper_1402_5168_gb300 as eo
    w = W.dataclasses.replace(W.WAVE_32X32_P16, nlx=8, nly=8)
    g = eo.Grid(8, 8, 16)
    x, y = g.nodes()
    c = W.wave_c(w, x, y)
    assert c.min() >= 0.5 and c.max() <= 2.0
    R = 9
    kw = dict(band=W.BAND[W.WAVE_32X32_P16.name], n_poles=61, c2=c * c, max_rhs=R)
    op = eo.Operator(g, eo.WAVE_DIRICHLET, precision="fp64", **kw)
    U0 = np.stack([np.stack(W.initial_fields(w, x, y, r)) for r in range(R)])
    st = Stepper(Problem(sem.Grid(8, 8, 16), "wave", op.tau, c2=c * c), op.alpha, op.b)
    # rounding floor of two FP64 computations of the same step: the oracle against
    # itself with another sparse-LU column ordering (the clipped GRF coefficient and
    # the pole sum's cancellation amplify rounding to ~1e-10 here)
    st2 = Stepper(st.prob, op.alpha, op.b)
    st2._lu = {i: spla.splu(st.prob.system(op.alpha[i]), permc_spec="MMD_AT_PLUS_A")
               for i in range(op.alpha.size) if op.alpha[i].imag >= 0}
    want = [st.step(U0[r]) for r in range(R)]
    floor = [rel(st2.step(U0[r]), want[r]) for r in range(R)]
    return g, kw, U0, want, floor, op


@pytest.mark.parametrize("precision", ["fp64", "df32"])
def test_batched_wave_grf_p16_61_poles_9_rhs(precision, grf_case):
    import paper_1402_5168_gb300 as eo
    g, kw, U0, want, floor, op64 = grf_case
    op = op64 if precision == "fp64" else eo.Operator(g, eo.WAVE_DIRICHLET, precision=precision, **kw)
    u = torch.tensor(U0, device="cuda")
    op.apply(u, 1)
    torch.cuda.synchronize()
    got = u.cpu().numpy()
    for r in range(U0.shape[0]):
        e = rel(got[r], want[r])
        print(f"wave GRF 8x8/p16, 61 poles, {precision}, rhs {r}: rel L2 vs oracle {e:.3e} "
              f"(oracle rounding floor {floor[r]:.3e})")
        assert e <= max(1e-10, 2 * floor[r]), (r, e, floor[r])
