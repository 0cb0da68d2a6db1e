"""Fused low merge levels (opts.merge_fuse): levels 1 .. Lf of both sweeps in one launch
each, against one launch per level (merge_fuse = 0, the default) of the same build and against
the oracle.  Shared per-level operators exist for shallow water (constant
coefficients), so that is the problem kind fused.

The fused kernels run the per-column arithmetic of the per-level kernels with another
split of the block products over threads, so the two agree to rounding (1e-12 relative
in FP64 and 1e-10 in FP32 pairs after three steps), not bit for bit.  Grids cover every
fused depth (1 .. 4), rectangular subtrees, an odd q (p = 5, where the reflection
blocks do not apply to every level and fusion stops below the first such level), and
several right-hand sides, so that column groups of 8, 4, 2 and 1 and a ragged group
all run.
"""
import numpy as np
import pytest

import workloads as W
from oracle import sem
from oracle.resolvent import Problem, Stepper

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def state(g, seed=1000, R=1):
    x, y = g.nodes()
    out = []
    for r in range(R):
        c, s, a = W.draw_gaussians(seed + r, 3, (0.1, 0.15), (0.1, 1.0), (0.3, 0.7))
        h = W.gaussian_sum(x, y, c, s, a)
        out.append(np.stack([0.3 * np.sin(np.pi * y) * x * (1 - x), -0.2 * np.sin(np.pi * x) * y * (1 - y), h]))
    return out[0] if R == 1 else np.stack(out)


def levels(nlx, nly):
    return int(np.log2(nlx)) + int(np.log2(nly))


def up_merge_launches(op, u):
    op.set_timing(True)
    op.timing()
    op.apply(u, 1)
    t = op.timing()
    op.set_timing(False)
    return t["up_merge"][0], t["down_merge"][0]


@pytest.mark.parametrize("nlx,nly,p,precision,R", [(2, 2, 8, "fp64", 1), (4, 4, 10, "df32", 1),
                                                   (2, 8, 16, "fp64", 1), (8, 8, 12, "df32", 1),
                                                   (16, 16, 6, "fp64", 1), (4, 4, 8, "fp64", 5),
                                                   (8, 4, 8, "df32", 3), (4, 2, 5, "fp64", 1)])
def test_fused_levels_match_one_launch_per_level(nlx, nly, p, precision, R):
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(nlx, nly, p)
    kw = dict(band=60.0, n_poles=21, f=10.0, g=1.0, H=1.0, shared_ops=True, precision=precision, max_rhs=R)
    L = levels(nlx, nly)
    u0 = state(g, R=R)
    base = eo.Operator(g, eo.SW_WALLS, **kw)
    b = torch.tensor(u0, device="cuda")
    nu, nd = up_merge_launches(base, b)
    assert nu == L and nd == L and base.fused_levels(R) == 0
    b = torch.tensor(u0, device="cuda")
    base.apply(b, 3)
    want = b.cpu().numpy()
    tol = 1e-12 if precision == "fp64" else 1e-10
    for k in (1, 2, 3, 4):
        op = eo.Operator(g, eo.SW_WALLS, merge_fuse=k, **kw)
        a = torch.tensor(u0, device="cuda")
        nu, nd = up_merge_launches(op, a)
        a = torch.tensor(u0, device="cuda")
        op.apply(a, 3)
        e = rel(a.cpu().numpy(), want)
        print(f"{nlx}x{nly} p={p} {precision} R={R} merge_fuse={k}: {nu} up / {nd} down merge launches, "
              f"vs one launch per level after 3 steps {e:.1e}")
        lf = op.fused_levels(R)
        assert nu == nd == L - lf + (1 if lf else 0), (nu, nd, lf)
        if p % 2 == 0:   # even q: every level symmetric, fused depth min(k, L - 1)
            assert lf == min(k, L - 1), (lf, k)
        else:            # q odd: level 1 (n3 = q) has no even/odd split, nothing fused
            assert lf == 0
        assert e <= tol, (k, e)


def test_fused_levels_match_the_oracle_multi_rhs():
    import paper_1402_5168_gb300 as eo
    g = eo.Grid(8, 4, 8)
    R = 3
    op = eo.Operator(g, eo.SW_WALLS, band=60.0, n_poles=21, f=10.0, g=1.0, H=1.0, shared_ops=True, max_rhs=R,
                     precision="df32", merge_fuse=4)
    U0 = state(g, 1003, R=R)
    u = torch.tensor(U0, device="cuda")
    nu, _ = up_merge_launches(op, u)
    assert op.fused_levels(R) == 4 and nu == levels(8, 4) - 4 + 1
    u = torch.tensor(U0, device="cuda")
    op.apply(u, 1)
    got = u.cpu().numpy()
    st = Stepper(Problem(sem.Grid(8, 4, 8), "sw", op.tau, f=10.0, g=1.0, H=1.0), op.alpha, op.b)
    for r in range(R):
        e = rel(got[r], st.step(U0[r]))
        print(f"8x4 p=8 df32, fused levels 1-4, rhs {r}: vs oracle {e:.1e}")
        assert e <= 1e-10


def test_merge_fuse_out_of_range_rejected():
    import paper_1402_5168_gb300 as eo
    from paper_1402_5168_gb300 import ExpopError
    g = eo.Grid(2, 2, 8)
    for k in (-1, 5):
        with pytest.raises(ExpopError, match="merge_fuse"):
            eo.Operator(g, eo.SW_WALLS, band=60.0, n_poles=21, f=10.0, shared_ops=True, merge_fuse=k)
