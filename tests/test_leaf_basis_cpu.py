"""Host checks of the separable leaf eigenbasis (eo_leaf_basis) against the
oracle's collocated operator: on a constant-coefficient leaf the interior block
of div(a grad) (Section 2.2, nested 1-D differentiation) must be the Kronecker
sum I (x) M_x + M_y (x) I with M = V diag(lam) V^{-1} from the library, and the
leaf solve through that basis must equal a direct sparse solve."""
import numpy as np
import pytest

from oracle import sem


@pytest.fixture(scope="module")
def eo():
    import os
    from paper_1402_5168_gb300 import _capi, build_ext
    if not os.path.exists(_capi.LIB_PATH):
        build_ext.build()
    import paper_1402_5168_gb300 as m
    return m


def interior_block(p, hx, hy, a):
    g = sem.Grid(1, 1, p, 0.0, hx, 0.0, hy)
    A = sem.divgrad_operator(g, np.full(g.n_nodes, a)).tocsr()
    ii = np.arange(g.n_int)          # interior ids of leaf 0: (j-1) q + (k-1)
    return A[ii][:, ii].toarray()


@pytest.mark.parametrize("p,hx,hy,a", [(4, 1.0, 1.0, 1.0), (6, 0.5, 0.25, 2.5), (10, 1 / 16, 1 / 16, 1.0),
                                       (16, 1 / 16, 1 / 8, 0.7), (24, 0.1, 0.3, 1.0)])
def test_interior_block_is_a_kronecker_sum_in_the_library_basis(eo, p, hx, hy, a):
    q = p - 2
    lx, Vx, Vxi = eo.leaf_basis(p, hx, a)
    ly, Vy, Vyi = eo.leaf_basis(p, hy, a)
    Mx = Vx @ np.diag(lx) @ Vxi
    My = Vy @ np.diag(ly) @ Vyi
    Aii = interior_block(p, hx, hy, a)
    K = np.kron(np.eye(q), Mx) + np.kron(My, np.eye(q))
    assert np.abs(K - Aii).max() <= 1e-12 * np.abs(Aii).max()
    # eigenvalues real, negative and descending; V Vinv = I
    assert np.all(lx < 0) and np.all(np.diff(lx) < 0)
    assert np.allclose(Vx @ Vxi, np.eye(q), atol=1e-13)


@pytest.mark.parametrize("p", [8, 12, 16])
def test_fast_diagonal_leaf_solve_equals_sparse_solve(eo, p):
    """(A_ii - kappa^2) z = f through (V_y (x) V_x) diag(1/(lx_a + ly_b - kappa^2)) (V_y (x) V_x)^{-1}
    for a complex kappa^2 like those of the shallow-water poles."""
    q = p - 2
    hx, hy = 1 / 16, 1 / 8
    lx, Vx, Vxi = eo.leaf_basis(p, hx, 1.0)
    ly, Vy, Vyi = eo.leaf_basis(p, hy, 1.0)
    Aii = interior_block(p, hx, hy, 1.0)
    rng = np.random.default_rng(p)
    f = rng.standard_normal(q * q) + 1j * rng.standard_normal(q * q)
    for k2 in (3.0 + 40.0j, -250.0 + 7.0j, 1e4 - 1e3j):
        z_ref = np.linalg.solve(Aii - k2 * np.eye(q * q), f)
        F = f.reshape(q, q).T                      # F[k, j]
        Fh = Vxi @ F @ Vyi.T                       # hat(a, b)
        Zh = Fh / (lx[:, None] + ly[None, :] - k2)
        Z = Vx @ Zh @ Vy.T
        z = Z.T.ravel()
        assert np.linalg.norm(z - z_ref) <= 1e-12 * np.linalg.norm(z_ref)


def test_eigenvalues_match_a_dense_eigensolver(eo):
    p, h = 16, 0.25
    g = sem.Grid(1, 1, p, 0.0, h, 0.0, h)
    M = (g.Dx @ g.Dx)[1:-1, 1:-1]
    lam, V, Vi = eo.leaf_basis(p, h, 1.0)
    ref = np.sort(np.linalg.eigvals(M).real)[::-1]
    assert np.abs(lam - ref).max() <= 1e-13 * np.abs(ref).max()
    assert np.allclose(np.linalg.norm(V, axis=0), 1.0, atol=1e-14)


def test_leaf_basis_rejects_bad_arguments(eo):
    from paper_1402_5168_gb300 import ExpopError
    for args in [(3, 1.0, 1.0), (25, 1.0, 1.0), (8, 0.0, 1.0), (8, 1.0, -1.0)]:
        with pytest.raises(ExpopError):
            eo.leaf_basis(*args)
