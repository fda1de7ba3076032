"""Pins of the naive VEM prolongation (Eq. 16, the "Ours^np" ablation) in the
oracle: it still reproduces linear functions and its multigrid PCG still
solves the system, but its coarse operators couple DOFs that share no coarse
cell (the diffusion the paper shows for it), so they have more nonzeros than
the diffusion-free ones (Eq. 17)."""
import numpy as np
import pytest

import scenes


@pytest.fixture(scope="module")
def both():
    from oracle.pipeline import build_system
    sc = scenes.config(0, 8)
    return build_system(sc), build_system(sc, naive_prolongation=True)


def test_naive_prolongation_reproduces_linears(both):
    _, N = both
    for l, P in enumerate(N.Pfull):
        Vf, Vc = N.meshes[l].V, N.meshes[l + 1].V
        q = np.array([0.3, -1.1, 0.7])
        used = np.diff(P.tocsc().indptr) > 0
        rows = np.diff(P.indptr) > 0
        err = P @ (Vc @ q + 0.25) - (Vf @ q + 0.25)
        assert np.abs(err[rows]).max() <= 1e-12, l
        assert used.any()


def test_naive_coarse_operators_spread_across_cells(both):
    """Level 1: every nonzero of the diffusion-free operator joins two DOFs of
    one coarse cell; the naive operator has nonzeros that do not, and more of
    them."""
    D, N = both
    A_d, A_n = D.H.A[1].tocoo(), N.H.A[1].tocoo()
    M1 = D.meshes[1]
    fr = D.free[1]
    cells = [set(vs) for vs in M1.cell_verts]
    def local(i, j):
        a, b = fr[i], fr[j]
        return any(a in c and b in c for c in cells)
    assert all(local(i, j) for i, j in zip(A_d.row, A_d.col))
    frn = N.free[1]
    cells_n = [set(vs) for vs in N.meshes[1].cell_verts]
    nonlocal_n = sum(1 for i, j in zip(A_n.row, A_n.col)
                     if not any(frn[i] in c and frn[j] in c for c in cells_n))
    assert nonlocal_n > 0
    assert A_n.nnz > A_d.nnz


def test_naive_mgpcg_matches_direct_solve(both):
    import scipy.sparse.linalg as spla
    from oracle.multigrid import pcg
    _, N = both
    A = N.H.A[0]
    b = np.cos(np.arange(A.shape[0]) * 0.37)
    x, its, _ = pcg(A, b, N.H.vcycle, tol=1e-10)
    xd = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-8


# ---- second order (k = 2): Eq. 16 with the cell projector Pi_2, the setting
# of the paper's ablation

@pytest.fixture(scope="module")
def both_k2():
    from oracle.system2 import build_hierarchy2
    sc = scenes.config(0, 4)
    return build_hierarchy2(sc, L=2), build_hierarchy2(sc, L=2, naive_prolongation=True)


def test_naive_k2_prolongation_reproduces_quadratics(both_k2):
    """Pi_2 reproduces quadratics, so the naive P maps the coarse DOFs of a
    quadratic (vertex values, edge midpoints, face and cell means) to its
    fine DOFs, like the diffusion-free one."""
    _, N = both_k2
    a = np.random.default_rng(2).standard_normal(10)

    def q(X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        return (a[0] + a[1] * x + a[2] * y + a[3] * z + a[4] * x * x + a[5] * x * y + a[6] * x * z
                + a[7] * y * y + a[8] * y * z + a[9] * z * z)

    def dofs(Lv):
        d = np.zeros(Lv.n)
        for E, dm in zip(Lv.cells, Lv.dofmap):
            d[dm] = E.dofs_of(q)
        return d

    df, dc = dofs(N.levels[0]), dofs(N.levels[1])
    assert np.abs(N.Pfull[0] @ dc - df).max() <= 1e-11 * np.abs(df).max()


def test_naive_k2_rows_use_whole_cells_and_coarse_operator_fills_in(both_k2):
    """Every naive row that is not a vertex copy uses all of its parent cell's
    DOFs; the diffusion-free rows of fine DOFs on coarse faces use only that
    face's.  The naive level-1 operator holds several times the nonzeros."""
    D, N = both_k2
    Pd, Pn = D.Pfull[0].tocsr(), N.Pfull[0].tocsr()
    ld, ln = np.diff(Pd.indptr), np.diff(Pn.indptr)
    assert (ln >= ld).all() and (ln > ld).sum() > 0
    cell_sizes = {len(dm) for dm in N.levels[1].dofmap}
    assert set(np.unique(ln[ln > 1])) <= cell_sizes
    assert N.H.A[1].nnz > 3 * D.H.A[1].nnz


def test_naive_k2_mgpcg_matches_direct_solve(both_k2):
    import scipy.sparse.linalg as spla
    from oracle.multigrid import pcg
    _, N = both_k2
    A = N.H.A[0]
    b = np.cos(np.arange(A.shape[0]) * 0.29)
    x, its, _ = pcg(A, b, N.H.vcycle, tol=1e-10)
    xd = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-8
