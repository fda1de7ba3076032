"""Pins of the k = 2 VEM element of the oracle (Sec. 3.1, Eq. 11-14): what the
mathematics fixes for any convex polyhedron.  CPU only."""
import numpy as np
import pytest

from oracle.vem2 import CellVEM2, Face2, polyhedron_quadrature


def _cube(h=1.0, skew=0.0):
    V = np.array([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], dtype=float) * h
    V[:, 0] += skew * V[:, 2]                      # a sheared (still convex) hexahedron
    idx = lambda i, j, k: i + 2 * j + 4 * k
    faces = [[idx(0, 0, 0), idx(0, 0, 1), idx(0, 1, 1), idx(0, 1, 0)],
             [idx(1, 0, 0), idx(1, 1, 0), idx(1, 1, 1), idx(1, 0, 1)],
             [idx(0, 0, 0), idx(1, 0, 0), idx(1, 0, 1), idx(0, 0, 1)],
             [idx(0, 1, 0), idx(0, 1, 1), idx(1, 1, 1), idx(1, 1, 0)],
             [idx(0, 0, 0), idx(0, 1, 0), idx(1, 1, 0), idx(1, 0, 0)],
             [idx(0, 0, 1), idx(1, 0, 1), idx(1, 1, 1), idx(0, 1, 1)]]
    return V, faces, list(range(8))


def _quadratic(seed):
    c = np.random.default_rng(seed).standard_normal(10)

    def q(X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        return (c[0] + c[1] * x + c[2] * y + c[3] * z + c[4] * x * x + c[5] * x * y + c[6] * x * z
                + c[7] * y * y + c[8] * y * z + c[9] * z * z)

    def grad(X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        return np.stack([c[1] + 2 * c[4] * x + c[5] * y + c[6] * z,
                         c[2] + c[5] * x + 2 * c[7] * y + c[8] * z,
                         c[3] + c[6] * x + c[8] * y + 2 * c[9] * z], axis=1)
    return q, grad


def _cells(sphere8, count=12):
    """The cube, a sheared hexahedron, and the cut cells of the 8^3 sphere
    scene with the most faces."""
    out = [_cube(0.37), _cube(1.0, skew=0.3)]
    M = sphere8.meshes[0]
    order = sorted(range(len(M.cell_faces)), key=lambda c: -len(M.cell_faces[c]))[:count]
    for c in order:
        out.append((M.V, [f[2] for f in M.cell_faces[c]], M.cell_verts[c]))
    return out


def test_face_projector_reproduces_quadratics(sphere8):
    for V, faces, _ in _cells(sphere8, 4):
        for cyc in faces:
            F = Face2(V, cyc)
            q, _ = _quadratic(len(cyc))
            P = V[cyc]
            mids = 0.5 * (P + np.roll(P, -1, axis=0))
            d = np.concatenate([q(P), q(mids), [float(F.qw @ q(F.qp)) / F.area]])
            coef = F.Pis @ d
            assert np.allclose(F.mono2(F.qp)[0] @ coef, q(F.qp), atol=1e-11 * max(1.0, np.abs(q(F.qp)).max()))


def test_cell_projector_reproduces_quadratics(sphere8):
    for V, faces, verts in _cells(sphere8):
        E = CellVEM2(V, faces, verts)
        q, _ = _quadratic(E.n)
        d = E.dofs_of(q)
        assert np.allclose(E.Pi @ d, d, atol=1e-10 * max(1.0, np.abs(d).max()))


def test_energy_of_quadratics_is_exact(sphere8):
    """For q in P2 the stabilisation vanishes and d(q)^T K d(q) = int_E |grad q|^2
    (right side by independent quadrature, exact for degree 2)."""
    for V, faces, verts in _cells(sphere8):
        E = CellVEM2(V, faces, verts)
        q, gq = _quadratic(3 * E.n)
        d = E.dofs_of(q)
        qp, qw = polyhedron_quadrature(V, faces)
        ref = float(qw @ (gq(qp) ** 2).sum(axis=1))
        assert abs(d @ E.K @ d - ref) <= 1e-10 * max(1.0, ref)


def test_element_symmetric_psd_with_constant_kernel(sphere8):
    """Rounding bound 1e-14 cond(G) max|K|: cut cells with tiny sub-faces give
    ill-conditioned projectors (Eq. 14)."""
    for V, faces, verts in _cells(sphere8):
        E = CellVEM2(V, faces, verts)
        K = E.K
        tol = 1e-14 * np.linalg.cond(E.G) * np.abs(K).max()
        assert np.abs(K - K.T).max() <= tol
        ev = np.linalg.eigvalsh(K)
        assert ev[0] > -tol
        assert np.abs(K @ np.ones(E.n)).max() <= tol
        assert (ev > 1e-8 * ev[-1]).sum() == E.n - 1


def test_element_scales_with_h():
    V, faces, verts = _cube(1.0, skew=0.2)
    K1 = CellVEM2(V, faces, verts).K
    K3 = CellVEM2(V * 0.25, faces, verts).K
    assert np.allclose(K3, 0.25 * K1, atol=1e-13)


def test_cube_dof_counts():
    V, faces, verts = _cube()
    E = CellVEM2(V, faces, verts)
    assert (len(E.verts), len(E.edges), E.n) == (8, 12, 8 + 12 + 6 + 1)


# ------------------------------------------------------------------ global system (level 0)

@pytest.fixture(scope="module")
def sphere6_k2():
    import scenes
    from oracle.system2 import build_system2
    return build_system2(scenes.config(0, 6))


def test_k2_system_symmetric_with_constant_kernel(sphere6_k2):
    S = sphere6_k2
    K = S.K
    assert abs(K - K.T).max() <= 1e-13 * abs(K).max()
    assert np.abs(K @ np.ones(S.n)).max() <= 1e-10 * abs(K).max()
    assert S.n == S.nv + S.ne + S.nf + len(S.cells)


def test_k2_global_patch_test_quadratic_pressure(sphere6_k2):
    """u' = grad q with q quadratic and q = 0 on y = 1: Pi_1 u' = grad q, the
    element is exact on P2, so the k = 2 system returns q's DOFs exactly (a
    first-order discretisation cannot)."""
    from oracle.system2 import dofs_of2, solve2
    S = sphere6_k2
    a, b, c, d = 0.3, -0.7, 0.4, 1.1
    q = lambda X: (1 - X[:, 1]) * (a + b * X[:, 0] + c * X[:, 1] + d * X[:, 2])
    gq = lambda X: np.stack([(1 - X[:, 1]) * b,
                             -(a + b * X[:, 0] + c * X[:, 1] + d * X[:, 2]) + (1 - X[:, 1]) * c,
                             (1 - X[:, 1]) * d], axis=1)
    p = solve2(S, gq(S.mesh.V))
    dq = dofs_of2(S, q)
    assert np.abs(p - dq).max() <= 1e-10 * np.abs(dq).max()


@pytest.mark.slow
def test_k2_third_order_convergence():
    """With the exact grad q integrated against grad Pi_2 phi_i (so that only
    the element and the assembly are tested, not the first-order velocity
    representation), the k = 2 vertex error falls at third order: observed
    about 3.2 from 4^3 to 8^3 on the empty box (first order VEM: 2)."""
    import scenes
    import scipy.sparse.linalg as spla
    from oracle.system2 import build_system2
    from oracle.vem2 import mono3

    def q(V):
        x, y, z = V[:, 0], V[:, 1], V[:, 2]
        return np.cos(np.pi * x) * np.cos(np.pi * z) * np.sin(0.5 * np.pi * (1 - y))

    def gq(V):
        x, y, z = V[:, 0], V[:, 1], V[:, 2]
        a, b, c = np.cos(np.pi * x), np.sin(0.5 * np.pi * (1 - y)), np.cos(np.pi * z)
        return np.stack([-np.pi * np.sin(np.pi * x) * b * c,
                         -0.5 * np.pi * a * np.cos(0.5 * np.pi * (1 - y)) * c,
                         -np.pi * a * b * np.sin(np.pi * z)], axis=1)

    err = []
    for N in (4, 8):
        S = build_system2(scenes.empty_scene(N))
        r = np.zeros(S.n)
        for E, dm in zip(S.cells, S.dofmap):
            qp, qw = polyhedron_quadrature(S.mesh.V, E._faces)
            _, g = mono3(qp, E.xE, E.hE)
            r[dm] += np.einsum("q,qd,qid->i", qw, gq(qp), np.einsum("qad,ai->qid", g, E.Pis))
        f = S.free
        p = np.zeros(S.n)
        p[f] = spla.spsolve(S.K[f][:, f].tocsc(), r[f])
        e = p[:S.nv] - q(S.mesh.V)
        err.append((np.abs(e).max(), np.sqrt(np.mean(e ** 2))))
    for k in range(2):
        assert np.log2(err[0][k] / err[1][k]) >= 2.8, err


# ------------------------------------------------------------------ hierarchy (k = 2)

@pytest.fixture(scope="module")
def sphere4_k2_mg():
    import scenes
    from oracle.system2 import build_hierarchy2
    return build_hierarchy2(scenes.config(0, 4), L=2)


def test_k2_prolongation_reproduces_quadratics(sphere4_k2_mg):
    """Vertex, edge-midpoint, face-mean and cell-mean DOFs of a quadratic on the
    coarse level map to those of the same quadratic on the fine level: the
    quadratic through a coarse edge's DOFs, the face projector Pi_{2,F} and
    the cell projector Pi_2 all reproduce P2."""
    S = sphere4_k2_mg
    a = np.random.default_rng(1).standard_normal(10)

    def q(X):
        x, y, z = X[:, 0], X[:, 1], X[:, 2]
        return (a[0] + a[1] * x + a[2] * y + a[3] * z + a[4] * x * x + a[5] * x * y + a[6] * x * z
                + a[7] * y * y + a[8] * y * z + a[9] * z * z)

    def dofs(Lv):
        d = np.zeros(Lv.n)
        for E, dm in zip(Lv.cells, Lv.dofmap):
            d[dm] = E.dofs_of(q)
        return d

    for l, P in enumerate(S.Pfull):
        df, dc = dofs(S.levels[l]), dofs(S.levels[l + 1])
        assert np.abs(P @ dc - df).max() <= 1e-11 * np.abs(df).max(), l


def test_k2_mgpcg_matches_direct_solve(sphere4_k2_mg):
    """Both V-cycles (unscaled, and the diagonally scaled k = 2 reading) give
    PCG solutions equal to the sparse direct solve."""
    import scipy.sparse.linalg as spla
    from oracle.multigrid import pcg
    S = sphere4_k2_mg
    A = S.H.A[0]
    b = np.random.default_rng(2).standard_normal(A.shape[0])
    xd = spla.spsolve(A.tocsc(), b)
    for M in (S.H.vcycle, S.Hs):
        x, its, _ = pcg(A, b, M, 1e-11, max_iters=1000)
        assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-8


@pytest.mark.slow
def test_k2_scaled_mgpcg_iterations_in_paper_range():
    """Empty box at 8^3, 3 levels, tolerance 1e-10: the diagonally scaled k = 2
    V-cycle keeps PCG within Table 4's 7-16 iterations (measured 14; the
    unscaled k = 1 smoother needs 26 here), and so does the condensed one."""
    import scenes
    from oracle.multigrid import pcg
    from oracle.system2 import build_hierarchy2
    S = build_hierarchy2(scenes.empty_scene(8), L=3)
    A = S.H.A[0]
    b = np.random.default_rng(2).standard_normal(A.shape[0])
    _, its, _ = pcg(A, b, S.Hs, 1e-10, max_iters=200)
    assert its <= 16
    bc = np.random.default_rng(3).standard_normal(S.S0.shape[0])
    _, its_c, _ = pcg(S.S0, bc, S.Hc, 1e-10, max_iters=200)
    assert its_c <= 16


def test_k2_condensed_solve_matches_direct(sphere4_k2_mg):
    """The condensed solve (Schur complement on the non-cell DOFs, cell DOFs
    recovered per cell) equals the direct solve of the full k = 2 system."""
    import scipy.sparse.linalg as spla
    from oracle.multigrid import pcg
    S = sphere4_k2_mg
    A = S.levels[0].K
    f = S.free[0]
    r = np.zeros(S.n)
    r[f] = np.random.default_rng(4).standard_normal(len(f))
    xd = np.zeros(S.n)
    xd[f] = spla.spsolve(A[f][:, f].tocsc(), r[f])
    rb = r[S.b0] - S.Kbc0 @ (S.dinv0 * r[S.c0])
    xb, _, _ = pcg(S.S0, rb, S.Hc, 1e-12, max_iters=1000)
    x = np.zeros(S.n)
    x[S.b0] = xb
    x[S.c0] = S.dinv0 * (r[S.c0] - S.Kbc0.T @ xb)
    assert np.linalg.norm(x - xd) / np.linalg.norm(xd) <= 1e-8


def test_k2_projection_patch_test(sphere4_k2_mg):
    """u' = grad q, q quadratic and zero on y = 1 (Sec. 3.2-3.3): the k = 2
    projection (multigrid PCG with the scaled V-cycle) returns p = q on every
    DOF and a divergence-free correction that vanishes, Pi_1 u_new = 0."""
    from oracle.system2 import dofs_of2, project2
    S = sphere4_k2_mg
    a, b, c, d = 0.3, -0.7, 0.4, 1.1
    q = lambda X: (1 - X[:, 1]) * (a + b * X[:, 0] + c * X[:, 1] + d * X[:, 2])
    gq = lambda X: np.stack([(1 - X[:, 1]) * b,
                             -(a + b * X[:, 0] + c * X[:, 1] + d * X[:, 2]) + (1 - X[:, 1]) * c,
                             (1 - X[:, 1]) * d], axis=1)
    p, cellpoly, its = project2(S, gq(S.mesh.V), tol=1e-12, max_iters=1000)
    dq = dofs_of2(S, q)
    assert np.abs(p - dq).max() <= 1e-9 * np.abs(dq).max()
    assert np.abs(cellpoly).max() <= 1e-8
