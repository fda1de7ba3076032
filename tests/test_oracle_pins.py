"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix
(closed forms, invariants, library special cases).  CPU only."""
import os

import numpy as np
import pytest
import scipy.sparse as sp

import scenes
from oracle.geometry import PlaneTable, winding_number
from oracle.multigrid import chebyshev, pcg, prolongation
from oracle.pipeline import dense_solve, dirichlet_mask, project, rhs_full
from oracle.vem import CellVEM

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ------------------------------------------------------------------ inputs

def test_splitmix64_published_vectors():
    vals = [l.strip() for l in open(os.path.join(GOLDEN, "splitmix64_seed0.txt"))
            if l.strip() and not l.startswith("#")]
    r = scenes.SplitMix64(0)
    assert [f"{r.next_u64():016x}" for _ in vals] == vals


def test_winding_number_inside_outside():
    tris = scenes.icosphere((0.5, 0.5, 0.5), 0.2, 2)
    assert abs(winding_number(tris, np.array([0.5, 0.5, 0.5])) - 1.0) < 1e-12
    assert abs(winding_number(tris, np.array([0.1, 0.9, 0.5]))) < 1e-12


# ------------------------------------------------------------------ geometry

def _faces(M, c):
    return [f[2] for f in M.cell_faces[c]]


def test_fluid_volume_equals_box_minus_obstacle(sphere8):
    M = sphere8.meshes[0]
    vol = sum(cv.vol for cv in sphere8.cells)
    assert abs(vol - (1.0 - scenes.mesh_volume(sphere8.scene.tris))) < 1e-10


def test_cells_convex_closed_euler(sphere8):
    for l, M in enumerate(sphere8.meshes):
        for c in range(len(M.cell_faces)):
            faces = _faces(M, c)
            verts = sorted({v for f in faces for v in f})
            edges = {tuple(sorted((f[i], f[(i + 1) % len(f)]))) for f in faces for i in range(len(f))}
            assert len(verts) - len(edges) + len(faces) == 2
            A = np.zeros(3)
            for f in faces:
                P = M.V[f]
                a = 0.5 * sum(np.cross(P[i], P[(i + 1) % len(f)]) for i in range(len(f)))
                A += a
                n = a / np.linalg.norm(a)
                s = (M.V[verts] - P[0]) @ n
                assert s.max() <= 1e-9            # convex: all vertices inside every face plane
            assert np.linalg.norm(A) < 1e-12      # closed surface: sum of vector areas vanishes


def test_interior_faces_match(sphere8):
    """Conformity: every face is either matched (same vertex cycle, reversed)
    by exactly one other cell, or lies on the boundary (box wall or obstacle)."""
    PT = PlaneTable(sphere8.scene.N, sphere8.scene.tris)
    for M in sphere8.meshes:
        seen = {}
        for c in range(len(M.cell_faces)):
            for (pid, sg, cyc) in M.cell_faces[c]:
                key = tuple(sorted(cyc))
                seen.setdefault(key, []).append((c, pid, sg, cyc))
        for key, lst in seen.items():
            assert len(lst) <= 2
            if len(lst) == 2:
                (c1, p1, s1, y1), (c2, p2, s2, y2) = lst
                assert p1 == p2 and s1 == -s2 and c1 != c2
                k = len(y1)
                i = y2.index(y1[0])
                assert [y2[(i - m) % k] for m in range(k)] == y1


def test_levels_nested_and_nonempty(sphere8):
    for l in range(len(sphere8.meshes) - 1):
        par = sphere8.meshes[l].parent
        assert len(par) == len(sphere8.meshes[l].cell_faces)
        assert set(par.tolist()) == set(range(len(sphere8.meshes[l + 1].cell_faces)))


# ------------------------------------------------------------------ VEM element

def _cube_cell(h, origin=(0.0, 0.0, 0.0)):
    o = np.array(origin)
    V = np.array([[i, j, k] for k in (0, 1) for j in (0, 1) for i in (0, 1)], dtype=float) * h + o
    idx = lambda i, j, k: i + 2 * j + 4 * k
    faces = [[idx(0, 0, 0), idx(0, 0, 1), idx(0, 1, 1), idx(0, 1, 0)],
             [idx(1, 0, 0), idx(1, 1, 0), idx(1, 1, 1), idx(1, 0, 1)],
             [idx(0, 0, 0), idx(1, 0, 0), idx(1, 0, 1), idx(0, 0, 1)],
             [idx(0, 1, 0), idx(0, 1, 1), idx(1, 1, 1), idx(1, 1, 0)],
             [idx(0, 0, 0), idx(0, 1, 0), idx(1, 1, 0), idx(1, 0, 0)],
             [idx(0, 0, 1), idx(1, 0, 1), idx(1, 1, 1), idx(0, 1, 1)]]
    return V, faces


def test_uncut_cube_consistency_closed_form():
    """On a cube the k=1 face space is bilinear, so grad Pi phi_i = s_i / (4h)
    and the consistency block is (h/16) s_i . s_j (s_i the corner sign vector)."""
    h = 0.37
    V, faces = _cube_cell(h)
    cv = CellVEM(V, faces, list(range(8)))
    s = np.sign(V - V.mean(axis=0))
    cons = cv.Pis.T @ cv.Gt @ cv.Pis
    assert np.allclose(cons, h / 16.0 * (s @ s.T), rtol=0, atol=1e-14)
    # scaling: K(h) = h K(1)
    V1, _ = _cube_cell(1.0)
    K1 = CellVEM(V1, faces, list(range(8))).K
    assert np.allclose(cv.K, h * K1, atol=1e-13)


def test_element_matrices_sym_psd_kernel(sphere8):
    for cv in sphere8.cells:
        K = cv.K
        assert np.allclose(K, K.T, atol=1e-14)
        ev = np.linalg.eigvalsh(K)
        assert ev[0] > -1e-13 * ev[-1]
        assert np.abs(K.sum(axis=1)).max() < 1e-12 * np.abs(K).max() + 1e-16
        assert (ev > 1e-10 * ev[-1]).sum() == len(ev) - 1       # rank n-1


def test_patch_test_every_cell(sphere8):
    """VEM is exact on P_1: with u' = grad q (q linear), K^E q = r^E."""
    g = np.array([0.3, -1.1, 0.7])
    V = sphere8.meshes[0].V
    for cv in sphere8.cells:
        q = V[cv.verts] @ g + 0.25
        u = np.tile(g, (len(cv.verts), 1))
        assert np.allclose(cv.K @ q, cv.rhs(u), atol=1e-13 * max(1.0, np.abs(cv.K).max()))
        assert np.allclose(cv.Pi @ q, q, atol=1e-13)


def test_global_patch_test_neumann_and_dirichlet(sphere8):
    S = sphere8
    V = S.meshes[0].V
    # pure Neumann: K 1 = 0 and p = q + const for u' = grad q
    assert np.abs(S.K @ np.ones(len(V))).max() < 1e-13
    g = np.array([0.5, 0.2, -0.4])
    r = rhs_full(S, np.tile(g, (len(V), 1)))
    q = V @ g
    assert np.abs(S.K @ q - r).max() < 1e-13
    # Dirichlet p = 0 at y = 1: q = c (y - 1) is reproduced exactly, u_new = 0
    u = np.tile(np.array([0.0, 0.8, 0.0]), (len(V), 1))
    p = dense_solve(S, u)
    assert np.abs(p - 0.8 * (V[:, 1] - 1.0)).max() < 1e-12
    _, cellpoly, _, _ = project(S, u, tol=1e-13)
    assert np.abs(cellpoly).max() < 1e-9


def test_global_K_symmetric(sphere8):
    K = sphere8.K
    assert abs(K - K.T).max() < 1e-15


# ------------------------------------------------------------------ multigrid

def test_prolongation_reproduces_linears(sphere8):
    for l, P in enumerate(sphere8.Pfull):
        Vf, Vc = sphere8.meshes[l].V, sphere8.meshes[l + 1].V
        for q in (lambda X: np.ones(len(X)), lambda X: X[:, 0], lambda X: X[:, 1],
                  lambda X: X[:, 2] - 0.3 * X[:, 0]):
            assert np.abs(P @ q(Vc) - q(Vf)).max() < 1e-12


def test_regular_aggregation_is_trilinear(empty4):
    """Uncut 2x2x2 aggregation: the diffusion-free P is trilinear interpolation
    (copy at corners, 1/2 at edge midpoints, 1/4 at face centres, 1/8 at the
    cube centre)."""
    Mf, Mc = empty4.meshes
    P = empty4.Pfull[0].toarray()
    for v in range(len(Mf.V)):
        x = Mf.V[v]
        w = np.array([np.prod(1.0 - np.abs(x - y) / 0.5) if np.all(np.abs(x - y) < 0.5 + 1e-12) else 0.0
                      for y in Mc.V])
        w[w < 0] = 0.0
        assert np.allclose(P[v], w, atol=1e-14)


def test_galerkin_is_diffusion_free(sphere8):
    """A_c(i,j) != 0 only if coarse DOFs i and j share a coarse cell (Sec. 4.3)."""
    S = sphere8
    for l in range(1, len(S.meshes)):
        free = S.free[l]
        pos = -np.ones(len(S.meshes[l].V), dtype=np.int64)
        pos[free] = np.arange(len(free))
        allowed = set()
        for vs in S.meshes[l].cell_verts:
            loc = [pos[v] for v in vs if pos[v] >= 0]
            allowed.update((a, b) for a in loc for b in loc)
        A = S.H.A[l].tocoo()
        nz = np.abs(A.data) > 0
        got = set(zip(A.row[nz].tolist(), A.col[nz].tolist()))
        assert got <= allowed


def test_coarse_constants_map_to_fine_constants(sphere8):
    for l, P in enumerate(sphere8.Pfull):
        assert np.allclose(P @ np.ones(P.shape[1]), 1.0, atol=1e-13)


def test_chebyshev_matches_closed_form_polynomial():
    """On a diagonal matrix the degree-d Chebyshev iteration from x0 = 0
    leaves error e_i = T_d((theta - l_i)/delta)/T_d(theta/delta) x*_i."""
    from numpy.polynomial import chebyshev as C
    lam = np.linspace(0.05, 2.0, 40)
    A = sp.diags(lam).tocsr()
    xs = np.cos(np.arange(40))
    b = lam * xs
    lmax = 2.2
    x = chebyshev(A, b, None, lmax, 5)
    beta, alpha = lmax, lmax / 30.0
    th, de = (beta + alpha) / 2, (beta - alpha) / 2
    Td = C.Chebyshev.basis(5)
    e = Td((th - lam) / de) / Td(th / de) * xs
    assert np.allclose(xs - x, e, atol=1e-13)


def test_fixed_cg_is_exact_after_n_distinct_eigenvalues():
    """CG terminates (in exact arithmetic) after as many steps as A has
    distinct eigenvalues; with 6 of them, 6 iterations give the solution."""
    from oracle.multigrid import fixed_cg
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    lam = np.repeat([0.5, 1.0, 2.0, 3.0, 5.0, 8.0], [7, 7, 7, 7, 6, 6])
    A = sp.csr_matrix((Q * lam) @ Q.T)
    b = rng.standard_normal(40)
    x = fixed_cg(A, b, 6)
    assert np.allclose(x, np.linalg.solve(A.toarray(), b), atol=1e-9)
    assert not np.allclose(fixed_cg(A, b, 3), x, atol=1e-3)


def test_lanczos_lmax_matches_dense_eigenvalue():
    """The Chebyshev upper bound is 1.1 x the largest eigenvalue (Lanczos)."""
    from oracle.multigrid import lanczos_lmax
    rng = np.random.default_rng(1)
    B = rng.standard_normal((200, 200))
    A = sp.csr_matrix(B @ B.T / 200 + np.eye(200))
    lam = np.linalg.eigvalsh(A.toarray())[-1]
    assert abs(lanczos_lmax(A) / 1.1 - lam) <= 1e-8 * lam


def test_pcg_matches_library_solve():
    rng = np.random.default_rng(0)
    B = rng.standard_normal((30, 30))
    A = sp.csr_matrix(B @ B.T + 30 * np.eye(30))
    b = rng.standard_normal(30)
    x, it, _ = pcg(A, b, lambda r: r / A.diagonal(), 1e-13)
    assert np.allclose(x, np.linalg.solve(A.toarray(), b), atol=1e-10)


def test_mgpcg_matches_dense_direct(sphere8):
    S = sphere8
    u = S.scene.velocity(S.meshes[0].V)
    p, _, it, hist = project(S, u, tol=1e-10)
    pd = dense_solve(S, u)
    assert np.linalg.norm(p - pd) / np.linalg.norm(pd) < 1e-9
    assert hist[-1] <= 1e-10 and it < 40


def test_dirichlet_rows_removed(sphere8):
    V = sphere8.meshes[0].V
    d = dirichlet_mask(V)
    assert d.sum() > 0
    assert not np.any(np.isin(np.nonzero(d)[0], sphere8.free[0]))


def _q(V):
    """Smooth pressure that vanishes on the Dirichlet plane y = 1."""
    x, y, z = V[:, 0], V[:, 1], V[:, 2]
    return np.cos(np.pi * x) * np.cos(np.pi * z) * np.sin(0.5 * np.pi * (1 - y))


def _grad_q(V):
    x, y, z = V[:, 0], V[:, 1], V[:, 2]
    a, b, c = np.cos(np.pi * x), np.sin(0.5 * np.pi * (1 - y)), np.cos(np.pi * z)
    return np.stack([-np.pi * np.sin(np.pi * x) * b * c,
                     -0.5 * np.pi * a * np.cos(0.5 * np.pi * (1 - y)) * c,
                     -np.pi * a * b * np.sin(np.pi * z)], axis=1)


@pytest.mark.slow
def test_second_order_convergence_to_manufactured_pressure(sphere8):
    """With u' = grad q and q = 0 on y = 1, the weak problem of Sec. 3.2
    (int grad p . grad phi = int u' . grad phi, Neumann elsewhere) has p = q.
    The first-order VEM pressure then converges at second order at the
    vertices: the observed order from 8^3 to 16^3 is about 2 on the empty box
    and with the sphere's cut cells (a dropped RHS term, a wrong sign or a
    wrong stabilisation scale breaks it)."""
    from oracle.pipeline import build_system, project
    # one level suffices here: the projection's solve is checked elsewhere
    cases = {"empty": [build_system(scenes.empty_scene(8), L=1), build_system(scenes.empty_scene(16), L=1)],
             "sphere": [sphere8, build_system(scenes.config(0, 16), L=1)]}
    for name, systems in cases.items():
        err = []
        for S in systems:
            V = S.meshes[0].V
            p, _, _, _ = project(S, _grad_q(V), 0.0, tol=1e-12)
            e = p - _q(V)
            err.append((np.abs(e).max(), np.sqrt(np.mean(e ** 2))))
        for k in range(2):
            order = np.log2(err[0][k] / err[1][k])
            assert 1.8 <= order <= 2.3, (name, k, order)
