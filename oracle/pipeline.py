"""Oracle: the whole pressure projection, end to end (Alg. 1 precompute + the
"VEM-based pressure projection" step).

TEST INFRASTRUCTURE ONLY: only tests, the smoke check and the benchmark's CPU
baseline may import this package.

Boundary conditions (reading): Neumann (no-through-flow) on the box walls and
the obstacles, Dirichlet p = 0 on the top face y = 1 (the paper's buoyancy
axis is y); all pressure DOFs on that face are removed.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .cutcell import build_cut_grid
from .geometry import EPS
from .hierarchy import build_hierarchy
from .mesh import build_meshes
from .multigrid import Hierarchy, pcg, prolongation
from .vem import CellVEM


class OracleSystem:
    pass


def dirichlet_mask(V):
    return np.abs(V[:, 1] - 1.0) <= EPS


def assemble_K(M, cells):
    n = len(M.V)
    rows, cols, vals = [], [], []
    for cv in cells:
        g = np.array(cv.verts)
        rows.append(np.repeat(g, len(g)))
        cols.append(np.tile(g, len(g)))
        vals.append(cv.K.reshape(-1))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def build_system(scene, L=5, G=None, balance=True, naive_prolongation=False):
    """Cut grid, hierarchy, level meshes, level-0 elements and operator, and
    the multigrid hierarchy; naive_prolongation: Eq. 16 (the "Ours^np"
    ablation) instead of the diffusion-free Eq. 17."""
    S = OracleSystem()
    S.scene = scene
    S.G = G if G is not None else build_cut_grid(scene.N, scene.tris)
    S.levels = build_hierarchy(S.G, L, balance)
    S.meshes = build_meshes(S.G, S.levels)
    M0 = S.meshes[0]
    S.cells = [CellVEM(M0.V, [f[2] for f in cf], vs)
               for cf, vs in zip(M0.cell_faces, M0.cell_verts)]
    S.K = assemble_K(M0, S.cells)
    # free DOFs per level
    S.free = []
    S.Pfull = []
    dir0 = dirichlet_mask(M0.V)
    S.free.append(np.nonzero(~dir0)[0])
    for l in range(L - 1):
        P = prolongation(S.meshes[l], S.meshes[l + 1], naive=naive_prolongation)
        S.Pfull.append(P)
        Pc = P.tocsc()
        nonempty = np.diff(Pc.indptr) > 0
        dirc = dirichlet_mask(S.meshes[l + 1].V)
        S.free.append(np.nonzero(nonempty & ~dirc)[0])
    Ps = [S.Pfull[l][S.free[l]][:, S.free[l + 1]] for l in range(L - 1)]
    A0 = S.K[S.free[0]][:, S.free[0]].tocsr()
    S.H = Hierarchy(A0, Ps)
    return S


def rhs_full(S, u_vert, u_inflow=0.0):
    M0 = S.meshes[0]
    r = np.zeros(len(M0.V))
    for cv in S.cells:
        r[cv.verts] += cv.rhs(u_vert[cv.verts])
    if u_inflow != 0.0:
        # inflow face x = 0: grid plane id 0 with outward sign -1
        from .vem import face_phi_integrals
        for cf in M0.cell_faces:
            for (pid, sg, cyc) in cf:
                if pid == 0 and sg < 0:
                    r[cyc] += u_inflow * face_phi_integrals(M0.V, cyc)
    return r


def project(S, u_vert, u_inflow=0.0, tol=None, max_iters=500):
    tol = S.scene.tol if tol is None else tol
    r = rhs_full(S, u_vert, u_inflow)
    b = r[S.free[0]]
    A = S.H.A[0]
    pf, iters, hist = pcg(A, b, S.H.vcycle, tol, max_iters)
    p = np.zeros(len(S.meshes[0].V))
    p[S.free[0]] = pf
    cellpoly = np.array([cv.correct(u_vert[cv.verts], p[cv.verts]) for cv in S.cells])
    return p, cellpoly, iters, hist


def dense_solve(S, u_vert, u_inflow=0.0):
    r = rhs_full(S, u_vert, u_inflow)
    A = S.H.A[0].toarray()
    p = np.zeros(len(S.meshes[0].V))
    p[S.free[0]] = np.linalg.solve(A, r[S.free[0]])
    return p


def operators(S, u_inflow=1.0):
    """Explicit sparse matrices of the affine map u' -> cellpoly (Sec. 3.2-3.3):
    R (free x 3nv, SoA columns), b_in (free), C_u (12nc x 3nv), C_p (12nc x nv)."""
    M0 = S.meshes[0]
    nv, nc = len(M0.V), len(S.cells)
    free = S.free[0]
    pos = -np.ones(nv, dtype=np.int64)
    pos[free] = np.arange(len(free))
    Rr, Rc, Rv, Ur, Uc, Uv, Pr, Pc, Pv = [], [], [], [], [], [], [], [], []
    for e, cv in enumerate(S.cells):
        n = len(cv.verts)
        g = cv.grad_coeffs()                    # (3, n)
        for c in range(3):
            # r_i = sum_c g[c,i] |E| s^c_1,  s^c_1 = Pis[0] . u_c
            for i in range(n):
                if pos[cv.verts[i]] < 0:
                    continue
                for j in range(n):
                    Rr.append(pos[cv.verts[i]]); Rc.append(c * nv + cv.verts[j])
                    Rv.append(g[c, i] * cv.vol * cv.Pis[0, j])
            for a in range(4):
                for j in range(n):
                    Ur.append(12 * e + 4 * c + a); Uc.append(c * nv + cv.verts[j]); Uv.append(cv.Pis[a, j])
            for j in range(n):
                Pr.append(12 * e + 4 * c); Pc.append(cv.verts[j]); Pv.append(-g[c, j])
    R = sp.csr_matrix((Rv, (Rr, Rc)), shape=(len(free), 3 * nv))
    Cu = sp.csr_matrix((Uv, (Ur, Uc)), shape=(12 * nc, 3 * nv))
    Cp = sp.csr_matrix((Pv, (Pr, Pc)), shape=(12 * nc, nv))
    b_in = rhs_full(S, np.zeros((nv, 3)), 1.0)[free]
    return R, b_in, Cu, Cp


def dense_adjoint(S, g):
    """J^T g of the projection by a dense solve: returns (g_u (3,nv) SoA, g_inflow)."""
    R, b_in, Cu, Cp = operators(S)
    free = S.free[0]
    A = S.H.A[0].toarray()
    lam = np.linalg.solve(A, (Cp[:, free].T @ g))
    gu = Cu.T @ g + R.T @ lam
    return gu.reshape(3, -1), float(b_in @ lam)
