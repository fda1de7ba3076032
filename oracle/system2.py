"""Oracle: the second-order (k = 2) pressure system on the finest mesh
(Sec. 3.1-3.2 with the k = 2 DOFs of Sec. 3.1).  Level 0 only: no hierarchy
and no prolongation for k = 2 yet.

TEST INFRASTRUCTURE ONLY (never imported by the product path).

Global DOFs: the mesh vertices (canonical order), then one per mesh edge
(edges sorted by their (smaller, larger) vertex ids), one per mesh face (faces
sorted by their sorted vertex ids; a face shared by two cells is one DOF),
then one per cell.  Dirichlet p = 0 on y = 1 (the same boundary reading as
for k = 1) removes the vertices on that plane, the edges with both ends on it
and the faces with all vertices on it.
RHS (Sec. 3.2, Delta t = 1): r_i = sum_E int_E Pi_1 u' . grad Pi_2 phi_i,
with u' given at the vertices and Pi_1 u' its first-order projection per
component (the k = 1 element of the same cell), integrated with the cell
quadrature (degree 2, exact for this integrand).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .cutcell import build_cut_grid
from .geometry import EPS
from .hierarchy import build_hierarchy
from .mesh import build_meshes
from .vem import CellVEM
from .vem2 import CellVEM2, mono3, polyhedron_quadrature


class System2:
    pass


def build_system2(scene, G=None):
    S = System2()
    S.scene = scene
    S.G = G if G is not None else build_cut_grid(scene.N, scene.tris)
    M = build_meshes(S.G, build_hierarchy(S.G, 1))[0]
    S.mesh = M
    V = M.V
    nv = len(V)
    cycles = [[f[2] for f in cf] for cf in M.cell_faces]
    edges = sorted({(min(a, b), max(a, b)) for fs in cycles for cyc in fs
                    for a, b in zip(cyc, cyc[1:] + cyc[:1])})
    eid = {e: nv + i for i, e in enumerate(edges)}
    fkeys = sorted({tuple(sorted(cyc)) for fs in cycles for cyc in fs})
    fid = {k: nv + len(edges) + i for i, k in enumerate(fkeys)}
    base_c = nv + len(edges) + len(fkeys)
    S.n = base_c + len(cycles)
    S.nv, S.ne, S.nf = nv, len(edges), len(fkeys)
    S.cells, S.cells1, S.dofmap = [], [], []
    rows, cols, vals = [], [], []
    for c, (fs, vs) in enumerate(zip(cycles, M.cell_verts)):
        E = CellVEM2(V, fs, vs)
        dm = np.array(list(E.verts) + [eid[e] for e in E.edges] + [fid[tuple(sorted(f))] for f in fs]
                      + [base_c + c])
        S.cells.append(E)
        S.cells1.append(CellVEM(V, fs, vs))
        S.dofmap.append(dm)
        rows.append(np.repeat(dm, len(dm)))
        cols.append(np.tile(dm, len(dm)))
        vals.append(E.K.reshape(-1))
    S.K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                        shape=(S.n, S.n))
    on = np.abs(V[:, 1] - 1.0) <= EPS
    dirichlet = np.zeros(S.n, bool)
    dirichlet[:nv] = on
    for e, g in eid.items():
        dirichlet[g] = on[e[0]] and on[e[1]]
    for k, g in fid.items():
        dirichlet[g] = bool(on[list(k)].all())
    S.dirichlet = dirichlet
    S.free = np.nonzero(~dirichlet)[0]
    return S


def rhs2(S, u_vert):
    """r_i = sum_E int_E Pi_1 u' . grad Pi_2 phi_i over all global DOFs."""
    V = S.mesh.V
    r = np.zeros(S.n)
    for E, E1, dm in zip(S.cells, S.cells1, S.dofmap):
        s = E1.Pis @ u_vert[E1.verts]                 # (4, 3): Pi_1 u' per component
        qp, qw = polyhedron_quadrature(V, E._faces)
        Y = (qp - E1.xE) / E1.h
        u1 = s[0][None, :] + Y @ s[1:]                # (q, 3)
        _, g = mono3(qp, E.xE, E.hE)                  # (q, 10, 3)
        grad_phi = np.einsum("qad,ai->qid", g, E.Pis)  # (q, n_E, 3)
        r[dm] += np.einsum("q,qd,qid->i", qw, u1, grad_phi)
    return r


def dofs_of2(S, q):
    """Global DOF vector of a function q (callable on (n, 3) points)."""
    d = np.zeros(S.n)
    for E, dm in zip(S.cells, S.dofmap):
        d[dm] = E.dofs_of(q)
    return d


def solve2(S, u_vert):
    """Pressure DOFs of the k = 2 system (sparse direct solve; 0 on y = 1)."""
    r = rhs2(S, u_vert)
    f = S.free
    p = np.zeros(S.n)
    p[f] = spla.spsolve(S.K[f][:, f].tocsc(), r[f])
    return p
