"""Oracle: the second-order (k = 2) pressure system (Sec. 3.1-3.2 with the
k = 2 DOFs of Sec. 3.1) on the finest mesh, and its multigrid hierarchy
(Sec. 4: diffusion-free prolongation extended to the k = 2 DOFs, Galerkin
coarse operators, the same Chebyshev / coarsest-CG V-cycle as for k = 1).

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
from .vem2 import EXP3, CellVEM2, mono3, polyhedron_quadrature


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


# ---------------------------------------------------------------- multilevel (Sec. 4)

class Level2:
    pass


def level2(M, elements=True):
    """k = 2 DOFs, elements and assembled K of one level mesh (with
    elements=False: the DOF numbering, element DOF lists and Dirichlet mask
    only)."""
    Lv = Level2()
    Lv.mesh = M
    V = M.V
    nv = len(V)
    cycles = [[f[2] for f in cf] for cf in M.cell_faces]
    edges = sorted({(min(a, b), max(a, b)) for fs in cycles for cyc in fs
                    for a, b in zip(cyc, cyc[1:] + cyc[:1])})
    Lv.eid = {e: nv + i for i, e in enumerate(edges)}
    fk = {}
    for fs in cycles:
        for cyc in fs:
            fk.setdefault(tuple(sorted(cyc)), cyc)
    keys = sorted(fk)
    Lv.fid = {k: nv + len(edges) + i for i, k in enumerate(keys)}
    Lv.fcyc = fk
    base_c = nv + len(edges) + len(keys)
    Lv.cdof = base_c
    Lv.n = base_c + len(cycles)
    Lv.nv, Lv.ne, Lv.nf = nv, len(edges), len(keys)
    Lv.cycles = cycles
    Lv.cells, Lv.dofmap = [], []
    rows, cols, vals = [], [], []
    for c, (fs, vs) in enumerate(zip(cycles, M.cell_verts)):
        es = sorted({(min(f[m], f[(m + 1) % len(f)]), max(f[m], f[(m + 1) % len(f)]))
                     for f in fs for m in range(len(f))})
        dm = np.array(sorted(vs) + [Lv.eid[e] for e in es] + [Lv.fid[tuple(sorted(f))] for f in fs] + [base_c + c])
        Lv.dofmap.append(dm)
        if not elements:
            continue
        E = CellVEM2(V, fs, vs)
        Lv.cells.append(E)
        rows.append(np.repeat(dm, len(dm)))
        cols.append(np.tile(dm, len(dm)))
        vals.append(E.K.reshape(-1))
    if elements:
        Lv.K = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                             shape=(Lv.n, Lv.n))
    on = np.abs(V[:, 1] - 1.0) <= EPS
    dirichlet = np.zeros(Lv.n, bool)
    dirichlet[:nv] = on
    for e, g in Lv.eid.items():
        dirichlet[g] = on[e[0]] and on[e[1]]
    for k, g in Lv.fid.items():
        dirichlet[g] = bool(on[list(k)].all())
    Lv.dirichlet = dirichlet
    return Lv


def prolongation2(Lf, Lc, naive=False):
    """Diffusion-free prolongation for k = 2 (Sec. 4.3, Eq. 17, extended to the
    k = 2 DOFs): point DOFs of the fine level (vertices, edge midpoints) take
    the coarse function at their placement (coarse vertex: copy; coarse edge:
    the quadratic through that edge's DOFs; coarse face: Pi_{2,F}; coarse cell:
    Pi_2); mean DOFs (fine faces, fine cells) take the mean over the fine
    entity of the coarse face or cell polynomial that holds it.

    naive: the naive prolongation of Eq. 16 (Sec. 4.2): fine vertices on
    coarse vertices copy them (the shared vertex DOFs); every other fine DOF
    is that functional of the parent cell's Pi_2 polynomial."""
    from .multigrid import classify_vertex
    from .vem2 import Face2
    Mf, Mc = Lf.mesh, Lc.mesh
    Vf, Vc = Mf.V, Mc.V
    face_cache = {}

    def cface(cyc):
        # keyed by the oriented cycle: the projector's columns follow its order
        k = tuple(cyc)
        if k not in face_cache:
            face_cache[k] = Face2(Vc, list(cyc))
        return face_cache[k]

    def face_dofs(cyc):
        k = len(cyc)
        return ([cyc[m] for m in range(k)]
                + [Lc.eid[(min(cyc[m], cyc[(m + 1) % k]), max(cyc[m], cyc[(m + 1) % k]))] for m in range(k)]
                + [Lc.fid[tuple(sorted(cyc))]])

    def at_point(x, C):
        cf = Lc.cycles[C]
        pl = classify_vertex(Vc, cf, x)
        if pl[0] == "vertex":
            return [(pl[1], 1.0)]
        if naive:
            pl = ("cell",)
        if pl[0] == "edge":
            _, a, b, t = pl
            mid = Lc.eid[(min(a, b), max(a, b))]
            return [(a, (1 - t) * (1 - 2 * t)), (mid, 4 * t * (1 - t)), (b, t * (2 * t - 1))]
        if pl[0] == "face":
            F = cface(pl[1])
            w = F.mono2(x[None])[0][0] @ F.Pis
            return list(zip(face_dofs(pl[1]), w))
        E = Lc.cells[C]
        w = mono3(x[None], E.xE, E.hE)[0][0] @ E.Pis
        return list(zip(Lc.dofmap[C], w))

    # a fine cell holding each fine vertex, edge and face
    vcell = {}
    ecell, fcell = {}, {}
    for c, fs in enumerate(Lf.cycles):
        for cyc in fs:
            fcell.setdefault(tuple(sorted(cyc)), c)
            for a, b in zip(cyc, cyc[1:] + cyc[:1]):
                vcell.setdefault(a, c)
                ecell.setdefault((min(a, b), max(a, b)), c)
    rows, cols, vals = [], [], []

    def put(i, ent):
        for j, w in ent:
            rows.append(i)
            cols.append(j)
            vals.append(w)

    for v in range(Lf.nv):
        put(v, at_point(Vf[v], int(Mf.parent[vcell[v]])))
    for e, g in Lf.eid.items():
        put(g, at_point(0.5 * (Vf[e[0]] + Vf[e[1]]), int(Mf.parent[ecell[e]])))
    for k, g in Lf.fid.items():
        C = int(Mf.parent[fcell[k]])
        Ff = Face2(Vf, list(Lf.fcyc[k]))
        pl = classify_vertex(Vc, Lc.cycles[C], Ff.xf)
        if pl[0] == "face" and not naive:
            F = cface(pl[1])
            w = (Ff.qw @ F.mono2(Ff.qp)[0]) @ F.Pis / Ff.area
            put(g, zip(face_dofs(pl[1]), w))
        else:
            E = Lc.cells[C]
            w = (Ff.qw @ mono3(Ff.qp, E.xE, E.hE)[0]) @ E.Pis / Ff.area
            put(g, zip(Lc.dofmap[C], w))
    for c, E in enumerate(Lf.cells):
        C = int(Mf.parent[c])
        Ec = Lc.cells[C]
        qp, qw = polyhedron_quadrature(Vf, E._faces)
        w = (qw @ mono3(qp, Ec.xE, Ec.hE)[0]) @ Ec.Pis / E.vol
        put(Lf.cdof + c, zip(Lc.dofmap[C], w))
    return sp.csr_matrix((vals, (rows, cols)), shape=(Lf.n, Lc.n))


def build_hierarchy2(scene, L=3, G=None, naive_prolongation=False):
    """k = 2 levels, prolongations and the free-DOF multigrid hierarchy;
    naive_prolongation: Eq. 16 instead of Eq. 17."""
    from .multigrid import Hierarchy
    S = System2()
    S.scene = scene
    S.G = G if G is not None else build_cut_grid(scene.N, scene.tris)
    meshes = build_meshes(S.G, build_hierarchy(S.G, L))
    S.levels = [level2(M) for M in meshes]
    S.Pfull = [prolongation2(S.levels[l], S.levels[l + 1], naive_prolongation) for l in range(L - 1)]
    S.free = [np.nonzero(~S.levels[0].dirichlet)[0]]
    for l in range(L - 1):
        nonempty = np.diff(S.Pfull[l].tocsc().indptr) > 0
        S.free.append(np.nonzero(nonempty & ~S.levels[l + 1].dirichlet)[0])
    Ps = [S.Pfull[l][S.free[l]][:, S.free[l + 1]] for l in range(L - 1)]
    L0 = S.levels[0]
    S.H = Hierarchy(L0.K[S.free[0]][:, S.free[0]].tocsr(), Ps)
    S.Hs = ScaledVcycle(S.H)
    condense(S)
    # finest-level views used by rhs2 / project2
    S.mesh, S.n, S.cells, S.dofmap = L0.mesh, L0.n, L0.cells, L0.dofmap
    S.cells1 = [CellVEM(L0.mesh.V, fs, vs) for fs, vs in zip(L0.cycles, L0.mesh.cell_verts)]
    return S


def correction2(S, u_vert, p):
    """Sec. 3.3 for k = 2: Pi_1 u_new = Pi_1 u' - grad Pi_2 p per cell.  grad Pi_2 p
    is linear, so the result keeps the k = 1 layout: 12 coefficients per cell,
    [component c][monomial a] in the monomials 1, (x_d - x_E,d)/h_E."""
    out = np.zeros((len(S.cells), 3, 4))
    for c, (E, E1, dm) in enumerate(zip(S.cells, S.cells1, S.dofmap)):
        coef = E.Pis @ p[dm]                          # Pi_2 p in the k = 2 monomials
        g = np.zeros((3, 4))                          # grad in (1, Y_1, Y_2, Y_3), Y = (x - x_E)/h_E
        for a, e in enumerate(EXP3):
            for d in range(3):
                if e[d] == 0:
                    continue
                rest = list(e)
                rest[d] -= 1
                if sum(rest) == 0:
                    g[d, 0] += coef[a] * e[d] / E.hE
                else:
                    g[d, 1 + rest.index(1)] += coef[a] * e[d] / E.hE
        assert np.allclose(E1.xE, E.xE, atol=1e-13) and abs(E1.h - E.hE) <= 1e-13
        out[c] = E1.velocity_coeffs(u_vert[E1.verts]) - g
    return out


def project2(S, u_vert, tol=1e-10, max_iters=500):
    """k = 2 projection: RHS; multigrid PCG on the condensed system (reading K2,
    scaled V-cycle K1), then the cell DOFs from their cells; correction.
    Returns (p over all level-0 DOFs, cell coefficients, iters)."""
    from .multigrid import pcg
    r = rhs2(S, u_vert)
    rb = r[S.b0] - S.Kbc0 @ (S.dinv0 * r[S.c0])
    xb, its, _ = pcg(S.S0, rb, S.Hc, tol, max_iters)
    p = np.zeros(S.n)
    p[S.b0] = xb
    p[S.c0] = S.dinv0 * (r[S.c0] - S.Kbc0.T @ xb)
    return p, correction2(S, u_vert, p), its


def _split_cells(Lv, free):
    f = np.asarray(free)
    return f[f < Lv.cdof], f[f >= Lv.cdof]


def _schur(K, b, c):
    """K_bb - K_bc K_cc^-1 K_cb with K_cc diagonal (a cell DOF couples only
    within its own cell, and each cell has one)."""
    Kbc = K[b][:, c].tocsr()
    dinv = 1.0 / K[c][:, c].diagonal()
    return (K[b][:, b] - Kbc @ sp.diags(dinv) @ Kbc.T).tocsr(), Kbc, dinv


def condense(S):
    """Reading K2 for k = 2: static condensation of the cell-mean DOFs.  Level 0
    solves the Schur complement on its other free DOFs; each coarse level's
    cell DOFs follow their boundary DOFs by the discrete harmonic extension of
    that level's K, so the prolongation of the condensed system is
    P_b [I; -K_cc^-1 K_cb].  Multigrid on the condensed system uses the scaled
    V-cycle (reading K1)."""
    from .multigrid import Hierarchy
    Ls = S.levels
    S.b0, S.c0 = _split_cells(Ls[0], S.free[0])
    S.S0, S.Kbc0, S.dinv0 = _schur(Ls[0].K, S.b0, S.c0)
    Ps = []
    for l in range(len(Ls) - 1):
        bf, _ = _split_cells(Ls[l], S.free[l])
        bc, cc = _split_cells(Ls[l + 1], S.free[l + 1])
        _, Kbc, dinv = _schur(Ls[l + 1].K, bc, cc)
        E = sp.vstack([sp.identity(len(bc)), -sp.diags(dinv) @ Kbc.T]).tocsr()
        Ps.append((S.Pfull[l][bf][:, np.concatenate([bc, cc])] @ E).tocsr())
    S.Hc = ScaledVcycle(Hierarchy(S.S0, Ps))


class ScaledVcycle:
    """Reading for k = 2: Chebyshev smoothing of every level scaled by that
    level's diagonal.  The k = 2 operators are badly scaled (vertex, edge,
    face and cell DOFs; diagonals spanning several orders of magnitude), and
    the unscaled smoother needs 26 CG iterations on the empty 8^3 box against
    14 scaled (Table 4: 7-16).  Level l uses A'_l = D_l^-1/2 A_l D_l^-1/2 and
    P'_l = D_l^1/2 P_l D_{l+1}^-1/2, which keeps A'_{l+1} = P'_l^T A'_l P'_l;
    as a preconditioner of the unscaled system, M r = D_0^-1/2 V'(D_0^-1/2 r)."""

    def __init__(self, H):
        from .multigrid import Hierarchy
        d = [A.diagonal() for A in H.A]
        Pp = [(sp.diags(np.sqrt(d[l])) @ H.P[l] @ sp.diags(1.0 / np.sqrt(d[l + 1]))).tocsr()
              for l in range(len(H.P))]
        A0 = (sp.diags(1.0 / np.sqrt(d[0])) @ H.A[0] @ sp.diags(1.0 / np.sqrt(d[0]))).tocsr()
        self.H = Hierarchy(A0, Pp)
        self.s0 = 1.0 / np.sqrt(d[0])

    def __call__(self, r):
        return self.s0 * self.H.vcycle(self.s0 * r)
