"""Oracle: second-order (k = 2) conforming VEM on a polyhedral cell (Sec. 3.1,
Eq. 11-14, App. A).  Element level only (rows A2/A3 for k = 2): projector and
element matrix.  Assembly, prolongation and the right-hand side for k = 2 are
not written yet.

TEST INFRASTRUCTURE ONLY (never imported by the product path).

DOFs of a cell E (Sec. 3.1, the four DOF families for k = 2), in this order:
  vertex values (vertices in ascending global id), values at edge midpoints
  (the one interior point of the 3-point Gauss-Lobatto rule; edges sorted by
  their (smaller, larger) global vertex ids), face means (1/|f|) int_f v (faces
  in the given order), and the cell mean (1/|E|) int_E v.
Scaled monomials (App. A): m = prod_c ((x_c - x_E,c)/h_E)^{a_c}, |a| <= 2,
  N_2 = 10, x_E the centroid, h_E the largest vertex-vertex distance.
Projector (Eq. 14): G_ab = int_E grad m_a . grad m_b with the first row
  replaced by P0(m_b); B_ai = int_E grad phi_i . grad m_a with the first row
  P0(phi_i); P0 = cell mean for k >= 2 (Eq. 13), which is the cell DOF.
  By parts, int_E grad phi_i . grad m_a = -Delta m_a int_E phi_i
  + sum_f int_f phi_i (grad m_a . n_f): Delta m_a is a constant and
  int_E phi_i is |E| times the cell DOF; grad m_a . n_f is linear on f.
Face term (reading, enhanced face space): the moments of phi_i of order 1 on a
  face are those of its face projector Pi_{2,f} phi_i, the 2D analogue built
  from the face's DOFs (vertex values, edge-midpoint values and the face mean):
  G_f with first row P0_f = face mean, B_f by parts in 2D, with
  -Delta m int_f phi_i = -Delta m |f| (face DOF) and the boundary integrals of
  phi_i (quadratic along each edge) times the linear normal derivative, exact
  by Simpson's rule.
K^E = Pi*^T Gt Pi* + s_E (I - Pi)^T (I - Pi), Pi = D Pi*, D_ia = DOF_i(m_a),
  Gt = G with the first row zeroed, s_E = h_E (the same reading as for k = 1).
Integrals of polynomials: faces by a fan of triangles with the 7-point
  degree-5 rule, cells by a fan of tetrahedra (cell vertex mean as apex) with
  the 4-point degree-2 rule; both exact for the degrees used here.
"""
from __future__ import annotations

import numpy as np

# exponents of the 10 monomials of degree <= 2 in 3D and of the 6 in 2D
EXP3 = [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1), (2, 0, 0), (1, 1, 0), (1, 0, 1), (0, 2, 0), (0, 1, 1),
        (0, 0, 2)]
EXP2 = [(0, 0), (1, 0), (0, 1), (2, 0), (1, 1), (0, 2)]

# 7-point degree-5 triangle rule (Radon): barycentric points and weights
_A1, _B1 = (6.0 - np.sqrt(15.0)) / 21.0, (9.0 + 2.0 * np.sqrt(15.0)) / 21.0
_A2, _B2 = (6.0 + np.sqrt(15.0)) / 21.0, (9.0 - 2.0 * np.sqrt(15.0)) / 21.0
_W1, _W2 = (155.0 - np.sqrt(15.0)) / 1200.0, (155.0 + np.sqrt(15.0)) / 1200.0
TRI_BARY = np.array([[1 / 3, 1 / 3, 1 / 3],
                     [_A1, _A1, _B1], [_A1, _B1, _A1], [_B1, _A1, _A1],
                     [_A2, _A2, _B2], [_A2, _B2, _A2], [_B2, _A2, _A2]])
TRI_W = np.array([9.0 / 40.0, _W1, _W1, _W1, _W2, _W2, _W2])   # sum 1 (times the area)
# 4-point degree-2 tetrahedron rule
_TA, _TB = 0.5854101966249685, 0.1381966011250105
TET_BARY = np.array([[_TA, _TB, _TB, _TB], [_TB, _TA, _TB, _TB], [_TB, _TB, _TA, _TB], [_TB, _TB, _TB, _TA]])
TET_W = np.full(4, 0.25)


def polygon_quadrature(P):
    """Points and weights integrating polynomials of degree <= 5 exactly over
    the convex polygon with vertices P (fan from P[0])."""
    pts, wts = [], []
    for m in range(1, len(P) - 1):
        a, b, c = P[0], P[m], P[m + 1]
        area = 0.5 * np.linalg.norm(np.cross(b - a, c - a))
        pts.append(TRI_BARY @ np.array([a, b, c]))
        wts.append(TRI_W * area)
    return np.vstack(pts), np.concatenate(wts)


def polyhedron_quadrature(V, faces):
    """Points and weights integrating polynomials of degree <= 2 exactly over
    the convex polyhedron (fan of tetrahedra from the vertex mean)."""
    verts = sorted({v for f in faces for v in f})
    apex = V[verts].mean(axis=0)
    pts, wts = [], []
    for cyc in faces:
        for m in range(1, len(cyc) - 1):
            a, b, c = V[cyc[0]], V[cyc[m]], V[cyc[m + 1]]
            vol = abs(np.dot(np.cross(b - a, c - a), apex - a)) / 6.0
            pts.append(TET_BARY @ np.array([a, b, c, apex]))
            wts.append(TET_W * vol)
    return np.vstack(pts), np.concatenate(wts)


def mono3(X, xE, hE):
    """Values (n, 10) and gradients (n, 10, 3) of the scaled 3D monomials."""
    Y = (np.atleast_2d(X) - xE) / hE
    val = np.ones((len(Y), 10))
    grd = np.zeros((len(Y), 10, 3))
    for a, e in enumerate(EXP3):
        val[:, a] = Y[:, 0] ** e[0] * Y[:, 1] ** e[1] * Y[:, 2] ** e[2]
        for c in range(3):
            if e[c] == 0:
                continue
            ee = list(e)
            ee[c] -= 1
            grd[:, a, c] = e[c] * Y[:, 0] ** ee[0] * Y[:, 1] ** ee[1] * Y[:, 2] ** ee[2] / hE
    return val, grd


def laplacian3(hE):
    """Delta m_a of the scaled monomials (constants)."""
    return np.array([2.0 / hE ** 2 * sum(1 for c in range(3) if e[c] == 2) for e in EXP3])


class Face2:
    """A planar face with its k = 2 DOFs: cycle vertices, edge midpoints (edge m
    joins cycle[m] and cycle[m+1]) and the face mean; the 2D projector Pi_{2,f}."""

    def __init__(self, V, cyc):
        P = V[cyc]
        A = 0.5 * sum(np.cross(P[i], P[(i + 1) % len(P)]) for i in range(len(P)))
        self.area = float(np.linalg.norm(A))
        self.n = A / self.area
        self.qp, self.qw = polygon_quadrature(P)
        self.xf = (self.qw @ self.qp) / self.area
        t1 = P[1] - P[0]
        t1 = t1 - np.dot(t1, self.n) * self.n
        self.t1 = t1 / np.linalg.norm(t1)
        self.t2 = np.cross(self.n, self.t1)
        self.hf = max(np.linalg.norm(P[i] - P[j]) for i in range(len(P)) for j in range(i + 1, len(P)))
        k = len(cyc)
        self.k = k
        mids = 0.5 * (P + np.roll(P, -1, axis=0))
        # G_f
        mv, mg = self.mono2(self.qp)
        G = np.einsum("q,qad,qbd->ab", self.qw, mg, mg)
        G[0] = (self.qw @ mv) / self.area
        # B_f over local DOFs [k vertices, k midpoints, face mean]
        B = np.zeros((6, 2 * k + 1))
        B[0, 2 * k] = 1.0
        lap = np.array([2.0 / self.hf ** 2 * sum(1 for c in range(2) if e[c] == 2) for e in EXP2])
        B[:, 2 * k] += -lap * self.area
        B[0, 2 * k] = 1.0
        for m in range(k):
            a, b = P[m], P[(m + 1) % k]
            L = np.linalg.norm(b - a)
            ne = np.cross(b - a, self.n) / L          # outward in-plane normal (CCW cycle)
            for node, w, dof in ((a, 1.0 / 6.0, m), (mids[m], 4.0 / 6.0, k + m), (b, 1.0 / 6.0, (m + 1) % k)):
                _, g = self.mono2(node[None])
                dn = g[0] @ ne
                B[1:, dof] += L * w * dn[1:]
        self.Pis = np.linalg.solve(G, B)

    def local(self, X):
        Y = np.atleast_2d(X) - self.xf
        return np.stack([Y @ self.t1, Y @ self.t2], axis=1) / self.hf

    def mono2(self, X):
        """Values (n, 6) and 3D gradients (n, 6, 3) of the scaled face monomials."""
        Z = self.local(X)
        val = np.ones((len(Z), 6))
        grd = np.zeros((len(Z), 6, 3))
        T = np.stack([self.t1, self.t2]) / self.hf
        for a, e in enumerate(EXP2):
            val[:, a] = Z[:, 0] ** e[0] * Z[:, 1] ** e[1]
            d0 = e[0] * Z[:, 0] ** max(e[0] - 1, 0) * Z[:, 1] ** e[1] if e[0] else 0.0 * Z[:, 0]
            d1 = e[1] * Z[:, 0] ** e[0] * Z[:, 1] ** max(e[1] - 1, 0) if e[1] else 0.0 * Z[:, 0]
            grd[:, a] = np.outer(d0, T[0]) + np.outer(d1, T[1])
        return val, grd

    def moments(self, q_at_qp):
        """int_f (Pi_{2,f} phi_j) q for the local DOFs j, q given at the face
        quadrature points (q linear here, so the integrand has degree 3)."""
        mv, _ = self.mono2(self.qp)
        return (self.qw * q_at_qp) @ mv @ self.Pis


class CellVEM2:
    """k = 2 VEM element on a convex polyhedron given by its face cycles (CCW
    about the outward normal) and the global ids of its vertices."""

    def __init__(self, V, faces, verts):
        self.verts = sorted(verts)
        vloc = {v: i for i, v in enumerate(self.verts)}
        edges = sorted({(min(f[m], f[(m + 1) % len(f)]), max(f[m], f[(m + 1) % len(f)]))
                        for f in faces for m in range(len(f))})
        eloc = {e: i for i, e in enumerate(edges)}
        nv, ne, nf = len(self.verts), len(edges), len(faces)
        self.edges = edges
        self.n = nv + ne + nf + 1
        cdof = self.n - 1
        qp, qw = polyhedron_quadrature(V, faces)
        self.vol = float(qw.sum())
        self.xE = (qw @ qp) / self.vol
        X = V[self.verts]
        self.hE = max(np.linalg.norm(X[i] - X[j]) for i in range(nv) for j in range(i + 1, nv))
        mv, mg = mono3(qp, self.xE, self.hE)
        G = np.einsum("q,qad,qbd->ab", qw, mg, mg)
        self.Gt = G.copy()
        self.Gt[0] = 0.0
        G[0] = (qw @ mv) / self.vol
        # B: volume term, then faces by the enhanced face moments
        B = np.zeros((10, self.n))
        B[:, cdof] += -laplacian3(self.hE) * self.vol
        for fi, cyc in enumerate(faces):
            F = Face2(V, cyc)
            _, g = mono3(F.qp, self.xE, self.hE)
            dn = g @ F.n                                   # (q, 10): grad m_a . n_f
            for a in range(1, 10):
                mom = F.moments(dn[:, a])                  # local face DOFs
                k = F.k
                for m in range(k):
                    B[a, vloc[cyc[m]]] += mom[m]
                    e = (min(cyc[m], cyc[(m + 1) % k]), max(cyc[m], cyc[(m + 1) % k]))
                    B[a, nv + eloc[e]] += mom[k + m]
                B[a, nv + ne + fi] += mom[2 * k]
        B[0] = 0.0
        B[0, cdof] = 1.0
        self.G, self.B = G, B
        self.Pis = np.linalg.solve(G, B)
        # D: DOFs of the monomials
        D = np.zeros((self.n, 10))
        D[:nv] = mono3(X, self.xE, self.hE)[0]
        mids = np.array([0.5 * (V[a] + V[b]) for a, b in edges])
        D[nv:nv + ne] = mono3(mids, self.xE, self.hE)[0]
        for fi, cyc in enumerate(faces):
            F = Face2(V, cyc)
            D[nv + ne + fi] = (F.qw @ mono3(F.qp, self.xE, self.hE)[0]) / F.area
        D[cdof] = (qw @ mv) / self.vol
        self.D = D
        self.Pi = D @ self.Pis
        I = np.eye(self.n)
        self.K = self.Pis.T @ self.Gt @ self.Pis + self.hE * (I - self.Pi).T @ (I - self.Pi)
        self._faces = [list(f) for f in faces]
        self._V = V

    def dofs_of(self, q):
        """DOF vector of a function q (callable on (n, 3) points): vertex values,
        midpoint values, face means, cell mean (exact for polynomials of degree
        <= 5 on faces and <= 2 in the cell)."""
        V = self._V
        out = [q(V[self.verts])]
        out.append(q(np.array([0.5 * (V[a] + V[b]) for a, b in self.edges])))
        fm = []
        for cyc in self._faces:
            F = Face2(V, cyc)
            fm.append(float(F.qw @ q(F.qp)) / F.area)
        out.append(np.array(fm))
        qp, qw = polyhedron_quadrature(V, self._faces)
        out.append(np.array([float(qw @ q(qp)) / self.vol]))
        return np.concatenate(out)
