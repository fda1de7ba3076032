"""Oracle: first-order conforming VEM on a polyhedral cell (Sec. 3.1-3.3, App. A).

TEST INFRASTRUCTURE ONLY (never imported by the product path).

Per cell E with vertices x_i (local order = ascending global id):
  scaled monomials m_1 = 1, m_{1+c} = (x_c - x_E,c)/h_E (App. A; x_E the
  centroid, h_E the largest vertex-vertex distance);
  G_ab = int_E grad m_a . grad m_b, first row replaced by P0(m_b) (Eq. 14);
  B_ai = int_E grad phi_i . grad m_a = sum_f int_f phi_i (grad m_a . n_f)
         (integration by parts; Delta m_a = 0 for k = 1), first row P0(phi_i);
         P0 = mean of the vertex values (Eq. 13, k = 1);
  int_f phi_i = int_f Pi_{1,f} phi_i (enhanced face space; reading), with the
         2D projector of the face polygon: Pi_{1,f} phi_i = 1/n_f + g_i.(x - xbar_f),
         g_i = (1/|f|) int_{df} phi_i n ds, xbar_f the face vertex mean;
  Pi* = G^{-1} B (coefficients), Pi = D Pi* with D_ia = m_a(x_i);
  K^E = Pi*^T Gt Pi* + s_E (I - Pi)^T (I - Pi)  (Sec. 3.1, the dofi-dofi
         stabilisation), Gt = G with the first row zeroed, s_E = h_E (reading:
         the 3D scaling of int |grad phi|^2; the printed sum has no factor).
RHS (Sec. 3.2): r_i = sum_E int_E Pi_1 u' . grad Pi_1 phi_i  (Delta t = 1),
       u' the vertex interpolant, Pi_1 per component; inflow on x = 0:
       r_i += U_in int_{Gamma_in} phi_i  (from dp/dn = (u' - u_b).n, u_b = U_in e_x).
Correction (Sec. 3.3): Pi_1 u_new = Pi_1 u' - grad Pi_1 p, 12 coefficients per
       cell, layout [component c][monomial a].
"""
from __future__ import annotations

import numpy as np

STAB_SCALE = "h"          # s_E = h_E


def face_geometry(V, cyc):
    """Area, unit normal (from the CCW cycle), area centroid, vertex mean."""
    P = V[cyc]
    A = np.zeros(3)
    for i in range(len(cyc)):
        A = A + np.cross(P[i], P[(i + 1) % len(cyc)])
    A = 0.5 * A
    area = float(np.linalg.norm(A))
    n = A / area
    cen = np.zeros(3)
    tot = 0.0
    for m in range(1, len(cyc) - 1):
        a = 0.5 * float(np.dot(np.cross(P[m] - P[0], P[m + 1] - P[0]), n))
        cen += a * (P[0] + P[m] + P[m + 1]) / 3.0
        tot += a
    cen /= tot
    return area, n, cen, P.mean(axis=0)


def face_phi_integrals(V, cyc):
    """int_f phi_j for the vertices of a face (k = 1 enhanced face space)."""
    area, n, cen, xbar = face_geometry(V, cyc)
    k = len(cyc)
    out = np.zeros(k)
    for m in range(k):
        g = np.cross(V[cyc[(m + 1) % k]] - V[cyc[m - 1]], n) / (2.0 * area)
        out[m] = area * (1.0 / k + float(np.dot(g, cen - xbar)))
    return out


def face_projector_weights(V, cyc, x):
    """Pi_{1,f} phi_j evaluated at x, for the vertices of the face cycle."""
    area, n, cen, xbar = face_geometry(V, cyc)
    k = len(cyc)
    w = np.zeros(k)
    for m in range(k):
        g = np.cross(V[cyc[(m + 1) % k]] - V[cyc[m - 1]], n) / (2.0 * area)
        w[m] = 1.0 / k + float(np.dot(g, x - xbar))
    return w


def cell_volume_centroid(V, faces):
    verts = sorted({v for f in faces for v in f})
    c0 = V[verts].mean(axis=0)
    vol = 0.0
    cen = np.zeros(3)
    for cyc in faces:
        a = V[cyc[0]]
        for m in range(1, len(cyc) - 1):
            b, c = V[cyc[m]], V[cyc[m + 1]]
            t = float(np.dot(a - c0, np.cross(b - c0, c - c0))) / 6.0
            vol += t
            cen += t * (c0 + a + b + c) / 4.0
    return vol, cen / vol


class CellVEM:
    """Local k = 1 VEM quantities of one cell."""

    def __init__(self, V, faces, verts):
        self.verts = list(verts)
        loc = {g: i for i, g in enumerate(self.verts)}
        nv = len(self.verts)
        X = V[self.verts]
        self.vol, self.xE = cell_volume_centroid(V, faces)
        d = X[:, None, :] - X[None, :, :]
        self.h = float(np.sqrt((d * d).sum(-1)).max())
        h, vol = self.h, self.vol
        # monomials at the vertices: D_ia = m_a(x_i)
        D = np.ones((nv, 4))
        D[:, 1:] = (X - self.xE) / h
        self.D = D
        # G: int grad m_a . grad m_b ; grad m_{1+c} = e_c / h
        G = np.zeros((4, 4))
        G[1:, 1:] = np.eye(3) * vol / h ** 2
        Gt = G.copy()
        G[0, :] = D.mean(axis=0)             # P0(m_b) = mean of vertex values
        # B: boundary integrals
        B = np.zeros((4, nv))
        B[0, :] = 1.0 / nv                    # P0(phi_i)
        self.face_int = []
        for cyc in faces:
            area, n, _, _ = face_geometry(V, cyc)
            fi = face_phi_integrals(V, cyc)
            self.face_int.append(fi)
            for m, g in enumerate(cyc):
                B[1:, loc[g]] += n / h * fi[m]
        self.G, self.Gt, self.B = G, Gt, B
        self.Pis = np.linalg.solve(G, B)      # Pi* (4 x nv)
        self.Pi = D @ self.Pis                # Pi (nv x nv)
        s = h if STAB_SCALE == "h" else 1.0
        I = np.eye(nv)
        self.K = self.Pis.T @ Gt @ self.Pis + s * (I - self.Pi).T @ (I - self.Pi)
        # int_E m_a (first moments; exact for linear monomials)
        self.mom1 = np.array([vol, 0.0, 0.0, 0.0])

    def grad_coeffs(self):
        """Constant gradient of Pi_1 phi_i: (3 x nv)."""
        return self.Pis[1:, :] / self.h

    def rhs(self, u_loc):
        """Local r_i = int_E Pi_1 u' . grad Pi_1 phi_i ; u_loc (nv,3)."""
        s = self.Pis @ u_loc                  # (4,3): coefficients per component
        mean_u = (self.mom1 @ s)              # int_E Pi_1 u'_c (3,)
        return self.grad_coeffs().T @ mean_u

    def velocity_coeffs(self, u_loc):
        """Pi_1 u' coefficients, (3,4) [component][monomial]."""
        return (self.Pis @ u_loc).T

    def correct(self, u_loc, p_loc):
        c = self.velocity_coeffs(u_loc).copy()
        gp = self.grad_coeffs() @ p_loc       # (3,)
        c[:, 0] -= gp
        return c


def mass_moments(V, faces, xE, h):
    """int_E m_a m_b for k = 1 monomials (4x4), from second moments computed on
    the fan tetrahedra (exact quadrature for quadratics: vertices + centroid)."""
    M = np.zeros((4, 4))
    verts = sorted({v for f in faces for v in f})
    c0 = V[verts].mean(axis=0)
    for cyc in faces:
        a = V[cyc[0]]
        for m in range(1, len(cyc) - 1):
            b, c = V[cyc[m]], V[cyc[m + 1]]
            vol = float(np.dot(a - c0, np.cross(b - c0, c - c0))) / 6.0
            P = np.array([c0, a, b, c])
            # exact for degree 2 on a tetrahedron: int q = vol/20 * (sum q(v_i) + 16 q(centroid))
            # (the Keast/Stroud 5-point rule is used instead for clarity:)
            pts, wts = _tet_rule(P)
            for x, wgt in zip(pts, wts):
                mv = np.array([1.0, *((x - xE) / h)])
                M += vol * wgt * np.outer(mv, mv)
    return M


def _tet_rule(P):
    """Degree-2 exact rule on a tetrahedron: 4 points with barycentric
    (a,b,b,b), a = 0.5854101966249685, b = 0.1381966011250105, weights 1/4."""
    a, b = 0.5854101966249685, 0.1381966011250105
    pts = []
    for i in range(4):
        lam = np.full(4, b)
        lam[i] = a
        pts.append(lam @ P)
    return pts, [0.25] * 4
