"""Oracle: diffusion-free prolongation, Galerkin operators, Chebyshev smoother,
V-cycle and multigrid-preconditioned CG (Sec. 4; Eq. 15, Eq. 17).

TEST INFRASTRUCTURE ONLY (never imported by the product path).

Prolongation (k = 1) -- each fine vertex is placed relative to the *coarse*
topology (reading of Eq. 17 that makes the new-DOF sets cover the fine
vertices and keeps A_c cell-local):
  * coincides with a coarse vertex          -> copy (shared DOF);
  * inside a coarse edge (a, b)             -> 1D projector = linear interpolation;
  * inside a coarse face F                  -> 2D projector Pi_{1,F};
  * inside a coarse cell C                  -> 3D projector Pi_1 of C.
The placement is taken in the parent of the lowest-numbered fine cell that has
the vertex.  Coarse operators are formed literally as A_c = P^T A_f P (Eq. 15)
with a library sparse product.

The naive VEM prolongation of Eq. 16 (the ablation "Ours^np") copies the
shared (coincident) vertex DOFs and evaluates every other fine vertex, on a
coarse edge or face too, from the projected coarse function Pi_1 of that same
parent cell; rows of vertices on coarse faces then reach the whole parent
cell, and the Galerkin products spread the coupling across cells.

Smoother (reading of "AMGCL default Chebyshev"): the textbook Chebyshev
semi-iteration (Saad, Iterative Methods, Alg. 12.1) of degree 5 in A itself on
[lmax/30, lmax], lmax = 1.1 x (largest Ritz value of 40 Lanczos steps started
from x_i = 1 + (i mod 7)/7; a 15-step power iteration underestimated lmax by
10% on a 96^3 grid, and the Chebyshev polynomial then amplifies the top of the
spectrum and CG breaks down);
one pre- and one post-sweep.  Coarsest level (the paper is silent): CG from
x0 = 0 for a fixed number of iterations (default 40) in the Chronopoulos-Gear
arrangement (Chronopoulos & Gear 1989: both inner products of an iteration in
one reduction), stopped early when ||r|| <= 1e-10 ||b|| (on a singular coarse
operator the rounding-level null-space part of the iterate drifts once the
range part has converged) or an inner product loses positivity; the
band of cut cells never aggregates, so this level stays large and a low-degree
polynomial leaves its smooth modes in place.
CG: x0 = 0, stop when ||r||/||r0|| <= tol; Polak-Ribiere beta (flexible CG),
which equals Fletcher-Reeves for a fixed SPD preconditioner in exact arithmetic.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .geometry import EPS, WELD
from .vem import CellVEM, face_projector_weights

CHEB_DEGREE = 5
COARSE_DEGREE = 20        # Chebyshev degree when COARSE_SOLVER == "cheb"
COARSE_SOLVER = "cg"
COARSE_ITERS = 80
COARSE_RTOL = 1e-10       # the coarsest CG also stops at this relative residual
LANCZOS_STEPS = 40
LMAX_SAFETY = 1.1
LMIN_RATIO = 30.0


# ---------------------------------------------------------------- prolongation

def classify_vertex(Vc, cfaces, x):
    """Placement of point x relative to a coarse cell given by its face cycles.
    Returns ('vertex', v) | ('edge', a, b, t) | ('face', cyc) | ('cell',)."""
    verts = sorted({v for f in cfaces for v in f})
    for v in verts:
        if np.max(np.abs(Vc[v] - x)) <= WELD:
            return ("vertex", v)
    for cyc in cfaces:
        k = len(cyc)
        for m in range(k):
            a, b = cyc[m], cyc[(m + 1) % k]
            e = Vc[b] - Vc[a]
            L2 = float(e @ e)
            t = float((x - Vc[a]) @ e) / L2
            L = np.sqrt(L2)
            if t * L > WELD and (1 - t) * L > WELD and \
                    np.linalg.norm(x - Vc[a] - t * e) <= WELD:
                return ("edge", a, b, t)
    for cyc in cfaces:
        P = Vc[cyc]
        A = np.zeros(3)
        for m in range(len(cyc)):
            A += np.cross(P[m], P[(m + 1) % len(cyc)])
        n = A / np.linalg.norm(A)
        if abs(float(n @ (x - P[0]))) > EPS:
            continue
        inside = True
        for m in range(len(cyc)):
            if float(np.cross(P[(m + 1) % len(cyc)] - P[m], x - P[m]) @ n) < -EPS:
                inside = False
                break
        if inside:
            return ("face", cyc)
    return ("cell",)


def prolongation(Mf, Mc, naive=False):
    """Full P (nf x nc) between level meshes (all vertices); naive: Eq. 16
    instead of the diffusion-free Eq. 17."""
    nf, nc = len(Mf.V), len(Mc.V)
    vcell = np.full(nf, -1, dtype=np.int64)
    for c, vs in enumerate(Mf.cell_verts):
        for v in vs:
            if vcell[v] < 0:
                vcell[v] = c
    cache = {}
    rows, cols, vals = [], [], []
    for v in range(nf):
        C = int(Mf.parent[vcell[v]])
        cfaces = [f[2] for f in Mc.cell_faces[C]]
        pl = classify_vertex(Mc.V, cfaces, Mf.V[v])
        if naive and pl[0] in ("edge", "face"):
            pl = ("cell",)
        if pl[0] == "vertex":
            ent = [(pl[1], 1.0)]
        elif pl[0] == "edge":
            _, a, b, t = pl
            ent = [(a, 1.0 - t), (b, t)]
        elif pl[0] == "face":
            cyc = pl[1]
            w = face_projector_weights(Mc.V, cyc, Mf.V[v])
            ent = list(zip(cyc, w))
        else:
            if C not in cache:
                cache[C] = CellVEM(Mc.V, cfaces, Mc.cell_verts[C])
            cv = cache[C]
            m = np.array([1.0, *((Mf.V[v] - cv.xE) / cv.h)])
            w = m @ cv.Pis
            ent = list(zip(cv.verts, w))
        for (c, w) in ent:
            rows.append(v)
            cols.append(c)
            vals.append(w)
    return sp.csr_matrix((vals, (rows, cols)), shape=(nf, nc))


# ---------------------------------------------------------------- smoother / cycle

def lanczos_lmax(A):
    """1.1 x the largest eigenvalue of the Lanczos tridiagonal matrix (no
    reorthogonalisation: extreme Ritz values are unaffected by ghost copies)."""
    n = A.shape[0]
    v = 1.0 + (np.arange(n) % 7) / 7.0
    v = v / np.linalg.norm(v)
    v_prev = np.zeros(n)
    alphas, betas = [], []
    beta = 0.0
    for _ in range(min(LANCZOS_STEPS, n)):
        w = A @ v
        a = float(v @ w)
        alphas.append(a)
        w = w - a * v - beta * v_prev
        beta = float(np.linalg.norm(w))
        if beta <= 1e-14 * max(abs(a), 1e-300):
            break
        betas.append(beta)
        v_prev, v = v, w / beta
    m = len(alphas)
    T = np.diag(alphas) + np.diag(betas[:m - 1], 1) + np.diag(betas[:m - 1], -1)
    return LMAX_SAFETY * float(np.linalg.eigvalsh(T)[-1])


def chebyshev(A, b, x0, lmax, degree, want_residual=False):
    """Chebyshev semi-iteration for A x = b on [lmax/30, lmax] (Saad Alg. 12.1)."""
    beta = lmax
    alpha = lmax / LMIN_RATIO
    theta = 0.5 * (beta + alpha)
    delta = 0.5 * (beta - alpha)
    sigma = theta / delta
    rho = 1.0 / sigma
    x = np.zeros_like(b) if x0 is None else x0.copy()
    r = b.copy() if x0 is None else b - A @ x
    d = r / theta
    for k in range(degree):
        x = x + d
        if k == degree - 1 and not want_residual:
            break
        r = r - A @ d
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * r
        rho = rho_new
    return (x, r) if want_residual else x


def fixed_cg(A, b, iters):
    """CG from x0 = 0 for `iters` iterations, in the Chronopoulos-Gear
    arrangement (both inner products of an iteration formed together; equal to
    plain CG in exact arithmetic).  Stops at ||r|| <= COARSE_RTOL ||b|| or if an
    inner product loses positivity."""
    x = np.zeros_like(b)
    r = b.copy()
    w = A @ r
    gamma = float(r @ r)
    delta = float(w @ r)
    if not (gamma > 0.0 and delta > 0.0):
        return x
    alpha = gamma / delta
    beta = 0.0
    stop = COARSE_RTOL ** 2 * gamma
    p = np.zeros_like(b)
    s = np.zeros_like(b)
    for it in range(iters):
        p = r + beta * p
        s = w + beta * s
        x = x + alpha * p
        r = r - alpha * s
        if it == iters - 1:
            break
        w = A @ r
        gamma_new = float(r @ r)
        delta = float(w @ r)
        if not gamma_new > stop:
            break
        beta = gamma_new / gamma
        den = delta - beta * gamma_new / alpha
        if not den > 0.0:
            break
        alpha = gamma_new / den
        gamma = gamma_new
    return x


class Hierarchy:
    """Free-DOF operators of every level: A[l], P[l] (level l+1 -> l)."""

    def __init__(self, A0, Ps):
        self.A = [A0]
        self.P = []
        for P in Ps:
            Ac = (P.T @ self.A[-1] @ P).tocsr()
            self.P.append(P.tocsr())
            self.A.append(Ac)
        self.lmax = [lanczos_lmax(A) for A in self.A]

    def vcycle(self, b, l=0):
        A = self.A[l]
        if l == len(self.A) - 1:
            if COARSE_SOLVER == "cg":
                return fixed_cg(A, b, COARSE_ITERS)
            return chebyshev(A, b, None, self.lmax[l], COARSE_DEGREE)
        x, r = chebyshev(A, b, None, self.lmax[l], CHEB_DEGREE, want_residual=True)
        P = self.P[l]
        e = self.vcycle(P.T @ r, l + 1)
        x = x + P @ e
        return chebyshev(A, b, x, self.lmax[l], CHEB_DEGREE)


def pcg(A, b, M, tol, max_iters=500):
    """Preconditioned CG, x0 = 0, Polak-Ribiere beta; returns (x, iters, relres history)."""
    x = np.zeros_like(b)
    r = b.copy()
    r0 = np.linalg.norm(r)
    hist = [1.0]
    if r0 == 0.0:
        return x, 0, hist
    z = M(r)
    p = z.copy()
    rz = float(r @ z)
    it = 0
    while it < max_iters:
        Ap = A @ p
        alpha = rz / float(p @ Ap)
        x = x + alpha * p
        r_new = r - alpha * Ap
        it += 1
        rel = np.linalg.norm(r_new) / r0
        hist.append(rel)
        if rel <= tol:
            break
        z_new = M(r_new)
        rz_new = float(r_new @ z_new)
        beta = (rz_new - float(r @ z_new)) / rz
        p = z_new + beta * p
        r, z, rz = r_new, z_new, rz_new
    return x, it, hist
