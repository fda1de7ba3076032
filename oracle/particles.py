"""Oracle: the particle transfers around the projection (Sec. 3.2 P2G,
Sec. 3.3 G2P and advection), plain FP64, brute force over all pairs.

TEST INFRASTRUCTURE ONLY (never imported by the product path).

P2G (Sec. 3.2): the value at vertex i is the normalised radial-kernel
average of the particles' values,
    f_i = sum_p f_p w_ip / sum_p w_ip,   w_ip = k(|x_p - x_i|^2 / R^2),
    k(q) = max(0, 1 - q)^3,
with R the edge length h = 1/N of the background grid.

G2P (Sec. 3.3): with Pi_1 u_h the cell polynomials of the P2G velocity and
Pi_1 u_new those of the projected velocity, Delta u = Pi_1 u_new - Pi_1 u_h
and every particle takes the FLIP / PIC blend at its position x_p in its
cell.

Advection (Sec. 3.3): second-order Runge-Kutta in the projected velocity
field, with particles that cross an obstacle mirrored back across it.

Readings (the paper leaves these open or prints them garbled):
  * Sigma_p w_ip = 0 (no particle within R) gives f_i = 0; particles whose
    cell is -1 (inside an obstacle or outside the grid) carry no value;
  * the printed FLIP update adds the increment outside the FLIP weight, so at
    alpha = 0 it would not be the PIC update; it is read as the standard
    blend of the cited FLIP scheme:
        u_p <- alpha (u_p + Delta u(x_p)) + (1 - alpha) Pi_1 u_new(x_p);
  * the cell of a point is the lowest-numbered level-0 cell whose closed
    face half-spaces hold it within 1e-10 (the side tolerance of the grid
    construction), -1 if none; the outward plane of a face occurrence is
    its normalised Newell normal through the mean of its vertices;
  * RK2 is the midpoint rule: x_m = x + dt/2 v(x), x_new = x + dt v(x_m);
  * each stage's end point y (from start x) is handled in this order:
    (1) the first obstacle triangle that the segment x -> y crosses (least
        parameter t in (0, 1], ties to the lower triangle index) mirrors y
        across that triangle's plane;
    (2) a coordinate outside [0, 1] is mirrored across that wall of the box;
    (3) if y then lies in no fluid cell, the particle stays at x (in x's
        cell) for that stage;
  * particles whose cell is -1 are left as they are by G2P and advection.
"""
from __future__ import annotations

import numpy as np

LOCATE_TOL = 1e-10


def kernel_weight(q):
    """k(q) = max(0, 1 - q)^3 (Sec. 3.2)."""
    return np.maximum(0.0, 1.0 - np.asarray(q, dtype=np.float64)) ** 3


def p2g(V, xp, fp, R, alive=None):
    """f_i for every vertex.  V: (nv,3); xp: (np,3); fp: (np,C); returns
    (nv,C).  alive: optional (np,) bool, particles that count."""
    xp = np.asarray(xp, dtype=np.float64)
    fp = np.asarray(fp, dtype=np.float64)
    if alive is not None:
        xp, fp = xp[alive], fp[alive]
    out = np.zeros((len(V), fp.shape[1]))
    for i in range(len(V)):
        d = xp - V[i]
        w = kernel_weight((d * d).sum(axis=1) / (R * R))
        s = w.sum()
        if s > 0.0:
            out[i] = (w[:, None] * fp).sum(axis=0) / s
    return out


def face_planes(mesh):
    """Per cell, the (n, d) of its face occurrences: n the unit outward
    Newell normal, d = n . (mean of the face's vertices)."""
    V = mesh.V
    planes = []
    for cf in mesh.cell_faces:
        pl = []
        for (_, _, cyc) in cf:
            P = V[cyc]
            n = np.zeros(3)
            for m in range(len(cyc)):
                n = n + np.cross(P[m], P[(m + 1) % len(cyc)])
            n = n / np.linalg.norm(n)
            pl.append((n, float(n @ P.mean(axis=0))))
        planes.append(pl)
    return planes


def cell_boxes(mesh):
    """Per cell, its vertices' bounding box grown by 1e-9 (lo, hi)."""
    lo = np.array([mesh.V[v].min(axis=0) for v in mesh.cell_verts]) - 1e-9
    hi = np.array([mesh.V[v].max(axis=0) for v in mesh.cell_verts]) + 1e-9
    return lo, hi


def locate(mesh, xp, planes=None, boxes=None):
    """Cell of every point (reading above), -1 if none.  Cells are tried in
    ascending order; one whose vertex bounding box (grown by 1e-9) misses
    the point cannot hold it and is skipped, which only saves time."""
    planes = face_planes(mesh) if planes is None else planes
    lo, hi = cell_boxes(mesh) if boxes is None else boxes
    xp = np.asarray(xp, dtype=np.float64)
    out = np.full(len(xp), -1, dtype=np.int64)
    for p, x in enumerate(xp):
        for c in np.nonzero(np.all((lo <= x) & (x <= hi), axis=1))[0]:
            if all(float(n @ x) - d <= LOCATE_TOL for n, d in planes[c]):
                out[p] = int(c)
                break
    return out


def cell_linear(cells, u_vert):
    """Pi_1 u per cell, (nc,3,4) [component][monomial 1, (x-x_E)/h_E]."""
    return np.array([cv.velocity_coeffs(u_vert[cv.verts]) for cv in cells])


def eval_linear(cells, coef, c, x):
    """Velocity of cell c's linear polynomial at x."""
    cv = cells[c]
    y = (np.asarray(x, dtype=np.float64) - cv.xE) / cv.h
    return coef[c][:, 0] + coef[c][:, 1:] @ y


def g2p(cells, xp, cell, u_old_vert, cellpoly_new, alpha, up):
    """New particle velocities (reading above); up: (np,3)."""
    old = cell_linear(cells, u_old_vert)
    out = np.array(up, dtype=np.float64, copy=True)
    for p in range(len(xp)):
        c = int(cell[p])
        if c < 0:
            continue
        vn = eval_linear(cells, cellpoly_new, c, xp[p])
        vo = eval_linear(cells, old, c, xp[p])
        out[p] = alpha * (out[p] + (vn - vo)) + (1.0 - alpha) * vn
    return out


def segment_triangle_t(x0, x1, tri):
    """Parameter t in (0, 1] where the segment x0 -> x1 meets triangle tri
    (3x3), or None (Moller-Trumbore; parallel segments never meet)."""
    d = x1 - x0
    e1, e2 = tri[1] - tri[0], tri[2] - tri[0]
    pv = np.cross(d, e2)
    det = float(e1 @ pv)
    if det == 0.0:
        return None
    inv = 1.0 / det
    tv = x0 - tri[0]
    u = float(tv @ pv) * inv
    if u < 0.0 or u > 1.0:
        return None
    qv = np.cross(tv, e1)
    v = float(d @ qv) * inv
    if v < 0.0 or u + v > 1.0:
        return None
    t = float(e2 @ qv) * inv
    return t if 0.0 < t <= 1.0 else None


def _stage_end(mesh, planes, boxes, tris, x0, c0, y):
    best, bi = None, -1
    # triangles whose bounding box misses the segment's cannot meet it
    smin, smax = np.minimum(x0, y), np.maximum(x0, y)
    near = np.nonzero(np.all((tris.min(axis=1) <= smax) & (tris.max(axis=1) >= smin), axis=1))[0]
    for i in near:
        tri = tris[i]
        t = segment_triangle_t(x0, y, tri)
        if t is not None and (best is None or t < best):
            best, bi = t, i
    if bi >= 0:
        tri = tris[bi]
        n = np.cross(tri[1] - tri[0], tri[2] - tri[0])
        n = n / np.linalg.norm(n)
        y = y - 2.0 * float((y - tri[0]) @ n) * n
    y = np.where(y < 0.0, -y, y)
    y = np.where(y > 1.0, 2.0 - y, y)
    c = int(locate(mesh, y[None], planes, boxes)[0])
    if c < 0:
        return np.array(x0, dtype=np.float64), c0
    return y, c


def advect(mesh, cells, tris, cellpoly, dt, xp, cell):
    """RK2 (midpoint) step of every live particle (reading above)."""
    planes, boxes = face_planes(mesh), cell_boxes(mesh)
    X = np.array(xp, dtype=np.float64, copy=True)
    C = np.array(cell, dtype=np.int64, copy=True)
    tris = np.asarray(tris, dtype=np.float64).reshape(-1, 3, 3)
    for p in range(len(X)):
        c0 = int(C[p])
        if c0 < 0:
            continue
        x0 = X[p].copy()
        v0 = eval_linear(cells, cellpoly, c0, x0)
        xm, cm = _stage_end(mesh, planes, boxes, tris, x0, c0, x0 + 0.5 * dt * v0)
        vm = eval_linear(cells, cellpoly, cm, xm)
        X[p], C[p] = _stage_end(mesh, planes, boxes, tris, x0, c0, x0 + dt * vm)
    return X, C
