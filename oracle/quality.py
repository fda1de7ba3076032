"""Oracle: the VEM element quality indicator (Eq. 18, Eq. 19 and App. C).

TEST INFRASTRUCTURE ONLY (never imported by the product path).

For a cell E with faces f (vertex cycles, counter-clockwise about the outward
normal) and the edges e of each face:

  rho1(E) = |k(E)| / |E| * prod_f |k(f)| / |f|,
            k(.) the kernel: the points from which the whole element is
            visible, i.e. the intersection of the inner half-spaces of its
            faces (cell) or of its edges (face, in the face's plane);
  rho2(E) = min(|E|^(1/3), min_f h_f) / h_E
            + (1 / #f) sum_f min(|f|^(1/2), min_{e in f} |e|) / h_f;
  rho3(E) = 4 / #f + (1 / #f) sum_f 3 / #e_f;
  rho(E)  = sqrt(rho1 rho2 + rho1 rho3) / 2                       (Eq. 18);
  rho(P)  = sqrt(mean over the cut cells of rho(E)^2)             (Eq. 19).

h_E and h_f are diameters (largest distance between two vertices).

Readings (the printed formulas are garbled in two places):
  * the face term of rho2 prints the cube root of the face's area, which is
    not a length; read as the square root, the 2D counterpart of the cell's
    cube root of its volume;
  * Eq. 19 is cut off after the sum; read as the root mean square over the
    cut cells;
  * a cut cell is a cell that is not an axis-aligned cube: its bounding box
    is not a cube, or its volume differs from the box's (relative 1e-9).

Kernels are computed for any polyhedron: the half-spaces are intersected by
scipy.spatial.HalfspaceIntersection around an interior point found by a
linear program (the largest inscribed ball), and the volume / area of the
intersection is that of its convex hull; the linear program's and the hull's
tolerances leave about 1e-9 relative error in rho1.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import linprog
from scipy.spatial import ConvexHull, HalfspaceIntersection


def _kernel_measure(A, b):
    """Measure (volume in 3D, area in 2D) of {x : A x <= b}, 0 if empty."""
    dim = A.shape[1]
    norms = np.linalg.norm(A, axis=1)
    # largest ball inside: max r with A x + r |a| <= b
    c = np.zeros(dim + 1)
    c[-1] = -1.0
    res = linprog(c, A_ub=np.hstack([A, norms[:, None]]), b_ub=b, bounds=[(None, None)] * dim + [(0, None)],
                  method="highs")
    if not res.success or res.x[-1] <= 1e-14 * max(1.0, float(np.abs(b).max())):
        return 0.0
    x0 = res.x[:dim]
    hs = HalfspaceIntersection(np.hstack([A, -b[:, None]]), x0)
    return float(ConvexHull(hs.intersections).volume)


def _face_frame(V, cyc):
    P = V[cyc]
    A = np.zeros(3)
    for i in range(len(cyc)):
        A = A + np.cross(P[i], P[(i + 1) % len(cyc)])
    area = 0.5 * float(np.linalg.norm(A))
    n = A / np.linalg.norm(A)
    t1 = P[1] - P[0]
    t1 = t1 - np.dot(t1, n) * n
    t1 /= np.linalg.norm(t1)
    t2 = np.cross(n, t1)
    return P, area, n, t1, t2


def face_kernel_area(V, cyc):
    """Area of the kernel of a planar polygon (its cycle CCW about n),
    computed in coordinates centred on the polygon and scaled by its
    diameter (so the linear program and the hull see unit-size data)."""
    P, area, n, t1, t2 = _face_frame(V, cyc)
    s = _diameter(P)
    Q = np.stack([(P - P.mean(axis=0)) @ t1, (P - P.mean(axis=0)) @ t2], axis=1) / s
    A, b = [], []
    k = len(cyc)
    for i in range(k):
        e = Q[(i + 1) % k] - Q[i]
        if np.linalg.norm(e) == 0.0:
            continue
        out = np.array([e[1], -e[0]])  # outward normal of a CCW polygon's edge
        A.append(out)
        b.append(float(out @ Q[i]))
    return _kernel_measure(np.array(A), np.array(b)) * s * s


def cell_kernel_volume(V, faces):
    """Volume of the kernel of a polyhedron (faces CCW about outward
    normals), computed in coordinates centred on the cell's vertices and
    scaled by its diameter."""
    verts = sorted({v for f in faces for v in f})
    c = V[verts].mean(axis=0)
    s = _diameter(V[verts])
    W = (V - c) / s
    A, b = [], []
    for cyc in faces:
        P, area, n, _, _ = _face_frame(W, cyc)
        A.append(n)
        b.append(float(n @ P.mean(axis=0)))
    return _kernel_measure(np.array(A), np.array(b)) * s ** 3


def _volume(V, faces):
    verts = sorted({v for f in faces for v in f})
    c0 = V[verts].mean(axis=0)
    vol = 0.0
    for cyc in faces:
        a = V[cyc[0]]
        for m in range(1, len(cyc) - 1):
            vol += float(np.dot(a - c0, np.cross(V[cyc[m]] - c0, V[cyc[m + 1]] - c0))) / 6.0
    return vol


def _diameter(X):
    d = X[:, None, :] - X[None, :, :]
    return float(np.sqrt((d * d).sum(-1)).max())


def cell_quality(V, faces):
    """(rho, rho1, rho2, rho3) of one cell (App. C, Eq. 18)."""
    verts = sorted({v for f in faces for v in f})
    vol = _volume(V, faces)
    hE = _diameter(V[verts])
    rho1 = cell_kernel_volume(V, faces) / vol
    nf = len(faces)
    min_hf = np.inf
    s2 = s3 = 0.0
    for cyc in faces:
        P, area, _, _, _ = _face_frame(V, cyc)
        rho1 *= face_kernel_area(V, cyc) / area
        hf = _diameter(P)
        emin = min(float(np.linalg.norm(P[(i + 1) % len(cyc)] - P[i])) for i in range(len(cyc)))
        min_hf = min(min_hf, hf)
        s2 += min(np.sqrt(area), emin) / hf
        s3 += 3.0 / len(cyc)
    rho2 = min(np.cbrt(vol), min_hf) / hE + s2 / nf
    rho3 = 4.0 / nf + s3 / nf
    return float(np.sqrt(rho1 * rho2 + rho1 * rho3) / 2.0), rho1, rho2, rho3


def is_cut(V, faces, rel=1e-9):
    """Not an axis-aligned cube (reading of "cut cell" above)."""
    verts = sorted({v for f in faces for v in f})
    X = V[verts]
    ext = X.max(axis=0) - X.min(axis=0)
    cube = abs(ext[0] - ext[1]) <= rel * ext[0] and abs(ext[1] - ext[2]) <= rel * ext[0]
    return not (cube and abs(_volume(V, faces) - float(np.prod(ext))) <= rel * float(np.prod(ext)))


def mesh_quality(mesh):
    """Per-cell rho, the cut mask and rho(P) of a LevelMesh (Eq. 19)."""
    V = mesh.V
    rho = np.zeros(len(mesh.cell_faces))
    cut = np.zeros(len(mesh.cell_faces), dtype=bool)
    for c, cf in enumerate(mesh.cell_faces):
        faces = [f[2] for f in cf]
        rho[c] = cell_quality(V, faces)[0]
        cut[c] = is_cut(V, faces)
    grid = float(np.sqrt(np.mean(rho[cut] ** 2))) if cut.any() else float("nan")
    return rho, cut, grid
