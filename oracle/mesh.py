"""Oracle: conforming polyhedral mesh of one hierarchy level, canonical numbering.

TEST INFRASTRUCTURE ONLY (never imported by the product path).

The paper cuts every background cell independently (Sec. 5.1) and coarsens
locally (Sec. 5.2); faces of neighbouring cells then do not match, yet the
conforming VEM space (Sec. 3) needs shared vertices, edges and faces.  Reading
taken here (the paper is silent on it):
  * overlay: every face of a fluid cell is replaced by its intersections with
    the opposite faces (same plane, opposite orientation) of the pieces that
    tile the other side -- fluid cells of the level and convex solid pieces;
  * vertices: all face vertices are welded (max-norm 1e-9); the coordinates
    of a welded vertex are those of its smallest plane-triple key;
  * T-junctions: every face edge is split at all welded vertices lying in its
    interior (distance <= 1e-9).  Cells keep their convex shape and gain
    coplanar sub-faces and collinear vertices, which the VEM allows;
  * numbering: vertices sorted by (z, y, x) on the 2^-30 lattice, then by the
    raw coordinates; face cycles start at their smallest vertex id and run
    counter-clockwise about the outward normal; a cell's faces are sorted by
    their cycles.
"""
from __future__ import annotations

import numpy as np
from scipy.spatial import cKDTree

from .cutcell import CutGrid, TREE, root_index
from .geometry import EPS, WELD, cube_H, face_polygon, make_polytope, polygon_area
from .hierarchy import Level, cell_H

Q30 = float(2 ** 30)


class LevelMesh:
    """Conforming mesh of the fluid cells of one level.

    V          (nv,3) vertex coordinates, canonical order
    cell_faces per cell: list of (pid, sg, [vertex ids, CCW about outward normal])
    cell_verts per cell: sorted vertex ids
    """

    def __init__(self):
        self.V = None
        self.cell_faces = []
        self.cell_verts = []
        self.parent = None


def build_level_mesh(G: CutGrid, lv: Level) -> LevelMesh:
    N = G.N
    PT = G.PT
    # ---- pieces: fluid cells first (piece id = cell position), then solids
    H_list = [cell_H(G, c) for c in lv.cells] + list(lv.solid_pieces)
    nfl = len(lv.cells)
    polys = [None] * len(H_list)

    def poly(p):
        if polys[p] is None:
            polys[p] = make_polytope(PT, H_list[p])
        return polys[p]

    # ---- root registry: background cell -> pieces that meet it
    reg = {}

    def footprint(H):
        """Background cells covered by a piece: its cube range for cubes, the
        single root for BSP pieces (first six half-spaces are the root cube)."""
        lo = [0, 0, 0]
        hi = [0, 0, 0]
        for a in range(3):
            pa_lo, _ = H[2 * a]
            pa_hi, _ = H[2 * a + 1]
            lo[a] = pa_lo - a * (N + 1)
            hi[a] = pa_hi - a * (N + 1)
        return lo, hi

    for p, H in enumerate(H_list):
        lo, hi = footprint(H)
        for k in range(lo[2], hi[2]):
            for j in range(lo[1], hi[1]):
                for i in range(lo[0], hi[0]):
                    reg.setdefault(root_index(N, i, j, k), []).append(p)

    # ---- overlay
    occ = []            # per fluid cell: list of faces; face = (pid, sg, [(keys, xyz), ...])
    for c in range(nfl):
        P = poly(c)
        H = H_list[c]
        lo, hi = footprint(H)
        faces = []
        for (pid, sg, cyc) in P.faces:
            fverts = [(P.vkeys[v], P.verts[v]) for v in cyc]
            if PT.is_grid(pid):
                a, idx = PT.grid_axis_index(pid)
                o = idx if sg > 0 else idx - 1
                if o < 0 or o >= N:
                    faces.append((pid, sg, fverts))      # domain wall
                    continue
                rng = [range(lo[b], hi[b]) for b in range(3)]
                rng[a] = range(o, o + 1)
                cand = set()
                for k in rng[2]:
                    for j in rng[1]:
                        for i in rng[0]:
                            cand.update(reg.get(root_index(N, i, j, k), []))
            else:
                cand = set(reg.get(root_index(N, lo[0], lo[1], lo[2]), []))
            cand.discard(c)
            area_f = polygon_area(P.verts[cyc], sg * PT.n[pid])
            pieces = []
            fkeys = frozenset(min(P.vkeys[v]) for v in cyc)
            for q in sorted(cand):
                if (pid, -sg) not in H_list[q]:
                    continue
                Pq = poly(q)
                same = False
                for (qp, qs, qcyc) in Pq.faces:
                    if qp == pid and qs == -sg:
                        same = frozenset(min(Pq.vkeys[v]) for v in qcyc) == fkeys
                        break
                if same:
                    pieces.append(list(fverts))
                    continue
                Hu = list(H) + [h for h in H_list[q] if h not in H]
                keys, xyz = face_polygon(PT, Hu, pid, sg)
                if len(keys) >= 3:
                    pieces.append(list(zip(keys, xyz)))
            tot = sum(polygon_area(np.array([x for _, x in pc]), sg * PT.n[pid]) for pc in pieces)
            # relative to the face, plus a floor of 1e-11 of a background
            # cell face: sliver faces (width ~1e-6 h) carry rounding of their
            # long edges, which is not small relative to their own area
            if abs(tot - area_f) > 1e-9 * max(area_f, 1e-30) + 1e-11 / (N * N):
                raise RuntimeError(f"overlay does not cover face: cell {c} pid {pid} "
                                   f"area {area_f} covered {tot}")
            for pc in pieces:
                faces.append((pid, sg, pc))
        occ.append(faces)

    # ---- global weld
    cand = {}
    for faces in occ:
        for (_, _, fv) in faces:
            for keys, x in fv:
                k0 = min(keys)
                if k0 not in cand:
                    cand[k0] = x
    keys_sorted = sorted(cand)
    grid = {}
    rep_of = {}
    reps = []
    inv = 1.0 / (4.0 * WELD)
    for key in keys_sorted:
        x = cand[key]
        b = tuple(int(np.floor(x[a] * inv)) for a in range(3))
        hit = -1
        for dz in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dx in (-1, 0, 1):
                    for r in grid.get((b[0] + dx, b[1] + dy, b[2] + dz), ()):
                        if np.max(np.abs(reps[r] - x)) <= WELD:
                            hit = r
                            break
                    if hit >= 0:
                        break
                if hit >= 0:
                    break
            if hit >= 0:
                break
        if hit < 0:
            hit = len(reps)
            reps.append(x)
            grid.setdefault(b, []).append(hit)
        rep_of[key] = hit
    R = np.array(reps)

    cells_faces = []
    for faces in occ:
        cf = []
        for (pid, sg, fv) in faces:
            cyc = []
            for keys, _ in fv:
                g = rep_of[min(keys)]
                if not cyc or cyc[-1] != g:
                    cyc.append(g)
            while len(cyc) > 1 and cyc[0] == cyc[-1]:
                cyc.pop()
            cf.append((pid, sg, cyc))
        cells_faces.append(cf)

    # ---- T-junctions: split face edges at welded vertices inside them
    used = sorted({g for cf in cells_faces for (_, _, cyc) in cf for g in cyc})
    Ru = R[used]
    tree = cKDTree(Ru)
    split_cache = {}

    def inner(a, b):
        key = (a, b) if a < b else (b, a)
        if key not in split_cache:
            pa, pb = R[key[0]], R[key[1]]
            e = pb - pa
            L2 = float(e @ e)
            L = np.sqrt(L2)
            mids = tree.query_ball_point((pa + pb) / 2.0, L / 2.0 + 2 * WELD)
            res = []
            for m in mids:
                v = used[m]
                if v == key[0] or v == key[1]:
                    continue
                w = R[v] - pa
                t = float(w @ e) / L2
                dist = np.linalg.norm(w - t * e)
                if dist <= WELD and t * L > WELD and (1.0 - t) * L > WELD:
                    res.append((t, v))
            res.sort()
            split_cache[key] = [v for _, v in res]
        out = split_cache[key]
        return out if a < b else out[::-1]

    for cf in cells_faces:
        for fi, (pid, sg, cyc) in enumerate(cf):
            new = []
            for i in range(len(cyc)):
                a, b = cyc[i], cyc[(i + 1) % len(cyc)]
                new.append(a)
                new.extend(inner(a, b))
            cf[fi] = (pid, sg, new)

    # ---- canonical numbering
    used = sorted({g for cf in cells_faces for (_, _, cyc) in cf for g in cyc})
    U = R[used]
    q = np.floor(U * Q30 + 0.5)
    order = np.lexsort((U[:, 0], U[:, 1], U[:, 2], q[:, 0], q[:, 1], q[:, 2]))
    newid = {}
    for rank, o in enumerate(order):
        newid[used[o]] = rank
    M = LevelMesh()
    M.V = U[order]
    for cf in cells_faces:
        faces = []
        for (pid, sg, cyc) in cf:
            ids = [newid[g] for g in cyc]
            s = int(np.argmin(ids))
            ids = ids[s:] + ids[:s]
            faces.append((pid, sg, ids))
        faces.sort(key=lambda f: f[2])
        M.cell_faces.append(faces)
        M.cell_verts.append(sorted({v for f in faces for v in f[2]}))
    M.parent = None if lv.parent is None else np.array(lv.parent, dtype=np.int64)
    return M


def build_meshes(G: CutGrid, levels):
    return [build_level_mesh(G, lv) for lv in levels]
