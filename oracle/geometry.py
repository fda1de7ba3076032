"""Oracle geometry: planes, convex polytopes from half-space lists, clipping.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this module;
it is the independent FP64 CPU reference that the CUDA library is checked
against.

Every geometric *decision* (which side of a plane, is a vertex feasible, do two
points coincide) is taken in IEEE-754 binary64 with the fixed evaluation order
written out below, so that an independent implementation that follows the same
written rules reaches the same integer topology:

  dot(a,b)   = (a0*b0 + a1*b1) + a2*b2
  cross(a,b) = (a1*b2 - a2*b1, a2*b0 - a0*b2, a0*b1 - a1*b0)
  s_p(x)     = dot(n_p, x) + d_p                      (signed distance)
  grid plane (axis a, index i):  n = e_a, d = -(i / N)
  triangle plane: c = cross(v1-v0, v2-v0), L = sqrt((c0*c0 + c1*c1) + c2*c2),
                  n = c / L, d = -dot(n, v0)
  vertex of planes i<j<k (ascending plane ids), Cramer's rule:
      cjk = cross(nj,nk), cki = cross(nk,ni), cij = cross(ni,nj)
      det = dot(ni, cjk)        (|det| < 1e-12 -> no vertex)
      x_c = ((((-di)*cjk_c) - (dj*cki_c)) - (dk*cij_c)) / det

Tolerances (unit domain [0,1]^3, unit normals): EPS = 1e-10 for side tests,
WELD = 1e-9 (max-norm) for coincident points.  These stand in for the exact
predicates the paper obtains from CGAL (Sec. 5.1).
"""
from __future__ import annotations

import functools
import itertools

import numpy as np

EPS = 1e-10
WELD = 1e-9
DET_MIN = 1e-12
VOL_MIN = 1e-12          # Sec. 5.1: partitions giving cells below 1e-12 are discarded
AREA_MIN = 1e-20


# ---------------------------------------------------------------- primitives

def dot3(a, b):
    return (a[..., 0] * b[..., 0] + a[..., 1] * b[..., 1]) + a[..., 2] * b[..., 2]


def cross3(a, b):
    return np.stack([a[..., 1] * b[..., 2] - a[..., 2] * b[..., 1],
                     a[..., 2] * b[..., 0] - a[..., 0] * b[..., 2],
                     a[..., 0] * b[..., 1] - a[..., 1] * b[..., 0]], axis=-1)


def _cross_s(a, b):
    a0, a1, a2 = float(a[0]), float(a[1]), float(a[2])
    b0, b1, b2 = float(b[0]), float(b[1]), float(b[2])
    return (a1 * b2 - a2 * b1, a2 * b0 - a0 * b2, a0 * b1 - a1 * b0)


def _dot_s(a, b):
    return (float(a[0]) * float(b[0]) + float(a[1]) * float(b[1])) + float(a[2]) * float(b[2])


def _sub_s(a, b):
    return (float(a[0]) - float(b[0]), float(a[1]) - float(b[1]), float(a[2]) - float(b[2]))


class PlaneTable:
    """All planes of one scene: 3(N+1) grid planes, then one per triangle."""

    def __init__(self, N: int, tris: np.ndarray):
        self.N = N
        self.ngrid = 3 * (N + 1)
        T = len(tris)
        n = np.zeros((self.ngrid + T, 3))
        d = np.zeros(self.ngrid + T)
        for a in range(3):
            for i in range(N + 1):
                pid = a * (N + 1) + i
                n[pid, a] = 1.0
                d[pid] = -(float(i) / float(N))
        v0, v1, v2 = tris[:, 0], tris[:, 1], tris[:, 2]
        c = cross3(v1 - v0, v2 - v0)
        L = np.sqrt((c[:, 0] * c[:, 0] + c[:, 1] * c[:, 1]) + c[:, 2] * c[:, 2])
        nt = c / L[:, None]
        n[self.ngrid:] = nt
        d[self.ngrid:] = -dot3(nt, v0)
        self.n = n
        self.d = d

    def grid_pid(self, axis, i):
        return axis * (self.N + 1) + i

    def tri_pid(self, t):
        return self.ngrid + t

    def is_grid(self, pid):
        return pid < self.ngrid

    def grid_axis_index(self, pid):
        return divmod(pid, self.N + 1)

    def side(self, pid, x):
        """s_p(x) for points x (...,3)."""
        return dot3(self.n[pid], x) + self.d[pid]


@functools.lru_cache(maxsize=None)
def _triples(m):
    return np.array(list(itertools.combinations(range(m), 3)), dtype=np.int64).reshape(-1, 3)


def solve_triples(PT: PlaneTable, tri_pids: np.ndarray):
    """Vertices of plane triples (rows of ascending plane ids).  Returns
    (coords (k,3), ok mask)."""
    ni, nj, nk = PT.n[tri_pids[:, 0]], PT.n[tri_pids[:, 1]], PT.n[tri_pids[:, 2]]
    di, dj, dk = PT.d[tri_pids[:, 0]], PT.d[tri_pids[:, 1]], PT.d[tri_pids[:, 2]]
    cjk, cki, cij = cross3(nj, nk), cross3(nk, ni), cross3(ni, nj)
    det = dot3(ni, cjk)
    ok = np.abs(det) >= DET_MIN
    safe = np.where(ok, det, 1.0)
    x = ((((-di)[:, None] * cjk) - (dj[:, None] * cki)) - (dk[:, None] * cij)) / safe[:, None]
    return x, ok


# ---------------------------------------------------------------- polytopes

class Polytope:
    """Convex polytope {x : sg * s_p(x) <= 0 for (p, sg) in H}.

    verts : (nv,3) representative coordinates (the candidate with the smallest
            plane-triple key among those that coincide)
    vkeys : per vertex, the list of plane-triple keys that produced it
    faces : list of (pid, sg, [vertex indices counter-clockwise about the
            outward normal sg*n_p])
    """

    __slots__ = ("H", "verts", "vkeys", "faces", "volume", "centroid")

    def __init__(self):
        self.H = []
        self.verts = np.zeros((0, 3))
        self.vkeys = []
        self.faces = []
        self.volume = 0.0
        self.centroid = np.zeros(3)


def _feasible(PT, H, x):
    pids = np.array([p for p, _ in H], dtype=np.int64)
    sg = np.array([s for _, s in H], dtype=np.float64)
    n = PT.n[pids]
    d = PT.d[pids]
    s = ((x[:, None, 0] * n[None, :, 0] + x[:, None, 1] * n[None, :, 1])
         + x[:, None, 2] * n[None, :, 2]) + d[None, :]
    return np.all(sg[None, :] * s <= EPS, axis=1)


def _weld_sorted(keys, x):
    """Candidates in ascending key order -> representatives (first wins)."""
    reps, rkeys = [], []
    for key, p in zip(keys, x):
        for r, q in enumerate(reps):
            if np.max(np.abs(p - q)) <= WELD:
                rkeys[r].append(key)
                break
        else:
            reps.append(p)
            rkeys.append([key])
    return (np.array(reps) if reps else np.zeros((0, 3))), rkeys


def order_ccw(points, normal, idx):
    """Sort polygon vertex indices counter-clockwise about `normal`, starting
    at idx[0] (convex position assumed)."""
    pivot = points[idx[0]]

    def cmp(a, b):
        c = _dot_s(_cross_s(_sub_s(points[a], pivot), _sub_s(points[b], pivot)), normal)
        return -1 if c > 0 else (1 if c < 0 else 0)
    rest = sorted(idx[1:], key=functools.cmp_to_key(cmp))
    return [idx[0]] + rest


def vertex_candidates(PT, H, pids=None, must=None):
    """Feasible plane-triple vertices of the polytope H (keys ascending).
    If `must` is given, only triples containing plane `must` are formed."""
    if pids is None:
        pids = sorted(set(p for p, _ in H))
    pids = np.array(pids, dtype=np.int64)
    if must is not None:
        others = pids[pids != must]
        if len(others) < 2:
            return [], np.zeros((0, 3))
        pr = np.array(list(itertools.combinations(range(len(others)), 2)), dtype=np.int64)
        trip = np.stack([np.full(len(pr), must), others[pr[:, 0]], others[pr[:, 1]]], axis=1)
        trip = np.sort(trip, axis=1)
    else:
        if len(pids) < 3:
            return [], np.zeros((0, 3))
        trip = pids[_triples(len(pids))]
    x, ok = solve_triples(PT, trip)
    trip, x = trip[ok], x[ok]
    if len(x) == 0:
        return [], x
    feas = _feasible(PT, H, x)
    trip, x = trip[feas], x[feas]
    order = np.lexsort((trip[:, 2], trip[:, 1], trip[:, 0]))
    keys = [tuple(int(v) for v in trip[o]) for o in order]
    return keys, x[order]


def cube_polytope(PT, H):
    """Axis-aligned cube (H from cube_H): the same result as make_polytope,
    built directly (grid-plane triples solve exactly to i/N)."""
    N1 = PT.N + 1
    px = (H[0][0], H[1][0])
    py = (H[2][0], H[3][0])
    pz = (H[4][0], H[5][0])
    P = Polytope()
    P.H = list(H)
    verts, keys = [], []
    for c in range(8):
        a, b, e = px[(c >> 0) & 1], py[(c >> 1) & 1], pz[(c >> 2) & 1]
        verts.append((-PT.d[a], -PT.d[b], -PT.d[e]))
        keys.append([(a, b, e)])
    # candidates come out in ascending key order: (x, y, z) with x fastest
    order = sorted(range(8), key=lambda c: keys[c][0])
    P.verts = np.array([verts[c] for c in order], dtype=np.float64) + 0.0
    P.vkeys = [keys[c] for c in order]
    pos = {order[i]: i for i in range(8)}
    quads = {0: [0, 4, 6, 2], 1: [1, 3, 7, 5], 2: [0, 1, 5, 4], 3: [2, 6, 7, 3],
             4: [0, 2, 3, 1], 5: [4, 5, 7, 6]}
    for f, (pid, sg) in enumerate(P.H):
        cyc = [pos[c] for c in quads[f]]
        nrm = sg * PT.n[pid]
        P.faces.append((pid, sg, order_ccw(P.verts, nrm, sorted(cyc))))
    P.volume, P.centroid = volume_centroid(P.verts, [f[2] for f in P.faces])
    return P


def make_polytope(PT, H, with_faces=True):
    if len(H) == 6 and all(PT.is_grid(p) for p, _ in H) and with_faces:
        return cube_polytope(PT, H)
    P = Polytope()
    P.H = list(H)
    keys, x = vertex_candidates(PT, H)
    P.verts, P.vkeys = _weld_sorted(keys, x)
    if len(P.verts) < 4 or not with_faces:
        return P
    for (pid, sg) in P.H:
        s = PT.side(pid, P.verts)
        on = [i for i in range(len(P.verts)) if abs(s[i]) <= EPS]
        if len(on) < 3:
            continue
        nrm = sg * PT.n[pid]
        cyc = order_ccw(P.verts, nrm, on)
        if polygon_area(P.verts[cyc], nrm) <= AREA_MIN:
            continue
        P.faces.append((pid, sg, cyc))
    P.volume, P.centroid = volume_centroid(P.verts, [f[2] for f in P.faces])
    return P


def polygon_area(pts, normal):
    """Area of a planar polygon (vector area projected on its unit normal)."""
    a0 = a1 = a2 = 0.0
    for i in range(len(pts)):
        c = _cross_s(pts[i], pts[(i + 1) % len(pts)])
        a0 += c[0]
        a1 += c[1]
        a2 += c[2]
    return 0.5 * _dot_s((a0, a1, a2), normal)


def volume_centroid(verts, cycles):
    """Volume and centroid of a closed polyhedron: fan tetrahedra from the
    vertex mean, summed face by face in the given order."""
    if len(verts) == 0 or not cycles:
        return 0.0, np.zeros(3)
    c0 = np.zeros(3)
    for v in verts:
        c0 = c0 + v
    c0 = c0 / float(len(verts))
    vol = 0.0
    cen = np.zeros(3)
    for cyc in cycles:
        a = verts[cyc[0]]
        for m in range(1, len(cyc) - 1):
            b, c = verts[cyc[m]], verts[cyc[m + 1]]
            t = _dot_s(_sub_s(a, c0), _cross_s(_sub_s(b, c0), _sub_s(c, c0))) / 6.0
            vol += t
            cen = cen + t * (((c0 + a) + b) + c) / 4.0
    if vol != 0.0:
        cen = cen / vol
    return vol, cen


def face_polygon(PT, Hunion, pid, sg):
    """Vertices of the flat polygon {x in plane pid} within the constraint set
    Hunion (which contains pid with both signs for an overlay piece).
    Returns (keys per vertex, coords (k,3) ordered CCW about sg*n_pid)."""
    keys, x = vertex_candidates(PT, Hunion, must=pid)
    reps, rkeys = _weld_sorted(keys, x)
    if len(reps) < 3:
        return [], reps[:0]
    nrm = sg * PT.n[pid]
    cyc = order_ccw(reps, nrm, list(range(len(reps))))
    if polygon_area(reps[cyc], nrm) <= AREA_MIN:
        return [], reps[:0]
    return [rkeys[i] for i in cyc], reps[cyc]


def cube_H(PT, i0, j0, k0, size):
    """Half-spaces of the axis-aligned cube [i0,i0+size]x... in grid units."""
    N1 = PT.N + 1
    return [(0 * N1 + i0, -1), (0 * N1 + i0 + size, 1),
            (1 * N1 + j0, -1), (1 * N1 + j0 + size, 1),
            (2 * N1 + k0, -1), (2 * N1 + k0 + size, 1)]


# ---------------------------------------------------------------- polygon clipping

def clip_polygon(PT, poly, pid, keep_sign):
    """Sutherland-Hodgman clip of a planar polygon (k,3) to the closed side
    keep_sign * s_pid <= 0.  Intersection points use the edge parameter
    t = s_a / (s_a - s_b)."""
    if len(poly) == 0:
        return poly
    s = keep_sign * PT.side(pid, poly)
    out = []
    k = len(poly)
    for i in range(k):
        a, b = poly[i], poly[(i + 1) % k]
        sa, sb = s[i], s[(i + 1) % k]
        ina, inb = sa <= EPS, sb <= EPS
        if ina:
            out.append(a)
        if ina != inb:
            t = sa / (sa - sb)
            out.append(a + (b - a) * t)
    return np.array(out) if out else np.zeros((0, 3))


def triangle_area_poly(poly):
    """Area of a planar polygon from its own vertex order (fan from vertex 0)."""
    if len(poly) < 3:
        return 0.0
    acc = 0.0
    for m in range(1, len(poly) - 1):
        c = _cross_s(_sub_s(poly[m], poly[0]), _sub_s(poly[m + 1], poly[0]))
        acc += 0.5 * float(np.sqrt(_dot_s(c, c)))
    return acc


# ---------------------------------------------------------------- inside test

def winding_number(tris, p):
    """Generalised winding number of a closed triangle soup about point p
    (solid angles, Van Oosterom & Strackee 1983), divided by 4 pi."""
    A = tris[:, 0] - p
    B = tris[:, 1] - p
    C = tris[:, 2] - p
    la = np.sqrt(dot3(A, A))
    lb = np.sqrt(dot3(B, B))
    lc = np.sqrt(dot3(C, C))
    num = dot3(A, cross3(B, C))
    den = la * lb * lc + dot3(A, B) * lc + dot3(B, C) * la + dot3(C, A) * lb
    return float(np.sum(2.0 * np.arctan2(num, den)) / (4.0 * np.pi))
