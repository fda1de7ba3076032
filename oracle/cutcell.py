"""Oracle: binary-space-partition cut cells (Sec. 5.1) and cut weights (Sec. 5.2).

TEST INFRASTRUCTURE ONLY (never imported by the product path).

Readings of the paper taken here (each listed in the design notes):
  * association (Sec. 5.1, "uniform sampling" with no density given): a
    triangle belongs to every background cell its closed clip against the
    cube is non-empty for (a superset of any sampling);
  * cut order: per cell, a triangle's count is the number of *other triangles
    of that cell* that its supporting plane crosses strictly; ascending count,
    ties by triangle index;
  * a plane is applied only if it splits the current region strictly and both
    children keep volume >= 1e-12; otherwise the triangle is skipped;
  * the remaining triangles go to the child (or both) on whose side their
    clipped part lies ("spatial relationship to the cutting plane");
  * inside/outside (Sec. 5.1 ray vote): the generalised winding number of the
    closed obstacle mesh at the leaf centroid, > 1/2 means solid.  For closed
    meshes every fair ray vote gives the same answer;
  * importance weight (Sec. 5.2): area of the triangles coplanar with the cut
    that lie in the node's region, over the total mesh area; stored also as
    the integer round(w * 2^40) so that greedy order and the running sum are
    exact.
"""
from __future__ import annotations

import numpy as np
from scipy import ndimage

from .geometry import (EPS, VOL_MIN, PlaneTable, clip_polygon, cube_H, make_polytope,
                       triangle_area_poly, winding_number)

WQ = float(2 ** 40)

# root kinds
UNCUT_FLUID, UNCUT_SOLID, SINGLE_FLUID, SINGLE_SOLID, TREE = 0, 1, 2, 3, 4


class Node:
    __slots__ = ("id", "parent", "left", "right", "pid", "H", "poly", "w", "wq",
                 "solid", "nfluid", "leaf_id")

    def __init__(self, nid, parent, H):
        self.id = nid
        self.parent = parent
        self.left = -1
        self.right = -1
        self.pid = -1
        self.H = H
        self.poly = None
        self.w = 0.0
        self.wq = 0
        self.solid = False
        self.nfluid = 0
        self.leaf_id = -1

    @property
    def is_leaf(self):
        return self.left < 0


class RootTree:
    def __init__(self, r, ijk):
        self.r = r
        self.ijk = ijk
        self.nodes: list[Node] = []


def root_index(N, i, j, k):
    return i + N * (j + N * k)


class CutGrid:
    """Finest-level cut-cell grid: per background cell a kind, and a BSP tree
    for cells split into more than one leaf."""

    def __init__(self, N, tris, total_area, kinds, trees, assoc):
        self.N = N
        self.tris = tris
        self.PT = PlaneTable(N, tris)
        self.total_area = total_area
        self.kinds = kinds          # (N^3,) int8
        self.trees = trees          # r -> RootTree
        self.assoc = assoc          # r -> ordered list of triangle ids


def associate(PT: PlaneTable, tris):
    """Triangle -> background cells whose closed cube it touches; returns
    dict r -> list of (t, clipped polygon)."""
    N = PT.N
    out = {}
    lo = np.floor((tris.min(axis=1) - EPS) * N).astype(np.int64)
    hi = np.floor((tris.max(axis=1) + EPS) * N).astype(np.int64)
    lo = np.clip(lo, 0, N - 1)
    hi = np.clip(hi, 0, N - 1)
    for t in range(len(tris)):
        if np.any(tris[t].max(axis=0) < -EPS) or np.any(tris[t].min(axis=0) > 1 + EPS):
            continue
        for k in range(lo[t, 2], hi[t, 2] + 1):
            for j in range(lo[t, 1], hi[t, 1] + 1):
                for i in range(lo[t, 0], hi[t, 0] + 1):
                    poly = tris[t].copy()
                    for (pid, sg) in cube_H(PT, i, j, k, 1):
                        poly = clip_polygon(PT, poly, pid, sg)
                        if len(poly) == 0:
                            break
                    if len(poly):
                        out.setdefault(root_index(N, i, j, k), []).append((t, poly))
    return out


def cut_order(PT: PlaneTable, tris, tlist):
    """Sort a cell's triangles by how many other cell triangles their plane
    crosses strictly (ascending), ties by index."""
    ids = [t for t, _ in tlist]
    counts = []
    for t in ids:
        pid = PT.tri_pid(t)
        c = 0
        for u in ids:
            if u == t:
                continue
            s = PT.side(pid, tris[u])
            if s.max() > EPS and s.min() < -EPS:
                c += 1
        counts.append(c)
    order = sorted(range(len(ids)), key=lambda a: (counts[a], ids[a]))
    return [tlist[a] for a in order]


def _split_list(PT, rest, pid):
    left, right = [], []
    for (t, poly) in rest:
        s = PT.side(pid, poly)
        flat = bool(np.all(np.abs(s) <= EPS))
        if flat or s.min() < -EPS:
            lp = clip_polygon(PT, poly, pid, 1.0)
            if len(lp):
                left.append((t, lp))
        if flat or s.max() > EPS:
            rp = clip_polygon(PT, poly, pid, -1.0)
            if len(rp):
                right.append((t, rp))
    return left, right


def build_tree(PT: PlaneTable, tris, total_area, r, ijk, tlist):
    tree = RootTree(r, ijk)

    def rec(H, lst, parent):
        node = Node(len(tree.nodes), parent, H)
        tree.nodes.append(node)
        P = make_polytope(PT, H)
        node.poly = P
        for idx, (t, _poly) in enumerate(lst):
            pid = PT.tri_pid(t)
            s = PT.side(pid, P.verts)
            if not (s.max() > EPS and s.min() < -EPS):
                continue
            HL = H + [(pid, 1)]
            HR = H + [(pid, -1)]
            PL = make_polytope(PT, HL)
            PR = make_polytope(PT, HR)
            if PL.volume < VOL_MIN or PR.volume < VOL_MIN:
                continue
            area = 0.0
            for (u, upoly) in lst:
                su = PT.side(pid, tris[u])
                if np.all(np.abs(su) <= EPS):
                    area += triangle_area_poly(upoly)
            node.pid = pid
            node.w = area / total_area
            node.wq = int(round(node.w * WQ))
            left, right = _split_list(PT, lst[idx + 1:], pid)
            node.left = rec(HL, left, node.id)
            node.right = rec(HR, right, node.id)
            return node.id
        return node.id

    rec(cube_H(PT, *ijk, 1), tlist, -1)
    return tree


def build_cut_grid(N, tris) -> CutGrid:
    tris = np.asarray(tris, dtype=np.float64)
    PT = PlaneTable(N, tris)
    total_area = 0.0
    for t in range(len(tris)):
        total_area += triangle_area_poly(tris[t])
    assoc = associate(PT, tris)
    kinds = np.full(N ** 3, UNCUT_FLUID, dtype=np.int8)
    trees = {}
    order = {}
    for r in sorted(assoc):
        k, rem = divmod(r, N * N)
        j, i = divmod(rem, N)
        lst = cut_order(PT, tris, assoc[r])
        order[r] = [t for t, _ in lst]
        tree = build_tree(PT, tris, total_area, r, (i, j, k), lst)
        if len(tree.nodes) == 1:
            c = (np.array([i, j, k], dtype=np.float64) + 0.5) / N
            kinds[r] = SINGLE_SOLID if winding_number(tris, c) > 0.5 else SINGLE_FLUID
            continue
        kinds[r] = TREE
        for nd in tree.nodes:
            if nd.is_leaf:
                nd.solid = winding_number(tris, nd.poly.centroid) > 0.5
        # fluid counts bottom-up (children have larger preorder ids)
        for nd in reversed(tree.nodes):
            if nd.is_leaf:
                nd.nfluid = 0 if nd.solid else 1
            else:
                nd.nfluid = tree.nodes[nd.left].nfluid + tree.nodes[nd.right].nfluid
        trees[r] = tree
    # uncut cells: connected components (6-neighbour) share the inside status
    uncut = np.ones(N ** 3, dtype=bool)
    uncut[list(assoc.keys())] = False
    lab, nlab = ndimage.label(uncut.reshape(N, N, N))   # array index [k][j][i]
    lab = lab.reshape(-1)
    if nlab:
        first = np.full(nlab + 1, -1, dtype=np.int64)
        idx = np.nonzero(lab)[0]
        for r in idx[::-1]:
            first[lab[r]] = r
        for comp in range(1, nlab + 1):
            r = first[comp]
            k, rem = divmod(r, N * N)
            j, i = divmod(rem, N)
            c = (np.array([i, j, k], dtype=np.float64) + 0.5) / N
            if winding_number(tris, c) > 0.5:
                kinds[(lab == comp)] = UNCUT_SOLID
    return CutGrid(N, tris, total_area, kinds, trees, order)
