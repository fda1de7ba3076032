"""Pins of the oracle's cut order (Sec. 5.1), importance weights and greedy
cut removal (Sec. 5.2) on hand-built scenes whose answers are worked out by
hand below, not by the oracle:

* cut order: per cell, a triangle's count is the number of *other triangles
  of the same cell* that its supporting plane crosses strictly; ascending
  count, ties by triangle index;
* weight of a cut: area of the triangles coplanar with the cut plane that lie
  in the node's region, over the total mesh area;
* greedy removal: removable cuts (both children current leaves) are popped
  smallest weight first (ties by background cell index, then node id), and
  the iteration stops once the removed weight exceeds 1/L (the removal that
  crosses 1/L is kept).
"""
from fractions import Fraction as F

import numpy as np

from oracle.cutcell import associate, build_cut_grid, build_tree, cut_order, root_index
from oracle.geometry import PlaneTable
from oracle.hierarchy import HierarchyState, build_hierarchy


def _tri(*v):
    return np.array(v, dtype=np.float64)


# ---------------------------------------------------------------- cut order
# One background cell [0,1]^3 (N = 1) holding three triangles, and a fourth
# triangle outside the cell (y = 2) that only a count over the whole mesh
# would see.
#   T0 in z = 0.5, x, y in [0.1, 0.9]           (area 0.32)
#   T1 in x = 0.4, y in [0.05, 0.8], z in [0.2, 0.8] (right triangle, area 0.225)
#   T2 in y = 0.7, x in [0.5, 0.9], z in [0.6, 0.9]  (area 0.06)
#   T3 in y = 2,   x in [0.6, 0.8], z in [0.3, 0.7]  (area 0.04, not in the cell)
# Counts within the cell: T0's plane crosses T1 only (1); T1's plane crosses
# T0 only (1); T2's plane crosses T0 and T1 (2).  Ascending with ties by index
# gives T0, T1, T2.  (Descending: T2 first; ties by descending index: T1
# first; counting T3 too: T0 would count 2 and T1 would come first.)
CUT_TRIS = np.array([
    _tri((0.1, 0.1, 0.5), (0.9, 0.1, 0.5), (0.1, 0.9, 0.5)),
    _tri((0.4, 0.05, 0.2), (0.4, 0.8, 0.2), (0.4, 0.05, 0.8)),
    _tri((0.5, 0.7, 0.6), (0.9, 0.7, 0.6), (0.5, 0.7, 0.9)),
    _tri((0.6, 2.0, 0.3), (0.8, 2.0, 0.3), (0.6, 2.0, 0.7)),
])


def _cut_cell():
    PT = PlaneTable(1, CUT_TRIS)
    assoc = associate(PT, CUT_TRIS)
    assert sorted(assoc) == [0] and [t for t, _ in assoc[0]] == [0, 1, 2]
    return PT, assoc[0]


def test_cut_order_ascending_count_ties_by_index():
    PT, lst = _cut_cell()
    order = [t for t, _ in cut_order(PT, CUT_TRIS, lst)]
    assert order == [0, 1, 2]


def test_cut_tree_and_weights_by_area_in_node_region():
    """Splits: the root by T0 (z = 0.5); T1 reaches both children (it spans
    z 0.2..0.8) and splits each; T2 reaches only the upper child (z >= 0.6)
    and, inside it, only the side x > 0.4, where it splits once more.
    Weights over the total area 0.645: root 0.32; T1 below z = 0.5: 0.16875
    (the part of T1 above z = 0.5 is the similar triangle with legs 0.375 and
    0.3, area 0.05625, and 0.225 - 0.05625 = 0.16875); T1 above: 0.05625; T2:
    0.06."""
    PT, lst = _cut_cell()
    total = 0.32 + 0.225 + 0.06 + 0.04
    tree = build_tree(PT, CUT_TRIS, total, 0, (0, 0, 0), cut_order(PT, CUT_TRIS, lst))
    internal = [nd for nd in tree.nodes if not nd.is_leaf]
    got = {}
    for nd in internal:
        t = nd.pid - PT.ngrid
        if t == 1:
            # which side of z = 0.5 is this node's region on?
            zc = nd.poly.centroid[2]
            got[("T1", "below" if zc < 0.5 else "above")] = nd.w
        else:
            got[("T%d" % t,)] = nd.w
    expect = {("T0",): 0.32 / total, ("T1", "below"): 0.16875 / total, ("T1", "above"): 0.05625 / total,
              ("T2",): 0.06 / total}
    assert set(got) == set(expect)
    for k in expect:
        assert abs(got[k] - expect[k]) <= 1e-14 * expect[k], (k, got[k], expect[k])
    assert tree.nodes[0].pid == PT.tri_pid(0)
    # T2 cuts the upper T1 child's side x > 0.4 only: four cuts, five leaves
    assert len(internal) == 4 and sum(nd.is_leaf for nd in tree.nodes) == 5


# ---------------------------------------------------------------- greedy removal
# A closed, outward-oriented box on the N = 4 grid (cells of 1/4), with
# dyadic extents so every piece area is exact:
#   x in [0.3125, 0.5625], y in [0.375, 0.578125], z in [0.28125, 0.59375].
# It lies in the 8 cells (i, j, k) in {1, 2}^3 and holds one corner in each.
# Per axis, the box part in cell index 1 / 2:
#   lx = 3/16, 1/16;  ly = 1/8, 5/64;  lz = 7/32, 3/32.
# Total area 2 (1/4 * 13/64 + 1/4 * 5/16 + 13/64 * 5/16) = 197/512.
# Triangles are listed face by face (x-, x+, y-, y+, z-, z+), so in every cell
# the three face planes tie at count 0 and are cut in index order: x, then y,
# then z, each tree a chain whose weights are the face pieces in the cell:
#   w_x = ly lz / A,  w_y = lx lz / A,  w_z = lx ly / A.
BOX_LO = (0.3125, 0.375, 0.28125)
BOX_HI = (0.5625, 0.578125, 0.59375)
LX = {1: F(3, 16), 2: F(1, 16)}
LY = {1: F(1, 8), 2: F(5, 64)}
LZ = {1: F(7, 32), 2: F(3, 32)}
AREA = F(197, 512)


def box_tris(lo=BOX_LO, hi=BOX_HI):
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    q = []
    # each face: two triangles, counter-clockwise seen from outside
    faces = [
        [(x0, y0, z0), (x0, y0, z1), (x0, y1, z1), (x0, y1, z0)],   # x-
        [(x1, y0, z0), (x1, y1, z0), (x1, y1, z1), (x1, y0, z1)],   # x+
        [(x0, y0, z0), (x1, y0, z0), (x1, y0, z1), (x0, y0, z1)],   # y-
        [(x0, y1, z0), (x0, y1, z1), (x1, y1, z1), (x1, y1, z0)],   # y+
        [(x0, y0, z0), (x0, y1, z0), (x1, y1, z0), (x1, y0, z0)],   # z-
        [(x0, y0, z1), (x1, y0, z1), (x1, y1, z1), (x0, y1, z1)],   # z+
    ]
    for a, b, c, d in faces:
        q.append(_tri(a, b, c))
        q.append(_tri(a, c, d))
    return np.array(q)


def _axis_of(G, r, n):
    t = G.trees[r].nodes[n].pid - G.PT.ngrid
    return "xyz"[(t // 2) // 2]


def _ijk(r, N=4):
    k, rem = divmod(r, N * N)
    j, i = divmod(rem, N)
    return (i, j, k)


def test_box_scene_weights_are_face_pieces():
    tris = box_tris()
    n = np.cross(tris[:, 1] - tris[:, 0], tris[:, 2] - tris[:, 0])
    c = tris.mean(axis=1) - 0.5 * (np.array(BOX_LO) + np.array(BOX_HI))
    assert np.all((n * c).sum(axis=1) > 0)          # outward
    G = build_cut_grid(4, tris)
    assert sorted(G.trees) == sorted(root_index(4, i, j, k) for i in (1, 2) for j in (1, 2) for k in (1, 2))
    assert abs(G.total_area - float(AREA)) <= 1e-16
    for r, tree in G.trees.items():
        i, j, k = _ijk(r)
        chain = [nd for nd in tree.nodes if not nd.is_leaf]
        assert [_axis_of(G, r, nd.id) for nd in chain] == ["x", "y", "z"]
        expect = {"x": LY[j] * LZ[k] / AREA, "y": LX[i] * LZ[k] / AREA, "z": LX[i] * LY[j] / AREA}
        for nd in chain:
            e = float(expect[_axis_of(G, r, nd.id)])
            assert abs(nd.w - e) <= 1e-15 * e


# Greedy removal with L = 5 (stop once the removed weight exceeds 1/5), worked
# by hand from the weights above (in units of 1/394):
#   candidates at the start are the z cuts: (2,2,1) 5, (2,2,2) 5, (2,1,1) 8,
#   (2,1,2) 8, (1,2,1) 15, (1,2,2) 15, (1,1,1) 24, (1,1,2) 24.
#   pop (2,2,1)z 5 [tie with (2,2,2), smaller cell index]  -> y of (2,2,1): 14
#   pop (2,2,2)z 5                                          -> y of (2,2,2): 6
#   pop (2,2,2)y 6                                          -> x of (2,2,2): 7.5
#   pop (2,2,2)x 7.5 (the whole cell becomes a cube)
#   pop (2,1,1)z 8                                          -> y of (2,1,1): 14
#   pop (2,1,2)z 8                                          -> y of (2,1,2): 6
#   pop (2,1,2)y 6                                          -> x of (2,1,2): 12
#   pop (2,1,2)x 12 (a cube)                 running sum 57.5 <= 78.8 (= 1/5)
#   pop (2,1,1)y 14 [tie with (2,2,1)y]      running sum 71.5 <= 78.8
#   pop (2,2,1)y 14                          running sum 85.5 >  78.8: stop.
GREEDY = [((2, 2, 1), "z"), ((2, 2, 2), "z"), ((2, 2, 2), "y"), ((2, 2, 2), "x"), ((2, 1, 1), "z"),
          ((2, 1, 2), "z"), ((2, 1, 2), "y"), ((2, 1, 2), "x"), ((2, 1, 1), "y"), ((2, 2, 1), "y")]


def test_greedy_removal_min_first_until_over_one_over_L():
    G = build_cut_grid(4, box_tris())
    st = HierarchyState(G)
    st.aggregate()
    st.remove_cuts(5)
    got = [(_ijk(r), _axis_of(G, r, n)) for r, n in st.removed]
    assert got == GREEDY
    assert st.full == {root_index(4, 2, 2, 2), root_index(4, 2, 1, 2)}
    assert {(2, 2, 2), (2, 1, 2)} <= set(st.cubes)


def test_hierarchy_levels_of_box_scene():
    """Level 1 of the box scene, from the removal above: the two fully
    collapsed cells are single cubes, (2,2,1) keeps only its x cut (two
    cells: one fluid, one holding the box corner, which is kept because it
    contains a finest fluid cell), (2,1,1) likewise, and the other four trees
    keep their three cuts (their finest fluid leaves, three each)."""
    G = build_cut_grid(4, box_tris())
    lv = build_hierarchy(G, 5)
    nodes = [c for c in lv[1].cells if c[0] == "node"]
    per = {}
    for c in nodes:
        per.setdefault(_ijk(c[1]), []).append(c[2])
    assert {k: len(v) for k, v in per.items()} == {(1, 1, 1): 3, (1, 2, 1): 3, (1, 1, 2): 3, (1, 2, 2): 3,
                                                    (2, 1, 1): 2, (2, 2, 1): 2}
    cubes = {c[1] for c in lv[1].cells if c[0] == "cube"}
    assert (2, 2, 2) in cubes and (2, 1, 2) in cubes
