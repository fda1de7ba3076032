"""Oracle: nested, boundary-aware grid hierarchy (Sec. 5.2).

TEST INFRASTRUCTURE ONLY (never imported by the product path).

Each coarsening iteration (L-1 of them) does, in the paper's order:
  (i)  aggregate regular cubes 2x2x2: an aligned block becomes one cube of
       twice the size when all 8 members are current single cubes of the same
       size s that hold fluid (reading: keeps coarse cells convex; a background
       cell whose cuts were all removed counts as a cube).  With `balance`
       (the default) also every fluid cell touching the block (faces, edges,
       corners) must have size >= s before the step (2:1 balance, the usual
       practice of geometric multigrid on locally refined grids; without it
       coarse cubes next to the boundary band collect hundreds of hanging
       vertices and their cliques grow); balance=False is the rule as
       Sec. 5.2 prints it;
  (ii) greedily remove removable cuts (internal BSP nodes whose two children
       are current leaves), smallest weight first (ties: background cell
       index, node preorder id), until the removed weight of this iteration
       exceeds 1/L; the weights are summed as integers round(w * 2^40);
  (iii) extract: a coarse cell is kept if it contains at least one finest
       fluid cell (reading of the contradictory extraction sentence: fluid
       cells are the retained "exterior" ones of Sec. 5.1).
Cells: ("cube", (i0,j0,k0), size) or ("node", r, node_id).  Canonical cell
order: (linear index of the background cell at the cell's min corner, node
preorder id; -1 for cubes).
"""
from __future__ import annotations

import heapq

import numpy as np

from .cutcell import SINGLE_FLUID, SINGLE_SOLID, TREE, UNCUT_FLUID, UNCUT_SOLID, CutGrid, root_index
from .geometry import cube_H


class Level:
    def __init__(self):
        self.cells = []          # canonical order; ("cube", ijk, size) / ("node", r, nid)
        self.index = {}          # cell -> position
        self.solid_pieces = []   # H lists of convex solid regions completing the tiling
        self.parent = None       # array: cell -> coarse cell position (set for l < L-1)


def cell_key(N, cell):
    if cell[0] == "cube":
        i, j, k = cell[1]
        return (root_index(N, i, j, k), -1)
    return (cell[1], cell[2])


def cell_H(G: CutGrid, cell):
    if cell[0] == "cube":
        i, j, k = cell[1]
        return cube_H(G.PT, i, j, k, cell[2])
    return G.trees[cell[1]].nodes[cell[2]].H


class HierarchyState:
    def __init__(self, G: CutGrid):
        self.G = G
        self.removed = []         # (root, node id) of every removed cut, in removal order
        N = G.N
        self.cubes = {}           # (i,j,k) -> size, fluid cube cells
        self.collapsed = {r: set() for r in G.trees}
        self.full = set()         # tree roots collapsed to a single cube
        for r in range(N ** 3):
            if G.kinds[r] in (UNCUT_FLUID, SINGLE_FLUID):
                k, rem = divmod(r, N * N)
                j, i = divmod(rem, N)
                self.cubes[(i, j, k)] = 1

    def current_leaf(self, r, nid):
        """Highest collapsed ancestor of node nid (or nid itself)."""
        nodes = self.G.trees[r].nodes
        best = nid
        a = nodes[nid].parent
        while a >= 0:
            if a in self.collapsed[r]:
                best = a
            a = nodes[a].parent
        return best

    def leaves(self, r):
        """Current leaves of tree r (preorder)."""
        nodes = self.G.trees[r].nodes
        out = []
        stack = [0]
        while stack:
            n = stack.pop()
            if nodes[n].is_leaf or n in self.collapsed[r]:
                out.append(n)
            else:
                stack.append(nodes[n].right)
                stack.append(nodes[n].left)
        return sorted(out)

    def extract(self) -> Level:
        G = self.G
        N = G.N
        lv = Level()
        cells = [("cube", ijk, s) for ijk, s in self.cubes.items()]
        for r, tree in G.trees.items():
            if r in self.full:
                continue
            for n in self.leaves(r):
                if tree.nodes[n].nfluid > 0:
                    cells.append(("node", r, n))
                else:
                    lv.solid_pieces.append(tree.nodes[n].H)
        for r, tree in G.trees.items():
            if r in self.full and tree.nodes[0].nfluid == 0:
                lv.solid_pieces.append(tree.nodes[0].H)
        for r in range(N ** 3):
            if G.kinds[r] in (UNCUT_SOLID, SINGLE_SOLID):
                k, rem = divmod(r, N * N)
                j, i = divmod(rem, N)
                lv.solid_pieces.append(cube_H(G.PT, i, j, k, 1))
        cells.sort(key=lambda c: cell_key(N, c))
        lv.cells = cells
        lv.index = {c: p for p, c in enumerate(cells)}
        return lv

    def sizes_of_roots(self):
        """Size of the current fluid cell holding each background cell (0 if none)."""
        G = self.G
        N = G.N
        sz = np.zeros((N, N, N), dtype=np.int64)           # indexed [k, j, i]
        for (i, j, k), s in self.cubes.items():
            sz[k:k + s, j:j + s, i:i + s] = s
        for r, tree in G.trees.items():
            if r not in self.full and tree.nodes[0].nfluid > 0:
                k, rem = divmod(r, N * N)
                jj, ii = divmod(rem, N)
                sz[k, jj, ii] = 1
        return sz

    def aggregate(self, balance=True):
        N = self.G.N
        sz = self.sizes_of_roots()
        new = dict(self.cubes)
        for (i, j, k), s in sorted(self.cubes.items(), key=lambda kv: root_index(N, *kv[0])):
            s2 = 2 * s
            if i % s2 or j % s2 or k % s2 or i + s2 > N or j + s2 > N or k + s2 > N:
                continue
            members = [(i + di * s, j + dj * s, k + dk * s)
                       for dk in (0, 1) for dj in (0, 1) for di in (0, 1)]
            if not all(self.cubes.get(m) == s for m in members):
                continue
            # the block and its one-cell shell: the block holds size-s cubes only,
            # so a size below s can only come from a neighbour
            near = sz[max(0, k - 1):k + s2 + 1, max(0, j - 1):j + s2 + 1, max(0, i - 1):i + s2 + 1]
            if balance and np.any((near > 0) & (near < s)):
                continue
            for m in members:
                del new[m]
            new[(i, j, k)] = s2
        self.cubes = new

    def remove_cuts(self, L):
        G = self.G
        limit = int(round(2 ** 40)) // L   # floor(2^40 / L) in integer units
        heap = []

        def removable(r, n):
            nodes = G.trees[r].nodes
            nd = nodes[n]
            if nd.is_leaf or n in self.collapsed[r]:
                return False
            for c in (nd.left, nd.right):
                if not (nodes[c].is_leaf or c in self.collapsed[r]):
                    return False
            return self.current_leaf(r, n) == n

        for r, tree in G.trees.items():
            if r in self.full:
                continue
            for nd in tree.nodes:
                if removable(r, nd.id):
                    heapq.heappush(heap, (nd.wq, r, nd.id))
        acc = 0
        while heap and acc <= limit:
            wq, r, n = heapq.heappop(heap)
            self.collapsed[r].add(n)
            self.removed.append((r, n))
            acc += wq
            p = G.trees[r].nodes[n].parent
            if p >= 0 and removable(r, p):
                heapq.heappush(heap, (G.trees[r].nodes[p].wq, r, p))
            if p < 0:
                self.full.add(r)
                if G.trees[r].nodes[0].nfluid > 0:
                    self.cubes[G.trees[r].ijk] = 1

    def map_cell(self, cell):
        """Cell of the current state that contains the given (older) cell."""
        if cell[0] == "cube":
            ijk = self._cube_containing(*cell[1])
            return ("cube", ijk, self.cubes[ijk])
        r, n = cell[1], cell[2]
        if r in self.full:
            ijk = self._cube_containing(*self.G.trees[r].ijk)
            return ("cube", ijk, self.cubes[ijk])
        return ("node", r, self.current_leaf(r, n))

    def _cube_containing(self, i, j, k):
        s = 1
        while s <= self.G.N:
            c = (i - i % s, j - j % s, k - k % s)
            if self.cubes.get(c) == s:
                return c
            s *= 2
        raise KeyError((i, j, k))


def build_hierarchy(G: CutGrid, L: int = 5, balance: bool = True):
    """Returns the list of L levels (0 = finest) with parent maps."""
    st = HierarchyState(G)
    levels = [st.extract()]
    for _ in range(L - 1):
        st.aggregate(balance)
        st.remove_cuts(L)
        lv = st.extract()
        prev = levels[-1]
        prev.parent = [lv.index[st.map_cell(c)] for c in prev.cells]
        levels.append(lv)
    return levels
