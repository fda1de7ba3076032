// Host-side cut-cell topology and grid hierarchy (the precompute of Alg. 1).
//
// Builds, from a closed obstacle triangle soup and an N^3 background grid, the
// binary-space-partition cut cells (Sec. 5.1), the nested boundary-aware
// hierarchy (Sec. 5.2), one conforming polyhedral mesh per level with a
// canonical numbering, and the placement of every fine vertex in the next
// coarser mesh that the diffusion-free prolongation needs (Sec. 4.3, Eq. 17).
// All geometric decisions follow fixed FP64 evaluation rules (see topo.cpp),
// so the integer topology is reproducible bit for bit.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace fvem {

struct LevelMesh {
  int nv = 0;
  std::vector<double> V;              // 3*nv, canonical vertex order
  int nc = 0;
  std::vector<int32_t> cell_vptr;     // nc+1
  std::vector<int32_t> cell_v;        // sorted vertex ids per cell
  std::vector<int32_t> cell_fptr;     // nc+1, faces per cell (canonical order)
  std::vector<int32_t> face_pid;      // plane id of each face occurrence
  std::vector<int8_t> face_sg;        // outward sign
  std::vector<int32_t> face_vptr;     // nfaces+1
  std::vector<int32_t> face_v;        // vertex cycles, CCW about the outward normal
  std::vector<int32_t> parent;        // coarse cell of each cell (empty on the coarsest level)
};

// Placement of a fine vertex in the coarse mesh (Eq. 17 reading).
enum PlaceType : int8_t { PLACE_VERTEX = 0, PLACE_EDGE = 1, PLACE_FACE = 2, PLACE_CELL = 3 };

struct Placement {
  std::vector<int8_t> type;           // per fine vertex
  std::vector<int32_t> cell;          // coarse cell used for the placement
  std::vector<int32_t> a, b;          // vertex: a; edge: a,b (coarse vertex ids); face: a = face occurrence index
};

// Placement of point x relative to coarse cell C of level mesh Cm (coarse
// vertex, edge interior, face, or cell; see Placement for a, b).
void classify_point(const LevelMesh& Cm, int C, const double* x, int8_t& type, int32_t& a, int32_t& b);

struct Topology {
  int N = 0, L = 0;
  std::vector<LevelMesh> levels;
  std::vector<Placement> place;       // place[l]: level l vertices in level l+1 mesh
  double total_area = 0.0;
  int64_t n_trees = 0;
};

// Returns 0 on success; on failure a message in err.  balance: 2x2x2
// aggregation only where every fluid cell touching the block is at least as
// large as its members (2:1 balance); false aggregates every block of 8 equal
// cubes, as the hierarchy rule of Sec. 5.2 states it.
// naive: prolongation placements of Eq. 16 (a new fine vertex on a coarse
// edge or face is placed in its parent cell) instead of Eq. 17
int build_topology(int N, const double* tris, int ntri, int L, bool balance, Topology& out, std::string& err,
                   bool naive = false);

}  // namespace fvem
