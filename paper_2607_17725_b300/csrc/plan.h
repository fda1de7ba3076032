// Integer plan of the solver built on the host from the topology: free-DOF
// numbering, sparsity patterns (structural clique unions), prolongation row
// patterns, sliced-ELL layouts and the index maps the device kernels use.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "topo.h"

namespace fvem {

constexpr int SELL_C = 32;  // rows per slice (one warp)

struct LevelPlan {
  int nv = 0, nc = 0, ndof = 0;
  std::vector<int32_t> dof_of_vertex, vertex_of_dof;
  // Element vertex lists: the DOFs an element block K^E couples.  Level 0:
  // the cell's vertices.  Coarser levels: the sorted union of the cell's
  // vertices and the prolongation columns of its children's element lists,
  // so K^C = sum_e P_e^T K^e P_e is the exact Galerkin block for any P; it
  // equals the cell list whenever the prolongation is local to the parent
  // (elem_is_cell), which exact geometry guarantees (Sec. 4.3).
  std::vector<int32_t> elem_vptr, elem_v;
  bool elem_is_cell = true;
  std::vector<int64_t> kptr;                       // nc+1 offsets of n_E^2 element blocks (element lists)
  std::vector<int32_t> inc_ptr, inc_cell, inc_loc; // vertex -> (cell, index in its element list)
  std::vector<int64_t> a_rowptr;                   // CSR of A over free DOFs
  std::vector<int32_t> a_col;
  int64_t nslices = 0;
  std::vector<int64_t> sell_ptr;                   // nslices+1
  std::vector<int32_t> sell_w;                     // width per slice
  std::vector<int32_t> sell_col;                   // padded columns (pad = own row)
  bool sell_d16 = false;                           // every column - row offset fits 16 bits
  std::vector<int16_t> sell_dcol;                  // column - row (pad: own row, or row n-1 past the end)
  std::vector<int64_t> sell_of_csr;                // csr nnz -> sell slot
  // prolongation from the next coarser level (only levels < L-1)
  std::vector<int32_t> prow_ptr, prow_col;         // full rows over all vertices, coarse vertex ids
  std::vector<int64_t> pf_rowptr, pf_src;          // free rows/cols: rows = free DOFs here
  std::vector<int32_t> pf_col;                     //   cols = free DOFs of level l+1
  std::vector<int64_t> pt_rowptr, pt_src;          // transpose of pf
  std::vector<int32_t> pt_col;
  // children: cells of level l-1 grouped by their parent cell of this level
  std::vector<int32_t> child_ptr, child_cell;
  int max_nv = 0, max_nf = 0, max_ne = 0;         // cell vertices, cell faces, element list length
  bool has_inflow = false;
};

int build_plan(const Topology& T, std::vector<LevelPlan>& plan, std::string& err);

// Second-order (k = 2) DOFs of one level (Sec. 3.1): the vertices, then one per
// edge (sorted by (smaller, larger) vertex id), one per face (sorted by its
// sorted vertex ids; a face shared by two cells is one DOF), one per cell.
// Element DOF lists follow the element order: the cell's vertices ascending,
// its edges sorted, its faces in the cell's face order, the cell DOF.
// Dirichlet (y = 1, |y - 1| <= 1e-10): vertices on the plane, edges with both
// ends on it, faces with all vertices on it.
struct DofsK2 {
  int64_t nv = 0, ne = 0, nf = 0, nc = 0, n = 0;
  std::vector<int64_t> elem_ptr;  // nc + 1
  std::vector<int64_t> elem_dof;
  std::vector<uint8_t> dirichlet; // n
  // free DOFs (not Dirichlet) in global order, and the pattern of A over them:
  // the union of the cells' element-list cliques (structural)
  std::vector<int64_t> free_of;     // n: free index or -1
  std::vector<int64_t> a_rowptr;
  std::vector<int64_t> a_col;
};

void build_dofs_k2(const LevelMesh& M, DofsK2& D);

// Pattern of the k = 2 prolongation from coarse level Cm to fine level F over
// all DOFs (rows: fine k = 2 DOFs, columns: coarse ones), sorted columns.
// Point DOFs (vertices, edge midpoints) use the DOFs of the coarse entity that
// holds them: vertex; edge (its two vertices and its midpoint DOF); face (its
// vertices, edge midpoints and face DOF); cell (the cell's element list).
// Face-mean DOFs use the coarse face or cell that holds the face's centroid;
// cell-mean DOFs use the parent cell.  The containing fine cell of a vertex,
// edge or face is the first in cell order.
void build_prolongation_pattern_k2(const LevelMesh& F, const LevelMesh& Cm, const DofsK2& Df, const DofsK2& Dc,
                                   std::vector<int64_t>& rowptr, std::vector<int64_t>& col);

}  // namespace fvem
