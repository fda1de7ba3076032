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
                                   std::vector<int64_t>& rowptr, std::vector<int64_t>& col, bool naive = false);

// ------------------------------------------------------------------ k = 2
// The second-order solver works on the condensed system (reading K2): the
// cell-mean DOFs are eliminated per cell, so the unknowns of every level are
// its free "boundary" DOFs (vertices, edges, faces; global ids < cdof).  The
// level's LevelPlan then describes that system with the boundary ids in the
// role the vertices play for k = 1 (dof_of_vertex / vertex_of_dof over ids <
// cdof, element lists = each cell's sorted boundary ids, incidence, pattern,
// sliced-ELL layout, prolongation rows over fine boundary ids with coarse
// boundary columns).  LevelK2 holds what the k = 2 kernels need besides.
struct LevelK2 {
  DofsK2 D;            // all k = 2 DOFs (element order per cell: vertices, edges, faces, cell)
  int64_t cdof = 0;    // first cell-DOF id (nv + ne + nf)
  // element-order tables of the element kernel
  std::vector<int32_t> edge_ptr;  // nc + 1: local edges per cell
  std::vector<int32_t> edge_v;    // two global vertex ids (u < w) per local edge, sorted
  std::vector<int32_t> fpos_v;    // per face_v entry: local vertex index of cycle[m]
  std::vector<int32_t> fpos_e;    // per face_v entry: local edge index of (cycle[m], cycle[m+1])
  std::vector<int32_t> perm;      // per element-order entry: position in the sorted boundary list (-1: cell DOF)
  std::vector<int64_t> k2_off;    // nc + 1: offsets of the n_E^2 element matrices
  std::vector<int64_t> face_off;  // n_face_occ + 1: offsets of the face data
  int max_ne = 0, max_nf = 0, max_fk = 0;
  // prolongation into this level from level l+1 (rows: this level's boundary
  // ids; the columns, coarse boundary ids, are LevelPlan::prow_col in the
  // order the kernel writes them):
  //   kind 0: coarse vertex a (weight 1)
  //   kind 1: point on the coarse edge (a, b): columns a, b, edge DOF
  //   kind 2: point on coarse face occurrence a: its cycle vertices, cycle
  //           edge DOFs, face DOF (the face projector's order)
  //   kind 3: point in coarse cell C: C's element DOFs but the cell DOF
  //   kind 4: mean over fine face occurrence b of coarse face occurrence a
  //   kind 5: mean over fine face occurrence b of coarse cell C
  // points: 3 doubles per row (kinds 0-3)
  std::vector<int8_t> pk;
  std::vector<int32_t> pC, pa, pb;
  std::vector<double> px;
};

// Build the condensed k = 2 plan of every level (LevelPlan fields as described
// above, LevelK2 alongside).  Returns 0 on success.
// naive: the naive prolongation of Eq. 16 (only fine vertices on coarse
// vertices are copied; every other fine DOF from the parent cell's Pi_2)
int build_plan_k2(const Topology& T, std::vector<LevelPlan>& plan, std::vector<LevelK2>& k2, std::string& err,
                  bool naive = false);

}  // namespace fvem
