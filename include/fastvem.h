/*
 * fastvem.h -- C ABI of the B300 cut-cell VEM pressure projection.
 *
 * The library computes the pressure projection of "Fast VEM Fluid Simulation"
 * (Zhang & Ren, ACM TOG 45(4), 2026): Alg. 1 precompute (body-fitted grid,
 * Sec. 5.1; nested boundary-aware hierarchy, Sec. 5.2; diffusion-free
 * prolongation and Galerkin coarse operators A_c = P^T A_f P, Sec. 4.3, Eq. 15
 * and Eq. 17) and the projection step (right-hand side, Sec. 3.2; multigrid
 * preconditioned CG with a Chebyshev V-cycle, Sec. 4 and Sec. 6; velocity
 * correction, Sec. 3.3).  First-order VEM (k = 1) on the first-order velocity
 * space, Delta t = 1.
 *
 * Conventions for every entry point:
 *  - pointers named d_* are device pointers on the context's device, h_* are
 *    host pointers; the caller owns all input and output buffers, the context
 *    owns everything it allocates;
 *  - device work is issued on the stream given to fvem_create; calls return
 *    after that stream has been synchronised, so outputs are ready;
 *  - inputs are never modified;
 *  - no exception crosses the ABI; on error a status is returned, the context
 *    stays valid (a failed build leaves it unbuilt), and fvem_last_error()
 *    gives a one-line reason;
 *  - a context is not thread-safe; different contexts are independent.
 */
#ifndef FASTVEM_H
#define FASTVEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fvem_ctx fvem_ctx;

typedef enum {
  FVEM_OK = 0,
  FVEM_EINVAL = 1,     /* bad argument or call order                              */
  FVEM_ENOMEM = 2,     /* device or host allocation failed                        */
  FVEM_EGEOM = 3,      /* degenerate input or topology (non-nested, empty level)  */
  FVEM_ENOCONV = 4,    /* CG reached max_iters before rel_tol                     */
  FVEM_EBREAKDOWN = 5, /* CG breakdown: p^T A p <= 0 or r^T z <= 0                */
  FVEM_ENAN = 6,       /* NaN or Inf met in the input or in a reduction           */
  FVEM_ECUDA = 7,      /* a CUDA call failed (message in fvem_last_error)         */
  FVEM_ENODEV = 8,     /* no CUDA device: only host-side calls are available      */
  FVEM_ETIMEOUT = 9    /* a bounded wait inside a persistent kernel ran out (the
                          kernel stopped cleanly; the context was reset)         */
} fvem_status;

typedef enum {
  FVEM_PREC_FP64 = 0,  /* V-cycle and CG in FP64                                  */
  FVEM_PREC_FP32 = 1,  /* FP32 V-cycle (level values and vectors) inside FP64 CG  */
  FVEM_PREC_BF16 = 2,  /* FP32 V-cycle whose level matrices (all but the coarsest)
                          are read as packed BF16 values, accumulated in FP32;
                          the coarsest CG keeps FP32 values; FP64 outer CG      */
  FVEM_PREC_FP16 = 3   /* as FVEM_PREC_BF16 with packed FP16 (binary16) values:
                          eleven significand bits against BF16's eight, range
                          6e-8 (subnormal) to 65504; values below round to 0  */
} fvem_precision;

typedef enum {
  FVEM_COARSE_CHEBYSHEV = 0, /* coarsest level: Chebyshev of degree coarse_degree  */
  FVEM_COARSE_CG = 1         /* coarsest level: coarse_degree plain CG iterations  */
} fvem_coarse_solver;

typedef struct {
  int order_k;        /* VEM order: 1 or 2 (second order needs levels >= 2)        */
  int levels;         /* hierarchy levels L (Sec. 6: 5)                           */
  int cheb_degree;    /* Chebyshev smoother degree per sweep (default 5)          */
  int coarse_degree;  /* coarsest level: Chebyshev degree or CG iterations (80)    */
  int precision;      /* fvem_precision                                           */
  double rel_tol;     /* stop when ||r_k|| / ||r_0|| <= rel_tol                   */
  int max_iters;      /* CG iteration cap                                         */
  int coarse_solver;  /* fvem_coarse_solver (default FVEM_COARSE_CG)              */
  int balance;        /* hierarchy (Sec. 5.2): 1 (default) aggregates a 2x2x2
                         block of equal cubes only where every fluid cell
                         touching it is at least as large as its members (2:1
                         balance); 0 aggregates every such block, as Sec. 5.2
                         states the rule                                        */
  int naive_prolongation; /* 0 (default): the diffusion-free prolongation
                         (Eq. 17); 1: the naive VEM prolongation of Eq. 16,
                         for the ablation: fine vertices on coarse vertices
                         copy them, and every other fine DOF (a vertex on a
                         coarse edge or face too; for k = 2 also edge
                         midpoints and face means) is that functional of its
                         parent cell's projector Pi_k                      */
} fvem_params;

typedef struct {
  int N;              /* background resolution                                    */
  int levels;
  int order_k;        /* VEM order of the context                                 */
  int64_t n_cells[16];    /* fluid cells per level                                */
  int64_t n_vertices[16]; /* mesh vertices per level                              */
  int64_t n_dofs[16];     /* unknowns of the CG / V-cycle system per level: free
                             vertices (k = 1), free vertex, edge and face DOFs
                             of the condensed system (k = 2)                    */
  int64_t n_dofs_all[16]; /* all pressure DOFs per level: vertices (k = 1), or
                             vertices + edges + faces + cells (k = 2)           */
  int64_t nnz[16];        /* stored nonzeros of A_l                               */
  int64_t nnz_p[16];      /* stored nonzeros of P_l (level l+1 -> l)              */
  int64_t n_trees;        /* background cells split by the BSP                    */
  double lmax[16];        /* Chebyshev upper bounds per level                     */
  int coarse_mode;        /* FP64 coarsest CG chosen at build: 0 one cooperative
                             launch, 1 kernel sequence replayed from a graph,
                             2 persistent launch with the level's matrix in
                             shared memory                                      */
  double coarse_ms[2];    /* build-time timing of one FP64 coarsest solve, [0]
                             cooperative (best shape), [1] kernel sequence        */
  int sell_cfg64[16];     /* tuned sliced-ELL launch shape per level, FP64 and   */
  int sell_cfg32[16];     /* FP32: (gathers in flight, warps per slice) =
                             (2,1) (4,1) (2,2) (4,2) (2,4) (4,4) (2,8) (4,8) (8,1) (8,2)
                             (16,1) (16,2)                                      */
  int coarse_cfg[2];      /* tuned product shape of the coarsest kernel-sequence
                             CG: [0] FP64, [1] FP32 (the FP32 V-cycle's); 0-11 as
                             sell_cfg64, 12-17 a mixed split (each slice gets the
                             fewest of 1, 2, 4, 8 warps that keep its slots per
                             warp under a bound): (gathers in flight, bound) =
                             (4,8) (4,12) (4,16) (8,16) (8,24) (8,32); -1 where
                             not built                                          */
  double coarse_ms32;     /* build-time timing of one FP32 coarsest solve as a
                             kernel sequence (best shape)                       */
  int coarse_mode32;      /* FP32 coarsest CG chosen at build: 0 cooperative,
                             1 kernel sequence, 2 persistent (shared-memory
                             matrix), -1 not built                              */
  double coarse_ms32_coop; /* build-time timing of one FP32 coarsest solve as
                             one cooperative launch (best shape and grid)       */
  int64_t stencil_slices32[16]; /* per level, stencil slices of the FP32 copy:
                             32 rows whose entries all sit at lattice positions
                             of their vertex (uncut cubes, walls, removed
                             Dirichlet neighbours), with columns in runs of
                             three consecutive indices per line; the FP32
                             V-cycle reads their values from a class table and
                             their columns from eight 16-bit line offsets per
                             row (the stored products up to summation order)    */
  int64_t stencil_classes32[16]; /* distinct 27-value rows (classes) per level */
  int stencil_used32[16]; /* 1 where the build-time tuner kept the stencil
                             slices for the level's FP32 products               */
  double coarse_ms_persist[2]; /* build-time timing of one coarsest solve in the
                             persistent form, [0] FP64, [1] FP32 (0: the level
                             does not fit in shared memory, or not built)      */
  int persist_ctas;       /* CTAs of the persistent form (one per SM)         */
  double setup_s[2];      /* wall time of the last set-up: [0] topology and plan
                             (host, A0-A1 and patterns), [1] device build
                             (elements, P, Galerkin, assembly, bounds, tuning)  */
} fvem_info;

typedef struct {
  int iters;          /* CG iterations taken                                      */
  double rel_res;     /* final ||r|| / ||r0|| (FP64, recomputed r)                */
  double r0_norm;     /* ||r0|| = ||b||                                           */
  double solve_ms;    /* device time of the CG loop (CUDA events)                 */
  double total_ms;    /* device time of RHS + CG + correction                     */
} fvem_solve_stats;

/* Default parameters: k=1, L=5, Chebyshev degree 5, coarsest CG 80 iterations,
 * FP64, rel_tol 1e-6, 500 iterations, 2:1 balance on. */
void fvem_default_params(fvem_params* p);

/* Create a context bound to the current CUDA device and `cuda_stream`
 * (a cudaStream_t, NULL = legacy default stream).  Host-only use (topology
 * export) works without a device. */
fvem_status fvem_create(const fvem_params* params, void* cuda_stream, fvem_ctx** out);
void fvem_destroy(fvem_ctx* ctx);

/* A0-A1 (Sec. 5.1-5.2): cut-cell grid, hierarchy, conforming level meshes and
 * prolongation placements, on the host.  h_tris: ntri triangles, 9 doubles
 * each (v0,v1,v2), closed and outward oriented, inside or crossing [0,1]^3.
 * N in [2,1024].  Needs no device. */
fvem_status fvem_build_topology(fvem_ctx* ctx, int N, const double* h_tris, int ntri);

/* A0-A6: fvem_build_topology, then on the device: per-cell projectors and
 * element matrices (Sec. 3.1), assembly of A_0, diffusion-free prolongations
 * (Eq. 17) and Galerkin operators A_{l+1} = P^T A_l P (Eq. 15) per coarse
 * cell, Chebyshev bounds, coarsest-level setup. */
fvem_status fvem_build(fvem_ctx* ctx, int N, const double* h_tris, int ntri);

fvem_status fvem_query(const fvem_ctx* ctx, fvem_info* out);

/* Integer topology of level l for parity checks (host copies).  Pass NULL to
 * get only the sizes.  Sizes: counts[0]=n_vertices, [1]=n_cells,
 * [2]=len(cell_v), [3]=n_face_occurrences, [4]=len(face_v).
 * h_V: 3*n_vertices doubles; cell_vptr: n_cells+1; face_vptr: n_faces+1;
 * cell_fptr: n_cells+1; face_pid: n_faces; face_sg: n_faces (int8);
 * parent: n_cells (or nothing on the coarsest level). */
fvem_status fvem_export_level(const fvem_ctx* ctx, int level, int64_t* counts, double* h_V,
                              int32_t* h_cell_vptr, int32_t* h_cell_v, int32_t* h_cell_fptr,
                              int32_t* h_face_vptr, int32_t* h_face_v, int32_t* h_face_pid,
                              int8_t* h_face_sg, int32_t* h_parent);

/* Placement of level-l vertices in the level-(l+1) mesh (Eq. 17 reading):
 * type 0 vertex (a), 1 edge (a,b), 2 face (a = face occurrence), 3 cell;
 * cell = coarse cell used.  Arrays of n_vertices(l). */
fvem_status fvem_export_placement(const fvem_ctx* ctx, int level, int8_t* h_type, int32_t* h_cell,
                                  int32_t* h_a, int32_t* h_b);

/* Free-DOF numbering of level l: h_dof_of_vertex[v] = free index or -1. */
fvem_status fvem_export_dofs(const fvem_ctx* ctx, int level, int32_t* h_dof_of_vertex);

/* Second-order (k = 2) DOF numbering of level l (Sec. 3.1, the four DOF
 * families; host only, available after fvem_build_topology).  Global DOFs:
 * vertices, then edges sorted by (smaller, larger) vertex id, then faces
 * sorted by their sorted vertex ids (shared faces once), then cells.
 * counts[6] = {n, n_vertices, n_edges, n_faces, n_cells, element list length}
 * (call with null buffers first).  h_elem_ptr[n_cells + 1], h_elem_dof: each
 * cell's DOFs in element order (vertices ascending, edges sorted, faces in
 * the cell's face order, the cell); h_dirichlet[n]: 1 on the plane y = 1.
 * The solver itself is first order (order_k = 1); this export serves the
 * parity of the k = 2 numbering. */
fvem_status fvem_export_dofs_k2(const fvem_ctx* ctx, int level, int64_t* counts, int64_t* h_elem_ptr,
                                int64_t* h_elem_dof, uint8_t* h_dirichlet);

/* Pattern of the k = 2 operator of level l over its free DOFs (numbered in
 * global order, Dirichlet DOFs skipped): the union of the cells' element-list
 * cliques, CSR with sorted columns.  counts[2] = {rows, nonzeros} (call with
 * null buffers first); h_rowptr[rows + 1], h_col[nonzeros].  Host only. */
fvem_status fvem_export_pattern_k2(const fvem_ctx* ctx, int level, int64_t* counts, int64_t* h_rowptr,
                                   int64_t* h_col);

/* Pattern of the k = 2 prolongation from level l+1 to level l (Sec. 4.2,
 * Eq. 17, extended to the k = 2 DOFs) over all DOFs: row i lists the coarse
 * DOFs of the coarse entity holding fine DOF i (a point DOF's vertex, edge,
 * face or cell; a face mean's coarse face or cell; a cell mean's parent).
 * counts[3] = {fine DOFs, coarse DOFs, nonzeros} (null buffers first);
 * h_rowptr[fine DOFs + 1], h_col (sorted per row).  Host only. */
fvem_status fvem_export_prolongation_pattern_k2(const fvem_ctx* ctx, int level, int64_t* counts,
                                                int64_t* h_rowptr, int64_t* h_col);

/* CSR of A_l (FP64 values) or of P_l (level l+1 -> l; rows = free DOFs of l,
 * columns = free DOFs of l+1), copied to the host.  which: 0 = A, 1 = P.
 * Pass NULL pointers to get sizes in counts[0]=rows, [1]=cols, [2]=nnz. */
fvem_status fvem_export_matrix(const fvem_ctx* ctx, int which, int level, int64_t* counts,
                               int64_t* h_rowptr, int32_t* h_col, double* h_val);

/* Per-cell projector data of level 0 (host copies, n_cells entries):
 * vol, centroid (3), h_E, and the element matrices (n_E^2 per cell, row-major,
 * local order = ascending vertex id). Pass NULL for parts not wanted. */
fvem_status fvem_export_cells(const fvem_ctx* ctx, double* h_vol, double* h_centroid, double* h_h,
                              double* h_K);

/* A7-A13: one pressure projection (Sec. 3.2-3.3, Sec. 4).
 * d_u:        3*n_vertices(0) doubles, SoA (all x, then y, then z): the
 *             intermediate velocity u' at the level-0 vertices;
 * u_inflow:   uniform inflow speed through the x = 0 face (0 = wall);
 * d_p:        out, n_dofs_all(0) doubles: pressure at every vertex (k = 1),
 *             or at every k = 2 DOF in the numbering of fvem_export_dofs_k2
 *             (vertex values, edge midpoints, face means, cell means; the
 *             cell means recovered from the condensed solve), 0 on the
 *             Dirichlet face y = 1;
 * d_cellpoly: out, 12*n_cells(0) doubles: per cell the linear velocity
 *             Pi_1 u_new, [cell][component][monomial 1, x, y, z] in the scaled
 *             monomials of the cell (centroid, diameter h_E);
 * stats:      out (may be NULL).
 * Second order (order_k = 2, Sec. 3.1-3.3 with the k = 2 DOFs): the cell-mean
 * DOFs are condensed out per cell, CG runs on the remaining DOFs with the
 * diagonally scaled V-cycle, u_inflow must be 0.
 * Returns FVEM_ENOCONV / FVEM_EBREAKDOWN / FVEM_ENAN from the solve (outputs
 * then hold the last iterate). */
fvem_status fvem_project(fvem_ctx* ctx, const double* d_u, double u_inflow, double* d_p,
                         double* d_cellpoly, fvem_solve_stats* stats);

/* Same computation from host buffers: h_u is copied to the device, the results
 * are copied back (h_p, h_cellpoly may be NULL). */
fvem_status fvem_project_host(fvem_ctx* ctx, const double* h_u, double u_inflow, double* h_p,
                              double* h_cellpoly, fvem_solve_stats* stats);

/* A15: n independent projections run in lockstep.  Every scene keeps its own
 * context (hierarchy, tuned launch shapes, V-cycle graph) and its own stream;
 * the host issues one CG step of every unconverged scene, then waits once
 * for all of them, so kernels of different scenes overlap on the device and
 * converged scenes drop out (per-scene convergence mask).  Arrays of n:
 * contexts (distinct, each built; give them distinct non-null streams for
 * overlap), device velocities, inflow speeds (NULL = all 0), device outputs
 * as for fvem_project, stats (may be NULL).  Returns the first non-OK status
 * of any scene (its message in that scene's fvem_last_error); the others
 * still finish. */
fvem_status fvem_project_batched(fvem_ctx* const* ctxs, int n, const double* const* d_u, const double* u_inflow,
                                 double* const* d_p, double* const* d_cellpoly, fvem_solve_stats* stats);

/* Apply the V-cycle preconditioner once: d_z = M^{-1} d_r on free DOFs of
 * level 0 (n_dofs[0] doubles each), in the context's precision. */
fvem_status fvem_vcycle(fvem_ctx* ctx, const double* d_r, double* d_z);

/* y = A_l x on free DOFs of level l (FP64).  For order_k = 2, A_0 is the
 * condensed operator and the coarser A_l are diagonally scaled (the V-cycle's
 * operators). */
fvem_status fvem_spmv(fvem_ctx* ctx, int level, const double* d_x, double* d_y);

/* Second-order element data of level l (host copies, after fvem_build with
 * order_k = 2), every cell in element order (vertex values ascending,
 * edge midpoints by sorted edge, face means in the cell's face order, the
 * cell mean): h_K the element matrices K^E (n_E^2 per cell, row-major),
 * h_Pis the projectors Pi* (10 x n_E per cell, row-major; monomials 1, x,
 * y, z, xx, xy, xz, yy, yz, zz scaled by the centroid and diameter), h_mom
 * the cell moments int_E m_a (10 per cell).  counts[3] = {len(K), len(Pis),
 * len(mom)} (pass NULL buffers first).  Sec. 3.1, Eq. 11-14 for k = 2. */
fvem_status fvem_export_elements_k2(const fvem_ctx* ctx, int level, int64_t* counts, double* h_K, double* h_Pis,
                                    double* h_mom);

/* Adjoint of fvem_project (the map u', u_inflow -> cellpoly is affine):
 * given d_gcell (12*n_cells(0)), returns d_gu (3*n_vertices(0), SoA) and
 * *h_ginflow = dL/du_inflow, using the same hierarchy for the transposed
 * (symmetric) solve. */
fvem_status fvem_project_adjoint(fvem_ctx* ctx, const double* d_gcell, double* d_gu, double* h_ginflow,
                                 fvem_solve_stats* stats);

/* Measurement hook (not part of the paper's method): when on, every launch of
 * the dominant kernel -- the fused level-0 Chebyshev step (sliced-ELL product
 * plus three vector updates) -- is bracketed by CUDA events on the context
 * stream.  fvem_get_profile returns the launches and their summed device time
 * since the last fvem_set_profiling call, and the algorithmic bytes of one
 * launch: nnz_g*(s_v + s_i) + 17*n_s + 6*n*s_v (values and columns of the
 * generic rows once; per row of an FP32 stencil slice its class byte and
 * eight 16-bit line offsets; the gathered vector, x, r read once; x, r, d
 * written), nnz_g = stored
 * nonzeros outside the stencil slices used, n_s = their rows, s_v = 8 (FP64)
 * or 4, s_i = 2 when the level stores 16-bit column offsets, else 4. */
fvem_status fvem_set_profiling(fvem_ctx* ctx, int on);
fvem_status fvem_get_profile(fvem_ctx* ctx, int64_t* launches, double* total_ms, double* bytes_per_launch);

/* Switch the V-cycle precision of a built context.  FP64 is always
 * available; FP32 only if the context was created with FVEM_PREC_FP32,
 * FVEM_PREC_BF16 or FVEM_PREC_FP16 (which keep FP32 copies of the level
 * operators next to the FP64 ones); BF16 and FP16 only if it was created with
 * one of those two, which also keep a packed 16-bit copy of the level values
 * (all levels but the coarsest): built from the FP64 values in the creation
 * format, and re-packed from the FP32 copy when the other format is selected.  In FP32 the whole V-cycle, its coarsest-level CG
 * included, runs on the FP32 copies (the coarsest CG forms its inner
 * products in FP64, or in float-float arithmetic in its persistent form); the
 * outer CG is FP64 in every mode. */
fvem_status fvem_set_precision(fvem_ctx* ctx, int precision);

/* Change the CG stopping rule of a context. */
fvem_status fvem_set_tolerance(fvem_ctx* ctx, double rel_tol, int max_iters);

/* Replay the V-cycle of the CG loop from a CUDA graph (default on; captured
 * on first use on an internal stream, launched on the context stream).  Off:
 * every kernel is launched one by one. */
fvem_status fvem_set_graphs(fvem_ctx* ctx, int on);

/* Override the Chebyshev upper bound lambda_max of level l (the smoother's
 * interval becomes [lmax/30, lmax]); the build estimates it by Lanczos.  A
 * bound far below the true largest eigenvalue makes the V-cycle indefinite,
 * and CG then stops with FVEM_EBREAKDOWN.  lmax must be finite and > 0. */
fvem_status fvem_set_cheb_lmax(fvem_ctx* ctx, int level, double lmax);

/* Use (on = 1) or skip (0) the stencil slices of level l in the FP32 V-cycle
 * (the build-time tuner picks one per level; fvem_query's stencil_used32
 * reports the current choice).  FVEM_EINVAL if the level has none. */
fvem_status fvem_set_stencil(fvem_ctx* ctx, int level, int on);

/* Number of kernels this context has launched so far (all entry points;
 * kernels inside a graph replay count once per replay). */
fvem_status fvem_launch_count(const fvem_ctx* ctx, int64_t* n);

/* Not in the paper (it has no counterpart there): fvem_vcycle without any
 * device allocation, for callers that may not call cudaMalloc once set-up is
 * done (a pre-planned memory budget, a pool that owns the device, a host that
 * forbids allocation on its serving path).  Same arguments and result as
 * fvem_vcycle in FP64: d_z = M^{-1} d_r on the free DOFs of level 0.
 * The work vectors of all levels live in one file-scope device array of
 * 2^21 doubles (16 MiB) that every device loading the library holds until
 * the process exits; a hierarchy that needs more than
 * 5 * sum_l n_dofs(l) + n_dofs(coarsest) + 4 * max(cooperative blocks of the
 * FP64 and FP32 coarsest CG) doubles (the level vectors, the coarsest CG's
 * extra vector and its reduction slots) is rejected with FVEM_EINVAL, and so
 * is a second-order context.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress) with that device
 * current; make that first call before any stream capture.  All calls share
 * the array and it keeps the last call's contents (every vector is written
 * before it is read); calls that overlap on the GPU, from any context or
 * stream, race on it.  No cudaMalloc, cudaFree or allocating library call. */
fvem_status fvem_vcycle_static(fvem_ctx* ctx, const double* d_r, double* d_z);

/* VEM element quality indicator (Eq. 18 and App. C; grid value Eq. 19) of
 * the cells of a level, as a diagnostic of the grid (not part of the solve):
 *   rho(E) = sqrt(rho1 rho2 + rho1 rho3) / 2 with
 *   rho1 = |k(E)|/|E| prod_f |k(f)|/|f| (kernel ratios; 1 for the convex
 *          cells and faces these grids consist of),
 *   rho2 = min(|E|^(1/3), min_f h_f)/h_E + (1/#f) sum_f min(|f|^(1/2), min_e |e|)/h_f,
 *   rho3 = 4/#f + (1/#f) sum_f 3/#e_f (h: diameters; the face term reads the
 *          printed cube root of the face area as its square root),
 * and rho(P) = the root mean square of rho(E) over the cut cells (cells that
 * are not axis-aligned cubes).
 * d_rho:  n_cells(level) doubles on the device (cell order of
 *         fvem_export_level), or NULL;
 * h_grid: rho(P), NaN when the level has no cut cell (host, may be NULL);
 * h_ncut: the number of cut cells (host, may be NULL).
 * FVEM_EINVAL for a bad level or an unbuilt context; FVEM_EGEOM if a cell is
 * not convex to 1e-8 in distance (its kernel is not computed; its rho is
 * NaN). */
fvem_status fvem_quality(fvem_ctx* ctx, int level, double* d_rho, double* h_grid, int64_t* h_ncut);

/* ---- Particle transfers around the projection (Sec. 3.2, Sec. 3.3) ----
 * Particles live in [0,1]^3.  Layouts (device pointers, on the context's
 * stream; every call synchronises it before returning):
 *   d_xp:   3*n doubles, SoA (all x, then y, then z);
 *   d_cell: n int32, the level-0 cell holding each particle, -1 inside an
 *           obstacle or outside the box (fvem_locate writes it; G2P and
 *           advection leave particles with an id outside [0, n_cells(0))
 *           as they are);
 *   vertex fields: n_ch*n_vertices(0) doubles, SoA, in the vertex order of
 *           fvem_export_level(0);
 *   d_cellpoly: 12*n_cells(0) doubles as fvem_project writes them.
 * The first particle call of a built context bins the level-0 cells and
 * the obstacle triangles by background cube (host set-up, kept until the
 * next build).  All four need a built context (FVEM_EINVAL otherwise) and
 * 0 <= n < 2^31; they work for order_k 1 and 2 (the level-0 mesh and its
 * first-order projectors are the same). */

/* P2G (Sec. 3.2): vertex value i = sum_p f_p w_ip / sum_p w_ip with
 * w_ip = max(0, 1 - |x_p - x_i|^2 / R^2)^3 and R = 1/N (the background
 * grid's edge), 0 where no particle is within R.  d_fp: n_ch*n doubles SoA
 * (n_ch in 1..4); d_fv: out, n_ch*n_vertices(0) doubles; d_cell may be NULL
 * (every particle with finite coordinates counts), else particles with
 * cell -1 are skipped.  Distances and sums in FP32 on offsets from each
 * particle's background cube (relative error about 1e-6 of the largest
 * |f_p|), the quotient in FP64; the result does not depend on the order of
 * the particles in memory beyond their ids (bitwise reproducible while no
 * background cube holds more than 1024 particles; a fuller cube's sums
 * follow the order of atomic updates and differ between runs by rounding). */
fvem_status fvem_p2g(fvem_ctx* ctx, int64_t n, const double* d_xp, const int32_t* d_cell, int n_ch,
                     const double* d_fp, double* d_fv);

/* The level-0 cell of every particle: the lowest-numbered cell of its
 * background cube whose closed face half-spaces hold it within 1e-10, -1
 * if none or outside [0,1]^3 (also for non-finite coordinates). */
fvem_status fvem_locate(fvem_ctx* ctx, int64_t n, const double* d_xp, int32_t* d_cell);

/* G2P (Sec. 3.3), FLIP/PIC blend: with Pi_1 u_old the cell polynomials of
 * d_u_old (3*n_vertices(0), the P2G velocity before forces) and Pi_1 u_new
 * = d_cellpoly (the projection's output), every particle with cell >= 0 takes
 *   u_p <- alpha (u_p + (Pi_1 u_new - Pi_1 u_old)(x_p)) + (1 - alpha) Pi_1 u_new(x_p)
 * (the standard blend: the printed update's increment read inside the FLIP
 * weight).  d_up: in/out, 3*n SoA.  alpha in [0, 1], else FVEM_EINVAL. */
fvem_status fvem_g2p(fvem_ctx* ctx, int64_t n, const double* d_xp, const int32_t* d_cell, const double* d_u_old,
                     const double* d_cellpoly, double alpha, double* d_up);

/* Advection (Sec. 3.3): one midpoint Runge-Kutta step of every particle with
 * cell >= 0 in the velocity d_cellpoly: x_m = x + dt/2 v(x), x_new = x + dt
 * v(x_m).  Each stage's end point: mirrored across the plane of the first
 * obstacle triangle its segment crosses (least parameter, ties to the lower
 * triangle index), then across any box wall it passed, then kept only if it
 * lies in a fluid cell (else the particle stays at the stage's start).
 * d_xp and d_cell: in/out.  dt finite and >= 0, else FVEM_EINVAL; a stage
 * spanning more than 3 background cubes along an axis leaves that particle
 * in place and the call returns FVEM_EINVAL (reduce dt). */
fvem_status fvem_advect(fvem_ctx* ctx, int64_t n, double dt, const double* d_cellpoly, double* d_xp,
                        int32_t* d_cell);

/* Failure-path hook (for tests; not part of the paper's method): sets the
 * abort word of the persistent coarsest-level CG, which its CTAs otherwise
 * set when a bounded wait runs out.  Its next launch then leaves before its
 * first copy through the same exit: the call that issued it (fvem_project,
 * fvem_vcycle, ...) returns FVEM_ETIMEOUT, its outputs are not valid, and the
 * context is reset, so the following calls run normally.  No GPU fault or
 * hang is involved.  FVEM_EINVAL when the context is not built or its
 * coarsest CG does not use the persistent form in either precision. */
fvem_status fvem_arm_coarse_abort(fvem_ctx* ctx);

const char* fvem_status_str(fvem_status s);
const char* fvem_last_error(const fvem_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* FASTVEM_H */
