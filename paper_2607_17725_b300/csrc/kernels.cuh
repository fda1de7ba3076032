// Device kernels of the cut-cell VEM pressure projection (sm_103a).
//
// Element kernels (precompute): one warp per polyhedral cell.  Solve kernels:
// sliced-ELL (32 rows per slice, one warp per slice, column-major slots so each
// step of the row loop is one coalesced 32-wide load of values and of column
// indices), Chebyshev steps fused with the sparse product, deterministic
// reductions (fixed per-block trees, then one block over the partials).
#pragma once
#include <cooperative_groups.h>
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <type_traits>

namespace fvem {

constexpr int RED_THREADS = 256;
constexpr int RED_BLOCKS = 592;  // 4 x 148 SMs

struct MeshView {
  const double* V;
  const int32_t* cell_vptr;
  const int32_t* cell_v;
  const int32_t* cell_fptr;
  const int32_t* face_vptr;
  const int32_t* face_v;
  const int32_t* face_pid;
  const int8_t* face_sg;
  int nc;
};

template <typename T>
struct SellView {
  const int64_t* ptr;
  const int32_t* w;
  const int32_t* col;   // absolute columns (32-bit), or
  const int16_t* dcol;  // column - row (16-bit), when every offset of the level fits
  const T* val;
  int64_t n;   // rows
  int64_t ns;  // slices of 32 rows
  // Stencil slices: reg[s] == 2 marks a slice whose 32 rows are stencil rows
  // (every entry at a lattice position of the row's vertex); they take the
  // first nsched_st entries of the block schedule below.  The row in lane
  // `lane` of schedule entry q has class c = cls[32 q + lane]; its 27 values
  // are the class row stc[28 c ..] (28 floats per class, the last one zero
  // padding for 16-byte loads; zero where an entry is missing); slot
  // j = 3k + dx + 1 (k = 3 (dz+1) + (dy+1), dx = -1, 0, 1) is column
  // row + line(k) + dx, with line(4) = 0 and the other eight line offsets in
  // lines[8 (32 q + lane) + k'] (k' = k, or k - 1 past 4; 16 bytes per row).
  // Stored by schedule position, they load in the same round as the slice id;
  // no values or column offsets are read, and all 27 gathers issue after it.
  const uint8_t* reg;  // per slice, or null
  const T* stc;        // class table, 28 values per class
  const uint8_t* cls;  // class per row, by schedule position
  const int16_t* lines;
  // Block schedule where a level has lattice slices: slot q of the launch
  // takes slice order[q] (-1: none); lattice slices come first, then the
  // others, each list padded to a multiple of 8, so that no block mixes the
  // short lattice warps with the long generic ones (a block holds its SM
  // slots until its slowest warp ends).
  const int32_t* order;  // or null: slot q takes slice q
  int64_t nsched;
  // Packed BF16 copy of the values (FP32 V-cycle only): when set, the product
  // reads the stored values from here, converts them to T and accumulates in T.
  const __nv_bfloat16* valb = nullptr;
  // Packed FP16 copy of the values, read the same way (at most one of valb,
  // valh is set)
  const __half* valh = nullptr;
  // schedule entries of the stencil part (the first entries of `order`, a
  // multiple of 8)
  int64_t nsched_st = 0;
  // per slice: its schedule position if a stencil slice, else -1; set by
  // launches whose `order` is another list (the stencil data stay indexed by
  // the level's schedule position)
  const int32_t* stpos = nullptr;
};



// slice groups (blocks of 8 / KS slices) a plain launch over A covers
template <int KS, typename T>
__host__ __device__ __forceinline__ int64_t sell_groups(const SellView<T>& A) {
  return (A.ns + 8 / KS - 1) / (8 / KS);
}

__device__ __forceinline__ double warp_sum_bcast(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return __shfl_sync(0xffffffffu, v, 0);
}
__device__ __forceinline__ double warp_max_bcast(double v) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  return __shfl_sync(0xffffffffu, v, 0);
}

struct D3 {
  double x, y, z;
};
__device__ __forceinline__ D3 ld3(const double* V, int g) { return D3{V[3 * g], V[3 * g + 1], V[3 * g + 2]}; }
__device__ __forceinline__ D3 sub3(D3 a, D3 b) { return D3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ D3 add3(D3 a, D3 b) { return D3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ D3 mul3(D3 a, double s) { return D3{a.x * s, a.y * s, a.z * s}; }
__device__ __forceinline__ D3 crs3(D3 a, D3 b) {
  return D3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double dt3(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// Face quantities of a CCW cycle: area, unit normal, area centroid, vertex mean.
__device__ inline void face_geom(const double* V, const int32_t* cyc, int k, double& area, D3& n, D3& cen,
                                 D3& xbar) {
  D3 A{0, 0, 0}, m{0, 0, 0};
  for (int q = 0; q < k; ++q) {
    D3 p = ld3(V, cyc[q]), pn = ld3(V, cyc[(q + 1) % k]);
    A = add3(A, crs3(p, pn));
    m = add3(m, p);
  }
  A = mul3(A, 0.5);
  area = sqrt(dt3(A, A));
  n = mul3(A, 1.0 / area);
  xbar = mul3(m, 1.0 / k);
  D3 p0 = ld3(V, cyc[0]);
  D3 c{0, 0, 0};
  double tot = 0.0;
  for (int q = 1; q + 1 < k; ++q) {
    D3 a = ld3(V, cyc[q]), b = ld3(V, cyc[q + 1]);
    double t = 0.5 * dt3(crs3(sub3(a, p0), sub3(b, p0)), n);
    c = add3(c, mul3(add3(add3(p0, a), b), t / 3.0));
    tot += t;
  }
  cen = mul3(c, 1.0 / tot);
}

// ---------------------------------------------------------------- A2 / A3
// Per cell (one warp): volume, centroid, diameter h_E, the k=1 projector
// coefficients Pi* = G^{-1} B (4 x n_E, stored row-major at 4*cell_vptr[c]),
// and optionally the element matrix
//   K^E = Pi*^T Gt Pi* + h_E (I - Pi)^T (I - Pi),  Pi = D Pi*   (Sec. 3.1),
// formed through the 4x4 middle matrix M = Gt + h_E D^T D, so the cost is
// O(n_E^2) per cell.  Face integrals of phi_i use the 2D face projector
// (enhanced face space): int_f phi_i = |f| (1/k + g_i.(x_f - xbar_f)).
__global__ void k_cell_vem(MeshView m, int maxf, double* vol_o, double* xE_o, double* h_o, double* Pis,
                           const int64_t* kptr, double* Kel) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  double* fg = smem + size_t(warp) * maxf * 10;
  for (int c = blockIdx.x * wpb + warp; c < m.nc; c += gridDim.x * wpb) {
    const int vb = m.cell_vptr[c], nv = m.cell_vptr[c + 1] - vb;
    const int fb = m.cell_fptr[c], nf = m.cell_fptr[c + 1] - fb;
    D3 c0{0, 0, 0};
    for (int i = lane; i < nv; i += 32) c0 = add3(c0, ld3(m.V, m.cell_v[vb + i]));
    c0 = D3{warp_sum_bcast(c0.x) / nv, warp_sum_bcast(c0.y) / nv, warp_sum_bcast(c0.z) / nv};
    double vol = 0.0;
    D3 cc{0, 0, 0};
    for (int f = lane; f < nf; f += 32) {
      const int s = m.face_vptr[fb + f], k = m.face_vptr[fb + f + 1] - s;
      double area;
      D3 n, cen, xbar;
      face_geom(m.V, m.face_v + s, k, area, n, cen, xbar);
      double* g = fg + f * 10;
      g[0] = area;
      g[1] = n.x; g[2] = n.y; g[3] = n.z;
      g[4] = cen.x; g[5] = cen.y; g[6] = cen.z;
      g[7] = xbar.x; g[8] = xbar.y; g[9] = xbar.z;
      D3 a = ld3(m.V, m.face_v[s]);
      for (int q = 1; q + 1 < k; ++q) {
        D3 b = ld3(m.V, m.face_v[s + q]), d = ld3(m.V, m.face_v[s + q + 1]);
        double t = dt3(sub3(a, c0), crs3(sub3(b, c0), sub3(d, c0))) / 6.0;
        vol += t;
        cc = add3(cc, mul3(add3(add3(add3(c0, a), b), d), t / 4.0));
      }
    }
    vol = warp_sum_bcast(vol);
    D3 xE{warp_sum_bcast(cc.x) / vol, warp_sum_bcast(cc.y) / vol, warp_sum_bcast(cc.z) / vol};
    double h2 = 0.0;
    for (int p = lane; p < nv * nv; p += 32) {
      int i = p / nv, j = p % nv;
      if (j <= i) continue;
      D3 d = sub3(ld3(m.V, m.cell_v[vb + i]), ld3(m.V, m.cell_v[vb + j]));
      h2 = fmax(h2, dt3(d, d));
    }
    const double h = sqrt(warp_max_bcast(h2));
    __syncwarp();
    double* Pc = Pis + 4 * size_t(vb);
    D3 mean{0, 0, 0};
    for (int i = lane; i < nv; i += 32) {
      const int gv = m.cell_v[vb + i];
      D3 B{0, 0, 0};
      for (int f = 0; f < nf; ++f) {
        const int s = m.face_vptr[fb + f], k = m.face_vptr[fb + f + 1] - s;
        int pos = -1;
        for (int q = 0; q < k; ++q)
          if (m.face_v[s + q] == gv) { pos = q; break; }
        if (pos < 0) continue;
        const double* g = fg + f * 10;
        D3 n{g[1], g[2], g[3]}, cen{g[4], g[5], g[6]}, xbar{g[7], g[8], g[9]};
        D3 pn = ld3(m.V, m.face_v[s + (pos + 1) % k]), pp = ld3(m.V, m.face_v[s + (pos + k - 1) % k]);
        D3 gv3 = mul3(crs3(sub3(pn, pp), n), 1.0 / (2.0 * g[0]));
        double fi = g[0] * (1.0 / k + dt3(gv3, sub3(cen, xbar)));
        B = add3(B, mul3(n, fi / h));
      }
      const double sc = h * h / vol;
      Pc[1 * nv + i] = B.x * sc;
      Pc[2 * nv + i] = B.y * sc;
      Pc[3 * nv + i] = B.z * sc;
      mean = add3(mean, mul3(sub3(ld3(m.V, gv), xE), 1.0 / h));
    }
    mean = D3{warp_sum_bcast(mean.x) / nv, warp_sum_bcast(mean.y) / nv, warp_sum_bcast(mean.z) / nv};
    for (int i = lane; i < nv; i += 32)
      Pc[i] = 1.0 / nv - (mean.x * Pc[nv + i] + mean.y * Pc[2 * nv + i] + mean.z * Pc[3 * nv + i]);
    if (lane == 0) {
      vol_o[c] = vol;
      xE_o[3 * c] = xE.x;
      xE_o[3 * c + 1] = xE.y;
      xE_o[3 * c + 2] = xE.z;
      h_o[c] = h;
    }
    __syncwarp();
    if (Kel) {
      double DtD[10];
#pragma unroll
      for (int q = 0; q < 10; ++q) DtD[q] = 0.0;
      for (int i = lane; i < nv; i += 32) {
        D3 y = mul3(sub3(ld3(m.V, m.cell_v[vb + i]), xE), 1.0 / h);
        double d[4] = {1.0, y.x, y.y, y.z};
        int q = 0;
        for (int a = 0; a < 4; ++a)
          for (int b = a; b < 4; ++b) DtD[q++] += d[a] * d[b];
      }
      double M[4][4];
      {
        int q = 0;
        for (int a = 0; a < 4; ++a)
          for (int b = a; b < 4; ++b) {
            double v = h * warp_sum_bcast(DtD[q++]);
            if (a == b && a > 0) v += vol / (h * h);
            M[a][b] = v;
            M[b][a] = v;
          }
      }
      double* K = Kel + kptr[c];
      for (int p = lane; p < nv * nv; p += 32) {
        const int i = p / nv, j = p % nv;
        D3 yi = mul3(sub3(ld3(m.V, m.cell_v[vb + i]), xE), 1.0 / h);
        D3 yj = mul3(sub3(ld3(m.V, m.cell_v[vb + j]), xE), 1.0 / h);
        double Di[4] = {1.0, yi.x, yi.y, yi.z}, Dj[4] = {1.0, yj.x, yj.y, yj.z};
        double Pi_[4], Pj[4];
        for (int a = 0; a < 4; ++a) {
          Pi_[a] = Pc[a * nv + i];
          Pj[a] = Pc[a * nv + j];
        }
        double cons = 0.0, PIij = 0.0, PIji = 0.0;
        for (int a = 0; a < 4; ++a) {
          double t = 0.0;
          for (int b = 0; b < 4; ++b) t += M[a][b] * Pj[b];
          cons += Pi_[a] * t;
          PIij += Di[a] * Pj[a];
          PIji += Dj[a] * Pi_[a];
        }
        K[p] = cons + h * ((i == j ? 1.0 : 0.0) - PIij - PIji);
      }
    }
  }
}

// ---------------------------------------------------------------- A4
// Row-owner assembly: thread per free row, contributions of every incident
// cell added in cell order into the row's own slots (deterministic, no atomics).
__global__ void k_assemble(int ndof, const int32_t* vertex_of_dof, const int32_t* dof_of_vertex,
                           const int32_t* inc_ptr, const int32_t* inc_cell, const int32_t* inc_loc,
                           const int32_t* cell_vptr, const int32_t* cell_v, const int64_t* kptr, const double* Kel,
                           const int64_t* rowptr, const int32_t* col, double* val, int* err) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ndof) return;
  const int64_t rs = rowptr[i], re = rowptr[i + 1];
  for (int64_t q = rs; q < re; ++q) val[q] = 0.0;
  const int v = vertex_of_dof[i];
  for (int q = inc_ptr[v]; q < inc_ptr[v + 1]; ++q) {
    const int c = inc_cell[q], a = inc_loc[q];
    const int vb = cell_vptr[c], n = cell_vptr[c + 1] - vb;
    const double* K = Kel + kptr[c] + int64_t(a) * n;
    for (int b = 0; b < n; ++b) {
      const int j = dof_of_vertex[cell_v[vb + b]];
      if (j < 0) continue;
      int64_t lo = rs, hi = re;
      while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (col[mid] < j) lo = mid + 1; else hi = mid;
      }
      if (lo >= re || col[lo] != j) { atomicExch(err, 1); continue; }
      val[lo] += K[b];
    }
  }
}

template <typename T>
__global__ void k_scatter_sell(int64_t nnz, const int64_t* sell_of_csr, const double* csr_val, T* sell_val) {
  int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < nnz) sell_val[sell_of_csr[k]] = T(csr_val[k]);
}
// packed BF16 copy of the values (round to nearest); padding slots stay 0
__global__ void k_scatter_sell_bf16(int64_t nnz, const int64_t* sell_of_csr, const double* csr_val,
                                    __nv_bfloat16* sell_val) {
  int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < nnz) sell_val[sell_of_csr[k]] = __double2bfloat16(csr_val[k]);
}
__global__ void k_scatter_sell_fp16(int64_t nnz, const int64_t* sell_of_csr, const double* csr_val,
                                    __half* sell_val) {
  int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k < nnz) sell_val[sell_of_csr[k]] = __double2half(csr_val[k]);
}
// A 16-bit plane re-packed from the FP32 copy of the same sliced-ELL slots
// (FP16 or BF16, round to nearest even).
__global__ void k_pack16(int64_t n, const float* __restrict__ in, void* out, int half) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    if (half)
      static_cast<__half*>(out)[i] = __float2half_rn(in[i]);
    else
      static_cast<__nv_bfloat16*>(out)[i] = __float2bfloat16_rn(in[i]);
  }
}

template <typename T>
__global__ void k_gather_vals(int64_t n, const int64_t* src, const double* from, double* to64, T* toT) {
  int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (k >= n) return;
  double v = from[src[k]];
  if (to64) to64[k] = v;
  if (toT) toT[k] = T(v);
}

// ---------------------------------------------------------------- A5
// Diffusion-free prolongation rows (Eq. 17 reading), one thread per fine
// vertex: copy / linear on a coarse edge / 2D face projector / 3D cell projector.
__global__ void k_prolong_rows(int nf, const double* Vf, const int8_t* type, const int32_t* pcell,
                               const int32_t* pa, const int32_t* pb, MeshView cm, const double* cPis,
                               const double* cxE, const double* ch, const int32_t* prow_ptr, double* prow_val) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nf) return;
  const D3 x = ld3(Vf, v);
  double* w = prow_val + prow_ptr[v];
  const int t = type[v];
  if (t == 0) {
    w[0] = 1.0;
  } else if (t == 1) {
    D3 a = ld3(cm.V, pa[v]), b = ld3(cm.V, pb[v]);
    D3 e = sub3(b, a);
    double tt = dt3(sub3(x, a), e) / dt3(e, e);
    w[0] = 1.0 - tt;
    w[1] = tt;
  } else if (t == 2) {
    const int f = pa[v];
    const int s = cm.face_vptr[f], k = cm.face_vptr[f + 1] - s;
    double area;
    D3 n, cen, xbar;
    face_geom(cm.V, cm.face_v + s, k, area, n, cen, xbar);
    for (int q = 0; q < k; ++q) {
      D3 pn = ld3(cm.V, cm.face_v[s + (q + 1) % k]), pp = ld3(cm.V, cm.face_v[s + (q + k - 1) % k]);
      D3 g = mul3(crs3(sub3(pn, pp), n), 1.0 / (2.0 * area));
      w[q] = 1.0 / k + dt3(g, sub3(x, xbar));
    }
  } else {
    const int C = pcell[v];
    const int vb = cm.cell_vptr[C], n = cm.cell_vptr[C + 1] - vb;
    const double* P = cPis + 4 * size_t(vb);
    const double h = ch[C];
    D3 y = mul3(sub3(x, D3{cxE[3 * C], cxE[3 * C + 1], cxE[3 * C + 2]}), 1.0 / h);
    for (int j = 0; j < n; ++j) w[j] = P[j] + y.x * P[n + j] + y.y * P[2 * n + j] + y.z * P[3 * n + j];
  }
}

// ---------------------------------------------------------------- A6
// Galerkin coarse element blocks without SpGEMM: K^C = sum_{e in C} P_e^T K^e P_e
// over element lists (sorted; every prolongation column of a child's list is
// in its parent's list by construction, so the sum is P^T A P exactly; with
// exact geometry the lists are the cells' vertices, Sec. 4.3).  P is the
// free-row restriction: a fine vertex with no DOF (f_dof < 0: Dirichlet, or
// referenced by no prolongation row) contributes nothing, which matters where
// a Dirichlet vertex's row reaches free coarse vertices (the naive
// prolongation of Eq. 16 places top-wall vertices in cells).  One thread per
// coarse cell, fixed summation order.
__global__ void k_galerkin(int ncc, const int32_t* child_ptr, const int32_t* child_cell, const int32_t* f_vptr,
                           const int32_t* f_v, const int64_t* f_kptr, const double* f_K, const int32_t* prow_ptr,
                           const int32_t* prow_col, const double* prow_val, const int32_t* f_dof,
                           const int32_t* c_vptr, const int32_t* c_v, const int64_t* c_kptr, double* c_K, int* err) {
  int C = blockIdx.x * blockDim.x + threadIdx.x;
  if (C >= ncc) return;
  const int cb = c_vptr[C], nC = c_vptr[C + 1] - cb;
  double* KC = c_K + c_kptr[C];
  for (int64_t q = 0; q < int64_t(nC) * nC; ++q) KC[q] = 0.0;
  auto loc = [&](int cv) -> int {
    int lo = 0, hi = nC;
    while (lo < hi) {
      int mid = (lo + hi) >> 1;
      if (c_v[cb + mid] < cv) lo = mid + 1; else hi = mid;
    }
    return (lo < nC && c_v[cb + lo] == cv) ? lo : -1;
  };
  for (int q = child_ptr[C]; q < child_ptr[C + 1]; ++q) {
    const int e = child_cell[q];
    const int eb = f_vptr[e], ne = f_vptr[e + 1] - eb;
    const double* Ke = f_K + f_kptr[e];
    for (int a = 0; a < ne; ++a) {
      const int ua = f_v[eb + a];
      if (f_dof[ua] < 0) continue;
      for (int pa = prow_ptr[ua]; pa < prow_ptr[ua + 1]; ++pa) {
        const int ia = loc(prow_col[pa]);
        if (ia < 0) { atomicExch(err, 2); continue; }
        const double wa = prow_val[pa];
        for (int b = 0; b < ne; ++b) {
          const double kab = wa * Ke[a * ne + b];
          if (kab == 0.0) continue;
          const int ub = f_v[eb + b];
          if (f_dof[ub] < 0) continue;
          for (int pb = prow_ptr[ub]; pb < prow_ptr[ub + 1]; ++pb) {
            const int jb = loc(prow_col[pb]);
            if (jb < 0) { atomicExch(err, 2); continue; }
            KC[int64_t(ia) * nC + jb] += kab * prow_val[pb];
          }
        }
      }
    }
  }
}

// The same Galerkin blocks with one warp per coarse cell.  Per child e, with
// P_e its prolongation rows (sparse, columns located in the coarse list):
//   T = K^e P_e     (n_e x n_C, in shared memory; lane a owns row a),
//   K^C += P_e^T T  (lane j owns column j of K^C),
// so every entry is accumulated by one lane in a fixed order (deterministic,
// no atomics).  K^C itself is accumulated in place in global memory.  tcap:
// doubles of shared memory per warp for T (n_e n_C <= tcap).
__device__ __forceinline__ int find_sorted(const int32_t* v, int n, int key) {
  int lo = 0, hi = n;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (v[mid] < key) lo = mid + 1; else hi = mid;
  }
  return (lo < n && v[lo] == key) ? lo : -1;
}

__global__ void k_galerkin_warp(int ncc, const int32_t* child_ptr, const int32_t* child_cell, const int32_t* f_vptr,
                                const int32_t* f_v, const int64_t* f_kptr, const double* f_K,
                                const int32_t* prow_ptr, const int32_t* prow_col, const double* prow_val,
                                const int32_t* f_dof, const int32_t* c_vptr, const int32_t* c_v,
                                const int64_t* c_kptr, double* c_K, int tcap, int* err) {
  extern __shared__ double gsm[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  double* T = gsm + size_t(warp) * tcap;
  for (int C = blockIdx.x * wpb + warp; C < ncc; C += gridDim.x * wpb) {
    const int cb = c_vptr[C], nC = c_vptr[C + 1] - cb;
    const int32_t* cv = c_v + cb;
    double* KC = c_K + c_kptr[C];
    for (int64_t q = lane; q < int64_t(nC) * nC; q += 32) KC[q] = 0.0;
    __syncwarp();
    for (int q = child_ptr[C]; q < child_ptr[C + 1]; ++q) {
      const int e = child_cell[q];
      const int eb = f_vptr[e], ne = f_vptr[e + 1] - eb;
      if (ne * nC > tcap) {
        if (lane == 0) atomicExch(err, 4);
        continue;
      }
      const double* Ke = f_K + f_kptr[e];
      // T = K^e P_e
      for (int a = lane; a < ne; a += 32)
        for (int j = 0; j < nC; ++j) T[a * nC + j] = 0.0;
      for (int b = 0; b < ne; ++b) {
        const int ub = f_v[eb + b];
        if (f_dof[ub] < 0) continue;
        for (int pb = prow_ptr[ub]; pb < prow_ptr[ub + 1]; ++pb) {
          const int jb = find_sorted(cv, nC, prow_col[pb]);
          if (jb < 0) {
            if (lane == 0) atomicExch(err, 2);
            continue;
          }
          const double w = prow_val[pb];
          for (int a = lane; a < ne; a += 32) T[a * nC + jb] += Ke[a * ne + b] * w;
        }
      }
      __syncwarp();
      // K^C += P_e^T T
      for (int a = 0; a < ne; ++a) {
        const int ua = f_v[eb + a];
        if (f_dof[ua] < 0) continue;
        for (int pa = prow_ptr[ua]; pa < prow_ptr[ua + 1]; ++pa) {
          const int ia = find_sorted(cv, nC, prow_col[pa]);
          if (ia < 0) continue;
          const double w = prow_val[pa];
          for (int j = lane; j < nC; j += 32) KC[int64_t(ia) * nC + j] += w * T[a * nC + j];
        }
      }
      __syncwarp();
    }
  }
}

// ---------------------------------------------------------------- A7 / A13 / A14 per-cell maps
// RHS (Sec. 3.2): local r_i = sum_c (Pi*_{1+c,i}/h) |E| s^c_1 with s^c = Pi* u'_c,
// plus the inflow term u_in int_f phi_i on faces of the x = 0 wall.
__global__ void k_rhs_local(MeshView m, const double* Pis, const double* vol, const double* hE, const double* u,
                            int64_t nvtx, double u_in, double* rloc) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.nc) return;
  const int vb = m.cell_vptr[c], n = m.cell_vptr[c + 1] - vb;
  const double* P = Pis + 4 * size_t(vb);
  double s0[3] = {0, 0, 0};
  for (int j = 0; j < n; ++j) {
    const int g = m.cell_v[vb + j];
    s0[0] += P[j] * u[g];
    s0[1] += P[j] * u[nvtx + g];
    s0[2] += P[j] * u[2 * nvtx + g];
  }
  const double f = vol[c] / hE[c];
  for (int i = 0; i < n; ++i)
    rloc[vb + i] = f * (P[n + i] * s0[0] + P[2 * n + i] * s0[1] + P[3 * n + i] * s0[2]);
  if (u_in != 0.0) {
    for (int fi = m.cell_fptr[c]; fi < m.cell_fptr[c + 1]; ++fi) {
      if (!(m.face_pid[fi] == 0 && m.face_sg[fi] < 0)) continue;
      const int s = m.face_vptr[fi], k = m.face_vptr[fi + 1] - s;
      double area;
      D3 nn, cen, xbar;
      face_geom(m.V, m.face_v + s, k, area, nn, cen, xbar);
      for (int q = 0; q < k; ++q) {
        D3 pn = ld3(m.V, m.face_v[s + (q + 1) % k]), pp = ld3(m.V, m.face_v[s + (q + k - 1) % k]);
        D3 g = mul3(crs3(sub3(pn, pp), nn), 1.0 / (2.0 * area));
        double phi = area * (1.0 / k + dt3(g, sub3(cen, xbar)));
        int gv = m.face_v[s + q], lo = 0, hi = n;
        while (lo < hi) {
          int mid = (lo + hi) >> 1;
          if (m.cell_v[vb + mid] < gv) lo = mid + 1; else hi = mid;
        }
        rloc[vb + lo] += u_in * phi;
      }
    }
  }
}

// Gather per-cell local values to free DOFs (or to all vertices when dof_of_vertex is null).
__global__ void k_gather_dofs(int n, const int32_t* vertex_of_dof, const int32_t* inc_ptr, const int32_t* inc_cell,
                              const int32_t* inc_loc, const int32_t* cell_vptr, const double* loc, double* out) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int v = vertex_of_dof ? vertex_of_dof[i] : i;
  double s = 0.0;
  for (int q = inc_ptr[v]; q < inc_ptr[v + 1]; ++q) s += loc[cell_vptr[inc_cell[q]] + inc_loc[q]];
  out[i] = s;
}

// Velocity correction (Sec. 3.3): Pi_1 u_new = Pi_1 u' - grad Pi_1 p, 12 numbers per cell.
__global__ void k_correct(MeshView m, const double* Pis, const double* hE, const double* u, int64_t nvtx,
                          const double* pv, double* out) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.nc) return;
  const int vb = m.cell_vptr[c], n = m.cell_vptr[c + 1] - vb;
  const double* P = Pis + 4 * size_t(vb);
  double s[3][4], gp[3] = {0, 0, 0};
  for (int cc = 0; cc < 3; ++cc)
    for (int a = 0; a < 4; ++a) s[cc][a] = 0.0;
  for (int j = 0; j < n; ++j) {
    const int g = m.cell_v[vb + j];
    const double uj[3] = {u[g], u[nvtx + g], u[2 * nvtx + g]};
    for (int a = 0; a < 4; ++a) {
      const double pa = P[a * n + j];
      s[0][a] += pa * uj[0];
      s[1][a] += pa * uj[1];
      s[2][a] += pa * uj[2];
    }
    const double pj = pv[g];
    gp[0] += P[n + j] * pj;
    gp[1] += P[2 * n + j] * pj;
    gp[2] += P[3 * n + j] * pj;
  }
  const double ih = 1.0 / hE[c];
  for (int cc = 0; cc < 3; ++cc) {
    out[12 * size_t(c) + 4 * cc] = s[cc][0] - gp[cc] * ih;
    for (int a = 1; a < 4; ++a) out[12 * size_t(c) + 4 * cc + a] = s[cc][a];
  }
}

// Adjoint pieces.  (a) local d(cellpoly)/dp ^T g: -sum_c g[c][0] Pi*_{1+c,i}/h
__global__ void k_adj_pcoef(MeshView m, const double* Pis, const double* hE, const double* g, double* loc) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.nc) return;
  const int vb = m.cell_vptr[c], n = m.cell_vptr[c + 1] - vb;
  const double* P = Pis + 4 * size_t(vb);
  const double* gc = g + 12 * size_t(c);
  const double ih = 1.0 / hE[c];
  for (int i = 0; i < n; ++i)
    loc[vb + i] = -(gc[0] * P[n + i] + gc[4] * P[2 * n + i] + gc[8] * P[3 * n + i]) * ih;
}
// (b) local velocity gradient: C_u^T g + R^T lambda, per cell and component.
__global__ void k_adj_u(MeshView m, const double* Pis, const double* vol, const double* hE, const double* g,
                        const double* lam_v, double* loc3, int64_t nloc) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.nc) return;
  const int vb = m.cell_vptr[c], n = m.cell_vptr[c + 1] - vb;
  const double* P = Pis + 4 * size_t(vb);
  const double* gc = g + 12 * size_t(c);
  const double f = vol[c] / hE[c];
  double a[3] = {0, 0, 0};
  for (int i = 0; i < n; ++i) {
    const double li = lam_v[m.cell_v[vb + i]];
    a[0] += P[n + i] * li;
    a[1] += P[2 * n + i] * li;
    a[2] += P[3 * n + i] * li;
  }
  for (int j = 0; j < n; ++j)
    for (int cc = 0; cc < 3; ++cc) {
      double s = f * a[cc] * P[j];
      for (int al = 0; al < 4; ++al) s += gc[4 * cc + al] * P[al * n + j];
      loc3[cc * nloc + vb + j] = s;
    }
}

// ---------------------------------------------------------------- A8 / A9 solve kernels
// Split sliced-ELL product: a block of 256 threads covers 8/KS slices; the KS
// warps of a slice take every KS-th slot of its rows (each warp load stays one
// coalesced 32-wide access), their partial sums meet in shared memory, and the
// first warp of the slice runs the epilogue epi(row, y) for rows < n.
// STC = false compiles the plain product, which ignores the stencil flags,
// the lattice offsets and the block schedule (correct on every level: marked
// slices keep their stored values and offsets); STC = true serves marked
// slices from the canonical row and follows the schedule.
// The nine line offsets of the stencil row in lane `lane` of schedule entry q
// (one 16-byte load; line 4 is the row's own line, offset 0).
template <typename T>
__device__ __forceinline__ void stencil_lines(const SellView<T>& A, int64_t q, int lane, int lo[9]) {
  const int4 v = __ldg(reinterpret_cast<const int4*>(A.lines) + (q * 32 + lane));
  const int w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const int o = int(int16_t(uint16_t((unsigned(w[k >> 1]) >> (16 * (k & 1))) & 0xffffu)));
    lo[k < 4 ? k : k + 1] = o;
  }
  lo[4] = 0;
}

template <int U, int KS, bool D16, bool STC = false, typename T, typename Epi>
__device__ __forceinline__ void sell_split(const SellView<T>& A, int64_t slice_group, const T* __restrict__ x,
                                           T* sh, Epi epi) {
  constexpr int SPB = 8 / KS;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int sib = warp / KS, part = warp % KS;
  const int64_t q = slice_group * SPB + sib;
  const int64_t s = (STC && A.order) ? (q < A.nsched ? int64_t(__ldg(A.order + q)) : int64_t(-1)) : q;
  T acc = T(0);
  if (s >= 0 && s < A.ns) {
    const int32_t row = int32_t(s * 32 + lane);
    // schedule position of a stencil slice (uniform over the warp), else -1
    int64_t qs = -1;
    if (STC && A.order != nullptr) qs = A.stpos != nullptr ? int64_t(__ldg(A.stpos + s)) : (q < A.nsched_st ? q : -1);
    const bool stq = qs >= 0;
    const int w = stq ? 0 : A.w[s];
    const int64_t base = stq ? 0 : A.ptr[s] + lane;
    T y[U];
#pragma unroll
    for (int u = 0; u < U; ++u) y[u] = T(0);
    int j = part;
    if (stq) {
      // lattice slice: the KS warps take lines k = part, part + KS, ...
      int lo[9];
      stencil_lines(A, qs, lane, lo);
      const T* tab = A.stc + 28 * int(__ldg(A.cls + qs * 32 + lane));
      const int last = int(A.n - 1);
      T t = T(0);
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        if (k % KS != part) continue;
        // missing neighbours carry value 0; their index is clamped in bounds
        const int c = row + lo[k];
        t += __ldg(tab + 3 * k) * __ldg(x + max(c - 1, 0)) + __ldg(tab + 3 * k + 1) * __ldg(x + c) +
             __ldg(tab + 3 * k + 2) * __ldg(x + min(c + 1, last));
      }
      y[0] = t;
    }
    // the value source is uniform over the launch: one loop per source
    auto slots = [&](auto valat) {
      for (; j + KS * (U - 1) < w; j += KS * U) {
        int c[U];
        T v[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (D16)
            c[u] = row + int(__ldg(A.dcol + base + (j + KS * u) * 32));
          else
            c[u] = __ldg(A.col + base + (j + KS * u) * 32);
          v[u] = valat(base + (j + KS * u) * 32);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) y[u] += v[u] * __ldg(x + c[u]);
      }
      for (; j < w; j += KS) {
        const int c = D16 ? row + int(__ldg(A.dcol + base + j * 32)) : __ldg(A.col + base + j * 32);
        y[0] += valat(base + j * 32) * __ldg(x + c);
      }
    };
    if (!std::is_same<T, double>::value && A.valb != nullptr)
      slots([&](int64_t i) { return T(__bfloat162float(__ldg(A.valb + i))); });
    else if (!std::is_same<T, double>::value && A.valh != nullptr)
      slots([&](int64_t i) { return T(__half2float(__ldg(A.valh + i))); });
    else
      slots([&](int64_t i) { return __ldg(A.val + i); });
    acc = y[0];
#pragma unroll
    for (int u = 1; u < U; ++u) acc += y[u];
  }
  if (KS > 1) {
    sh[threadIdx.x] = acc;
    __syncthreads();
    if (part == 0)
      for (int p = 1; p < KS; ++p) acc += sh[(sib * KS + p) * 32 + lane];
    __syncthreads();
  }
  if (part == 0 && s >= 0 && s < A.ns) {
    const int64_t row = s * 32 + lane;
    if (row < A.n) epi(row, acc);
  }
}

template <int KS>
__host__ __device__ constexpr int slices_per_block() {
  return 8 / KS;
}

// Stencil slices per warp of the Chebyshev launches' stencil blocks.
constexpr int kStencilPerWarp = 1;

// One warp per kStencilPerWarp stencil slices (schedule entries q, q + 8,
// ... < nsched_st): their slice ids, line offsets and classes load in one
// round, the epilogue's own-row operands (pre) in the next, together with the
// gathers they do not wait for, so each warp keeps the loads of several
// slices in flight; epi(row, y, pre(row)) then finishes each row.  Class
// rows come as float4 loads.
template <typename T, typename Pre, typename Epi>
__device__ __forceinline__ void stencil_warp(const SellView<T>& A, int64_t q0, const T* __restrict__ x, Pre pre,
                                             Epi epi) {
  static_assert(std::is_same<T, float>::value, "stencil slices are FP32");
  constexpr int NS = kStencilPerWarp;
  const int lane = threadIdx.x & 31;
  int s[NS], lo[NS][9], ci[NS];
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    const int64_t q = q0 + 8 * j;
    s[j] = __ldg(A.order + q);
    stencil_lines(A, q, lane, lo[j]);
    ci[j] = __ldg(A.cls + q * 32 + lane);
  }
  using PT = decltype(pre(0));
  PT P[NS];
#pragma unroll
  for (int j = 0; j < NS; ++j)
    if (s[j] >= 0) P[j] = pre(s[j] * 32 + lane);
  const int last = int(A.n - 1);
  T t[NS];
#pragma unroll
  for (int j = 0; j < NS; ++j) {
    t[j] = T(0);
    if (s[j] < 0) continue;  // schedule padding
    const int row = s[j] * 32 + lane;
    const float4* t4 = reinterpret_cast<const float4*>(A.stc) + 7 * ci[j];
#pragma unroll
    for (int g = 0; g < 3; ++g) {
      // coefficients 9g .. 9g + 8 (lines 3g .. 3g + 2) from float4 b .. b + 2
      constexpr int kb[3] = {0, 2, 4};
      const int b = kb[g], o = 9 * g - 4 * kb[g];
      const float4 f0 = __ldg(t4 + b), f1 = __ldg(t4 + b + 1), f2 = __ldg(t4 + b + 2);
      const float cf[12] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w, f2.x, f2.y, f2.z, f2.w};
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        // missing neighbours carry value 0; their index is clamped in bounds
        const int c = row + lo[j][3 * g + m];
        t[j] += cf[o + 3 * m] * __ldg(x + max(c - 1, 0)) + cf[o + 3 * m + 1] * __ldg(x + c) +
                cf[o + 3 * m + 2] * __ldg(x + min(c + 1, last));
      }
    }
  }
#pragma unroll
  for (int j = 0; j < NS; ++j)
    if (s[j] >= 0) epi(s[j] * 32 + lane, t[j], P[j]);
}

// Product launch of the Chebyshev kernels.  On stencil levels (STC, with a
// block schedule) launched with one warp per slice, the blocks of the generic
// slices, which take several times longer, are launched first (longest
// first, so they do not form the launch's tail), then the stencil blocks
// (stencil_warp).  pre(row) loads the epilogue's own-row operands; epi(row,
// y, pre(row)) finishes row `row`.
template <int U, int KS, bool D16, bool STC, typename T, typename Pre, typename Epi>
__device__ __forceinline__ void sell_any(const SellView<T>& A, const T* __restrict__ x, T* sh, Pre pre, Epi epi) {
  auto fin = [&](int64_t row, T y) { epi(row, y, pre(row)); };
  if constexpr (STC && KS == 1) {
    if (A.order != nullptr && A.nsched_st > 0) {
      const int64_t b = blockIdx.x, ngen = (A.nsched - A.nsched_st) / 8;
      if (b >= ngen)
        stencil_warp(A, (b - ngen) * 8 * kStencilPerWarp + (threadIdx.x >> 5), x, pre, epi);
      else
        sell_split<U, 1, D16, STC>(A, A.nsched_st / 8 + b, x, sh, fin);
      return;
    }
  }
  sell_split<U, KS, D16, STC>(A, blockIdx.x, x, sh, fin);
}

// Resident blocks of 256 threads per SM the Chebyshev kernels are compiled
// for (65536 registers / (256 x registers per thread)): 32 registers for the
// plain product with up to 4 gathers in flight (FP32: 8), 40 with 8 (FP32:
// 16), 64 with 16 FP64 gathers.
template <typename T, int U, int KS, bool STC>
__host__ __device__ constexpr int cheb_min_blocks() {
  constexpr bool f64 = sizeof(T) == 8;
  if (U >= 16) return f64 ? 4 : 6;
  if (U >= 8) return f64 ? 6 : 8;
  return 8;
}

template <typename T, int U = 4, int KS = 1, bool D16 = false>
__global__ void __launch_bounds__(256) k_spmv(SellView<T> A, const T* __restrict__ x, T* __restrict__ y) {
  __shared__ T sh[256];
  sell_split<U, KS, D16>(A, blockIdx.x, x, sh, [&](int64_t row, T v) { y[row] = v; });
}

// Chebyshev (Saad Alg. 12.1) first step from x0 = 0: d0 = b/theta, x = d0,
// r = b - A d0, d1 = c1 d0 + c2 r; with `fold`, x += d1 as well.
template <typename T, int U = 4, int KS = 1, bool D16 = false, bool STC = false>
__global__ void __launch_bounds__(256, cheb_min_blocks<T, U, KS, STC>()) k_cheb_first(SellView<T> A, const T* __restrict__ b, T* __restrict__ x,
                                                    T* __restrict__ r, T* __restrict__ dout, T inv_theta, T c1, T c2,
                                                    int want_d, int fold) {
  __shared__ T sh[256];
  sell_any<U, KS, D16, STC>(A, b, sh, [&](int64_t row) { return b[row]; }, [&](int64_t row, T y, T bi) {
    const T d0 = bi * inv_theta;
    const T rr = bi - y * inv_theta;
    r[row] = rr;
    T xi = d0;
    if (want_d) {
      const T d1 = c1 * d0 + c2 * rr;
      dout[row] = d1;
      if (fold) xi += d1;
    }
    x[row] = xi;
  });
}

// Chebyshev step: x += d, r -= A d, d' = c1 d + c2 r; with `fold`, x += d'.
template <typename T, int U = 4, int KS = 1, bool D16 = false, bool STC = false>
__global__ void __launch_bounds__(256, cheb_min_blocks<T, U, KS, STC>()) k_cheb_step(SellView<T> A, const T* __restrict__ din, T* __restrict__ x,
                                                   T* __restrict__ r, T* __restrict__ dout, T c1, T c2, int want_d,
                                                   int fold) {
  __shared__ T sh[256];
  struct RX {
    T r, x;
  };
  sell_any<U, KS, D16, STC>(
      A, din, sh, [&](int64_t row) { return RX{r[row], x[row]}; },
      [&](int64_t row, T y, RX o) {
    const T di = din[row];
    const T rr = o.r - y;
    r[row] = rr;
    T xi = o.x + di;
    if (want_d) {
      const T d1 = c1 * di + c2 * rr;
      dout[row] = d1;
      if (fold) xi += d1;
    }
    x[row] = xi;
  });
}

// Post-smoothing start: r = b - A x, d = r/theta (degree 1: the caller adds
// d to x in a separate launch, after every row of this product has read x).
template <typename T, int U = 4, int KS = 1, bool D16 = false, bool STC = false>
__global__ void __launch_bounds__(256, cheb_min_blocks<T, U, KS, STC>()) k_cheb_resid(SellView<T> A, const T* __restrict__ b, const T* __restrict__ x,
                                                    T* __restrict__ r, T* __restrict__ d, T inv_theta) {
  __shared__ T sh[256];
  sell_any<U, KS, D16, STC>(A, x, sh, [&](int64_t row) { return b[row]; }, [&](int64_t row, T y, T bi) {
    const T rr = bi - y;
    r[row] = rr;
    d[row] = rr * inv_theta;
  });
}

// CSR product (restriction P^T r, prolongation x += P e), thread per row.
template <typename T>
__global__ void k_csr(int64_t n, const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                      const T* __restrict__ val, const T* __restrict__ x, T* __restrict__ y, int add) {
  int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T s = T(0);
  for (int64_t k = rp[i]; k < rp[i + 1]; ++k) s += val[k] * __ldg(x + col[k]);
  y[i] = add ? y[i] + s : s;
}

// ---------------------------------------------------------------- A12 reductions (deterministic)
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < int(blockDim.x >> 5); ++q) t += sh[q];
  __syncthreads();
  return t;
}

// Block partial -> global array; the last block to finish (atomic ticket)
// sums all partials in block order into `out` (k sums of nb partials each,
// partial j of sum q at part[q*nb + j]) and returns true in every thread of
// that block.  The ticket counter is reset for the next use.
template <int K>
__device__ __forceinline__ bool last_block_sum(const double (&v)[K], double* part, unsigned* ticket, double* out,
                                               double* sh) {
  __shared__ bool last;
  const int nb = gridDim.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  double t[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    t[q] = v[q];
    for (int o = 16; o > 0; o >>= 1) t[q] += __shfl_down_sync(0xffffffffu, t[q], o);
  }
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < K; ++q) sh[K * w + q] = t[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < K; ++q) {
      double a = 0.0;
      for (int j = 0; j < nw; ++j) a += sh[K * j + q];
      part[q * nb + blockIdx.x] = a;
    }
    __threadfence();
    last = atomicAdd(ticket, 1u) == unsigned(nb - 1);
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  double u[K];
#pragma unroll
  for (int q = 0; q < K; ++q) {
    u[q] = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) u[q] += part[q * nb + i];
    for (int o = 16; o > 0; o >>= 1) u[q] += __shfl_down_sync(0xffffffffu, u[q], o);
  }
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int q = 0; q < K; ++q) sh[K * w + q] = u[q];
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 0; q < K; ++q) {
      double a = 0.0;
      for (int j = 0; j < nw; ++j) a += sh[K * j + q];
      out[q] = a;
    }
    *ticket = 0u;
  }
  __syncthreads();
  return true;
}

// y = A x with the partial sum of x.y of each block (outer FP64 CG); one
// slice group per block, partials summed afterwards by k_finalize.
template <int U, int KS = 1, bool D16 = false>
__global__ void __launch_bounds__(256) k_spmv_dot(SellView<double> A, const double* __restrict__ x,
                                                  double* __restrict__ y, double* part) {
  __shared__ double sh[256];
  __shared__ double shr[32];
  double acc = 0.0;
  sell_split<U, KS, D16>(A, blockIdx.x, x, sh, [&](int64_t row, double v) {
    y[row] = v;
    acc += v * x[row];
  });
  double t = block_sum(acc, shr);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// Two dot products a.b and c.b in one pass.
__global__ void k_dot2(int64_t n, const double* __restrict__ a, const double* __restrict__ b, const double* __restrict__ c,
                       double* part) {
  __shared__ double sh[32];
  double s0 = 0.0, s1 = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    s0 += a[i] * b[i];
    if (c) s1 += c[i] * b[i];
  }
  double t0 = block_sum(s0, sh);
  double t1 = block_sum(s1, sh);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = t0;
    part[gridDim.x + blockIdx.x] = t1;
  }
}

// Sum the per-block partials in a fixed order; k scalars of nb partials each.
__global__ void k_finalize(const double* part, int nb, int k, double* out) {
  __shared__ double sh[32];
  for (int s = 0; s < k; ++s) {
    double v = 0.0;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) v += part[s * nb + i];
    double t = block_sum(v, sh);
    if (threadIdx.x == 0) out[s] = t;
  }
}

// Fused CG steps (scalars in sc: 0 rz, 1 pq, 2 rr, 3 qz, 4 alpha, 5 beta,
// 6 rr0, 10..12 ticket counters).  q = A p with pq = p.q and alpha = rz / pq:
template <int U, int KS = 1, bool D16 = false>
__global__ void __launch_bounds__(256) k_cg_spmv_alpha(SellView<double> A, const double* __restrict__ p,
                                                       double* __restrict__ q, double* part, double* sc) {
  __shared__ double sh[256];
  __shared__ double shr[64];
  double acc = 0.0;
  sell_split<U, KS, D16>(A, blockIdx.x, p, sh, [&](int64_t row, double v) {
    q[row] = v;
    acc += v * p[row];
  });
  double v1[1] = {acc};
  double out[1];
  if (last_block_sum<1>(v1, part, reinterpret_cast<unsigned*>(sc + 10), out, shr) && threadIdx.x == 0) {
    sc[1] = out[0];
    sc[4] = sc[0] / out[0];
  }
}

// x += alpha p, r -= alpha q, rr = r.r
__global__ void k_cg_update_fused(int64_t n, double* __restrict__ x, double* __restrict__ r,
                                  const double* __restrict__ p, const double* __restrict__ q, double* part, double* sc) {
  __shared__ double shr[64];
  const double alpha = sc[4];
  double acc = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    acc += ri * ri;
  }
  double v1[1] = {acc};
  double out[1];
  if (last_block_sum<1>(v1, part, reinterpret_cast<unsigned*>(sc + 11), out, shr) && threadIdx.x == 0) sc[2] = out[0];
}

// rz_new = r.z, qz = q.z, beta = -qz / pq (flexible), rz = rz_new
__global__ void k_cg_dots_beta(int64_t n, const double* __restrict__ r, const double* __restrict__ z,
                               const double* __restrict__ q, double* part, double* sc) {
  __shared__ double shr[64];
  double a0 = 0.0, a1 = 0.0;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const double zi = z[i];
    a0 += r[i] * zi;
    a1 += q[i] * zi;
  }
  double v2[2] = {a0, a1};
  double out[2];
  if (last_block_sum<2>(v2, part, reinterpret_cast<unsigned*>(sc + 12), out, shr) && threadIdx.x == 0) {
    sc[5] = -out[1] / sc[1];
    sc[0] = out[0];
    sc[3] = out[1];
  }
}

// Device-side control of the whole-PCG graph (one thread).  Scalars in sc as
// above, plus 7 the coarsest-solve timeout flag, 13 rel_res, 14 iterations
// taken, 15 status (an fvem_status value; -1 while the solve runs).  The
// tests follow the host loop: a timeout, a non-finite scalar, then a
// breakdown (p.Ap <= 0 or r.z <= 0), then ||r|| / ||r0|| <= tol, then the
// iteration cap.  `loop` continues the while node and `dir` runs the next
// direction (preconditioner, beta, p) inside it.
__global__ void k_pcg_check_start(double* sc, cudaGraphConditionalHandle loop) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double rr0 = sc[6];
  int st = -1;
  if (sc[7] != 0.0)
    st = 9;
  else if (!isfinite(rr0))
    st = 6;
  else if (rr0 == 0.0)
    st = 0;
  sc[13] = st == -1 ? 1.0 : 0.0;
  sc[14] = 0.0;
  sc[15] = double(st);
  cudaGraphSetConditional(loop, st == -1 ? 1u : 0u);
}

__global__ void k_pcg_check_step(double* sc, double tol, int max_iters, cudaGraphConditionalHandle loop,
                                 cudaGraphConditionalHandle dir) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double it = sc[14] + 1.0;
  sc[14] = it;
  const double rz = sc[0], pq = sc[1], rr = sc[2], rr0 = sc[6];
  int st = -1;
  if (sc[7] != 0.0) {
    st = 9;
  } else if (!isfinite(rz) || !isfinite(pq) || !isfinite(rr)) {
    st = 6;
  } else if (pq <= 0.0 || rz <= 0.0) {
    st = 5;
  } else {
    const double rel = sqrt(rr / rr0);
    sc[13] = rel;
    if (rel <= tol)
      st = 0;
    else if (it >= double(max_iters))
      st = 4;
  }
  sc[15] = double(st);
  cudaGraphSetConditional(loop, st == -1 ? 1u : 0u);
  cudaGraphSetConditional(dir, st == -1 ? 1u : 0u);
}

// p = z + beta p (outer CG scalars in sc as above)
__global__ void k_cg_dir(int64_t n, double* __restrict__ p, const double* __restrict__ z, const double* sc) {
  const double beta = sc[5];
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

template <typename A, typename B>
__global__ void k_convert(int64_t n, const A* __restrict__ a, B* __restrict__ b) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = B(a[i]);
}

__global__ void k_scale_copy(int64_t n, const double* a, double s, double* b) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    b[i] = a[i] * s;
}

// p at all vertices from the free DOF vector (0 on removed DOFs).
__global__ void k_expand(int nv, const int32_t* dof_of_vertex, const double* x, double* out) {
  int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const int i = dof_of_vertex[v];
  out[v] = i >= 0 ? x[i] : 0.0;
}

// Lanczos step pieces: w -= a v + b vprev ; then vprev = v, v = w / beta.
__global__ void k_lanczos_orth(int64_t n, double* w, const double* v, const double* vprev, double a, double b) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    w[i] = (w[i] - a * v[i]) - b * vprev[i];
}
__global__ void k_lanczos_shift(int64_t n, const double* w, double* v, double* vprev, double inv_beta) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    vprev[i] = v[i];
    v[i] = w[i] * inv_beta;
  }
}

__global__ void k_power_init(int64_t n, double* x) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] = 1.0 + double(i % 7) / 7.0;
}

// ---------------------------------------------------------------- A11 coarsest level
// Plain CG from x0 = 0 for a fixed number of iterations on the coarsest level,
// as one cooperative (co-resident) launch: the grid-wide barriers of the
// cooperative-groups API separate the product, the axpys and the reductions.
// Reductions are in FP64; every block sums the per-block partials in the same
// order, so all blocks take identical, deterministic scalar decisions.
// red: 3 * gridDim.x doubles (three slots, so no slot is rewritten while a
// slower block may still read it).
__device__ __forceinline__ double grid_partial_sum(const double* part, int nb, double* sh) {
  double v = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v += part[i];
  double t = block_sum(v, sh);
  if (threadIdx.x == 0) sh[0] = t;
  __syncthreads();
  t = sh[0];
  __syncthreads();
  return t;
}

// Coarsest-level CG in the Chronopoulos-Gear arrangement (two grid barriers
// per iteration: after the row updates, and after the product w = A r with
// both inner products r.r and w.r accumulated in its epilogue).
// red: 4 * gridDim.x doubles (two slot sets used alternately, so a set is only
// rewritten after every block has passed the next barrier).
// Sum two per-block partial arrays in one pass (same fixed order in every block).
__device__ __forceinline__ void grid_partial_sum2(const double* a, const double* b, int nb, double* sh, double& sa,
                                                  double& sb) {
  double va = 0.0, vb = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    va += a[i];
    vb += b[i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    va += __shfl_down_sync(0xffffffffu, va, o);
    vb += __shfl_down_sync(0xffffffffu, vb, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    sh[2 * w] = va;
    sh[2 * w + 1] = vb;
  }
  __syncthreads();
  double ta = 0.0, tb = 0.0;
  for (int q = 0; q < int(blockDim.x >> 5); ++q) {
    ta += sh[2 * q];
    tb += sh[2 * q + 1];
  }
  __syncthreads();
  sa = ta;
  sb = tb;
}

template <typename T, bool D16 = false, int KS = 4, int U = 4>
__global__ void __launch_bounds__(256, 5) k_coarse_cg(SellView<T> A, const T* __restrict__ b, T* x, T* r, T* p, T* s,
                                                      T* w, int iters, double* red) {
  namespace cg = cooperative_groups;
  cg::grid_group grid = cg::this_grid();
  __shared__ double sh[33];
  __shared__ T shT[256];
  const int nb = gridDim.x;
  const int64_t n = A.n;
  const int64_t groups = sell_groups<KS>(A);
  const int64_t tid = int64_t(blockIdx.x) * blockDim.x + threadIdx.x, stride = int64_t(gridDim.x) * blockDim.x;
  for (int64_t i = tid; i < n; i += stride) {
    x[i] = T(0);
    r[i] = b[i];
    p[i] = T(0);
    s[i] = T(0);
  }
  grid.sync();
  auto product = [&](double* slot) {
    double g_acc = 0.0, d_acc = 0.0;
    for (int64_t g = blockIdx.x; g < groups; g += gridDim.x)
      sell_split<U, KS, D16>(A, g, r, shT, [&](int64_t row, T wi) {
        w[row] = wi;
        const double ri = double(r[row]);
        g_acc += ri * ri;
        d_acc += double(wi) * ri;
      });
    for (int o = 16; o > 0; o >>= 1) {
      g_acc += __shfl_down_sync(0xffffffffu, g_acc, o);
      d_acc += __shfl_down_sync(0xffffffffu, d_acc, o);
    }
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    if (lane == 0) {
      sh[2 * wp] = g_acc;
      sh[2 * wp + 1] = d_acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double ta = 0.0, tb = 0.0;
      for (int q = 0; q < 8; ++q) {
        ta += sh[2 * q];
        tb += sh[2 * q + 1];
      }
      slot[blockIdx.x] = ta;
      slot[nb + blockIdx.x] = tb;
    }
    __syncthreads();
  };
  product(red);
  grid.sync();
  double gamma, delta;
  grid_partial_sum2(red, red + nb, nb, sh, gamma, delta);
  if (!(gamma > 0.0 && delta > 0.0)) return;
  double alpha = gamma / delta, beta = 0.0;
  const double stop = 1e-20 * gamma;  // ||r|| <= 1e-10 ||b||
  for (int it = 0; it < iters; ++it) {
    const T ta = T(alpha), tb = T(beta);
    for (int64_t i = tid; i < n; i += stride) {
      const T pi = r[i] + tb * p[i];
      const T si = w[i] + tb * s[i];
      p[i] = pi;
      s[i] = si;
      x[i] += ta * pi;
      r[i] -= ta * si;
    }
    if (it == iters - 1) break;
    grid.sync();
    double* slot = red + 2 * nb * ((it + 1) & 1);
    product(slot);
    grid.sync();
    double gn;
    grid_partial_sum2(slot, slot + nb, nb, sh, gn, delta);
    if (!(gn > stop)) break;
    beta = gn / gamma;
    const double den = delta - beta * gn / alpha;
    if (!(den > 0.0)) break;
    alpha = gn / den;
    gamma = gn;
  }
}

// ---------------------------------------------------------------- A11, kernel-sequence form
// The same Chronopoulos-Gear CG as k_coarse_cg, as two kernels per iteration
// (replayed from the V-cycle graph): k_ccg_upd (row updates) and k_ccg_prod
// (w = A r with the partial sums of r.r and w.r).  The last block of each
// product (atomic ticket) sums the partials in block order and updates the
// scalars; a breakdown or the 1e-10 floor sets `done`, after which every
// remaining kernel of the sequence returns at once.
// cs: 0 gamma, 1 alpha, 2 beta, 3 stop, 4 done, 5 ticket (as unsigned)
template <typename T>
__global__ void k_ccg_init(int64_t n, const T* __restrict__ b, T* x, T* r, T* p, T* s, double* cs) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    x[i] = T(0);
    r[i] = b[i];
    p[i] = T(0);
    s[i] = T(0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    cs[4] = 0.0;
    reinterpret_cast<unsigned*>(cs + 5)[0] = 0u;
  }
}

// Row updates in the vectors' type T; the scalars stay FP64 (rounded to T once).
template <typename T>
__global__ void k_ccg_upd(int64_t n, T* x, T* r, T* p, T* s, const T* w, const double* cs) {
  if (cs[4] != 0.0) return;
  const T a = T(cs[1]), be = T(cs[2]);
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const T pi = r[i] + be * p[i];
    const T si = w[i] + be * s[i];
    p[i] = pi;
    s[i] = si;
    x[i] += a * pi;
    r[i] -= a * si;
  }
}

// w = A r in the type T of the matrix and vectors (FP64, or FP32 inside the
// FP32 V-cycle, where B300's FP64 pipe would bound the product); the inner
// products are accumulated in FP64 either way.
// Block sums of (r.r, w.r) -> per-block partials; the last block to finish
// (atomic ticket in cs[5]) sums all partials in block order and updates the
// scalars (first: gamma, alpha, stop; else the Chronopoulos-Gear step, or
// `done` at the floor or on breakdown).  Called by every thread of the block.
__device__ __forceinline__ void ccg_finish(double g_acc, double d_acc, double* part, double* cs, int first) {
  __shared__ double s2[16];
  __shared__ bool last;
  for (int o = 16; o > 0; o >>= 1) {
    g_acc += __shfl_down_sync(0xffffffffu, g_acc, o);
    d_acc += __shfl_down_sync(0xffffffffu, d_acc, o);
  }
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  if (lane == 0) {
    s2[2 * wp] = g_acc;
    s2[2 * wp + 1] = d_acc;
  }
  __syncthreads();
  const int nb = gridDim.x;
  if (threadIdx.x == 0) {
    double ta = 0.0, tb = 0.0;
    for (int q = 0; q < 8; ++q) {
      ta += s2[2 * q];
      tb += s2[2 * q + 1];
    }
    part[blockIdx.x] = ta;
    part[nb + blockIdx.x] = tb;
    __threadfence();
    const unsigned t = atomicAdd(reinterpret_cast<unsigned*>(cs + 5), 1u);
    last = (t == unsigned(nb - 1));
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double va = 0.0, vb = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    va += part[i];
    vb += part[nb + i];
  }
  for (int o = 16; o > 0; o >>= 1) {
    va += __shfl_down_sync(0xffffffffu, va, o);
    vb += __shfl_down_sync(0xffffffffu, vb, o);
  }
  __syncthreads();
  if (lane == 0) {
    s2[2 * wp] = va;
    s2[2 * wp + 1] = vb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double gn = 0.0, delta = 0.0;
    for (int q = 0; q < 8; ++q) {
      gn += s2[2 * q];
      delta += s2[2 * q + 1];
    }
    if (first) {
      if (gn > 0.0 && delta > 0.0) {
        cs[0] = gn;
        cs[1] = gn / delta;
        cs[2] = 0.0;
        cs[3] = 1e-20 * gn;
      } else {
        cs[4] = 1.0;
      }
    } else {
      const double gamma = cs[0], alpha = cs[1];
      if (!(gn > cs[3])) {
        cs[4] = 1.0;
      } else {
        const double beta = gn / gamma;
        const double den = delta - beta * gn / alpha;
        if (!(den > 0.0)) {
          cs[4] = 1.0;
        } else {
          cs[1] = gn / den;
          cs[2] = beta;
          cs[0] = gn;
        }
      }
    }
    reinterpret_cast<unsigned*>(cs + 5)[0] = 0u;
  }
}

template <typename T, int U, int KS, bool D16, bool STC = false>
__global__ void __launch_bounds__(256) k_ccg_prod(SellView<T> A, const T* __restrict__ r, T* w, double* part,
                                                  double* cs, int first) {
  if (cs[4] != 0.0) return;
  __shared__ T sh[256];
  double g_acc = 0.0, d_acc = 0.0;
  sell_split<U, KS, D16, STC>(A, blockIdx.x, r, sh, [&](int64_t row, T wi) {
    w[row] = wi;
    const double ri = double(r[row]);
    g_acc += ri * ri;
    d_acc += double(wi) * ri;
  });
  ccg_finish(g_acc, d_acc, part, cs, first);
}

// Mixed split: slice lists by warps per slice (class c uses KS = 1, 2, 4, 8;
// a slice gets the fewest warps that keep its per-warp share of slots under
// a tuned bound), each list padded to its slices per block with -1; class c
// owns blocks [blk[c], blk[c+1]) of one launch, so wide slices get more
// warps without splitting the narrow ones.
struct MixSched {
  const int32_t* list;  // the four class lists, concatenated
  int64_t off[4], len[4];
  int blk[5];
  const int32_t* stpos;  // per slice: stencil schedule position or -1 (null: no stencil slices)
};

template <typename T, int U, bool D16>
__global__ void __launch_bounds__(256) k_ccg_prod_mix(SellView<T> A, MixSched M, const T* __restrict__ r, T* w,
                                                      double* part, double* cs, int first) {
  if (cs[4] != 0.0) return;
  __shared__ T sh[256];
  double g_acc = 0.0, d_acc = 0.0;
  auto epi = [&](int64_t row, T wi) {
    w[row] = wi;
    const double ri = double(r[row]);
    g_acc += ri * ri;
    d_acc += double(wi) * ri;
  };
  const int b = blockIdx.x;
  const int c = b < M.blk[1] ? 0 : (b < M.blk[2] ? 1 : (b < M.blk[3] ? 2 : 3));
  SellView<T> V = A;
  V.order = M.list + M.off[c];
  V.nsched = M.len[c];
  V.nsched_st = 0;
  V.stpos = A.reg != nullptr ? M.stpos : nullptr;
  const int64_t g = b - M.blk[c];
  if (c == 0)
    sell_split<U, 1, D16, true>(V, g, r, sh, epi);
  else if (c == 1)
    sell_split<U, 2, D16, true>(V, g, r, sh, epi);
  else if (c == 2)
    sell_split<U, 4, D16, true>(V, g, r, sh, epi);
  else
    sell_split<U, 8, D16, true>(V, g, r, sh, epi);
  ccg_finish(g_acc, d_acc, part, cs, first);
}

// ---------------------------------------------------------------- A11, persistent form
// The Chronopoulos-Gear CG of k_ccg_* as one cooperative launch with one CTA
// per SM and one grid barrier per iteration.  Each CTA owns a contiguous run
// of rows [row0, row1), stored in its own compact layout: the run's rows
// sorted by length (longest first) in slices of 32, each slice as wide as its
// first row, slots column-major (slot = slice start + 32 j + lane), so the
// padding stays small.  Its halo is the sorted list of distinct columns its
// rows reference (own rows included, at a known offset); the stored column
// of a slot is its position in the halo.  At the start the CTA copies, with
// bulk asynchronous copies (cp.async.bulk, completion on an mbarrier), its
// values, halo positions, halo row list and sorted-row order into shared
// memory.  It keeps r and s on its whole halo and p, x on its own rows in
// shared memory, and updates the halo copies of r and s itself from the
// published products w, so r never travels through global memory.  Per
// iteration t:
//   w = A r on own rows (shared memory only) -> w_g[t & 1], and the CTA's
//   partial sums of r.r and w.r (FP64) -> part[t & 1];
//   grid barrier;
//   warp 0 sums the partials in CTA order and one thread runs the scalar
//   recurrence (identical scalars in every CTA; B300's FP64 pipe is narrow,
//   so no FP64 work is spread over the whole CTA); the other warps load
//   w_g[t & 1] on the halo; then p, x (own rows) and s, r (halo) are updated.
// Every CTA computes a halo row's r and s with the same operations on the
// same values as the row's owner, so all copies agree bit for bit.  w_g is
// double buffered: w_g[t & 1] is rewritten at step t + 2, after the barrier of
// step t + 1, which every reader of step t has reached.
// The grid barrier is one monotonic 64-bit arrival counter: at the start a
// CTA reads it (fewer than nb arrivals of this launch can precede the read)
// and rounds down to a multiple of nb; barrier k is passed when the counter
// reaches that base + (k + 1) nb.  Every wait is bounded (kSpinLimit polls);
// on a timeout the CTA records status 1, raises `abort` so the others stop
// waiting, and returns (its bulk copies have completed by then, or their
// bounded wait ran out first).
constexpr long long kSpinLimit = 1ll << 22;

struct PersistPlan {
  const int32_t* rb;        // nb + 1 row bounds
  const int64_t* p_off;     // nb + 1 offsets of the CTAs' pair rows (32 lanes x 2 slots each)
  const int32_t* t_off;     // nb + 1 offsets into tasks
  const int4* tasks;        // per CTA: {first pair row (CTA-relative), pair rows, slice, part}
  const int32_t* perm_off;  // nb + 1 offsets into perm (multiples of 8)
  const int16_t* perm;      // per CTA, sorted position -> local row
  const void* val;          // per pair row and lane, two values (type T; padding 0)
  const uint32_t* lidx2;    // per pair row and lane, the two slots' halo positions (16 bits each; padding 0)
  const int32_t* halo_ptr;  // nb + 1 (each run padded to a multiple of 4)
  const int32_t* halo_col;  // halo rows per CTA
  const int32_t* halo_own;  // nb: position of the CTA's first own row in its halo
  unsigned long long* count;  // grid-barrier arrival counter
  double* part;               // 2 parities x 2 sums x nb
  void* w_g;                  // 2 parities x n values of w = A r (type T)
  int* abort_;
  double* status;  // set to 1 on a timeout (host-visible scalar)
  int64_t n;
  int rows_cap, pairs_cap, tasks_cap, halo_cap, ks;  // ks: most parts of one slice
  int val_smem;  // 1: the values are copied to shared memory; 0: read from global memory (L2) each product
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// bulk copy global -> this CTA's shared memory; dst, src 16-byte aligned, bytes % 16 == 0
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
// bounded wait for phase `parity` of the mbarrier
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  for (long long it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier number k on the monotonic counter (thread 0 arrives and
// polls); false on the poll limit or when another CTA aborted.  Called by all
// threads of the CTA.
__device__ __forceinline__ bool grid_barrier(unsigned long long* count, unsigned long long target, const int* abort_,
                                             int* fail) {
  __syncthreads();
  if (threadIdx.x == 0) {
    // release: the CTA's writes (ordered before this thread by the barrier
    // above) become visible with the arrival; acquire: every arrival's
    // writes are visible to this CTA after the barrier below
    asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(count), "l"(1ull) : "memory");
    bool ok = false;
    for (long long it = 0; it < kSpinLimit; ++it) {
      if (ld_acquire_u64(count) >= target) {
        ok = true;
        break;
      }
      if ((it & 255) == 255 && *reinterpret_cast<const volatile int*>(abort_)) break;
    }
    if (!ok) *fail = 1;
  }
  __syncthreads();
  return *reinterpret_cast<volatile int*>(fail) == 0;
}

// Values of the compact layout from the assembled CSR values (FP64):
// out[k] = T(csr[map[k]]), or 0 where map[k] < 0 (padding).
template <typename T>
__global__ void k_gather_pad(int64_t n, const int64_t* __restrict__ map, const double* __restrict__ csr,
                             T* __restrict__ out) {
  for (int64_t k = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; k < n; k += int64_t(gridDim.x) * blockDim.x) {
    const int64_t m = map[k];
    out[k] = m >= 0 ? T(csr[m]) : T(0);
  }
}

// Float-float ("double-single") arithmetic of the FP32 persistent CG's dot
// products and scalar recurrence: a value is the unevaluated sum h + l of two
// floats with |l| <= ulp(h) / 2, about 48 significand bits carried by FP32
// instructions alone (B300's FP64 pipe is narrow, and the scalar chain of a CG
// iteration is latency-bound).  Error-free transformations: Knuth's TwoSum
// and the FMA form of Dekker's TwoProduct; sum, product and quotient after
// Dekker (1971).
struct ff2 {
  float h, l;
};
// |a| >= |b| or a == 0
__device__ __forceinline__ ff2 ff_fast(float a, float b) {
  const float s = a + b;
  return ff2{s, b - (s - a)};
}
__device__ __forceinline__ ff2 ff_two_sum(float a, float b) {
  const float s = a + b, bb = s - a;
  return ff2{s, (a - (s - bb)) + (b - bb)};
}
// a * b exactly (barring underflow)
__device__ __forceinline__ ff2 ff_prod(float a, float b) {
  const float p = a * b;
  return ff2{p, fmaf(a, b, -p)};
}
__device__ __forceinline__ ff2 ff_add(ff2 x, ff2 y) {
  ff2 s = ff_two_sum(x.h, y.h);
  const ff2 t = ff_two_sum(x.l, y.l);
  s = ff_fast(s.h, s.l + t.h);
  return ff_fast(s.h, s.l + t.l);
}
// Sum for reduction trees: one TwoSum on the high parts, the low parts added
// plainly; its error stays within a few units of 2^-48 (|x| + |y|), the
// bound a dot product's rounding is judged by.
__device__ __forceinline__ ff2 ff_add_tree(ff2 x, ff2 y) {
  const ff2 s = ff_two_sum(x.h, y.h);
  return ff_fast(s.h, s.l + (x.l + y.l));
}
__device__ __forceinline__ ff2 ff_mul(ff2 x, ff2 y) {
  const ff2 p = ff_prod(x.h, y.h);
  return ff_fast(p.h, fmaf(x.h, y.l, fmaf(x.l, y.h, p.l)));
}
// x / y: a first quotient from the correctly rounded reciprocal of y.h, then
// one correction step on the exact remainder (about 2^-46 relative)
__device__ __forceinline__ ff2 ff_div(ff2 x, ff2 y) {
  const float ry = __frcp_rn(y.h);
  const float q1 = x.h * ry;
  const ff2 p = ff_mul(y, ff2{q1, 0.0f});
  const ff2 r = ff_add(x, ff2{-p.h, -p.l});
  return ff_fast(q1, r.h * ry);
}
__device__ __forceinline__ ff2 ff_shfl_down(ff2 v, int o) {
  return ff2{__shfl_down_sync(0xffffffffu, v.h, o), __shfl_down_sync(0xffffffffu, v.l, o)};
}

// two consecutive values of shared memory in one access (p aligned to 2 T)
template <typename T>
__device__ __forceinline__ void ld_pair(const T* p, T& a, T& b) {
  if constexpr (std::is_same<T, float>::value) {
    const float2 v = *reinterpret_cast<const float2*>(p);
    a = v.x;
    b = v.y;
  } else {
    const double2 v = *reinterpret_cast<const double2*>(p);
    a = v.x;
    b = v.y;
  }
}

template <typename T>
__global__ void __launch_bounds__(1024, 1) k_ccg_persist(PersistPlan P, const T* __restrict__ b,
                                                         T* __restrict__ x_out, int iters) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ uint64_t bar;
  __shared__ double sc[4];  // gamma, alpha, beta, stop (lane 0 of warp 0; FP64 copies)
  __shared__ ff2 sf[6];     // the same in float-float (FP32 copies), then 1/gamma, 1/(gamma alpha)
  __shared__ float4 bpart[32];  // FP32 copies: per-warp float-float partial sums
  __shared__ T ab[2];       // alpha, beta rounded to T
  __shared__ int go_s;
  __shared__ int fail;
  __shared__ unsigned long long base;
  const int tid = threadIdx.x, lane = tid & 31, wp = tid >> 5, nw = blockDim.x >> 5;
  const int blk = blockIdx.x, nb = gridDim.x;
  const int64_t row0 = P.rb[blk];
  const int rows = P.rb[blk + 1] - P.rb[blk];
  const int64_t g0 = P.p_off[blk], npair = P.p_off[blk + 1] - g0;
  const int t0 = P.t_off[blk], ntask = P.t_off[blk + 1] - t0;
  const int pm0 = P.perm_off[blk], npm = P.perm_off[blk + 1] - pm0;
  const int h0 = P.halo_ptr[blk], nhalo = P.halo_ptr[blk + 1] - h0;
  const int own = P.halo_own[blk];
  T* w_g = static_cast<T*>(P.w_g);
  // shared layout: value pairs | halo-position pairs (uint32) | tasks (int4)
  //                | halo rows (int32) | sorted order (int16) | halo r, s, w
  //                | own p, x | product partials | per-row FP64 sums
  T* val = reinterpret_cast<T*>(sm);
  uint32_t* lidx2 = reinterpret_cast<uint32_t*>(val + (P.val_smem ? size_t(P.pairs_cap) * 64 : size_t(0)));
  int4* task = reinterpret_cast<int4*>(lidx2 + size_t(P.pairs_cap) * 32);
  int32_t* hcol = reinterpret_cast<int32_t*>(task + P.tasks_cap);
  int16_t* perm = reinterpret_cast<int16_t*>(hcol + P.halo_cap);
  T* hr = reinterpret_cast<T*>(perm + P.rows_cap);
  T* hs = hr + P.halo_cap;
  T* hw = hs + P.halo_cap;
  T* vp = hw + P.halo_cap;
  T* vx = vp + P.rows_cap;
  T* wpart = vx + P.rows_cap;  // ks x rows_cap product partials (sorted positions)
  double* rg = reinterpret_cast<double*>((reinterpret_cast<uintptr_t>(wpart + size_t(P.ks) * P.rows_cap) + 7) &
                                         ~uintptr_t(7));
  double* rd = rg + P.rows_cap;
  const int ks = P.ks;
  auto abort_all = [&]() {
    fail = 1;
    atomicExch(P.abort_, 1);
    *reinterpret_cast<volatile double*>(P.status) = 1.0;
  };
  if (tid == 0) {
    // a set abort word (an earlier launch gave up, or the host armed it) ends
    // the launch before it issues any copy, through the timeout's exit
    fail = *reinterpret_cast<const volatile int*>(P.abort_) != 0 ? 1 : 0;
    if (fail) *reinterpret_cast<volatile double*>(P.status) = 1.0;
  }
  if (tid == 0 && !fail) {
    base = (ld_relaxed_u64(P.count) / unsigned(nb)) * unsigned(nb);
    mbar_init(&bar, 1);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const unsigned bv = P.val_smem ? unsigned(npair * 64 * sizeof(T)) : 0u;
    const unsigned bi = unsigned(npair * 32 * sizeof(uint32_t)), bt = unsigned(ntask * sizeof(int4));
    const unsigned bh = unsigned(nhalo * sizeof(int32_t)), bp = unsigned(npm * sizeof(int16_t));
    mbar_expect_tx(&bar, bv + bi + bt + bh + bp);
    if (bv) bulk_g2s(val, static_cast<const T*>(P.val) + g0 * 64, bv, &bar);
    bulk_g2s(lidx2, P.lidx2 + g0 * 32, bi, &bar);
    bulk_g2s(task, P.tasks + t0, bt, &bar);
    bulk_g2s(hcol, P.halo_col + h0, bh, &bar);
    bulk_g2s(perm, P.perm + pm0, bp, &bar);
  }
  for (int i = tid; i < rows; i += blockDim.x) {
    vx[i] = T(0);
    vp[i] = T(0);
  }
  // parts a slice does not have stay zero in the partial sums
  for (int i = tid; i < ks * P.rows_cap; i += blockDim.x) wpart[i] = T(0);
  __syncthreads();
  if (fail) return;
  if (tid == 0 && !mbar_wait(&bar, 0)) abort_all();
  __syncthreads();
  if (fail) return;
  for (int h = tid; h < nhalo; h += blockDim.x) {
    hr[h] = b[hcol[h]];
    hs[h] = T(0);
  }
  __syncthreads();
  // the product's values: this CTA's copy in shared memory, or its run of the
  // global array (L2-resident across the iterations) when they do not fit
  const T* vals = P.val_smem ? val : static_cast<const T*>(P.val) + g0 * 64;
  for (int t = 0; t < iters; ++t) {
    // FP32 copies: the reciprocals the next scalar step needs, formed by
    // warp 0 (which takes the shortest product task) off the critical path
    if constexpr (std::is_same<T, float>::value) {
      if (tid == 0 && t > 0) {
        sf[4] = ff_div(ff2{1.0f, 0.0f}, sf[0]);
        sf[5] = ff_div(ff2{1.0f, 0.0f}, ff_mul(sf[0], sf[1]));
      }
    }
    // w = A r on own rows: task {first pair row, pair rows, slice, part}
    // takes part `part` of its slice's slots, two slots per pair row, one
    // task per warp in turn (the host balanced the tasks over the warps;
    // tasks come longest first, and the last warp takes the first)
    for (int k = nw - 1 - wp; k < ntask; k += nw) {
      const int4 d = task[k];
      const T* v2 = vals + (size_t(d.x) * 32 + lane) * 2;
      const uint32_t* l2 = lidx2 + size_t(d.x) * 32 + lane;
      T y0 = T(0), y1 = T(0), y2 = T(0), y3 = T(0);
      int r = 0;
      for (; r + 1 < d.y; r += 2) {
        const uint32_t la = l2[r * 32], lb = l2[(r + 1) * 32];
        T a0, a1, b0, b1;
        ld_pair(v2 + r * 64, a0, a1);
        ld_pair(v2 + (r + 1) * 64, b0, b1);
        y0 += a0 * hr[la & 0xffffu];
        y1 += a1 * hr[la >> 16];
        y2 += b0 * hr[lb & 0xffffu];
        y3 += b1 * hr[lb >> 16];
      }
      if (r < d.y) {
        const uint32_t la = l2[r * 32];
        T a0, a1;
        ld_pair(v2 + r * 64, a0, a1);
        y0 += a0 * hr[la & 0xffffu];
        y1 += a1 * hr[la >> 16];
      }
      wpart[d.w * P.rows_cap + d.z * 32 + lane] = (y0 + y2) + (y1 + y3);
    }
    __syncthreads();
    T* wt = w_g + size_t(t & 1) * size_t(P.n);
    constexpr bool kF = std::is_same<T, float>::value;
    ff2 ag{0.0f, 0.0f}, ad{0.0f, 0.0f};  // FP32 copies: this thread's (r, r), (w, r)
    for (int i = tid; i < rows; i += blockDim.x) {
      T wi = wpart[i];
      for (int pt = 1; pt < ks; ++pt) wi += wpart[pt * P.rows_cap + i];
      const int lr = perm[i];
      wt[row0 + lr] = wi;
      if constexpr (kF) {
        const float ri = hr[own + lr];
        ag = ff_add_tree(ag, ff_prod(ri, ri));
        ad = ff_add_tree(ad, ff_prod(wi, ri));
      } else {
        const double ri = double(hr[own + lr]);
        rg[i] = ri * ri;
        rd[i] = double(wi) * ri;
      }
    }
    if constexpr (kF) {
      // fixed-order tree over the block: lanes, then the warps' partials
      // (warps past the last row hold zeros and skip the tree)
      if (wp * 32 < rows) {
        for (int o = 16; o > 0; o >>= 1) {
          ag = ff_add_tree(ag, ff_shfl_down(ag, o));
          ad = ff_add_tree(ad, ff_shfl_down(ad, o));
        }
      }
      if (lane == 0) bpart[wp] = make_float4(ag.h, ag.l, ad.h, ad.l);
    }
    __syncthreads();
    double* pp = P.part + size_t(t & 1) * 2 * nb;
    float4* pf = reinterpret_cast<float4*>(P.part) + size_t(t & 1) * nb;  // FP32 copies (same bytes)
    if (kF && wp == 0) {
      const float4 v = lane < nw ? bpart[lane] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      ff2 a{v.x, v.y}, d{v.z, v.w};
      for (int o = 16; o > 0; o >>= 1) {
        a = ff_add_tree(a, ff_shfl_down(a, o));
        d = ff_add_tree(d, ff_shfl_down(d, o));
      }
      if (lane == 0) pf[blk] = make_float4(a.h, a.l, d.h, d.l);
    } else if (!kF && wp == 0) {
      double a = 0.0, d = 0.0;
      for (int i = lane; i < rows; i += 32) {
        a += rg[i];
        d += rd[i];
      }
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        d += __shfl_down_sync(0xffffffffu, d, o);
      }
      if (lane == 0) {
        pp[blk] = a;
        pp[nb + blk] = d;
      }
    }
    // every CTA's product and partial sums of this step are published
    if (!grid_barrier(P.count, base + (unsigned long long)(t + 1) * unsigned(nb), P.abort_, &fail)) {
      if (tid == 0) abort_all();
      return;
    }
    if (kF && wp == 0) {
      // the CTAs' partials, five loads in flight per lane, then a fixed tree
      ff2 a{0.0f, 0.0f}, d{0.0f, 0.0f};
      for (int q0 = 0; q0 < nb; q0 += 160) {
        float4 v[5];
#pragma unroll
        for (int u = 0; u < 5; ++u) {
          const int q = q0 + lane + 32 * u;
          v[u] = q < nb ? __ldcg(pf + q) : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
#pragma unroll
        for (int u = 0; u < 5; ++u) {
          a = ff_add_tree(a, ff2{v[u].x, v[u].y});
          d = ff_add_tree(d, ff2{v[u].z, v[u].w});
        }
      }
      for (int o = 16; o > 0; o >>= 1) {
        a = ff_add_tree(a, ff_shfl_down(a, o));
        d = ff_add_tree(d, ff_shfl_down(d, o));
      }
      if (lane == 0) {
        // Chronopoulos-Gear recurrence, as in the FP64 branch below
        const ff2 gn = a, delta = d;
        bool go = true;
        if (t == 0) {
          if (gn.h > 0.0f && delta.h > 0.0f) {
            sf[0] = gn;
            sf[1] = ff_div(gn, delta);
            sf[2] = ff2{0.0f, 0.0f};
            sf[3] = ff2{1e-20f * gn.h, 0.0f};
          } else {
            go = false;
          }
        } else if (!(gn.h > sf[3].h)) {
          go = false;
        } else {
          // beta = gn / gamma, den = delta - gn^2 / (gamma alpha): products
          // with the reciprocals formed during the product phase
          const ff2 bt = ff_mul(gn, sf[4]);
          const ff2 q = ff_mul(ff_mul(gn, gn), sf[5]);
          const ff2 den = ff_add(delta, ff2{-q.h, -q.l});
          if (!(den.h > 0.0f)) {
            go = false;
          } else {
            sf[1] = ff_div(gn, den);
            sf[2] = bt;
            sf[0] = gn;
          }
        }
        go_s = go ? 1 : 0;
        ab[0] = T(sf[1].h);
        ab[1] = T(sf[2].h);
      }
    } else if (wp == 0) {
      double a = 0.0, d = 0.0;
      for (int q = lane; q < nb; q += 32) {
        a += __ldcg(pp + q);
        d += __ldcg(pp + nb + q);
      }
      for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_down_sync(0xffffffffu, a, o);
        d += __shfl_down_sync(0xffffffffu, d, o);
      }
      if (lane == 0) {
        const double gn = a, delta = d;
        bool go = true;
        if (t == 0) {
          if (gn > 0.0 && delta > 0.0) {
            sc[0] = gn;          // gamma
            sc[1] = gn / delta;  // alpha
            sc[2] = 0.0;         // beta
            sc[3] = 1e-20 * gn;  // stop
          } else {
            go = false;
          }
        } else if (!(gn > sc[3])) {
          go = false;
        } else {
          const double bt = gn / sc[0];
          const double den = delta - bt * gn / sc[1];
          if (!(den > 0.0)) {
            go = false;
          } else {
            sc[1] = gn / den;
            sc[2] = bt;
            sc[0] = gn;
          }
        }
        go_s = go ? 1 : 0;
        ab[0] = T(sc[1]);
        ab[1] = T(sc[2]);
      }
    } else {
      // the halo's products, eight independent loads in flight per thread
      const int stride = blockDim.x - 32;
      int h = tid - 32;
      for (; h + 7 * stride < nhalo; h += 8 * stride) {
        T v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __ldcg(wt + hcol[h + u * stride]);
#pragma unroll
        for (int u = 0; u < 8; ++u) hw[h + u * stride] = v[u];
      }
      for (; h < nhalo; h += stride) hw[h] = __ldcg(wt + hcol[h]);
    }
    __syncthreads();
    if (!go_s) break;
    const T ta = ab[0], tb = ab[1];
    // own rows first (p needs the old r), then r and s on the whole halo
    for (int i = tid; i < rows; i += blockDim.x) {
      const T pi = hr[own + i] + tb * vp[i];
      vp[i] = pi;
      vx[i] += ta * pi;
    }
    __syncthreads();
    for (int h = tid; h < nhalo; h += blockDim.x) {
      const T si = hw[h] + tb * hs[h];
      hs[h] = si;
      hr[h] = hr[h] - ta * si;
    }
    __syncthreads();
  }
  __syncthreads();
  for (int i = tid; i < rows; i += blockDim.x) x_out[row0 + i] = vx[i];
}

// ---------------------------------------------------------------- element quality (Eq. 18, App. C)
// rho(E) = sqrt(rho1 rho2 + rho1 rho3) / 2 per cell, thread per cell:
//   rho1 = |k(E)|/|E| prod_f |k(f)|/|f| (kernels: the points that see the
//          whole element); the cells of these grids are convex polyhedra with
//          convex faces (BSP cells and overlay faces), so every kernel is the
//          element itself and rho1 = 1.  The kernel checks that (every cell
//          vertex on the inner side of every face plane, every face turning
//          one way, both to 1e-8 in distance: ten times the distance at which
//          the topology welds vertices) and flags a cell that is not convex,
//          whose rho it leaves undefined (NaN);
//   rho2 = min(|E|^(1/3), min_f h_f)/h_E + (1/#f) sum_f min(|f|^(1/2), min_e |e|)/h_f
//          (the face term read with the square root of the area);
//   rho3 = 4/#f + (1/#f) sum_f 3/#e_f,
// h_E, h_f diameters.  flag bit 0: a cut cell (not an axis-aligned cube: its
// bounding box not a cube, or its volume off the box's by 1e-9 relative);
// bit 1: not convex.
__global__ void k_quality(MeshView m, double* __restrict__ rho, int* __restrict__ flag) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.nc) return;
  const int vb = m.cell_vptr[c], nv = m.cell_vptr[c + 1] - vb;
  const int fb = m.cell_fptr[c], nf = m.cell_fptr[c + 1] - fb;
  D3 c0{0, 0, 0}, lo{1e300, 1e300, 1e300}, hi{-1e300, -1e300, -1e300};
  double hE = 0.0;
  for (int i = 0; i < nv; ++i) {
    const D3 a = ld3(m.V, m.cell_v[vb + i]);
    c0 = add3(c0, a);
    lo = D3{fmin(lo.x, a.x), fmin(lo.y, a.y), fmin(lo.z, a.z)};
    hi = D3{fmax(hi.x, a.x), fmax(hi.y, a.y), fmax(hi.z, a.z)};
    for (int j = i + 1; j < nv; ++j) {
      const D3 d = sub3(a, ld3(m.V, m.cell_v[vb + j]));
      hE = fmax(hE, sqrt(dt3(d, d)));
    }
  }
  c0 = mul3(c0, 1.0 / nv);
  const double tol = 1e-9;   // relative, the cube test of the cut flag
  const double dtol = 1e-8;  // distance, the convexity tests
  bool convex = true;
  double vol = 0.0, minhf = 1e300, s2 = 0.0, s3 = 0.0;
  for (int f = 0; f < nf; ++f) {
    const int s = m.face_vptr[fb + f], k = m.face_vptr[fb + f + 1] - s;
    const int32_t* cyc = m.face_v + s;
    double area;
    D3 n, cen, xbar;
    face_geom(m.V, cyc, k, area, n, cen, xbar);
    double hf = 0.0, emin = 1e300;
    const D3 a0 = ld3(m.V, cyc[0]);
    for (int q = 0; q < k; ++q) {
      const D3 p = ld3(m.V, cyc[q]), pn = ld3(m.V, cyc[(q + 1) % k]), pnn = ld3(m.V, cyc[(q + 2) % k]);
      const D3 e = sub3(pn, p);
      emin = fmin(emin, sqrt(dt3(e, e)));
      for (int r = q + 1; r < k; ++r) {
        const D3 d = sub3(p, ld3(m.V, cyc[r]));
        hf = fmax(hf, sqrt(dt3(d, d)));
      }
      // a convex face turns one way (collinear vertices allowed): the next
      // vertex lies left of this edge's line, or within dtol of it
      const double le = sqrt(dt3(e, e));
      if (le > 0.0 && dt3(crs3(e, sub3(pnn, pn)), n) < -dtol * le) convex = false;
      if (q >= 1 && q + 1 < k) vol += dt3(sub3(a0, c0), crs3(sub3(p, c0), sub3(pn, c0))) / 6.0;
    }
    // a convex cell lies on the inner side of each face plane
    for (int i = 0; i < nv; ++i)
      if (dt3(sub3(ld3(m.V, m.cell_v[vb + i]), cen), n) > dtol) convex = false;
    minhf = fmin(minhf, hf);
    s2 += fmin(sqrt(area), emin) / hf;
    s3 += 3.0 / k;
  }
  const double rho2 = fmin(cbrt(vol), minhf) / hE + s2 / nf;
  const double rho3 = 4.0 / nf + s3 / nf;
  rho[c] = convex ? sqrt(rho2 + rho3) / 2.0 : nan("");
  const D3 ext = sub3(hi, lo);
  const double bv = ext.x * ext.y * ext.z;
  const bool cube = fabs(ext.x - ext.y) <= tol * ext.x && fabs(ext.y - ext.z) <= tol * ext.x &&
                    fabs(vol - bv) <= tol * bv;
  flag[c] = (cube ? 0 : 1) | (convex ? 0 : 2);
}

// Per block, in a fixed order: the sum of rho^2 over cut cells, the number of
// cut cells and the number of non-convex cells (3 doubles per block).
__global__ void k_quality_sum(int nc, const double* __restrict__ rho, const int* __restrict__ flag,
                              double* __restrict__ part) {
  __shared__ double sh[3][256];
  double a = 0.0, b = 0.0, d = 0.0;
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < nc; c += gridDim.x * blockDim.x) {
    const int f = flag[c];
    if (f & 1) {
      a += rho[c] * rho[c];
      b += 1.0;
    }
    if (f & 2) d += 1.0;
  }
  sh[0][threadIdx.x] = a;
  sh[1][threadIdx.x] = b;
  sh[2][threadIdx.x] = d;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (int(threadIdx.x) < o)
      for (int q = 0; q < 3; ++q) sh[q][threadIdx.x] += sh[q][threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int q = 0; q < 3; ++q) part[3 * blockIdx.x + q] = sh[q][0];
}

template <typename T>
__global__ void k_axpy(int64_t n, T* __restrict__ x, const T* __restrict__ d) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] += d[i];
}

}  // namespace fvem
