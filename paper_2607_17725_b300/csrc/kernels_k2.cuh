// Device kernels of the second-order (k = 2) VEM path (sm_103a).
//
// Element kernel (Sec. 3.1, Eq. 11-14, App. A for k = 2): one warp per
// polyhedral cell, every matrix in shared memory.  DOFs of a cell in element
// order: vertex values (vertices ascending), values at edge midpoints (edges
// sorted by their vertex ids), face means (the cell's face order), the cell
// mean.  Scaled monomials m_a = ((x - x_E)/h_E)^e_a, |e_a| <= 2, in the order
// 1, x, y, z, xx, xy, xz, yy, yz, zz; on a face, m2_b = z^e_b in the face's
// local coordinates z = ((x - x_f).t1, (x - x_f).t2)/h_f, order 1, z1, z2,
// z1z1, z1z2, z2z2.  Integrals of polynomials are exact: cells by a fan of
// tetrahedra from the vertex mean with the degree-2 rule on the vertices
// (weight -1/20) and edge midpoints (1/5); faces by a fan of triangles with
// the degree-3 rule on the vertices (1/20), edge midpoints (2/15) and
// centroid (9/20); the edge integrals of the face projector by Simpson's rule
// (quadratic times linear).  The face terms of B use the face projector
// Pi_{2,f} (enhanced face space): int_f phi_i q = int_f Pi_{2,f} phi_i q for
// linear q.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace fvem {

// exponents of the scaled monomials (3D: 10, 2D up to degree 3: 10)
__constant__ int8_t kE3[10][3] = {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 0},
                                  {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};
__constant__ int8_t kE2[10][2] = {{0, 0}, {1, 0}, {0, 1}, {2, 0}, {1, 1}, {0, 2}, {3, 0}, {2, 1}, {1, 2}, {0, 3}};

// index of a 3D exponent of degree <= 2 in kE3 (-1 if none)
__device__ __forceinline__ int idx3(int a, int b, int c) {
  if (a < 0 || b < 0 || c < 0) return -1;
  const int d = a + b + c;
  if (d == 0) return 0;
  if (d == 1) return a ? 1 : (b ? 2 : 3);
  if (d == 2) {
    if (a == 2) return 4;
    if (a == 1) return b ? 5 : 6;
    if (b == 2) return 7;
    if (b == 1) return 8;
    return 9;
  }
  return -1;
}
// index of a 2D exponent of degree <= 3 in kE2
__device__ __forceinline__ int idx2(int a, int b) {
  if (a < 0 || b < 0) return -1;
  const int d = a + b;
  if (d > 3) return -1;
  const int base = d == 0 ? 0 : (d == 1 ? 1 : (d == 2 ? 3 : 6));
  return base + b;
}
__device__ __forceinline__ void mono3v(D3 y, double* m) {
  m[0] = 1.0;
  m[1] = y.x;
  m[2] = y.y;
  m[3] = y.z;
  m[4] = y.x * y.x;
  m[5] = y.x * y.y;
  m[6] = y.x * y.z;
  m[7] = y.y * y.y;
  m[8] = y.y * y.z;
  m[9] = y.z * y.z;
}
// z-monomials of degree <= 3 at z
__device__ __forceinline__ void mono2v(double z1, double z2, double* m) {
  m[0] = 1.0;
  m[1] = z1;
  m[2] = z2;
  m[3] = z1 * z1;
  m[4] = z1 * z2;
  m[5] = z2 * z2;
  m[6] = z1 * z1 * z1;
  m[7] = z1 * z1 * z2;
  m[8] = z1 * z2 * z2;
  m[9] = z2 * z2 * z2;
}

// Dense solve A X = B in place (A n x n row-major, B n x m row-major, one
// thread), Gaussian elimination with partial pivoting.
__device__ inline void small_solve(double* A, int n, double* B, int m) {
  for (int k = 0; k < n; ++k) {
    int p = k;
    double best = fabs(A[k * n + k]);
    for (int i = k + 1; i < n; ++i)
      if (fabs(A[i * n + k]) > best) {
        best = fabs(A[i * n + k]);
        p = i;
      }
    if (p != k) {
      for (int j = 0; j < n; ++j) {
        const double t = A[k * n + j];
        A[k * n + j] = A[p * n + j];
        A[p * n + j] = t;
      }
      for (int j = 0; j < m; ++j) {
        const double t = B[k * m + j];
        B[k * m + j] = B[p * m + j];
        B[p * m + j] = t;
      }
    }
    const double inv = 1.0 / A[k * n + k];
    for (int i = k + 1; i < n; ++i) {
      const double f = A[i * n + k] * inv;
      if (f == 0.0) continue;
      for (int j = k; j < n; ++j) A[i * n + j] -= f * A[k * n + j];
      for (int j = 0; j < m; ++j) B[i * m + j] -= f * B[k * m + j];
    }
  }
  for (int j = 0; j < m; ++j)
    for (int i = n - 1; i >= 0; --i) {
      double s = B[i * m + j];
      for (int q = i + 1; q < n; ++q) s -= A[i * n + q] * B[q * m + j];
      B[i * m + j] = s / A[i * n + i];
    }
}

struct K2View {
  const int32_t* edge_ptr;  // nc + 1
  const int32_t* edge_v;    // 2 per local edge
  const int32_t* fpos_v;    // per face_v entry
  const int32_t* fpos_e;
  const int64_t* eptr;      // nc + 1 element-order offsets (n_E per cell)
  const int64_t* k2_off;    // nc + 1
  const int64_t* face_off;  // n_occ + 1
};

// Face data layout (global, per face occurrence): Pi_f (6 x (2k+1)), then
// x_f (3), t1 (3), t2 (3), h_f, area, n (3), one unused.
constexpr int kFaceExtra = 16;

// Per-warp shared layout of the element kernel (doubles):
//   face slots (nf_cap x fslot): F[10] (z-moments), fm[10] (3D monomial face
//   means), frame[14] (xf, t1, t2, hf, area, n), Pi_f (6 x (2 kcap + 1));
//   M[10], G[100], Mm[100], Gf scratch (32 lanes x 36), B, Pis, D, Q.
__host__ __device__ inline int k2_fslot(int kcap) { return 34 + 6 * (2 * kcap + 1); }
__host__ __device__ inline size_t k2_warp_doubles(int nf_cap, int kcap, int ne_cap) {
  return size_t(nf_cap) * k2_fslot(kcap) + 10 + 100 + 100 + 32 * 36 + 4 * size_t(10) * ne_cap;
}

__global__ void k_elem_k2(MeshView m, K2View kv, const double* vol_in, const double* xE_in, const double* h_in,
                          int nf_cap, int kcap, int ne_cap, double* Pis2, double* K2, double* mom_o,
                          double* face_o, int* err) {
  extern __shared__ double smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  const int fslot = k2_fslot(kcap);
  double* base = smem + size_t(warp) * k2_warp_doubles(nf_cap, kcap, ne_cap);
  double* fs = base;
  double* M = fs + size_t(nf_cap) * fslot;
  double* G = M + 10;
  double* Mm = G + 100;
  double* Gf = Mm + 100;  // 32 x 36
  double* B = Gf + 32 * 36;
  double* Pis = B + 10 * ne_cap;
  double* Dm = Pis + 10 * ne_cap;
  double* Q = Dm + 10 * ne_cap;
  for (int c = blockIdx.x * wpb + warp; c < m.nc; c += gridDim.x * wpb) {
    const int vb = m.cell_vptr[c], nv = m.cell_vptr[c + 1] - vb;
    const int fb = m.cell_fptr[c], nf = m.cell_fptr[c + 1] - fb;
    const int eb = kv.edge_ptr[c], ne = kv.edge_ptr[c + 1] - eb;
    const int nE = nv + ne + nf + 1;
    if (nf > nf_cap || nE > ne_cap) {
      if (lane == 0) atomicExch(err, 3);
      continue;
    }
    const double vol = vol_in[c], h = h_in[c];
    const D3 xE{xE_in[3 * c], xE_in[3 * c + 1], xE_in[3 * c + 2]};
    const double ih = 1.0 / h;
    // vertex mean (apex of the tetrahedra)
    D3 c0{0, 0, 0};
    for (int i = lane; i < nv; i += 32) c0 = add3(c0, ld3(m.V, m.cell_v[vb + i]));
    c0 = D3{warp_sum_bcast(c0.x) / nv, warp_sum_bcast(c0.y) / nv, warp_sum_bcast(c0.z) / nv};
    // ---- faces: geometry, moments, face projector (one lane per face)
    double macc[10];
#pragma unroll
    for (int q = 0; q < 10; ++q) macc[q] = 0.0;
    for (int f = lane; f < nf; f += 32) {
      const int s = m.face_vptr[fb + f], k = m.face_vptr[fb + f + 1] - s;
      const int32_t* cyc = m.face_v + s;
      double* F = fs + size_t(f) * fslot;
      double* fm = F + 10;
      double* fr = F + 20;  // xf(3) t1(3) t2(3) hf area n(3)
      double* Pf = F + 34;
      D3 A{0, 0, 0};
      for (int q = 0; q < k; ++q) A = add3(A, crs3(ld3(m.V, cyc[q]), ld3(m.V, cyc[(q + 1) % k])));
      A = mul3(A, 0.5);
      const double area = sqrt(dt3(A, A));
      const D3 n = mul3(A, 1.0 / area);
      const D3 p0 = ld3(m.V, cyc[0]);
      D3 xf{0, 0, 0};
      for (int q = 1; q + 1 < k; ++q) {
        const D3 a = ld3(m.V, cyc[q]), b = ld3(m.V, cyc[q + 1]);
        const D3 cr = crs3(sub3(a, p0), sub3(b, p0));
        const double ar = 0.5 * sqrt(dt3(cr, cr));
        xf = add3(xf, mul3(add3(add3(p0, a), b), ar / 3.0));
      }
      xf = mul3(xf, 1.0 / area);
      D3 t1 = sub3(ld3(m.V, cyc[1]), p0);
      t1 = sub3(t1, mul3(n, dt3(t1, n)));
      t1 = mul3(t1, 1.0 / sqrt(dt3(t1, t1)));
      const D3 t2 = crs3(n, t1);
      double hf2 = 0.0;
      for (int i = 0; i < k; ++i)
        for (int j = i + 1; j < k; ++j) {
          const D3 d = sub3(ld3(m.V, cyc[i]), ld3(m.V, cyc[j]));
          hf2 = fmax(hf2, dt3(d, d));
        }
      const double hf = sqrt(hf2), ihf = 1.0 / hf;
      // z-moments (degree <= 3) and 3D monomial integrals (degree <= 2)
      double Fz[10], F3[10];
#pragma unroll
      for (int q = 0; q < 10; ++q) Fz[q] = F3[q] = 0.0;
      for (int q = 1; q + 1 < k; ++q) {
        const D3 a = ld3(m.V, cyc[q]), b = ld3(m.V, cyc[q + 1]);
        const D3 cr = crs3(sub3(a, p0), sub3(b, p0));
        const double ar = 0.5 * sqrt(dt3(cr, cr));
        D3 pts[7] = {p0, a, b, mul3(add3(p0, a), 0.5), mul3(add3(a, b), 0.5), mul3(add3(b, p0), 0.5),
                     mul3(add3(add3(p0, a), b), 1.0 / 3.0)};
        const double wts[7] = {1.0 / 20, 1.0 / 20, 1.0 / 20, 2.0 / 15, 2.0 / 15, 2.0 / 15, 9.0 / 20};
        for (int p = 0; p < 7; ++p) {
          const D3 d = sub3(pts[p], xf);
          double mz[10], m3[10];
          mono2v(dt3(d, t1) * ihf, dt3(d, t2) * ihf, mz);
          mono3v(mul3(sub3(pts[p], xE), ih), m3);
          const double w = wts[p] * ar;
#pragma unroll
          for (int q = 0; q < 10; ++q) {
            Fz[q] += w * mz[q];
            F3[q] += w * m3[q];
          }
        }
      }
      for (int q = 0; q < 10; ++q) {
        F[q] = Fz[q];
        fm[q] = F3[q] / area;
      }
      fr[0] = xf.x; fr[1] = xf.y; fr[2] = xf.z;
      fr[3] = t1.x; fr[4] = t1.y; fr[5] = t1.z;
      fr[6] = t2.x; fr[7] = t2.y; fr[8] = t2.z;
      fr[9] = hf; fr[10] = area;
      fr[11] = n.x; fr[12] = n.y; fr[13] = n.z;
      // G_f (6 x 6): first row P0 = face mean; B_f (6 x (2k+1)) into Pf
      double* g = Gf + lane * 36;
      for (int a = 0; a < 6; ++a)
        for (int b2 = 0; b2 < 6; ++b2) {
          double v = 0.0;
          for (int d = 0; d < 2; ++d) {
            const int ea = kE2[a][d], eb2 = kE2[b2][d];
            if (!ea || !eb2) continue;
            const int i0 = idx2(kE2[a][0] + kE2[b2][0] - 2 * (d == 0), kE2[a][1] + kE2[b2][1] - 2 * (d == 1));
            v += double(ea * eb2) * Fz[i0];
          }
          g[a * 6 + b2] = v * ihf * ihf;
        }
      for (int b2 = 0; b2 < 6; ++b2) g[b2] = Fz[b2] / area;
      const int nfd = 2 * k + 1;
      for (int q = 0; q < 6 * nfd; ++q) Pf[q] = 0.0;
      Pf[2 * k] = 1.0;
      for (int a = 1; a < 6; ++a) {
        const int sq = (kE2[a][0] == 2) + (kE2[a][1] == 2);
        Pf[a * nfd + 2 * k] = -(2.0 * sq * ihf * ihf) * area;
      }
      for (int q = 0; q < k; ++q) {
        const D3 a = ld3(m.V, cyc[q]), b = ld3(m.V, cyc[(q + 1) % k]);
        const D3 e = sub3(b, a);
        const double L = sqrt(dt3(e, e));
        const D3 nE = mul3(crs3(e, n), 1.0 / L);
        const double c1 = dt3(t1, nE) * ihf, c2 = dt3(t2, nE) * ihf;
        const D3 nodes[3] = {a, mul3(add3(a, b), 0.5), b};
        const double w3[3] = {1.0 / 6.0, 4.0 / 6.0, 1.0 / 6.0};
        const int dofs[3] = {q, k + q, (q + 1) % k};
        for (int p = 0; p < 3; ++p) {
          const D3 d = sub3(nodes[p], xf);
          const double z1 = dt3(d, t1) * ihf, z2 = dt3(d, t2) * ihf;
          // d/dz of 1, z1, z2, z1^2, z1 z2, z2^2
          const double d1[6] = {0, 1, 0, 2 * z1, z2, 0}, d2[6] = {0, 0, 1, 0, z1, 2 * z2};
          for (int a2 = 1; a2 < 6; ++a2) Pf[a2 * nfd + dofs[p]] += L * w3[p] * (d1[a2] * c1 + d2[a2] * c2);
        }
      }
      small_solve(g, 6, Pf, nfd);
      // the same face data to global memory (coarse levels use it in the prolongation)
      double* go = face_o + kv.face_off[fb + f];
      for (int q = 0; q < 6 * nfd; ++q) go[q] = Pf[q];
      for (int q = 0; q < 14; ++q) go[6 * nfd + q] = fr[q];
      go[6 * nfd + 14] = 0.0;
      go[6 * nfd + 15] = 0.0;
      // cell moments over this face's tetrahedra (apex c0)
      for (int q = 1; q + 1 < k; ++q) {
        const D3 a = ld3(m.V, cyc[q]), b = ld3(m.V, cyc[q + 1]);
        const double tv = fabs(dt3(sub3(p0, c0), crs3(sub3(a, c0), sub3(b, c0)))) / 6.0;
        const D3 vt[4] = {c0, p0, a, b};
        for (int i = 0; i < 4; ++i) {
          double m3[10];
          mono3v(mul3(sub3(vt[i], xE), ih), m3);
          for (int r = 0; r < 10; ++r) macc[r] -= tv / 20.0 * m3[r];
          for (int j = i + 1; j < 4; ++j) {
            mono3v(mul3(sub3(mul3(add3(vt[i], vt[j]), 0.5), xE), ih), m3);
            for (int r = 0; r < 10; ++r) macc[r] += tv / 5.0 * m3[r];
          }
        }
      }
    }
    for (int r = 0; r < 10; ++r) {
      const double v = warp_sum_bcast(macc[r]);
      if (lane == 0) M[r] = v;
    }
    __syncwarp();
    // ---- G (10 x 10), first row P0 = cell mean; Gt = G with row 0 zeroed goes to Mm
    for (int p = lane; p < 100; p += 32) {
      const int a = p / 10, b = p % 10;
      double v = 0.0;
      for (int d = 0; d < 3; ++d) {
        const int ea = kE3[a][d], eb = kE3[b][d];
        if (!ea || !eb) continue;
        const int i0 = idx3(kE3[a][0] + kE3[b][0] - 2 * (d == 0), kE3[a][1] + kE3[b][1] - 2 * (d == 1),
                            kE3[a][2] + kE3[b][2] - 2 * (d == 2));
        v += double(ea * eb) * M[i0];
      }
      v *= ih * ih;
      Mm[p] = a == 0 ? 0.0 : v;
      G[p] = a == 0 ? M[b] / vol : v;
    }
    // ---- B (10 x nE): volume term and row 0
    for (int p = lane; p < 10 * nE; p += 32) B[p] = 0.0;
    __syncwarp();
    if (lane == 0) {
      B[nE - 1] = 1.0;
      for (int a = 1; a < 10; ++a) {
        const int sq = (kE3[a][0] == 2) + (kE3[a][1] == 2) + (kE3[a][2] == 2);
        B[a * nE + nE - 1] = -(2.0 * sq * ih * ih) * vol;
      }
    }
    __syncwarp();
    // face terms: int_f Pi_f phi_j (grad m_a . n_f), grad m_a . n_f linear on f
    for (int f = 0; f < nf; ++f) {
      const int s = m.face_vptr[fb + f], k = m.face_vptr[fb + f + 1] - s;
      const double* F = fs + size_t(f) * fslot;
      const double* fr = F + 20;
      const double* Pf = F + 34;
      const int nfd = 2 * k + 1;
      const D3 xf{fr[0], fr[1], fr[2]}, t1{fr[3], fr[4], fr[5]}, t2{fr[6], fr[7], fr[8]}, n{fr[11], fr[12], fr[13]};
      const double hf = fr[9];
      const D3 y0 = mul3(sub3(xf, xE), ih);
      for (int p = lane; p < 9 * nfd; p += 32) {
        const int a = 1 + p / nfd, j = p % nfd;
        // q_a(x) = grad m_a . n = (1/h) sum_d e_d Y^(e - e_d) n_d, linear in Y
        double q0 = 0.0;  // value at x_f
        D3 gq{0, 0, 0};   // gradient in x
        for (int d = 0; d < 3; ++d) {
          const int ed = kE3[a][d];
          if (!ed) continue;
          const double nd = d == 0 ? n.x : (d == 1 ? n.y : n.z);
          int e0 = kE3[a][0] - (d == 0), e1 = kE3[a][1] - (d == 1), e2 = kE3[a][2] - (d == 2);
          // the remaining monomial has degree 0 or 1
          const double yv = (e0 ? y0.x : 1.0) * (e1 ? y0.y : 1.0) * (e2 ? y0.z : 1.0);
          q0 += ed * nd * ih * yv;
          if (e0) gq.x += ed * nd * ih * ih;
          if (e1) gq.y += ed * nd * ih * ih;
          if (e2) gq.z += ed * nd * ih * ih;
        }
        const double c1 = hf * dt3(gq, t1), c2 = hf * dt3(gq, t2);
        double mom = 0.0;
        for (int b2 = 0; b2 < 6; ++b2) {
          const int ez1 = kE2[b2][0], ez2 = kE2[b2][1];
          mom += Pf[b2 * nfd + j] * (q0 * F[b2] + c1 * F[idx2(ez1 + 1, ez2)] + c2 * F[idx2(ez1, ez2 + 1)]);
        }
        int pos;
        if (j < k)
          pos = kv.fpos_v[s + j];
        else if (j < 2 * k)
          pos = nv + kv.fpos_e[s + (j - k)];
        else
          pos = nv + ne + f;
        B[a * nE + pos] += mom;
      }
      __syncwarp();
    }
    // ---- Pi* = G^-1 B
    for (int p = lane; p < 10 * nE; p += 32) Pis[p] = B[p];
    __syncwarp();
    if (lane == 0) small_solve(G, 10, Pis, nE);
    __syncwarp();
    // ---- D (nE x 10): DOFs of the monomials
    for (int i = lane; i < nE; i += 32) {
      double mv[10];
      if (i < nv) {
        mono3v(mul3(sub3(ld3(m.V, m.cell_v[vb + i]), xE), ih), mv);
      } else if (i < nv + ne) {
        const int q = eb + (i - nv);
        const D3 x = mul3(add3(ld3(m.V, kv.edge_v[2 * q]), ld3(m.V, kv.edge_v[2 * q + 1])), 0.5);
        mono3v(mul3(sub3(x, xE), ih), mv);
      } else if (i < nv + ne + nf) {
        const double* fm = fs + size_t(i - nv - ne) * fslot + 10;
        for (int a = 0; a < 10; ++a) mv[a] = fm[a];
      } else {
        for (int a = 0; a < 10; ++a) mv[a] = M[a] / vol;
      }
      for (int a = 0; a < 10; ++a) Dm[i * 10 + a] = mv[a];
    }
    __syncwarp();
    // ---- Mm = Gt + h D^T D
    for (int p = lane; p < 100; p += 32) {
      const int a = p / 10, b = p % 10;
      double v = 0.0;
      for (int i = 0; i < nE; ++i) v += Dm[i * 10 + a] * Dm[i * 10 + b];
      Mm[p] += h * v;
    }
    __syncwarp();
    // ---- Q = Mm Pi*
    for (int p = lane; p < 10 * nE; p += 32) {
      const int a = p / nE, j = p % nE;
      double v = 0.0;
      for (int b = 0; b < 10; ++b) v += Mm[a * 10 + b] * Pis[b * nE + j];
      Q[p] = v;
    }
    __syncwarp();
    // ---- K = Pi*^T Q - h (Pi + Pi^T) + h I,  Pi = D Pi*
    double* Ko = K2 + kv.k2_off[c];
    for (int p = lane; p < nE * nE; p += 32) {
      const int i = p / nE, j = p % nE;
      double cons = 0.0, pij = 0.0, pji = 0.0;
      for (int a = 0; a < 10; ++a) {
        cons += Pis[a * nE + i] * Q[a * nE + j];
        pij += Dm[i * 10 + a] * Pis[a * nE + j];
        pji += Dm[j * 10 + a] * Pis[a * nE + i];
      }
      Ko[p] = cons + h * ((i == j ? 1.0 : 0.0) - pij - pji);
    }
    double* Po = Pis2 + 10 * kv.eptr[c];
    for (int p = lane; p < 10 * nE; p += 32) Po[p] = Pis[p];
    if (lane < 10) mom_o[10 * size_t(c) + lane] = M[lane];
    __syncwarp();
  }
}

// Condensed element blocks (reading K2): for the cell DOF c (last in element
// order) K~ = K_bb - K_bc K_cb / K_cc, written in the order of the sorted
// boundary list (perm: element position -> sorted position).
__global__ void k_condense_k2(int nc, const int64_t* eptr, const int64_t* k2_off, const double* K2,
                              const int32_t* perm, const int64_t* kptr, double* Kt) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, wpb = blockDim.x >> 5;
  for (int c = blockIdx.x * wpb + warp; c < nc; c += gridDim.x * wpb) {
    const int nE = int(eptr[c + 1] - eptr[c]), nb = nE - 1;
    const double* K = K2 + k2_off[c];
    const int32_t* pm = perm + eptr[c];
    double* out = Kt + kptr[c];
    const double icc = 1.0 / K[nb * nE + nb];
    for (int p = lane; p < nb * nb; p += 32) {
      const int i = p / nb, j = p % nb;
      out[size_t(pm[i]) * nb + pm[j]] = K[i * nE + j] - K[i * nE + nb] * K[nb * nE + j] * icc;
    }
  }
}

// k = 2 right-hand side (Sec. 3.2): r_i = int_E Pi_1 u' . grad Pi_2 phi_i with
// Pi_1 u' from the k = 1 projector of the same cell (same centroid and
// diameter), condensed per cell: r~_b = r_b - K_bc r_c / K_cc (sorted boundary
// order into rloc at elem_vptr offsets); the cell entry r_c is kept for the
// recovery of the cell DOF.
__global__ void k_rhs_k2(MeshView m, const double* Pis1, const double* hE, const double* u, int64_t nvtx,
                         const int64_t* eptr, const double* Pis2, const double* mom, const int64_t* k2_off,
                         const double* K2, const int32_t* perm, const int32_t* elem_vptr, double* rloc, double* rc) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.nc) return;
  const int vb = m.cell_vptr[c], nv = m.cell_vptr[c + 1] - vb;
  const double* P1 = Pis1 + 4 * size_t(vb);
  double s[3][4];
  for (int d = 0; d < 3; ++d)
    for (int a = 0; a < 4; ++a) s[d][a] = 0.0;
  for (int j = 0; j < nv; ++j) {
    const int g = m.cell_v[vb + j];
    const double uj[3] = {u[g], u[nvtx + g], u[2 * nvtx + g]};
    for (int a = 0; a < 4; ++a) {
      const double pa = P1[a * nv + j];
      for (int d = 0; d < 3; ++d) s[d][a] += pa * uj[d];
    }
  }
  const double* M = mom + 10 * size_t(c);
  const double ih = 1.0 / hE[c];
  double I[10];
  for (int a = 0; a < 10; ++a) {
    double v = 0.0;
    for (int d = 0; d < 3; ++d) {
      const int ed = kE3[a][d];
      if (!ed) continue;
      const int e0 = kE3[a][0] - (d == 0), e1 = kE3[a][1] - (d == 1), e2 = kE3[a][2] - (d == 2);
      double t = s[d][0] * M[idx3(e0, e1, e2)];
      t += s[d][1] * M[idx3(e0 + 1, e1, e2)] + s[d][2] * M[idx3(e0, e1 + 1, e2)] + s[d][3] * M[idx3(e0, e1, e2 + 1)];
      v += ed * t;
    }
    I[a] = v * ih;
  }
  const int nE = int(eptr[c + 1] - eptr[c]), nb = nE - 1;
  const double* P2 = Pis2 + 10 * eptr[c];
  const double* K = K2 + k2_off[c];
  double r_c = 0.0;
  for (int a = 0; a < 10; ++a) r_c += P2[a * nE + nb] * I[a];
  const double f = r_c / K[nb * nE + nb];
  const int32_t* pm = perm + eptr[c];
  double* out = rloc + elem_vptr[c];
  for (int i = 0; i < nb; ++i) {
    double ri = 0.0;
    for (int a = 0; a < 10; ++a) ri += P2[a * nE + i] * I[a];
    out[pm[i]] = ri - K[i * nE + nb] * f;
  }
  rc[c] = r_c;
}

// Recovery of the cell DOFs and the velocity correction (Sec. 3.3) for k = 2:
// p_c = (r_c - sum_b K_cb p_b) / K_cc; Pi_1 u_new = Pi_1 u' - grad Pi_2 p, 12
// numbers per cell in the k = 1 layout; the cell DOFs go to p_all[cdof + c].
__global__ void k_correct_k2(MeshView m, const double* Pis1, const double* hE, const double* u, int64_t nvtx,
                             const int64_t* eptr, const int64_t* edof, const double* Pis2, const int64_t* k2_off,
                             const double* K2, const double* rc, const double* p_all_b, int64_t cdof, double* p_all,
                             double* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.nc) return;
  const int nE = int(eptr[c + 1] - eptr[c]), nb = nE - 1;
  const int64_t* ids = edof + eptr[c];
  const double* K = K2 + k2_off[c];
  const double* P2 = Pis2 + 10 * eptr[c];
  double coef[10];
  for (int a = 0; a < 10; ++a) coef[a] = 0.0;
  double acc = rc[c];
  for (int i = 0; i < nb; ++i) {
    const double pi = p_all_b[ids[i]];
    acc -= K[nb * nE + i] * pi;
    for (int a = 0; a < 10; ++a) coef[a] += P2[a * nE + i] * pi;
  }
  const double pcell = acc / K[nb * nE + nb];
  for (int a = 0; a < 10; ++a) coef[a] += P2[a * nE + nb] * pcell;
  p_all[cdof + c] = pcell;
  const double ih = 1.0 / hE[c];
  double g[3][4];
  for (int d = 0; d < 3; ++d)
    for (int a = 0; a < 4; ++a) g[d][a] = 0.0;
  for (int a = 1; a < 10; ++a)
    for (int d = 0; d < 3; ++d) {
      const int ed = kE3[a][d];
      if (!ed) continue;
      const int e0 = kE3[a][0] - (d == 0), e1 = kE3[a][1] - (d == 1), e2 = kE3[a][2] - (d == 2);
      const int slot = (e0 + e1 + e2 == 0) ? 0 : (e0 ? 1 : (e1 ? 2 : 3));
      g[d][slot] += coef[a] * ed * ih;
    }
  const int vb = m.cell_vptr[c], nv = m.cell_vptr[c + 1] - vb;
  const double* P1 = Pis1 + 4 * size_t(vb);
  for (int d = 0; d < 3; ++d)
    for (int a = 0; a < 4; ++a) {
      double s = 0.0;
      for (int j = 0; j < nv; ++j) s += P1[a * nv + j] * u[d * nvtx + m.cell_v[vb + j]];
      out[12 * size_t(c) + 4 * d + a] = s - g[d][a];
    }
}

// Diffusion-free prolongation for k = 2 (Sec. 4.2, Eq. 17 extended to the
// k = 2 DOFs), one thread per fine boundary DOF: point DOFs take the coarse
// function at their placement (a copy, the quadratic through a coarse edge's
// three DOFs, Pi_{2,F}, Pi_2 of the coarse cell), face means the mean over
// the fine face of the coarse face or cell polynomial; weights on a coarse
// cell DOF are folded into that cell's boundary DOFs by the harmonic
// extension of the coarse element (reading K2): w_b -= w_c K_bc / K_cc.
struct ProlongK2 {
  const int8_t* kind;
  const int32_t* C;
  const int32_t* a;
  const int32_t* b;
  const double* x;
};

__device__ __forceinline__ void face_frame(const double* fd, int nfd, D3& xf, D3& t1, D3& t2, double& hf) {
  const double* fr = fd + 6 * nfd;
  xf = D3{fr[0], fr[1], fr[2]};
  t1 = D3{fr[3], fr[4], fr[5]};
  t2 = D3{fr[6], fr[7], fr[8]};
  hf = fr[9];
}

__global__ void k_prolong_k2(int64_t nrows, ProlongK2 pr, MeshView fm, MeshView cm, const int64_t* c_eptr,
                             const double* c_Pis2, const double* c_xE, const double* c_h, const int64_t* c_k2_off,
                             const double* c_K2, const double* c_face, const int64_t* c_face_off,
                             const int32_t* prow_ptr, double* prow_val) {
  const int64_t g = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (g >= nrows) return;
  double* w = prow_val + prow_ptr[g];
  const int kind = pr.kind[g];
  const D3 x{pr.x[3 * g], pr.x[3 * g + 1], pr.x[3 * g + 2]};
  if (kind == 0) {
    w[0] = 1.0;
    return;
  }
  if (kind == 1) {
    const D3 a = ld3(cm.V, pr.a[g]), b = ld3(cm.V, pr.b[g]);
    const D3 e = sub3(b, a);
    const double t = dt3(sub3(x, a), e) / dt3(e, e);
    w[0] = (1.0 - t) * (1.0 - 2.0 * t);
    w[1] = t * (2.0 * t - 1.0);
    w[2] = 4.0 * t * (1.0 - t);
    return;
  }
  if (kind == 2 || kind == 4) {
    const int fo = pr.a[g];
    const int k = cm.face_vptr[fo + 1] - cm.face_vptr[fo], nfd = 2 * k + 1;
    const double* fd = c_face + c_face_off[fo];
    D3 xf, t1, t2;
    double hf;
    face_frame(fd, nfd, xf, t1, t2, hf);
    double mz[10];
    if (kind == 2) {
      const D3 d = sub3(x, xf);
      mono2v(dt3(d, t1) / hf, dt3(d, t2) / hf, mz);
    } else {
      // mean over the fine face of the coarse face's monomials (fan of
      // triangles, edge-midpoint rule, exact for degree 2)
      const int fo_f = pr.b[g];
      const int s = fm.face_vptr[fo_f], kk = fm.face_vptr[fo_f + 1] - s;
      for (int q = 0; q < 6; ++q) mz[q] = 0.0;
      double tot = 0.0;
      const D3 p0 = ld3(fm.V, fm.face_v[s]);
      for (int q = 1; q + 1 < kk; ++q) {
        const D3 pa = ld3(fm.V, fm.face_v[s + q]), pb = ld3(fm.V, fm.face_v[s + q + 1]);
        const D3 cr = crs3(sub3(pa, p0), sub3(pb, p0));
        const double ar = 0.5 * sqrt(dt3(cr, cr));
        const D3 mids[3] = {mul3(add3(p0, pa), 0.5), mul3(add3(pa, pb), 0.5), mul3(add3(pb, p0), 0.5)};
        for (int p = 0; p < 3; ++p) {
          const D3 d = sub3(mids[p], xf);
          double mm[10];
          mono2v(dt3(d, t1) / hf, dt3(d, t2) / hf, mm);
          for (int q2 = 0; q2 < 6; ++q2) mz[q2] += ar / 3.0 * mm[q2];
        }
        tot += ar;
      }
      for (int q = 0; q < 6; ++q) mz[q] /= tot;
    }
    for (int j = 0; j < nfd; ++j) {
      double v = 0.0;
      for (int b2 = 0; b2 < 6; ++b2) v += mz[b2] * fd[b2 * nfd + j];
      w[j] = v;
    }
    return;
  }
  // kinds 3 and 5: coarse cell polynomial Pi_2 of cell C
  const int C = pr.C[g];
  const int nE = int(c_eptr[C + 1] - c_eptr[C]), nb = nE - 1;
  const D3 xc{c_xE[3 * C], c_xE[3 * C + 1], c_xE[3 * C + 2]};
  const double ihc = 1.0 / c_h[C];
  double mv[10];
  if (kind == 3) {
    mono3v(mul3(sub3(x, xc), ihc), mv);
  } else {
    const int fo_f = pr.b[g];
    const int s = fm.face_vptr[fo_f], kk = fm.face_vptr[fo_f + 1] - s;
    for (int q = 0; q < 10; ++q) mv[q] = 0.0;
    double tot = 0.0;
    const D3 p0 = ld3(fm.V, fm.face_v[s]);
    for (int q = 1; q + 1 < kk; ++q) {
      const D3 pa = ld3(fm.V, fm.face_v[s + q]), pb = ld3(fm.V, fm.face_v[s + q + 1]);
      const D3 cr = crs3(sub3(pa, p0), sub3(pb, p0));
      const double ar = 0.5 * sqrt(dt3(cr, cr));
      const D3 mids[3] = {mul3(add3(p0, pa), 0.5), mul3(add3(pa, pb), 0.5), mul3(add3(pb, p0), 0.5)};
      for (int p = 0; p < 3; ++p) {
        double mm[10];
        mono3v(mul3(sub3(mids[p], xc), ihc), mm);
        for (int q2 = 0; q2 < 10; ++q2) mv[q2] += ar / 3.0 * mm[q2];
      }
      tot += ar;
    }
    for (int q = 0; q < 10; ++q) mv[q] /= tot;
  }
  const double* P2 = c_Pis2 + 10 * c_eptr[C];
  const double* K = c_K2 + c_k2_off[C];
  double wc = 0.0;
  for (int a = 0; a < 10; ++a) wc += mv[a] * P2[a * nE + nb];
  const double f = wc / K[nb * nE + nb];
  for (int j = 0; j < nb; ++j) {
    double v = 0.0;
    for (int a = 0; a < 10; ++a) v += mv[a] * P2[a * nE + j];
    w[j] = v - K[j * nE + nb] * f;
  }
}

// ---- diagonal scaling of the k = 2 hierarchy (reading K1)
// s[i] = 1/sqrt(A_ii) from the CSR of a level.
__global__ void k_csr_invsqrt_diag(int64_t n, const int64_t* rp, const int32_t* col, const double* val, double* s) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double d = 0.0;
  for (int64_t q = rp[i]; q < rp[i + 1]; ++q)
    if (col[q] == i) d = val[q];
  s[i] = 1.0 / sqrt(d);
}
// A'_ij = s_i A_ij s_j (in place), one thread per row
__global__ void k_csr_scale_sym(int64_t n, const int64_t* rp, const int32_t* col, const double* s, double* val) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double si = s[i];
  for (int64_t q = rp[i]; q < rp[i + 1]; ++q) val[q] *= si * s[col[q]];
}
// P'_ij = P_ij s_c[j] / s_f[i] (P' = D_f^1/2 P D_c^-1/2 with s = D^-1/2), in place
__global__ void k_csr_scale_p(int64_t n, const int64_t* rp, const int32_t* col, const double* sf, const double* sc,
                              double* val) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double inv = 1.0 / sf[i];
  for (int64_t q = rp[i]; q < rp[i + 1]; ++q) val[q] *= sc[col[q]] * inv;
}
// y = s .* x in the type of y
template <typename A, typename B>
__global__ void k_scale_to(int64_t n, const double* __restrict__ s, const A* __restrict__ x, B* __restrict__ y) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = B(s[i] * double(x[i]));
}

}  // namespace fvem
