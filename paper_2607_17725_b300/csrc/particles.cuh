// Particle transfers around the projection (Sec. 3.2 P2G, Sec. 3.3 G2P and
// advection) on the level-0 cut-cell grid.
//
// Layouts: particle positions and velocities are SoA (all x, then y, then z;
// n_p each), per-particle cells int32 (-1: inside an obstacle or outside the
// box), vertex values SoA over the level-0 vertices, cell polynomials
// [cell][component][monomial 1, (x - x_E)/h_E] (12 per cell).
//
// Binning: the N^3 background cubes.  Particles are counted per cube,
// scattered by an exclusive scan and each cube's list sorted by particle id,
// so every vertex sums its particles in one fixed order (bitwise
// reproducible).  A particle record holds its offset from its cube's corner
// in FP32 (|offset| < h, so rounding is about 6e-8 h) and up to four values.
#pragma once
#include <cstdint>

namespace fvem {

constexpr int kScanTile = 2048;  // elements per block of the scan (256 threads x 8)
constexpr double kLocateTol = 1e-10;

struct PartGridView {
  int N;
  double h;
  const int32_t* cbin_ptr;   // N^3 + 1: level-0 cells per cube, ascending
  const int32_t* cbin_cell;
  const uint8_t* cbin_full;  // 1: the cube's one cell is the whole cube
  const double4* fplane;     // per face occurrence: outward unit normal, d = n . face mean
  const int32_t* cell_fptr;
  const double* tri;         // 9 per obstacle triangle
  const int32_t* tbin_ptr;   // N^3 + 1: triangles whose box meets each cube
  const int32_t* tbin_tri;
};

__device__ __forceinline__ int cube_index(double x, int N) {
  const double t = x * double(N);
  if (!(t >= 0.0)) return 0;  // also NaN
  return t >= double(N) ? N - 1 : int(t);
}

// ------------------------------------------------------------------ binning

__global__ void k_part_count(int64_t np, const double* x, const int32_t* cell, int N, int32_t* count,
                             int32_t* bin, int32_t* rank) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const double a = x[p], b = x[np + p], c = x[2 * np + p];
  const bool ok = (cell == nullptr || cell[p] >= 0) && isfinite(a) && isfinite(b) && isfinite(c);
  if (!ok) {
    bin[p] = -1;
    return;
  }
  const int q = (cube_index(c, N) * N + cube_index(b, N)) * N + cube_index(a, N);
  bin[p] = q;
  rank[p] = atomicAdd(&count[q], 1);
}

// Exclusive scan of n int32 in three passes: per-tile scans with tile sums,
// one block over the tile sums (carried across chunks), then the tile
// offsets added.  out may alias in.
__global__ void __launch_bounds__(256) k_scan_tiles(int64_t n, const int32_t* in, int32_t* out, int32_t* tsum) {
  __shared__ int32_t wsum[8];
  const int64_t base = int64_t(blockIdx.x) * kScanTile + int64_t(threadIdx.x) * 8;
  int32_t v[8], s = 0;
  for (int k = 0; k < 8; ++k) {
    v[k] = base + k < n ? in[base + k] : 0;
    s += v[k];
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int32_t inc = s;
  for (int o = 1; o < 32; o <<= 1) {
    const int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  int32_t wpre = 0;
  for (int k = 0; k < w; ++k) wpre += wsum[k];
  int32_t run = wpre + inc - s;
  for (int k = 0; k < 8; ++k) {
    if (base + k < n) out[base + k] = run;
    run += v[k];
  }
  if (threadIdx.x == 255) tsum[blockIdx.x] = wpre + inc;
}

__global__ void __launch_bounds__(1024) k_scan_sums(int64_t nt, int32_t* tsum) {
  __shared__ int32_t wsum[32];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t b0 = 0; b0 < nt; b0 += 1024) {
    const int64_t i = b0 + threadIdx.x;
    const int32_t v = i < nt ? tsum[i] : 0;
    int32_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
      const int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += t;
    }
    if (lane == 31) wsum[w] = inc;
    __syncthreads();
    int32_t wpre = 0;
    for (int k = 0; k < w; ++k) wpre += wsum[k];
    const int32_t c = carry;
    if (i < nt) tsum[i] = c + wpre + inc - v;
    __syncthreads();
    if (threadIdx.x == 1023) carry = c + wpre + inc;
    __syncthreads();
  }
}

__global__ void k_scan_add(int64_t n, int32_t* out, const int32_t* tsum) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i < n) out[i] += tsum[i / kScanTile];
}

__global__ void k_part_scatter(int64_t np, const int32_t* bin, const int32_t* rank, const int32_t* off,
                               int32_t* idx) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= np || bin[p] < 0) return;
  idx[off[bin[p]] + rank[p]] = int32_t(p);
}

// Each cube's particle ids in ascending order (the atomic ranks are not
// reproducible; the sorted order is).  Insertion sort: cubes hold a handful.
// A cube with more than kSortCap particles keeps its atomic order, which
// bounds every thread's work (kSortCap^2 steps); its sums then differ
// between runs by rounding only.
constexpr int kSortCap = 1024;

__global__ void k_part_sort(int64_t nbin, const int32_t* off, int32_t* idx) {
  const int64_t b = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (b >= nbin) return;
  const int s = off[b], e = off[b + 1];
  if (e - s > kSortCap) return;
  for (int i = s + 1; i < e; ++i) {
    const int32_t v = idx[i];
    int j = i - 1;
    while (j >= s && idx[j] > v) {
      idx[j + 1] = idx[j];
      --j;
    }
    idx[j + 1] = v;
  }
}

// Sorted records: offset from the cube's corner (FP32) and the values.
__global__ void k_part_pack(const int32_t* nrec, const int32_t* idx, const int32_t* bin, int64_t np, const double* x,
                            const double* f, int nch, int N, double h, float4* rpos, float4* rval) {
  const int64_t j = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (j >= *nrec) return;  // the live particles: the scan's last offset
  const int32_t p = idx[j];
  const int q = bin[p];
  const int i = q % N, jj = (q / N) % N, k = q / (N * N);
  rpos[j] = make_float4(float(x[p] - i * h), float(x[np + p] - jj * h), float(x[2 * np + p] - k * h), 0.f);
  float v[4] = {0.f, 0.f, 0.f, 0.f};
  for (int c = 0; c < nch; ++c) v[c] = float(f[int64_t(c) * np + p]);
  rval[j] = make_float4(v[0], v[1], v[2], v[3]);
}

// P2G gather (Sec. 3.2): thread per vertex; the cubes that can hold a
// particle within R = h of x_i are floor((x - R) N) .. ceil((x + R) N) - 1
// per axis (2 per axis for a lattice vertex, 3 otherwise).  Distances in
// FP32 from the cube corner's offset (FP64, rounded once) plus the record's
// offset; sums in FP32, the normalisation in FP64.  No particle in range: 0.
__global__ void __launch_bounds__(256) k_p2g(int nv, const double* V, int N, double h, const int32_t* off,
                                             const float4* rpos, const float4* rval, int nch, double* out) {
  const int v = blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const double px = V[3 * size_t(v)], py = V[3 * size_t(v) + 1], pz = V[3 * size_t(v) + 2];
  const double dN = double(N);
  int lo[3], hi[3];
  const double pc[3] = {px, py, pz};
  for (int d = 0; d < 3; ++d) {
    lo[d] = max(0, int(floor((pc[d] - h) * dN)));
    hi[d] = min(N - 1, int(ceil((pc[d] + h) * dN)) - 1);
  }
  const float inv_r2 = float(1.0 / (h * h));
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  float ws = 0.f;
  for (int k = lo[2]; k <= hi[2]; ++k) {
    const float oz = float(k * h - pz);
    for (int j = lo[1]; j <= hi[1]; ++j) {
      const float oy = float(j * h - py);
      for (int i = lo[0]; i <= hi[0]; ++i) {
        const float ox = float(i * h - px);
        const int q = (k * N + j) * N + i;
        for (int r = off[q]; r < off[q + 1]; ++r) {
          const float4 o = rpos[r];
          const float dx = ox + o.x, dy = oy + o.y, dz = oz + o.z;
          const float qq = (dx * dx + dy * dy + dz * dz) * inv_r2;
          if (qq < 1.f) {
            const float t = 1.f - qq, w = t * t * t;
            const float4 f = rval[r];
            acc.x += w * f.x;
            acc.y += w * f.y;
            acc.z += w * f.z;
            acc.w += w * f.w;
            ws += w;
          }
        }
      }
    }
  }
  const double iw = ws > 0.f ? 1.0 / double(ws) : 0.0;
  out[v] = double(acc.x) * iw;
  if (nch > 1) out[int64_t(nv) + v] = double(acc.y) * iw;
  if (nch > 2) out[2 * int64_t(nv) + v] = double(acc.z) * iw;
  if (nch > 3) out[3 * int64_t(nv) + v] = double(acc.w) * iw;
}

// ------------------------------------------------------------------ location

// Lowest-numbered cell of x's cube whose closed face half-spaces hold x
// within kLocateTol; -1 outside [0, 1]^3 or in no fluid cell of the cube.
__device__ int locate_point(const PartGridView& g, double x, double y, double z) {
  if (!(x >= 0.0 && x <= 1.0 && y >= 0.0 && y <= 1.0 && z >= 0.0 && z <= 1.0)) return -1;
  const int q = (cube_index(z, g.N) * g.N + cube_index(y, g.N)) * g.N + cube_index(x, g.N);
  const int s = g.cbin_ptr[q], e = g.cbin_ptr[q + 1];
  if (e - s == 1 && g.cbin_full[q]) return g.cbin_cell[s];
  for (int r = s; r < e; ++r) {
    const int c = g.cbin_cell[r];
    bool in = true;
    for (int f = g.cell_fptr[c]; f < g.cell_fptr[c + 1] && in; ++f) {
      const double4 P = g.fplane[f];
      in = P.x * x + P.y * y + P.z * z - P.w <= kLocateTol;
    }
    if (in) return c;
  }
  return -1;
}

__global__ void k_locate(int64_t np, const double* x, PartGridView g, int32_t* cell) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= np) return;
  cell[p] = locate_point(g, x[p], x[np + p], x[2 * np + p]);
}

// ------------------------------------------------------------------ G2P

// Pi_1 u per cell from vertex values (the velocity part of the correction).
__global__ void k_cell_linear(MeshView m, const double* Pis, const double* u, int64_t nvtx, double* out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= m.nc) return;
  const int vb = m.cell_vptr[c], n = m.cell_vptr[c + 1] - vb;
  const double* P = Pis + 4 * size_t(vb);
  double s[3][4] = {};
  for (int j = 0; j < n; ++j) {
    const int g = m.cell_v[vb + j];
    const double uj[3] = {u[g], u[nvtx + g], u[2 * nvtx + g]};
    for (int a = 0; a < 4; ++a) {
      const double pa = P[a * n + j];
      s[0][a] += pa * uj[0];
      s[1][a] += pa * uj[1];
      s[2][a] += pa * uj[2];
    }
  }
  for (int cc = 0; cc < 3; ++cc)
    for (int a = 0; a < 4; ++a) out[12 * size_t(c) + 4 * cc + a] = s[cc][a];
}

__device__ __forceinline__ void eval_linear(const double* poly, const double* xE, const double* hE, int c, double x,
                                            double y, double z, double v[3]) {
  const double ih = 1.0 / hE[c];
  const double a = (x - xE[3 * size_t(c)]) * ih, b = (y - xE[3 * size_t(c) + 1]) * ih,
               d = (z - xE[3 * size_t(c) + 2]) * ih;
  const double* P = poly + 12 * size_t(c);
  for (int k = 0; k < 3; ++k) v[k] = P[4 * k] + P[4 * k + 1] * a + P[4 * k + 2] * b + P[4 * k + 3] * d;
}

// u_p <- alpha (u_p + Delta u(x_p)) + (1 - alpha) Pi_1 u_new(x_p), the
// standard FLIP blend; particles with cell -1 (or no valid cell id) keep
// their velocity.
__global__ void k_g2p(int64_t np, const double* x, const int32_t* cell, int nc, const double* xE, const double* hE,
                      const double* lin_old, const double* lin_new, double alpha, double* up) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int c = cell[p];
  if (c < 0 || c >= nc) return;
  double vo[3], vn[3];
  eval_linear(lin_old, xE, hE, c, x[p], x[np + p], x[2 * np + p], vo);
  eval_linear(lin_new, xE, hE, c, x[p], x[np + p], x[2 * np + p], vn);
  for (int k = 0; k < 3; ++k) {
    const double u = up[int64_t(k) * np + p];
    up[int64_t(k) * np + p] = alpha * (u + (vn[k] - vo[k])) + (1.0 - alpha) * vn[k];
  }
}

// ------------------------------------------------------------------ advection

// Parameter t in (0, 1] where segment a -> b meets triangle T, else -1
// (Moller-Trumbore; parallel segments never meet).
__device__ double seg_tri(const double a[3], const double b[3], const double* T) {
  const double d[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
  const double e1[3] = {T[3] - T[0], T[4] - T[1], T[5] - T[2]};
  const double e2[3] = {T[6] - T[0], T[7] - T[1], T[8] - T[2]};
  const double pv[3] = {d[1] * e2[2] - d[2] * e2[1], d[2] * e2[0] - d[0] * e2[2], d[0] * e2[1] - d[1] * e2[0]};
  const double det = e1[0] * pv[0] + e1[1] * pv[1] + e1[2] * pv[2];
  if (det == 0.0) return -1.0;
  const double inv = 1.0 / det;
  const double tv[3] = {a[0] - T[0], a[1] - T[1], a[2] - T[2]};
  const double u = (tv[0] * pv[0] + tv[1] * pv[1] + tv[2] * pv[2]) * inv;
  if (u < 0.0 || u > 1.0) return -1.0;
  const double qv[3] = {tv[1] * e1[2] - tv[2] * e1[1], tv[2] * e1[0] - tv[0] * e1[2], tv[0] * e1[1] - tv[1] * e1[0]};
  const double v = (d[0] * qv[0] + d[1] * qv[1] + d[2] * qv[2]) * inv;
  if (v < 0.0 || u + v > 1.0) return -1.0;
  const double t = (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]) * inv;
  return (t > 0.0 && t <= 1.0) ? t : -1.0;
}

constexpr int kMaxStepCubes = 4;  // cubes per axis one stage's segment may span

// End of one stage from (a, ca) to y: first obstacle crossing mirrors y
// across that triangle's plane, then the box walls mirror it, then it must
// lie in a fluid cell, else the stage stays at a.  Returns false when the
// segment spans more than kMaxStepCubes cubes along an axis (step too long).
__device__ bool stage_end(const PartGridView& g, const double a[3], int ca, double y[3], int& cy) {
  int lo[3], hi[3];
  for (int d = 0; d < 3; ++d) {
    const double mn = fmin(a[d], y[d]), mx = fmax(a[d], y[d]);
    if (!(isfinite(mn) && isfinite(mx))) return false;
    lo[d] = max(0, min(g.N - 1, int(floor(mn * g.N))));
    hi[d] = max(0, min(g.N - 1, int(floor(mx * g.N))));
    if (hi[d] - lo[d] >= kMaxStepCubes) return false;
  }
  double best = 2.0;
  int bi = -1;
  for (int k = lo[2]; k <= hi[2]; ++k)
    for (int j = lo[1]; j <= hi[1]; ++j)
      for (int i = lo[0]; i <= hi[0]; ++i) {
        const int q = (k * g.N + j) * g.N + i;
        for (int r = g.tbin_ptr[q]; r < g.tbin_ptr[q + 1]; ++r) {
          const int t = g.tbin_tri[r];
          const double s = seg_tri(a, y, g.tri + 9 * size_t(t));
          if (s > 0.0 && (s < best || (s == best && t < bi))) {
            best = s;
            bi = t;
          }
        }
      }
  if (bi >= 0) {
    const double* T = g.tri + 9 * size_t(bi);
    const double e1[3] = {T[3] - T[0], T[4] - T[1], T[5] - T[2]};
    const double e2[3] = {T[6] - T[0], T[7] - T[1], T[8] - T[2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const double L = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int d = 0; d < 3; ++d) n[d] /= L;
    const double s = 2.0 * ((y[0] - T[0]) * n[0] + (y[1] - T[1]) * n[1] + (y[2] - T[2]) * n[2]);
    for (int d = 0; d < 3; ++d) y[d] -= s * n[d];
  }
  for (int d = 0; d < 3; ++d) {
    if (y[d] < 0.0) y[d] = -y[d];
    if (y[d] > 1.0) y[d] = 2.0 - y[d];
  }
  cy = locate_point(g, y[0], y[1], y[2]);
  if (cy < 0) {
    for (int d = 0; d < 3; ++d) y[d] = a[d];
    cy = ca;
  }
  return true;
}

// One midpoint RK2 step per live particle (Sec. 3.3): x_m = x + dt/2 v(x),
// x_new = x + dt v(x_m), each stage's end handled by stage_end.  A particle
// whose step is too long keeps its position and sets *err = 1; particles
// with cell -1 (or no valid cell id) are left as they are.
__global__ void k_advect(int64_t np, double dt, const double* poly, const double* xE, const double* hE, int nc,
                         PartGridView g, double* x, int32_t* cell, int* err) {
  const int64_t p = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (p >= np) return;
  const int c0 = cell[p];
  if (c0 < 0 || c0 >= nc) return;
  const double a[3] = {x[p], x[np + p], x[2 * np + p]};
  double v[3];
  eval_linear(poly, xE, hE, c0, a[0], a[1], a[2], v);
  double m[3] = {a[0] + 0.5 * dt * v[0], a[1] + 0.5 * dt * v[1], a[2] + 0.5 * dt * v[2]};
  int cm;
  if (!stage_end(g, a, c0, m, cm)) {
    atomicExch(err, 1);
    return;
  }
  eval_linear(poly, xE, hE, cm, m[0], m[1], m[2], v);
  double y[3] = {a[0] + dt * v[0], a[1] + dt * v[1], a[2] + dt * v[2]};
  int cy;
  if (!stage_end(g, a, c0, y, cy)) {
    atomicExch(err, 1);
    return;
  }
  x[p] = y[0];
  x[np + p] = y[1];
  x[2 * np + p] = y[2];
  cell[p] = cy;
}

}  // namespace fvem
