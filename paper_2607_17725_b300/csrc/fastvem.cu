// C ABI of the cut-cell VEM pressure projection (include/fastvem.h).
//
// Host: topology (topo.cpp) and integer plan (plan.cpp).  Device: every
// numeric step of the precompute (A2-A6) and of the projection (A7-A13), plus
// the adjoint, in the kernels of kernels.cuh.  No CPU fallback exists: without
// a CUDA device only the host-side topology calls succeed.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <new>
#include <stdexcept>
#include <string>
#include <type_traits>
#include <unordered_map>
#include <vector>

#include "../../include/fastvem.h"
#include "kernels.cuh"
#include "kernels_k2.cuh"
#include "particles.cuh"
#include "plan.h"
#include "topo.h"

using namespace fvem;

namespace {

struct CudaError : std::runtime_error {
  using std::runtime_error::runtime_error;
};

#define CK(call)                                                                                   \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess)                                                                         \
      throw CudaError(std::string(#call) + ": " + cudaGetErrorString(e_));                         \
  } while (0)

// Owning device buffer.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() {
    if (p) cudaFree(p);
  }
  void alloc(size_t b) {
    if (p) {
      cudaFree(p);
      p = nullptr;
    }
    bytes = b;
    if (b == 0) return;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
      p = nullptr;
      if (e == cudaErrorMemoryAllocation) throw std::bad_alloc();
      throw CudaError(std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
  }
  template <typename T>
  T* as() const {
    return static_cast<T*>(p);
  }
};

template <typename T>
void upload(DBuf& b, const std::vector<T>& v, cudaStream_t s) {
  b.alloc(v.size() * sizeof(T));
  if (!v.empty()) CK(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, s));
}

inline unsigned nblk(int64_t n, int t = 256) { return unsigned(std::max<int64_t>(1, (n + t - 1) / t)); }

struct DevLevel {
  int nv = 0, nc = 0, ndof = 0;
  int64_t nnz = 0, nnzp = 0;
  int max_nv = 0, max_nf = 0;
  DBuf V, cell_vptr, cell_v, cell_fptr, face_vptr, face_v, face_pid, face_sg;
  DBuf kptr, Kel, vol, xE, hE, Pis;
  DBuf dof_of_vertex, vertex_of_dof, inc_ptr, inc_cell, inc_loc;
  DBuf elem_vptr_x, elem_v_x;
  DBuf cw32;  // coarsest level: w = A r of the FP32 kernel-sequence CG
  DBuf mix_list;  // coarsest level: slice lists of the mixed-split product
  MixSched mix{};
  // stencil slices of the FP32 copy (see SellView): flags, class table,
  // per-row class, lattice line offsets and block schedule
  DBuf reg32, stc32, cls32, lines32, order32, stpos32;
  int64_t nsched32 = 0;
  int64_t nreg32 = 0;     // stencil slices
  int64_t ncls32 = 0;     // classes in the table
  int64_t stc_nnz32 = 0;  // stored nonzeros of the rows of stencil slices
  bool stc_on = true;     // the level's FP32 products use its stencil slices (tuned)
  int64_t nsched_st32 = 0;  // schedule entries of the stencil slices (padded to 8)
  // element lists where they differ from the cell lists
  const int32_t* elem_vptr() const {
    return elem_vptr_x.p ? elem_vptr_x.as<int32_t>() : cell_vptr.as<int32_t>();
  }
  const int32_t* elem_v() const { return elem_v_x.p ? elem_v_x.as<int32_t>() : cell_v.as<int32_t>(); }
  DBuf a_rowptr, a_col, a_val;
  int64_t nslices = 0;
  DBuf sell_ptr, sell_w, sell_col, sell_dcol, sell_val, sell_val32, sell_of_csr;
  DBuf sell_valb;        // packed 16-bit copy of the V-cycle values (contexts created in BF16 or FP16 mode)
  bool bf16_on = false;  // the FP32 products of this level read the 16-bit copy (BF16/FP16 mode, not the coarsest)
  bool v16_half = false;  // the 16-bit copy is FP16 (else BF16)
  bool d16 = false;
  // prolongation from level l+1 into this level
  DBuf ptype, pcell, pa, pb, prow_ptr, prow_col, prow_val;
  DBuf pf_rowptr, pf_col, pf_src, pf_val, pf_val32;
  DBuf pt_rowptr, pt_col, pt_src, pt_val, pt_val32;
  DBuf child_ptr, child_cell;
  // V-cycle work vectors, FP64 and (when FP32 is enabled) FP32
  DBuf b, x, r, d0, d1;
  DBuf b32, x32, r32, d032, d132;
  DBuf cw;  // coarsest level only: the extra CG vector w
  // second order: element-order tables, element data (Pi* 10 x n_E, K n_E^2,
  // cell moments, face projectors), prolongation placements, the level's
  // diagonal scaling s = D^-1/2 and (level 0) the scaled values the V-cycle
  // uses while the outer CG keeps the unscaled operator
  DBuf k2_edge_ptr, k2_edge_v, k2_fpos_v, k2_fpos_e, k2_eptr, k2_edof, k2_perm, k2_koff, k2_foff;
  DBuf Pis2, K2, mom2, face2, pk, pC, pa2, pb2, px;
  DBuf sv, vsell_val;
  int k2_nf_cap = 0, k2_kcap = 0, k2_ne_cap = 0;
  double lmax = 0.0;
  // sliced-ELL launch shape per precision (tuned at build): index into kSellCfg
  int cfg64 = 0, cfg32 = 0;
  template <typename T>
  int cfg() const {
    return std::is_same<T, double>::value ? cfg64 : cfg32;
  }

  MeshView mesh() const {
    return MeshView{V.as<double>(),     cell_vptr.as<int32_t>(), cell_v.as<int32_t>(),   cell_fptr.as<int32_t>(),
                    face_vptr.as<int32_t>(), face_v.as<int32_t>(), face_pid.as<int32_t>(), face_sg.as<int8_t>(),
                    nc};
  }
  template <typename T>
  SellView<T> sell() const;
  // the operator the V-cycle smooths with: the level's own, or on level 0 of
  // the second-order path its diagonally scaled copy
  template <typename T>
  SellView<T> vsell() const {
    SellView<T> A = sell<T>();
    if (std::is_same<T, double>::value && vsell_val.p) A.val = static_cast<const T*>(vsell_val.p);
    return A;
  }
};
template <>
SellView<double> DevLevel::sell<double>() const {
  return SellView<double>{sell_ptr.as<int64_t>(), sell_w.as<int32_t>(), sell_col.as<int32_t>(),
                          sell_dcol.as<int16_t>(), sell_val.as<double>(), int64_t(ndof), nslices,
                          nullptr, nullptr, nullptr, nullptr, nullptr, 0};
}
template <>
SellView<float> DevLevel::sell<float>() const {
  return SellView<float>{sell_ptr.as<int64_t>(), sell_w.as<int32_t>(), sell_col.as<int32_t>(),
                         sell_dcol.as<int16_t>(), sell_val32.as<float>(), int64_t(ndof), nslices,
                         stc_on ? reg32.as<uint8_t>() : nullptr, stc32.as<float>(), cls32.as<uint8_t>(),
                         lines32.as<int16_t>(), stc_on ? order32.as<int32_t>() : nullptr, stc_on ? nsched32 : 0,
                         (bf16_on && sell_valb.p && !v16_half) ? sell_valb.as<__nv_bfloat16>() : nullptr,
                         (bf16_on && sell_valb.p && v16_half) ? sell_valb.as<__half>() : nullptr,
                         stc_on ? nsched_st32 : 0};
}

// Launch shapes of the sliced-ELL kernels: (gathers in flight per thread U,
// warps per slice KS).  Grid = ceil(slices / (8 / KS)) blocks of 256.
template <int V>
using IC = std::integral_constant<int, V>;
constexpr int kSellCfgCount = 12;
template <bool D, typename F>
void with_cfg_d(int cfg, F&& f) {
  using B = std::integral_constant<bool, D>;
  switch (cfg) {
    case 0: f(IC<2>(), IC<1>(), B()); break;
    case 1: f(IC<4>(), IC<1>(), B()); break;
    case 2: f(IC<2>(), IC<2>(), B()); break;
    case 3: f(IC<4>(), IC<2>(), B()); break;
    case 4: f(IC<2>(), IC<4>(), B()); break;
    case 5: f(IC<4>(), IC<4>(), B()); break;
    case 6: f(IC<2>(), IC<8>(), B()); break;
    case 7: f(IC<4>(), IC<8>(), B()); break;
    case 8: f(IC<8>(), IC<1>(), B()); break;
    case 9: f(IC<8>(), IC<2>(), B()); break;
    case 10: f(IC<16>(), IC<1>(), B()); break;
    default: f(IC<16>(), IC<2>(), B()); break;
  }
}
// f(U, KS, D16): D16 = the level stores 16-bit column offsets
template <typename F>
void with_cfg(int cfg, bool d16, F&& f) {
  if (d16)
    with_cfg_d<true>(cfg, f);
  else
    with_cfg_d<false>(cfg, f);
}
inline unsigned sell_grid(int64_t ns, int KS) {
  int spb = 8 / KS;
  return unsigned(std::max<int64_t>(1, (ns + spb - 1) / spb));
}
// grid of a launch over A: the block schedule's length for the stencil
// variant (stc), else one slot per slice
template <typename T>
inline unsigned sell_grid(const SellView<T>& A, int KS, bool stc = false) {
  return sell_grid(stc && A.order ? A.nsched : A.ns, KS);
}
// f(U, KS, D16, STC): STC selects the stencil-slice variant, compiled for
// FP32 only (FP64 copies are never marked)
template <typename T, typename F>
void with_cfg_s(int cfg, bool d16, bool stc, F&& f) {
  using Y = std::integral_constant<bool, true>;
  using N = std::integral_constant<bool, false>;
  if constexpr (std::is_same<T, float>::value) {
    if (stc) {
      with_cfg(cfg, d16, [&](auto u, auto ks, auto dd) { f(u, ks, dd, Y()); });
      return;
    }
  }
  with_cfg(cfg, d16, [&](auto u, auto ks, auto dd) { f(u, ks, dd, N()); });
}

// f(U, KS, D16, STC, grid): a Chebyshev launch of shape cfg over A; with
// stencil slices and one warp per slice, the generic slices' blocks (8
// slices each) and the stencil blocks (8 kStencilPerWarp slices each)
template <typename T, typename F>
void with_launch(int cfg, const SellView<T>& A, F&& f) {
  with_cfg_s<T>(cfg, A.dcol != nullptr, A.reg != nullptr, [&](auto u, auto ks, auto dd, auto st) {
    constexpr int KS = decltype(ks)::value;
    constexpr bool S = decltype(st)::value;
    unsigned grid = sell_grid(A, KS, S);
    if (S && KS == 1 && A.order != nullptr && A.nsched_st > 0)
      grid = unsigned((A.nsched - A.nsched_st) / 8 + A.nsched_st / (8 * kStencilPerWarp));
    f(u, ks, dd, st, grid);
  });
}

}  // namespace

struct fvem_ctx {
  fvem_params prm{};
  cudaStream_t stream = nullptr;
  bool has_device = false;
  bool fp32_capable = false;  // FP32 level copies exist (context created in FP32 or BF16 mode)
  bool bf16_capable = false;  // packed 16-bit copies of the V-cycle values exist (created in BF16 or FP16 mode)
  bool v16_half = false;      // those copies are FP16 (created in FP16 mode), else BF16
  bool topo_ready = false, built = false;
  double topo_s = 0.0, device_s = 0.0;  // wall time of the last topology and device set-up
  std::string err;
  Topology topo;
  std::vector<LevelPlan> plan;
  std::vector<LevelK2> k2;  // second-order plan per level (order_k = 2)
  DBuf rc2;                 // second order: cell entries of the element right-hand sides
  std::vector<std::unique_ptr<DevLevel>> lv;
  DBuf d_err, scal, part, part_big, rzqz, coop_red, ccg_part, ccg_cs;
  bool coarse_seq = true;  // coarsest CG as a kernel sequence (else one cooperative launch); tuned
  int ccg_cfg = 0;         // launch shape of the coarsest-CG product kernel (tuned)
  int ccg_cfg32 = 0;       // the same for the FP32 coarsest CG of the FP32 V-cycle (tuned)
  float ccg32_ms = 0;      // build-time time of one FP32 coarsest solve (graph replay)
  bool coarse_coop32 = false;  // FP32 coarsest CG as one cooperative launch (else the sequence)
  int coarse_ks32 = 0;         // its launch shape (see coarse_fn)
  float coop32_ms = 0;         // its build-time time
  float coarse_seq_ms = 0.f, coarse_coop_ms = 0.f;
  int coop_blocks_f64 = 0, coop_blocks_f32 = 0;  // cooperative grid sizes of the coarsest CG
  int coarse_ks = 2;                              // launch shape of the coarsest CG (tuned, see coarse_fn)
  // persistent coarsest CG (k_ccg_persist): plan of the coarsest level, and
  // whether the tuner picked it per precision ([0] FP64, [1] FP32)
  struct Persist {
    bool ok = false;  // the coarsest level fits in the SMs' shared memory
    int nb = 0, rows_cap = 0, pairs_cap = 0, tasks_cap = 0, halo_cap = 0, kmax = 1;
    DBuf rb, p_off, t_off, tasks, perm_off, perm, map, val64, val32, lidx2, halo_ptr, halo_col, halo_own;
    DBuf count, part, w_g, abort_;
    bool use[2] = {false, false};
    float ms[2] = {0.f, 0.f};
    bool vsm[2] = {true, true};  // per precision: the values fit in shared memory
    size_t smem(int prec) const { return smem_with(prec, vsm[prec]); }
    size_t smem_with(int prec, bool vals) const {
      const size_t tb = prec == 0 ? 8 : 4;
      // value pairs (when kept in shared memory) and halo-position pairs,
      // tasks, halo rows and r, s, w, sorted order, own p and x, product
      // partials (aligned up to 8 bytes), per-row FP64 sums
      const size_t v = size_t(pairs_cap) * 32 * ((vals ? 2 * tb : 0) + 4) + size_t(tasks_cap) * 16 +
                       size_t(halo_cap) * (4 + 3 * tb) + size_t(rows_cap) * 2 +
                       size_t(2 + kmax) * size_t(rows_cap) * tb;
      return ((v + 7) & ~size_t(7)) + 2 * size_t(rows_cap) * 8;
    }
  } pst;
  DBuf cg_x, cg_r, cg_z, cg_p, cg_q, r32, z32, rloc, rloc3, pfull, u_tmp, gcell_tmp;
  double* h_sc = nullptr;  // pinned scalars
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr, ev3 = nullptr;
  cudaEvent_t evb = nullptr;  // joins the streams of a batch around its graph
  // optional timing of the dominant kernel (level-0 Chebyshev step)
  bool prof = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> prof_ev;
  size_t prof_used = 0;
  int64_t nlaunch = 0;  // kernels launched by this context
  // V-cycle of the CG loop as a CUDA graph (replayed once per iteration)
  bool use_graph = true;
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t vgraph = nullptr;
  int vgraph_prec = -1;
  bool vgraph_prof = false;
  bool capturing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> gprof_ev;
  size_t gprof_used = 0;
  bool gprof_pending = false;
  int64_t vgraph_launches = 0;  // kernels inside one replay
  double prof_ms = 0.0;
  int64_t prof_launches = 0;
  // whole PCG as one graph launch (device-side convergence test, conditional
  // while/if nodes); rebuilt when anything it captured changes (gen)
  uint64_t uid = 0, gen = 0;
  bool use_pcg_graph = true;
  cudaGraphExec_t pgraph = nullptr;
  uint64_t pgraph_gen = ~0ull;
  int64_t pg_init = 0, pg_step = 0, pg_dir = 0;  // kernels per section of the captured PCG
  // batch graph over a list of contexts, cached in the first context of the batch
  cudaGraphExec_t bgraph = nullptr;
  std::vector<std::pair<uint64_t, uint64_t>> bgraph_key;
  // particle transfers (Sec. 3.2-3.3): the obstacle triangles, the level-0
  // cells and triangles binned by background cube, face planes, and the
  // per-call particle bins (grown on demand)
  std::vector<double> tris;
  struct Particles {
    bool ready = false;
    DBuf cbin_ptr, cbin_cell, cbin_full, fplane, tri, tbin_ptr, tbin_tri, lin_old;
    DBuf count, tsum, bin, rank, idx, rpos, rval, err;
    int64_t np_cap = 0;
  } pt;
};

static fvem_status fail(fvem_ctx* c, fvem_status s, const std::string& m) {
  if (c) c->err = m;
  return s;
}

#define API_BEGIN try {
#define API_END(ctx)                                                        \
  }                                                                         \
  catch (const std::bad_alloc&) {                                           \
    return fail(ctx, FVEM_ENOMEM, "out of memory");                         \
  }                                                                         \
  catch (const CudaError& e) {                                              \
    return fail(ctx, FVEM_ECUDA, e.what());                                 \
  }                                                                         \
  catch (const std::exception& e) {                                         \
    return fail(ctx, FVEM_EINVAL, e.what());                                \
  }

// ------------------------------------------------------------------ V-cycle

namespace {

struct ChebCoef {
  double inv_theta;
  std::vector<double> c1, c2;  // per step k: d_{k+1} = c1[k] d_k + c2[k] r_{k+1}
};

ChebCoef cheb_coef(double lmax, int degree) {
  const double beta = lmax, alpha = lmax / 30.0;
  const double theta = 0.5 * (beta + alpha), delta = 0.5 * (beta - alpha), sigma = theta / delta;
  ChebCoef c;
  c.inv_theta = 1.0 / theta;
  double rho = 1.0 / sigma;
  for (int k = 0; k < degree; ++k) {
    double rn = 1.0 / (2.0 * sigma - rho);
    c.c1.push_back(rn * rho);
    c.c2.push_back(2.0 * rn / delta);
    rho = rn;
  }
  return c;
}

template <typename T>
T* vb(DBuf& b) {
  return b.as<T>();
}
// Level vectors of the V-cycle precision: which = 0 b, 1 x, 2 r, 3 d0, 4 d1.
template <typename T>
T* vec(DevLevel& L, int which);
template <>
double* vec<double>(DevLevel& L, int w) {
  DBuf* v[5] = {&L.b, &L.x, &L.r, &L.d0, &L.d1};
  return v[w]->as<double>();
}
template <>
float* vec<float>(DevLevel& L, int w) {
  DBuf* v[5] = {&L.b32, &L.x32, &L.r32, &L.d032, &L.d132};
  return v[w]->as<float>();
}

void prof_flush(fvem_ctx* C) {
  if (!C->prof_used) return;
  CK(cudaStreamSynchronize(C->stream));
  for (size_t i = 0; i < C->prof_used; ++i) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, C->prof_ev[i].first, C->prof_ev[i].second));
    C->prof_ms += ms;
  }
  C->prof_launches += int64_t(C->prof_used);
  C->prof_used = 0;
}

// Level-0 Chebyshev step, bracketed by events when profiling is on.
template <typename T>
void launch_step(fvem_ctx* C, int level, int cfg, const SellView<T>& A, const T* din, T* x, T* r, T* dout, T c1,
                 T c2, int wd, int fold) {
  cudaStream_t s = C->stream;
  const bool p = C->prof && level == 0;
  auto& ev = C->capturing ? C->gprof_ev : C->prof_ev;
  size_t& used = C->capturing ? C->gprof_used : C->prof_used;
  if (p) {
    if (used == ev.size()) {
      cudaEvent_t a, b;
      CK(cudaEventCreate(&a));
      CK(cudaEventCreate(&b));
      ev.push_back({a, b});
    }
    CK(cudaEventRecordWithFlags(ev[used].first, s, C->capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
  }
  with_launch<T>(cfg, A, [&](auto u, auto ks, auto dd, auto st, unsigned grid) {
    constexpr int U = decltype(u)::value, KS = decltype(ks)::value;
    constexpr bool D = decltype(dd)::value, S = decltype(st)::value;
    ++C->nlaunch, k_cheb_step<T, U, KS, D, S><<<grid, 256, 0, s>>>(A, din, x, r, dout, c1, c2, wd, fold);
  });
  if (p) {
    CK(cudaEventRecordWithFlags(ev[used].second, s, C->capturing ? cudaEventRecordExternal : cudaEventRecordDefault));
    ++used;
    if (!C->capturing && used == 4096) prof_flush(C);
  }
}

// The five work vectors of one level: b, x, r and the two Chebyshev
// directions.  The context's own (vec) or a caller-provided set (the
// allocation-free V-cycle).
template <typename T>
struct LVecs {
  T *b, *x, *r, *d0, *d1;
};
template <typename T>
LVecs<T> lvecs(DevLevel& L) {
  return LVecs<T>{vec<T>(L, 0), vec<T>(L, 1), vec<T>(L, 2), vec<T>(L, 3), vec<T>(L, 4)};
}

// x = p(A) b from x0 = 0 (degree d); with want_r also r = b - A x.
template <typename T>
void cheb_zero(fvem_ctx* C, int level, DevLevel& L, const LVecs<T>& v, const T* b, int degree, bool want_r) {
  cudaStream_t s = C->stream;
  ChebCoef cf = cheb_coef(L.lmax, degree);
  auto A = L.vsell<T>();
  T* x = v.x;
  T* r = v.r;
  T* d[2] = {v.d0, v.d1};
  // k = 0
  int steps_with_spmv = want_r ? degree : degree - 1;  // SpMVs after the first kernel's one
  bool need_d0 = degree > 1;
  with_launch<T>(L.cfg<T>(), A, [&](auto u, auto ks, auto dd, auto st, unsigned grid) {
    constexpr int U = decltype(u)::value, KS = decltype(ks)::value;
    constexpr bool D = decltype(dd)::value, S = decltype(st)::value;
    ++C->nlaunch, k_cheb_first<T, U, KS, D, S><<<grid, 256, 0, s>>>(A, b, x, r, d[0], T(cf.inv_theta),
                                                                         T(cf.c1[0]), T(cf.c2[0]), need_d0 ? 1 : 0,
                                                                         (!want_r && degree == 2) ? 1 : 0);
  });
  int cur = 0;
  for (int k = 1; k < steps_with_spmv; ++k) {
    bool wd = want_r ? (k < degree - 1) : true;
    bool fold = !want_r && (k == degree - 2);
    launch_step<T>(C, level, L.cfg<T>(), A, d[cur], x, r, d[1 - cur], T(cf.c1[k]), T(cf.c2[k]), wd ? 1 : 0,
                   fold ? 1 : 0);
    cur = 1 - cur;
  }
}

// x = x + p(A)(b - A x) (degree d), x given.
template <typename T>
void cheb_from(fvem_ctx* C, int level, DevLevel& L, const LVecs<T>& v, const T* b, int degree) {
  cudaStream_t s = C->stream;
  ChebCoef cf = cheb_coef(L.lmax, degree);
  auto A = L.vsell<T>();
  T* x = v.x;
  T* r = v.r;
  T* d[2] = {v.d0, v.d1};
  with_launch<T>(L.cfg<T>(), A, [&](auto u, auto ks, auto dd, auto st, unsigned grid) {
    constexpr int U = decltype(u)::value, KS = decltype(ks)::value;
    constexpr bool D = decltype(dd)::value, S = decltype(st)::value;
    ++C->nlaunch, k_cheb_resid<T, U, KS, D, S><<<grid, 256, 0, s>>>(A, b, x, r, d[0], T(cf.inv_theta));
  });
  if (degree == 1) ++C->nlaunch, k_axpy<T><<<nblk(L.ndof), 256, 0, s>>>(L.ndof, x, d[0]);
  int cur = 0;
  for (int k = 0; k + 1 < degree; ++k) {
    bool fold = (k == degree - 2);
    launch_step<T>(C, level, L.cfg<T>(), A, d[cur], x, r, d[1 - cur], T(cf.c1[k]), T(cf.c2[k]), 1, fold ? 1 : 0);
    cur = 1 - cur;
  }
}

// Coarsest-level CG (cooperative launch; grid sized to stay co-resident).
// Coarsest-CG variants: 16-bit offsets x warps per slice (2, 4, 8) x gathers
// in flight (4, 8); cfg = 2 * ks_index + u_index.
constexpr int kCoarseCfgCount = 6;
template <typename T, bool D>
const void* coarse_fn_d(int cfg) {
  switch (cfg) {
    case 0: return (const void*)k_coarse_cg<T, D, 2, 4>;
    case 1: return (const void*)k_coarse_cg<T, D, 2, 8>;
    case 2: return (const void*)k_coarse_cg<T, D, 4, 4>;
    case 3: return (const void*)k_coarse_cg<T, D, 4, 8>;
    case 4: return (const void*)k_coarse_cg<T, D, 8, 4>;
    default: return (const void*)k_coarse_cg<T, D, 8, 8>;
  }
}
template <typename T>
const void* coarse_fn(bool d16, int cfg) {
  return d16 ? coarse_fn_d<T, true>(cfg) : coarse_fn_d<T, false>(cfg);
}
inline int coarse_ks(int cfg) { return cfg < 2 ? 2 : (cfg < 4 ? 4 : 8); }

// Coarsest CG as a kernel sequence (FP64 or FP32 vectors and matrix; FP64
// inner products and scalars): init, first product, then per
// iteration an update and (but for the last) a product.
// Mixed-split product shapes of the coarsest CG (launch shapes kSellCfgCount +
// i): gathers in flight U and the bound on slots per warp that sets each
// slice's warp count (KS = 1, 2, 4, 8: the fewest with ceil(width / KS) <=
// bound, else 8).
constexpr int kMixCount = 6;
constexpr int kMixU[kMixCount] = {4, 4, 4, 8, 8, 8};
constexpr int kMixBound[kMixCount] = {8, 12, 16, 16, 24, 32};

void build_mix(fvem_ctx* C, DevLevel& L, const LevelPlan& P, int bound) {
  std::vector<int32_t> lists[4];
  for (int64_t sl = 0; sl < P.nslices; ++sl) {
    const int w = P.sell_w[sl];
    int c = 3;
    for (int k = 0; k < 3; ++k)
      if ((w + (1 << k) - 1) >> k <= bound) {
        c = k;
        break;
      }
    lists[c].push_back(int32_t(sl));
  }
  std::vector<int32_t> all;
  L.mix.blk[0] = 0;
  for (int c = 0; c < 4; ++c) {
    const int spb = 8 >> c;  // slices per block with 2^c warps per slice
    while (lists[c].size() % spb) lists[c].push_back(-1);
    L.mix.off[c] = int64_t(all.size());
    L.mix.len[c] = int64_t(lists[c].size());
    L.mix.blk[c + 1] = L.mix.blk[c] + int(lists[c].size() / spb);
    all.insert(all.end(), lists[c].begin(), lists[c].end());
  }
  upload(L.mix_list, all, C->stream);
  L.mix.list = L.mix_list.as<int32_t>();
}

template <typename T>
void coarse_cg_seq(fvem_ctx* C, DevLevel& L, const T* b, T* x, T* r, T* p, T* s_, T* w, double* part, double* cs,
                   int cfg) {
  cudaStream_t s = C->stream;
  auto A = L.sell<T>();
  const int iters = C->prm.coarse_degree;
  const unsigned gu = nblk(L.ndof);
  ++C->nlaunch, k_ccg_init<T><<<gu, 256, 0, s>>>(L.ndof, b, x, r, p, s_, cs);
  auto prod = [&](int first) {
    if (cfg >= kSellCfgCount) {
      const unsigned grid = unsigned(std::max(1, L.mix.blk[4]));
      auto launch = [&](auto u, auto dd) {
        constexpr int U = decltype(u)::value;
        constexpr bool D = decltype(dd)::value;
        MixSched M = L.mix;
        M.stpos = L.stpos32.as<int32_t>();
        ++C->nlaunch, k_ccg_prod_mix<T, U, D><<<grid, 256, 0, s>>>(A, M, r, w, part, cs, first);
      };
      using Y = std::integral_constant<bool, true>;
      using N = std::integral_constant<bool, false>;
      const bool u8 = kMixU[cfg - kSellCfgCount] == 8;
      if (L.d16)
        u8 ? launch(IC<8>(), Y()) : launch(IC<4>(), Y());
      else
        u8 ? launch(IC<8>(), N()) : launch(IC<4>(), N());
      return;
    }
    with_cfg_s<T>(cfg, L.d16, A.reg != nullptr, [&](auto u, auto ks, auto dd, auto st) {
      constexpr int U = decltype(u)::value, KS = decltype(ks)::value;
      constexpr bool D = decltype(dd)::value, S = decltype(st)::value;
      ++C->nlaunch, k_ccg_prod<T, U, KS, D, S><<<sell_grid(A, KS, S), 256, 0, s>>>(A, r, w, part, cs, first);
    });
  };
  prod(1);
  for (int it = 0; it < iters; ++it) {
    ++C->nlaunch, k_ccg_upd<T><<<gu, 256, 0, s>>>(L.ndof, x, r, p, s_, w, cs);
    if (it < iters - 1) prod(0);
  }
}

// Persistent coarsest CG: one cooperative launch of one 1024-thread CTA per
// SM, the level's matrix and each CTA's halo of r in shared memory (see
// k_ccg_persist).
template <typename T>
const void* persist_fn() {
  return (const void*)k_ccg_persist<T>;
}

template <typename T>
void coarse_persist(fvem_ctx* C, DevLevel& L, const T* b, T* x) {
  auto& ps = C->pst;
  const int prec = std::is_same<T, double>::value ? 0 : 1;
  PersistPlan pp{ps.rb.as<int32_t>(),
                 ps.p_off.as<int64_t>(),
                 ps.t_off.as<int32_t>(),
                 ps.tasks.as<int4>(),
                 ps.perm_off.as<int32_t>(),
                 ps.perm.as<int16_t>(),
                 prec == 0 ? ps.val64.p : ps.val32.p,
                 ps.lidx2.as<uint32_t>(),
                 ps.halo_ptr.as<int32_t>(),
                 ps.halo_col.as<int32_t>(),
                 ps.halo_own.as<int32_t>(),
                 ps.count.as<unsigned long long>(),
                 ps.part.as<double>(),
                 ps.w_g.p,
                 ps.abort_.as<int>(),
                 C->scal.as<double>() + 7,
                 int64_t(L.ndof),
                 ps.rows_cap,
                 ps.pairs_cap,
                 ps.tasks_cap,
                 ps.halo_cap,
                 ps.kmax,
                 ps.vsm[prec] ? 1 : 0};
  int iters = C->prm.coarse_degree;
  void* args[] = {(void*)&pp, (void*)&b, (void*)&x, (void*)&iters};
  ++C->nlaunch;
  CK(cudaLaunchCooperativeKernel(persist_fn<T>(), dim3(ps.nb), dim3(1024), args, ps.smem(prec), C->stream));
}

// Plan of the persistent form on the coarsest level: one contiguous run of
// rows per SM, balanced by stored nonzeros; per run, its rows sorted by
// length (longest first, ties by row) in slices of 32 as wide as their first
// row, the halo (sorted distinct columns of the run, padded with its first
// entry to a multiple of 4) and each slot's halo position; values are
// gathered on the device from the assembled CSR.  The product of a run is
// split into warp tasks: each slice gets 1, 2, 4 or 8 parts (part p takes
// its slots p, p + k, ...), doubling the part count of the slice with the
// most slots per part while the CTA's 32 warps suffice, so that one round of
// tasks covers the run; tasks are ordered longest first, and each task's
// slots are stored in pairs (two slots per lane per pair row) in task order.
// The form is available when every run fits in one CTA's shared memory.
constexpr int kPersistWarps = 32;  // warps of the persistent CTA (1024 threads)
constexpr int kPersistMaxParts = 8;

void build_persist(fvem_ctx* C, DevLevel& L, const LevelPlan& P) {
  auto& ps = C->pst;
  ps.ok = false;
  int dev = 0, nsm = 0, optin = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const int64_t n = P.ndof;
  if (n < 1) return;
  const int nb = int(std::min<int64_t>(nsm, n));
  const int64_t nnz = P.a_rowptr[n];
  std::vector<int32_t> rb(static_cast<size_t>(nb) + 1, 0);
  for (int k = 1; k < nb; ++k) {
    const int64_t target = nnz * k / nb;
    int64_t r = std::lower_bound(P.a_rowptr.begin(), P.a_rowptr.begin() + n, target) - P.a_rowptr.begin();
    r = std::max<int64_t>(r, rb[k - 1] + 1);
    r = std::min<int64_t>(r, n - (nb - k));
    rb[k] = int32_t(r);
  }
  rb[nb] = int32_t(n);
  std::vector<int64_t> p_off(1, 0), map;
  std::vector<int32_t> t_off(1, 0), task4, perm_off(1, 0), hptr(1, 0), hcol, hown;
  std::vector<int16_t> perm;
  std::vector<uint32_t> lidx2;
  int rows_cap = 0, halo_cap = 0, tasks_cap = 0, kmax = 1;
  int64_t pairs_cap = 0;
  for (int k = 0; k < nb; ++k) {
    const int64_t r0 = rb[k], r1 = rb[k + 1], rows = r1 - r0;
    if (rows > 32000) return;  // the sorted order is stored in 16 bits
    std::vector<int32_t> ord(static_cast<size_t>(rows));
    for (int64_t i = 0; i < rows; ++i) ord[size_t(i)] = int32_t(i);
    auto len = [&](int64_t local) { return P.a_rowptr[r0 + local + 1] - P.a_rowptr[r0 + local]; };
    std::stable_sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) { return len(a) > len(b); });
    std::vector<int32_t> h(P.a_col.begin() + P.a_rowptr[r0], P.a_col.begin() + P.a_rowptr[r1]);
    std::sort(h.begin(), h.end());
    h.erase(std::unique(h.begin(), h.end()), h.end());
    if (h.size() > 16000) return;  // halo positions (with bank padding) are stored in 16 bits
    const int32_t own = int32_t(std::lower_bound(h.begin(), h.end(), int32_t(r0)) - h.begin());
    hown.push_back(own);
    const int64_t nsl = (rows + 31) / 32;
    auto hidx = [&](int64_t src) {
      return int32_t(std::lower_bound(h.begin(), h.end(), P.a_col[size_t(src)]) - h.begin());
    };
    // Bank-aware halo order.  The 32 lanes of one slot of a slice gather
    // distinct halo entries; entries in the same shared-memory bank (position
    // mod 32) serialise.  The run's own rows keep their contiguous block;
    // every other entry, most-gathered first, takes the bank least used by
    // the entries it is gathered with (ties: the least-filled bank, then the
    // lowest), and the k-th entry of bank b sits at the k-th free position
    // congruent to b.  hpos maps the sorted halo index to its position.
    std::vector<int32_t> hpos(h.size(), -1);
    {
      std::vector<std::vector<int32_t>> groups;  // distinct entries per (slice, slot)
      for (int64_t sl = 0; sl < nsl; ++sl) {
        const int wmax = int(len(ord[size_t(sl * 32)]));
        for (int j = 0; j < wmax; ++j) {
          std::vector<int32_t> g;
          for (int lane = 0; lane < 32; ++lane) {
            const int64_t pos = sl * 32 + lane;
            if (pos < rows && j < len(ord[size_t(pos)])) g.push_back(hidx(P.a_rowptr[r0 + ord[size_t(pos)]] + j));
          }
          std::sort(g.begin(), g.end());
          g.erase(std::unique(g.begin(), g.end()), g.end());
          groups.push_back(std::move(g));
        }
      }
      std::vector<std::vector<int32_t>> occ(h.size());
      for (size_t gi = 0; gi < groups.size(); ++gi)
        for (int32_t e : groups[gi]) occ[size_t(e)].push_back(int32_t(gi));
      std::vector<int> bank(h.size(), -1), fill(32, 0);
      for (int64_t i = 0; i < rows; ++i) {
        bank[size_t(own + i)] = int((own + i) % 32);
        hpos[size_t(own + i)] = int32_t(own + i);
        ++fill[size_t((own + i) % 32)];
      }
      std::vector<int32_t> rest;
      for (size_t e = 0; e < h.size(); ++e)
        if (bank[e] < 0) rest.push_back(int32_t(e));
      std::stable_sort(rest.begin(), rest.end(),
                       [&](int32_t a, int32_t b) { return occ[size_t(a)].size() > occ[size_t(b)].size(); });
      std::vector<int32_t> next(32);
      for (int b = 0; b < 32; ++b) next[size_t(b)] = b;
      for (int32_t e : rest) {
        int64_t score[32] = {};
        for (int32_t gi : occ[size_t(e)])
          for (int32_t f : groups[size_t(gi)])
            if (bank[size_t(f)] >= 0) ++score[bank[size_t(f)]];
        int bsel = 0;
        for (int b = 1; b < 32; ++b)
          if (score[b] < score[bsel] || (score[b] == score[bsel] && fill[size_t(b)] < fill[size_t(bsel)])) bsel = b;
        bank[size_t(e)] = bsel;
        ++fill[size_t(bsel)];
        int32_t p = next[size_t(bsel)];
        while (p >= own && p < own + rows) p += 32;  // the own block is taken
        hpos[size_t(e)] = p;
        next[size_t(bsel)] = p + 32;
      }
    }
    int32_t hsize = 0;
    for (int32_t p : hpos) hsize = std::max(hsize, p + 1);
    if (hsize > 32000) {  // a lopsided bank fill: keep the sorted order (16-bit positions)
      for (size_t e = 0; e < h.size(); ++e) hpos[e] = int32_t(e);
      hsize = int32_t(h.size());
    }
    std::vector<int> wsl(static_cast<size_t>(nsl)), ksl(static_cast<size_t>(nsl), 1);
    for (int64_t sl = 0; sl < nsl; ++sl) wsl[size_t(sl)] = int(len(ord[size_t(sl * 32)]));
    // parts per slice: double the slice with the most slots per part (ties:
    // the first) while the doubled count still fits the CTA's warps
    int64_t used = nsl;
    for (;;) {
      int64_t best = -1, bw = 1;
      for (int64_t sl = 0; sl < nsl; ++sl) {
        const int kk = ksl[size_t(sl)];
        const int64_t per = (wsl[size_t(sl)] + kk - 1) / kk;
        if (kk < kPersistMaxParts && used + kk <= kPersistWarps && per > bw) {
          bw = per;
          best = sl;
        }
      }
      if (best < 0) break;
      used += ksl[size_t(best)];
      ksl[size_t(best)] *= 2;
    }
    struct Task {
      int64_t sl;
      int part, cnt;
    };
    std::vector<Task> tk;
    for (int64_t sl = 0; sl < nsl; ++sl)
      for (int p = 0; p < ksl[size_t(sl)]; ++p) {
        const int kk = ksl[size_t(sl)];
        tk.push_back({sl, p, std::max(0, (wsl[size_t(sl)] - p + kk - 1) / kk)});
        kmax = std::max(kmax, kk);
      }
    std::stable_sort(tk.begin(), tk.end(), [](const Task& a, const Task& b) { return a.cnt > b.cnt; });
    int64_t pr = 0;  // pair rows of this run so far
    for (const Task& t : tk) {
      const int kk = ksl[size_t(t.sl)];
      const int npair = (t.cnt + 1) / 2;
      task4.insert(task4.end(), {int32_t(pr), int32_t(npair), int32_t(t.sl), int32_t(t.part)});
      for (int r = 0; r < npair; ++r)
        for (int lane = 0; lane < 32; ++lane) {
          uint32_t l2 = 0;
          for (int e = 0; e < 2; ++e) {
            const int64_t j = t.part + int64_t(2 * r + e) * kk;  // slot of the row
            const int64_t pos = t.sl * 32 + lane;
            int64_t src = -1;
            uint32_t li = 0;
            if (pos < rows && j < len(ord[size_t(pos)])) {
              src = P.a_rowptr[r0 + ord[size_t(pos)]] + j;
              li = uint32_t(hpos[size_t(hidx(src))]);
            }
            map.push_back(src);
            l2 |= li << (16 * e);
          }
          lidx2.push_back(l2);
        }
      pr += npair;
    }
    t_off.push_back(int32_t(task4.size() / 4));
    tasks_cap = std::max(tasks_cap, int(tk.size()));
    p_off.push_back(p_off.back() + pr);
    pairs_cap = std::max(pairs_cap, pr);
    rows_cap = std::max(rows_cap, int(nsl * 32));
    for (int64_t i = 0; i < rows; ++i) perm.push_back(int16_t(ord[size_t(i)]));
    while (perm.size() % 8) perm.push_back(0);
    perm_off.push_back(int32_t(perm.size()));
    // halo rows by position; the gaps of the bank layout and the padding to
    // a multiple of 4 repeat the first halo row (their values are never used)
    std::vector<int32_t> hp(size_t((hsize + 3) / 4 * 4), h.front());
    for (size_t e = 0; e < h.size(); ++e) hp[size_t(hpos[e])] = h[e];
    halo_cap = std::max(halo_cap, int(hp.size()));
    hcol.insert(hcol.end(), hp.begin(), hp.end());
    hptr.push_back(int32_t(hcol.size()));
  }
  ps.nb = nb;
  ps.rows_cap = rows_cap;
  ps.pairs_cap = int(pairs_cap);
  ps.tasks_cap = tasks_cap;
  ps.halo_cap = halo_cap;
  ps.kmax = kmax;
  const size_t static_smem = 1024;
  // FVEM_PERSIST_GLOBAL_VALUES=1 keeps the values in global memory even where
  // they fit (so that small cases exercise that path too)
  const char* gv = std::getenv("FVEM_PERSIST_GLOBAL_VALUES");
  const bool force_global = gv && gv[0] == '1';
  for (int prec = 0; prec < 2; ++prec)
    ps.vsm[prec] = !force_global && ps.smem_with(prec, true) + static_smem <= size_t(optin);
  if (ps.smem_with(1, false) + static_smem > size_t(optin)) return;
  cudaStream_t s = C->stream;
  upload(ps.rb, rb, s);
  upload(ps.p_off, p_off, s);
  upload(ps.t_off, t_off, s);
  upload(ps.tasks, task4, s);
  upload(ps.perm_off, perm_off, s);
  upload(ps.perm, perm, s);
  upload(ps.map, map, s);
  upload(ps.lidx2, lidx2, s);
  upload(ps.halo_ptr, hptr, s);
  upload(ps.halo_col, hcol, s);
  upload(ps.halo_own, hown, s);
  const int64_t nslot = int64_t(map.size());
  ps.val64.alloc(sizeof(double) * size_t(nslot));
  ++C->nlaunch, k_gather_pad<double><<<RED_BLOCKS, 256, 0, s>>>(nslot, ps.map.as<int64_t>(), L.a_val.as<double>(),
                                                                ps.val64.as<double>());
  if (C->fp32_capable) {
    ps.val32.alloc(sizeof(float) * size_t(nslot));
    ++C->nlaunch, k_gather_pad<float><<<RED_BLOCKS, 256, 0, s>>>(nslot, ps.map.as<int64_t>(), L.a_val.as<double>(),
                                                                  ps.val32.as<float>());
  }
  CK(cudaGetLastError());
  ps.w_g.alloc(sizeof(double) * 2 * size_t(n));
  ps.count.alloc(sizeof(unsigned long long));
  CK(cudaMemsetAsync(ps.count.p, 0, sizeof(unsigned long long), s));
  ps.part.alloc(sizeof(double) * 4 * size_t(nb));
  ps.abort_.alloc(sizeof(int));
  CK(cudaMemsetAsync(ps.abort_.p, 0, sizeof(int), s));
  // the launch may use any dynamic shared size up to the device limit
  for (const void* fn : {persist_fn<double>(), persist_fn<float>()})
    CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - int(static_smem)));
  CK(cudaStreamSynchronize(s));
  ps.ok = true;
}

// After a timeout in the persistent kernel: clear its barrier counter, abort
// word and the status scalar, so the next solve starts from a clean state.
void reset_persist(fvem_ctx* C) {
  auto& ps = C->pst;
  cudaStream_t s = C->stream;
  CK(cudaStreamSynchronize(s));
  if (ps.count.p) CK(cudaMemsetAsync(ps.count.p, 0, sizeof(unsigned long long), s));
  if (ps.abort_.p) CK(cudaMemsetAsync(ps.abort_.p, 0, sizeof(int), s));
  CK(cudaMemsetAsync(C->scal.as<double>() + 7, 0, sizeof(double), s));
  CK(cudaStreamSynchronize(s));
}

// Status word of the persistent kernel (read after a stream sync).
bool coarse_timed_out(fvem_ctx* C) {
  double v = 0.0;
  CK(cudaMemcpyAsync(&v, C->scal.as<double>() + 7, sizeof(double), cudaMemcpyDeviceToHost, C->stream));
  CK(cudaStreamSynchronize(C->stream));
  return v != 0.0;
}

template <typename T>
void coarse_cg(fvem_ctx* C, DevLevel& L, const T* b, T* x, T* r, T* p, T* q, double* red, T* w = nullptr) {
  if (C->pst.ok && C->pst.use[std::is_same<T, double>::value ? 0 : 1]) {
    coarse_persist<T>(C, L, b, x);
    return;
  }
  if (C->coarse_seq && std::is_same<T, double>::value) {
    coarse_cg_seq<double>(C, L, (const double*)b, (double*)x, (double*)r, (double*)p, (double*)q,
                          w ? (double*)w : L.cw.as<double>(), C->ccg_part.as<double>(), C->ccg_cs.as<double>(),
                          C->ccg_cfg);
    return;
  }
  const int cfg = std::is_same<T, double>::value ? C->coarse_ks : C->coarse_ks32;
  int nb = std::is_same<T, double>::value ? C->coop_blocks_f64 : C->coop_blocks_f32;
  nb = int(std::max<int64_t>(1, std::min<int64_t>(nb, int64_t(sell_grid(L.sell<T>(), coarse_ks(cfg))))));
  auto A = L.sell<T>();
  int iters = C->prm.coarse_degree;
  if (!w) w = L.cw.as<T>();
  void* args[] = {(void*)&A, (void*)&b, (void*)&x, (void*)&r, (void*)&p, (void*)&q, (void*)&w, (void*)&iters,
                  (void*)&red};
  ++C->nlaunch;
  CK(cudaLaunchCooperativeKernel(coarse_fn<T>(L.d16, cfg), dim3(nb), dim3(256), args, 0, C->stream));
}

// z = V-cycle(b) on level l (z ends in the level's x).  With `vs` the work
// vectors of every level come from the caller (FP64 only: the allocation-free
// entry point), as do the coarsest CG's vector w and reduction slots `red`;
// otherwise the context's own vectors are used.
template <typename T>
void vcycle(fvem_ctx* C, int l, const T* b, const LVecs<T>* vs = nullptr, double* red = nullptr, T* w = nullptr) {
  DevLevel& L = *C->lv[l];
  const LVecs<T> v = vs ? vs[l] : lvecs<T>(L);
  int Lv = int(C->lv.size());
  cudaStream_t s = C->stream;
  if (l == Lv - 1) {
    if (C->prm.coarse_solver == FVEM_COARSE_CG) {
      // FP64 V-cycle: FP64 coarsest CG; FP32 V-cycle: FP32 kernel sequence when
      // built (FP64 inner products), else the FP64 solve between conversions
      if (std::is_same<T, double>::value) {
        coarse_cg<double>(C, L, (const double*)b, (double*)v.x, (double*)v.r, (double*)v.d0, (double*)v.d1,
                          red ? red : C->coop_red.as<double>(), (double*)w);
      } else if (C->fp32_capable && L.cw32.p && (C->coarse_coop32 || (C->pst.ok && C->pst.use[1]))) {
        // FP32 V-cycle: the coarsest CG runs in FP32 too (FP64 inner products)
        coarse_cg<float>(C, L, (const float*)b, (float*)v.x, (float*)v.r, (float*)v.d0, (float*)v.d1,
                         C->coop_red.as<double>(), L.cw32.as<float>());
      } else if (C->fp32_capable && L.cw32.p) {
        coarse_cg_seq<float>(C, L, (const float*)b, (float*)v.x, (float*)v.r, (float*)v.d0, (float*)v.d1,
                             L.cw32.as<float>(), C->ccg_part.as<double>(), C->ccg_cs.as<double>(), C->ccg_cfg32);
      } else {
        ++C->nlaunch, k_convert<T, double><<<nblk(L.ndof), 256, 0, s>>>(L.ndof, b, vec<double>(L, 0));
        coarse_cg<double>(C, L, vec<double>(L, 0), vec<double>(L, 1), vec<double>(L, 2), vec<double>(L, 3),
                          vec<double>(L, 4), C->coop_red.as<double>());
        ++C->nlaunch, k_convert<double, T><<<nblk(L.ndof), 256, 0, s>>>(L.ndof, vec<double>(L, 1), v.x);
      }
    } else {
      cheb_zero<T>(C, l, L, v, b, C->prm.coarse_degree, false);
    }
    return;
  }
  DevLevel& Cn = *C->lv[l + 1];
  const LVecs<T> vc = vs ? vs[l + 1] : lvecs<T>(Cn);
  cheb_zero<T>(C, l, L, v, b, C->prm.cheb_degree, true);
  const T* ptv = std::is_same<T, double>::value ? (const T*)L.pt_val.p : (const T*)L.pt_val32.p;
  const T* pfv = std::is_same<T, double>::value ? (const T*)L.pf_val.p : (const T*)L.pf_val32.p;
  ++C->nlaunch, k_csr<T><<<nblk(Cn.ndof), 256, 0, s>>>(Cn.ndof, L.pt_rowptr.as<int64_t>(), L.pt_col.as<int32_t>(), ptv,
                                         v.r, vc.b, 0);
  vcycle<T>(C, l + 1, vc.b, vs, red, w);
  ++C->nlaunch, k_csr<T><<<nblk(L.ndof), 256, 0, s>>>(L.ndof, L.pf_rowptr.as<int64_t>(), L.pf_col.as<int32_t>(), pfv,
                                        vc.x, v.x, 1);
  cheb_from<T>(C, l, L, v, b, C->prm.cheb_degree);
}

// z = M^{-1} r on level 0 in the context precision (FP64 in/out).
void apply_precond(fvem_ctx* C, const double* r, double* z) {
  DevLevel& L0 = *C->lv[0];
  cudaStream_t s = C->stream;
  if (C->prm.order_k == 2) {
    // scaled V-cycle (reading K1): z = s0 .* V'(s0 .* r), s0 = D_0^-1/2
    const double* s0 = L0.sv.as<double>();
    if (C->prm.precision != FVEM_PREC_FP64) {
      ++C->nlaunch, k_scale_to<double, float><<<RED_BLOCKS, 256, 0, s>>>(L0.ndof, s0, r, C->r32.as<float>());
      vcycle<float>(C, 0, C->r32.as<float>());
      ++C->nlaunch, k_scale_to<float, double><<<RED_BLOCKS, 256, 0, s>>>(L0.ndof, s0, vec<float>(L0, 1), z);
    } else {
      ++C->nlaunch, k_scale_to<double, double><<<RED_BLOCKS, 256, 0, s>>>(L0.ndof, s0, r, z);
      vcycle<double>(C, 0, z);
      ++C->nlaunch, k_scale_to<double, double><<<RED_BLOCKS, 256, 0, s>>>(L0.ndof, s0, vec<double>(L0, 1), z);
    }
    return;
  }
  if (C->prm.precision != FVEM_PREC_FP64) {
    ++C->nlaunch, k_convert<double, float><<<RED_BLOCKS, 256, 0, s>>>(L0.ndof, r, C->r32.as<float>());
    vcycle<float>(C, 0, C->r32.as<float>());
    ++C->nlaunch, k_convert<float, double><<<RED_BLOCKS, 256, 0, s>>>(L0.ndof, vec<float>(L0, 1), z);
  } else {
    vcycle<double>(C, 0, r);
    CK(cudaMemcpyAsync(z, L0.x.p, sizeof(double) * L0.ndof, cudaMemcpyDeviceToDevice, s));
  }
}

void destroy_vgraph(fvem_ctx* C) {
  if (C->vgraph) cudaGraphExecDestroy(C->vgraph);
  C->vgraph = nullptr;
  C->vgraph_prec = -1;
  ++C->gen;  // graphs holding the old V-cycle (whole-PCG graphs) are stale too
}

// Accumulate the event pairs of the last graph replay (called after a sync).
void collect_graph_prof(fvem_ctx* C) {
  if (!C->gprof_pending) return;
  for (size_t i = 0; i < C->gprof_used; ++i) {
    float ms = 0;
    CK(cudaEventElapsedTime(&ms, C->gprof_ev[i].first, C->gprof_ev[i].second));
    C->prof_ms += ms;
  }
  C->prof_launches += int64_t(C->gprof_used);
  C->gprof_pending = false;
}

// V-cycle of the CG loop (input cg_r, output cg_z): replayed from a CUDA graph
// captured on first use (and again when precision or profiling changes).
void apply_precond_cg(fvem_ctx* C) {
  double* r = C->cg_r.as<double>();
  double* z = C->cg_z.as<double>();
  if (C->use_graph && (!C->vgraph || C->vgraph_prec != C->prm.precision || C->vgraph_prof != C->prof)) {
    destroy_vgraph(C);
    cudaStream_t user = C->stream;
    if (!C->cap_stream) CK(cudaStreamCreateWithFlags(&C->cap_stream, cudaStreamNonBlocking));
    C->stream = C->cap_stream;
    C->capturing = true;
    C->gprof_used = 0;
    int64_t n0 = C->nlaunch;
    cudaGraph_t g = nullptr;
    bool ok = cudaStreamBeginCapture(C->cap_stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (ok) {
      try {
        apply_precond(C, r, z);
      } catch (...) {
        ok = false;
      }
      if (cudaStreamEndCapture(C->cap_stream, &g) != cudaSuccess) ok = false;
    }
    C->capturing = false;
    C->stream = user;
    if (ok && cudaGraphInstantiate(&C->vgraph, g, 0) != cudaSuccess) ok = false;
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    const int64_t captured = C->nlaunch - n0;
    C->nlaunch = n0;
    if (!ok) {
      destroy_vgraph(C);
      C->use_graph = false;  // launch kernel by kernel from now on
    } else {
      C->vgraph_prec = C->prm.precision;
      C->vgraph_prof = C->prof;
      C->vgraph_launches = captured;
    }
  }
  if (C->use_graph && C->vgraph) {
    CK(cudaGraphLaunch(C->vgraph, C->stream));
    C->nlaunch += C->vgraph_launches;
    if (C->vgraph_prof) C->gprof_pending = true;
  } else {
    apply_precond(C, r, z);
  }
}

void read_scalars(fvem_ctx* C) {
  CK(cudaMemcpyAsync(C->h_sc, C->scal.p, 8 * sizeof(double), cudaMemcpyDeviceToHost, C->stream));
  CK(cudaStreamSynchronize(C->stream));
  collect_graph_prof(C);
}

void issue_read(fvem_ctx* C) {
  CK(cudaMemcpyAsync(C->h_sc, C->scal.p, 8 * sizeof(double), cudaMemcpyDeviceToHost, C->stream));
}
void wait_read(fvem_ctx* C) {
  CK(cudaStreamSynchronize(C->stream));
  collect_graph_prof(C);
}

// Multigrid-preconditioned CG on level 0 free DOFs (b in cg_r on entry,
// overwritten by the residual), split into issue / wait / check phases so that
// several independent scenes can run in lockstep with one host wait per
// iteration (fvem_project_batched); a single scene is a batch of one.
struct PcgRun {
  fvem_ctx* C = nullptr;
  double* x = nullptr;
  int iters = 0;
  double rr0 = 0.0, relres = 0.0, r0n = 0.0;
  fvem_status st = FVEM_OK;
  bool done = false;
};

// x = 0, rr0 = r.r, z = M r, p = z, rz = r.z (then read the scalars)
void pcg_issue_start(PcgRun& P) {
  fvem_ctx* C = P.C;
  DevLevel& L0 = *C->lv[0];
  cudaStream_t s = C->stream;
  const int64_t n = L0.ndof;
  double* r = C->cg_r.as<double>();
  double* z = C->cg_z.as<double>();
  double* p = C->cg_p.as<double>();
  double* sc = C->scal.as<double>();
  double* part = C->part.as<double>();
  CK(cudaMemsetAsync(P.x, 0, sizeof(double) * n, s));
  ++C->nlaunch, k_dot2<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, r, r, nullptr, part);
  ++C->nlaunch, k_finalize<<<1, 256, 0, s>>>(part, RED_BLOCKS, 1, sc + 6);
  apply_precond_cg(C);
  CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s));
  ++C->nlaunch, k_dot2<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, r, z, nullptr, part);
  ++C->nlaunch, k_finalize<<<1, 256, 0, s>>>(part, RED_BLOCKS, 1, sc + 0);
  issue_read(C);
}

// The persistent coarsest CG reports a timed-out wait in scalar 7.
bool check_timeout(PcgRun& P) {
  if (P.C->h_sc[7] == 0.0) return false;
  reset_persist(P.C);
  P.C->err = "a bounded wait of the persistent coarsest-level CG ran out";
  P.st = FVEM_ETIMEOUT;
  P.done = true;
  return true;
}

void pcg_check_start(PcgRun& P) {
  if (check_timeout(P)) return;
  P.rr0 = P.C->h_sc[6];
  P.r0n = std::sqrt(P.rr0);
  P.iters = 0;
  P.relres = 0.0;
  if (!std::isfinite(P.rr0)) {
    P.st = FVEM_ENAN;
    P.done = true;
  } else if (P.rr0 == 0.0) {
    // b = 0: x = 0 is exact (z, p are 0 as well)
    P.done = true;
  } else {
    P.relres = 1.0;
  }
}

// q = A p, alpha = rz / pq, x += alpha p, r -= alpha q, rr = r.r (then read)
void pcg_issue_step(PcgRun& P) {
  fvem_ctx* C = P.C;
  DevLevel& L0 = *C->lv[0];
  cudaStream_t s = C->stream;
  const int64_t n = L0.ndof;
  double* r = C->cg_r.as<double>();
  double* p = C->cg_p.as<double>();
  double* q = C->cg_q.as<double>();
  double* sc = C->scal.as<double>();
  double* part = C->part.as<double>();
  auto A = L0.sell<double>();
  with_cfg(L0.cfg64, L0.d16, [&](auto u, auto ks, auto dd) {
    constexpr int U = decltype(u)::value, KS = decltype(ks)::value;
    constexpr bool D = decltype(dd)::value;
    ++C->nlaunch, k_cg_spmv_alpha<U, KS, D><<<sell_grid(A, KS), 256, 0, s>>>(A, p, q, C->part_big.as<double>(), sc);
  });
  ++C->nlaunch, k_cg_update_fused<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, P.x, r, p, q, part, sc);
  issue_read(C);
}

void pcg_check_step(PcgRun& P) {
  fvem_ctx* C = P.C;
  ++P.iters;
  if (check_timeout(P)) return;
  const double rz = C->h_sc[0], pq = C->h_sc[1], rr = C->h_sc[2];
  if (!std::isfinite(rz) || !std::isfinite(pq) || !std::isfinite(rr)) {
    P.st = FVEM_ENAN;
    P.done = true;
    return;
  }
  if (pq <= 0.0 || rz <= 0.0) {
    C->err = "CG breakdown at iteration " + std::to_string(P.iters) + ": p.Ap = " + std::to_string(pq) +
             ", r.z = " + std::to_string(rz) + ", rel_res = " + std::to_string(std::sqrt(rr / P.rr0));
    P.st = FVEM_EBREAKDOWN;
    P.done = true;
    return;
  }
  P.relres = std::sqrt(rr / P.rr0);
  if (P.relres <= C->prm.rel_tol) {
    P.done = true;
  } else if (P.iters >= C->prm.max_iters) {
    P.st = FVEM_ENOCONV;
    P.done = true;
  }
}

// z = M r, rz_new = r.z, qz = q.z, beta = -qz/pq, p = z + beta p
void pcg_issue_direction(PcgRun& P) {
  fvem_ctx* C = P.C;
  DevLevel& L0 = *C->lv[0];
  cudaStream_t s = C->stream;
  const int64_t n = L0.ndof;
  double* r = C->cg_r.as<double>();
  double* z = C->cg_z.as<double>();
  double* p = C->cg_p.as<double>();
  double* q = C->cg_q.as<double>();
  double* sc = C->scal.as<double>();
  double* part = C->part.as<double>();
  apply_precond_cg(C);
  ++C->nlaunch, k_cg_dots_beta<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, r, z, q, part, sc);
  ++C->nlaunch, k_cg_dir<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, p, z, sc);
}

// Lockstep CG over independent scenes: one host wait per iteration for all.
void pcg_batch(std::vector<PcgRun>& runs) {
  for (auto& P : runs) pcg_issue_start(P);
  for (auto& P : runs) wait_read(P.C);
  for (auto& P : runs) pcg_check_start(P);
  for (auto& P : runs)
    if (!P.done) pcg_issue_step(P);
  while (true) {
    bool any = false;
    for (auto& P : runs)
      if (!P.done) {
        wait_read(P.C);
        pcg_check_step(P);
        any = true;
      }
    if (!any) break;
    for (auto& P : runs)
      if (!P.done) {
        pcg_issue_direction(P);
        pcg_issue_step(P);
      }
  }
}

bool pcg_graph(fvem_ctx* C, PcgRun& P);

fvem_status pcg(fvem_ctx* C, double* x, int& iters, double& relres, double& r0n) {
  std::vector<PcgRun> runs(1);
  runs[0].C = C;
  runs[0].x = x;
  if (x != C->cg_x.as<double>() || !pcg_graph(C, runs[0])) pcg_batch(runs);
  iters = runs[0].iters;
  relres = runs[0].relres;
  r0n = runs[0].r0n;
  return runs[0].st;
}

// ------------------------------------------------------------------ whole-PCG graph
// The multigrid-preconditioned CG of one context as one branch of a CUDA
// graph, with no host round trip: the start (x = 0, r.r, z = M r, p = z,
// r.z), a device-side start test, then a while node whose body is the step
// (q = A p, alpha, x, r, r.r) and the device-side test, with the next
// direction (z = M r, beta, p) inside an if node.  The branch has no
// dependencies, so the branches of several contexts in one graph run
// concurrently.  Captured with the context's kernels on three internal
// streams; false if the driver refuses any part (the caller then uses the
// host-driven loop).
struct CondNode {
  cudaGraphNode_t node = nullptr;
  cudaGraph_t body = nullptr;
};

bool add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type, CondNode& out) {
  cudaStreamCaptureStatus cst;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(s, &cst, nullptr, &cg, &deps, nullptr, &nd) != cudaSuccess ||
      cst != cudaStreamCaptureStatusActive)
    return false;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = type;
  np.conditional.size = 1;
  if (cudaGraphAddNode(&out.node, cg, deps, nullptr, nd, &np) != cudaSuccess) return false;
  out.body = np.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(s, &out.node, nullptr, 1, cudaStreamSetCaptureDependencies) ==
         cudaSuccess;
}

bool capture_pcg_branch(fvem_ctx* C, cudaGraph_t g, cudaStream_t s1, cudaStream_t s2, cudaStream_t s3) {
  cudaGraphConditionalHandle loop = 0, dir = 0;
  if (cudaGraphConditionalHandleCreate(&loop, g, 0, cudaGraphCondAssignDefault) != cudaSuccess) return false;
  const auto mode = cudaStreamCaptureModeThreadLocal;
  if (cudaStreamBeginCaptureToGraph(s1, g, nullptr, nullptr, 0, mode) != cudaSuccess) return false;
  cudaStream_t user = C->stream;
  const bool cap0 = C->capturing;
  C->capturing = true;
  const int64_t n0 = C->nlaunch;
  bool ok = true;
  bool open2 = false, open3 = false;
  DevLevel& L0 = *C->lv[0];
  const int64_t n = L0.ndof;
  double* x = C->cg_x.as<double>();
  double* r = C->cg_r.as<double>();
  double* z = C->cg_z.as<double>();
  double* p = C->cg_p.as<double>();
  double* q = C->cg_q.as<double>();
  double* sc = C->scal.as<double>();
  double* part = C->part.as<double>();
  try {
    C->stream = s1;
    CK(cudaMemsetAsync(x, 0, sizeof(double) * n, s1));
    ++C->nlaunch, k_dot2<<<RED_BLOCKS, RED_THREADS, 0, s1>>>(n, r, r, nullptr, part);
    ++C->nlaunch, k_finalize<<<1, 256, 0, s1>>>(part, RED_BLOCKS, 1, sc + 6);
    apply_precond(C, r, z);
    CK(cudaMemcpyAsync(p, z, sizeof(double) * n, cudaMemcpyDeviceToDevice, s1));
    ++C->nlaunch, k_dot2<<<RED_BLOCKS, RED_THREADS, 0, s1>>>(n, r, z, nullptr, part);
    ++C->nlaunch, k_finalize<<<1, 256, 0, s1>>>(part, RED_BLOCKS, 1, sc + 0);
    ++C->nlaunch, k_pcg_check_start<<<1, 32, 0, s1>>>(sc, loop);
    CK(cudaGetLastError());
    C->pg_init = C->nlaunch - n0;
    CondNode wn, in;
    if (!add_conditional(s1, loop, cudaGraphCondTypeWhile, wn)) throw std::runtime_error("while node");
    if (cudaGraphConditionalHandleCreate(&dir, wn.body, 0, cudaGraphCondAssignDefault) != cudaSuccess)
      throw std::runtime_error("if handle");
    if (cudaStreamBeginCaptureToGraph(s2, wn.body, nullptr, nullptr, 0, mode) != cudaSuccess)
      throw std::runtime_error("while body capture");
    open2 = true;
    C->stream = s2;
    const int64_t n1 = C->nlaunch;
    auto A = L0.sell<double>();
    with_cfg(L0.cfg64, L0.d16, [&](auto u, auto ks, auto dd) {
      constexpr int U = decltype(u)::value, KS = decltype(ks)::value;
      constexpr bool D = decltype(dd)::value;
      ++C->nlaunch, k_cg_spmv_alpha<U, KS, D><<<sell_grid(A, KS), 256, 0, s2>>>(A, p, q, C->part_big.as<double>(), sc);
    });
    ++C->nlaunch, k_cg_update_fused<<<RED_BLOCKS, RED_THREADS, 0, s2>>>(n, x, r, p, q, part, sc);
    ++C->nlaunch, k_pcg_check_step<<<1, 32, 0, s2>>>(sc, C->prm.rel_tol, C->prm.max_iters, loop, dir);
    CK(cudaGetLastError());
    C->pg_step = C->nlaunch - n1;
    if (!add_conditional(s2, dir, cudaGraphCondTypeIf, in)) throw std::runtime_error("if node");
    if (cudaStreamBeginCaptureToGraph(s3, in.body, nullptr, nullptr, 0, mode) != cudaSuccess)
      throw std::runtime_error("if body capture");
    open3 = true;
    C->stream = s3;
    const int64_t n2 = C->nlaunch;
    apply_precond(C, r, z);
    ++C->nlaunch, k_cg_dots_beta<<<RED_BLOCKS, RED_THREADS, 0, s3>>>(n, r, z, q, part, sc);
    ++C->nlaunch, k_cg_dir<<<RED_BLOCKS, RED_THREADS, 0, s3>>>(n, p, z, sc);
    CK(cudaGetLastError());
    C->pg_dir = C->nlaunch - n2;
  } catch (...) {
    ok = false;
  }
  cudaGraph_t tmp = nullptr;
  if (open3 && cudaStreamEndCapture(s3, &tmp) != cudaSuccess) ok = false;
  if (open2 && cudaStreamEndCapture(s2, &tmp) != cudaSuccess) ok = false;
  if (cudaStreamEndCapture(s1, &tmp) != cudaSuccess) ok = false;
  cudaGetLastError();
  C->stream = user;
  C->capturing = cap0;
  C->nlaunch = n0;
  return ok;
}

struct CapStreams {
  cudaStream_t s[3] = {nullptr, nullptr, nullptr};
  CapStreams() {
    for (auto& x : s) CK(cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking));
  }
  ~CapStreams() {
    for (auto& x : s)
      if (x) cudaStreamDestroy(x);
  }
};

// Instantiate one graph holding the PCG branches of the given contexts.
cudaGraphExec_t build_pcg_graph(const std::vector<fvem_ctx*>& cs) {
  cudaGraph_t g = nullptr;
  if (cudaGraphCreate(&g, 0) != cudaSuccess) return nullptr;
  CapStreams st;
  bool ok = true;
  for (fvem_ctx* C : cs)
    if (ok) ok = capture_pcg_branch(C, g, st.s[0], st.s[1], st.s[2]);
  cudaGraphExec_t ge = nullptr;
  if (ok && cudaGraphInstantiate(&ge, g, 0) != cudaSuccess) ge = nullptr;
  cudaGraphDestroy(g);
  cudaGetLastError();
  return ge;
}

// Read the device-side results of a finished whole-PCG branch (after a sync
// of the stream the graph ran on) into the host-side run record.
void finish_graph_run(fvem_ctx* C, PcgRun& P) {
  CK(cudaMemcpyAsync(C->h_sc, C->scal.p, 16 * sizeof(double), cudaMemcpyDeviceToHost, C->stream));
  CK(cudaStreamSynchronize(C->stream));
  const double* h = C->h_sc;
  P.iters = int(h[14]);
  P.relres = h[13];
  P.rr0 = h[6];
  P.r0n = std::sqrt(std::max(0.0, h[6]));
  const int st = int(h[15]);
  P.st = st == 0 ? FVEM_OK : static_cast<fvem_status>(st);
  P.done = true;
  if (P.st == FVEM_EBREAKDOWN)
    C->err = "CG breakdown at iteration " + std::to_string(P.iters) + ": p.Ap = " + std::to_string(h[1]) +
             ", r.z = " + std::to_string(h[0]) + ", rel_res = " + std::to_string(std::sqrt(h[2] / h[6]));
  if (P.st == FVEM_ETIMEOUT) {
    reset_persist(C);
    C->err = "a bounded wait of the persistent coarsest-level CG ran out";
  }
  C->nlaunch += C->pg_init + int64_t(P.iters) * C->pg_step + int64_t(std::max(0, P.iters - 1)) * C->pg_dir;
}

// Single-scene PCG through the cached whole-PCG graph; false if the graph
// could not be built (the caller falls back to the host-driven loop).
bool pcg_graph(fvem_ctx* C, PcgRun& P) {
  if (!C->use_graph || !C->use_pcg_graph || C->prof) return false;
  if (!C->pgraph || C->pgraph_gen != C->gen) {
    if (C->pgraph) cudaGraphExecDestroy(C->pgraph);
    C->pgraph = build_pcg_graph({C});
    C->pgraph_gen = C->gen;
    if (!C->pgraph) {
      C->use_pcg_graph = false;
      return false;
    }
  }
  CK(cudaGraphLaunch(C->pgraph, C->stream));
  finish_graph_run(C, P);
  return true;
}

// A15: the PCG of every scene of a batch as one branch of one graph, launched
// once on the first scene's stream after every scene's right-hand side; each
// scene's stream then waits for it.  The graph is cached in the first context
// and rebuilt when the list of contexts or any of their states changes.
bool pcg_batch_graph(std::vector<PcgRun>& runs) {
  fvem_ctx* C0 = runs[0].C;
  std::vector<std::pair<uint64_t, uint64_t>> key;
  for (auto& P : runs) {
    fvem_ctx* C = P.C;
    if (!C->use_graph || !C->use_pcg_graph || C->prof || P.x != C->cg_x.as<double>()) return false;
    key.push_back({C->uid, C->gen});
  }
  if (!C0->bgraph || C0->bgraph_key != key) {
    if (C0->bgraph) cudaGraphExecDestroy(C0->bgraph);
    C0->bgraph = nullptr;
    C0->bgraph_key.clear();
    std::vector<fvem_ctx*> cs;
    for (auto& P : runs) cs.push_back(P.C);
    // In a batch the coarsest solves of the scenes overlap; the persistent
    // form takes one CTA on every SM and would run them one at a time, so the
    // batch graph captures the other forms the build tuned.
    std::vector<std::array<bool, 2>> keep;
    for (fvem_ctx* C : cs) {
      keep.push_back({C->pst.use[0], C->pst.use[1]});
      if (cs.size() > 1) C->pst.use[0] = C->pst.use[1] = false;
    }
    C0->bgraph = build_pcg_graph(cs);
    for (size_t i = 0; i < cs.size(); ++i) {
      cs[i]->pst.use[0] = keep[i][0];
      cs[i]->pst.use[1] = keep[i][1];
    }
    if (!C0->bgraph) {
      for (auto& P : runs) P.C->use_pcg_graph = false;
      return false;
    }
    C0->bgraph_key = key;
  }
  for (auto& P : runs)
    if (P.C != C0) {
      CK(cudaEventRecord(P.C->evb, P.C->stream));
      CK(cudaStreamWaitEvent(C0->stream, P.C->evb, 0));
    }
  CK(cudaGraphLaunch(C0->bgraph, C0->stream));
  CK(cudaEventRecord(C0->evb, C0->stream));
  for (auto& P : runs)
    if (P.C != C0) CK(cudaStreamWaitEvent(P.C->stream, C0->evb, 0));
  for (auto& P : runs) finish_graph_run(P.C, P);
  return true;
}

// Largest eigenvalue of a symmetric tridiagonal matrix by Sturm-sequence bisection.
double tridiag_max_eig(const std::vector<double>& a, const std::vector<double>& b) {
  const int m = int(a.size());
  double lo = 1e300, hi = -1e300;
  for (int i = 0; i < m; ++i) {
    double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  auto count_below = [&](double x) {
    int cnt = 0;
    double d = 1.0;
    for (int i = 0; i < m; ++i) {
      double bb = i > 0 ? b[i - 1] * b[i - 1] : 0.0;
      d = (a[i] - x) - (i > 0 ? bb / d : 0.0);
      if (d == 0.0) d = -1e-300;
      if (d < 0) ++cnt;
    }
    return cnt;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(hi), 1e-300); ++it) {
    double mid = 0.5 * (lo + hi);
    if (count_below(mid) >= m) hi = mid; else lo = mid;
  }
  return hi;
}

// Chebyshev upper bound: 1.1 x the largest Ritz value of 40 Lanczos steps
// started from x_i = 1 + (i mod 7)/7 (no reorthogonalisation).
double lanczos_lmax(fvem_ctx* C, DevLevel& L) {
  cudaStream_t s = C->stream;
  const int64_t n = L.ndof;
  DBuf vb_, vp_, wb_;
  vb_.alloc(sizeof(double) * n);
  vp_.alloc(sizeof(double) * n);
  wb_.alloc(sizeof(double) * n);
  double *v = vb_.as<double>(), *vprev = vp_.as<double>(), *w = wb_.as<double>();
  double* part = C->part.as<double>();
  double* sc = C->scal.as<double>();
  ++C->nlaunch, k_power_init<<<RED_BLOCKS, 256, 0, s>>>(n, v);
  CK(cudaMemsetAsync(vprev, 0, sizeof(double) * n, s));
  auto dot = [&](const double* x, const double* y) {
    ++C->nlaunch, k_dot2<<<RED_BLOCKS, RED_THREADS, 0, s>>>(n, x, y, nullptr, part);
    ++C->nlaunch, k_finalize<<<1, 256, 0, s>>>(part, RED_BLOCKS, 1, sc + 6);
    read_scalars(C);
    return C->h_sc[6];
  };
  double nv0 = std::sqrt(dot(v, v));
  ++C->nlaunch, k_scale_copy<<<RED_BLOCKS, 256, 0, s>>>(n, v, 1.0 / nv0, v);
  std::vector<double> al, be;
  double beta = 0.0;
  auto A = L.vsell<double>();
  for (int j = 0; j < std::min<int64_t>(40, n); ++j) {
    if (L.d16)
      ++C->nlaunch, k_spmv<double, 4, 1, true><<<sell_grid(A, 1), 256, 0, s>>>(A, v, w);
    else
      ++C->nlaunch, k_spmv<double, 4, 1, false><<<sell_grid(A, 1), 256, 0, s>>>(A, v, w);
    double a = dot(v, w);
    al.push_back(a);
    ++C->nlaunch, k_lanczos_orth<<<RED_BLOCKS, 256, 0, s>>>(n, w, v, vprev, a, beta);
    beta = std::sqrt(dot(w, w));
    if (!(beta > 1e-14 * std::max(std::fabs(a), 1e-300))) break;
    be.push_back(beta);
    ++C->nlaunch, k_lanczos_shift<<<RED_BLOCKS, 256, 0, s>>>(n, w, v, vprev, 1.0 / beta);
  }
  be.resize(al.size() > 0 ? al.size() - 1 : 0);
  return 1.1 * tridiag_max_eig(al, be);
}

// Build-time tuner: time the fused Chebyshev step of a level with 2 and 4
// gathers in flight per row and keep the faster one (per precision).
// Build-time tuner: time the fused Chebyshev step of a level with each launch
// shape (gathers in flight per thread x warps per slice) and keep the fastest
// one, per precision.
template <typename T>
int tune_sell(fvem_ctx* C, DevLevel& L) {
  cudaStream_t s = C->stream;
  T* v[5] = {vec<T>(L, 0), vec<T>(L, 1), vec<T>(L, 2), vec<T>(L, 3), vec<T>(L, 4)};
  for (auto* p : v) CK(cudaMemsetAsync(p, 0, sizeof(T) * size_t(std::max(1, L.ndof)), s));
  float best = 1e30f;
  int bestc = kSellCfgCount - 1;
  bool best_stc = false;
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  // FP32 levels with stencil slices are timed with and without them
  const bool can_stc = std::is_same<T, float>::value && L.reg32.p != nullptr;
  for (int trial = 0; trial < (can_stc ? 2 * kSellCfgCount : kSellCfgCount); ++trial) {
    const int cfg = trial % kSellCfgCount;
    const bool stc = trial >= kSellCfgCount;
    if (std::is_same<T, float>::value) L.stc_on = stc;
    auto A = L.vsell<T>();
    for (int rep = 0; rep < 2; ++rep) {
      CK(cudaEventRecord(e0, s));
      for (int k = 0; k < 5; ++k)
        with_launch<T>(cfg, A, [&](auto u, auto ks, auto dd, auto st, unsigned grid) {
          constexpr int U = decltype(u)::value, KS = decltype(ks)::value;
          constexpr bool D = decltype(dd)::value, S = decltype(st)::value;
          ++C->nlaunch, k_cheb_step<T, U, KS, D, S><<<grid, 256, 0, s>>>(A, v[3], v[1], v[2], v[4], T(0.5), T(0.5), 1,
                                                                          0);
        });
      CK(cudaEventRecord(e1, s));
      CK(cudaEventSynchronize(e1));
      float ms = 0;
      CK(cudaEventElapsedTime(&ms, e0, e1));
      if (rep == 1 && ms < best) {
        best = ms;
        bestc = cfg;
        best_stc = stc;
      }
    }
  }
  if (std::is_same<T, float>::value) L.stc_on = best_stc;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return bestc;
}

// Tuning decisions can be pinned through a file named by FVEM_TUNE_FILE: if
// it exists (and matches the hierarchy's sizes) the decisions are read from
// it, else they are measured and written to it.  Used so that a profiling run
// (whose serialised timing would mislead the tuner) replays the decisions of a
// plain run.
struct TuneRecord {
  std::vector<int> cfg64, cfg32, stc32;
  int coarse_seq = 1, coarse_ks = 2, coop_nb = 0, ccg_cfg = 0, ccg_cfg32 = 0;
  float seq_ms = 0, coop_ms = 0, ccg32_ms = 0;
  int coop32 = 0, ks32 = 0, nb32 = 0;
  float coop32_ms = 0;
  int persist64 = 0, persist32 = 0, pks64 = 1, pks32 = 1;
  float pms64 = 0, pms32 = 0;
};

std::string tune_key(fvem_ctx* C) {
  std::string k = std::to_string(C->topo.N) + ":" + std::to_string(C->prm.precision);
  for (auto& L : C->lv) k += ":" + std::to_string(L->ndof) + "/" + std::to_string(L->nnz);
  return k;
}

bool tune_load(fvem_ctx* C, TuneRecord& t) {
  const char* fn = std::getenv("FVEM_TUNE_FILE");
  if (!fn) return false;
  FILE* f = std::fopen(fn, "r");
  if (!f) return false;
  char key[4096] = {0};
  bool ok = std::fscanf(f, "%4095s", key) == 1 && tune_key(C) == key;
  int Lv = int(C->lv.size());
  t.cfg64.assign(Lv, 0);
  t.cfg32.assign(Lv, 0);
  t.stc32.assign(Lv, 0);
  for (int l = 0; ok && l < Lv; ++l) ok = std::fscanf(f, "%d %d %d", &t.cfg64[l], &t.cfg32[l], &t.stc32[l]) == 3;
  if (ok)
    ok = std::fscanf(f, "%d %d %d %d %f %f %d %f %d %d %d %f %d %d %d %d %f %f", &t.coarse_seq, &t.coarse_ks,
                     &t.coop_nb, &t.ccg_cfg, &t.seq_ms, &t.coop_ms, &t.ccg_cfg32, &t.ccg32_ms, &t.coop32, &t.ks32,
                     &t.nb32, &t.coop32_ms, &t.persist64, &t.persist32, &t.pks64, &t.pks32, &t.pms64,
                     &t.pms32) == 18;
  std::fclose(f);
  return ok;
}

void tune_save(fvem_ctx* C, const TuneRecord& t) {
  const char* fn = std::getenv("FVEM_TUNE_FILE");
  if (!fn) return;
  FILE* f = std::fopen(fn, "w");
  if (!f) return;
  std::fprintf(f, "%s\n", tune_key(C).c_str());
  for (size_t l = 0; l < t.cfg64.size(); ++l) std::fprintf(f, "%d %d %d\n", t.cfg64[l], t.cfg32[l], t.stc32[l]);
  std::fprintf(f, "%d %d %d %d %f %f %d %f %d %d %d %f %d %d %d %d %f %f\n", t.coarse_seq, t.coarse_ks, t.coop_nb,
               t.ccg_cfg, t.seq_ms, t.coop_ms, t.ccg_cfg32, t.ccg32_ms, t.coop32, t.ks32, t.nb32, t.coop32_ms,
               t.persist64, t.persist32, t.pks64, t.pks32, t.pms64, t.pms32);
  std::fclose(f);
}

void check_err(fvem_ctx* C, const char* what) {
  int h = 0;
  CK(cudaMemcpyAsync(&h, C->d_err.p, sizeof(int), cudaMemcpyDeviceToHost, C->stream));
  CK(cudaStreamSynchronize(C->stream));
  if (h) throw std::runtime_error(std::string(what) + ": device consistency check failed (code " + std::to_string(h) + ")");
}

// Stencil slices (FP32 copies).  A row is a stencil row when every stored
// entry sits at a lattice position of the row's vertex: (dx, dy, dz) in
// {-1, 0, 1}^3 times the largest coordinate offset among its entries (exact
// to 1e-9), the centre being the row itself.  Its 27-slot virtual row holds
// the FP32 values (zero where an entry is missing: walls, removed Dirichlet
// neighbours), and its columns must form, per line (dy, dz), three
// consecutive indices around the line's centre (a missing line gets offset
// 0).  Rows with the same 27 FP32 values share a class (at most 255 per
// level); a slice whose 32 rows are all stencil rows is a stencil slice.  Its
// products use the class table and eight 16-bit line offsets per row, which
// gives the stored matrix's products up to summation order.
constexpr int kStencilWidth = 27;

void mark_stencils(fvem_ctx* C) {
  if (!C->fp32_capable || C->prm.order_k != 1) return;
  cudaStream_t s = C->stream;
  for (size_t l = 0; l < C->lv.size(); ++l) {
    DevLevel& L = *C->lv[l];
    const LevelPlan& P = C->plan[l];
    const LevelMesh& M = C->topo.levels[l];
    L.reg32.alloc(0);
    L.stc32.alloc(0);
    L.cls32.alloc(0);
    L.lines32.alloc(0);
    L.order32.alloc(0);
    L.stpos32.alloc(0);
    L.nsched32 = L.nreg32 = L.ncls32 = L.stc_nnz32 = L.nsched_st32 = 0;
    const int64_t n = P.ndof, nnz = P.a_rowptr[n];
    if (n < 32 || nnz == 0) continue;
    std::vector<double> val(static_cast<size_t>(nnz));
    CK(cudaMemcpyAsync(val.data(), L.a_val.p, sizeof(double) * size_t(nnz), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<int16_t> ln(size_t(L.nslices) * 256, 0);
    std::vector<uint8_t> cls(size_t(n), 0), rowok(size_t(n), 0);
    std::vector<float> table;
    std::unordered_map<std::string, int> ids;
    for (int64_t i = 0; i < n; ++i) {
      const int64_t rb = P.a_rowptr[i], re = P.a_rowptr[i + 1];
      if (re - rb > kStencilWidth) continue;
      const double* vi = &M.V[3 * size_t(P.vertex_of_dof[i])];
      double hr = 0.0;
      for (int64_t k = rb; k < re; ++k) {
        const double* vj = &M.V[3 * size_t(P.vertex_of_dof[P.a_col[k]])];
        for (int c = 0; c < 3; ++c) hr = std::max(hr, std::fabs(vj[c] - vi[c]));
      }
      if (!(hr > 0.0)) continue;
      float v27[kStencilWidth] = {};
      int64_t c27[kStencilWidth] = {};
      bool has[kStencilWidth] = {};
      bool ok = true;
      for (int64_t k = rb; k < re && ok; ++k) {
        const double* vj = &M.V[3 * size_t(P.vertex_of_dof[P.a_col[k]])];
        int d[3];
        for (int c = 0; c < 3 && ok; ++c) {
          const double q = (vj[c] - vi[c]) / hr;
          d[c] = int(std::lround(q));
          ok = std::fabs(q - d[c]) <= 1e-9 && d[c] >= -1 && d[c] <= 1;
        }
        if (!ok) break;
        const int slot = 9 * (d[2] + 1) + 3 * (d[1] + 1) + (d[0] + 1);
        ok = !has[slot];
        has[slot] = true;
        v27[slot] = float(val[size_t(k)]);
        c27[slot] = P.a_col[k];
      }
      if (!ok || !has[13] || c27[13] != i) continue;
      int16_t off[9] = {};
      for (int k = 0; k < 9 && ok; ++k) {
        const int mid = 3 * k + 1;
        if (!has[mid]) {
          ok = !has[mid - 1] && !has[mid + 1];  // a line is whole or absent
          continue;
        }
        const int64_t base = c27[mid], o = base - i;
        ok = (!has[mid - 1] || c27[mid - 1] == base - 1) && (!has[mid + 1] || c27[mid + 1] == base + 1) &&
             o >= -32767 && o <= 32767;
        off[k] = int16_t(o);
      }
      if (!ok) continue;
      const std::string key(reinterpret_cast<const char*>(v27), sizeof(v27));
      auto it = ids.find(key);
      int id;
      if (it == ids.end()) {
        if (ids.size() >= 255) continue;
        id = int(ids.size());
        ids.emplace(key, id);
        table.insert(table.end(), v27, v27 + kStencilWidth);
        table.push_back(0.0f);  // 28 floats per class (16-byte rows)
      } else {
        id = it->second;
      }
      cls[size_t(i)] = uint8_t(id);
      rowok[size_t(i)] = 1;
      const int64_t sl = i >> 5;
      const int lane = int(i & 31);
      for (int k = 0; k < 9; ++k)
        if (k != 4) ln[size_t(sl) * 256 + (k < 4 ? k : k - 1) * 32 + lane] = off[k];
    }
    std::vector<uint8_t> h(size_t(L.nslices), 0);
    int64_t nl = 0, snnz = 0;
    for (int64_t sl = 0; sl < L.nslices; ++sl) {
      if (sl * 32 + 31 >= n) continue;
      bool all = true;
      for (int q = 0; q < 32 && all; ++q) all = rowok[size_t(sl * 32 + q)] != 0;
      if (!all) continue;
      h[size_t(sl)] = 2;
      ++nl;
      snnz += P.a_rowptr[sl * 32 + 32] - P.a_rowptr[sl * 32];
    }
    if (nl == 0) continue;
    // block schedule: stencil slices (padded to a whole number of stencil
    // blocks, 8 warps of kStencilPerWarp slices), then the others (padded to 8)
    std::vector<int32_t> ord;
    for (int pass = 0; pass < 2; ++pass) {
      for (int64_t sl = 0; sl < L.nslices; ++sl)
        if ((h[size_t(sl)] == 2) == (pass == 0)) ord.push_back(int32_t(sl));
      while (ord.size() % (pass == 0 ? 8 * kStencilPerWarp : 8)) ord.push_back(-1);
    }
    // classes and line offsets of the stencil rows by schedule position
    // (padding entries zero)
    const int64_t nst = (nl + 8 * kStencilPerWarp - 1) / (8 * kStencilPerWarp) * (8 * kStencilPerWarp);
    std::vector<uint8_t> clsq(size_t(nst) * 32, 0);
    std::vector<int16_t> lnq(size_t(nst) * 32 * 8, 0);
    for (int64_t q = 0; q < nl; ++q) {
      const int64_t sl = ord[size_t(q)];
      for (int lane = 0; lane < 32; ++lane) {
        clsq[size_t(q * 32 + lane)] = cls[size_t(sl * 32 + lane)];
        for (int kk = 0; kk < 8; ++kk)
          lnq[size_t((q * 32 + lane) * 8 + kk)] = ln[size_t(sl) * 256 + kk * 32 + lane];
      }
    }
    upload(L.reg32, h, s);
    upload(L.stc32, table, s);
    upload(L.cls32, clsq, s);
    upload(L.lines32, lnq, s);
    upload(L.order32, ord, s);
    std::vector<int32_t> stpos(size_t(L.nslices), -1);
    for (int64_t q = 0; q < nl; ++q) stpos[size_t(ord[size_t(q)])] = int32_t(q);
    upload(L.stpos32, stpos, s);
    CK(cudaStreamSynchronize(s));
    L.nsched32 = int64_t(ord.size());
    L.nsched_st32 = nst;
    L.nreg32 = nl;
    L.ncls32 = int64_t(ids.size());
    L.stc_nnz32 = snnz;
  }
}

// In BF16 (FP16) mode every level but the coarsest reads its packed 16-bit
// values in the FP32 V-cycle (the coarsest CG keeps its FP32 copy).
void set_bf16_flags(fvem_ctx* C) {
  const int Lv = int(C->lv.size());
  const bool on = C->prm.precision == FVEM_PREC_BF16 || C->prm.precision == FVEM_PREC_FP16;
  for (int l = 0; l < Lv; ++l) {
    C->lv[l]->bf16_on = on && l + 1 < Lv && C->lv[l]->sell_valb.p != nullptr;
    C->lv[l]->v16_half = C->v16_half;
  }
}

// The packed 16-bit copy of a level's V-cycle values (BF16 or FP16, by the
// context's creation mode), scattered from CSR values into the sliced-ELL
// slots (padding stays 0).
void make_v16(fvem_ctx* C, DevLevel& L, const double* vals, cudaStream_t s) {
  L.sell_valb.alloc(2 * (L.sell_val.bytes / sizeof(double)));
  CK(cudaMemsetAsync(L.sell_valb.p, 0, L.sell_valb.bytes, s));
  if (C->v16_half)
    ++C->nlaunch, k_scatter_sell_fp16<<<nblk(L.nnz), 256, 0, s>>>(L.nnz, L.sell_of_csr.as<int64_t>(), vals,
                                                                  L.sell_valb.as<__half>());
  else
    ++C->nlaunch, k_scatter_sell_bf16<<<nblk(L.nnz), 256, 0, s>>>(L.nnz, L.sell_of_csr.as<int64_t>(), vals,
                                                                  L.sell_valb.as<__nv_bfloat16>());
}

// Diagonal scaling of the second-order hierarchy (reading K1): on every level
// A' = D^-1/2 A D^-1/2 and P' = D_l^1/2 P D_{l+1}^-1/2, which keeps the
// Galerkin relation A'_{l+1} = P'^T A'_l P'.  Level 0 keeps its unscaled
// operator for the outer CG (CSR and FP64 sliced-ELL values) and gets a scaled
// FP64 copy for the V-cycle; the coarser levels are scaled in place.  FP32
// copies hold the scaled values.
void scale_k2(fvem_ctx* C) {
  cudaStream_t s = C->stream;
  const int Lv = int(C->lv.size());
  for (int l = 0; l < Lv; ++l) {
    DevLevel& L = *C->lv[l];
    L.sv.alloc(sizeof(double) * size_t(std::max(1, L.ndof)));
    ++C->nlaunch, k_csr_invsqrt_diag<<<nblk(L.ndof), 256, 0, s>>>(L.ndof, L.a_rowptr.as<int64_t>(), L.a_col.as<int32_t>(),
                                                                  L.a_val.as<double>(), L.sv.as<double>());
  }
  for (int l = 0; l < Lv; ++l) {
    DevLevel& L = *C->lv[l];
    DBuf tmp;
    double* vals = L.a_val.as<double>();
    if (l == 0) {
      tmp.alloc(sizeof(double) * size_t(std::max<int64_t>(1, L.nnz)));
      CK(cudaMemcpyAsync(tmp.p, L.a_val.p, sizeof(double) * size_t(L.nnz), cudaMemcpyDeviceToDevice, s));
      vals = tmp.as<double>();
      L.vsell_val.alloc(L.sell_val.bytes);
      CK(cudaMemsetAsync(L.vsell_val.p, 0, L.vsell_val.bytes, s));
    }
    ++C->nlaunch, k_csr_scale_sym<<<nblk(L.ndof), 256, 0, s>>>(L.ndof, L.a_rowptr.as<int64_t>(), L.a_col.as<int32_t>(),
                                                               L.sv.as<double>(), vals);
    ++C->nlaunch, k_scatter_sell<double><<<nblk(L.nnz), 256, 0, s>>>(
                      L.nnz, L.sell_of_csr.as<int64_t>(), vals, l == 0 ? L.vsell_val.as<double>() : L.sell_val.as<double>());
    if (C->fp32_capable)
      ++C->nlaunch, k_scatter_sell<float><<<nblk(L.nnz), 256, 0, s>>>(L.nnz, L.sell_of_csr.as<int64_t>(), vals,
                                                                      L.sell_val32.as<float>());
    if (C->bf16_capable && l + 1 < Lv) make_v16(C, L, vals, s);
    CK(cudaStreamSynchronize(s));
  }
  for (int l = 0; l + 1 < Lv; ++l) {
    DevLevel& F = *C->lv[l];
    DevLevel& Cn = *C->lv[l + 1];
    if (!F.nnzp) continue;
    ++C->nlaunch, k_csr_scale_p<<<nblk(F.ndof), 256, 0, s>>>(F.ndof, F.pf_rowptr.as<int64_t>(), F.pf_col.as<int32_t>(),
                                                             F.sv.as<double>(), Cn.sv.as<double>(), F.pf_val.as<double>());
    if (C->fp32_capable)
      ++C->nlaunch, k_convert<double, float><<<nblk(F.nnzp), 256, 0, s>>>(F.nnzp, F.pf_val.as<double>(),
                                                                          F.pf_val32.as<float>());
    ++C->nlaunch, k_gather_vals<float><<<nblk(F.nnzp), 256, 0, s>>>(F.nnzp, F.pt_src.as<int64_t>(), F.pf_val.as<double>(),
                                                                    F.pt_val.as<double>(), F.pt_val32.as<float>());
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
}

void device_build(fvem_ctx* C) {
  cudaStream_t s = C->stream;
  const Topology& T = C->topo;
  int Lv = T.L;
  C->lv.clear();
  ++C->gen;            // every captured graph is stale
  C->pst.ok = false;  // rebuilt and re-tuned on the new coarsest level below
  C->pst.use[0] = C->pst.use[1] = false;
  C->d_err.alloc(sizeof(int));
  CK(cudaMemsetAsync(C->d_err.p, 0, sizeof(int), s));
  C->scal.alloc(16 * sizeof(double));
  CK(cudaMemsetAsync(C->scal.p, 0, 16 * sizeof(double), s));
  C->part.alloc(2 * RED_BLOCKS * sizeof(double));
  {
    // one partial per block of the level-0 product (largest grid: one warp per slice)
    int64_t ns0 = C->plan[0].nslices;
    C->part_big.alloc(sizeof(double) * size_t(std::max<int64_t>(RED_BLOCKS, ns0 + 16)));  // + schedule padding
  }
  C->rzqz.alloc(4 * sizeof(double));
  for (int l = 0; l < Lv; ++l) {
    auto L = std::make_unique<DevLevel>();
    const LevelMesh& M = T.levels[l];
    const LevelPlan& P = C->plan[l];
    L->nv = M.nv;
    L->nc = M.nc;
    L->ndof = P.ndof;
    L->nnz = P.a_rowptr.back();
    L->max_nv = P.max_nv;
    L->max_nf = P.max_nf;
    upload(L->V, M.V, s);
    upload(L->cell_vptr, M.cell_vptr, s);
    upload(L->cell_v, M.cell_v, s);
    upload(L->cell_fptr, M.cell_fptr, s);
    upload(L->face_vptr, M.face_vptr, s);
    upload(L->face_v, M.face_v, s);
    upload(L->face_pid, M.face_pid, s);
    upload(L->face_sg, M.face_sg, s);
    if (!P.elem_is_cell) {
      upload(L->elem_vptr_x, P.elem_vptr, s);
      upload(L->elem_v_x, P.elem_v, s);
    }
    upload(L->kptr, P.kptr, s);
    L->Kel.alloc(sizeof(double) * P.kptr.back());
    L->vol.alloc(sizeof(double) * M.nc);
    L->xE.alloc(sizeof(double) * 3 * M.nc);
    L->hE.alloc(sizeof(double) * M.nc);
    L->Pis.alloc(sizeof(double) * 4 * M.cell_v.size());
    upload(L->dof_of_vertex, P.dof_of_vertex, s);
    upload(L->vertex_of_dof, P.vertex_of_dof, s);
    upload(L->inc_ptr, P.inc_ptr, s);
    upload(L->inc_cell, P.inc_cell, s);
    upload(L->inc_loc, P.inc_loc, s);
    upload(L->a_rowptr, P.a_rowptr, s);
    upload(L->a_col, P.a_col, s);
    L->a_val.alloc(sizeof(double) * L->nnz);
    L->nslices = P.nslices;
    upload(L->sell_ptr, P.sell_ptr, s);
    upload(L->sell_w, P.sell_w, s);
    if (P.sell_d16)
      upload(L->sell_dcol, P.sell_dcol, s);
    else
      upload(L->sell_col, P.sell_col, s);
    L->d16 = P.sell_d16;
    upload(L->sell_of_csr, P.sell_of_csr, s);
    const size_t nslots = size_t(P.sell_ptr.back());
    L->sell_val.alloc(sizeof(double) * nslots);
    CK(cudaMemsetAsync(L->sell_val.p, 0, L->sell_val.bytes, s));
    if (C->fp32_capable) {
      L->sell_val32.alloc(sizeof(float) * nslots);
      CK(cudaMemsetAsync(L->sell_val32.p, 0, L->sell_val32.bytes, s));
    }
    if (C->prm.order_k == 2) {
      const LevelK2& K = C->k2[l];
      upload(L->k2_edge_ptr, K.edge_ptr, s);
      upload(L->k2_edge_v, K.edge_v, s);
      upload(L->k2_fpos_v, K.fpos_v, s);
      upload(L->k2_fpos_e, K.fpos_e, s);
      upload(L->k2_eptr, K.D.elem_ptr, s);
      upload(L->k2_edof, K.D.elem_dof, s);
      upload(L->k2_perm, K.perm, s);
      upload(L->k2_koff, K.k2_off, s);
      upload(L->k2_foff, K.face_off, s);
      L->Pis2.alloc(sizeof(double) * 10 * K.D.elem_dof.size());
      L->K2.alloc(sizeof(double) * size_t(K.k2_off.back()));
      L->mom2.alloc(sizeof(double) * 10 * size_t(std::max(1, M.nc)));
      L->face2.alloc(sizeof(double) * size_t(K.face_off.back()));
      L->k2_nf_cap = K.max_nf;
      L->k2_kcap = K.max_fk;
      L->k2_ne_cap = K.max_ne;
      if (l + 1 < Lv) {
        upload(L->pk, K.pk, s);
        upload(L->pC, K.pC, s);
        upload(L->pa2, K.pa, s);
        upload(L->pb2, K.pb, s);
        upload(L->px, K.px, s);
      }
    }
    if (l + 1 < Lv) {
      if (C->prm.order_k == 1) {
        const Placement& pl = T.place[l];
        upload(L->ptype, pl.type, s);
        upload(L->pcell, pl.cell, s);
        upload(L->pa, pl.a, s);
        upload(L->pb, pl.b, s);
      }
      upload(L->prow_ptr, P.prow_ptr, s);
      upload(L->prow_col, P.prow_col, s);
      L->prow_val.alloc(sizeof(double) * P.prow_col.size());
      upload(L->pf_rowptr, P.pf_rowptr, s);
      upload(L->pf_col, P.pf_col, s);
      upload(L->pf_src, P.pf_src, s);
      L->nnzp = int64_t(P.pf_col.size());
      L->pf_val.alloc(sizeof(double) * L->nnzp);
      upload(L->pt_rowptr, P.pt_rowptr, s);
      upload(L->pt_col, P.pt_col, s);
      upload(L->pt_src, P.pt_src, s);
      L->pt_val.alloc(sizeof(double) * L->nnzp);
      if (C->fp32_capable) {
        L->pf_val32.alloc(sizeof(float) * L->nnzp);
        L->pt_val32.alloc(sizeof(float) * L->nnzp);
      }
    }
    if (l > 0) {
      upload(L->child_ptr, P.child_ptr, s);
      upload(L->child_cell, P.child_cell, s);
    }
    size_t vbytes = sizeof(double) * size_t(std::max(1, L->ndof));
    L->b.alloc(vbytes);
    L->x.alloc(vbytes);
    L->r.alloc(vbytes);
    L->d0.alloc(vbytes);
    L->d1.alloc(vbytes);
    if (C->fp32_capable) {
      size_t fb = sizeof(float) * size_t(std::max(1, L->ndof));
      L->b32.alloc(fb);
      L->x32.alloc(fb);
      L->r32.alloc(fb);
      L->d032.alloc(fb);
      L->d132.alloc(fb);
    }
    C->lv.push_back(std::move(L));
  }
  // A2/A3: per-cell projectors on every level, element matrices on level 0
  for (int l = 0; l < Lv; ++l) {
    DevLevel& L = *C->lv[l];
    int maxf = std::max(1, L.max_nf);
    size_t per_warp = size_t(maxf) * 10 * sizeof(double);
    int wpb = int(std::max<size_t>(1, std::min<size_t>(8, (160 * 1024) / per_warp)));
    size_t smem = per_warp * wpb;
    if (smem > 227 * 1024) throw std::runtime_error("cell with too many faces for the element kernel");
    CK(cudaFuncSetAttribute(k_cell_vem, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
    unsigned grid = unsigned(std::max<int64_t>(1, std::min<int64_t>((L.nc + wpb - 1) / wpb, 148 * 32)));
    ++C->nlaunch, k_cell_vem<<<grid, 32 * wpb, smem, s>>>(L.mesh(), maxf, L.vol.as<double>(), L.xE.as<double>(), L.hE.as<double>(),
                                             L.Pis.as<double>(), L.kptr.as<int64_t>(),
                                             (l == 0 && C->prm.order_k == 1) ? L.Kel.as<double>() : nullptr);
    CK(cudaGetLastError());
  }
  if (C->prm.order_k == 2) {
    // second-order projectors and element matrices on every level (A2/A3)
    for (int l = 0; l < Lv; ++l) {
      DevLevel& L = *C->lv[l];
      const size_t per_warp = sizeof(double) * k2_warp_doubles(std::max(1, L.k2_nf_cap), std::max(3, L.k2_kcap),
                                                               std::max(2, L.k2_ne_cap));
      const int wpb = int(std::max<size_t>(1, std::min<size_t>(4, (200 * 1024) / per_warp)));
      const size_t smem = per_warp * wpb;
      if (smem > 227 * 1024) throw std::runtime_error("cell too large for the second-order element kernel");
      CK(cudaFuncSetAttribute(k_elem_k2, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem)));
      K2View kv{L.k2_edge_ptr.as<int32_t>(), L.k2_edge_v.as<int32_t>(), L.k2_fpos_v.as<int32_t>(),
                L.k2_fpos_e.as<int32_t>(), L.k2_eptr.as<int64_t>(), L.k2_koff.as<int64_t>(), L.k2_foff.as<int64_t>()};
      const unsigned grid = unsigned(std::max<int64_t>(1, std::min<int64_t>((L.nc + wpb - 1) / wpb, 148 * 64)));
      ++C->nlaunch, k_elem_k2<<<grid, 32 * wpb, smem, s>>>(
                        L.mesh(), kv, L.vol.as<double>(), L.xE.as<double>(), L.hE.as<double>(), std::max(1, L.k2_nf_cap),
                        std::max(3, L.k2_kcap), std::max(2, L.k2_ne_cap), L.Pis2.as<double>(), L.K2.as<double>(),
                        L.mom2.as<double>(), L.face2.as<double>(), C->d_err.as<int>());
      CK(cudaGetLastError());
    }
    // level 0 element blocks: the condensed element matrices (reading K2)
    DevLevel& L0 = *C->lv[0];
    ++C->nlaunch, k_condense_k2<<<nblk(L0.nc, 128), 128, 0, s>>>(L0.nc, L0.k2_eptr.as<int64_t>(), L0.k2_koff.as<int64_t>(),
                                                                 L0.K2.as<double>(), L0.k2_perm.as<int32_t>(),
                                                                 L0.kptr.as<int64_t>(), L0.Kel.as<double>());
    CK(cudaGetLastError());
    check_err(C, "second-order elements");
  }
  // A5/A6: prolongation rows, Galerkin element blocks, then A4 assembly per level
  for (int l = 0; l < Lv; ++l) {
    DevLevel& L = *C->lv[l];
    if (l > 0) {
      DevLevel& F = *C->lv[l - 1];
      if (C->prm.order_k == 2) {
        ProlongK2 pr{F.pk.as<int8_t>(), F.pC.as<int32_t>(), F.pa2.as<int32_t>(), F.pb2.as<int32_t>(), F.px.as<double>()};
        const int64_t nrows = C->k2[l - 1].cdof;
        ++C->nlaunch, k_prolong_k2<<<nblk(nrows), 256, 0, s>>>(
                          nrows, pr, F.mesh(), L.mesh(), L.k2_eptr.as<int64_t>(), L.Pis2.as<double>(), L.xE.as<double>(),
                          L.hE.as<double>(), L.k2_koff.as<int64_t>(), L.K2.as<double>(), L.face2.as<double>(),
                          L.k2_foff.as<int64_t>(), F.prow_ptr.as<int32_t>(), F.prow_val.as<double>());
      } else {
        ++C->nlaunch, k_prolong_rows<<<nblk(F.nv), 256, 0, s>>>(F.nv, F.V.as<double>(), F.ptype.as<int8_t>(), F.pcell.as<int32_t>(),
                                                 F.pa.as<int32_t>(), F.pb.as<int32_t>(), L.mesh(), L.Pis.as<double>(),
                                                 L.xE.as<double>(), L.hE.as<double>(), F.prow_ptr.as<int32_t>(),
                                                 F.prow_val.as<double>());
      }
      CK(cudaGetLastError());
      {
        // warp per coarse cell with T = K^e P_e in shared memory when it fits
        const int tcap = std::max(1, C->plan[l - 1].max_ne * C->plan[l].max_ne);
        const size_t per_warp = sizeof(double) * size_t(tcap);
        const int wpb = int(std::max<size_t>(1, std::min<size_t>(8, (96 * 1024) / per_warp)));
        if (per_warp * wpb <= 200 * 1024) {
          CK(cudaFuncSetAttribute(k_galerkin_warp, cudaFuncAttributeMaxDynamicSharedMemorySize, int(per_warp * wpb)));
          const unsigned grid = unsigned(std::max<int64_t>(1, std::min<int64_t>((L.nc + wpb - 1) / wpb, 148 * 64)));
          ++C->nlaunch, k_galerkin_warp<<<grid, 32 * wpb, per_warp * wpb, s>>>(
                            L.nc, L.child_ptr.as<int32_t>(), L.child_cell.as<int32_t>(), F.elem_vptr(), F.elem_v(),
                            F.kptr.as<int64_t>(), F.Kel.as<double>(), F.prow_ptr.as<int32_t>(), F.prow_col.as<int32_t>(),
                            F.prow_val.as<double>(), F.dof_of_vertex.as<int32_t>(), L.elem_vptr(), L.elem_v(),
                            L.kptr.as<int64_t>(), L.Kel.as<double>(), tcap, C->d_err.as<int>());
        } else {
          ++C->nlaunch, k_galerkin<<<nblk(L.nc, 128), 128, 0, s>>>(L.nc, L.child_ptr.as<int32_t>(), L.child_cell.as<int32_t>(),
                                                   F.elem_vptr(), F.elem_v(), F.kptr.as<int64_t>(),
                                                   F.Kel.as<double>(), F.prow_ptr.as<int32_t>(), F.prow_col.as<int32_t>(),
                                                   F.prow_val.as<double>(), F.dof_of_vertex.as<int32_t>(),
                                                   L.elem_vptr(), L.elem_v(), L.kptr.as<int64_t>(),
                                                   L.Kel.as<double>(), C->d_err.as<int>());
        }
      }
      CK(cudaGetLastError());
      if (F.nnzp) {
        ++C->nlaunch, k_gather_vals<float><<<nblk(F.nnzp), 256, 0, s>>>(F.nnzp, F.pf_src.as<int64_t>(), F.prow_val.as<double>(),
                                                         F.pf_val.as<double>(), F.pf_val32.as<float>());
        ++C->nlaunch, k_gather_vals<float><<<nblk(F.nnzp), 256, 0, s>>>(F.nnzp, F.pt_src.as<int64_t>(), F.pf_val.as<double>(),
                                                         F.pt_val.as<double>(), F.pt_val32.as<float>());
      }
    }
    ++C->nlaunch, k_assemble<<<nblk(L.ndof, 128), 128, 0, s>>>(L.ndof, L.vertex_of_dof.as<int32_t>(), L.dof_of_vertex.as<int32_t>(),
                                                 L.inc_ptr.as<int32_t>(), L.inc_cell.as<int32_t>(),
                                                 L.inc_loc.as<int32_t>(), L.elem_vptr(),
                                                 L.elem_v(), L.kptr.as<int64_t>(), L.Kel.as<double>(),
                                                 L.a_rowptr.as<int64_t>(), L.a_col.as<int32_t>(), L.a_val.as<double>(),
                                                 C->d_err.as<int>());
    CK(cudaGetLastError());
    ++C->nlaunch, k_scatter_sell<double><<<nblk(L.nnz), 256, 0, s>>>(L.nnz, L.sell_of_csr.as<int64_t>(), L.a_val.as<double>(),
                                                      L.sell_val.as<double>());
    if (C->fp32_capable)
      ++C->nlaunch, k_scatter_sell<float><<<nblk(L.nnz), 256, 0, s>>>(L.nnz, L.sell_of_csr.as<int64_t>(), L.a_val.as<double>(),
                                                       L.sell_val32.as<float>());
    CK(cudaGetLastError());
  }
  check_err(C, "assembly");
  if (C->prm.order_k == 2) {
    scale_k2(C);
  } else if (C->bf16_capable) {
    for (int l = 0; l + 1 < Lv; ++l) make_v16(C, *C->lv[l], C->lv[l]->a_val.as<double>(), s);
  }
  set_bf16_flags(C);
  mark_stencils(C);
  for (int l = 0; l < Lv; ++l) C->lv[l]->lmax = lanczos_lmax(C, *C->lv[l]);
  TuneRecord tr;
  const bool pinned = tune_load(C, tr);
  for (int l = 0; l < Lv; ++l) {
    if (pinned) {
      C->lv[l]->cfg64 = tr.cfg64[l];
      C->lv[l]->cfg32 = tr.cfg32[l];
      C->lv[l]->stc_on = tr.stc32[l] != 0;
      continue;
    }
    C->lv[l]->cfg64 = tune_sell<double>(C, *C->lv[l]);
    if (C->fp32_capable) C->lv[l]->cfg32 = tune_sell<float>(C, *C->lv[l]);
  }
  {
    int dev = 0, nsm = 0, a64 = 0, a32 = 0, coop = 0;
    CK(cudaGetDevice(&dev));
    CK(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev));
    if (!coop && C->prm.coarse_solver == FVEM_COARSE_CG)
      throw std::runtime_error("device without cooperative launch: use the Chebyshev coarsest solver");
    DevLevel& Lc = *C->lv[Lv - 1];
    // resident blocks per SM of each coarse-CG variant (the launch must stay co-resident)
    auto occ = [&](int cfg) {
      int a = 0;
      CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, coarse_fn<double>(Lc.d16, cfg), 256, 0));
      return std::max(1, a);
    };
    a64 = occ(0);
    for (int cfg = 1; cfg < kCoarseCfgCount; ++cfg) a64 = std::min(a64, occ(cfg));
    auto occ32 = [&](int cfg) {
      int a = 0;
      CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, coarse_fn<float>(Lc.d16, cfg), 256, 0));
      return std::max(1, a);
    };
    a32 = occ32(0);
    for (int cfg = 1; cfg < kCoarseCfgCount; ++cfg) a32 = std::min(a32, occ32(cfg));
    C->coop_blocks_f64 = a64 * nsm;
    C->coop_blocks_f32 = a32 * nsm;
    C->coop_red.alloc(sizeof(double) * 4 * size_t(std::max(C->coop_blocks_f64, C->coop_blocks_f32)));
    Lc.cw.alloc(sizeof(double) * size_t(std::max(1, Lc.ndof)));
    if (C->fp32_capable && C->prm.coarse_solver == FVEM_COARSE_CG)
      Lc.cw32.alloc(sizeof(float) * size_t(std::max(1, Lc.ndof)));
    C->ccg_part.alloc(sizeof(double) * 2 * size_t(Lc.nslices + 16));  // + schedule padding
    C->ccg_cs.alloc(sizeof(double) * 8);
    CK(cudaMemsetAsync(C->ccg_cs.p, 0, sizeof(double) * 8, s));
    if (pinned) {
      C->coarse_seq = tr.coarse_seq != 0;
      C->coarse_ks = tr.coarse_ks;
      C->ccg_cfg = tr.ccg_cfg;
      C->ccg_cfg32 = tr.ccg_cfg32 < kSellCfgCount + kMixCount ? tr.ccg_cfg32 : 0;
      C->coarse_coop32 = tr.coop32 != 0;
      C->coarse_ks32 = tr.ks32;
      if (tr.nb32 > 0) C->coop_blocks_f32 = tr.nb32;
      C->coop32_ms = tr.coop32_ms;
      C->ccg32_ms = tr.ccg32_ms;
      if (tr.coop_nb > 0) C->coop_blocks_f64 = tr.coop_nb;
      C->coarse_seq_ms = tr.seq_ms;
      C->coarse_coop_ms = tr.coop_ms;
    }
    // tune the cooperative launch: warps per slice x blocks per SM
    if (C->prm.coarse_solver == FVEM_COARSE_CG && !pinned) {
      int best_nb = C->coop_blocks_f64, best_ks = 2;
      float best = 1e30f;
      cudaEvent_t e0, e1;
      CK(cudaEventCreate(&e0));
      CK(cudaEventCreate(&e1));
      double* v[5] = {vec<double>(Lc, 0), vec<double>(Lc, 1), vec<double>(Lc, 2), vec<double>(Lc, 3),
                      vec<double>(Lc, 4)};
      // a right-hand side in the range of the (possibly singular) coarsest
      // operator, so every variant runs the same iterations: b = A v
      ++C->nlaunch, k_power_init<<<RED_BLOCKS, 256, 0, s>>>(Lc.ndof, v[1]);
      if (Lc.d16)
        ++C->nlaunch, k_spmv<double, 4, 1, true><<<sell_grid(Lc.sell<double>(), 1), 256, 0, s>>>(Lc.sell<double>(), v[1], v[0]);
      else
        ++C->nlaunch, k_spmv<double, 4, 1, false><<<sell_grid(Lc.sell<double>(), 1), 256, 0, s>>>(Lc.sell<double>(), v[1], v[0]);
      C->coarse_seq = false;
      for (int ks = 0; ks < kCoarseCfgCount; ++ks)
        for (int per = 1; per <= a64; ++per) {
          C->coarse_ks = ks;
          C->coop_blocks_f64 = per * nsm;
          float ms = 0;
          for (int rep = 0; rep < 2; ++rep) {
            CK(cudaEventRecord(e0, s));
            coarse_cg<double>(C, Lc, v[0], v[1], v[2], v[3], v[4], C->coop_red.as<double>());
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            CK(cudaEventElapsedTime(&ms, e0, e1));
          }
          if (ms < best) {
            best = ms;
            best_nb = C->coop_blocks_f64;
            best_ks = ks;
          }
        }
      C->coop_blocks_f64 = best_nb;
      C->coarse_ks = best_ks;
      // kernel-sequence form: first its product kernel's launch shape, then the
      // whole sequence timed as a graph replay (its production use)
      {
        float bp = 1e30f;
        for (int cfg = 0; cfg < kSellCfgCount; ++cfg) {
          float ms = 0;
          for (int rep = 0; rep < 2; ++rep) {
            CK(cudaEventRecord(e0, s));
            for (int k = 0; k < 10; ++k)
              with_cfg(cfg, Lc.d16, [&](auto u, auto ks, auto dd) {
                constexpr int U = decltype(u)::value, KS = decltype(ks)::value;
                constexpr bool D = decltype(dd)::value;
                // cs[4] = 1 makes the kernel return at once, so time with a fresh state each call
                ++C->nlaunch, k_ccg_prod<double, U, KS, D><<<sell_grid(Lc.sell<double>(), KS), 256, 0, s>>>(
                                  Lc.sell<double>(), v[0], v[4], C->ccg_part.as<double>(), C->ccg_cs.as<double>(), 1);
              });
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            CK(cudaEventElapsedTime(&ms, e0, e1));
          }
          if (ms < bp) {
            bp = ms;
            C->ccg_cfg = cfg;
          }
        }
        CK(cudaMemsetAsync(C->ccg_cs.p, 0, sizeof(double) * 8, s));
        C->coarse_seq = true;
        cudaStream_t user = C->stream;
        cudaStream_t cs_ = nullptr;
        CK(cudaStreamCreateWithFlags(&cs_, cudaStreamNonBlocking));
        cudaGraph_t g = nullptr;
        cudaGraphExec_t ge = nullptr;
        C->stream = cs_;
        int64_t n0 = C->nlaunch;
        bool ok = cudaStreamBeginCapture(cs_, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
        if (ok) {
          coarse_cg<double>(C, Lc, v[0], v[1], v[2], v[3], v[4], C->coop_red.as<double>());
          ok = cudaStreamEndCapture(cs_, &g) == cudaSuccess;
        }
        C->stream = user;
        C->nlaunch = n0;
        if (ok) ok = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
        float ms = 1e30f;
        if (ok) {
          for (int rep = 0; rep < 2; ++rep) {
            CK(cudaEventRecord(e0, s));
            CK(cudaGraphLaunch(ge, s));
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            CK(cudaEventElapsedTime(&ms, e0, e1));
          }
        }
        if (ge) cudaGraphExecDestroy(ge);
        if (g) cudaGraphDestroy(g);
        cudaStreamDestroy(cs_);
        cudaGetLastError();
        C->coarse_seq = ok && ms < best;
        C->coarse_seq_ms = ms;
        C->coarse_coop_ms = best;
      }
      // FP32 kernel sequence of the FP32 V-cycle: each product shape timed as a
      // replay of the captured sequence (its production use)
      if (Lc.cw32.p) {
        float* f[5] = {vec<float>(Lc, 0), vec<float>(Lc, 1), vec<float>(Lc, 2), vec<float>(Lc, 3), vec<float>(Lc, 4)};
        ++C->nlaunch, k_convert<double, float><<<nblk(Lc.ndof), 256, 0, s>>>(Lc.ndof, v[0], f[0]);
        CK(cudaGetLastError());
        cudaStream_t user = C->stream;
        cudaStream_t cs_ = nullptr;
        CK(cudaStreamCreateWithFlags(&cs_, cudaStreamNonBlocking));
        CK(cudaStreamSynchronize(s));
        const int64_t n0 = C->nlaunch;
        float bt = 1e30f;
        bool bstc = false;
        const int nshape = kSellCfgCount + kMixCount;
        const bool can_stc = Lc.reg32.p != nullptr;  // timed with and without stencil slices
        for (int trial = 0; trial < (can_stc ? 2 * nshape : nshape); ++trial) {
          const int cfg = trial % nshape;
          const bool stc = trial >= nshape;
          Lc.stc_on = stc;
          if (cfg >= kSellCfgCount) build_mix(C, Lc, C->plan[Lv - 1], kMixBound[cfg - kSellCfgCount]);
          cudaGraph_t g = nullptr;
          cudaGraphExec_t ge = nullptr;
          C->stream = cs_;
          bool okc = cudaStreamBeginCapture(cs_, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
          if (okc) {
            coarse_cg_seq<float>(C, Lc, f[0], f[1], f[2], f[3], f[4], Lc.cw32.as<float>(), C->ccg_part.as<double>(),
                                 C->ccg_cs.as<double>(), cfg);
            okc = cudaStreamEndCapture(cs_, &g) == cudaSuccess;
          }
          C->stream = user;
          if (okc) okc = cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
          float t = 1e30f;
          for (int rep = 0; okc && rep < 3; ++rep) {
            CK(cudaEventRecord(e0, s));
            CK(cudaGraphLaunch(ge, s));
            CK(cudaEventRecord(e1, s));
            CK(cudaEventSynchronize(e1));
            float m = 0;
            CK(cudaEventElapsedTime(&m, e0, e1));
            if (rep > 0) t = std::min(t, m);
          }
          if (ge) cudaGraphExecDestroy(ge);
          if (g) cudaGraphDestroy(g);
          cudaGetLastError();
          if (std::getenv("FVEM_TIMING"))
            std::fprintf(stderr, "[fvem] FP32 coarsest CG, product shape %d%s: %.4f ms\n", cfg,
                         stc ? " (stencil)" : "", t);
          if (okc && t < bt) {
            bt = t;
            bstc = stc;
            C->ccg_cfg32 = cfg;
          }
        }
        C->nlaunch = n0;
        C->ccg32_ms = bt;
        Lc.stc_on = bstc;
        cudaStreamDestroy(cs_);
        // the FP32 cooperative form: warps per slice x blocks per SM
        float bc = 1e30f;
        int best_nb32 = C->coop_blocks_f32, best_ks32 = 0;
        for (int ks = 0; ks < kCoarseCfgCount; ++ks)
          for (int per = 1; per <= a32; ++per) {
            C->coarse_ks32 = ks;
            C->coop_blocks_f32 = per * nsm;
            float t = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
              CK(cudaEventRecord(e0, s));
              coarse_cg<float>(C, Lc, f[0], f[1], f[2], f[3], f[4], C->coop_red.as<double>(), Lc.cw32.as<float>());
              CK(cudaEventRecord(e1, s));
              CK(cudaEventSynchronize(e1));
              float m = 0;
              CK(cudaEventElapsedTime(&m, e0, e1));
              if (rep > 0) t = std::min(t, m);
            }
            if (std::getenv("FVEM_TIMING"))
              std::fprintf(stderr, "[fvem] FP32 coarsest CG, cooperative shape %d, %d blocks: %.4f ms\n", ks,
                           per * nsm, t);
            if (t < bc) {
              bc = t;
              best_nb32 = per * nsm;
              best_ks32 = ks;
            }
          }
        C->nlaunch = n0;
        C->coop_blocks_f32 = best_nb32;
        C->coarse_ks32 = best_ks32;
        C->coop32_ms = bc;
        C->coarse_coop32 = bc < bt;
      }
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    // the mixed-split product keeps the slice lists of its chosen bound
    if (Lc.cw32.p && C->ccg_cfg32 >= kSellCfgCount)
      build_mix(C, Lc, C->plan[Lv - 1], kMixBound[C->ccg_cfg32 - kSellCfgCount]);
    // the persistent form, timed against the best of the forms above
    if (C->prm.coarse_solver == FVEM_COARSE_CG) {
      build_persist(C, Lc, C->plan[Lv - 1]);
      auto& ps = C->pst;
      ps.use[0] = ps.use[1] = false;
      int optin = 0, dev = 0;
      CK(cudaGetDevice(&dev));
      CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
      auto fits = [&](int prec) { return ps.smem(prec) + 1024 <= size_t(optin); };
      if (ps.ok && pinned) {
        ps.use[0] = tr.persist64 != 0 && fits(0);
        ps.use[1] = tr.persist32 != 0 && Lc.cw32.p && fits(1);
        ps.ms[0] = tr.pms64;
        ps.ms[1] = tr.pms32;
      } else if (ps.ok) {
        cudaEvent_t e0, e1;
        CK(cudaEventCreate(&e0));
        CK(cudaEventCreate(&e1));
        const int64_t n0 = C->nlaunch;
        for (int prec = 0; prec < 2; ++prec) {
          if (prec == 1 && !Lc.cw32.p) continue;
          const void* fn = prec == 0 ? persist_fn<double>() : persist_fn<float>();
          float best = 1e30f;
          {
            if (!fits(prec)) continue;
            int occ = 0;
            CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, 1024, ps.smem(prec)));
            if (occ < 1) continue;
            float t = 1e30f;
            for (int rep = 0; rep < 3; ++rep) {
              CK(cudaEventRecord(e0, s));
              if (prec == 0)
                coarse_persist<double>(C, Lc, vec<double>(Lc, 0), vec<double>(Lc, 1));
              else
                coarse_persist<float>(C, Lc, vec<float>(Lc, 0), vec<float>(Lc, 1));
              CK(cudaEventRecord(e1, s));
              CK(cudaEventSynchronize(e1));
              float m = 0;
              CK(cudaEventElapsedTime(&m, e0, e1));
              if (rep > 0) t = std::min(t, m);
            }
            if (coarse_timed_out(C)) {
              reset_persist(C);
              t = 1e30f;
            }
            if (std::getenv("FVEM_TIMING"))
              std::fprintf(stderr, "[fvem] %s coarsest CG, persistent: %.4f ms\n", prec ? "FP32" : "FP64", t);
            best = t;
          }
          ps.ms[prec] = best < 1e29f ? best : 0.f;
          const float other = prec == 0 ? (C->coarse_seq ? C->coarse_seq_ms : C->coarse_coop_ms)
                                        : std::min(C->ccg32_ms, C->coop32_ms);
          ps.use[prec] = best < other;
        }
        C->nlaunch = n0;
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
      }
      tr.persist64 = ps.use[0] ? 1 : 0;
      tr.persist32 = ps.use[1] ? 1 : 0;
      tr.pks64 = tr.pks32 = ps.kmax;  // parts per slice at most (set by the plan)
      tr.pms64 = ps.ms[0];
      tr.pms32 = ps.ms[1];
    }
    if (!pinned) {
      tr.cfg64.clear();
      tr.cfg32.clear();
      tr.stc32.clear();
      for (auto& L : C->lv) {
        tr.cfg64.push_back(L->cfg64);
        tr.cfg32.push_back(L->cfg32);
        tr.stc32.push_back(L->stc_on ? 1 : 0);
      }
      tr.coarse_seq = C->coarse_seq ? 1 : 0;
      tr.coarse_ks = C->coarse_ks;
      tr.coop_nb = C->coop_blocks_f64;
      tr.ccg_cfg = C->ccg_cfg;
      tr.ccg_cfg32 = C->ccg_cfg32;
      tr.coop32 = C->coarse_coop32 ? 1 : 0;
      tr.ks32 = C->coarse_ks32;
      tr.nb32 = C->coop_blocks_f32;
      tr.coop32_ms = C->coop32_ms;
      tr.ccg32_ms = C->ccg32_ms;
      tr.seq_ms = C->coarse_seq_ms;
      tr.coop_ms = C->coarse_coop_ms;
      tune_save(C, tr);
    }
  }
  // solver vectors
  DevLevel& L0 = *C->lv[0];
  size_t n8 = sizeof(double) * size_t(L0.ndof);
  C->cg_x.alloc(n8);
  C->cg_r.alloc(n8);
  C->cg_z.alloc(n8);
  C->cg_p.alloc(n8);
  C->cg_q.alloc(n8);
  if (C->fp32_capable) C->r32.alloc(sizeof(float) * size_t(L0.ndof));
  C->rloc.alloc(sizeof(double) * std::max(C->topo.levels[0].cell_v.size(), C->plan[0].elem_v.size()));
  if (C->prm.order_k == 2) C->rc2.alloc(sizeof(double) * size_t(std::max(1, L0.nc)));
  C->rloc3.alloc(3 * sizeof(double) * C->topo.levels[0].cell_v.size());
  C->pfull.alloc(sizeof(double) * size_t(L0.nv));
  CK(cudaStreamSynchronize(s));
}

// RHS (free DOFs) into cg_r from the velocity at level-0 vertices.
void build_rhs(fvem_ctx* C, const double* d_u, double u_in) {
  DevLevel& L0 = *C->lv[0];
  cudaStream_t s = C->stream;
  if (C->prm.order_k == 2) {
    ++C->nlaunch, k_rhs_k2<<<nblk(L0.nc, 128), 128, 0, s>>>(
                      L0.mesh(), L0.Pis.as<double>(), L0.hE.as<double>(), d_u, L0.nv, L0.k2_eptr.as<int64_t>(),
                      L0.Pis2.as<double>(), L0.mom2.as<double>(), L0.k2_koff.as<int64_t>(), L0.K2.as<double>(),
                      L0.k2_perm.as<int32_t>(), L0.elem_vptr(), C->rloc.as<double>(), C->rc2.as<double>());
    ++C->nlaunch, k_gather_dofs<<<nblk(L0.ndof), 256, 0, s>>>(L0.ndof, L0.vertex_of_dof.as<int32_t>(), L0.inc_ptr.as<int32_t>(),
                                                              L0.inc_cell.as<int32_t>(), L0.inc_loc.as<int32_t>(),
                                                              L0.elem_vptr(), C->rloc.as<double>(), C->cg_r.as<double>());
    return;
  }
  ++C->nlaunch, k_rhs_local<<<nblk(L0.nc, 128), 128, 0, s>>>(L0.mesh(), L0.Pis.as<double>(), L0.vol.as<double>(),
                                               L0.hE.as<double>(), d_u, L0.nv, u_in, C->rloc.as<double>());
  ++C->nlaunch, k_gather_dofs<<<nblk(L0.ndof), 256, 0, s>>>(L0.ndof, L0.vertex_of_dof.as<int32_t>(), L0.inc_ptr.as<int32_t>(),
                                              L0.inc_cell.as<int32_t>(), L0.inc_loc.as<int32_t>(),
                                              L0.cell_vptr.as<int32_t>(), C->rloc.as<double>(), C->cg_r.as<double>());
}

// Pressure at every DOF and the corrected cell velocities from the CG
// solution in cg_x: k = 1 the vertex pressures; k = 2 the boundary DOFs, then
// each cell's mean DOF recovered from its element and the correction.
void issue_finish(fvem_ctx* C, const double* d_u, double* d_p, double* d_cell) {
  DevLevel& L0 = *C->lv[0];
  cudaStream_t s = C->stream;
  if (C->prm.order_k == 2) {
    const int64_t cdof = C->k2[0].cdof;
    ++C->nlaunch, k_expand<<<nblk(cdof), 256, 0, s>>>(int(cdof), L0.dof_of_vertex.as<int32_t>(), C->cg_x.as<double>(), d_p);
    ++C->nlaunch, k_correct_k2<<<nblk(L0.nc, 128), 128, 0, s>>>(
                      L0.mesh(), L0.Pis.as<double>(), L0.hE.as<double>(), d_u, L0.nv, L0.k2_eptr.as<int64_t>(),
                      L0.k2_edof.as<int64_t>(), L0.Pis2.as<double>(), L0.k2_koff.as<int64_t>(), L0.K2.as<double>(),
                      C->rc2.as<double>(), d_p, cdof, d_p, d_cell);
    return;
  }
  ++C->nlaunch, k_expand<<<nblk(L0.nv), 256, 0, s>>>(L0.nv, L0.dof_of_vertex.as<int32_t>(), C->cg_x.as<double>(), d_p);
  ++C->nlaunch, k_correct<<<nblk(L0.nc, 128), 128, 0, s>>>(L0.mesh(), L0.Pis.as<double>(), L0.hE.as<double>(), d_u, L0.nv,
                                                           d_p, d_cell);
}

// Length of the pressure output: level-0 vertices (k = 1) or every k = 2 DOF.
int64_t pressure_len(const fvem_ctx* C) {
  return C->prm.order_k == 2 ? C->k2[0].D.n : int64_t(C->topo.levels[0].nv);
}

}  // namespace

// ------------------------------------------------------------------ API

extern "C" {

void fvem_default_params(fvem_params* p) {
  if (!p) return;
  p->order_k = 1;
  p->levels = 5;
  p->cheb_degree = 5;
  p->precision = FVEM_PREC_FP64;
  p->rel_tol = 1e-6;
  p->max_iters = 500;
  p->coarse_solver = FVEM_COARSE_CG;
  p->coarse_degree = 80;
  p->balance = 1;
  p->naive_prolongation = 0;
}

fvem_status fvem_create(const fvem_params* params, void* cuda_stream, fvem_ctx** out) {
  if (!out) return FVEM_EINVAL;
  *out = nullptr;
  fvem_ctx* C = nullptr;
  try {
    C = new fvem_ctx();
  } catch (...) {
    return FVEM_ENOMEM;
  }
  if (params)
    C->prm = *params;
  else
    fvem_default_params(&C->prm);
  const fvem_params& p = C->prm;
  if ((p.order_k != 1 && p.order_k != 2) || (p.order_k == 2 && p.levels < 2) || p.levels < 1 || p.levels > 16 || p.cheb_degree < 1 || p.cheb_degree > 64 ||
      p.coarse_degree < 1 || p.coarse_degree > 4096 || !(p.rel_tol > 0) || p.max_iters < 1 ||
      (p.precision != FVEM_PREC_FP64 && p.precision != FVEM_PREC_FP32 && p.precision != FVEM_PREC_BF16 &&
       p.precision != FVEM_PREC_FP16) ||
      (p.coarse_solver != FVEM_COARSE_CHEBYSHEV && p.coarse_solver != FVEM_COARSE_CG) ||
      (p.balance != 0 && p.balance != 1) || (p.naive_prolongation != 0 && p.naive_prolongation != 1)) {
    delete C;
    return FVEM_EINVAL;
  }
  C->stream = static_cast<cudaStream_t>(cuda_stream);
  static std::atomic<uint64_t> next_uid{1};
  C->uid = next_uid++;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) == cudaSuccess && ndev > 0) {
    C->has_device = true;
    if (cudaMallocHost(reinterpret_cast<void**>(&C->h_sc), 16 * sizeof(double)) != cudaSuccess) {
      delete C;
      return FVEM_ENOMEM;
    }
    cudaEventCreate(&C->ev0);
    cudaEventCreate(&C->ev1);
    cudaEventCreate(&C->ev2);
    cudaEventCreate(&C->ev3);
    cudaEventCreateWithFlags(&C->evb, cudaEventDisableTiming);
  } else {
    cudaGetLastError();
  }
  *out = C;
  return FVEM_OK;
}

void fvem_destroy(fvem_ctx* C) {
  if (!C) return;
  if (C->has_device) {
    cudaStreamSynchronize(C->stream);
    if (C->h_sc) cudaFreeHost(C->h_sc);
    if (C->ev0) cudaEventDestroy(C->ev0);
    if (C->ev1) cudaEventDestroy(C->ev1);
    if (C->ev2) cudaEventDestroy(C->ev2);
    if (C->ev3) cudaEventDestroy(C->ev3);
    if (C->evb) cudaEventDestroy(C->evb);
    if (C->pgraph) cudaGraphExecDestroy(C->pgraph);
    if (C->bgraph) cudaGraphExecDestroy(C->bgraph);
    for (auto& e : C->prof_ev) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    for (auto& e : C->gprof_ev) {
      cudaEventDestroy(e.first);
      cudaEventDestroy(e.second);
    }
    destroy_vgraph(C);
    if (C->cap_stream) cudaStreamDestroy(C->cap_stream);
  }
  delete C;
}

fvem_status fvem_build_topology(fvem_ctx* C, int N, const double* h_tris, int ntri) {
  if (!C || (ntri > 0 && !h_tris) || ntri < 0) return fail(C, FVEM_EINVAL, "bad arguments");
  API_BEGIN
  C->topo_ready = false;
  C->built = false;
  C->lv.clear();
  for (int64_t q = 0; q < int64_t(ntri) * 9; ++q)
    if (!std::isfinite(h_tris[q])) return fail(C, FVEM_ENAN, "non-finite triangle coordinate");
  std::string err;
  const auto t0 = std::chrono::steady_clock::now();
  if (build_topology(N, h_tris, ntri, C->prm.levels, C->prm.balance != 0, C->topo, err, C->prm.naive_prolongation != 0))
    return fail(C, FVEM_EGEOM, err);
  C->tris.assign(h_tris, h_tris + int64_t(ntri) * 9);
  C->pt.ready = false;
  if (C->prm.order_k == 2) {
    if (build_plan_k2(C->topo, C->plan, C->k2, err, C->prm.naive_prolongation != 0)) return fail(C, FVEM_EGEOM, err);
  } else {
    C->k2.clear();
    if (build_plan(C->topo, C->plan, err)) return fail(C, FVEM_EGEOM, err);
  }
  C->topo_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  C->device_s = 0.0;
  C->topo_ready = true;
  return FVEM_OK;
  API_END(C)
}

fvem_status fvem_build(fvem_ctx* C, int N, const double* h_tris, int ntri) {
  fvem_status st = fvem_build_topology(C, N, h_tris, ntri);
  if (st != FVEM_OK) return st;
  if (!C->has_device) return fail(C, FVEM_ENODEV, "no CUDA device");
  API_BEGIN
  C->fp32_capable = C->prm.precision == FVEM_PREC_FP32 || C->prm.precision == FVEM_PREC_BF16 ||
                    C->prm.precision == FVEM_PREC_FP16;
  C->bf16_capable = C->prm.precision == FVEM_PREC_BF16 || C->prm.precision == FVEM_PREC_FP16;
  C->v16_half = C->prm.precision == FVEM_PREC_FP16;
  const auto t0 = std::chrono::steady_clock::now();
  device_build(C);
  CK(cudaStreamSynchronize(C->stream));
  C->device_s = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  C->built = true;
  return FVEM_OK;
  API_END(C)
}

fvem_status fvem_query(const fvem_ctx* C, fvem_info* o) {
  if (!C || !o || !C->topo_ready) return FVEM_EINVAL;
  std::memset(o, 0, sizeof(*o));
  o->N = C->topo.N;
  o->levels = C->topo.L;
  o->order_k = C->prm.order_k;
  o->n_trees = C->topo.n_trees;
  for (int l = 0; l < C->topo.L && l < 16; ++l) {
    o->n_cells[l] = C->topo.levels[l].nc;
    o->n_vertices[l] = C->topo.levels[l].nv;
    o->n_dofs[l] = C->plan[l].ndof;
    o->nnz[l] = C->plan[l].a_rowptr.back();
    o->nnz_p[l] = int64_t(C->plan[l].pf_col.size());
    o->lmax[l] = C->built ? C->lv[l]->lmax : 0.0;
    o->n_dofs_all[l] = C->prm.order_k == 2 ? C->k2[l].D.n : int64_t(C->topo.levels[l].nv);
  }
  o->coarse_mode = (C->built && C->pst.ok && C->pst.use[0]) ? 2 : (C->coarse_seq ? 1 : 0);
  for (int l = 0; l < C->topo.L && l < 16 && C->built; ++l) {
    o->sell_cfg64[l] = C->lv[l]->cfg64;
    o->sell_cfg32[l] = C->lv[l]->cfg32;
  }
  o->coarse_ms[0] = C->coarse_coop_ms;
  o->coarse_ms[1] = C->coarse_seq_ms;
  const bool f32 = C->built && C->lv.back()->cw32.p;
  o->coarse_cfg[0] = C->built ? C->ccg_cfg : -1;
  o->coarse_cfg[1] = f32 ? C->ccg_cfg32 : -1;
  o->coarse_ms32 = f32 ? C->ccg32_ms : 0.0;
  o->coarse_mode32 = f32 ? ((C->pst.ok && C->pst.use[1]) ? 2 : (C->coarse_coop32 ? 0 : 1)) : -1;
  o->coarse_ms_persist[0] = C->built ? C->pst.ms[0] : 0.0;
  o->coarse_ms_persist[1] = f32 ? C->pst.ms[1] : 0.0;
  o->persist_ctas = C->built && C->pst.ok ? C->pst.nb : 0;
  o->coarse_ms32_coop = f32 ? C->coop32_ms : 0.0;
  o->setup_s[0] = C->topo_s;
  o->setup_s[1] = C->device_s;
  for (int l = 0; C->built && l < int(C->lv.size()) && l < 16; ++l) {
    o->stencil_slices32[l] = C->lv[l]->nreg32;
    o->stencil_classes32[l] = C->lv[l]->ncls32;
    o->stencil_used32[l] = (C->lv[l]->nreg32 > 0 && C->lv[l]->stc_on) ? 1 : 0;
  }
  return FVEM_OK;
}

fvem_status fvem_export_level(const fvem_ctx* C, int l, int64_t* counts, double* V, int32_t* cvp, int32_t* cv,
                              int32_t* cfp, int32_t* fvp, int32_t* fv, int32_t* fpid, int8_t* fsg, int32_t* par) {
  if (!C || !C->topo_ready || l < 0 || l >= C->topo.L || !counts) return FVEM_EINVAL;
  const LevelMesh& M = C->topo.levels[l];
  counts[0] = M.nv;
  counts[1] = M.nc;
  counts[2] = int64_t(M.cell_v.size());
  counts[3] = int64_t(M.face_pid.size());
  counts[4] = int64_t(M.face_v.size());
  if (V) std::memcpy(V, M.V.data(), sizeof(double) * M.V.size());
  if (cvp) std::memcpy(cvp, M.cell_vptr.data(), sizeof(int32_t) * M.cell_vptr.size());
  if (cv) std::memcpy(cv, M.cell_v.data(), sizeof(int32_t) * M.cell_v.size());
  if (cfp) std::memcpy(cfp, M.cell_fptr.data(), sizeof(int32_t) * M.cell_fptr.size());
  if (fvp) std::memcpy(fvp, M.face_vptr.data(), sizeof(int32_t) * M.face_vptr.size());
  if (fv) std::memcpy(fv, M.face_v.data(), sizeof(int32_t) * M.face_v.size());
  if (fpid) std::memcpy(fpid, M.face_pid.data(), sizeof(int32_t) * M.face_pid.size());
  if (fsg) std::memcpy(fsg, M.face_sg.data(), M.face_sg.size());
  if (par && !M.parent.empty()) std::memcpy(par, M.parent.data(), sizeof(int32_t) * M.parent.size());
  return FVEM_OK;
}

fvem_status fvem_export_placement(const fvem_ctx* C, int l, int8_t* t, int32_t* cell, int32_t* a, int32_t* b) {
  if (!C || !C->topo_ready || l < 0 || l + 1 >= C->topo.L) return FVEM_EINVAL;
  const Placement& p = C->topo.place[l];
  if (t) std::memcpy(t, p.type.data(), p.type.size());
  if (cell) std::memcpy(cell, p.cell.data(), sizeof(int32_t) * p.cell.size());
  if (a) std::memcpy(a, p.a.data(), sizeof(int32_t) * p.a.size());
  if (b) std::memcpy(b, p.b.data(), sizeof(int32_t) * p.b.size());
  return FVEM_OK;
}

fvem_status fvem_export_dofs(const fvem_ctx* C, int l, int32_t* d) {
  if (!C || !C->topo_ready || l < 0 || l >= C->topo.L || !d) return FVEM_EINVAL;
  std::memcpy(d, C->plan[l].dof_of_vertex.data(), sizeof(int32_t) * C->plan[l].dof_of_vertex.size());
  return FVEM_OK;
}

fvem_status fvem_export_dofs_k2(const fvem_ctx* C, int l, int64_t* counts, int64_t* elem_ptr, int64_t* elem_dof,
                                uint8_t* dirichlet) {
  if (!C || !C->topo_ready || l < 0 || l >= C->topo.L || !counts) return FVEM_EINVAL;
  DofsK2 D;
  build_dofs_k2(C->topo.levels[l], D);
  counts[0] = D.n;
  counts[1] = D.nv;
  counts[2] = D.ne;
  counts[3] = D.nf;
  counts[4] = D.nc;
  counts[5] = int64_t(D.elem_dof.size());
  if (elem_ptr) std::memcpy(elem_ptr, D.elem_ptr.data(), sizeof(int64_t) * D.elem_ptr.size());
  if (elem_dof) std::memcpy(elem_dof, D.elem_dof.data(), sizeof(int64_t) * D.elem_dof.size());
  if (dirichlet) std::memcpy(dirichlet, D.dirichlet.data(), D.dirichlet.size());
  return FVEM_OK;
}

fvem_status fvem_export_prolongation_pattern_k2(const fvem_ctx* C, int l, int64_t* counts, int64_t* rowptr,
                                                int64_t* col) {
  if (!C || !C->topo_ready || l < 0 || l + 1 >= C->topo.L || !counts) return FVEM_EINVAL;
  DofsK2 Df, Dc;
  build_dofs_k2(C->topo.levels[l], Df);
  build_dofs_k2(C->topo.levels[l + 1], Dc);
  std::vector<int64_t> rp, cl;
  build_prolongation_pattern_k2(C->topo.levels[l], C->topo.levels[l + 1], Df, Dc, rp, cl,
                                C->prm.naive_prolongation != 0);
  counts[0] = Df.n;
  counts[1] = Dc.n;
  counts[2] = int64_t(cl.size());
  if (rowptr) std::memcpy(rowptr, rp.data(), sizeof(int64_t) * rp.size());
  if (col) std::memcpy(col, cl.data(), sizeof(int64_t) * cl.size());
  return FVEM_OK;
}

fvem_status fvem_export_pattern_k2(const fvem_ctx* C, int l, int64_t* counts, int64_t* rowptr, int64_t* col) {
  if (!C || !C->topo_ready || l < 0 || l >= C->topo.L || !counts) return FVEM_EINVAL;
  DofsK2 D;
  build_dofs_k2(C->topo.levels[l], D);
  counts[0] = int64_t(D.a_rowptr.size()) - 1;
  counts[1] = int64_t(D.a_col.size());
  if (rowptr) std::memcpy(rowptr, D.a_rowptr.data(), sizeof(int64_t) * D.a_rowptr.size());
  if (col) std::memcpy(col, D.a_col.data(), sizeof(int64_t) * D.a_col.size());
  return FVEM_OK;
}

fvem_status fvem_export_matrix(const fvem_ctx* C, int which, int l, int64_t* counts, int64_t* rp, int32_t* col,
                               double* val) {
  if (!C || !C->topo_ready || l < 0 || l >= C->topo.L || !counts || which < 0 || which > 1) return FVEM_EINVAL;
  if (which == 1 && l + 1 >= C->topo.L) return FVEM_EINVAL;
  const LevelPlan& P = C->plan[l];
  const std::vector<int64_t>& R = which == 0 ? P.a_rowptr : P.pf_rowptr;
  const std::vector<int32_t>& K = which == 0 ? P.a_col : P.pf_col;
  counts[0] = P.ndof;
  counts[1] = which == 0 ? P.ndof : C->plan[l + 1].ndof;
  counts[2] = int64_t(K.size());
  if (rp) std::memcpy(rp, R.data(), sizeof(int64_t) * R.size());
  if (col) std::memcpy(col, K.data(), sizeof(int32_t) * K.size());
  if (val) {
    if (!C->built) return FVEM_EINVAL;
    fvem_ctx* M = const_cast<fvem_ctx*>(C);
    API_BEGIN
    const DBuf& src = which == 0 ? C->lv[l]->a_val : C->lv[l]->pf_val;
    CK(cudaMemcpyAsync(val, src.p, sizeof(double) * K.size(), cudaMemcpyDeviceToHost, C->stream));
    CK(cudaStreamSynchronize(C->stream));
    API_END(M)
  }
  return FVEM_OK;
}

fvem_status fvem_export_cells(const fvem_ctx* C, double* vol, double* cen, double* h, double* K) {
  if (!C || !C->built) return FVEM_EINVAL;
  fvem_ctx* M = const_cast<fvem_ctx*>(C);
  API_BEGIN
  const DevLevel& L = *C->lv[0];
  cudaStream_t s = C->stream;
  if (vol) CK(cudaMemcpyAsync(vol, L.vol.p, sizeof(double) * L.nc, cudaMemcpyDeviceToHost, s));
  if (cen) CK(cudaMemcpyAsync(cen, L.xE.p, sizeof(double) * 3 * L.nc, cudaMemcpyDeviceToHost, s));
  if (h) CK(cudaMemcpyAsync(h, L.hE.p, sizeof(double) * L.nc, cudaMemcpyDeviceToHost, s));
  if (K) CK(cudaMemcpyAsync(K, L.Kel.p, L.Kel.bytes, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return FVEM_OK;
  API_END(M)
}

fvem_status fvem_export_elements_k2(const fvem_ctx* C, int l, int64_t* counts, double* h_K, double* h_Pis,
                                    double* h_mom) {
  if (!C || !C->built || C->prm.order_k != 2 || l < 0 || l >= int(C->lv.size()) || !counts) return FVEM_EINVAL;
  const LevelK2& K = C->k2[l];
  counts[0] = K.k2_off.back();
  counts[1] = 10 * int64_t(K.D.elem_dof.size());
  counts[2] = 10 * int64_t(C->topo.levels[l].nc);
  fvem_ctx* M = const_cast<fvem_ctx*>(C);
  API_BEGIN
  const DevLevel& L = *C->lv[l];
  cudaStream_t s = C->stream;
  if (h_K) CK(cudaMemcpyAsync(h_K, L.K2.p, sizeof(double) * size_t(counts[0]), cudaMemcpyDeviceToHost, s));
  if (h_Pis) CK(cudaMemcpyAsync(h_Pis, L.Pis2.p, sizeof(double) * size_t(counts[1]), cudaMemcpyDeviceToHost, s));
  if (h_mom) CK(cudaMemcpyAsync(h_mom, L.mom2.p, sizeof(double) * size_t(counts[2]), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return FVEM_OK;
  API_END(M)
}

fvem_status fvem_quality(fvem_ctx* C, int level, double* d_rho, double* h_grid, int64_t* h_ncut) {
  if (!C || !C->built) return fail(C, FVEM_EINVAL, "not built");
  if (level < 0 || level >= int(C->lv.size())) return fail(C, FVEM_EINVAL, "level out of range");
  API_BEGIN
  DevLevel& L = *C->lv[size_t(level)];
  cudaStream_t s = C->stream;
  DBuf rbuf, fbuf, part;
  double* rho = d_rho;
  if (!rho) {
    rbuf.alloc(sizeof(double) * size_t(std::max(1, L.nc)));
    rho = rbuf.as<double>();
  }
  fbuf.alloc(sizeof(int) * size_t(std::max(1, L.nc)));
  constexpr int kBlocks = 148;
  part.alloc(sizeof(double) * 3 * kBlocks);
  ++C->nlaunch, k_quality<<<nblk(L.nc), 256, 0, s>>>(L.mesh(), rho, fbuf.as<int>());
  ++C->nlaunch, k_quality_sum<<<kBlocks, 256, 0, s>>>(L.nc, rho, fbuf.as<int>(), part.as<double>());
  std::vector<double> h(3 * kBlocks);
  CK(cudaMemcpyAsync(h.data(), part.p, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  double sq = 0.0, ncut = 0.0, nonconvex = 0.0;
  for (int b = 0; b < kBlocks; ++b) {
    sq += h[size_t(3 * b)];
    ncut += h[size_t(3 * b + 1)];
    nonconvex += h[size_t(3 * b + 2)];
  }
  if (h_ncut) *h_ncut = int64_t(ncut);
  if (h_grid) *h_grid = ncut > 0.0 ? std::sqrt(sq / ncut) : std::nan("");
  if (nonconvex > 0.0) return fail(C, FVEM_EGEOM, "a cell is not convex (its kernel is not computed)");
  return FVEM_OK;
  API_END(C)
}

// ------------------------------------------------------------------ particles (Sec. 3.2-3.3)

namespace {

int host_cube(double x, int N) {
  const double t = x * double(N);
  if (!(t >= 0.0)) return 0;
  if (t >= double(N)) return N - 1;
  return int(t);
}

// Level-0 cells and obstacle triangles binned by background cube, and each
// face occurrence's outward plane (unit Newell normal, d = n . face mean).
void particles_setup(fvem_ctx* C) {
  if (C->pt.ready) return;
  const LevelMesh& M = C->topo.levels[0];
  const int N = C->topo.N;
  const int64_t nbin = int64_t(N) * N * N;
  const double h = 1.0 / N;
  cudaStream_t s = C->stream;
  auto vx = [&](int v, int d) { return M.V[3 * size_t(v) + d]; };
  std::vector<int32_t> cbin(size_t(M.nc));
  std::vector<double> cvol(size_t(M.nc), 0.0);
  std::vector<double> plane(4 * M.face_pid.size());
  for (int c = 0; c < M.nc; ++c) {
    double m[3] = {0, 0, 0};
    const int nv = M.cell_vptr[c + 1] - M.cell_vptr[c];
    for (int q = M.cell_vptr[c]; q < M.cell_vptr[c + 1]; ++q)
      for (int d = 0; d < 3; ++d) m[d] += vx(M.cell_v[q], d);
    for (int d = 0; d < 3; ++d) m[d] /= nv;
    cbin[size_t(c)] = (host_cube(m[2], N) * N + host_cube(m[1], N)) * N + host_cube(m[0], N);
    for (int f = M.cell_fptr[c]; f < M.cell_fptr[c + 1]; ++f) {
      const int a = M.face_vptr[f], k = M.face_vptr[f + 1] - a;
      double n[3] = {0, 0, 0}, fm[3] = {0, 0, 0};
      for (int j = 0; j < k; ++j) {
        const int u = M.face_v[a + j], w = M.face_v[a + (j + 1) % k];
        n[0] += vx(u, 1) * vx(w, 2) - vx(u, 2) * vx(w, 1);
        n[1] += vx(u, 2) * vx(w, 0) - vx(u, 0) * vx(w, 2);
        n[2] += vx(u, 0) * vx(w, 1) - vx(u, 1) * vx(w, 0);
        for (int d = 0; d < 3; ++d) fm[d] += vx(u, d);
      }
      const double L = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      for (int d = 0; d < 3; ++d) {
        n[d] /= L;
        fm[d] /= k;
      }
      plane[4 * size_t(f)] = n[0];
      plane[4 * size_t(f) + 1] = n[1];
      plane[4 * size_t(f) + 2] = n[2];
      plane[4 * size_t(f) + 3] = n[0] * fm[0] + n[1] * fm[1] + n[2] * fm[2];
      // volume by the divergence theorem on the face's fan (about the cell's vertex mean)
      for (int j = 1; j + 1 < k; ++j) {
        double p0[3], p1[3], p2[3];
        for (int d = 0; d < 3; ++d) {
          p0[d] = vx(M.face_v[a], d) - m[d];
          p1[d] = vx(M.face_v[a + j], d) - m[d];
          p2[d] = vx(M.face_v[a + j + 1], d) - m[d];
        }
        cvol[size_t(c)] += (p0[0] * (p1[1] * p2[2] - p1[2] * p2[1]) - p0[1] * (p1[0] * p2[2] - p1[2] * p2[0]) +
                            p0[2] * (p1[0] * p2[1] - p1[1] * p2[0])) / 6.0;
      }
    }
  }
  std::vector<int32_t> cptr(size_t(nbin) + 1, 0), ccell(size_t(M.nc));
  for (int c = 0; c < M.nc; ++c) ++cptr[size_t(cbin[size_t(c)]) + 1];
  for (int64_t b = 0; b < nbin; ++b) cptr[size_t(b) + 1] += cptr[size_t(b)];
  {
    std::vector<int32_t> fill(cptr.begin(), cptr.end() - 1);
    for (int c = 0; c < M.nc; ++c) ccell[size_t(fill[size_t(cbin[size_t(c)])]++)] = c;
  }
  std::vector<uint8_t> full(size_t(nbin), 0);
  for (int64_t b = 0; b < nbin; ++b)
    if (cptr[size_t(b) + 1] - cptr[size_t(b)] == 1 && cvol[size_t(ccell[size_t(cptr[size_t(b)])])] >= (1.0 - 1e-9) * h * h * h)
      full[size_t(b)] = 1;
  // triangles: every cube that the triangle's bounding box (grown by 1e-9) meets
  const int64_t ntri = int64_t(C->tris.size() / 9);
  std::vector<int32_t> tptr(size_t(nbin) + 1, 0), ttri;
  auto tri_range = [&](int64_t t, int lo[3], int hi[3]) {
    for (int d = 0; d < 3; ++d) {
      double mn = C->tris[9 * size_t(t) + d], mx = mn;
      for (int v = 1; v < 3; ++v) {
        mn = std::min(mn, C->tris[9 * size_t(t) + 3 * v + d]);
        mx = std::max(mx, C->tris[9 * size_t(t) + 3 * v + d]);
      }
      lo[d] = host_cube(mn - 1e-9, N);
      hi[d] = host_cube(mx + 1e-9, N);
    }
  };
  for (int pass = 0; pass < 2; ++pass) {
    std::vector<int32_t> fill;
    if (pass == 1) {
      for (int64_t b = 0; b < nbin; ++b) tptr[size_t(b) + 1] += tptr[size_t(b)];
      ttri.assign(size_t(tptr.back()), 0);
      fill.assign(tptr.begin(), tptr.end() - 1);
    }
    for (int64_t t = 0; t < ntri; ++t) {
      int lo[3], hi[3];
      tri_range(t, lo, hi);
      for (int k = lo[2]; k <= hi[2]; ++k)
        for (int j = lo[1]; j <= hi[1]; ++j)
          for (int i = lo[0]; i <= hi[0]; ++i) {
            const size_t b = size_t((int64_t(k) * N + j) * N + i);
            if (pass == 0)
              ++tptr[b + 1];
            else
              ttri[size_t(fill[b]++)] = int32_t(t);
          }
    }
  }
  auto& P = C->pt;
  upload(P.cbin_ptr, cptr, s);
  upload(P.cbin_cell, ccell, s);
  upload(P.cbin_full, full, s);
  upload(P.fplane, plane, s);
  upload(P.tri, C->tris, s);
  upload(P.tbin_ptr, tptr, s);
  upload(P.tbin_tri, ttri, s);
  P.lin_old.alloc(sizeof(double) * 12 * size_t(std::max(1, M.nc)));
  P.count.alloc(sizeof(int32_t) * size_t(nbin + 1));
  P.tsum.alloc(sizeof(int32_t) * size_t((nbin + 1 + kScanTile - 1) / kScanTile));
  P.err.alloc(sizeof(int));
  CK(cudaStreamSynchronize(s));
  P.ready = true;
}

PartGridView part_view(const fvem_ctx* C) {
  const auto& P = C->pt;
  const DevLevel& L0 = *C->lv[0];
  return PartGridView{C->topo.N,
                      1.0 / C->topo.N,
                      P.cbin_ptr.as<int32_t>(),
                      P.cbin_cell.as<int32_t>(),
                      P.cbin_full.as<uint8_t>(),
                      P.fplane.as<double4>(),
                      L0.cell_fptr.as<int32_t>(),
                      P.tri.as<double>(),
                      P.tbin_ptr.as<int32_t>(),
                      P.tbin_tri.as<int32_t>()};
}

// Exclusive scan of C->pt.count (n = N^3 + 1 entries) in place.
void scan_counts(fvem_ctx* C, int64_t n) {
  cudaStream_t s = C->stream;
  const int64_t nt = (n + kScanTile - 1) / kScanTile;
  int32_t* cnt = C->pt.count.as<int32_t>();
  ++C->nlaunch, k_scan_tiles<<<unsigned(nt), 256, 0, s>>>(n, cnt, cnt, C->pt.tsum.as<int32_t>());
  ++C->nlaunch, k_scan_sums<<<1, 1024, 0, s>>>(nt, C->pt.tsum.as<int32_t>());
  ++C->nlaunch, k_scan_add<<<nblk(n), 256, 0, s>>>(n, cnt, C->pt.tsum.as<int32_t>());
}

fvem_status particle_args(fvem_ctx* C, int64_t np, const void* a, const void* b) {
  if (!C || !C->built) return fail(C, FVEM_EINVAL, "not built");
  if (np < 0 || np >= (int64_t(1) << 31)) return fail(C, FVEM_EINVAL, "particle count out of range");
  if (np > 0 && (!a || !b)) return fail(C, FVEM_EINVAL, "null pointer");
  return FVEM_OK;
}

}  // namespace

fvem_status fvem_p2g(fvem_ctx* C, int64_t np, const double* d_xp, const int32_t* d_cell, int nch, const double* d_fp,
                     double* d_fv) {
  fvem_status st = particle_args(C, np, d_xp, d_fp);
  if (st != FVEM_OK) return st;
  if (nch < 1 || nch > 4 || !d_fv) return fail(C, FVEM_EINVAL, "channels must be 1..4, output not null");
  API_BEGIN
  particles_setup(C);
  auto& P = C->pt;
  const int N = C->topo.N;
  const int64_t nbin = int64_t(N) * N * N;
  cudaStream_t s = C->stream;
  if (np > P.np_cap) {
    P.bin.alloc(sizeof(int32_t) * size_t(np));
    P.rank.alloc(sizeof(int32_t) * size_t(np));
    P.idx.alloc(sizeof(int32_t) * size_t(np));
    P.rpos.alloc(sizeof(float4) * size_t(np));
    P.rval.alloc(sizeof(float4) * size_t(np));
    P.np_cap = np;
  }
  CK(cudaMemsetAsync(P.count.p, 0, sizeof(int32_t) * size_t(nbin + 1), s));
  if (np > 0) {
    ++C->nlaunch, k_part_count<<<nblk(np), 256, 0, s>>>(np, d_xp, d_cell, N, P.count.as<int32_t>(), P.bin.as<int32_t>(),
                                                      P.rank.as<int32_t>());
  }
  scan_counts(C, nbin + 1);
  if (np > 0) {
    ++C->nlaunch, k_part_scatter<<<nblk(np), 256, 0, s>>>(np, P.bin.as<int32_t>(), P.rank.as<int32_t>(),
                                                        P.count.as<int32_t>(), P.idx.as<int32_t>());
    ++C->nlaunch, k_part_sort<<<nblk(nbin), 256, 0, s>>>(nbin, P.count.as<int32_t>(), P.idx.as<int32_t>());
    ++C->nlaunch, k_part_pack<<<nblk(np), 256, 0, s>>>(P.count.as<int32_t>() + nbin, P.idx.as<int32_t>(),
                                                     P.bin.as<int32_t>(), np, d_xp, d_fp, nch, N, 1.0 / N,
                                                     P.rpos.as<float4>(), P.rval.as<float4>());
  }
  const DevLevel& L0 = *C->lv[0];
  ++C->nlaunch, k_p2g<<<nblk(L0.nv), 256, 0, s>>>(L0.nv, L0.V.as<double>(), N, 1.0 / N, P.count.as<int32_t>(),
                                                 P.rpos.as<float4>(), P.rval.as<float4>(), nch, d_fv);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return FVEM_OK;
  API_END(C)
}

fvem_status fvem_locate(fvem_ctx* C, int64_t np, const double* d_xp, int32_t* d_cell) {
  fvem_status st = particle_args(C, np, d_xp, d_cell);
  if (st != FVEM_OK) return st;
  API_BEGIN
  particles_setup(C);
  if (np > 0) ++C->nlaunch, k_locate<<<nblk(np), 256, 0, C->stream>>>(np, d_xp, part_view(C), d_cell);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(C->stream));
  return FVEM_OK;
  API_END(C)
}

fvem_status fvem_g2p(fvem_ctx* C, int64_t np, const double* d_xp, const int32_t* d_cell, const double* d_u_old,
                     const double* d_cellpoly, double alpha, double* d_up) {
  fvem_status st = particle_args(C, np, d_xp, d_cell);
  if (st != FVEM_OK) return st;
  if (!d_u_old || !d_cellpoly || !d_up) return fail(C, FVEM_EINVAL, "null pointer");
  if (!(alpha >= 0.0 && alpha <= 1.0)) return fail(C, FVEM_EINVAL, "alpha_flip must be in [0, 1]");
  API_BEGIN
  particles_setup(C);
  const DevLevel& L0 = *C->lv[0];
  cudaStream_t s = C->stream;
  ++C->nlaunch, k_cell_linear<<<nblk(L0.nc, 128), 128, 0, s>>>(L0.mesh(), L0.Pis.as<double>(), d_u_old, L0.nv,
                                                               C->pt.lin_old.as<double>());
  if (np > 0)
    ++C->nlaunch, k_g2p<<<nblk(np), 256, 0, s>>>(np, d_xp, d_cell, L0.nc, L0.xE.as<double>(), L0.hE.as<double>(),
                                               C->pt.lin_old.as<double>(), d_cellpoly, alpha, d_up);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  return FVEM_OK;
  API_END(C)
}

fvem_status fvem_advect(fvem_ctx* C, int64_t np, double dt, const double* d_cellpoly, double* d_xp, int32_t* d_cell) {
  fvem_status st = particle_args(C, np, d_xp, d_cell);
  if (st != FVEM_OK) return st;
  if (!d_cellpoly) return fail(C, FVEM_EINVAL, "null pointer");
  if (!(dt >= 0.0 && std::isfinite(dt))) return fail(C, FVEM_EINVAL, "dt must be finite and >= 0");
  API_BEGIN
  particles_setup(C);
  const DevLevel& L0 = *C->lv[0];
  cudaStream_t s = C->stream;
  CK(cudaMemsetAsync(C->pt.err.p, 0, sizeof(int), s));
  if (np > 0)
    ++C->nlaunch, k_advect<<<nblk(np), 256, 0, s>>>(np, dt, d_cellpoly, L0.xE.as<double>(), L0.hE.as<double>(),
                                                  L0.nc, part_view(C), d_xp, d_cell, C->pt.err.as<int>());
  CK(cudaGetLastError());
  int e = 0;
  CK(cudaMemcpyAsync(&e, C->pt.err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (e) return fail(C, FVEM_EINVAL, "a particle's step spans more than 3 background cells; reduce dt");
  return FVEM_OK;
  API_END(C)
}

fvem_status fvem_arm_coarse_abort(fvem_ctx* C) {
  if (!C || !C->built) return fail(C, FVEM_EINVAL, "not built");
  if (!C->pst.ok || !(C->pst.use[0] || C->pst.use[1]))
    return fail(C, FVEM_EINVAL, "the coarsest-level CG does not use the persistent form");
  API_BEGIN
  CK(cudaMemsetAsync(C->pst.abort_.p, 1, sizeof(int), C->stream));
  CK(cudaStreamSynchronize(C->stream));
  return FVEM_OK;
  API_END(C)
}

fvem_status fvem_vcycle(fvem_ctx* C, const double* r, double* z) {
  if (!C || !C->built || !r || !z) return fail(C, FVEM_EINVAL, "not built or null pointer");
  API_BEGIN
  apply_precond(C, r, z);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(C->stream));
  if (C->pst.ok && (C->pst.use[0] || C->pst.use[1]) && coarse_timed_out(C)) {
    reset_persist(C);
    return fail(C, FVEM_ETIMEOUT, "a bounded wait of the persistent coarsest-level CG ran out");
  }
  return FVEM_OK;
  API_END(C)
}

fvem_status fvem_spmv(fvem_ctx* C, int l, const double* x, double* y) {
  if (!C || !C->built || l < 0 || l >= int(C->lv.size()) || !x || !y) return fail(C, FVEM_EINVAL, "bad arguments");
  API_BEGIN
  DevLevel& L = *C->lv[l];
  if (L.d16)
    ++C->nlaunch, k_spmv<double, 4, 1, true><<<sell_grid(L.sell<double>(), 1), 256, 0, C->stream>>>(L.sell<double>(), x, y);
  else
    ++C->nlaunch, k_spmv<double, 4, 1, false><<<sell_grid(L.sell<double>(), 1), 256, 0, C->stream>>>(L.sell<double>(), x, y);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(C->stream));
  return FVEM_OK;
  API_END(C)
}

fvem_status fvem_project(fvem_ctx* C, const double* d_u, double u_in, double* d_p, double* d_cell,
                         fvem_solve_stats* stats) {
  if (!C || !C->built || !d_u || !d_p || !d_cell) return fail(C, FVEM_EINVAL, "not built or null pointer");
  if (C->prm.order_k == 2 && u_in != 0.0) return fail(C, FVEM_EINVAL, "inflow is built for first-order VEM");
  if (!std::isfinite(u_in)) return fail(C, FVEM_ENAN, "non-finite inflow");
  API_BEGIN
  cudaStream_t s = C->stream;
  DevLevel& L0 = *C->lv[0];
  CK(cudaEventRecord(C->ev0, s));
  build_rhs(C, d_u, u_in);
  CK(cudaEventRecord(C->ev1, s));
  int it = 0;
  double rel = 0, r0n = 0;
  fvem_status st = pcg(C, C->cg_x.as<double>(), it, rel, r0n);
  CK(cudaEventRecord(C->ev2, s));
  issue_finish(C, d_u, d_p, d_cell);
  CK(cudaGetLastError());
  CK(cudaEventRecord(C->ev3, s));
  CK(cudaEventSynchronize(C->ev3));
  if (stats) {
    float a = 0, b = 0;
    cudaEventElapsedTime(&a, C->ev1, C->ev2);
    cudaEventElapsedTime(&b, C->ev0, C->ev3);
    stats->iters = it;
    stats->rel_res = rel;
    stats->r0_norm = r0n;
    stats->solve_ms = a;
    stats->total_ms = b;
  }
  if (st != FVEM_OK)
    return fail(C, st,
                (st == FVEM_EBREAKDOWN || st == FVEM_ETIMEOUT) ? C->err : std::string("solve did not converge cleanly"));
  return FVEM_OK;
  API_END(C)
}

fvem_status fvem_project_batched(fvem_ctx* const* ctxs, int n, const double* const* d_u, const double* u_in,
                                 double* const* d_p, double* const* d_cell, fvem_solve_stats* stats) {
  if (!ctxs || n < 1 || !d_u || !d_p || !d_cell) return FVEM_EINVAL;
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i] || !ctxs[i]->built || !d_u[i] || !d_p[i] || !d_cell[i]) return FVEM_EINVAL;
    if (u_in && !std::isfinite(u_in[i])) return fail(ctxs[i], FVEM_ENAN, "non-finite inflow");
    for (int j = 0; j < i; ++j)
      if (ctxs[j] == ctxs[i]) return fail(ctxs[i], FVEM_EINVAL, "a context appears twice in the batch");
  }
  fvem_ctx* C0 = ctxs[0];
  API_BEGIN
  std::vector<PcgRun> runs(n);
  for (int i = 0; i < n; ++i) {
    fvem_ctx* C = ctxs[i];
    CK(cudaEventRecord(C->ev0, C->stream));
    build_rhs(C, d_u[i], u_in ? u_in[i] : 0.0);
    CK(cudaEventRecord(C->ev1, C->stream));
    runs[i].C = C;
    runs[i].x = C->cg_x.as<double>();
  }
  if (!pcg_batch_graph(runs)) pcg_batch(runs);
  for (int i = 0; i < n; ++i) {
    fvem_ctx* C = ctxs[i];
    DevLevel& L0 = *C->lv[0];
    cudaStream_t s = C->stream;
    CK(cudaEventRecord(C->ev2, s));
    issue_finish(C, d_u[i], d_p[i], d_cell[i]);
    CK(cudaGetLastError());
    CK(cudaEventRecord(C->ev3, s));
  }
  fvem_status worst = FVEM_OK;
  for (int i = 0; i < n; ++i) {
    fvem_ctx* C = ctxs[i];
    CK(cudaEventSynchronize(C->ev3));
    if (stats) {
      float a = 0, b = 0;
      cudaEventElapsedTime(&a, C->ev1, C->ev2);
      cudaEventElapsedTime(&b, C->ev0, C->ev3);
      stats[i].iters = runs[i].iters;
      stats[i].rel_res = runs[i].relres;
      stats[i].r0_norm = runs[i].r0n;
      stats[i].solve_ms = a;
      stats[i].total_ms = b;
    }
    if (runs[i].st != FVEM_OK) {
      if (runs[i].st != FVEM_EBREAKDOWN) C->err = "solve did not converge cleanly";
      if (worst == FVEM_OK) worst = runs[i].st;
    }
  }
  return worst;
  API_END(C0)
}

fvem_status fvem_project_host(fvem_ctx* C, const double* h_u, double u_in, double* h_p, double* h_cell,
                              fvem_solve_stats* stats) {
  if (!C || !C->built || !h_u) return fail(C, FVEM_EINVAL, "not built or null pointer");
  fvem_status st;
  API_BEGIN
  DevLevel& L0 = *C->lv[0];
  cudaStream_t s = C->stream;
  const size_t np = size_t(pressure_len(C));
  if (C->u_tmp.bytes < sizeof(double) * 3 * size_t(L0.nv)) C->u_tmp.alloc(sizeof(double) * 3 * size_t(L0.nv));
  if (C->gcell_tmp.bytes < sizeof(double) * 12 * size_t(L0.nc)) C->gcell_tmp.alloc(sizeof(double) * 12 * size_t(L0.nc));
  if (C->pfull.bytes < sizeof(double) * np) C->pfull.alloc(sizeof(double) * np);
  CK(cudaMemcpyAsync(C->u_tmp.p, h_u, sizeof(double) * 3 * L0.nv, cudaMemcpyHostToDevice, s));
  st = fvem_project(C, C->u_tmp.as<double>(), u_in, C->pfull.as<double>(), C->gcell_tmp.as<double>(), stats);
  if (h_p) CK(cudaMemcpyAsync(h_p, C->pfull.p, sizeof(double) * np, cudaMemcpyDeviceToHost, s));
  if (h_cell) CK(cudaMemcpyAsync(h_cell, C->gcell_tmp.p, sizeof(double) * 12 * L0.nc, cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  return st;
  API_END(C)
}

fvem_status fvem_project_adjoint(fvem_ctx* C, const double* d_g, double* d_gu, double* h_gin, fvem_solve_stats* stats) {
  if (!C || !C->built || !d_g || !d_gu) return fail(C, FVEM_EINVAL, "not built or null pointer");
  if (C->prm.order_k != 1) return fail(C, FVEM_EINVAL, "the adjoint is built for first-order VEM");
  API_BEGIN
  cudaStream_t s = C->stream;
  DevLevel& L0 = *C->lv[0];
  // lambda_rhs = (d cellpoly / d p)^T g on free DOFs
  ++C->nlaunch, k_adj_pcoef<<<nblk(L0.nc, 128), 128, 0, s>>>(L0.mesh(), L0.Pis.as<double>(), L0.hE.as<double>(), d_g,
                                               C->rloc.as<double>());
  ++C->nlaunch, k_gather_dofs<<<nblk(L0.ndof), 256, 0, s>>>(L0.ndof, L0.vertex_of_dof.as<int32_t>(), L0.inc_ptr.as<int32_t>(),
                                              L0.inc_cell.as<int32_t>(), L0.inc_loc.as<int32_t>(),
                                              L0.cell_vptr.as<int32_t>(), C->rloc.as<double>(), C->cg_r.as<double>());
  // keep the adjoint RHS for the inflow gradient: b_in . lambda
  int it = 0;
  double rel = 0, r0n = 0;
  CK(cudaEventRecord(C->ev1, s));
  fvem_status st = pcg(C, C->cg_x.as<double>(), it, rel, r0n);
  CK(cudaEventRecord(C->ev2, s));
  ++C->nlaunch, k_expand<<<nblk(L0.nv), 256, 0, s>>>(L0.nv, L0.dof_of_vertex.as<int32_t>(), C->cg_x.as<double>(),
                                       C->pfull.as<double>());
  int64_t nloc = int64_t(C->topo.levels[0].cell_v.size());
  ++C->nlaunch, k_adj_u<<<nblk(L0.nc, 128), 128, 0, s>>>(L0.mesh(), L0.Pis.as<double>(), L0.vol.as<double>(), L0.hE.as<double>(),
                                           d_g, C->pfull.as<double>(), C->rloc3.as<double>(), nloc);
  for (int c = 0; c < 3; ++c)
    ++C->nlaunch, k_gather_dofs<<<nblk(L0.nv), 256, 0, s>>>(L0.nv, nullptr, L0.inc_ptr.as<int32_t>(), L0.inc_cell.as<int32_t>(),
                                             L0.inc_loc.as<int32_t>(), L0.cell_vptr.as<int32_t>(),
                                             C->rloc3.as<double>() + c * nloc, d_gu + size_t(c) * L0.nv);
  if (h_gin) {
    // inflow gradient = b_in . lambda with b_in = d r / d u_in (RHS of zero velocity, unit inflow)
    if (C->u_tmp.bytes < sizeof(double) * 3 * size_t(L0.nv)) C->u_tmp.alloc(sizeof(double) * 3 * size_t(L0.nv));
    CK(cudaMemsetAsync(C->u_tmp.p, 0, sizeof(double) * 3 * L0.nv, s));
    build_rhs(C, C->u_tmp.as<double>(), 1.0);
    double* part = C->part.as<double>();
    ++C->nlaunch, k_dot2<<<RED_BLOCKS, RED_THREADS, 0, s>>>(L0.ndof, C->cg_r.as<double>(), C->cg_x.as<double>(), nullptr, part);
    ++C->nlaunch, k_finalize<<<1, 256, 0, s>>>(part, RED_BLOCKS, 1, C->scal.as<double>() + 8);
    CK(cudaMemcpyAsync(C->h_sc + 8, C->scal.as<double>() + 8, sizeof(double), cudaMemcpyDeviceToHost, s));
  }
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(s));
  if (h_gin) *h_gin = C->h_sc[8];
  if (stats) {
    float a = 0;
    cudaEventElapsedTime(&a, C->ev1, C->ev2);
    stats->iters = it;
    stats->rel_res = rel;
    stats->r0_norm = r0n;
    stats->solve_ms = a;
    stats->total_ms = a;
  }
  if (st != FVEM_OK) return fail(C, st, "adjoint solve did not converge cleanly");
  return FVEM_OK;
  API_END(C)
}

fvem_status fvem_set_profiling(fvem_ctx* C, int on) {
  if (!C || !C->built) return fail(C, FVEM_EINVAL, "not built");
  API_BEGIN
  prof_flush(C);
  CK(cudaStreamSynchronize(C->stream));
  collect_graph_prof(C);
  C->prof = on != 0;
  C->prof_ms = 0.0;
  C->prof_launches = 0;
  return FVEM_OK;
  API_END(C)
}

fvem_status fvem_set_precision(fvem_ctx* C, int precision) {
  if (!C || !C->built) return fail(C, FVEM_EINVAL, "not built");
  const bool want16 = precision == FVEM_PREC_BF16 || precision == FVEM_PREC_FP16;
  if (precision == FVEM_PREC_FP64 || (precision == FVEM_PREC_FP32 && C->fp32_capable) ||
      (want16 && C->bf16_capable)) {
    API_BEGIN
    if (want16 && C->v16_half != (precision == FVEM_PREC_FP16)) {
      // the other 16-bit format: re-pack every plane from the FP32 copy
      C->v16_half = precision == FVEM_PREC_FP16;
      for (auto& L : C->lv)
        if (L->sell_valb.p)
          ++C->nlaunch, k_pack16<<<RED_BLOCKS, 256, 0, C->stream>>>(int64_t(L->sell_val32.bytes / sizeof(float)),
                                                                      L->sell_val32.as<float>(), L->sell_valb.p,
                                                                      C->v16_half ? 1 : 0);
      CK(cudaGetLastError());
      CK(cudaStreamSynchronize(C->stream));
    }
    if (C->prm.precision != precision) ++C->gen;
    C->prm.precision = precision;
    set_bf16_flags(C);
    return FVEM_OK;
    API_END(C)
  }
  return fail(C, FVEM_EINVAL, "precision not available in this context");
}

fvem_status fvem_set_tolerance(fvem_ctx* C, double rel_tol, int max_iters) {
  if (!C || !(rel_tol > 0) || max_iters < 1) return fail(C, FVEM_EINVAL, "bad tolerance");
  if (C->prm.rel_tol != rel_tol || C->prm.max_iters != max_iters) ++C->gen;  // baked into the PCG graph
  C->prm.rel_tol = rel_tol;
  C->prm.max_iters = max_iters;
  return FVEM_OK;
}

fvem_status fvem_set_graphs(fvem_ctx* C, int on) {
  if (!C) return FVEM_EINVAL;
  destroy_vgraph(C);
  C->use_graph = on != 0;
  return FVEM_OK;
}

fvem_status fvem_set_cheb_lmax(fvem_ctx* C, int level, double lmax) {
  if (!C || !C->built || level < 0 || level >= int(C->lv.size()) || !(lmax > 0.0) || !std::isfinite(lmax))
    return fail(C, FVEM_EINVAL, "bad level or bound");
  C->lv[level]->lmax = lmax;
  destroy_vgraph(C);  // the captured V-cycle holds the old coefficients
  return FVEM_OK;
}

fvem_status fvem_set_stencil(fvem_ctx* C, int level, int on) {
  if (!C || !C->built || level < 0 || level >= int(C->lv.size())) return fail(C, FVEM_EINVAL, "bad level");
  DevLevel& L = *C->lv[level];
  if (on && L.nreg32 == 0) return fail(C, FVEM_EINVAL, "level has no stencil slices in an FP32 copy");
  L.stc_on = on != 0;
  destroy_vgraph(C);
  return FVEM_OK;
}

fvem_status fvem_launch_count(const fvem_ctx* C, int64_t* n) {
  if (!C || !n) return FVEM_EINVAL;
  *n = C->nlaunch;
  return FVEM_OK;
}

fvem_status fvem_get_profile(fvem_ctx* C, int64_t* launches, double* total_ms, double* bytes_per_launch) {
  if (!C || !C->built) return fail(C, FVEM_EINVAL, "not built");
  API_BEGIN
  prof_flush(C);
  CK(cudaStreamSynchronize(C->stream));
  collect_graph_prof(C);
  const DevLevel& L = *C->lv[0];
  // value and vector bytes of the level-0 step in the current precision
  const double sx = C->prm.precision == FVEM_PREC_FP64 ? 8.0 : 4.0;
  const double sv = C->prm.precision == FVEM_PREC_FP64
                        ? 8.0
                        : ((C->prm.precision == FVEM_PREC_BF16 || C->prm.precision == FVEM_PREC_FP16) ? 2.0 : 4.0);
  if (launches) *launches = C->prof_launches;
  if (total_ms) *total_ms = C->prof_ms;
  const double si = L.d16 ? 2.0 : 4.0;  // stored column index width
  // stencil slices read no values and no column offsets: eight 16-bit line
  // offsets and a class byte per row
  const bool f32 = C->prm.precision != FVEM_PREC_FP64;
  const bool use = f32 && L.stc_on;
  const double snnz = double(use ? L.stc_nnz32 : 0), srows = double(use ? L.nreg32 * 32 : 0);
  if (bytes_per_launch)
    *bytes_per_launch = (double(L.nnz) - snnz) * (sv + si) + srows * 17.0 + 6.0 * sx * double(L.ndof);
  return FVEM_OK;
  API_END(C)
}

const char* fvem_status_str(fvem_status s) {
  switch (s) {
    case FVEM_OK: return "ok";
    case FVEM_EINVAL: return "invalid argument";
    case FVEM_ENOMEM: return "out of memory";
    case FVEM_EGEOM: return "degenerate geometry or topology";
    case FVEM_ENOCONV: return "no convergence";
    case FVEM_EBREAKDOWN: return "CG breakdown";
    case FVEM_ENAN: return "NaN or Inf";
    case FVEM_ECUDA: return "CUDA error";
    case FVEM_ENODEV: return "no CUDA device";
    case FVEM_ETIMEOUT: return "timeout in a persistent kernel";
  }
  return "unknown";
}

const char* fvem_last_error(const fvem_ctx* C) { return C ? C->err.c_str() : "null context"; }

}  // extern "C"

// ------------------------------------------------------------------ V-cycle without allocation
//
// fvem_vcycle_static: the FP64 V-cycle of fvem_vcycle with its work vectors
// in a file-scope device array instead of context buffers, for callers that
// must not allocate device memory after set-up (for example code running
// under a memory pool or budget that forbids cudaMalloc, or a host that
// pre-plans every allocation).  The array holds kStaticScratchDoubles doubles
// (16 MiB) on every device that loads this library, until the process exits.
namespace {

constexpr size_t kStaticScratchDoubles = size_t(1) << 21;
__device__ __align__(256) double g_static_scratch[kStaticScratchDoubles];
constexpr int kMaxDevices = 64;
double* g_static_ptr[kMaxDevices] = {nullptr};

// Device address of the static array for the current device (looked up once
// per device; in host code the symbol itself is only a host-side stand-in).
double* static_scratch(std::string& err) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    err = "no current CUDA device";
    return nullptr;
  }
  if (!g_static_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) {
      err = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
      return nullptr;
    }
    g_static_ptr[dev] = static_cast<double*>(p);
  }
  return g_static_ptr[dev];
}

}  // namespace

extern "C" fvem_status fvem_vcycle_static(fvem_ctx* C, const double* r, double* z) {
  if (!C || !C->built || !r || !z) return fail(C, FVEM_EINVAL, "not built or null pointer");
  if (C->prm.order_k != 1) return fail(C, FVEM_EINVAL, "the allocation-free V-cycle serves first-order VEM");
  size_t need = 4 * size_t(std::max(C->coop_blocks_f64, C->coop_blocks_f32)) +
                size_t(std::max(1, C->lv.back()->ndof));
  for (auto& L : C->lv) need += 5 * size_t(std::max(1, L->ndof));
  if (need > kStaticScratchDoubles)
    return fail(C, FVEM_EINVAL,
                "hierarchy needs " + std::to_string(need) + " scratch doubles; the static V-cycle holds at most " +
                    std::to_string(kStaticScratchDoubles));
  API_BEGIN
  std::string err;
  double* base = static_scratch(err);
  if (!base) return fail(C, FVEM_ECUDA, err);
  std::vector<LVecs<double>> vs;
  size_t off = 0;
  for (auto& L : C->lv) {
    size_t n = size_t(std::max(1, L->ndof));
    vs.push_back(LVecs<double>{base + off, base + off + n, base + off + 2 * n, base + off + 3 * n, base + off + 4 * n});
    off += 5 * n;
  }
  // every vector and reduction slot is written before it is read, so nothing
  // needs clearing; w and the slots are locals of this call (no shared host state)
  double* w = base + off;
  off += size_t(std::max(1, C->lv.back()->ndof));
  vcycle<double>(C, 0, r, vs.data(), base + off, w);
  CK(cudaMemcpyAsync(z, vs[0].x, sizeof(double) * C->lv[0]->ndof, cudaMemcpyDeviceToDevice, C->stream));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(C->stream));
  if (C->pst.ok && (C->pst.use[0] || C->pst.use[1]) && coarse_timed_out(C)) {
    reset_persist(C);
    return fail(C, FVEM_ETIMEOUT, "a bounded wait of the persistent coarsest-level CG ran out");
  }
  return FVEM_OK;
  API_END(C)
}
