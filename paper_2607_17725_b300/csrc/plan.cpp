// Host construction of the integer solver plan (see plan.h).
//
// Free DOFs (per level): vertices not on the Dirichlet face y = 1 (|y-1| <=
// 1e-10), and on coarse levels only vertices that some prolongation row uses
// (a coarse DOF with an empty P column is removed).  Free indices follow the
// canonical vertex order.  The pattern of A_l is the union of the cliques of
// the level's element lists over free DOFs (structural; numeric zeros are
// kept), which holds every entry of the Galerkin operator P^T A P.
#include "plan.h"

#include <algorithm>
#include <cmath>
#include <map>

namespace fvem {

static void build_sell(LevelPlan& L) {
  int64_t n = L.ndof;
  L.nslices = (n + SELL_C - 1) / SELL_C;
  L.sell_ptr.assign(L.nslices + 1, 0);
  L.sell_w.assign(L.nslices, 0);
  for (int64_t s = 0; s < L.nslices; ++s) {
    int w = 0;
    for (int64_t r = s * SELL_C; r < std::min<int64_t>(n, (s + 1) * SELL_C); ++r)
      w = std::max<int>(w, int(L.a_rowptr[r + 1] - L.a_rowptr[r]));
    L.sell_w[s] = w;
    L.sell_ptr[s + 1] = L.sell_ptr[s] + int64_t(w) * SELL_C;
  }
  L.sell_col.assign(L.sell_ptr[L.nslices], 0);
  L.sell_of_csr.assign(L.a_rowptr[n], 0);
  for (int64_t s = 0; s < L.nslices; ++s)
    for (int lane = 0; lane < SELL_C; ++lane) {
      int64_t r = s * SELL_C + lane;
      int64_t len = r < n ? L.a_rowptr[r + 1] - L.a_rowptr[r] : 0;
      int32_t pad = r < n ? int32_t(r) : 0;
      for (int j = 0; j < L.sell_w[s]; ++j) {
        int64_t slot = L.sell_ptr[s] + int64_t(j) * SELL_C + lane;
        if (j < len) {
          L.sell_col[slot] = L.a_col[L.a_rowptr[r] + j];
          L.sell_of_csr[L.a_rowptr[r] + j] = slot;
        } else {
          L.sell_col[slot] = pad;
        }
      }
    }
  // 16-bit offsets when every stored column is within +-32767 of its row
  bool fits = true;
  for (int64_t r = 0; r < n && fits; ++r)
    for (int64_t k = L.a_rowptr[r]; k < L.a_rowptr[r + 1]; ++k) {
      int64_t d = int64_t(L.a_col[k]) - r;
      if (d < -32767 || d > 32767) {
        fits = false;
        break;
      }
    }
  L.sell_d16 = fits && n > 0;
  if (L.sell_d16) {
    L.sell_dcol.assign(L.sell_col.size(), 0);
    for (int64_t s = 0; s < L.nslices; ++s)
      for (int lane = 0; lane < SELL_C; ++lane) {
        int64_t r = s * SELL_C + lane;
        for (int j = 0; j < L.sell_w[s]; ++j) {
          int64_t slot = L.sell_ptr[s] + int64_t(j) * SELL_C + lane;
          // rows past the end gather row n-1 (offset -31..-1), others their own column
          int64_t d = r < n ? int64_t(L.sell_col[slot]) - r : (n - 1) - r;
          L.sell_dcol[slot] = int16_t(d);
        }
      }
    L.sell_col.clear();
    L.sell_col.shrink_to_fit();
  }
}

int build_plan(const Topology& T, std::vector<LevelPlan>& plan, std::string& err) {
  int Lv = T.L;
  plan.assign(Lv, LevelPlan());
  // prolongation row patterns (full, over all vertices) for l -> l+1
  for (int l = 0; l + 1 < Lv; ++l) {
    const LevelMesh& F = T.levels[l];
    const LevelMesh& C = T.levels[l + 1];
    const Placement& pl = T.place[l];
    LevelPlan& P = plan[l];
    P.prow_ptr.assign(F.nv + 1, 0);
    P.prow_col.clear();
    for (int v = 0; v < F.nv; ++v) {
      switch (pl.type[v]) {
        case PLACE_VERTEX: P.prow_col.push_back(pl.a[v]); break;
        case PLACE_EDGE:
          P.prow_col.push_back(pl.a[v]);
          P.prow_col.push_back(pl.b[v]);
          break;
        case PLACE_FACE:
          for (int q = C.face_vptr[pl.a[v]]; q < C.face_vptr[pl.a[v] + 1]; ++q) P.prow_col.push_back(C.face_v[q]);
          break;
        default:
          for (int q = C.cell_vptr[pl.cell[v]]; q < C.cell_vptr[pl.cell[v] + 1]; ++q) P.prow_col.push_back(C.cell_v[q]);
      }
      P.prow_ptr[v + 1] = int32_t(P.prow_col.size());
    }
  }
  // children lists of coarse cells
  for (int l = 1; l < Lv; ++l) {
    const LevelMesh& F = T.levels[l - 1];
    LevelPlan& P = plan[l];
    P.nc = T.levels[l].nc;
    P.child_ptr.assign(P.nc + 1, 0);
    for (int c = 0; c < F.nc; ++c) P.child_ptr[F.parent[c] + 1]++;
    for (int c = 0; c < P.nc; ++c) P.child_ptr[c + 1] += P.child_ptr[c];
    P.child_cell.assign(F.nc, 0);
    std::vector<int32_t> fill(P.child_ptr.begin(), P.child_ptr.end() - 1);
    for (int c = 0; c < F.nc; ++c) P.child_cell[fill[F.parent[c]]++] = c;
  }
  // element vertex lists
  for (int l = 0; l < Lv; ++l) {
    const LevelMesh& M = T.levels[l];
    LevelPlan& P = plan[l];
    P.elem_vptr = M.cell_vptr;
    P.elem_v = M.cell_v;
    P.elem_is_cell = true;
    if (l == 0) continue;
    const LevelPlan& F = plan[l - 1];
    std::vector<int32_t> ev;
    std::vector<int32_t> nvp(1, 0), nv;
    for (int c = 0; c < M.nc; ++c) {
      ev.assign(M.cell_v.begin() + M.cell_vptr[c], M.cell_v.begin() + M.cell_vptr[c + 1]);
      const size_t own = ev.size();
      for (int q = P.child_ptr[c]; q < P.child_ptr[c + 1]; ++q) {
        const int e = P.child_cell[q];
        for (int u = F.elem_vptr[e]; u < F.elem_vptr[e + 1]; ++u) {
          const int fvx = F.elem_v[u];
          for (int r = F.prow_ptr[fvx]; r < F.prow_ptr[fvx + 1]; ++r) ev.push_back(F.prow_col[r]);
        }
      }
      std::sort(ev.begin(), ev.end());
      ev.erase(std::unique(ev.begin(), ev.end()), ev.end());
      if (ev.size() != own) P.elem_is_cell = false;
      nv.insert(nv.end(), ev.begin(), ev.end());
      nvp.push_back(int32_t(nv.size()));
    }
    if (!P.elem_is_cell) {
      P.elem_vptr.swap(nvp);
      P.elem_v.swap(nv);
    }
  }
  // free DOFs
  for (int l = 0; l < Lv; ++l) {
    const LevelMesh& M = T.levels[l];
    LevelPlan& P = plan[l];
    P.nv = M.nv;
    P.nc = M.nc;
    std::vector<char> used(M.nv, l == 0 ? 1 : 0);
    if (l > 0)
      for (int32_t c : plan[l - 1].prow_col) used[c] = 1;
    P.dof_of_vertex.assign(M.nv, -1);
    P.vertex_of_dof.clear();
    for (int v = 0; v < M.nv; ++v) {
      bool dir = std::fabs(M.V[3 * v + 1] - 1.0) <= 1e-10;
      if (used[v] && !dir) {
        P.dof_of_vertex[v] = int32_t(P.vertex_of_dof.size());
        P.vertex_of_dof.push_back(v);
      }
    }
    P.ndof = int(P.vertex_of_dof.size());
    if (P.ndof == 0) {
      err = "level " + std::to_string(l) + " has no free DOF";
      return 1;
    }
    // element block offsets, incidence lists, size maxima
    P.kptr.assign(M.nc + 1, 0);
    std::vector<int32_t> cnt(M.nv + 1, 0);
    for (int c = 0; c < M.nc; ++c) {
      int n = P.elem_vptr[c + 1] - P.elem_vptr[c];
      P.kptr[c + 1] = P.kptr[c] + int64_t(n) * n;
      P.max_nv = std::max(P.max_nv, M.cell_vptr[c + 1] - M.cell_vptr[c]);
      P.max_ne = std::max(P.max_ne, n);
      P.max_nf = std::max(P.max_nf, M.cell_fptr[c + 1] - M.cell_fptr[c]);
      for (int q = P.elem_vptr[c]; q < P.elem_vptr[c + 1]; ++q) cnt[P.elem_v[q] + 1]++;
    }
    P.inc_ptr.assign(M.nv + 1, 0);
    for (int v = 0; v < M.nv; ++v) P.inc_ptr[v + 1] = P.inc_ptr[v] + cnt[v + 1];
    P.inc_cell.assign(P.inc_ptr[M.nv], 0);
    P.inc_loc.assign(P.inc_ptr[M.nv], 0);
    std::vector<int32_t> fill(P.inc_ptr.begin(), P.inc_ptr.end() - 1);
    for (int c = 0; c < M.nc; ++c)
      for (int q = P.elem_vptr[c]; q < P.elem_vptr[c + 1]; ++q) {
        int v = P.elem_v[q];
        P.inc_cell[fill[v]] = c;
        P.inc_loc[fill[v]] = q - P.elem_vptr[c];
        fill[v]++;
      }
    for (int f = 0; f < int(M.face_pid.size()); ++f)
      if (M.face_pid[f] == 0 && M.face_sg[f] < 0) P.has_inflow = true;
    // pattern: clique union over free DOFs
    P.a_rowptr.assign(P.ndof + 1, 0);
    P.a_col.clear();
    std::vector<int32_t> cols;
    for (int i = 0; i < P.ndof; ++i) {
      int v = P.vertex_of_dof[i];
      cols.clear();
      for (int q = P.inc_ptr[v]; q < P.inc_ptr[v + 1]; ++q) {
        int c = P.inc_cell[q];
        for (int u = P.elem_vptr[c]; u < P.elem_vptr[c + 1]; ++u) {
          int j = P.dof_of_vertex[P.elem_v[u]];
          if (j >= 0) cols.push_back(j);
        }
      }
      std::sort(cols.begin(), cols.end());
      cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
      P.a_col.insert(P.a_col.end(), cols.begin(), cols.end());
      P.a_rowptr[i + 1] = int64_t(P.a_col.size());
    }
    if (P.a_rowptr[P.ndof] >= (int64_t(1) << 31)) {
      err = "too many nonzeros for 32-bit slot indices";
      return 1;
    }
    build_sell(P);
  }
  // free prolongation P (rows: free DOFs of l, cols: free DOFs of l+1) and P^T
  for (int l = 0; l + 1 < Lv; ++l) {
    LevelPlan& P = plan[l];
    const LevelPlan& Cp = plan[l + 1];
    P.pf_rowptr.assign(P.ndof + 1, 0);
    P.pf_col.clear();
    P.pf_src.clear();
    for (int i = 0; i < P.ndof; ++i) {
      int v = P.vertex_of_dof[i];
      for (int q = P.prow_ptr[v]; q < P.prow_ptr[v + 1]; ++q) {
        int j = Cp.dof_of_vertex[P.prow_col[q]];
        if (j < 0) continue;
        P.pf_col.push_back(j);
        P.pf_src.push_back(q);
      }
      P.pf_rowptr[i + 1] = int64_t(P.pf_col.size());
    }
    int nc = Cp.ndof;
    P.pt_rowptr.assign(nc + 1, 0);
    for (int32_t j : P.pf_col) P.pt_rowptr[j + 1]++;
    for (int j = 0; j < nc; ++j) P.pt_rowptr[j + 1] += P.pt_rowptr[j];
    P.pt_col.assign(P.pf_col.size(), 0);
    P.pt_src.assign(P.pf_col.size(), 0);
    std::vector<int64_t> fill(P.pt_rowptr.begin(), P.pt_rowptr.end() - 1);
    for (int i = 0; i < P.ndof; ++i)
      for (int64_t k = P.pf_rowptr[i]; k < P.pf_rowptr[i + 1]; ++k) {
        int j = P.pf_col[k];
        P.pt_col[fill[j]] = i;
        P.pt_src[fill[j]] = k;
        fill[j]++;
      }
  }
  return 0;
}

void build_dofs_k2(const LevelMesh& M, DofsK2& D) {
  const int64_t nv = M.nv, nc = M.nc;
  // edges and faces of every cell face occurrence
  std::vector<std::pair<int32_t, int32_t>> edges;
  std::vector<std::vector<int32_t>> fkeys;
  for (int c = 0; c < nc; ++c)
    for (int f = M.cell_fptr[c]; f < M.cell_fptr[c + 1]; ++f) {
      const int32_t b = M.face_vptr[f], e = M.face_vptr[f + 1];
      std::vector<int32_t> key(M.face_v.begin() + b, M.face_v.begin() + e);
      for (int32_t q = b; q < e; ++q) {
        const int32_t u = M.face_v[q], w = M.face_v[q + 1 < e ? q + 1 : b];
        edges.emplace_back(std::min(u, w), std::max(u, w));
      }
      std::sort(key.begin(), key.end());
      fkeys.push_back(std::move(key));
    }
  std::sort(edges.begin(), edges.end());
  edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
  std::vector<std::vector<int32_t>> fsorted = fkeys;
  std::sort(fsorted.begin(), fsorted.end());
  fsorted.erase(std::unique(fsorted.begin(), fsorted.end()), fsorted.end());
  D.nv = nv;
  D.ne = int64_t(edges.size());
  D.nf = int64_t(fsorted.size());
  D.nc = nc;
  D.n = nv + D.ne + D.nf + nc;
  auto edge_dof = [&](int32_t u, int32_t w) {
    const std::pair<int32_t, int32_t> k(std::min(u, w), std::max(u, w));
    return nv + int64_t(std::lower_bound(edges.begin(), edges.end(), k) - edges.begin());
  };
  auto face_dof = [&](const std::vector<int32_t>& key) {
    return nv + D.ne + int64_t(std::lower_bound(fsorted.begin(), fsorted.end(), key) - fsorted.begin());
  };
  D.elem_ptr.assign(1, 0);
  D.elem_dof.clear();
  size_t occ = 0;
  for (int c = 0; c < nc; ++c) {
    std::vector<int32_t> vs(M.cell_v.begin() + M.cell_vptr[c], M.cell_v.begin() + M.cell_vptr[c + 1]);
    std::vector<std::pair<int32_t, int32_t>> es;
    for (int f = M.cell_fptr[c]; f < M.cell_fptr[c + 1]; ++f) {
      const int32_t b = M.face_vptr[f], e = M.face_vptr[f + 1];
      for (int32_t q = b; q < e; ++q) {
        const int32_t u = M.face_v[q], w = M.face_v[q + 1 < e ? q + 1 : b];
        es.emplace_back(std::min(u, w), std::max(u, w));
      }
    }
    std::sort(es.begin(), es.end());
    es.erase(std::unique(es.begin(), es.end()), es.end());
    for (int32_t v : vs) D.elem_dof.push_back(v);
    for (auto& pr : es) D.elem_dof.push_back(edge_dof(pr.first, pr.second));
    for (int f = M.cell_fptr[c]; f < M.cell_fptr[c + 1]; ++f) D.elem_dof.push_back(face_dof(fkeys[occ++]));
    D.elem_dof.push_back(nv + D.ne + D.nf + c);
    D.elem_ptr.push_back(int64_t(D.elem_dof.size()));
  }
  std::vector<uint8_t> on(size_t(nv), 0);
  for (int64_t v = 0; v < nv; ++v) on[size_t(v)] = std::fabs(M.V[3 * v + 1] - 1.0) <= 1e-10 ? 1 : 0;
  D.dirichlet.assign(size_t(D.n), 0);
  for (int64_t v = 0; v < nv; ++v) D.dirichlet[size_t(v)] = on[size_t(v)];
  for (size_t i = 0; i < edges.size(); ++i)
    D.dirichlet[size_t(nv) + i] = on[size_t(edges[i].first)] && on[size_t(edges[i].second)];
  for (size_t i = 0; i < fsorted.size(); ++i) {
    bool all = true;
    for (int32_t v : fsorted[i]) all = all && on[size_t(v)];
    D.dirichlet[size_t(nv + D.ne) + i] = all ? 1 : 0;
  }
  // free numbering and the clique-union pattern over free DOFs
  D.free_of.assign(size_t(D.n), -1);
  int64_t nfree = 0;
  for (int64_t i = 0; i < D.n; ++i)
    if (!D.dirichlet[size_t(i)]) D.free_of[size_t(i)] = nfree++;
  std::vector<std::vector<int64_t>> rows(static_cast<size_t>(nfree));
  for (int64_t c = 0; c < nc; ++c)
    for (int64_t a = D.elem_ptr[c]; a < D.elem_ptr[c + 1]; ++a) {
      const int64_t ra = D.free_of[size_t(D.elem_dof[size_t(a)])];
      if (ra < 0) continue;
      for (int64_t b = D.elem_ptr[c]; b < D.elem_ptr[c + 1]; ++b) {
        const int64_t cb = D.free_of[size_t(D.elem_dof[size_t(b)])];
        if (cb >= 0) rows[size_t(ra)].push_back(cb);
      }
    }
  D.a_rowptr.assign(1, 0);
  D.a_col.clear();
  for (auto& r : rows) {
    std::sort(r.begin(), r.end());
    r.erase(std::unique(r.begin(), r.end()), r.end());
    D.a_col.insert(D.a_col.end(), r.begin(), r.end());
    D.a_rowptr.push_back(int64_t(D.a_col.size()));
  }
}

void build_prolongation_pattern_k2(const LevelMesh& F, const LevelMesh& Cm, const DofsK2& Df, const DofsK2& Dc,
                                   std::vector<int64_t>& rowptr, std::vector<int64_t>& col, bool naive) {
  // coarse lookups: edge -> DOF, sorted face key -> DOF (from the element lists)
  std::map<std::pair<int32_t, int32_t>, int64_t> cedge;
  std::map<std::vector<int32_t>, int64_t> cface;
  for (int c = 0; c < Cm.nc; ++c) {
    int64_t q = Dc.elem_ptr[c] + (Cm.cell_vptr[c + 1] - Cm.cell_vptr[c]);
    std::vector<std::pair<int32_t, int32_t>> es;
    for (int f = Cm.cell_fptr[c]; f < Cm.cell_fptr[c + 1]; ++f)
      for (int32_t m = Cm.face_vptr[f]; m < Cm.face_vptr[f + 1]; ++m) {
        const int32_t u = Cm.face_v[m], w = Cm.face_v[m + 1 < Cm.face_vptr[f + 1] ? m + 1 : Cm.face_vptr[f]];
        es.emplace_back(std::min(u, w), std::max(u, w));
      }
    std::sort(es.begin(), es.end());
    es.erase(std::unique(es.begin(), es.end()), es.end());
    for (auto& e : es) cedge[e] = Dc.elem_dof[size_t(q++)];
    for (int f = Cm.cell_fptr[c]; f < Cm.cell_fptr[c + 1]; ++f) {
      std::vector<int32_t> key(Cm.face_v.begin() + Cm.face_vptr[f], Cm.face_v.begin() + Cm.face_vptr[f + 1]);
      std::sort(key.begin(), key.end());
      cface[key] = Dc.elem_dof[size_t(q++)];
    }
  }
  auto entity_cols = [&](int8_t type, int32_t a, int32_t b, int C, std::vector<int64_t>& out) {
    out.clear();
    if (naive && (type == PLACE_EDGE || type == PLACE_FACE)) type = PLACE_CELL;  // Eq. 16
    if (type == PLACE_VERTEX) {
      out.push_back(a);
    } else if (type == PLACE_EDGE) {
      out.push_back(a);
      out.push_back(b);
      out.push_back(cedge.at({std::min(a, b), std::max(a, b)}));
    } else if (type == PLACE_FACE) {
      const int32_t s = Cm.face_vptr[a], e = Cm.face_vptr[a + 1];
      std::vector<int32_t> key(Cm.face_v.begin() + s, Cm.face_v.begin() + e);
      for (int32_t m = s; m < e; ++m) {
        const int32_t u = Cm.face_v[m], w = Cm.face_v[m + 1 < e ? m + 1 : s];
        out.push_back(u);
        out.push_back(cedge.at({std::min(u, w), std::max(u, w)}));
      }
      std::sort(key.begin(), key.end());
      out.push_back(cface.at(key));
    } else {
      out.assign(Dc.elem_dof.begin() + Dc.elem_ptr[C], Dc.elem_dof.begin() + Dc.elem_ptr[C + 1]);
    }
    std::sort(out.begin(), out.end());
    out.erase(std::unique(out.begin(), out.end()), out.end());
  };
  // first fine cell (cell order) holding each vertex, edge and face
  std::vector<int32_t> vcell(size_t(F.nv), -1);
  std::map<std::pair<int32_t, int32_t>, int32_t> ecell;
  std::map<std::vector<int32_t>, std::pair<int32_t, int32_t>> fcell;  // key -> (cell, occurrence)
  for (int c = 0; c < F.nc; ++c)
    for (int f = F.cell_fptr[c]; f < F.cell_fptr[c + 1]; ++f) {
      const int32_t s = F.face_vptr[f], e = F.face_vptr[f + 1];
      std::vector<int32_t> key(F.face_v.begin() + s, F.face_v.begin() + e);
      std::sort(key.begin(), key.end());
      fcell.emplace(key, std::make_pair(int32_t(c), int32_t(f)));
      for (int32_t m = s; m < e; ++m) {
        const int32_t u = F.face_v[m], w = F.face_v[m + 1 < e ? m + 1 : s];
        if (vcell[size_t(u)] < 0) vcell[size_t(u)] = c;
        ecell.emplace(std::make_pair(std::min(u, w), std::max(u, w)), c);
      }
    }
  std::vector<std::vector<int64_t>> rows(static_cast<size_t>(Df.n));
  std::vector<int64_t> cols;
  int8_t type;
  int32_t a, b;
  for (int32_t v = 0; v < F.nv; ++v) {
    const int C = F.parent[vcell[size_t(v)]];
    classify_point(Cm, C, &F.V[3 * size_t(v)], type, a, b);
    entity_cols(type, a, b, C, cols);
    rows[size_t(v)] = cols;
  }
  // edges: fine DOF ids from the fine element lists
  for (int c = 0; c < F.nc; ++c) {
    int64_t q = Df.elem_ptr[c] + (F.cell_vptr[c + 1] - F.cell_vptr[c]);
    std::vector<std::pair<int32_t, int32_t>> es;
    for (int f = F.cell_fptr[c]; f < F.cell_fptr[c + 1]; ++f)
      for (int32_t m = F.face_vptr[f]; m < F.face_vptr[f + 1]; ++m) {
        const int32_t u = F.face_v[m], w = F.face_v[m + 1 < F.face_vptr[f + 1] ? m + 1 : F.face_vptr[f]];
        es.emplace_back(std::min(u, w), std::max(u, w));
      }
    std::sort(es.begin(), es.end());
    es.erase(std::unique(es.begin(), es.end()), es.end());
    for (auto& e : es) {
      const int64_t g = Df.elem_dof[size_t(q++)];
      if (!rows[size_t(g)].empty()) continue;
      const int C = F.parent[ecell.at(e)];
      const double x[3] = {0.5 * (F.V[3 * size_t(e.first)] + F.V[3 * size_t(e.second)]),
                           0.5 * (F.V[3 * size_t(e.first) + 1] + F.V[3 * size_t(e.second) + 1]),
                           0.5 * (F.V[3 * size_t(e.first) + 2] + F.V[3 * size_t(e.second) + 2])};
      classify_point(Cm, C, x, type, a, b);
      entity_cols(type, a, b, C, cols);
      rows[size_t(g)] = cols;
    }
    for (int f = F.cell_fptr[c]; f < F.cell_fptr[c + 1]; ++f) {
      const int64_t g = Df.elem_dof[size_t(q++)];
      if (!rows[size_t(g)].empty()) continue;
      const int32_t s = F.face_vptr[f], e = F.face_vptr[f + 1];
      std::vector<int32_t> key(F.face_v.begin() + s, F.face_v.begin() + e);
      std::sort(key.begin(), key.end());
      const auto ce = fcell.at(key);
      const int C = F.parent[ce.first];
      // area centroid of the face (fan of triangles from its first vertex)
      const int32_t fs = F.face_vptr[ce.second], fe = F.face_vptr[ce.second + 1];
      const double* p0 = &F.V[3 * size_t(F.face_v[fs])];
      double cen[3] = {0, 0, 0}, area = 0;
      for (int32_t m = fs + 1; m + 1 < fe; ++m) {
        const double* p1 = &F.V[3 * size_t(F.face_v[m])];
        const double* p2 = &F.V[3 * size_t(F.face_v[m + 1])];
        const double u[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
        const double w[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
        const double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
        const double ar = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
        for (int d = 0; d < 3; ++d) cen[d] += ar * (p0[d] + p1[d] + p2[d]) / 3.0;
        area += ar;
      }
      for (int d = 0; d < 3; ++d) cen[d] /= area;
      classify_point(Cm, C, cen, type, a, b);
      if (type == PLACE_FACE)
        entity_cols(type, a, b, C, cols);
      else
        entity_cols(PLACE_CELL, -1, -1, C, cols);
      rows[size_t(g)] = cols;
    }
    entity_cols(PLACE_CELL, -1, -1, F.parent[c], cols);
    rows[size_t(Df.elem_dof[size_t(q)])] = cols;
  }
  rowptr.assign(1, 0);
  col.clear();
  for (auto& r : rows) {
    col.insert(col.end(), r.begin(), r.end());
    rowptr.push_back(int64_t(col.size()));
  }
}

}  // namespace fvem

namespace fvem {

namespace {

// Local edge tables of a level (element order of the k = 2 element kernel).
void element_tables_k2(const LevelMesh& M, LevelK2& K) {
  const DofsK2& D = K.D;
  K.cdof = D.nv + D.ne + D.nf;
  K.edge_ptr.assign(1, 0);
  K.edge_v.clear();
  K.fpos_v.assign(M.face_v.size(), 0);
  K.fpos_e.assign(M.face_v.size(), 0);
  K.perm.assign(D.elem_dof.size(), -1);
  K.k2_off.assign(1, 0);
  K.face_off.assign(1, 0);
  K.max_ne = K.max_nf = K.max_fk = 0;
  std::vector<std::pair<int32_t, int32_t>> es;
  for (int c = 0; c < M.nc; ++c) {
    es.clear();
    for (int f = M.cell_fptr[c]; f < M.cell_fptr[c + 1]; ++f)
      for (int32_t q = M.face_vptr[f]; q < M.face_vptr[f + 1]; ++q) {
        const int32_t u = M.face_v[q], w = M.face_v[q + 1 < M.face_vptr[f + 1] ? q + 1 : M.face_vptr[f]];
        es.emplace_back(std::min(u, w), std::max(u, w));
      }
    std::sort(es.begin(), es.end());
    es.erase(std::unique(es.begin(), es.end()), es.end());
    for (auto& e : es) {
      K.edge_v.push_back(e.first);
      K.edge_v.push_back(e.second);
    }
    K.edge_ptr.push_back(int32_t(K.edge_v.size() / 2));
    const int32_t vb = M.cell_vptr[c], nv = M.cell_vptr[c + 1] - vb;
    for (int f = M.cell_fptr[c]; f < M.cell_fptr[c + 1]; ++f) {
      const int32_t s = M.face_vptr[f], e = M.face_vptr[f + 1];
      K.max_fk = std::max(K.max_fk, int(e - s));
      for (int32_t q = s; q < e; ++q) {
        const int32_t u = M.face_v[q], w = M.face_v[q + 1 < e ? q + 1 : s];
        K.fpos_v[size_t(q)] =
            int32_t(std::lower_bound(M.cell_v.begin() + vb, M.cell_v.begin() + vb + nv, u) - (M.cell_v.begin() + vb));
        K.fpos_e[size_t(q)] = int32_t(std::lower_bound(es.begin(), es.end(), std::make_pair(std::min(u, w), std::max(u, w))) -
                                      es.begin());
      }
      K.face_off.push_back(K.face_off.back() + 6 * (2 * int64_t(e - s) + 1) + 16);
    }
    const int64_t eb = D.elem_ptr[c], ne = D.elem_ptr[c + 1] - eb;
    K.max_ne = std::max(K.max_ne, int(ne));
    K.max_nf = std::max(K.max_nf, M.cell_fptr[c + 1] - M.cell_fptr[c]);
    // sorted boundary ids: position of each element-order entry
    std::vector<int64_t> ids(D.elem_dof.begin() + eb, D.elem_dof.begin() + eb + ne - 1);
    std::sort(ids.begin(), ids.end());
    for (int64_t i = 0; i + 1 < ne; ++i)
      K.perm[size_t(eb + i)] =
          int32_t(std::lower_bound(ids.begin(), ids.end(), D.elem_dof[size_t(eb + i)]) - ids.begin());
    K.k2_off.push_back(K.k2_off.back() + ne * ne);
  }
}

}  // namespace

int build_plan_k2(const Topology& T, std::vector<LevelPlan>& plan, std::vector<LevelK2>& k2, std::string& err,
                  bool naive) {
  const int Lv = T.L;
  plan.assign(Lv, LevelPlan());
  k2.assign(Lv, LevelK2());
  for (int l = 0; l < Lv; ++l) {
    build_dofs_k2(T.levels[l], k2[l].D);
    element_tables_k2(T.levels[l], k2[l]);
  }
  // children lists of coarse cells
  for (int l = 1; l < Lv; ++l) {
    const LevelMesh& F = T.levels[l - 1];
    LevelPlan& P = plan[l];
    P.nc = T.levels[l].nc;
    P.child_ptr.assign(P.nc + 1, 0);
    for (int c = 0; c < F.nc; ++c) P.child_ptr[F.parent[c] + 1]++;
    for (int c = 0; c < P.nc; ++c) P.child_ptr[c + 1] += P.child_ptr[c];
    P.child_cell.assign(F.nc, 0);
    std::vector<int32_t> fill(P.child_ptr.begin(), P.child_ptr.end() - 1);
    for (int c = 0; c < F.nc; ++c) P.child_cell[fill[F.parent[c]]++] = c;
  }
  // Coarse DOFs the prolongation uses: every one.  The fine cell-mean rows of
  // the full k = 2 prolongation take all DOFs of their parent cell, and every
  // coarse cell has a child (the hierarchy is nested), so no coarse column
  // is empty; the free coarse DOFs are the non-Dirichlet ones.
  std::vector<std::vector<char>> used(Lv);
  for (int l = 1; l < Lv; ++l) used[l].assign(size_t(k2[l].D.n), 1);
  // condensed prolongation rows with their placements
  for (int l = 0; l + 1 < Lv; ++l) {
    const LevelMesh& F = T.levels[l];
    const LevelMesh& Cm = T.levels[l + 1];
    const LevelK2& Kf = k2[l];
    const LevelK2& Kc = k2[l + 1];
    LevelK2& R = k2[l];
    LevelPlan& P = plan[l];
    const int64_t nb = Kf.cdof;
    std::vector<std::pair<int32_t, int32_t>> cedges;
    for (size_t q = 0; q + 1 < Kc.edge_v.size(); q += 2) cedges.emplace_back(Kc.edge_v[q], Kc.edge_v[q + 1]);
    std::sort(cedges.begin(), cedges.end());
    cedges.erase(std::unique(cedges.begin(), cedges.end()), cedges.end());
    auto cedge = [&](int32_t u, int32_t w) {
      return int32_t(Kc.D.nv + (std::lower_bound(cedges.begin(), cedges.end(), std::make_pair(std::min(u, w), std::max(u, w))) -
                                cedges.begin()));
    };
    std::vector<int32_t> occ_cell(Cm.face_pid.size(), 0);
    for (int c = 0; c < Cm.nc; ++c)
      for (int f = Cm.cell_fptr[c]; f < Cm.cell_fptr[c + 1]; ++f) occ_cell[size_t(f)] = c;
    auto face_cols = [&](int32_t fo, std::vector<int32_t>& out) {
      const int c = occ_cell[size_t(fo)];
      const int32_t s = Cm.face_vptr[fo], e = Cm.face_vptr[fo + 1];
      for (int32_t q = s; q < e; ++q) out.push_back(Cm.face_v[q]);
      for (int32_t q = s; q < e; ++q) out.push_back(cedge(Cm.face_v[q], Cm.face_v[q + 1 < e ? q + 1 : s]));
      const int64_t eb = Kc.D.elem_ptr[c];
      const int64_t nvc = Cm.cell_vptr[c + 1] - Cm.cell_vptr[c], nec = Kc.edge_ptr[c + 1] - Kc.edge_ptr[c];
      out.push_back(int32_t(Kc.D.elem_dof[size_t(eb + nvc + nec + (fo - Cm.cell_fptr[c]))]));
    };
    auto cell_cols = [&](int c, std::vector<int32_t>& out) {
      for (int64_t q = Kc.D.elem_ptr[c]; q + 1 < Kc.D.elem_ptr[c + 1]; ++q) out.push_back(int32_t(Kc.D.elem_dof[size_t(q)]));
    };
    // first fine cell (cell order) holding each vertex, edge and face
    std::vector<int32_t> vcell(size_t(F.nv), -1);
    std::vector<int32_t> ecell(size_t(Kf.D.ne), -1), fcell(size_t(Kf.D.nf), -1), focc(size_t(Kf.D.nf), -1);
    for (int c = 0; c < F.nc; ++c) {
      const int64_t eb = Kf.D.elem_ptr[c];
      const int32_t nvc = F.cell_vptr[c + 1] - F.cell_vptr[c], nec = Kf.edge_ptr[c + 1] - Kf.edge_ptr[c];
      for (int32_t q = F.cell_vptr[c]; q < F.cell_vptr[c + 1]; ++q)
        if (vcell[size_t(F.cell_v[q])] < 0) vcell[size_t(F.cell_v[q])] = c;
      for (int32_t q = 0; q < nec; ++q) {
        const int64_t g = Kf.D.elem_dof[size_t(eb + nvc + q)] - Kf.D.nv;
        if (ecell[size_t(g)] < 0) ecell[size_t(g)] = c;
      }
      for (int f = F.cell_fptr[c]; f < F.cell_fptr[c + 1]; ++f) {
        const int64_t g = Kf.D.elem_dof[size_t(eb + nvc + nec + (f - F.cell_fptr[c]))] - Kf.D.nv - Kf.D.ne;
        if (fcell[size_t(g)] < 0) {
          fcell[size_t(g)] = c;
          focc[size_t(g)] = f;
        }
      }
    }
    // edge endpoints per edge DOF (from the fine cells' edge tables)
    std::vector<int32_t> eu(size_t(Kf.D.ne), -1), ew(size_t(Kf.D.ne), -1);
    for (int c = 0; c < F.nc; ++c) {
      const int64_t eb = Kf.D.elem_ptr[c];
      const int32_t nvc = F.cell_vptr[c + 1] - F.cell_vptr[c];
      for (int32_t q = Kf.edge_ptr[c]; q < Kf.edge_ptr[c + 1]; ++q) {
        const int64_t g = Kf.D.elem_dof[size_t(eb + nvc + (q - Kf.edge_ptr[c]))] - Kf.D.nv;
        eu[size_t(g)] = Kf.edge_v[2 * size_t(q)];
        ew[size_t(g)] = Kf.edge_v[2 * size_t(q) + 1];
      }
    }
    R.pk.assign(size_t(nb), 0);
    R.pC.assign(size_t(nb), -1);
    R.pa.assign(size_t(nb), -1);
    R.pb.assign(size_t(nb), -1);
    R.px.assign(3 * size_t(nb), 0.0);
    P.prow_ptr.assign(size_t(nb) + 1, 0);
    P.prow_col.clear();
    std::vector<int32_t> cols;
    auto place_point = [&](int64_t g, const double* x, int C) {
      int8_t type;
      int32_t a, b;
      classify_point(Cm, C, x, type, a, b);
      if (naive && (type == PLACE_EDGE || type == PLACE_FACE)) type = PLACE_CELL;  // Eq. 16: from the cell's Pi_2
      cols.clear();
      R.pC[size_t(g)] = C;
      for (int d = 0; d < 3; ++d) R.px[3 * size_t(g) + d] = x[d];
      if (type == PLACE_VERTEX) {
        R.pk[size_t(g)] = 0;
        R.pa[size_t(g)] = a;
        cols.push_back(a);
      } else if (type == PLACE_EDGE) {
        R.pk[size_t(g)] = 1;
        R.pa[size_t(g)] = a;
        R.pb[size_t(g)] = b;
        cols.push_back(a);
        cols.push_back(b);
        cols.push_back(cedge(a, b));
      } else if (type == PLACE_FACE) {
        R.pk[size_t(g)] = 2;
        R.pa[size_t(g)] = a;
        face_cols(a, cols);
      } else {
        R.pk[size_t(g)] = 3;
        cell_cols(C, cols);
      }
    };
    for (int64_t g = 0; g < nb; ++g) {
      if (g < Kf.D.nv) {
        place_point(g, &F.V[3 * size_t(g)], F.parent[vcell[size_t(g)]]);
      } else if (g < Kf.D.nv + Kf.D.ne) {
        const int64_t e = g - Kf.D.nv;
        const double x[3] = {0.5 * (F.V[3 * size_t(eu[size_t(e)])] + F.V[3 * size_t(ew[size_t(e)])]),
                             0.5 * (F.V[3 * size_t(eu[size_t(e)]) + 1] + F.V[3 * size_t(ew[size_t(e)]) + 1]),
                             0.5 * (F.V[3 * size_t(eu[size_t(e)]) + 2] + F.V[3 * size_t(ew[size_t(e)]) + 2])};
        place_point(g, x, F.parent[ecell[size_t(e)]]);
      } else {
        const int64_t fi = g - Kf.D.nv - Kf.D.ne;
        const int C = F.parent[fcell[size_t(fi)]];
        const int32_t fo = focc[size_t(fi)];
        // area centroid (fan of triangles from the first vertex)
        const int32_t fs = F.face_vptr[fo], fe = F.face_vptr[fo + 1];
        const double* p0 = &F.V[3 * size_t(F.face_v[fs])];
        double cen[3] = {0, 0, 0}, area = 0;
        for (int32_t m = fs + 1; m + 1 < fe; ++m) {
          const double* p1 = &F.V[3 * size_t(F.face_v[m])];
          const double* p2 = &F.V[3 * size_t(F.face_v[m + 1])];
          const double u[3] = {p1[0] - p0[0], p1[1] - p0[1], p1[2] - p0[2]};
          const double w[3] = {p2[0] - p0[0], p2[1] - p0[1], p2[2] - p0[2]};
          const double cr[3] = {u[1] * w[2] - u[2] * w[1], u[2] * w[0] - u[0] * w[2], u[0] * w[1] - u[1] * w[0]};
          const double ar = 0.5 * std::sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
          for (int d = 0; d < 3; ++d) cen[d] += ar * (p0[d] + p1[d] + p2[d]) / 3.0;
          area += ar;
        }
        for (int d = 0; d < 3; ++d) cen[d] /= area;
        int8_t type;
        int32_t a, b;
        classify_point(Cm, C, cen, type, a, b);
        cols.clear();
        R.pC[size_t(g)] = C;
        R.pb[size_t(g)] = fo;
        if (type == PLACE_FACE && !naive) {
          R.pk[size_t(g)] = 4;
          R.pa[size_t(g)] = a;
          face_cols(a, cols);
        } else {
          R.pk[size_t(g)] = 5;
          cell_cols(C, cols);
        }
      }
      P.prow_col.insert(P.prow_col.end(), cols.begin(), cols.end());
      P.prow_ptr[size_t(g) + 1] = int32_t(P.prow_col.size());
    }
  }
  // per level: free boundary DOFs, element lists, incidence, pattern, layout
  for (int l = 0; l < Lv; ++l) {
    const LevelMesh& M = T.levels[l];
    const LevelK2& K = k2[l];
    LevelPlan& P = plan[l];
    const int64_t nb = K.cdof;
    if (nb >= (int64_t(1) << 31) || K.D.n >= (int64_t(1) << 31)) {
      err = "too many k = 2 DOFs for 32-bit ids";
      return 1;
    }
    P.nv = int(nb);
    P.nc = M.nc;
    P.dof_of_vertex.assign(size_t(nb), -1);
    P.vertex_of_dof.clear();
    for (int64_t g = 0; g < nb; ++g)
      if (!K.D.dirichlet[size_t(g)] && (l == 0 || used[l][size_t(g)])) {
        P.dof_of_vertex[size_t(g)] = int32_t(P.vertex_of_dof.size());
        P.vertex_of_dof.push_back(int32_t(g));
      }
    P.ndof = int(P.vertex_of_dof.size());
    if (P.ndof == 0) {
      err = "level " + std::to_string(l) + " has no free DOF";
      return 1;
    }
    // element lists: the cell's sorted boundary ids; on coarse levels widened
    // by every prolongation column of the children's lists (as for k = 1), so
    // the per-cell Galerkin sum is P^T A P for any prolongation
    P.elem_is_cell = false;
    P.elem_vptr.assign(1, 0);
    P.elem_v.clear();
    P.kptr.assign(1, 0);
    std::vector<int32_t> cnt(size_t(nb) + 1, 0);
    for (int c = 0; c < M.nc; ++c) {
      std::vector<int32_t> ids;
      for (int64_t q = K.D.elem_ptr[c]; q + 1 < K.D.elem_ptr[c + 1]; ++q) ids.push_back(int32_t(K.D.elem_dof[size_t(q)]));
      if (l > 0) {
        const LevelPlan& Fp = plan[l - 1];
        for (int32_t q = P.child_ptr[c]; q < P.child_ptr[c + 1]; ++q) {
          const int e = P.child_cell[q];
          for (int32_t u = Fp.elem_vptr[e]; u < Fp.elem_vptr[e + 1]; ++u) {
            const int32_t g = Fp.elem_v[u];
            for (int32_t r = Fp.prow_ptr[size_t(g)]; r < Fp.prow_ptr[size_t(g) + 1]; ++r) ids.push_back(Fp.prow_col[size_t(r)]);
          }
        }
      }
      std::sort(ids.begin(), ids.end());
      ids.erase(std::unique(ids.begin(), ids.end()), ids.end());
      for (int32_t g : ids) cnt[size_t(g) + 1]++;
      P.elem_v.insert(P.elem_v.end(), ids.begin(), ids.end());
      P.elem_vptr.push_back(int32_t(P.elem_v.size()));
      const int64_t n = int64_t(ids.size());
      P.kptr.push_back(P.kptr.back() + n * n);
      P.max_ne = std::max(P.max_ne, int(n));
      P.max_nv = std::max(P.max_nv, M.cell_vptr[c + 1] - M.cell_vptr[c]);
      P.max_nf = std::max(P.max_nf, M.cell_fptr[c + 1] - M.cell_fptr[c]);
    }
    P.inc_ptr.assign(size_t(nb) + 1, 0);
    for (int64_t g = 0; g < nb; ++g) P.inc_ptr[size_t(g) + 1] = P.inc_ptr[size_t(g)] + cnt[size_t(g) + 1];
    P.inc_cell.assign(size_t(P.inc_ptr[size_t(nb)]), 0);
    P.inc_loc.assign(size_t(P.inc_ptr[size_t(nb)]), 0);
    std::vector<int32_t> fill(P.inc_ptr.begin(), P.inc_ptr.end() - 1);
    for (int c = 0; c < M.nc; ++c)
      for (int32_t q = P.elem_vptr[c]; q < P.elem_vptr[c + 1]; ++q) {
        const int32_t g = P.elem_v[q];
        P.inc_cell[fill[g]] = c;
        P.inc_loc[fill[g]] = q - P.elem_vptr[c];
        fill[g]++;
      }
    P.a_rowptr.assign(size_t(P.ndof) + 1, 0);
    P.a_col.clear();
    std::vector<int32_t> cols;
    for (int i = 0; i < P.ndof; ++i) {
      const int32_t g = P.vertex_of_dof[i];
      cols.clear();
      for (int32_t q = P.inc_ptr[g]; q < P.inc_ptr[g + 1]; ++q) {
        const int c = P.inc_cell[q];
        for (int32_t u = P.elem_vptr[c]; u < P.elem_vptr[c + 1]; ++u) {
          const int32_t j = P.dof_of_vertex[size_t(P.elem_v[u])];
          if (j >= 0) cols.push_back(j);
        }
      }
      std::sort(cols.begin(), cols.end());
      cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
      P.a_col.insert(P.a_col.end(), cols.begin(), cols.end());
      P.a_rowptr[size_t(i) + 1] = int64_t(P.a_col.size());
    }
    if (P.a_rowptr[size_t(P.ndof)] >= (int64_t(1) << 31)) {
      err = "too many nonzeros for 32-bit slot indices";
      return 1;
    }
    build_sell(P);
  }
  // free prolongation (rows: free DOFs of l, cols: free DOFs of l+1) and its transpose
  for (int l = 0; l + 1 < Lv; ++l) {
    LevelPlan& P = plan[l];
    const LevelPlan& Cp = plan[l + 1];
    P.pf_rowptr.assign(size_t(P.ndof) + 1, 0);
    P.pf_col.clear();
    P.pf_src.clear();
    for (int i = 0; i < P.ndof; ++i) {
      const int32_t g = P.vertex_of_dof[i];
      for (int32_t q = P.prow_ptr[size_t(g)]; q < P.prow_ptr[size_t(g) + 1]; ++q) {
        const int32_t j = Cp.dof_of_vertex[size_t(P.prow_col[size_t(q)])];
        if (j < 0) continue;
        P.pf_col.push_back(j);
        P.pf_src.push_back(q);
      }
      P.pf_rowptr[size_t(i) + 1] = int64_t(P.pf_col.size());
    }
    const int nc = Cp.ndof;
    P.pt_rowptr.assign(size_t(nc) + 1, 0);
    for (int32_t j : P.pf_col) P.pt_rowptr[size_t(j) + 1]++;
    for (int j = 0; j < nc; ++j) P.pt_rowptr[size_t(j) + 1] += P.pt_rowptr[size_t(j)];
    P.pt_col.assign(P.pf_col.size(), 0);
    P.pt_src.assign(P.pf_col.size(), 0);
    std::vector<int64_t> fill(P.pt_rowptr.begin(), P.pt_rowptr.end() - 1);
    for (int i = 0; i < P.ndof; ++i)
      for (int64_t k = P.pf_rowptr[size_t(i)]; k < P.pf_rowptr[size_t(i) + 1]; ++k) {
        const int32_t j = P.pf_col[size_t(k)];
        P.pt_col[size_t(fill[size_t(j)])] = i;
        P.pt_src[size_t(fill[size_t(j)])] = k;
        fill[size_t(j)]++;
      }
  }
  return 0;
}

}  // namespace fvem
