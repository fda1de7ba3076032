// Host precompute: cut cells (Sec. 5.1), hierarchy (Sec. 5.2), conforming level
// meshes and prolongation placements (Sec. 4.3).
//
// Evaluation rules for every FP64 decision (fixed order, no FMA contraction;
// this file is compiled with -ffp-contract=off):
//   dot(a,b)   = (a0*b0 + a1*b1) + a2*b2
//   cross(a,b) = (a1*b2 - a2*b1, a2*b0 - a0*b2, a0*b1 - a1*b0)
//   side_p(x)  = dot(n_p, x) + d_p
//   grid plane (axis a, index i): n = e_a, d = -(i/N); id = a*(N+1) + i
//   triangle t: c = cross(v1-v0, v2-v0), n = c / sqrt((c0*c0 + c1*c1) + c2*c2),
//               d = -dot(n, v0); id = 3*(N+1) + t
//   vertex of planes i<j<k by Cramer's rule with det = dot(ni, cross(nj,nk)),
//               x_c = ((((-di)*cjk_c) - (dj*cki_c)) - (dk*cij_c)) / det
// Tolerances: EPS = 1e-10 (side tests), WELD = 1e-9 (max-norm coincidence),
// |det| >= 1e-12, cells below volume 1e-12 are not created (Sec. 5.1).
#include "topo.h"

#include <algorithm>
#include <array>
#include <parallel/algorithm>
#include <cmath>
#include <cstring>
#include <deque>
#include <map>
#include <queue>
#include <set>
#include <tuple>
#include <unordered_map>
#include <unordered_set>
#include <chrono>
#include <cstdio>
#include <cstdlib>

namespace fvem {
namespace {

constexpr double EPS = 1e-10;
constexpr double WELD = 1e-9;
constexpr double DET_MIN = 1e-12;
constexpr double VOL_MIN = 1e-12;
constexpr double AREA_MIN = 1e-20;
constexpr double WQ = 1099511627776.0;  // 2^40
constexpr double Q30 = 1073741824.0;    // 2^30

// Open-addressing map from 64-bit keys to int32 values (linear probing,
// power-of-two capacity).  Same semantics as the standard map it replaces on
// the large level-0 tables: find returns -1 when absent, insert keeps the
// first value stored under a key.  find is safe from several threads once no
// thread inserts.
class FlatMap {
 public:
  explicit FlatMap(size_t expect = 16) { reset(expect); }
  void reset(size_t expect) {
    size_t cap = 16;
    while (cap < 2 * expect + 16) cap <<= 1;
    keys_.assign(cap, 0);
    vals_.assign(cap, -1);
    used_.assign(cap, 0);
    mask_ = cap - 1;
    n_ = 0;
  }
  int32_t find(uint64_t k) const {
    for (size_t i = slot(k);; i = (i + 1) & mask_) {
      if (!used_[i]) return -1;
      if (keys_[i] == k) return vals_[i];
    }
  }
  // returns the value stored under k (v if k was absent)
  int32_t insert(uint64_t k, int32_t v, bool& inserted) {
    if (2 * (n_ + 1) > keys_.size()) grow();
    for (size_t i = slot(k);; i = (i + 1) & mask_) {
      if (!used_[i]) {
        used_[i] = 1;
        keys_[i] = k;
        vals_[i] = v;
        ++n_;
        inserted = true;
        return v;
      }
      if (keys_[i] == k) {
        inserted = false;
        return vals_[i];
      }
    }
  }
  size_t size() const { return n_; }

 private:
  size_t slot(uint64_t k) const {
    k ^= k >> 30;
    k *= 0xBF58476D1CE4E5B9ULL;
    k ^= k >> 27;
    k *= 0x94D049BB133111EBULL;
    k ^= k >> 31;
    return size_t(k) & mask_;
  }
  void grow() {
    std::vector<uint64_t> ok = std::move(keys_);
    std::vector<int32_t> ov = std::move(vals_);
    std::vector<uint8_t> ou = std::move(used_);
    reset(ok.size());
    bool ins;
    for (size_t i = 0; i < ok.size(); ++i)
      if (ou[i]) insert(ok[i], ov[i], ins);
  }
  std::vector<uint64_t> keys_;
  std::vector<int32_t> vals_;
  std::vector<uint8_t> used_;
  size_t mask_ = 0, n_ = 0;
};

// Lists per 64-bit key in insertion order (head / next over element ids).
struct KeyLists {
  FlatMap head;
  std::vector<int32_t> tail, next;  // tail per list, next per element
  explicit KeyLists(size_t expect) : head(expect) {}
  void push(uint64_t k, int32_t e) {
    if (size_t(e) >= next.size()) next.resize(size_t(e) + 1, -1);
    bool ins;
    const int32_t l = head.insert(k, int32_t(tail.size()), ins);
    if (ins) {
      tail.push_back(e);
      heads.push_back(e);
    } else {
      next[size_t(tail[size_t(l)])] = e;
      tail[size_t(l)] = e;
    }
  }
  int32_t first(uint64_t k) const {
    const int32_t l = head.find(k);
    return l < 0 ? -1 : heads[size_t(l)];
  }
  int32_t after(int32_t e) const { return size_t(e) < next.size() ? next[size_t(e)] : -1; }
  std::vector<int32_t> heads;
};

struct V3 {
  double x, y, z;
  double operator[](int i) const { return i == 0 ? x : (i == 1 ? y : z); }
};
inline V3 sub(const V3& a, const V3& b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
inline V3 add(const V3& a, const V3& b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
inline V3 scl(const V3& a, double s) { return {a.x * s, a.y * s, a.z * s}; }
inline V3 cross(const V3& a, const V3& b) {
  return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
inline double dot(const V3& a, const V3& b) { return (a.x * b.x + a.y * b.y) + a.z * b.z; }
inline double maxabs(const V3& a, const V3& b) {
  return std::max(std::fabs(a.x - b.x), std::max(std::fabs(a.y - b.y), std::fabs(a.z - b.z)));
}

struct Key {
  int a, b, c;
  bool operator<(const Key& o) const {
    if (a != o.a) return a < o.a;
    if (b != o.b) return b < o.b;
    return c < o.c;
  }
  bool operator==(const Key& o) const { return a == o.a && b == o.b && c == o.c; }
};
inline uint64_t pack(const Key& k) {
  return (uint64_t(uint32_t(k.a)) << 42) | (uint64_t(uint32_t(k.b)) << 21) | uint64_t(uint32_t(k.c));
}

struct Planes {
  int N = 0, ngrid = 0;
  std::vector<V3> n;
  std::vector<double> d;
  double side(int p, const V3& x) const { return dot(n[p], x) + d[p]; }
  bool is_grid(int p) const { return p < ngrid; }
};

using HS = std::vector<std::pair<int, int>>;  // (plane id, sign): sign*side <= 0

struct Face {
  int pid, sg;
  std::vector<int> cyc;
};

struct Poly {
  HS H;
  std::vector<V3> v;
  std::vector<std::vector<Key>> vk;
  std::vector<Face> f;
  double vol = 0.0;
  V3 cen{0, 0, 0};
};

bool solve3(const Planes& P, int i, int j, int k, V3& out) {
  const V3 &ni = P.n[i], &nj = P.n[j], &nk = P.n[k];
  double di = P.d[i], dj = P.d[j], dk = P.d[k];
  V3 cjk = cross(nj, nk), cki = cross(nk, ni), cij = cross(ni, nj);
  double det = dot(ni, cjk);
  if (!(std::fabs(det) >= DET_MIN)) return false;
  out.x = ((((-di) * cjk.x) - (dj * cki.x)) - (dk * cij.x)) / det;
  out.y = ((((-di) * cjk.y) - (dj * cki.y)) - (dk * cij.y)) / det;
  out.z = ((((-di) * cjk.z) - (dj * cki.z)) - (dk * cij.z)) / det;
  return true;
}

bool feasible(const Planes& P, const HS& H, const V3& x) {
  for (auto& h : H) {
    double s = P.side(h.first, x);
    if (!(double(h.second) * s <= EPS)) return false;
  }
  return true;
}

void weld_sorted(const std::vector<Key>& keys, const std::vector<V3>& xs, std::vector<V3>& reps,
                 std::vector<std::vector<Key>>& rkeys) {
  reps.clear();
  rkeys.clear();
  for (size_t c = 0; c < keys.size(); ++c) {
    bool hit = false;
    for (size_t r = 0; r < reps.size(); ++r)
      if (maxabs(xs[c], reps[r]) <= WELD) {
        rkeys[r].push_back(keys[c]);
        hit = true;
        break;
      }
    if (!hit) {
      reps.push_back(xs[c]);
      rkeys.push_back({keys[c]});
    }
  }
}

// Counter-clockwise order about `nrm`, starting at idx[0] (insertion sort on a
// cross-product comparator; equal to any correct sort for convex position).
std::vector<int> order_ccw(const std::vector<V3>& pts, const V3& nrm, const std::vector<int>& idx) {
  std::vector<int> rest(idx.begin() + 1, idx.end());
  const V3 piv = pts[idx[0]];
  auto before = [&](int a, int b) {
    double c = dot(cross(sub(pts[a], piv), sub(pts[b], piv)), nrm);
    return c > 0;
  };
  for (size_t i = 1; i < rest.size(); ++i) {
    int x = rest[i];
    size_t j = i;
    while (j > 0 && before(x, rest[j - 1])) {
      rest[j] = rest[j - 1];
      --j;
    }
    rest[j] = x;
  }
  std::vector<int> out;
  out.push_back(idx[0]);
  out.insert(out.end(), rest.begin(), rest.end());
  return out;
}

double polygon_area(const std::vector<V3>& pts, const std::vector<int>& cyc, const V3& nrm) {
  double a0 = 0, a1 = 0, a2 = 0;
  size_t k = cyc.size();
  for (size_t i = 0; i < k; ++i) {
    V3 c = cross(pts[cyc[i]], pts[cyc[(i + 1) % k]]);
    a0 += c.x;
    a1 += c.y;
    a2 += c.z;
  }
  return 0.5 * dot(V3{a0, a1, a2}, nrm);
}

void volume_centroid(Poly& P) {
  P.vol = 0.0;
  P.cen = {0, 0, 0};
  if (P.v.empty() || P.f.empty()) return;
  V3 c0{0, 0, 0};
  for (auto& v : P.v) c0 = add(c0, v);
  double nv = double(P.v.size());
  c0 = {c0.x / nv, c0.y / nv, c0.z / nv};
  double vol = 0.0;
  V3 cen{0, 0, 0};
  for (auto& f : P.f) {
    const V3& a = P.v[f.cyc[0]];
    for (size_t m = 1; m + 1 < f.cyc.size(); ++m) {
      const V3& b = P.v[f.cyc[m]];
      const V3& c = P.v[f.cyc[m + 1]];
      double t = dot(sub(a, c0), cross(sub(b, c0), sub(c, c0))) / 6.0;
      vol += t;
      V3 s = add(add(add(c0, a), b), c);
      cen = add(cen, V3{(t * s.x) / 4.0, (t * s.y) / 4.0, (t * s.z) / 4.0});
    }
  }
  if (vol != 0.0) cen = {cen.x / vol, cen.y / vol, cen.z / vol};
  P.vol = vol;
  P.cen = cen;
}

std::vector<int> sorted_pids(const HS& H) {
  std::vector<int> p;
  for (auto& h : H) p.push_back(h.first);
  std::sort(p.begin(), p.end());
  p.erase(std::unique(p.begin(), p.end()), p.end());
  return p;
}

Poly make_poly(const Planes& P, const HS& H) {
  Poly out;
  out.H = H;
  std::vector<int> pids = sorted_pids(H);
  std::vector<Key> keys;
  std::vector<V3> xs;
  int m = int(pids.size());
  for (int i = 0; i < m; ++i)
    for (int j = i + 1; j < m; ++j)
      for (int k = j + 1; k < m; ++k) {
        V3 x;
        if (!solve3(P, pids[i], pids[j], pids[k], x)) continue;
        if (!feasible(P, H, x)) continue;
        keys.push_back({pids[i], pids[j], pids[k]});
        xs.push_back(x);
      }
  weld_sorted(keys, xs, out.v, out.vk);
  if (out.v.size() < 4) return out;
  for (auto& h : H) {
    std::vector<int> on;
    for (int i = 0; i < int(out.v.size()); ++i)
      if (std::fabs(P.side(h.first, out.v[i])) <= EPS) on.push_back(i);
    if (on.size() < 3) continue;
    V3 nrm = scl(P.n[h.first], double(h.second));
    std::vector<int> cyc = order_ccw(out.v, nrm, on);
    if (polygon_area(out.v, cyc, nrm) <= AREA_MIN) continue;
    out.f.push_back({h.first, h.second, cyc});
  }
  volume_centroid(out);
  return out;
}

// Flat polygon of plane `pid` inside the constraint set Hu; returns reps (CCW
// about sg*n_pid) with their key lists; empty when degenerate.
void face_polygon(const Planes& P, const HS& Hu, int pid, int sg, std::vector<V3>& pts,
                  std::vector<std::vector<Key>>& keys) {
  pts.clear();
  keys.clear();
  std::vector<int> pids = sorted_pids(Hu);
  std::vector<int> others;
  for (int p : pids)
    if (p != pid) others.push_back(p);
  std::vector<std::pair<Key, V3>> cand;
  for (size_t i = 0; i < others.size(); ++i)
    for (size_t j = i + 1; j < others.size(); ++j) {
      int t[3] = {pid, others[i], others[j]};
      std::sort(t, t + 3);
      V3 x;
      if (!solve3(P, t[0], t[1], t[2], x)) continue;
      if (!feasible(P, Hu, x)) continue;
      cand.push_back({Key{t[0], t[1], t[2]}, x});
    }
  std::sort(cand.begin(), cand.end(), [](const std::pair<Key, V3>& a, const std::pair<Key, V3>& b) {
    return a.first < b.first;
  });
  std::vector<Key> ks;
  std::vector<V3> xs;
  for (auto& c : cand) {
    ks.push_back(c.first);
    xs.push_back(c.second);
  }
  std::vector<V3> reps;
  std::vector<std::vector<Key>> rk;
  weld_sorted(ks, xs, reps, rk);
  if (reps.size() < 3) return;
  V3 nrm = scl(P.n[pid], double(sg));
  std::vector<int> idx(reps.size());
  for (size_t i = 0; i < idx.size(); ++i) idx[i] = int(i);
  std::vector<int> cyc = order_ccw(reps, nrm, idx);
  if (polygon_area(reps, cyc, nrm) <= AREA_MIN) return;
  for (int c : cyc) {
    pts.push_back(reps[c]);
    keys.push_back(rk[c]);
  }
}

std::vector<V3> clip_polygon(const Planes& P, const std::vector<V3>& poly, int pid, double keep) {
  std::vector<V3> out;
  size_t k = poly.size();
  if (!k) return out;
  std::vector<double> s(k);
  for (size_t i = 0; i < k; ++i) s[i] = keep * P.side(pid, poly[i]);
  for (size_t i = 0; i < k; ++i) {
    const V3& a = poly[i];
    const V3& b = poly[(i + 1) % k];
    double sa = s[i], sb = s[(i + 1) % k];
    bool ina = sa <= EPS, inb = sb <= EPS;
    if (ina) out.push_back(a);
    if (ina != inb) {
      double t = sa / (sa - sb);
      V3 e = sub(b, a);
      out.push_back(V3{a.x + e.x * t, a.y + e.y * t, a.z + e.z * t});
    }
  }
  return out;
}

double poly_area_fan(const std::vector<V3>& p) {
  if (p.size() < 3) return 0.0;
  double acc = 0.0;
  for (size_t m = 1; m + 1 < p.size(); ++m) {
    V3 c = cross(sub(p[m], p[0]), sub(p[m + 1], p[0]));
    acc += 0.5 * std::sqrt(dot(c, c));
  }
  return acc;
}

HS cube_H(int N, int i0, int j0, int k0, int s) {
  int N1 = N + 1;
  return {{i0, -1}, {i0 + s, 1}, {N1 + j0, -1}, {N1 + j0 + s, 1}, {2 * N1 + k0, -1}, {2 * N1 + k0 + s, 1}};
}

double winding(const std::vector<std::array<V3, 3>>& tris, const V3& p) {
  double acc = 0.0;
  for (auto& t : tris) {
    V3 A = sub(t[0], p), B = sub(t[1], p), C = sub(t[2], p);
    double la = std::sqrt(dot(A, A)), lb = std::sqrt(dot(B, B)), lc = std::sqrt(dot(C, C));
    double num = dot(A, cross(B, C));
    double den = la * lb * lc + dot(A, B) * lc + dot(B, C) * la + dot(C, A) * lb;
    acc += 2.0 * std::atan2(num, den);
  }
  return acc / (4.0 * M_PI);
}

// ------------------------------------------------------------------ BSP trees

enum RootKind : int8_t { UNCUT_FLUID = 0, UNCUT_SOLID = 1, SINGLE_FLUID = 2, SINGLE_SOLID = 3, TREE = 4 };

struct Node {
  int parent = -1, left = -1, right = -1, pid = -1;
  HS H;
  Poly poly;
  double w = 0.0;
  int64_t wq = 0;
  bool solid = false;
  int nfluid = 0;
  bool leaf() const { return left < 0; }
};

struct Tree {
  int r;
  int ijk[3];
  std::vector<Node> nodes;
};

struct TriEntry {
  int t;
  std::vector<V3> poly;
};

struct Ctx {
  int N;
  Planes P;
  std::vector<std::array<V3, 3>> tris;
  double total_area = 0.0;
  std::vector<int8_t> kind;
  std::map<int, Tree> trees;  // ordered by root index
};

inline int ridx(int N, int i, int j, int k) { return i + N * (j + N * k); }

int build_rec(Ctx& C, Tree& T, const HS& H, const std::vector<TriEntry>& lst, int parent, Poly&& poly) {
  int id = int(T.nodes.size());
  T.nodes.emplace_back();
  T.nodes[id].parent = parent;
  T.nodes[id].H = H;
  T.nodes[id].poly = std::move(poly);
  const Poly& Pn = T.nodes[id].poly;
  for (size_t idx = 0; idx < lst.size(); ++idx) {
    int t = lst[idx].t;
    int pid = C.P.ngrid + t;
    double smax = -1e300, smin = 1e300;
    for (auto& v : Pn.v) {
      double s = C.P.side(pid, v);
      smax = std::max(smax, s);
      smin = std::min(smin, s);
    }
    if (!(smax > EPS && smin < -EPS)) continue;
    HS HL = H, HR = H;
    HL.push_back({pid, 1});
    HR.push_back({pid, -1});
    Poly PL = make_poly(C.P, HL), PR = make_poly(C.P, HR);
    if (PL.vol < VOL_MIN || PR.vol < VOL_MIN) continue;
    double area = 0.0;
    for (auto& e : lst) {
      bool flat = true;
      for (int q = 0; q < 3; ++q)
        if (!(std::fabs(C.P.side(pid, C.tris[e.t][q])) <= EPS)) flat = false;
      if (flat) area += poly_area_fan(e.poly);
    }
    double w = area / C.total_area;
    std::vector<TriEntry> left, right;
    for (size_t m = idx + 1; m < lst.size(); ++m) {
      const auto& e = lst[m];
      double mx = -1e300, mn = 1e300;
      bool flat = true;
      for (auto& v : e.poly) {
        double s = C.P.side(pid, v);
        mx = std::max(mx, s);
        mn = std::min(mn, s);
        if (!(std::fabs(s) <= EPS)) flat = false;
      }
      if (flat || mn < -EPS) {
        auto lp = clip_polygon(C.P, e.poly, pid, 1.0);
        if (!lp.empty()) left.push_back({e.t, std::move(lp)});
      }
      if (flat || mx > EPS) {
        auto rp = clip_polygon(C.P, e.poly, pid, -1.0);
        if (!rp.empty()) right.push_back({e.t, std::move(rp)});
      }
    }
    T.nodes[id].pid = pid;
    T.nodes[id].w = w;
    T.nodes[id].wq = int64_t(std::nearbyint(w * WQ));
    int l = build_rec(C, T, HL, left, id, std::move(PL));
    T.nodes[id].left = l;
    int r = build_rec(C, T, HR, right, id, std::move(PR));
    T.nodes[id].right = r;
    return id;
  }
  return id;
}

void build_cut_grid(Ctx& C) {
  int N = C.N;
  const Planes& P = C.P;
  int T = int(C.tris.size());
  C.total_area = 0.0;
  for (int t = 0; t < T; ++t) {
    std::vector<V3> p = {C.tris[t][0], C.tris[t][1], C.tris[t][2]};
    C.total_area += poly_area_fan(p);
  }
  std::map<int, std::vector<TriEntry>> assoc;
  for (int t = 0; t < T; ++t) {
    double mn[3], mx[3];
    for (int a = 0; a < 3; ++a) {
      mn[a] = std::min(std::min(C.tris[t][0][a], C.tris[t][1][a]), C.tris[t][2][a]);
      mx[a] = std::max(std::max(C.tris[t][0][a], C.tris[t][1][a]), C.tris[t][2][a]);
    }
    bool out = false;
    for (int a = 0; a < 3; ++a)
      if (mx[a] < -EPS || mn[a] > 1 + EPS) out = true;
    if (out) continue;
    int lo[3], hi[3];
    for (int a = 0; a < 3; ++a) {
      lo[a] = std::min(std::max(int(std::floor((mn[a] - EPS) * N)), 0), N - 1);
      hi[a] = std::min(std::max(int(std::floor((mx[a] + EPS) * N)), 0), N - 1);
    }
    for (int k = lo[2]; k <= hi[2]; ++k)
      for (int j = lo[1]; j <= hi[1]; ++j)
        for (int i = lo[0]; i <= hi[0]; ++i) {
          std::vector<V3> poly = {C.tris[t][0], C.tris[t][1], C.tris[t][2]};
          for (auto& h : cube_H(N, i, j, k, 1)) {
            poly = clip_polygon(P, poly, h.first, double(h.second));
            if (poly.empty()) break;
          }
          if (!poly.empty()) assoc[ridx(N, i, j, k)].push_back({t, std::move(poly)});
        }
  }
  C.kind.assign(size_t(N) * N * N, UNCUT_FLUID);
  std::vector<char> cut(size_t(N) * N * N, 0);
  std::vector<int> roots;
  std::vector<std::vector<TriEntry>*> lists;
  for (auto& kv : assoc) {
    roots.push_back(kv.first);
    lists.push_back(&kv.second);
    cut[kv.first] = 1;
  }
  std::vector<Tree> built(roots.size());
  std::vector<int8_t> kinds(roots.size(), TREE);
#pragma omp parallel for schedule(dynamic, 4)
  for (long long q = 0; q < (long long)roots.size(); ++q) {
    int r = roots[q];
    auto& lst = *lists[q];
    // cut order: ascending count of other cell triangles crossed strictly, then index
    std::vector<int> cnt(lst.size(), 0);
    for (size_t a = 0; a < lst.size(); ++a) {
      int pid = P.ngrid + lst[a].t;
      for (size_t b = 0; b < lst.size(); ++b) {
        if (b == a) continue;
        double smax = -1e300, smin = 1e300;
        for (int e = 0; e < 3; ++e) {
          double sd = P.side(pid, C.tris[lst[b].t][e]);
          smax = std::max(smax, sd);
          smin = std::min(smin, sd);
        }
        if (smax > EPS && smin < -EPS) cnt[a]++;
      }
    }
    std::vector<int> ord(lst.size());
    for (size_t a = 0; a < ord.size(); ++a) ord[a] = int(a);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
      if (cnt[x] != cnt[y]) return cnt[x] < cnt[y];
      return lst[x].t < lst[y].t;
    });
    std::vector<TriEntry> sl;
    for (int a : ord) sl.push_back(lst[a]);
    int k = r / (N * N), rem = r % (N * N), j = rem / N, i = rem % N;
    Tree& tr = built[q];
    tr.r = r;
    tr.ijk[0] = i;
    tr.ijk[1] = j;
    tr.ijk[2] = k;
    HS H0 = cube_H(N, i, j, k, 1);
    Poly P0 = make_poly(P, H0);
    build_rec(C, tr, H0, sl, -1, std::move(P0));
    if (tr.nodes.size() == 1) {
      V3 c{(double(i) + 0.5) / N, (double(j) + 0.5) / N, (double(k) + 0.5) / N};
      kinds[q] = winding(C.tris, c) > 0.5 ? SINGLE_SOLID : SINGLE_FLUID;
      continue;
    }
    for (auto& nd : tr.nodes)
      if (nd.leaf()) nd.solid = winding(C.tris, nd.poly.cen) > 0.5;
    for (int n = int(tr.nodes.size()) - 1; n >= 0; --n) {
      Node& nd = tr.nodes[n];
      nd.nfluid = nd.leaf() ? (nd.solid ? 0 : 1) : tr.nodes[nd.left].nfluid + tr.nodes[nd.right].nfluid;
    }
  }
  for (size_t q = 0; q < roots.size(); ++q) {
    C.kind[roots[q]] = kinds[q];
    if (kinds[q] == TREE) C.trees.emplace(roots[q], std::move(built[q]));
  }
  // uncut cells: 6-connected components share the inside status
  size_t NN = size_t(N) * N * N;
  std::vector<int> comp(NN, -1);
  std::vector<int> stack;
  for (size_t r0 = 0; r0 < NN; ++r0) {
    if (cut[r0] || comp[r0] >= 0) continue;
    int k = int(r0 / (size_t(N) * N)), rem = int(r0 % (size_t(N) * N)), j = rem / N, i = rem % N;
    V3 c{(double(i) + 0.5) / N, (double(j) + 0.5) / N, (double(k) + 0.5) / N};
    bool solid = winding(C.tris, c) > 0.5;
    stack.clear();
    stack.push_back(int(r0));
    comp[r0] = 1;
    while (!stack.empty()) {
      int r = stack.back();
      stack.pop_back();
      if (solid) C.kind[r] = UNCUT_SOLID;
      int kk = r / (N * N), rr = r % (N * N), jj = rr / N, ii = rr % N;
      int nb[6][3] = {{ii - 1, jj, kk}, {ii + 1, jj, kk}, {ii, jj - 1, kk},
                      {ii, jj + 1, kk}, {ii, jj, kk - 1}, {ii, jj, kk + 1}};
      for (auto& q : nb) {
        if (q[0] < 0 || q[1] < 0 || q[2] < 0 || q[0] >= N || q[1] >= N || q[2] >= N) continue;
        int s = ridx(N, q[0], q[1], q[2]);
        if (cut[s] || comp[s] >= 0) continue;
        comp[s] = 1;
        stack.push_back(s);
      }
    }
  }
}

// ------------------------------------------------------------------ hierarchy

struct Cell {
  bool cube;
  int i, j, k, s;  // cube: min corner and size; node: root ijk
  int r, nid;      // node: root index and node id
};

struct LevelCells {
  std::vector<Cell> cells;
  std::vector<HS> solids;
  std::vector<int32_t> parent;
};

struct HState {
  Ctx& C;
  std::unordered_map<int, int> cubes;  // root index of min corner -> size
  std::map<int, std::unordered_set<int>> collapsed;
  std::unordered_set<int> full;
  explicit HState(Ctx& c) : C(c) {
    int N = C.N;
    for (int r = 0; r < N * N * N; ++r)
      if (C.kind[r] == UNCUT_FLUID || C.kind[r] == SINGLE_FLUID) cubes[r] = 1;
    for (auto& kv : C.trees) collapsed[kv.first];
  }
  bool is_cur_leaf(int r, int n) {
    const Node& nd = C.trees.at(r).nodes[n];
    return nd.leaf() || collapsed[r].count(n);
  }
  int current_leaf(int r, int n) {
    const auto& nodes = C.trees.at(r).nodes;
    int best = n;
    for (int a = nodes[n].parent; a >= 0; a = nodes[a].parent)
      if (collapsed[r].count(a)) best = a;
    return best;
  }
  std::vector<int> leaves(int r) {
    const auto& nodes = C.trees.at(r).nodes;
    std::vector<int> out, st = {0};
    while (!st.empty()) {
      int n = st.back();
      st.pop_back();
      if (nodes[n].leaf() || collapsed[r].count(n))
        out.push_back(n);
      else {
        st.push_back(nodes[n].right);
        st.push_back(nodes[n].left);
      }
    }
    std::sort(out.begin(), out.end());
    return out;
  }
  LevelCells extract() {
    int N = C.N;
    LevelCells lv;
    for (auto& kv : cubes) {
      int r = kv.first, k = r / (N * N), rem = r % (N * N);
      lv.cells.push_back(Cell{true, rem % N, rem / N, k, kv.second, r, -1});
    }
    for (auto& kv : C.trees) {
      int r = kv.first;
      if (full.count(r)) continue;
      for (int n : leaves(r)) {
        if (kv.second.nodes[n].nfluid > 0)
          lv.cells.push_back(Cell{false, kv.second.ijk[0], kv.second.ijk[1], kv.second.ijk[2], 1, r, n});
        else
          lv.solids.push_back(kv.second.nodes[n].H);
      }
    }
    for (auto& kv : C.trees)
      if (full.count(kv.first) && kv.second.nodes[0].nfluid == 0) lv.solids.push_back(kv.second.nodes[0].H);
    for (int r = 0; r < N * N * N; ++r)
      if (C.kind[r] == UNCUT_SOLID || C.kind[r] == SINGLE_SOLID) {
        int k = r / (N * N), rem = r % (N * N);
        lv.solids.push_back(cube_H(N, rem % N, rem / N, k, 1));
      }
    std::sort(lv.cells.begin(), lv.cells.end(), [](const Cell& a, const Cell& b) {
      if (a.r != b.r) return a.r < b.r;
      return a.nid < b.nid;
    });
    return lv;
  }
  // Size (in background cells) of the current cell holding each background
  // cell: cube size, 1 for a cell split by the BSP, 0 where no fluid cell is.
  std::vector<int16_t> sizes_of_roots() {
    int N = C.N;
    std::vector<int16_t> sz(size_t(N) * N * N, 0);
    for (auto& kv : cubes) {
      int r = kv.first, s = kv.second, k = r / (N * N), rem = r % (N * N), j = rem / N, i = rem % N;
      for (int dk = 0; dk < s; ++dk)
        for (int dj = 0; dj < s; ++dj)
          for (int di = 0; di < s; ++di) sz[ridx(N, i + di, j + dj, k + dk)] = int16_t(s);
    }
    for (auto& kv : C.trees)
      if (!full.count(kv.first) && kv.second.nodes[0].nfluid > 0) sz[kv.first] = 1;
    return sz;
  }
  // 2x2x2 aggregation: a block of 8 cubes of size s merges; with 2:1 balance
  // (balance = true) only if every fluid cell touching the block (faces,
  // edges, corners) has size >= s in the state before this step.
  void aggregate(bool balance) {
    int N = C.N;
    std::vector<int16_t> sz = sizes_of_roots();
    std::vector<std::pair<int, int>> items(cubes.begin(), cubes.end());
    std::sort(items.begin(), items.end());
    std::unordered_map<int, int> nw = cubes;
    for (auto& it : items) {
      int r = it.first, s = it.second, k = r / (N * N), rem = r % (N * N), j = rem / N, i = rem % N;
      int s2 = 2 * s;
      if (i % s2 || j % s2 || k % s2 || i + s2 > N || j + s2 > N || k + s2 > N) continue;
      bool all = true;
      int mem[8];
      int q = 0;
      for (int dk = 0; dk < 2; ++dk)
        for (int dj = 0; dj < 2; ++dj)
          for (int di = 0; di < 2; ++di) {
            int m = ridx(N, i + di * s, j + dj * s, k + dk * s);
            mem[q++] = m;
            auto f = cubes.find(m);
            if (f == cubes.end() || f->second != s) all = false;
          }
      if (!all) continue;
      bool balanced = true;
      for (int kk = std::max(0, k - 1); balance && kk <= std::min(N - 1, k + s2) && balanced; ++kk)
        for (int jj = std::max(0, j - 1); jj <= std::min(N - 1, j + s2) && balanced; ++jj)
          for (int ii = std::max(0, i - 1); ii <= std::min(N - 1, i + s2); ++ii) {
            bool inside = ii >= i && ii < i + s2 && jj >= j && jj < j + s2 && kk >= k && kk < k + s2;
            if (inside) continue;
            int t = sz[ridx(N, ii, jj, kk)];
            if (t != 0 && t < s) {
              balanced = false;
              break;
            }
          }
      if (!balanced) continue;
      for (int m : mem) nw.erase(m);
      nw[r] = s2;
    }
    cubes.swap(nw);
  }
  bool removable(int r, int n) {
    const auto& nodes = C.trees.at(r).nodes;
    const Node& nd = nodes[n];
    if (nd.leaf() || collapsed[r].count(n)) return false;
    if (!is_cur_leaf(r, nd.left) || !is_cur_leaf(r, nd.right)) return false;
    return current_leaf(r, n) == n;
  }
  void remove_cuts(int L) {
    int64_t limit = int64_t(1099511627776LL) / L;
    typedef std::tuple<int64_t, int, int> E;
    std::priority_queue<E, std::vector<E>, std::greater<E>> heap;
    for (auto& kv : C.trees) {
      if (full.count(kv.first)) continue;
      for (int n = 0; n < int(kv.second.nodes.size()); ++n)
        if (removable(kv.first, n)) heap.push(E{kv.second.nodes[n].wq, kv.first, n});
    }
    int64_t acc = 0;
    while (!heap.empty() && acc <= limit) {
      E e = heap.top();
      heap.pop();
      int r = std::get<1>(e), n = std::get<2>(e);
      collapsed[r].insert(n);
      acc += std::get<0>(e);
      const Tree& tr = C.trees.at(r);
      int p = tr.nodes[n].parent;
      if (p >= 0 && removable(r, p)) heap.push(E{tr.nodes[p].wq, r, p});
      if (p < 0) {
        full.insert(r);
        if (tr.nodes[0].nfluid > 0) cubes[r] = 1;
      }
    }
  }
  int cube_containing(int i, int j, int k) {
    int N = C.N;
    for (int s = 1; s <= N; s *= 2) {
      int r = ridx(N, i - i % s, j - j % s, k - k % s);
      auto f = cubes.find(r);
      if (f != cubes.end() && f->second == s) return r;
    }
    return -1;
  }
  // returns (root index, node id or -1 for cube) of the containing cell
  std::pair<int, int> map_cell(const Cell& c) {
    if (c.cube) return {cube_containing(c.i, c.j, c.k), -1};
    if (full.count(c.r)) return {cube_containing(c.i, c.j, c.k), -1};
    return {c.r, current_leaf(c.r, c.nid)};
  }
};

HS cell_H(Ctx& C, const Cell& c) {
  if (c.cube) return cube_H(C.N, c.i, c.j, c.k, c.s);
  return C.trees.at(c.r).nodes[c.nid].H;
}

// ------------------------------------------------------------------ level mesh

struct FaceOcc {
  int pid, sg;
  std::vector<uint64_t> keys;  // packed min key per vertex (cycle order)
  std::vector<V3> xs;          // representative coordinates
};

struct PieceGeom {
  bool cube = false;
  int lo[3], hi[3];
  HS H;
};

void footprint(int N, const HS& H, int lo[3], int hi[3]) {
  for (int a = 0; a < 3; ++a) {
    lo[a] = H[2 * a].first - a * (N + 1);
    hi[a] = H[2 * a + 1].first - a * (N + 1);
  }
}

bool has_h(const HS& H, int pid, int sg) {
  for (auto& h : H)
    if (h.first == pid && h.second == sg) return true;
  return false;
}

double now_s2() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int build_level_mesh(Ctx& C, const LevelCells& lv, LevelMesh& M, std::string& err) {
  const bool tm = std::getenv("FVEM_TIMING") != nullptr;
  double t0 = now_s2();
  auto lap = [&](const char* what) {
    if (tm) std::fprintf(stderr, "   [mesh] %-14s %8.3f s\n", what, now_s2() - t0);
    t0 = now_s2();
  };
  const int N = C.N;
  const Planes& P = C.P;
  int nfl = int(lv.cells.size());
  std::vector<HS> Hs;
  Hs.reserve(nfl + lv.solids.size());
  for (auto& c : lv.cells) Hs.push_back(cell_H(C, c));
  for (auto& s : lv.solids) Hs.push_back(s);
  int npieces = int(Hs.size());
  // polytopes of BSP pieces are kept in the trees; others are rebuilt on demand
  std::vector<const Poly*> cached(npieces, nullptr);
  for (int c = 0; c < nfl; ++c)
    if (!lv.cells[c].cube) cached[c] = &C.trees.at(lv.cells[c].r).nodes[lv.cells[c].nid].poly;
  // registry: root -> pieces (CSR)
  size_t NN = size_t(N) * N * N;
  std::vector<int64_t> rptr(NN + 1, 0);
  std::vector<std::array<int, 6>> fps(npieces);
  for (int p = 0; p < npieces; ++p) {
    int lo[3], hi[3];
    footprint(N, Hs[p], lo, hi);
    fps[p] = {lo[0], lo[1], lo[2], hi[0], hi[1], hi[2]};
    for (int k = lo[2]; k < hi[2]; ++k)
      for (int j = lo[1]; j < hi[1]; ++j)
        for (int i = lo[0]; i < hi[0]; ++i) rptr[ridx(N, i, j, k) + 1]++;
  }
  for (size_t r = 0; r < NN; ++r) rptr[r + 1] += rptr[r];
  std::vector<int> reg(rptr[NN]);
  {
    std::vector<int64_t> fill(rptr.begin(), rptr.end() - 1);
    for (int p = 0; p < npieces; ++p) {
      auto& f = fps[p];
      for (int k = f[2]; k < f[5]; ++k)
        for (int j = f[1]; j < f[4]; ++j)
          for (int i = f[0]; i < f[3]; ++i) reg[fill[ridx(N, i, j, k)]++] = p;
    }
  }
  lap("registry");
  auto getpoly = [&](int p, Poly& tmp) -> const Poly& {
    if (cached[p]) return *cached[p];
    tmp = make_poly(P, Hs[p]);
    return tmp;
  };

  // candidate coordinates by packed min key (first occurrence wins)
  FlatMap cand_id(size_t(nfl) * 4);
  std::vector<uint64_t> cand_key;
  std::vector<V3> cand_x;
  std::vector<std::vector<FaceOcc>> occ(nfl);
  auto minkey = [](const std::vector<Key>& ks) { return *std::min_element(ks.begin(), ks.end()); };

  std::vector<char> iscube(npieces, 0);
  for (int p = 0; p < npieces; ++p) {
    bool cb = Hs[p].size() == 6;
    for (auto& h : Hs[p])
      if (!P.is_grid(h.first)) cb = false;
    iscube[p] = cb;
  }
  std::vector<std::string> errs(nfl);
#pragma omp parallel for schedule(dynamic, 64)
  for (int c = 0; c < nfl; ++c) {
    Poly tmpc;
    const Poly& Pc = getpoly(c, tmpc);
    const HS& H = Hs[c];
    auto& fp = fps[c];
    for (auto& f : Pc.f) {
      int pid = f.pid, sg = f.sg;
      FaceOcc F;
      F.pid = pid;
      F.sg = sg;
      std::vector<uint64_t> fkeys;
      std::vector<V3> fx;
      for (int v : f.cyc) {
        Key k = minkey(Pc.vk[v]);
        fkeys.push_back(pack(k));
        fx.push_back(Pc.v[v]);
      }
      std::vector<int> cands;
      bool wall = false;
      if (P.is_grid(pid)) {
        int a = pid / (N + 1), idx = pid % (N + 1);
        int o = sg > 0 ? idx : idx - 1;
        if (o < 0 || o >= N) {
          wall = true;
        } else {
          int lo[3] = {fp[0], fp[1], fp[2]}, hi[3] = {fp[3], fp[4], fp[5]};
          lo[a] = o;
          hi[a] = o + 1;
          for (int k = lo[2]; k < hi[2]; ++k)
            for (int j = lo[1]; j < hi[1]; ++j)
              for (int i = lo[0]; i < hi[0]; ++i) {
                int r = ridx(N, i, j, k);
                for (int64_t q = rptr[r]; q < rptr[r + 1]; ++q) cands.push_back(reg[q]);
              }
        }
      } else {
        int r = ridx(N, fp[0], fp[1], fp[2]);
        for (int64_t q = rptr[r]; q < rptr[r + 1]; ++q) cands.push_back(reg[q]);
      }
      std::sort(cands.begin(), cands.end());
      cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
      auto push_piece = [&](const std::vector<uint64_t>& ks, const std::vector<V3>& xs) {
        FaceOcc G;
        G.pid = pid;
        G.sg = sg;
        G.keys = ks;
        G.xs = xs;
        occ[c].push_back(std::move(G));
      };
      if (wall) {
        push_piece(fkeys, fx);
        continue;
      }
      V3 nrm = scl(P.n[pid], double(sg));
      std::vector<int> cyc_all(fx.size());
      for (size_t m = 0; m < fx.size(); ++m) cyc_all[m] = int(m);
      double area_f = polygon_area(fx, cyc_all, nrm);
      double tot = 0.0;
      std::vector<uint64_t> fsorted = fkeys;
      std::sort(fsorted.begin(), fsorted.end());
      for (int q : cands) {
        if (q == c) continue;
        if (!has_h(Hs[q], pid, -sg)) continue;
        if (iscube[c] && iscube[q]) {
          int a = pid / (N + 1);
          bool ident = true;
          for (int b = 0; b < 3; ++b)
            if (b != a && (fps[q][b] != fp[b] || fps[q][b + 3] != fp[b + 3])) ident = false;
          if (ident) {
            push_piece(fkeys, fx);
            tot += area_f;
            continue;
          }
        }
        Poly tmpq;
        const Poly& Pq = getpoly(q, tmpq);
        bool same = false;
        for (auto& qf : Pq.f)
          if (qf.pid == pid && qf.sg == -sg) {
            std::vector<uint64_t> qk;
            for (int v : qf.cyc) qk.push_back(pack(minkey(Pq.vk[v])));
            std::sort(qk.begin(), qk.end());
            same = (qk == fsorted);
            break;
          }
        if (same) {
          push_piece(fkeys, fx);
          tot += area_f;
          continue;
        }
        HS Hu = H;
        for (auto& h : Hs[q])
          if (!has_h(H, h.first, h.second)) Hu.push_back(h);
        std::vector<V3> pts;
        std::vector<std::vector<Key>> ks;
        face_polygon(P, Hu, pid, sg, pts, ks);
        if (pts.size() >= 3) {
          std::vector<uint64_t> pk;
          for (auto& kl : ks) pk.push_back(pack(minkey(kl)));
          std::vector<int> cc(pts.size());
          for (size_t m = 0; m < pts.size(); ++m) cc[m] = int(m);
          tot += polygon_area(pts, cc, nrm);
          push_piece(pk, pts);
        }
      }
      // tolerance: relative to the face plus 1e-11 of a background cell face
      // (sliver faces carry the rounding of their long edges)
      if (std::fabs(tot - area_f) > 1e-9 * std::max(area_f, 1e-30) + 1e-11 / (double(N) * N))
        errs[c] = "overlay does not cover a face (cell " + std::to_string(c) + ")";
    }
  }
  lap("overlay");
  for (int c = 0; c < nfl; ++c)
    if (!errs[c].empty()) {
      err = errs[c];
      return 1;
    }
  for (int c = 0; c < nfl; ++c)
    for (auto& F : occ[c]) {
      for (size_t m = 0; m < F.keys.size(); ++m) {
        bool ins;
        cand_id.insert(F.keys[m], int32_t(cand_key.size()), ins);
        if (ins) {
          cand_key.push_back(F.keys[m]);
          cand_x.push_back(F.xs[m]);
        }
      }
      F.xs.clear();
      F.xs.shrink_to_fit();
    }
  lap("cand");
  // global weld (keys ascending; first representative within WELD wins)
  std::vector<int32_t> kord(cand_key.size());
  for (size_t i = 0; i < kord.size(); ++i) kord[i] = int32_t(i);
  // candidate keys are distinct, so any sort gives this order
  __gnu_parallel::sort(kord.begin(), kord.end(), [&](int32_t a, int32_t b) { return cand_key[a] < cand_key[b]; });
  std::vector<int32_t> rep_of(cand_key.size(), -1);  // by candidate id
  std::vector<V3> reps;
  KeyLists bucket(cand_key.size());
  const double inv = 1.0 / (4.0 * WELD);
  auto bkey = [](int64_t a, int64_t b, int64_t c) {
    return uint64_t(a) * 0x9E3779B97F4A7C15ULL ^ uint64_t(b) * 0xC2B2AE3D27D4EB4FULL ^
           uint64_t(c) * 0x165667B19E3779F9ULL;
  };
  for (int32_t ci : kord) {
    const V3 x = cand_x[size_t(ci)];
    int64_t b0 = int64_t(std::floor(x.x * inv)), b1 = int64_t(std::floor(x.y * inv)),
            b2 = int64_t(std::floor(x.z * inv));
    int hit = -1;
    for (int dz = -1; dz <= 1 && hit < 0; ++dz)
      for (int dy = -1; dy <= 1 && hit < 0; ++dy)
        for (int dx = -1; dx <= 1 && hit < 0; ++dx)
          for (int32_t r = bucket.first(bkey(b0 + dx, b1 + dy, b2 + dz)); r >= 0; r = bucket.after(r))
            if (maxabs(reps[size_t(r)], x) <= WELD) {
              hit = r;
              break;
            }
    if (hit < 0) {
      hit = int(reps.size());
      reps.push_back(x);
      bucket.push(bkey(b0, b1, b2), hit);
    }
    rep_of[size_t(ci)] = hit;
  }
  lap("weld");
  // face cycles in welded ids
  std::vector<std::vector<std::pair<std::pair<int, int>, std::vector<int>>>> cf(nfl);
#pragma omp parallel for schedule(dynamic, 256)
  for (int c = 0; c < nfl; ++c)
    for (auto& F : occ[c]) {
      std::vector<int> cyc;
      for (uint64_t k : F.keys) {
        int g = rep_of[size_t(cand_id.find(k))];
        if (cyc.empty() || cyc.back() != g) cyc.push_back(g);
      }
      while (cyc.size() > 1 && cyc.front() == cyc.back()) cyc.pop_back();
      cf[c].push_back({{F.pid, F.sg}, cyc});
    }
  occ.clear();
  occ.shrink_to_fit();
  // T-junctions: vertices inside face edges
  std::vector<char> usedf(reps.size(), 0);
  for (auto& cc : cf)
    for (auto& f : cc)
      for (int g : f.second) usedf[g] = 1;
  std::vector<int> used;
  for (size_t g = 0; g < reps.size(); ++g)
    if (usedf[g]) used.push_back(int(g));
  const double hb = 1.0 / N;
  KeyLists vgrid(reps.size());
  auto cellkey = [&](const V3& x, int64_t& a, int64_t& b, int64_t& c) {
    a = int64_t(std::floor(x.x / hb));
    b = int64_t(std::floor(x.y / hb));
    c = int64_t(std::floor(x.z / hb));
  };
  for (int g : used) {
    int64_t a, b, c;
    cellkey(reps[g], a, b, c);
    vgrid.push(bkey(a, b, c), g);
  }
  lap("cycles+vgrid");
  // unique undirected edges (keys (lo, hi) gathered per cell in parallel,
  // sorted, deduplicated; an edge's index only addresses its split list),
  // split points computed in parallel
  auto ekey = [](int a, int b) {
    return (uint64_t(uint32_t(std::min(a, b))) << 32) | uint32_t(std::max(a, b));
  };
  std::vector<int64_t> koff(size_t(nfl) + 1, 0);
#pragma omp parallel for schedule(static)
  for (int c = 0; c < nfl; ++c) {
    int64_t k = 0;
    for (auto& f : cf[c]) k += int64_t(f.second.size());
    koff[size_t(c) + 1] = k;
  }
  for (int c = 0; c < nfl; ++c) koff[size_t(c) + 1] += koff[size_t(c)];
  std::vector<uint64_t> edges(size_t(koff[size_t(nfl)]));
#pragma omp parallel for schedule(dynamic, 256)
  for (int c = 0; c < nfl; ++c) {
    int64_t k = koff[size_t(c)];
    for (auto& f : cf[c]) {
      const auto& cyc = f.second;
      for (size_t i = 0; i < cyc.size(); ++i) edges[size_t(k++)] = ekey(cyc[i], cyc[(i + 1) % cyc.size()]);
    }
  }
  std::vector<int64_t>().swap(koff);
  __gnu_parallel::sort(edges.begin(), edges.end());
  edges.erase(std::unique(edges.begin(), edges.end()), edges.end());
  std::vector<std::vector<int>> split(edges.size());
#pragma omp parallel for schedule(dynamic, 256)
  for (long long q = 0; q < (long long)edges.size(); ++q) {
    int lo = int(edges[q] >> 32), hi = int(edges[q] & 0xffffffffu);
    const V3 pa = reps[lo], pb = reps[hi];
    V3 e = sub(pb, pa);
    double L2 = dot(e, e), L = std::sqrt(L2);
    V3 mn{std::min(pa.x, pb.x) - 2 * WELD, std::min(pa.y, pb.y) - 2 * WELD, std::min(pa.z, pb.z) - 2 * WELD};
    V3 mx{std::max(pa.x, pb.x) + 2 * WELD, std::max(pa.y, pb.y) + 2 * WELD, std::max(pa.z, pb.z) + 2 * WELD};
    int64_t a0, a1, a2, b0, b1, b2;
    cellkey(mn, a0, a1, a2);
    cellkey(mx, b0, b1, b2);
    std::vector<std::pair<double, int>> res;
    for (int64_t z = a2; z <= b2; ++z)
      for (int64_t y = a1; y <= b1; ++y)
        for (int64_t x = a0; x <= b0; ++x) {
          for (int32_t v = vgrid.first(bkey(x, y, z)); v >= 0; v = vgrid.after(v)) {
            if (v == lo || v == hi) continue;
            V3 w = sub(reps[v], pa);
            double t = dot(w, e) / L2;
            V3 dv = sub(w, scl(e, t));
            double dist = std::sqrt(dot(dv, dv));
            if (dist <= WELD && t * L > WELD && (1.0 - t) * L > WELD) res.push_back({t, v});
          }
        }
    std::sort(res.begin(), res.end());
    for (auto& pr : res) split[q].push_back(pr.second);
  }
#pragma omp parallel for schedule(dynamic, 256)
  for (int c = 0; c < nfl; ++c)
    for (auto& f : cf[c]) {
      std::vector<int> nw;
      auto& cyc = f.second;
      for (size_t i = 0; i < cyc.size(); ++i) {
        int a = cyc[i], b = cyc[(i + 1) % cyc.size()];
        nw.push_back(a);
        int lo = std::min(a, b), hi = std::max(a, b);
        const auto& in = split[size_t(std::lower_bound(edges.begin(), edges.end(), ekey(lo, hi)) - edges.begin())];
        if (a < b)
          nw.insert(nw.end(), in.begin(), in.end());
        else
          nw.insert(nw.end(), in.rbegin(), in.rend());
      }
      cyc.swap(nw);
    }
  lap("tjunction");
  // canonical numbering: by (z, y, x) on the 2^-30 lattice, then raw
  // (z, y, x); keys computed once, the list index last (welded vertices
  // never tie, so it only makes the order independent of the sort used)
  struct NumKey {
    double k[6];
    int i;
  };
  std::vector<NumKey> keys(used.size());
  auto qz = [&](double v) { return std::floor(v * Q30 + 0.5); };
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < int64_t(used.size()); ++i) {
    const V3& a = reps[used[size_t(i)]];
    keys[size_t(i)] = NumKey{{qz(a.z), qz(a.y), qz(a.x), a.z, a.y, a.x}, int(i)};
  }
  __gnu_parallel::sort(keys.begin(), keys.end(), [](const NumKey& a, const NumKey& b) {
    for (int j = 0; j < 6; ++j)
      if (a.k[j] != b.k[j]) return a.k[j] < b.k[j];
    return a.i < b.i;
  });
  std::vector<int> ord(used.size());
  for (size_t i = 0; i < ord.size(); ++i) ord[i] = keys[i].i;
  std::vector<NumKey>().swap(keys);
  std::vector<int> newid(reps.size(), -1);
  M.nv = int(used.size());
  M.V.resize(size_t(3) * M.nv);
  for (size_t r = 0; r < ord.size(); ++r) {
    int g = used[ord[r]];
    newid[g] = int(r);
    M.V[3 * r] = reps[g].x;
    M.V[3 * r + 1] = reps[g].y;
    M.V[3 * r + 2] = reps[g].z;
  }
  M.nc = nfl;
  M.cell_vptr.assign(1, 0);
  M.cell_fptr.assign(1, 0);
  M.face_vptr.assign(1, 0);
  M.cell_v.clear();
  M.face_v.clear();
  M.face_pid.clear();
  M.face_sg.clear();
  // per cell in parallel: faces in new ids, rotated to their smallest id and
  // sorted; then appended in cell order
  std::vector<std::vector<std::tuple<std::vector<int>, int, int>>> cfaces(nfl);
#pragma omp parallel for schedule(dynamic, 256)
  for (int c = 0; c < nfl; ++c) {
    auto& faces = cfaces[c];
    for (auto& f : cf[c]) {
      std::vector<int> ids;
      for (int g : f.second) ids.push_back(newid[g]);
      size_t s = std::min_element(ids.begin(), ids.end()) - ids.begin();
      std::rotate(ids.begin(), ids.begin() + s, ids.end());
      faces.emplace_back(ids, f.first.first, f.first.second);
    }
    std::sort(faces.begin(), faces.end(),
              [](const std::tuple<std::vector<int>, int, int>& a, const std::tuple<std::vector<int>, int, int>& b) {
                return std::get<0>(a) < std::get<0>(b);
              });
    std::vector<std::pair<std::pair<int, int>, std::vector<int>>>().swap(cf[c]);
  }
  for (int c = 0; c < nfl; ++c) {
    auto& faces = cfaces[c];
    std::vector<int> vs;
    for (auto& f : faces) {
      auto& ids = std::get<0>(f);
      M.face_pid.push_back(std::get<1>(f));
      M.face_sg.push_back(int8_t(std::get<2>(f)));
      M.face_v.insert(M.face_v.end(), ids.begin(), ids.end());
      M.face_vptr.push_back(int32_t(M.face_v.size()));
      vs.insert(vs.end(), ids.begin(), ids.end());
    }
    std::sort(vs.begin(), vs.end());
    vs.erase(std::unique(vs.begin(), vs.end()), vs.end());
    M.cell_v.insert(M.cell_v.end(), vs.begin(), vs.end());
    M.cell_vptr.push_back(int32_t(M.cell_v.size()));
    M.cell_fptr.push_back(int32_t(M.face_pid.size()));
    std::vector<std::tuple<std::vector<int>, int, int>>().swap(faces);
  }
  lap("numbering");
  return 0;
}

// ------------------------------------------------------------------ placements

// Placement of point x relative to coarse cell C (the same tests, in the same
// order, as for vertices): a coarse vertex within WELD, else the interior of
// a coarse edge within WELD, else a coarse face (plane within EPS, inside
// every edge), else the cell.  a, b: vertex ids; for a face, a = occurrence.
void classify_in_cell(const LevelMesh& Cm, int C, V3 x, int8_t& type, int32_t& a_out, int32_t& b_out) {
  auto cv = [&](int v) { return V3{Cm.V[3 * v], Cm.V[3 * v + 1], Cm.V[3 * v + 2]}; };
  type = PLACE_CELL;
  a_out = b_out = -1;
  for (int q = Cm.cell_vptr[C]; q < Cm.cell_vptr[C + 1]; ++q)
    if (maxabs(cv(Cm.cell_v[q]), x) <= WELD) {
      type = PLACE_VERTEX;
      a_out = Cm.cell_v[q];
      return;
    }
  for (int f = Cm.cell_fptr[C]; f < Cm.cell_fptr[C + 1]; ++f) {
    int s = Cm.face_vptr[f], e = Cm.face_vptr[f + 1], k = e - s;
    for (int m = 0; m < k; ++m) {
      int a = Cm.face_v[s + m], b = Cm.face_v[s + (m + 1) % k];
      V3 pa = cv(a), ed = sub(cv(b), pa);
      double L2 = dot(ed, ed), L = std::sqrt(L2);
      V3 w = sub(x, pa);
      double t = dot(w, ed) / L2;
      V3 dv = sub(w, scl(ed, t));
      if (t * L > WELD && (1 - t) * L > WELD && std::sqrt(dot(dv, dv)) <= WELD) {
        type = PLACE_EDGE;
        a_out = a;
        b_out = b;
        return;
      }
    }
  }
  for (int f = Cm.cell_fptr[C]; f < Cm.cell_fptr[C + 1]; ++f) {
    int s = Cm.face_vptr[f], e = Cm.face_vptr[f + 1], k = e - s;
    V3 A{0, 0, 0};
    for (int m = 0; m < k; ++m) A = add(A, cross(cv(Cm.face_v[s + m]), cv(Cm.face_v[s + (m + 1) % k])));
    double nA = std::sqrt(dot(A, A));
    V3 n = scl(A, 1.0 / nA);
    V3 p0 = cv(Cm.face_v[s]);
    if (std::fabs(dot(n, sub(x, p0))) > EPS) continue;
    bool inside = true;
    for (int m = 0; m < k; ++m) {
      V3 pm = cv(Cm.face_v[s + m]), pn = cv(Cm.face_v[s + (m + 1) % k]);
      if (dot(cross(sub(pn, pm), sub(x, pm)), n) < -EPS) {
        inside = false;
        break;
      }
    }
    if (inside) {
      type = PLACE_FACE;
      a_out = f;
      return;
    }
  }
}

void compute_placement(const LevelMesh& F, const LevelMesh& Cm, Placement& pl) {
  int nf = F.nv;
  pl.type.assign(nf, PLACE_CELL);
  pl.cell.assign(nf, -1);
  pl.a.assign(nf, -1);
  pl.b.assign(nf, -1);
  std::vector<int> vcell(nf, -1);
  for (int c = 0; c < F.nc; ++c)
    for (int q = F.cell_vptr[c]; q < F.cell_vptr[c + 1]; ++q)
      if (vcell[F.cell_v[q]] < 0) vcell[F.cell_v[q]] = c;
#pragma omp parallel for schedule(dynamic, 1024)
  for (int v = 0; v < nf; ++v) {
    V3 x{F.V[3 * v], F.V[3 * v + 1], F.V[3 * v + 2]};
    int C = F.parent[vcell[v]];
    pl.cell[v] = C;
    classify_in_cell(Cm, C, x, pl.type[v], pl.a[v], pl.b[v]);
  }
}

}  // namespace

void classify_point(const LevelMesh& Cm, int C, const double* x, int8_t& type, int32_t& a, int32_t& b) {
  classify_in_cell(Cm, C, V3{x[0], x[1], x[2]}, type, a, b);
}

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

int build_topology(int N, const double* tris, int ntri, int L, bool balance, Topology& out, std::string& err,
                   bool naive) {
  const bool tm = std::getenv("FVEM_TIMING") != nullptr;
  double t0 = now_s();
  auto lap = [&](const char* what) {
    if (tm) std::fprintf(stderr, "[fvem topo] %-14s %8.3f s\n", what, now_s() - t0);
    t0 = now_s();
  };
  if (N < 2 || N > 1024 || L < 1 || L > 12 || ntri < 0) {
    err = "invalid grid size, level count or triangle count";
    return 1;
  }
  Ctx C;
  C.N = N;
  C.tris.resize(ntri);
  for (int t = 0; t < ntri; ++t)
    for (int q = 0; q < 3; ++q)
      C.tris[t][q] = V3{tris[9 * t + 3 * q], tris[9 * t + 3 * q + 1], tris[9 * t + 3 * q + 2]};
  Planes& P = C.P;
  P.N = N;
  P.ngrid = 3 * (N + 1);
  P.n.assign(P.ngrid + ntri, V3{0, 0, 0});
  P.d.assign(P.ngrid + ntri, 0.0);
  for (int a = 0; a < 3; ++a)
    for (int i = 0; i <= N; ++i) {
      int pid = a * (N + 1) + i;
      P.n[pid] = V3{a == 0 ? 1.0 : 0.0, a == 1 ? 1.0 : 0.0, a == 2 ? 1.0 : 0.0};
      P.d[pid] = -(double(i) / double(N));
    }
  for (int t = 0; t < ntri; ++t) {
    V3 c = cross(sub(C.tris[t][1], C.tris[t][0]), sub(C.tris[t][2], C.tris[t][0]));
    double Ln = std::sqrt((c.x * c.x + c.y * c.y) + c.z * c.z);
    if (!(Ln > 0)) {
      err = "degenerate triangle " + std::to_string(t);
      return 1;
    }
    V3 n{c.x / Ln, c.y / Ln, c.z / Ln};
    P.n[P.ngrid + t] = n;
    P.d[P.ngrid + t] = -dot(n, C.tris[t][0]);
  }
  build_cut_grid(C);
  lap("cut grid");
  out = Topology();
  out.N = N;
  out.L = L;
  out.total_area = C.total_area;
  out.n_trees = int64_t(C.trees.size());
  HState st(C);
  std::vector<LevelCells> lcs;
  lcs.push_back(st.extract());
  for (int l = 1; l < L; ++l) {
    st.aggregate(balance);
    st.remove_cuts(L);
    LevelCells nl = st.extract();
    std::map<std::pair<int, int>, int> pos;
    for (int c = 0; c < int(nl.cells.size()); ++c) pos[{nl.cells[c].r, nl.cells[c].nid}] = c;
    auto& prev = lcs.back();
    prev.parent.resize(prev.cells.size());
    for (size_t c = 0; c < prev.cells.size(); ++c) {
      auto key = st.map_cell(prev.cells[c]);
      auto f = pos.find(key);
      if (f == pos.end()) {
        err = "hierarchy is not nested";
        return 1;
      }
      prev.parent[c] = f->second;
    }
    lcs.push_back(std::move(nl));
  }
  lap("hierarchy");
  out.levels.resize(L);
  for (int l = 0; l < L; ++l) {
    if (build_level_mesh(C, lcs[l], out.levels[l], err)) return 1;
    out.levels[l].parent = lcs[l].parent;
    lap("level mesh");
    if (out.levels[l].nc == 0) {
      err = "level " + std::to_string(l) + " has no fluid cell";
      return 1;
    }
  }
  out.place.resize(L > 0 ? L - 1 : 0);
  for (int l = 0; l + 1 < L; ++l) {
    compute_placement(out.levels[l], out.levels[l + 1], out.place[l]);
    if (naive)  // Eq. 16: only coincident vertices are copied; every other new vertex uses its parent cell
      for (size_t v = 0; v < out.place[l].type.size(); ++v)
        if (out.place[l].type[v] == PLACE_EDGE || out.place[l].type[v] == PLACE_FACE) {
          out.place[l].type[v] = PLACE_CELL;
          out.place[l].a[v] = out.place[l].b[v] = -1;
        }
  }
  lap("placement");
  return 0;
}

}  // namespace fvem
