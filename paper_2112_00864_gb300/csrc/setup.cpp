// Host-side setup of the bcfmm library: mesh checks, element quadrature,
// the adaptive octree, per-task interaction / extended-neighbour lists, the
// near element-pair search and the translation tables.  FP64 throughout.
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "internal.h"

namespace bcfmm {

static double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

void MultiIndex::init(int P_) {
  P = P_;
  n = nterms(P);
  a.resize(n); b.resize(n); c.resize(n);
  lut.assign((P + 1) * (P + 1) * (P + 1), -1);
  int q = 0;
  for (int d = 0; d <= P; ++d)
    for (int i = d; i >= 0; --i)
      for (int j = d - i; j >= 0; --j) {
        int k = d - i - j;
        a[q] = i; b[q] = j; c[q] = k;
        lut[(i * (P + 1) + j) * (P + 1) + k] = q;
        ++q;
      }
}

// ---------------------------------------------------------------- geometry
static inline void vsub(const double* a, const double* b, double* o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static inline double vdot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void vcross(const double* a, const double* b, double* o) {
  o[0] = a[1] * b[2] - a[2] * b[1]; o[1] = a[2] * b[0] - a[0] * b[2]; o[2] = a[0] * b[1] - a[1] * b[0];
}

std::string setup_mesh(HostSetup& H, const double* verts, int64_t nvert, const int32_t* tets,
                       int64_t ntet, const int32_t* tris, int64_t ntri, bool* mesh_err) {
  *mesh_err = false;
  H.ntet = ntet; H.ntri = ntri;
  H.tet_v.resize(12 * ntet); H.tri_v.resize(9 * ntri);
  H.tet_vol.resize(ntet); H.tri_area.resize(ntri);
  for (int64_t i = 0; i < 3 * nvert; ++i)
    if (!std::isfinite(verts[i])) { *mesh_err = true; return "vertex " + std::to_string(i / 3) + " is not finite"; }
  for (int64_t t = 0; t < ntet; ++t) {
    for (int q = 0; q < 4; ++q) {
      int32_t v = tets[4 * t + q];
      if (v < 0 || v >= nvert) return "tet " + std::to_string(t) + " has vertex id out of range";
      std::memcpy(&H.tet_v[12 * t + 3 * q], verts + 3 * (int64_t)v, 3 * sizeof(double));
    }
    const double* v = &H.tet_v[12 * t];
    double a[3], b[3], c[3], n[3];
    vsub(v + 3, v, a); vsub(v + 6, v, b); vsub(v + 9, v, c); vcross(a, b, n);
    H.tet_vol[t] = std::fabs(vdot(n, c)) / 6.0;
    if (!(H.tet_vol[t] > 0)) { *mesh_err = true; return "tet " + std::to_string(t) + " has zero volume"; }
  }
  for (int64_t t = 0; t < ntri; ++t) {
    for (int q = 0; q < 3; ++q) {
      int32_t v = tris[3 * t + q];
      if (v < 0 || v >= nvert) return "triangle " + std::to_string(t) + " has vertex id out of range";
      std::memcpy(&H.tri_v[9 * t + 3 * q], verts + 3 * (int64_t)v, 3 * sizeof(double));
    }
    const double* v = &H.tri_v[9 * t];
    double a[3], b[3], n[3];
    vsub(v + 3, v, a); vsub(v + 6, v, b); vcross(a, b, n);
    H.tri_area[t] = 0.5 * std::sqrt(vdot(n, n));
    if (!(H.tri_area[t] > 0)) { *mesh_err = true; return "triangle " + std::to_string(t) + " has zero area"; }
  }
  // element quadrature: tet degree-2 4-point rule, triangle interior 3-point rule
  const double ta = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, tb = (5.0 - std::sqrt(5.0)) / 20.0;
  H.qp[0].resize(12 * ntet); H.qw[0].resize(4 * ntet);
  for (int64_t t = 0; t < ntet; ++t) {
    const double* v = &H.tet_v[12 * t];
    for (int q = 0; q < 4; ++q) {
      for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int i = 0; i < 4; ++i) s += (i == q ? ta : tb) * v[3 * i + k];
        H.qp[0][3 * (4 * t + q) + k] = s;
      }
      H.qw[0][4 * t + q] = 0.25 * H.tet_vol[t];
    }
  }
  H.qp[1].resize(9 * ntri); H.qw[1].resize(3 * ntri);
  for (int64_t t = 0; t < ntri; ++t) {
    const double* v = &H.tri_v[9 * t];
    for (int q = 0; q < 3; ++q) {
      for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int i = 0; i < 3; ++i) s += (i == q ? 2.0 / 3.0 : 1.0 / 6.0) * v[3 * i + k];
        H.qp[1][3 * (3 * t + q) + k] = s;
      }
      H.qw[1][3 * t + q] = H.tri_area[t] / 3.0;
    }
  }
  return "";
}

// -------------------------------------------------------------------- tree
// Root: bounding box of all element vertices, half width R0 = largest half
// extent; level-l box (i,j,k): side s = 2 R0 / 2^l, centre lo + (i+1/2) s.
// A box holding more than leaf_size points (both classes) is split; a point
// goes to the upper child along every axis where it is >= the box centre.
void build_tree(HostSetup& H, int leaf_size) {
  double t0 = now_s();
  double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
  for (size_t i = 0; i < H.tet_v.size(); ++i) { int a = i % 3; lo[a] = std::min(lo[a], H.tet_v[i]); hi[a] = std::max(hi[a], H.tet_v[i]); }
  for (size_t i = 0; i < H.tri_v.size(); ++i) { int a = i % 3; lo[a] = std::min(lo[a], H.tri_v[i]); hi[a] = std::max(hi[a], H.tri_v[i]); }
  double R0 = 0;
  for (int a = 0; a < 3; ++a) R0 = std::max(R0, 0.5 * (hi[a] - lo[a]));
  H.R0 = R0;
  for (int a = 0; a < 3; ++a) H.lo[a] = 0.5 * (lo[a] + hi[a]) - R0;
  int64_t np[2] = {4 * H.ntet, 3 * H.ntri};
  for (int c = 0; c < 2; ++c) { H.perm[c].resize(np[c]); for (int64_t i = 0; i < np[c]; ++i) H.perm[c][i] = (int)i; }
  H.box.clear();
  HostBox root{};
  root.level = 0; root.parent = -1; root.child0 = -1; root.nchild = 0; root.octant = 0;
  root.pt0[0] = 0; root.pt1[0] = (int)np[0]; root.pt0[1] = 0; root.pt1[1] = (int)np[1];
  root.s = 2.0 * R0;
  for (int a = 0; a < 3; ++a) root.c[a] = H.lo[a] + 0.5 * root.s;
  H.box.push_back(root);
  H.lvl_off = {0, 1};
  std::vector<int> tmp(std::max(np[0], np[1]) + 1);
  for (int level = 0; level < kMaxLevel; ++level) {
    int b0 = H.lvl_off[level], b1 = H.lvl_off[level + 1];
    for (int bi = b0; bi < b1; ++bi) {
      HostBox B = H.box[bi];
      int cnt = (B.pt1[0] - B.pt0[0]) + (B.pt1[1] - B.pt0[1]);
      if (cnt <= leaf_size) continue;
      int start[2][9];
      for (int c = 0; c < 2; ++c) {
        const double* P = H.qp[c].data();
        int* pm = H.perm[c].data();
        int cnt8[8] = {0};
        for (int q = B.pt0[c]; q < B.pt1[c]; ++q) {
          const double* x = P + 3 * (int64_t)pm[q];
          int o = (x[0] >= B.c[0]) | ((x[1] >= B.c[1]) << 1) | ((x[2] >= B.c[2]) << 2);
          cnt8[o]++;
        }
        start[c][0] = B.pt0[c];
        for (int o = 0; o < 8; ++o) start[c][o + 1] = start[c][o] + cnt8[o];
        int pos[8];
        for (int o = 0; o < 8; ++o) pos[o] = start[c][o];
        for (int q = B.pt0[c]; q < B.pt1[c]; ++q) {
          const double* x = P + 3 * (int64_t)pm[q];
          int o = (x[0] >= B.c[0]) | ((x[1] >= B.c[1]) << 1) | ((x[2] >= B.c[2]) << 2);
          tmp[pos[o]++] = pm[q];
        }
        std::memcpy(pm + B.pt0[c], tmp.data() + B.pt0[c], sizeof(int) * (B.pt1[c] - B.pt0[c]));
      }
      H.box[bi].child0 = (int)H.box.size();
      for (int o = 0; o < 8; ++o) {
        if (start[0][o + 1] - start[0][o] + start[1][o + 1] - start[1][o] == 0) continue;
        HostBox C{};
        C.level = level + 1; C.parent = bi; C.child0 = -1; C.nchild = 0; C.octant = o;
        C.ijk[0] = 2 * B.ijk[0] + (o & 1); C.ijk[1] = 2 * B.ijk[1] + ((o >> 1) & 1); C.ijk[2] = 2 * B.ijk[2] + ((o >> 2) & 1);
        for (int c = 0; c < 2; ++c) { C.pt0[c] = start[c][o]; C.pt1[c] = start[c][o + 1]; }
        C.s = std::ldexp(2.0 * R0, -(level + 1));
        for (int a = 0; a < 3; ++a) C.c[a] = H.lo[a] + ((double)C.ijk[a] + 0.5) * C.s;
        H.box.push_back(C);
        H.box[bi].nchild++;
      }
    }
    if ((int)H.box.size() == b1) break;
    H.lvl_off.push_back((int)H.box.size());
  }
  H.nlevels = (int)H.lvl_off.size() - 1;
  for (int c = 0; c < 2; ++c) {
    H.leaf_of[c].assign(np[c], -1);
    for (size_t bi = 0; bi < H.box.size(); ++bi) {
      const HostBox& B = H.box[bi];
      if (B.nchild) continue;
      for (int q = B.pt0[c]; q < B.pt1[c]; ++q) H.leaf_of[c][q] = (int)bi;
    }
  }
  H.seconds_tree = now_s() - t0;
}

// ------------------------------------------------------------------- lists
static inline uint64_t box_key(int level, int64_t i, int64_t j, int64_t k) {
  return ((uint64_t)(level + 1) << 57) | ((uint64_t)i << 38) | ((uint64_t)j << 19) | (uint64_t)k;
}

// Same-level boxes B, C are neighbours when eta = sqrt(3)/|o| > eta0 with
// o = ijk_B - ijk_C, i.e. |o|^2 eta0^2 < 3 (Eq. def:neighbors with the box
// circumradius as rho).
static std::vector<std::array<int, 3>> neighbour_offsets(double eta0) {
  std::vector<std::array<int, 3>> out;
  const int R = (int)std::floor(std::sqrt(3.0) / eta0) + 1;
  for (int z = -R; z <= R; ++z)
    for (int y = -R; y <= R; ++y)
      for (int x = -R; x <= R; ++x)
        if ((double)(x * x + y * y + z * z) * eta0 * eta0 < 3.0) out.push_back({x, y, z});
  return out;
}

void build_lists(HostSetup& H, double eta0) {
  double t0 = now_s();
  const auto NB = neighbour_offsets(eta0);
  auto is_nb = [&](int64_t dx, int64_t dy, int64_t dz) { return (double)(dx * dx + dy * dy + dz * dz) * eta0 * eta0 < 3.0; };
  std::unordered_map<uint64_t, int> idx;
  idx.reserve(H.box.size() * 2);
  for (size_t bi = 0; bi < H.box.size(); ++bi) {
    const HostBox& B = H.box[bi];
    idx[box_key(B.level, B.ijk[0], B.ijk[1], B.ijk[2])] = (int)bi;
  }
  auto find = [&](int level, int64_t i, int64_t j, int64_t k) -> int {
    int64_t lim = (int64_t)1 << level;
    if (i < 0 || j < 0 || k < 0 || i >= lim || j >= lim || k >= lim) return -1;
    auto it = idx.find(box_key(level, i, j, k));
    return it == idx.end() ? -1 : it->second;
  };
  const int nb = (int)H.box.size();
  // geometric lists (class independent)
  std::vector<std::vector<int>> nearb(nb), vlist(nb);
  for (int bi = 0; bi < nb; ++bi) {
    const HostBox& B = H.box[bi];
    if (B.nchild == 0) {
      // N*: all points in neighbour subtrees at the leaf's level ...
      for (const auto& o : NB) {
        int c = find(B.level, B.ijk[0] + o[0], B.ijk[1] + o[1], B.ijk[2] + o[2]);
        if (c >= 0) nearb[bi].push_back(c);
      }
      // ... and every coarser leaf that neighbours an ancestor
      for (int a = B.parent; a >= 0; a = H.box[a].parent) {
        const HostBox& A = H.box[a];
        for (const auto& o : NB) {
          int c = find(A.level, A.ijk[0] + o[0], A.ijk[1] + o[1], A.ijk[2] + o[2]);
          if (c >= 0 && H.box[c].nchild == 0) nearb[bi].push_back(c);
        }
      }
    }
    if (B.level >= 2) {
      const HostBox& P = H.box[B.parent];
      for (const auto& o : NB) {
        int q = find(P.level, P.ijk[0] + o[0], P.ijk[1] + o[1], P.ijk[2] + o[2]);
        if (q < 0) continue;
        const HostBox& Q = H.box[q];
        for (int c = Q.child0; c < Q.child0 + Q.nchild; ++c) {
          const HostBox& C = H.box[c];
          if (is_nb(B.ijk[0] - C.ijk[0], B.ijk[1] - C.ijk[1], B.ijk[2] - C.ijk[2])) continue;
          vlist[bi].push_back(c);
        }
      }
    }
  }
  // compact codes of the interaction offsets that occur
  std::unordered_map<int64_t, int> code_of;
  H.offsets.clear();
  auto code = [&](int ox, int oy, int oz) -> int {
    const int64_t key = ((int64_t)(ox + 64) << 16) | ((int64_t)(oy + 64) << 8) | (int64_t)(oz + 64);
    auto it = code_of.find(key);
    if (it != code_of.end()) return it->second;
    const int c = (int)(H.offsets.size() / 3);
    H.offsets.push_back(ox); H.offsets.push_back(oy); H.offsets.push_back(oz);
    code_of[key] = c;
    return c;
  };
  static const int cls[3][2] = {{0, 0}, {0, 1}, {1, 0}};   // {source class, target class}
  for (int t = 0; t < 3; ++t) {
    HostTask& T = H.task[t];
    T = HostTask();
    T.src_cls = cls[t][0]; T.tgt_cls = cls[t][1];
    int sc = T.src_cls, tc = T.tgt_cls;
    auto nsrc = [&](int b) { return H.box[b].pt1[sc] - H.box[b].pt0[sc]; };
    auto ntgt = [&](int b) { return H.box[b].pt1[tc] - H.box[b].pt0[tc]; };
    // far-field targets: VtV's local expansions also serve VtB (same source
    // class, so the same interaction lists): VtV covers every box with tet
    // or triangle points, and VtB evaluated right after VtV reuses them
    auto ftgt = [&](int b) {
      return t == 0 ? (H.box[b].pt1[0] - H.box[b].pt0[0]) + (H.box[b].pt1[1] - H.box[b].pt0[1]) : ntgt(b);
    };
    T.near_off.push_back(0);
    T.run_off.push_back(0);
    T.vl_off.push_back(0);
    T.m2m_parent.assign(H.nlevels, {});
    T.l2l_child.assign(H.nlevels, {});
    for (int bi = 0; bi < nb; ++bi) {
      const HostBox& B = H.box[bi];
      if (B.nchild == 0 && ntgt(bi) > 0) {
        // every target leaf is listed (its far field is evaluated here too)
        for (int c : nearb[bi]) if (nsrc(c) > 0) T.near_box.push_back(c);
        T.p2p_leaf.push_back(bi);
        T.near_off.push_back((int)T.near_box.size());
        // the same sources as merged runs of the sorted point array; for
        // VtV the leaf's own points come first (the only run that can hold
        // the target point itself)
        std::vector<std::pair<int, int>> rr;
        int self_s = -1, self_e = -1;
        for (int c : nearb[bi]) {
          if (nsrc(c) == 0) continue;
          const int s0 = H.box[c].pt0[sc], s1 = H.box[c].pt1[sc];
          if (sc == tc && c == bi) { self_s = s0; self_e = s1; continue; }
          rr.push_back({s0, s1});
        }
        std::sort(rr.begin(), rr.end());
        if (self_s >= 0) { T.runs.push_back(self_s); T.runs.push_back(self_e); }
        T.self_len.push_back(self_s >= 0 ? self_e - self_s : 0);
        for (size_t k = 0; k < rr.size(); ++k) {
          if (k > 0 && T.runs.back() == rr[k].first && (int)T.runs.size() / 2 > T.run_off.back() + (self_s >= 0 ? 1 : 0)) {
            T.runs.back() = rr[k].second;
          } else {
            T.runs.push_back(rr[k].first); T.runs.push_back(rr[k].second);
          }
        }
        T.run_off.push_back((int)T.runs.size() / 2);
      }
      if (B.nchild == 0 && nsrc(bi) > 0) T.p2m_leaf.push_back(bi);
      if (B.nchild > 0 && nsrc(bi) > 0) T.m2m_parent[B.level].push_back(bi);
      if (B.level >= 2 && ftgt(bi) > 0) {
        T.m2l_tgt.push_back(bi);
        for (int c : vlist[bi]) {
          if (nsrc(c) == 0) continue;
          const HostBox& C = H.box[c];
          int ox = (int)(B.ijk[0] - C.ijk[0]), oy = (int)(B.ijk[1] - C.ijk[1]), oz = (int)(B.ijk[2] - C.ijk[2]);
          T.vl_src.push_back(c);
          T.vl_code.push_back((uint16_t)code(ox, oy, oz));
        }
        T.vl_off.push_back((int)T.vl_src.size());
        if (B.level >= 3) T.l2l_child[B.level].push_back(bi);
        if (B.nchild == 0 && ntgt(bi) > 0) T.l2p_leaf.push_back(bi);
      }
    }
  }
  H.seconds_lists = now_s() - t0;
}

// Tiles of the tensor-core interaction phase: M2L targets grouped by
// (expansion order of their level, octant in the parent), tile_m per tile,
// levels of equal order and boxes in tree order inside a group (the
// box-scaled translation table of an offset serves every level, and
// same-octant boxes share the possible offsets); per tile the offsets that
// occur, each with the source box of every row.  box_q: order per box;
// targets whose order exceeds qmax get no tile (CUDA-core M2L).
void build_tc_tiles(HostSetup& H, int t, int tile_m, const std::vector<int>& box_q, int qmax) {
  HostTask& T = H.task[t];
  std::vector<int> order;
  for (int i = 0; i < (int)T.m2l_tgt.size(); ++i)
    if (box_q[T.m2l_tgt[i]] <= qmax) order.push_back(i);
  const int n = (int)order.size();
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    const int bx = T.m2l_tgt[x], by = T.m2l_tgt[y];
    if (box_q[bx] != box_q[by]) return box_q[bx] < box_q[by];
    return H.box[bx].octant < H.box[by].octant;
  });
  T.tc_tile_tgt.clear(); T.tc_tile_off.assign(1, 0); T.tc_ent_code.clear(); T.tc_ent_src.clear();
  T.tc_tile_q.clear();
  int i = 0;
  while (i < n) {
    const int f = T.m2l_tgt[order[i]];
    const HostBox& F = H.box[f];
    int j = i;
    std::vector<int> rows;
    while (j < n && (int)rows.size() < tile_m) {
      const int b = T.m2l_tgt[order[j]];
      if (box_q[b] != box_q[f] || H.box[b].octant != F.octant) break;
      rows.push_back(order[j]);
      ++j;
    }
    T.tc_tile_q.push_back(box_q[f]);
    std::unordered_map<int, int> ent_of;
    std::vector<std::pair<int, std::vector<int>>> ents;
    for (int r = 0; r < (int)rows.size(); ++r) {
      const int k = rows[r];
      for (int e = T.vl_off[k]; e < T.vl_off[k + 1]; ++e) {
        const int code = T.vl_code[e];
        auto it = ent_of.find(code);
        int idx;
        if (it == ent_of.end()) {
          idx = (int)ents.size();
          ent_of[code] = idx;
          ents.push_back({code, std::vector<int>(tile_m, -1)});
        } else {
          idx = it->second;
        }
        ents[idx].second[r] = T.vl_src[e];
      }
    }
    std::sort(ents.begin(), ents.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
    for (int r = 0; r < tile_m; ++r) T.tc_tile_tgt.push_back(r < (int)rows.size() ? T.m2l_tgt[rows[r]] : -1);
    for (auto& en : ents) {
      T.tc_ent_code.push_back(en.first);
      T.tc_ent_src.insert(T.tc_ent_src.end(), en.second.begin(), en.second.end());
    }
    T.tc_tile_off.push_back((int)T.tc_ent_code.size());
    i = j;
  }
}

// ------------------------------------------------------------ near pairs
// near iff eta = (rho_t + rho_s)/|x_t - x_s| > eta_ns (eta = inf for equal
// centres), x = centroid, rho = largest vertex distance from the centroid.
static void centre_radius(const double* v, int nv, double* c, double* rho) {
  c[0] = c[1] = c[2] = 0;
  for (int i = 0; i < nv; ++i) for (int k = 0; k < 3; ++k) c[k] += v[3 * i + k] / nv;
  double r = 0;
  for (int i = 0; i < nv; ++i) { double d[3]; vsub(v + 3 * i, c, d); double l = std::sqrt(vdot(d, d)); if (l > r) r = l; }
  *rho = r;
}

namespace {
struct ElemSet {
  int nv = 0;
  int64_t n = 0;
  std::vector<double> c, rho;
  std::vector<int> lev;
};

// Elements bucketed by size level; grid g holds every element with
// rho <= R0 2^-g in cells of side 2 R0 2^-g / eta.
struct LevelGrids {
  double cell[kMaxLevel + 8];
  int maxlev = 0;
  std::vector<std::unordered_map<uint64_t, std::vector<int>>> g;
};
}  // namespace

static int size_level(double rho, double R0) {
  int l = (int)std::floor(std::log2(R0 / rho));
  return std::max(0, std::min(l, kMaxLevel + 6));
}

static uint64_t cell_key(int64_t i, int64_t j, int64_t k) {
  return ((uint64_t)(i & 0x1FFFFF) << 42) | ((uint64_t)(j & 0x1FFFFF) << 21) | (uint64_t)(k & 0x1FFFFF);
}

static void make_elems(const std::vector<double>& V, int nv, int64_t n, double R0, ElemSet& E) {
  E.nv = nv; E.n = n;
  E.c.resize(3 * n); E.rho.resize(n); E.lev.resize(n);
  for (int64_t i = 0; i < n; ++i) {
    centre_radius(&V[3 * nv * i], nv, &E.c[3 * i], &E.rho[i]);
    E.lev[i] = size_level(E.rho[i], R0);
  }
}

static void make_grids(const ElemSet& E, double R0, const double* lo, double eta, LevelGrids& G) {
  G.maxlev = 0;
  for (int64_t i = 0; i < E.n; ++i) G.maxlev = std::max(G.maxlev, E.lev[i]);
  G.g.assign(G.maxlev + 1, {});
  for (int l = 0; l <= G.maxlev; ++l) G.cell[l] = 2.0 * std::ldexp(R0, -l) / eta;
  for (int64_t i = 0; i < E.n; ++i)
    for (int l = 0; l <= E.lev[i]; ++l) {
      int64_t ci = (int64_t)std::floor((E.c[3 * i] - lo[0]) / G.cell[l]);
      int64_t cj = (int64_t)std::floor((E.c[3 * i + 1] - lo[1]) / G.cell[l]);
      int64_t ck = (int64_t)std::floor((E.c[3 * i + 2] - lo[2]) / G.cell[l]);
      G.g[l][cell_key(ci, cj, ck)].push_back((int)i);
    }
}

static bool is_near_pair(const ElemSet& A, int64_t a, const ElemSet& B, int64_t b, double eta) {
  double d[3];
  vsub(&A.c[3 * a], &B.c[3 * b], d);
  double dist = std::sqrt(vdot(d, d));
  if (dist == 0.0) return true;
  return (A.rho[a] + B.rho[b]) / dist > eta;
}

// pairs (q in Q, e in E) with rho_e <= rho_q: query Q against E's grids
static void query_pairs(const ElemSet& Q, const ElemSet& E, const LevelGrids& G, const double* lo, double eta,
                        bool strict_smaller, std::vector<std::vector<int>>& out) {
  out.assign(Q.n, {});
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t q = 0; q < Q.n; ++q) {
    int l = std::min(Q.lev[q], G.maxlev);
    const double* c = &Q.c[3 * q];
    int64_t ci = (int64_t)std::floor((c[0] - lo[0]) / G.cell[l]);
    int64_t cj = (int64_t)std::floor((c[1] - lo[1]) / G.cell[l]);
    int64_t ck = (int64_t)std::floor((c[2] - lo[2]) / G.cell[l]);
    for (int dz = -1; dz <= 1; ++dz) for (int dy = -1; dy <= 1; ++dy) for (int dx = -1; dx <= 1; ++dx) {
      auto it = G.g[l].find(cell_key(ci + dx, cj + dy, ck + dz));
      if (it == G.g[l].end()) continue;
      for (int e : it->second) {
        if (strict_smaller ? !(E.rho[e] < Q.rho[q]) : !(E.rho[e] <= Q.rho[q])) continue;
        if (is_near_pair(Q, q, E, e, eta)) out[q].push_back(e);
      }
    }
  }
}

void find_near_pairs(HostSetup& H, double eta_ns) {
  double t0 = now_s();
  ElemSet tet, tri;
  make_elems(H.tet_v, 4, H.ntet, H.R0, tet);
  make_elems(H.tri_v, 3, H.ntri, H.R0, tri);
  const ElemSet* sets[2] = {&tet, &tri};
  LevelGrids grids[2];
  make_grids(tet, H.R0, H.lo, eta_ns, grids[0]);
  make_grids(tri, H.R0, H.lo, eta_ns, grids[1]);
  for (int t = 0; t < 3; ++t) {
    HostTask& T = H.task[t];
    const ElemSet& Tg = *sets[T.tgt_cls];
    const ElemSet& Sr = *sets[T.src_cls];
    // case A: rho_s <= rho_t, found from the targets; case B: rho_s > rho_t, from the sources
    std::vector<std::vector<int>> A, B;
    query_pairs(Tg, Sr, grids[T.src_cls], H.lo, eta_ns, false, A);
    query_pairs(Sr, Tg, grids[T.tgt_cls], H.lo, eta_ns, true, B);
    for (int64_t s = 0; s < Sr.n; ++s) for (int tt : B[s]) A[tt].push_back((int)s);
    T.cor_off.assign(Tg.n + 1, 0);
    for (int64_t i = 0; i < Tg.n; ++i) {
      std::sort(A[i].begin(), A[i].end());
      T.cor_off[i + 1] = T.cor_off[i] + (int64_t)A[i].size();
    }
    T.cor_col.resize(T.cor_off[Tg.n]);
    for (int64_t i = 0; i < Tg.n; ++i) std::copy(A[i].begin(), A[i].end(), T.cor_col.begin() + T.cor_off[i]);
  }
  H.seconds_near = now_s() - t0;
}

// ---------------------------------------------------------------- batches
void build_p2p_chunks(const HostSetup& H, int t, int64_t chunk, P2pChunks& out) {
  const HostTask& T = H.task[t];
  struct Blk { int leaf, self, grp, chunk, nt; int64_t ns; std::vector<int> runs; };
  std::vector<Blk> blk;
  out = P2pChunks();
  for (size_t i = 0; i < T.p2p_leaf.size(); ++i) {
    int64_t ns = 0;
    for (int r = T.run_off[i]; r < T.run_off[i + 1]; ++r) ns += T.runs[2 * r + 1] - T.runs[2 * r];
    const HostBox& B = H.box[T.p2p_leaf[i]];
    const int nt = B.pt1[T.tgt_cls] - B.pt0[T.tgt_cls];
    const int nch = (int)std::max<int64_t>(1, (ns + chunk - 1) / chunk);
    const int64_t per = (ns + nch - 1) / nch;
    const int g = nch > 1 ? (int)out.grp_row.size() : -1;
    if (nch > 1) {
      out.grp_row.push_back(out.rows);
      out.grp_n.push_back(nch);
      out.rows += nch;
    }
    Blk cur{T.p2p_leaf[i], T.self_len[i], g, 0, nt, 0, {}};
    for (int r = T.run_off[i]; r < T.run_off[i + 1]; ++r) {
      int s0 = T.runs[2 * r];
      const int e0 = T.runs[2 * r + 1];
      while (s0 < e0) {
        // the leaf's own run (first in a VtV list) is never cut
        const bool whole = cur.chunk + 1 == nch || (r == T.run_off[i] && T.self_len[i] > 0);
        const int take = whole ? e0 - s0 : (int)std::min<int64_t>(e0 - s0, per - cur.ns);
        cur.runs.push_back(s0);
        cur.runs.push_back(s0 + take);
        cur.ns += take;
        s0 += take;
        if (cur.chunk + 1 < nch && cur.ns >= per) {
          const int c = cur.chunk + 1;
          blk.push_back(std::move(cur));
          cur = Blk{T.p2p_leaf[i], 0, g, c, nt, 0, {}};
        }
      }
    }
    blk.push_back(std::move(cur));
  }
  std::stable_sort(blk.begin(), blk.end(), [](const Blk& a, const Blk& b) {
    return (double)a.ns * (a.nt + 8) > (double)b.ns * (b.nt + 8);
  });
  out.run_off.push_back(0);
  for (const Blk& k : blk) {
    out.leaf.push_back(k.leaf);
    out.self.push_back(k.self);
    out.grp.push_back(k.grp);
    out.chunk.push_back(k.chunk);
    out.runs.insert(out.runs.end(), k.runs.begin(), k.runs.end());
    out.run_off.push_back((int)out.runs.size() / 2);
  }
}

void merge_setups(std::vector<HostSetup>& P, HostSetup& H) {
  const int nm = (int)P.size();
  H = HostSetup();
  H.mesh_tet_off.assign(nm + 1, 0);
  H.mesh_tri_off.assign(nm + 1, 0);
  int nlev = 0;
  for (int m = 0; m < nm; ++m) {
    H.mesh_tet_off[m + 1] = H.mesh_tet_off[m] + P[m].ntet;
    H.mesh_tri_off[m + 1] = H.mesh_tri_off[m] + P[m].ntri;
    nlev = std::max(nlev, P[m].nlevels);
    H.seconds_tree += P[m].seconds_tree;
    H.seconds_lists += P[m].seconds_lists;
    H.seconds_near += P[m].seconds_near;
  }
  H.ntet = H.mesh_tet_off[nm];
  H.ntri = H.mesh_tri_off[nm];
  H.nlevels = nlev;
  for (int m = 0; m < nm; ++m) {
    const HostSetup& S = P[m];
    H.tet_v.insert(H.tet_v.end(), S.tet_v.begin(), S.tet_v.end());
    H.tri_v.insert(H.tri_v.end(), S.tri_v.begin(), S.tri_v.end());
    H.tet_vol.insert(H.tet_vol.end(), S.tet_vol.begin(), S.tet_vol.end());
    H.tri_area.insert(H.tri_area.end(), S.tri_area.begin(), S.tri_area.end());
    for (int c = 0; c < 2; ++c) {
      H.qp[c].insert(H.qp[c].end(), S.qp[c].begin(), S.qp[c].end());
      H.qw[c].insert(H.qw[c].end(), S.qw[c].begin(), S.qw[c].end());
    }
  }
  if (nm > 0) { std::memcpy(H.lo, P[0].lo, sizeof H.lo); H.R0 = P[0].R0; }
  // point offsets per class: points are element-major (4 per tet, 3 per triangle)
  auto pto = [&](int m, int c) -> int { return c == 0 ? (int)(4 * H.mesh_tet_off[m]) : (int)(3 * H.mesh_tri_off[m]); };
  // boxes, level-major
  std::vector<int> lcount(nlev, 0);
  for (int m = 0; m < nm; ++m)
    for (int l = 0; l < P[m].nlevels; ++l) lcount[l] += P[m].lvl_off[l + 1] - P[m].lvl_off[l];
  H.lvl_off.assign(nlev + 1, 0);
  for (int l = 0; l < nlev; ++l) H.lvl_off[l + 1] = H.lvl_off[l] + lcount[l];
  std::vector<std::vector<int>> bmap(nm);
  {
    std::vector<int> cursor(H.lvl_off.begin(), H.lvl_off.end() - 1);
    for (int m = 0; m < nm; ++m) {
      const HostSetup& S = P[m];
      bmap[m].resize(S.box.size());
      for (int l = 0; l < S.nlevels; ++l) {
        for (int b = S.lvl_off[l]; b < S.lvl_off[l + 1]; ++b) bmap[m][b] = cursor[l] + (b - S.lvl_off[l]);
        cursor[l] += S.lvl_off[l + 1] - S.lvl_off[l];
      }
    }
  }
  H.box.resize(H.lvl_off[nlev]);
  for (int m = 0; m < nm; ++m) {
    const HostSetup& S = P[m];
    for (size_t b = 0; b < S.box.size(); ++b) {
      HostBox B = S.box[b];
      if (B.parent >= 0) B.parent = bmap[m][B.parent];
      if (B.child0 >= 0) B.child0 = bmap[m][B.child0];
      for (int c = 0; c < 2; ++c) { B.pt0[c] += pto(m, c); B.pt1[c] += pto(m, c); }
      H.box[bmap[m][b]] = B;
    }
  }
  for (int c = 0; c < 2; ++c) {
    for (int m = 0; m < nm; ++m) {
      const int o = pto(m, c);
      for (int v : P[m].perm[c]) H.perm[c].push_back(o + v);
      for (int v : P[m].leaf_of[c]) H.leaf_of[c].push_back(v >= 0 ? bmap[m][v] : -1);
    }
  }
  // interaction offset codes
  std::unordered_map<int64_t, int> code_of;
  std::vector<std::vector<int>> cmap(nm);
  for (int m = 0; m < nm; ++m) {
    const std::vector<int>& O = P[m].offsets;
    for (size_t k = 0; k < O.size() / 3; ++k) {
      const int64_t key = ((int64_t)(O[3 * k] + 64) << 16) | ((int64_t)(O[3 * k + 1] + 64) << 8) | (int64_t)(O[3 * k + 2] + 64);
      auto it = code_of.find(key);
      int c;
      if (it == code_of.end()) {
        c = (int)(H.offsets.size() / 3);
        code_of[key] = c;
        H.offsets.insert(H.offsets.end(), {O[3 * k], O[3 * k + 1], O[3 * k + 2]});
      } else {
        c = it->second;
      }
      cmap[m].push_back(c);
    }
  }
  // per-task lists
  for (int t = 0; t < 3; ++t) {
    HostTask& T = H.task[t];
    T = HostTask();
    if (nm == 0) continue;
    T.src_cls = P[0].task[t].src_cls;
    T.tgt_cls = P[0].task[t].tgt_cls;
    const int sc = T.src_cls;
    T.near_off.push_back(0);
    T.run_off.push_back(0);
    T.vl_off.push_back(0);
    T.cor_off.push_back(0);
    T.m2m_parent.assign(nlev, {});
    T.l2l_child.assign(nlev, {});
    for (int m = 0; m < nm; ++m) {
      const HostTask& S = P[m].task[t];
      const std::vector<int>& bm = bmap[m];
      const int nb0 = (int)T.near_box.size(), rb0 = (int)(T.runs.size() / 2), vb0 = (int)T.vl_src.size();
      const int64_t nz0 = (int64_t)T.cor_col.size();
      for (int b : S.p2p_leaf) T.p2p_leaf.push_back(bm[b]);
      for (size_t i = 1; i < S.near_off.size(); ++i) T.near_off.push_back(S.near_off[i] + nb0);
      for (int b : S.near_box) T.near_box.push_back(bm[b]);
      for (size_t i = 1; i < S.run_off.size(); ++i) T.run_off.push_back(S.run_off[i] + rb0);
      for (int v : S.runs) T.runs.push_back(v + pto(m, sc));
      T.self_len.insert(T.self_len.end(), S.self_len.begin(), S.self_len.end());
      for (int b : S.m2l_tgt) T.m2l_tgt.push_back(bm[b]);
      for (size_t i = 1; i < S.vl_off.size(); ++i) T.vl_off.push_back(S.vl_off[i] + vb0);
      for (int b : S.vl_src) T.vl_src.push_back(bm[b]);
      for (uint16_t c : S.vl_code) T.vl_code.push_back((uint16_t)cmap[m][c]);
      for (int b : S.p2m_leaf) T.p2m_leaf.push_back(bm[b]);
      for (int b : S.l2p_leaf) T.l2p_leaf.push_back(bm[b]);
      for (size_t l = 0; l < S.m2m_parent.size(); ++l)
        for (int b : S.m2m_parent[l]) T.m2m_parent[l].push_back(bm[b]);
      for (size_t l = 0; l < S.l2l_child.size(); ++l)
        for (int b : S.l2l_child[l]) T.l2l_child[l].push_back(bm[b]);
      const int64_t so = sc == 0 ? H.mesh_tet_off[m] : H.mesh_tri_off[m];
      for (size_t i = 1; i < S.cor_off.size(); ++i) T.cor_off.push_back(S.cor_off[i] + nz0);
      for (int32_t c : S.cor_col) T.cor_col.push_back((int32_t)(c + so));
    }
  }
}

// ---------------------------------------------------------- quadrature
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.resize(n); w.resize(n);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) { double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k; p0 = p1; p1 = p2; }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[n - 1 - i] = 0.5 * (z + 1.0);
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

// ------------------------------------------------------- translations
static double binom(int n, int k) {
  if (k < 0 || k > n) return 0.0;
  double r = 1.0;
  for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
  return r;
}
static double fact(int n) { double r = 1; for (int i = 2; i <= n; ++i) r *= i; return r; }

// D^k (1/|x|) by differentiating F(u) = u^{-1/2}, u = |x|^2, axis by axis:
// d^a/dx^a F(x^2 + ...) = sum_j a!/(j!(a-2j)!) (2x)^{a-2j} F^{(a-j)}(u),
// F^{(n)}(u) = (-1)^n (2n-1)!! / 2^n u^{-1/2-n}.
static void derivatives_inv_r(const double* x, int P, const MultiIndex& M, std::vector<double>& D) {
  double u = x[0] * x[0] + x[1] * x[1] + x[2] * x[2];
  std::vector<double> Fn(P + 1);
  double dfact = 1.0;   // (2n-1)!!
  for (int n = 0; n <= P; ++n) {
    if (n > 0) dfact *= (2.0 * n - 1.0);
    Fn[n] = ((n & 1) ? -1.0 : 1.0) * dfact / std::ldexp(1.0, n) * std::pow(u, -0.5 - n);
  }
  // per-axis coefficient tables c(a, j) (2x)^{a-2j}
  D.assign(M.n, 0.0);
  for (int q = 0; q < M.n; ++q) {
    int al[3] = {M.a[q], M.b[q], M.c[q]};
    int tot = al[0] + al[1] + al[2];
    double s = 0.0;
    for (int j0 = 0; 2 * j0 <= al[0]; ++j0)
      for (int j1 = 0; 2 * j1 <= al[1]; ++j1)
        for (int j2 = 0; 2 * j2 <= al[2]; ++j2) {
          int jj[3] = {j0, j1, j2};
          double prod = 1.0;
          for (int ax = 0; ax < 3; ++ax) {
            int a = al[ax], j = jj[ax];
            prod *= fact(a) / (fact(j) * fact(a - 2 * j)) * std::pow(2.0 * x[ax], a - 2 * j);
          }
          s += prod * Fn[tot - j0 - j1 - j2];
        }
    D[q] = s;
  }
}

void m2l_matrix_scaled(int p, const double o[3], double* T) {
  MultiIndex M, M2;
  M.init(p); M2.init(2 * p);
  std::vector<double> D;
  derivatives_inv_r(o, 2 * p, M2, D);
  for (int a = 0; a < M.n; ++a)
    for (int b = 0; b < M.n; ++b) {
      double v = 0.0;
      int da = M.a[a] + M.b[a] + M.c[a], db = M.a[b] + M.b[b] + M.c[b];
      if (da + db <= p) {
        int k = M2.at(M.a[a] + M.a[b], M.b[a] + M.b[b], M.c[a] + M.c[b]);
        double den = fact(M.a[a]) * fact(M.b[a]) * fact(M.c[a]) * fact(M.a[b]) * fact(M.b[b]) * fact(M.c[b]);
        v = D[k] / kFourPi * ((db & 1) ? -1.0 : 1.0) / den;
      }
      T[a * M.n + b] = v;
    }
}

// D^gamma G(o) = D^gamma (1/r)(o) / (4 pi), |gamma| <= q, degree-major:
// the per-offset coefficients of the Taylor-form M2L (Sec. 3.3).
void m2l_taylor_coeffs(int q, const double o[3], double* g) {
  MultiIndex M;
  M.init(q);
  std::vector<double> D;
  derivatives_inv_r(o, q, M, D);
  for (int k = 0; k < M.n; ++k) g[k] = D[k] / kFourPi;
}

// child octant q: child centre = parent centre + sigma s_parent / 4,
// sigma_axis = +1 if the octant bit is set, else -1.
void m2m_matrices(int p, std::vector<double>& Mm) {
  MultiIndex M; M.init(p);
  int n = M.n;
  Mm.assign(8 * n * n, 0.0);
  for (int q = 0; q < 8; ++q) {
    double sg[3] = {(q & 1) ? 0.25 : -0.25, (q & 2) ? 0.25 : -0.25, (q & 4) ? 0.25 : -0.25};
    for (int b = 0; b < n; ++b)
      for (int g = 0; g < n; ++g) {
        int be[3] = {M.a[b], M.b[b], M.c[b]}, ga[3] = {M.a[g], M.b[g], M.c[g]};
        if (ga[0] > be[0] || ga[1] > be[1] || ga[2] > be[2]) continue;
        double v = std::ldexp(1.0, -(ga[0] + ga[1] + ga[2]));
        for (int ax = 0; ax < 3; ++ax) v *= binom(be[ax], ga[ax]) * std::pow(sg[ax], be[ax] - ga[ax]);
        Mm[(q * n + b) * n + g] = v;
      }
  }
}

void l2l_matrices(int p, std::vector<double>& Lm) {
  MultiIndex M; M.init(p);
  int n = M.n;
  Lm.assign(8 * n * n, 0.0);
  for (int q = 0; q < 8; ++q) {
    double sg[3] = {(q & 1) ? 0.25 : -0.25, (q & 2) ? 0.25 : -0.25, (q & 4) ? 0.25 : -0.25};
    for (int a = 0; a < n; ++a)
      for (int b = 0; b < n; ++b) {
        int al[3] = {M.a[a], M.b[a], M.c[a]}, be[3] = {M.a[b], M.b[b], M.c[b]};
        if (al[0] > be[0] || al[1] > be[1] || al[2] > be[2]) continue;
        double v = std::ldexp(1.0, -(al[0] + al[1] + al[2]));
        for (int ax = 0; ax < 3; ++ax) v *= binom(be[ax], al[ax]) * std::pow(sg[ax], be[ax] - al[ax]);
        Lm[(q * n + a) * n + b] = v;
      }
  }
}

}  // namespace bcfmm
