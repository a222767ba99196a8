// Internal declarations of the bcfmm library (not part of the C ABI).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace bcfmm {

constexpr double kFourPi = 12.566370614359172953850573533118;
constexpr int kMaxLevel = 18;
constexpr int kMaxP = 12;

inline int nterms(int p) { return (p + 1) * (p + 2) * (p + 3) / 6; }

// Multi-indices of total degree <= P: by degree, then (a desc, b desc).
struct MultiIndex {
  int P = 0, n = 0;
  std::vector<int> a, b, c;
  std::vector<int> lut;              // (P+1)^3
  void init(int P_);
  int at(int i, int j, int k) const {
    if (i < 0 || j < 0 || k < 0 || i + j + k > P) return -1;
    return lut[(i * (P + 1) + j) * (P + 1) + k];
  }
};

// Box of the adaptive octree.  Levels are stored contiguously (BFS order).
struct HostBox {
  int level;
  int64_t ijk[3];
  int parent;
  int child0, nchild;
  int octant;                        // position in the parent (bit0 x, bit1 y, bit2 z)
  int pt0[2], pt1[2];                // point ranges of class 0 (tet points) / 1 (tri points)
  double c[3], s;
};

// Per task (VtV, VtB, BtV) lists, host side.
struct HostTask {
  int src_cls = 0, tgt_cls = 0;
  // P2P: target leaves and their extended neighbour list N* as box ids
  std::vector<int> p2p_leaf, near_off, near_box;
  std::vector<int> run_off, runs, self_len;        // merged source runs (start, end) per target leaf
  // M2L: target boxes (level >= 2 with target points) and interaction lists
  std::vector<int> m2l_tgt, vl_off, vl_src;
  std::vector<uint16_t> vl_code;
  // upward / downward restricted to boxes with source / target points
  std::vector<int> p2m_leaf;                       // leaves with source points
  std::vector<std::vector<int>> m2m_parent;        // per level: non-leaf boxes with source points
  std::vector<std::vector<int>> l2l_child;         // per level: boxes (level>=3) with target points
  std::vector<int> l2p_leaf;                       // leaves (level >= 2) with target points
  // tensor-core M2L tiles (see DevTaskLists)
  std::vector<int> tc_tile_tgt, tc_tile_off, tc_ent_code, tc_ent_src, tc_tile_q;
  // near element pairs, CSR over target elements
  std::vector<int64_t> cor_off;
  std::vector<int32_t> cor_col;
};

struct HostSetup {
  int64_t ntet = 0, ntri = 0;
  std::vector<double> tet_v, tri_v;                // [ntet][4][3], [ntri][3][3]
  std::vector<double> tet_vol, tri_area;
  // quadrature points (original order): class 0 tet points 4/tet, class 1 tri points 3/tri
  std::vector<double> qp[2], qw[2];
  // tree
  double lo[3], R0;
  std::vector<HostBox> box;
  std::vector<int> lvl_off;                        // box index range per level
  int nlevels = 0;
  std::vector<int> perm[2];                        // sorted position -> original point index
  std::vector<int> leaf_of[2];                     // sorted position -> leaf box
  HostTask task[3];
  std::vector<int> offsets;                        // distinct interaction offsets (x,y,z) per code
  std::vector<int64_t> mesh_tet_off, mesh_tri_off; // element ranges of the meshes of a batch
  double seconds_tree = 0, seconds_lists = 0, seconds_near = 0;
};

// Validates the mesh, computes element geometry and quadrature points.
// Returns "" on success, else an error message; *mesh_err set when the
// failure is a degenerate element.
std::string setup_mesh(HostSetup& H, const double* verts, int64_t nvert, const int32_t* tets,
                       int64_t ntet, const int32_t* tris, int64_t ntri, bool* mesh_err);
void build_tree(HostSetup& H, int leaf_size);
void build_lists(HostSetup& H, double eta0);
void build_tc_tiles(HostSetup& H, int task, int tile_m, const std::vector<int>& box_q, int qmax);
void find_near_pairs(HostSetup& H, double eta_ns);
// Concatenates independently built meshes into one forest: elements and
// points mesh after mesh, boxes level-major (level l of every mesh, mesh
// order inside), lists and near pairs renumbered.  No list entry crosses
// meshes, so the result evaluates every mesh on its own.
void merge_setups(std::vector<HostSetup>& parts, HostSetup& H);

// Blocks of the packed FP32 near field for one task: a target leaf whose
// near list holds more than `chunk` source points is cut into near-equal
// chunks (runs split at the chunk boundaries; the leaf's own run, at most
// 128 points, stays whole at the front of chunk 0), one block per chunk;
// blocks in descending order of work, source points x (targets + 8).
struct P2pChunks {
  std::vector<int> leaf, run_off, runs, self;   // per block; runs as (start, end) pairs
  std::vector<int> grp, chunk;                  // split leaf index (-1: whole leaf), chunk index
  std::vector<int> grp_row, grp_n;              // per split leaf: first scratch row, chunks
  int rows = 0;                                 // scratch rows (chunks of split leaves)
};
constexpr int64_t kP2pChunk = 8192;
void build_p2p_chunks(const HostSetup& H, int task, int64_t chunk, P2pChunks& out);

// Gauss-Legendre nodes/weights on [0,1] (Newton iteration on P_n).
void gauss_legendre01(int n, std::vector<double>& x, std::vector<double>& w);

// Box-scaled translation tables (Sec. 3.3).
//  M2L: T[a][b] for one offset o (in box units).
//  M2M: for child octant q, m_parent[b] += sum_g M[q][b][g] m_child[g].
//  L2L: for child octant q, l_child[a] += sum_b L[q][a][b] l_parent[b].
void m2l_matrix_scaled(int p, const double o[3], double* T);
void m2l_taylor_coeffs(int q, const double o[3], double* g);
void m2m_matrices(int p, std::vector<double>& M);
void l2l_matrices(int p, std::vector<double>& L);

}  // namespace bcfmm
