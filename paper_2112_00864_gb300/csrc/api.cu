// C ABI of the bcfmm library: context setup (mesh, tree, lists, near-rule
// corrections, translation tables) and the VtV / VtB / BtV evaluations
// (Algorithms 1-3 of arXiv 2112.00864).
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/bcfmm.h"
#include "internal.h"
#include "kernels.cuh"
#include "m2l_taylor.cuh"
#include "m2l_tc.cuh"
#include "mlp.cuh"

using namespace bcfmm;

static thread_local std::string g_err;

static int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CU(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess) {                                                                \
      if (e_ == cudaErrorMemoryAllocation) return fail(BCFMM_ERR_OOM, std::string(#call) + ": " + cudaGetErrorString(e_)); \
      return fail(BCFMM_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));     \
    }                                                                                       \
  } while (0)

namespace {

struct DevAlloc {
  std::vector<void*> ptrs;
  template <typename T>
  cudaError_t alloc(T** p, size_t n) {
    *p = nullptr;
    if (n == 0) n = 1;
    cudaError_t e = cudaMalloc((void**)p, n * sizeof(T));
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
  }
  template <typename T>
  cudaError_t upload(T** p, const T* h, size_t n, cudaStream_t st) {
    cudaError_t e = alloc(p, n);
    if (e != cudaSuccess || n == 0) return e;
    return cudaMemcpyAsync(*p, h, n * sizeof(T), cudaMemcpyHostToDevice, st);
  }
  void release(void* p) {
    auto it = std::find(ptrs.begin(), ptrs.end(), p);
    if (it != ptrs.end()) { cudaFree(*it); ptrs.erase(it); }
  }
  void free_all() {
    for (void* p : ptrs) cudaFree(p);
    ptrs.clear();
  }
};

// Device copies of a task's element geometry kept after the build when the
// near-singular pairs are classified (training data is drawn from them).
struct NearGeom {
  double *tv = nullptr, *sv = nullptr, *tqp = nullptr, *tqw = nullptr, *sqp = nullptr, *sqw = nullptr;
  double *glx = nullptr, *glw = nullptr;
  int* row = nullptr;
  int64_t* ns_list = nullptr;          // CSR positions of the near-singular pairs
};

struct TaskDev {
  NearGeom ng{};
  int64_t n_singular = 0, n_learned = 0, n_fp64 = 0;   // near-pair classes (near_mode != 0)
  DevTaskLists L{};
  TcTaskSched tcs{};                   // tensor-core M2L launches, one per expansion order
  TaylorTaskSched tys{};               // CUDA-core Taylor-form M2L launches, one per expansion order
  std::vector<int> m2m_off, l2l_off;   // host offsets into the per-level arrays
  int* m2m_parent = nullptr;
  int* l2l_child = nullptr;
  int64_t p2p_pairs = 0, near_boxes = 0, m2l_pairs = 0, nnz = 0, tc_entries = 0, tc_rows = 0;
  int64_t m2l_pairs_q[kMaxP + 1] = {};     // box pairs of the interaction phase per expansion order
  double tc_mma_flop = 0;              // executed MMA flops of the tensor-core M2L per density
  int64_t p2p_src_q[5] = {};           // near-field source points per target leaf: min, median, p90, p99, max
};

}  // namespace

struct bcfmm_ctx {
  int device = 0;
  cudaStream_t st = nullptr;
  bcfmm_params prm{};
  int np = 0, ncode = 0;
  int nlevels = 0, nbox = 0, nleaf = 0;
  int64_t ntet = 0, ntri = 0, npts[2] = {0, 0};
  DevAlloc mem;
  DevGeom G{};
  TaskDev task[3];
  // translation tables
  double* T64 = nullptr;
  float* T32 = nullptr;
  M2LTensorTables tc{};
  // learned near-singular correction (near_mode 1): per task, FP32 master
  // parameters and per-bin calibrated errors, from the blob
  bool mlp_has[3] = {false, false, false};
  std::vector<float> mlp_params[3], mlp_eps[3];
  // densities
  // densities: [BCFMM_VOLUME], [BCFMM_BOUNDARY], [BCFMM_DIPOLE]
  int ndens[3] = {0, 0, 0}, ndp[3] = {0, 0, 0};
  double* dens[3] = {nullptr, nullptr, nullptr};
  int* err = nullptr;                  // device error word (bounded device waits)
  size_t tc_partial_per_dens = 0;      // largest tensor-core partial-sum need over the tasks (float2)
  // Taylor-form M2L (BCFMM_FP32): offset coefficients, prescaled moments,
  // chunk partial sums (largest need over the tasks, floats per density)
  TaylorTables ty{};
  float* ty_momp = nullptr;
  float* ty_partial = nullptr;
  size_t ty_partial_per_dens = 0;
  float2* tc_partial = nullptr;        // unit partial sums of the tensor-core M2L
  uint8_t* tc_momb = nullptr;          // BF16 split moments of the tensor-core M2L
  // work buffers (sized for the largest ndp seen)
  int work_ndp = 0;
  double *W64 = nullptr, *mom64 = nullptr, *loc64 = nullptr, *phi = nullptr, *out_dev = nullptr;
  float *W32 = nullptr, *mom32 = nullptr, *loc32 = nullptr;
  double* W64dl = nullptr;               // BtV double-layer point weights w g (double_layer)
  float* W32dl = nullptr;
  // stats
  int nmesh = 1;
  std::vector<int64_t> mesh_tet_off, mesh_tri_off;
  // host copy of the input meshes (bcfmm_build_like rebuilds from it)
  std::vector<double> h_verts;
  std::vector<int32_t> h_tets, h_tris;
  std::vector<int64_t> h_vo, h_to, h_ro;
  const bcfmm_ctx* reuse = nullptr;    // during a build: context whose near pairs are copied
  double sec_host = 0;
  double sec_setup = 0, sec_tree = 0, sec_lists = 0, sec_near_host = 0, sec_near_dev = 0;
  std::vector<int> leaves_per_level, boxes_per_level;
  // per task: CUDA events around the stages of the last evaluation; elapsed
  // times are read lazily by bcfmm_stats (no host sync inside an eval)
  cudaEvent_t ev[3][8] = {};
  bool ev_ok = false, ev_rec[3] = {false, false, false};
  // CUDA graph of bcfmm_eval_graph
  struct {
    cudaGraphExec_t exec = nullptr;
    int mask = 0, work_gen = -1, ndens[3] = {0, 0, 0};
    double* out[3] = {nullptr, nullptr, nullptr};
    int nodes = 0;
  } graph;
  cudaStream_t cap_st = nullptr;
  int work_gen = 0;                    // bumped whenever the work buffers move
};

// Expansion order of a level: p_level[level] when set (1..p), else p
// (Sec. 4.3: the interaction phase and the local expansions of level l use
// order q_l; moments are kept to order p on every level).
static int level_order(const bcfmm_params& prm, int level) {
  const int v = level < BCFMM_MAX_LEVELS ? prm.p_level[level] : 0;
  return v > 0 ? v : prm.p;
}

static double wall() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

static int pad_ndens(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

extern "C" void bcfmm_default_params(bcfmm_params* prm) {
  if (!prm) return;
  prm->p = 6;
  prm->leaf_size = 64;
  prm->eta_ns = 1.0 - std::ldexp(1.0, -20);
  prm->near_n = 3;
  prm->near_k = 1;
  prm->precision = BCFMM_FP64;
  prm->timing = 0;
  prm->eta0 = 0.5;
  prm->tc_unit = 0;
  prm->near_mode = 0;
  prm->mlp_tol = 5e-3;
  prm->mlp_blob = nullptr;
  prm->mlp_blob_bytes = 0;
  for (int l = 0; l < BCFMM_MAX_LEVELS; ++l) prm->p_level[l] = 0;
  prm->q0 = 0;
  prm->double_layer = 0;
}

extern "C" const char* bcfmm_last_error(void) { return g_err.c_str(); }

extern "C" int bcfmm_debug_shift_matrix(int32_t kind, int32_t p, int32_t octant, double* out) {
  if ((kind != 0 && kind != 1) || p < 0 || p > kMaxP || octant < 0 || octant > 7 || !out)
    return fail(BCFMM_ERR_ARG, "debug_shift_matrix: bad argument");
  std::vector<double> Mm;
  if (kind == 0) m2m_matrices(p, Mm); else l2l_matrices(p, Mm);
  const size_t n = (size_t)nterms(p);
  std::copy(Mm.begin() + octant * n * n, Mm.begin() + (octant + 1) * n * n, out);
  return BCFMM_OK;
}

extern "C" int bcfmm_debug_m2l_matrix(int32_t p, const double* o, double* T) {
  if (p < 0 || p > kMaxP || !o || !T) return fail(BCFMM_ERR_ARG, "debug_m2l_matrix: bad argument");
  m2l_matrix_scaled(p, o, T);
  return BCFMM_OK;
}

extern "C" int bcfmm_debug_m2l_taylor_coeffs(int32_t q, const double* o, double* g) {
  if (q < 0 || q > kMaxP || !o || !g) return fail(BCFMM_ERR_ARG, "debug_m2l_taylor_coeffs: bad argument");
  m2l_taylor_coeffs(q, o, g);
  return BCFMM_OK;
}

static int upload_task(bcfmm_ctx* C, const HostSetup& H, int t) {
  const HostTask& T = H.task[t];
  TaskDev& D = C->task[t];
  DevTaskLists& L = D.L;
  cudaStream_t st = C->st;
  auto& m = C->mem;
  L.src_cls = T.src_cls;
  L.tgt_cls = T.tgt_cls;
  L.n_p2p = (int)T.p2p_leaf.size();
  int *p2p_leaf, *near_off, *near_box, *m2l_tgt, *vl_off, *vl_src, *p2m_leaf, *l2p_leaf;
  uint16_t* vl_code;
  {
    // near-field blocks (one per target leaf) in descending order of work,
    // source points x (targets + 8): the longest blocks start first and the
    // launch ends without a tail of a few long leaves
    const int n = L.n_p2p;
    std::vector<int> ord(n);
    std::vector<double> work(n);
    for (int i = 0; i < n; ++i) {
      ord[i] = i;
      int64_t ns = 0;
      for (int r = T.run_off[i]; r < T.run_off[i + 1]; ++r) ns += T.runs[2 * r + 1] - T.runs[2 * r];
      const HostBox& B = H.box[T.p2p_leaf[i]];
      work[i] = (double)ns * (double)(B.pt1[T.tgt_cls] - B.pt0[T.tgt_cls] + 8);
    }
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) { return work[a] > work[b]; });
    std::vector<int> leaf(n), noff(1, 0), nbox, roff(1, 0), runs, self(n);
    for (int i = 0; i < n; ++i) {
      const int o = ord[i];
      leaf[i] = T.p2p_leaf[o];
      self[i] = T.self_len[o];
      for (int k = T.near_off[o]; k < T.near_off[o + 1]; ++k) nbox.push_back(T.near_box[k]);
      noff.push_back((int)nbox.size());
      for (int r = T.run_off[o]; r < T.run_off[o + 1]; ++r) { runs.push_back(T.runs[2 * r]); runs.push_back(T.runs[2 * r + 1]); }
      roff.push_back((int)runs.size() / 2);
    }
    CU(m.upload(&p2p_leaf, leaf.data(), leaf.size(), st));
    CU(m.upload(&near_off, noff.data(), noff.size(), st));
    CU(m.upload(&near_box, nbox.data(), nbox.size(), st));
    L.p2p_leaf = p2p_leaf; L.near_off = near_off; L.near_box = near_box;
    int *run_off, *self_len;
    int2* rd;
    CU(m.upload(&run_off, roff.data(), roff.size(), st));
    CU(m.upload(&self_len, self.data(), self.size(), st));
    CU(m.upload(&rd, reinterpret_cast<const int2*>(runs.data()), runs.size() / 2, st));
    L.run_off = run_off; L.runs = rd; L.self_len = self_len;
  }
  {
    // blocks of the packed FP32 near field (long leaves cut into chunks)
    P2pChunks K;
    build_p2p_chunks(H, t, kP2pChunk, K);
    std::vector<int2> grp(K.grp.size()), ginfo(K.grp_row.size());
    for (size_t b = 0; b < K.grp.size(); ++b) grp[b] = make_int2(K.grp[b], K.chunk[b]);
    for (size_t g = 0; g < K.grp_row.size(); ++g) ginfo[g] = make_int2(K.grp_row[g], K.grp_n[g]);
    int *sl, *sro, *ss;
    int2 *srn, *sg, *gi;
    unsigned* gc;
    float2* scr;
    L.sp_n = (int)K.leaf.size();
    CU(m.upload(&sl, K.leaf.data(), K.leaf.size(), st));
    CU(m.upload(&sro, K.run_off.data(), K.run_off.size(), st));
    CU(m.upload(&srn, reinterpret_cast<const int2*>(K.runs.data()), K.runs.size() / 2, st));
    CU(m.upload(&ss, K.self.data(), K.self.size(), st));
    CU(m.upload(&sg, grp.data(), grp.size(), st));
    CU(m.upload(&gi, ginfo.data(), ginfo.size(), st));
    CU(m.alloc(&gc, ginfo.size()));
    CU(cudaMemsetAsync(gc, 0, std::max<size_t>(1, ginfo.size()) * sizeof(unsigned), st));
    CU(m.alloc(&scr, (size_t)K.rows * 2 * 128));     // up to two densities
    L.sp_leaf = sl; L.sp_run_off = sro; L.sp_runs = srn; L.sp_self = ss;
    L.sp_grp = sg; L.grp_info = gi; L.grp_cnt = gc; L.sp_scratch = scr;
  }
  L.n_m2l = (int)T.m2l_tgt.size();
  CU(m.upload(&m2l_tgt, T.m2l_tgt.data(), T.m2l_tgt.size(), st));
  CU(m.upload(&vl_off, T.vl_off.data(), T.vl_off.size(), st));
  CU(m.upload(&vl_src, T.vl_src.data(), T.vl_src.size(), st));
  CU(m.upload(&vl_code, T.vl_code.data(), T.vl_code.size(), st));
  L.m2l_tgt = m2l_tgt; L.vl_off = vl_off; L.vl_src = vl_src; L.vl_code = vl_code;
  L.n_p2m = (int)T.p2m_leaf.size();
  CU(m.upload(&p2m_leaf, T.p2m_leaf.data(), T.p2m_leaf.size(), st));
  L.p2m_leaf = p2m_leaf;
  L.n_l2p = (int)T.l2p_leaf.size();
  CU(m.upload(&l2p_leaf, T.l2p_leaf.data(), T.l2p_leaf.size(), st));
  L.l2p_leaf = l2p_leaf;
  // per-level lists
  std::vector<int> flat;
  D.m2m_off.assign(1, 0);
  for (auto& v : T.m2m_parent) { flat.insert(flat.end(), v.begin(), v.end()); D.m2m_off.push_back((int)flat.size()); }
  CU(m.upload(&D.m2m_parent, flat.data(), flat.size(), st));
  flat.clear();
  D.l2l_off.assign(1, 0);
  for (auto& v : T.l2l_child) { flat.insert(flat.end(), v.begin(), v.end()); D.l2l_off.push_back((int)flat.size()); }
  CU(m.upload(&D.l2l_child, flat.data(), flat.size(), st));
  // target elements: sorted positions of their points
  const int tc = T.tgt_cls, sc = T.src_cls;
  const int nqt = tc == 0 ? 4 : 3;
  const int64_t nte = tc == 0 ? H.ntet : H.ntri;
  L.ntgt_el = nte;
  L.nsrc_el = sc == 0 ? H.ntet : H.ntri;
  L.nq_tgt = nqt;
  std::vector<int> pos_of(H.perm[tc].size());
  for (size_t j = 0; j < pos_of.size(); ++j) pos_of[H.perm[tc][j]] = (int)j;
  std::vector<int> ep(4 * nte, -1);
  for (int64_t e = 0; e < nte; ++e)
    for (int q = 0; q < nqt; ++q) ep[4 * e + q] = pos_of[nqt * e + q];
  int* elem_pts;
  CU(m.upload(&elem_pts, ep.data(), ep.size(), st));
  L.elem_pts = elem_pts;
  // tensor-core M2L tiles and their schedule: one persistent launch per
  // expansion order, units dealt to the SMs on the host
  L.err = C->err;
  L.tc_ntile = (int)T.tc_tile_off.size() > 0 ? (int)T.tc_tile_off.size() - 1 : 0;
  D.tcs = TcTaskSched();
  if (C->tc.nsplit > 0) {
    // targets of orders above the tensor cores' range: CUDA-core M2L (also
    // when no level's order is in range and there are no tiles at all)
    std::vector<int> sel;
    const int qmax = tc_max_order(C->tc.nsplit);
    for (size_t k = 0; k < T.m2l_tgt.size(); ++k)
      if (level_order(C->prm, H.box[T.m2l_tgt[k]].level) > qmax) sel.push_back((int)k);
    if (!sel.empty()) {
      int* dsel;
      CU(m.upload(&dsel, sel.data(), sel.size(), st));
      D.tcs.simt_sel = dsel;
      D.tcs.nsimt = (int)sel.size();
    }
  }
  if (L.tc_ntile > 0) {
    int* tt;
    CU(m.upload(&tt, T.tc_tile_tgt.data(), T.tc_tile_tgt.size(), st));
    L.tc_tile_tgt = tt;
    D.tc_entries = (int64_t)T.tc_ent_code.size();
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, C->device);
    std::vector<TcOrderSchedHost> sched;
    m2l_tc_schedule(T.tc_tile_off, T.tc_tile_q, T.tc_ent_src, nsm, C->tc.nsplit, C->prm.tc_unit, sched);
    for (const TcOrderSchedHost& O : sched) {
      TcOrderSched& S = D.tcs.ord[O.q];
      S.q = O.q;
      S.ncta = (int)O.seq_off.size() - 1;
      S.nunit = (int)O.units.size();
      S.nslot = O.nslot;
      S.nsplit_tiles = (int)O.splits.size();
      S.nent = O.nent;
      S.rows = O.rows;
      // per sequence item: the offset code and the 128 source rows of its
      // entry, in the order the CTA walks them (no indirection in the kernel)
      std::vector<int> seq_code(O.seq_e.size()), seq_src(O.seq_e.size() * 128);
      for (size_t i = 0; i < O.seq_e.size(); ++i) {
        const int e = O.seq_e[i];
        seq_code[i] = T.tc_ent_code[e];
        std::copy(T.tc_ent_src.begin() + (size_t)e * 128, T.tc_ent_src.begin() + (size_t)e * 128 + 128,
                  seq_src.begin() + i * 128);
      }
      int4 *du, *dsp;
      int *dsc, *dss, *dsu, *dso;
      CU(m.upload(&du, O.units.data(), O.units.size(), st));
      CU(m.upload(&dsp, O.splits.data(), O.splits.size(), st));
      CU(m.upload(&dsc, seq_code.data(), seq_code.size(), st));
      CU(m.upload(&dss, seq_src.data(), seq_src.size(), st));
      CU(m.upload(&dsu, O.seq_u.data(), O.seq_u.size(), st));
      CU(m.upload(&dso, O.seq_off.data(), O.seq_off.size(), st));
      S.units = du; S.splits = dsp; S.seq_code = dsc; S.seq_src = dss; S.seq_u = dsu; S.seq_off = dso;
      const int npad = m2l_tc_npad(O.q);
      D.tcs.partial_per_dens = std::max(D.tcs.partial_per_dens, (size_t)O.nslot * npad * 128);
      D.tc_rows += O.rows;
      D.tc_mma_flop += 2.0 * 128 * (C->tc.nsplit == 2 ? 3 : 6) * (double)npad * npad * (double)O.nent;
    }
    C->tc_partial_per_dens = std::max(C->tc_partial_per_dens, D.tcs.partial_per_dens);
  }
  // Taylor-form M2L: per order, the interaction lists cut into chunks and
  // interleaved per warp; targets of orders above the kernel's range go to
  // the generic kernel
  for (size_t k = 0; k < T.m2l_tgt.size(); ++k)
    D.m2l_pairs_q[level_order(C->prm, H.box[T.m2l_tgt[k]].level)] += T.vl_off[k + 1] - T.vl_off[k];
  if (C->ty.g && !T.m2l_tgt.empty()) {
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, C->device);
    std::vector<int> tq(T.m2l_tgt.size()), sel;
    for (size_t k = 0; k < tq.size(); ++k) tq[k] = level_order(C->prm, H.box[T.m2l_tgt[k]].level);
    std::vector<TaylorOrderHost> sched;
    D.tys = TaylorTaskSched();
    if (!m2l_taylor_schedule(T.m2l_tgt, T.vl_off, T.vl_src, T.vl_code, tq, C->nbox, C->ncode, nsm, sched, sel,
                             &D.tys.cbits)) {
      // indices too large for the packed lists: every target on the generic kernel
      sched.clear();
      sel.resize(T.m2l_tgt.size());
      for (size_t k = 0; k < sel.size(); ++k) sel[k] = (int)k;
    }
    for (const TaylorOrderHost& O : sched) {
      TaylorOrderSched& S = D.tys.ord[O.q];
      S.q = O.q;
      S.nwarp = (int)O.wb.size();
      S.nchunk = O.nchunk;
      S.ntgt = (int)O.tgt.size();
      S.chunk = O.chunk;
      S.pairs = O.pairs;
      int2* dwb;
      int *dlc, *dtg, *dtc;
      uint32_t* dpk;
      CU(m.upload(&dwb, O.wb.data(), O.wb.size(), st));
      CU(m.upload(&dlc, O.lane_chunk.data(), O.lane_chunk.size(), st));
      CU(m.upload(&dpk, O.pk.data(), O.pk.size(), st));
      CU(m.upload(&dtg, O.tgt.data(), O.tgt.size(), st));
      CU(m.upload(&dtc, O.tchunk.data(), O.tchunk.size(), st));
      S.wb = dwb; S.lane_chunk = dlc; S.pk = dpk; S.tgt = dtg; S.tchunk = dtc;
      D.tys.partial_per_dens = std::max(D.tys.partial_per_dens, (size_t)O.nchunk * nterms_q(O.q));
    }
    if (!sel.empty()) {
      int* dsel;
      CU(m.upload(&dsel, sel.data(), sel.size(), st));
      D.tys.simt_sel = dsel;
      D.tys.nsimt = (int)sel.size();
    }
    C->ty_partial_per_dens = std::max(C->ty_partial_per_dens, D.tys.partial_per_dens);
  }
  // near pairs + FP64 corrections computed on the device
  int64_t *cor_off;
  int *cor_col, *cor_row;
  double* cor_val;
  if (C->reuse) {
    // same meshes and near-pair parameters: the CSR and its FP64 values
    // do not depend on the tree, copy them
    const TaskDev& B = C->reuse->task[t];
    D.nnz = B.nnz;
    CU(m.alloc(&cor_off, nte + 1));
    CU(m.alloc(&cor_col, D.nnz));
    CU(m.alloc(&cor_val, D.nnz));
    CU(cudaMemcpyAsync(cor_off, B.L.cor_off, (nte + 1) * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    CU(cudaMemcpyAsync(cor_col, B.L.cor_col, D.nnz * sizeof(int), cudaMemcpyDeviceToDevice, st));
    CU(cudaMemcpyAsync(cor_val, B.L.cor_val, D.nnz * sizeof(double), cudaMemcpyDeviceToDevice, st));
    L.cor_off = cor_off; L.cor_col = cor_col; L.cor_val = cor_val;
  } else {
  D.nnz = (int64_t)T.cor_col.size();
  CU(m.upload(&cor_off, T.cor_off.data(), T.cor_off.size(), st));
  CU(m.upload(&cor_col, T.cor_col.data(), T.cor_col.size(), st));
  std::vector<int> row(T.cor_col.size());
  for (int64_t e = 0; e < nte; ++e)
    for (int64_t k = T.cor_off[e]; k < T.cor_off[e + 1]; ++k) row[k] = (int)e;
  CU(m.upload(&cor_row, row.data(), row.size(), st));
  CU(m.alloc(&cor_val, T.cor_col.size()));
  L.cor_off = cor_off; L.cor_col = cor_col; L.cor_val = cor_val;
  if (C->prm.near_mode == 0) {
    double *tv, *sv, *tqp, *tqw, *sqp, *sqw, *glx, *glw;
    const std::vector<double>& TV = tc == 0 ? H.tet_v : H.tri_v;
    const std::vector<double>& SV = sc == 0 ? H.tet_v : H.tri_v;
    CU(m.upload(&tv, TV.data(), TV.size(), st));
    CU(m.upload(&sv, SV.data(), SV.size(), st));
    CU(m.upload(&tqp, H.qp[tc].data(), H.qp[tc].size(), st));
    CU(m.upload(&tqw, H.qw[tc].data(), H.qw[tc].size(), st));
    CU(m.upload(&sqp, H.qp[sc].data(), H.qp[sc].size(), st));
    CU(m.upload(&sqw, H.qw[sc].data(), H.qw[sc].size(), st));
    std::vector<double> gx, gw;
    gauss_legendre01(C->prm.near_n, gx, gw);
    CU(m.upload(&glx, gx.data(), gx.size(), st));
    CU(m.upload(&glw, gw.data(), gw.size(), st));
    CU(launch_near_rule(t, D.nnz, nullptr, cor_row, cor_col, tv, sv, tqp, tqw, sqp, sqw, glx, glw, C->prm.near_n,
                        C->prm.near_k, 0, cor_val, st));
    CU(cudaStreamSynchronize(st));
    for (void* p : {(void*)tv, (void*)sv, (void*)tqp, (void*)tqw, (void*)sqp, (void*)sqw, (void*)glx, (void*)glw,
                    (void*)cor_row})
      m.release(p);
  } else {
    // classify: touching pairs -> FP64 near rule; near-singular pairs ->
    // learned correction (mode 1, bin accepted), FP64 near rule (mode 1,
    // bin rejected) or no correction (mode 2)
    NearGeom& g = D.ng;
    const std::vector<double>& TV = tc == 0 ? H.tet_v : H.tri_v;
    const std::vector<double>& SV = sc == 0 ? H.tet_v : H.tri_v;
    CU(m.upload(&g.tv, TV.data(), TV.size(), st));
    CU(m.upload(&g.sv, SV.data(), SV.size(), st));
    CU(m.upload(&g.tqp, H.qp[tc].data(), H.qp[tc].size(), st));
    CU(m.upload(&g.tqw, H.qw[tc].data(), H.qw[tc].size(), st));
    CU(m.upload(&g.sqp, H.qp[sc].data(), H.qp[sc].size(), st));
    CU(m.upload(&g.sqw, H.qw[sc].data(), H.qw[sc].size(), st));
    std::vector<double> gx, gw;
    gauss_legendre01(C->prm.near_n, gx, gw);
    CU(m.upload(&g.glx, gx.data(), gx.size(), st));
    CU(m.upload(&g.glw, gw.data(), gw.size(), st));
    g.row = cor_row;
    const bool learned = C->prm.near_mode == 1 && C->mlp_has[t];
    float *eps = nullptr, *par = nullptr;
    if (learned) {
      CU(m.upload(&eps, C->mlp_eps[t].data(), C->mlp_eps[t].size(), st));
      CU(m.upload(&par, C->mlp_params[t].data(), C->mlp_params[t].size(), st));
    }
    const int64_t cap = std::max<int64_t>(D.nnz, 1);
    int64_t* lists;
    unsigned long long* cnt;
    CU(m.alloc(&lists, 4 * cap));
    CU(m.alloc(&cnt, 4));
    CU(cudaMemsetAsync(cnt, 0, 4 * sizeof(unsigned long long), st));
    CU(cudaMemsetAsync(cor_val, 0, cap * sizeof(double), st));
    CU(launch_near_classify(t, D.nnz, cor_row, cor_col, g.tv, g.sv, C->prm.near_mode, eps, (float)C->prm.mlp_tol, lists,
                            cnt, cap, st));
    unsigned long long hc[4];
    CU(cudaMemcpyAsync(hc, cnt, sizeof hc, cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    D.n_fp64 = (int64_t)hc[0];
    D.n_learned = (int64_t)hc[1];
    D.n_singular = (int64_t)hc[3];
    CU(launch_near_rule(t, D.n_fp64, lists, cor_row, cor_col, g.tv, g.sv, g.tqp, g.tqw, g.sqp, g.sqw, g.glx, g.glw,
                        C->prm.near_n, C->prm.near_k, 0, cor_val, st));
    if (learned) CU(launch_near_mlp(t, lists + cap, D.n_learned, cor_row, cor_col, g.tv, g.sv, par, cor_val, st));
    CU(m.alloc(&g.ns_list, std::max<int64_t>(D.n_singular, 1)));
    CU(cudaMemcpyAsync(g.ns_list, lists + 3 * cap, D.n_singular * sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    CU(cudaStreamSynchronize(st));
    m.release(lists);
    m.release(cnt);
    if (eps) m.release(eps);
    if (par) m.release(par);
  }
  }
  // BtV double layer: FP64 near-rule corrections of dG/dn_y on the same
  // near-pair CSR (closed-form solid angle inside the composite rule)
  L.cor_val_dl = nullptr;
  if (t == 2 && C->prm.double_layer) {
    double* cdl;
    CU(m.alloc(&cdl, std::max<int64_t>(D.nnz, 1)));
    if (D.nnz == 0) {
    } else if (C->reuse) {
      CU(cudaMemcpyAsync(cdl, C->reuse->task[2].L.cor_val_dl, D.nnz * sizeof(double), cudaMemcpyDeviceToDevice, st));
    } else if (C->prm.near_mode == 2) {
      CU(cudaMemsetAsync(cdl, 0, D.nnz * sizeof(double), st));
    } else {
      std::vector<int> row(T.cor_col.size());
      for (int64_t e = 0; e < nte; ++e)
        for (int64_t k = T.cor_off[e]; k < T.cor_off[e + 1]; ++k) row[k] = (int)e;
      double *tv, *sv, *tqp, *tqw, *sqp, *sqw, *glx, *glw;
      int* drow;
      CU(m.upload(&drow, row.data(), row.size(), st));
      CU(m.upload(&tv, H.tet_v.data(), H.tet_v.size(), st));
      CU(m.upload(&sv, H.tri_v.data(), H.tri_v.size(), st));
      CU(m.upload(&tqp, H.qp[0].data(), H.qp[0].size(), st));
      CU(m.upload(&tqw, H.qw[0].data(), H.qw[0].size(), st));
      CU(m.upload(&sqp, H.qp[1].data(), H.qp[1].size(), st));
      CU(m.upload(&sqw, H.qw[1].data(), H.qw[1].size(), st));
      std::vector<double> gx, gw;
      gauss_legendre01(C->prm.near_n, gx, gw);
      CU(m.upload(&glx, gx.data(), gx.size(), st));
      CU(m.upload(&glw, gw.data(), gw.size(), st));
      CU(launch_near_rule(3, D.nnz, nullptr, drow, L.cor_col, tv, sv, tqp, tqw, sqp, sqw, glx, glw, C->prm.near_n,
                          C->prm.near_k, 0, cdl, st));
      CU(cudaStreamSynchronize(st));
      for (void* p : {(void*)tv, (void*)sv, (void*)tqp, (void*)tqw, (void*)sqp, (void*)sqw, (void*)glx, (void*)glw,
                      (void*)drow})
        m.release(p);
    }
    L.cor_val_dl = cdl;
  }
  // counts for the statistics and the roofline
  D.near_boxes = (int64_t)T.near_box.size();
  D.m2l_pairs = (int64_t)T.vl_src.size();
  D.p2p_pairs = 0;
  std::vector<int64_t> srcs;
  for (size_t i = 0; i < T.p2p_leaf.size(); ++i) {
    const HostBox& B = H.box[T.p2p_leaf[i]];
    int64_t nt = B.pt1[tc] - B.pt0[tc], ns = 0;
    for (int k = T.near_off[i]; k < T.near_off[i + 1]; ++k) {
      const HostBox& S = H.box[T.near_box[k]];
      ns += S.pt1[sc] - S.pt0[sc];
    }
    D.p2p_pairs += nt * ns;
    srcs.push_back(ns);
  }
  if (!srcs.empty()) {
    std::sort(srcs.begin(), srcs.end());
    const size_t n = srcs.size();
    const size_t at[5] = {0, n / 2, (n * 9) / 10, (n * 99) / 100, n - 1};
    for (int k = 0; k < 5; ++k) D.p2p_src_q[k] = srcs[at[k]];
  }
  return BCFMM_OK;
}

// Blob of the learned correction: 8 uint32 (magic "BCML" little-endian,
// version 1, parameters per network, bins, has[3], reserved), then per
// task t: float params[kMlpParams], float eps[kMlpBins].
struct MlpBlob {
  bool has[3] = {false, false, false};
  std::vector<float> params[3], eps[3];
};
constexpr uint32_t kMlpMagic = 0x4C4D4342u;
constexpr int64_t kMlpBlobBytes = 32 + 3 * (int64_t)(kMlpParams + kMlpBins) * 4;

static std::string parse_mlp_blob(const void* p, int64_t n, MlpBlob& B) {
  if (!p || n != kMlpBlobBytes) return "near_mode 1 needs an mlp_blob of bcfmm_mlp_blob_size() bytes";
  uint32_t h[8];
  std::memcpy(h, p, sizeof h);
  if (h[0] != kMlpMagic || h[1] != 1 || h[2] != (uint32_t)kMlpParams || h[3] != (uint32_t)kMlpBins)
    return "mlp_blob header does not match this library's network";
  const float* f = reinterpret_cast<const float*>(static_cast<const char*>(p) + 32);
  for (int t = 0; t < 3; ++t) {
    B.has[t] = h[4 + t] != 0;
    B.params[t].assign(f, f + kMlpParams);
    B.eps[t].assign(f + kMlpParams, f + kMlpParams + kMlpBins);
    for (float v : B.params[t])
      if (!std::isfinite(v)) return "mlp_blob holds a non-finite parameter";
    f += kMlpParams + kMlpBins;
  }
  return "";
}

// Host phase of one mesh: element geometry, octree, lists, near pairs.
static std::string build_host_mesh(HostSetup& H, const double* verts, int64_t nvert, const int32_t* tets, int64_t ntet,
                                   const int32_t* tris, int64_t ntri, const bcfmm_params& prm, bool near,
                                   bool* mesh_err) {
  std::string e = setup_mesh(H, verts, nvert, tets, ntet, tris, ntri, mesh_err);
  if (!e.empty()) return e;
  build_tree(H, prm.leaf_size);
  for (auto& B : H.box)
    if (!B.nchild && (B.pt1[0] - B.pt0[0] > 128 || B.pt1[1] - B.pt0[1] > 128)) {
      *mesh_err = true;
      return "more than 128 coincident points in one leaf at the deepest level";
    }
  build_lists(H, prm.eta0);
  if (near) find_near_pairs(H, prm.eta_ns);
  return "";
}

static int build_impl(const double* verts, const int64_t* vert_off, const int32_t* tets, const int64_t* tet_off,
                      const int32_t* tris, const int64_t* tri_off, int32_t nmesh, const bcfmm_params* prm_in,
                      void* stream, bcfmm_ctx** out, const bcfmm_ctx* reuse = nullptr) {
  double t0 = wall();
  bcfmm_params prm;
  bcfmm_default_params(&prm);
  if (prm_in) prm = *prm_in;
  if (!out) return fail(BCFMM_ERR_ARG, "build: out is NULL");
  *out = nullptr;
  if (nmesh < 1 || !vert_off || !tet_off || !tri_off) return fail(BCFMM_ERR_ARG, "build: nmesh < 1 or null offsets");
  for (int m = 0; m < nmesh; ++m)
    if (vert_off[m + 1] <= vert_off[m] || tet_off[m + 1] <= tet_off[m] || tri_off[m + 1] < tri_off[m] || vert_off[0] != 0 ||
        tet_off[0] != 0 || tri_off[0] != 0)
      return fail(BCFMM_ERR_ARG, "build: mesh " + std::to_string(m) + " is empty or the offsets are not prefix sums");
  const int64_t ntet = tet_off[nmesh], ntri = tri_off[nmesh];
  if (!verts || !tets || (ntri > 0 && !tris)) return fail(BCFMM_ERR_ARG, "build: null mesh arrays or empty mesh");
  if (4 * ntet > INT32_MAX / 2 || 3 * ntri > INT32_MAX / 2) return fail(BCFMM_ERR_ARG, "build: mesh too large");
  if (prm.p < 0 || prm.p > kMaxP) return fail(BCFMM_ERR_ARG, "build: p must be in 0..12");
  if (prm.leaf_size < 1 || prm.leaf_size > 128) return fail(BCFMM_ERR_ARG, "build: leaf_size must be in 1..128");
  for (int l = 0; l < BCFMM_MAX_LEVELS; ++l)
    if (prm.p_level[l] < 0 || prm.p_level[l] > prm.p)
      return fail(BCFMM_ERR_ARG, "build: p_level[" + std::to_string(l) + "] must be in 0..p (0: p)");
  if (!(prm.eta_ns > 0)) return fail(BCFMM_ERR_ARG, "build: eta_ns must be > 0");
  if (!(prm.eta0 >= 0.3 && prm.eta0 <= 1.0)) return fail(BCFMM_ERR_ARG, "build: eta0 must be in 0.3..1");
  if (prm.near_n < 1 || prm.near_n > 8 || prm.near_k < 0 || prm.near_k > 3)
    return fail(BCFMM_ERR_ARG, "build: near_n must be in 1..8 and near_k in 0..3");
  if (prm.precision < BCFMM_FP64 || prm.precision > BCFMM_FP32_BF16X3)
    return fail(BCFMM_ERR_ARG, "build: unknown precision");
  if (prm.tc_unit < 0 || prm.tc_unit > 4096) return fail(BCFMM_ERR_ARG, "build: tc_unit must be in 0..4096");
  if (prm.near_mode < 0 || prm.near_mode > 2) return fail(BCFMM_ERR_ARG, "build: near_mode must be 0, 1 or 2");
  MlpBlob blob;
  if (prm.near_mode == 1 && !reuse) {             // (a rebuild copies the corrections)
    if (!(prm.mlp_tol > 0)) return fail(BCFMM_ERR_ARG, "build: mlp_tol must be > 0");
    std::string be = parse_mlp_blob(prm.mlp_blob, prm.mlp_blob_bytes, blob);
    if (!be.empty()) return fail(BCFMM_ERR_ARG, "build: " + be);
  }
  const bool tc_mode = prm.precision == BCFMM_FP32_BF16X2 || prm.precision == BCFMM_FP32_BF16X3;
  const int nsplit = prm.precision == BCFMM_FP32_BF16X3 ? 3 : 2;
  if (prm.q0 < 0 || prm.q0 > kMaxP) return fail(BCFMM_ERR_ARG, "build: q0 must be in 0..12");
  if (prm.double_layer != 0 && prm.double_layer != 1) return fail(BCFMM_ERR_ARG, "build: double_layer must be 0 or 1");

  // host phase per mesh; meshes of a batch in parallel, largest first
  const double th = wall();
  HostSetup H;
  {
    std::vector<HostSetup> parts(nmesh);
    std::vector<std::string> errs(nmesh);
    std::vector<char> merr(nmesh, 0);
    auto one = [&](int m) {
      bool me = false;
      try {
        errs[m] = build_host_mesh(parts[m], verts + 3 * vert_off[m], vert_off[m + 1] - vert_off[m], tets + 4 * tet_off[m],
                                  tet_off[m + 1] - tet_off[m], ntri > 0 ? tris + 3 * tri_off[m] : nullptr,
                                  tri_off[m + 1] - tri_off[m], prm, reuse == nullptr, &me);
      } catch (const std::bad_alloc&) {
        errs[m] = "host allocation failed";
      } catch (const std::exception& ex) {
        errs[m] = ex.what();
      }
      merr[m] = me;
    };
    if (nmesh == 1) {
      one(0);
    } else {
      std::vector<int> order(nmesh);
      for (int m = 0; m < nmesh; ++m) order[m] = m;
      std::stable_sort(order.begin(), order.end(),
                       [&](int a, int b) { return tet_off[a + 1] - tet_off[a] > tet_off[b + 1] - tet_off[b]; });
#pragma omp parallel for schedule(dynamic, 1)
      for (int i = 0; i < nmesh; ++i) one(order[i]);
    }
    for (int m = 0; m < nmesh; ++m)
      if (!errs[m].empty())
        return fail(merr[m] ? BCFMM_ERR_MESH : BCFMM_ERR_ARG,
                    "build: " + (nmesh > 1 ? "mesh " + std::to_string(m) + ": " : std::string()) + errs[m]);
    if (nmesh == 1) {
      H = std::move(parts[0]);
      H.mesh_tet_off = {0, ntet};
      H.mesh_tri_off = {0, ntri};
    } else {
      merge_setups(parts, H);
    }
  }
  if (H.offsets.size() / 3 > 65535) return fail(BCFMM_ERR_ARG, "build: too many interaction offsets");
  if (prm.q0 > 0) {
    // Sec. 4.3 (Eq. def:q0): q_l = q0 + L - l, L the deepest level of the
    // tree (of every mesh of a batch), capped at p
    const int L = H.nlevels - 1;
    for (int l = 0; l < BCFMM_MAX_LEVELS; ++l) prm.p_level[l] = std::max(1, std::min(prm.p, prm.q0 + L - l));
  }
  std::vector<int> box_q(H.box.size());
  for (size_t i = 0; i < H.box.size(); ++i) box_q[i] = level_order(prm, H.box[i].level);
  // levels of higher order than the tensor cores take run the CUDA-core M2L
  if (tc_mode)
    for (int t = 0; t < 3; ++t) build_tc_tiles(H, t, 128, box_q, tc_max_order(nsplit));
  const double host_wall = wall() - th;

  int dev = 0;
  CU(cudaGetDevice(&dev));
  bcfmm_ctx* C = new bcfmm_ctx();
  C->device = dev;
  C->st = (cudaStream_t)stream;
  C->prm = prm;
  C->ntet = ntet;
  C->ntri = ntri;
  auto cleanup = [&](int code) { C->mem.free_all(); delete C; return code; };

  if (C->mem.alloc(&C->err, 1) != cudaSuccess || cudaMemsetAsync(C->err, 0, sizeof(int), C->st) != cudaSuccess)
    return cleanup(fail(BCFMM_ERR_OOM, "build: device allocation failed (error word)"));
  C->nmesh = nmesh;
  C->reuse = reuse;
  for (int t = 0; t < 3; ++t) {
    C->mlp_has[t] = blob.has[t];
    C->mlp_params[t] = blob.params[t];
    C->mlp_eps[t] = blob.eps[t];
  }
  C->prm.mlp_blob = nullptr;             // read during the build only
  C->prm.mlp_blob_bytes = 0;
  C->h_verts.assign(verts, verts + 3 * vert_off[nmesh]);
  C->h_tets.assign(tets, tets + 4 * ntet);
  if (ntri > 0) C->h_tris.assign(tris, tris + 3 * ntri);
  C->h_vo.assign(vert_off, vert_off + nmesh + 1);
  C->h_to.assign(tet_off, tet_off + nmesh + 1);
  C->h_ro.assign(tri_off, tri_off + nmesh + 1);
  C->mesh_tet_off = H.mesh_tet_off;
  C->mesh_tri_off = H.mesh_tri_off;
  C->sec_host = host_wall;
  C->sec_tree = H.seconds_tree;
  C->sec_lists = H.seconds_lists;
  C->sec_near_host = H.seconds_near;
  C->nlevels = H.nlevels;
  C->nbox = (int)H.box.size();
  C->np = nterms(prm.p);
  C->leaves_per_level.assign(H.nlevels, 0);
  C->boxes_per_level.assign(H.nlevels, 0);
  for (auto& B : H.box) { C->boxes_per_level[B.level]++; if (!B.nchild) { C->leaves_per_level[B.level]++; C->nleaf++; } }

  cudaStream_t st = C->st;
  auto& m = C->mem;
  DevGeom& G = C->G;
  G.np = C->np; G.ms = (C->np + 3) / 4 * 4; G.p = prm.p; G.nbox = C->nbox;
  {
    MultiIndex M; M.init(prm.p);
    std::vector<int> mi(M.n);
    for (int q = 0; q < M.n; ++q) mi[q] = M.a[q] | (M.b[q] << 8) | (M.c[q] << 16);
    int* dmi;
    if (m.upload(&dmi, mi.data(), mi.size(), st) != cudaSuccess)
      return cleanup(fail(BCFMM_ERR_OOM, "build: device allocation failed"));
    G.mi = dmi;
  }
  // boxes
  {
    const int nb = C->nbox;
    std::vector<double4_32a> cs(nb);
    std::vector<int> c0(nb), nc(nb), oc(nb), par(nb);
    std::vector<int2> rg[2] = {std::vector<int2>(nb), std::vector<int2>(nb)};
    for (int i = 0; i < nb; ++i) {
      const HostBox& B = H.box[i];
      cs[i] = make_double4_32a(B.c[0], B.c[1], B.c[2], B.s);
      c0[i] = B.child0; nc[i] = B.nchild; oc[i] = B.octant; par[i] = B.parent;
      for (int c = 0; c < 2; ++c) rg[c][i] = make_int2(B.pt0[c], B.pt1[c]);
    }
    const std::vector<int>& bq = box_q;
    double4_32a* dcs; int *dc0, *dnc, *doc, *dpar, *dbq; int2 *drg0, *drg1;
    bool ok = m.upload(&dcs, cs.data(), nb, st) == cudaSuccess && m.upload(&dc0, c0.data(), nb, st) == cudaSuccess &&
              m.upload(&dnc, nc.data(), nb, st) == cudaSuccess && m.upload(&doc, oc.data(), nb, st) == cudaSuccess &&
              m.upload(&dpar, par.data(), nb, st) == cudaSuccess && m.upload(&drg0, rg[0].data(), nb, st) == cudaSuccess &&
              m.upload(&drg1, rg[1].data(), nb, st) == cudaSuccess && m.upload(&dbq, bq.data(), nb, st) == cudaSuccess;
    if (!ok) return cleanup(fail(BCFMM_ERR_OOM, "build: device allocation failed (boxes)"));
    G.box_cs = dcs; G.box_child0 = dc0; G.box_nchild = dnc; G.box_octant = doc; G.box_parent = dpar;
    G.box_rng[0] = drg0; G.box_rng[1] = drg1; G.box_q = dbq;
  }
  // sorted points
  for (int c = 0; c < 2; ++c) {
    const int nq = c == 0 ? 4 : 3;
    const int64_t n = (int64_t)H.perm[c].size();
    C->npts[c] = n;
    std::vector<double4_32a> p64(n);
    std::vector<float4> hi(n), lo(n);
    std::vector<int> el(n);
    for (int64_t j = 0; j < n; ++j) {
      const int o = H.perm[c][j];
      const double* x = &H.qp[c][3 * (int64_t)o];
      p64[j] = make_double4_32a(x[0], x[1], x[2], H.qw[c][o]);
      float h[3], l[3];
      for (int a = 0; a < 3; ++a) { h[a] = (float)x[a]; l[a] = (float)(x[a] - (double)h[a]); }
      hi[j] = make_float4(h[0], h[1], h[2], (float)H.qw[c][o]);
      lo[j] = make_float4(l[0], l[1], l[2], 0.f);
      el[j] = o / nq;
    }
    double4_32a* dp; float4 *dh, *dl; int* de;
    bool ok = m.upload(&dp, p64.data(), n, st) == cudaSuccess && m.upload(&dh, hi.data(), n, st) == cudaSuccess &&
              m.upload(&dl, lo.data(), n, st) == cudaSuccess && m.upload(&de, el.data(), n, st) == cudaSuccess;
    if (!ok) return cleanup(fail(BCFMM_ERR_OOM, "build: device allocation failed (points)"));
    G.pt64[c] = dp; G.pthi[c] = dh; G.ptlo[c] = dl; G.pt_elem[c] = de;
  }
  // unit normal of every triangle (right-hand rule of its vertex order)
  {
    const int64_t nf = (int64_t)(H.tri_v.size() / 9);
    std::vector<double4_32a> nrm(std::max<int64_t>(nf, 1), make_double4_32a(0, 0, 0, 0));
    for (int64_t f = 0; f < nf; ++f) {
      const double* v = &H.tri_v[9 * f];
      const double a[3] = {v[3] - v[0], v[4] - v[1], v[5] - v[2]}, b[3] = {v[6] - v[0], v[7] - v[1], v[8] - v[2]};
      double n[3] = {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
      const double nn = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
      nrm[f] = make_double4_32a(n[0] / nn, n[1] / nn, n[2] / nn, 0.0);
    }
    double4_32a* dn;
    if (m.upload(&dn, nrm.data(), nrm.size(), st) != cudaSuccess)
      return cleanup(fail(BCFMM_ERR_OOM, "build: device allocation failed (normals)"));
    G.tri_nrm = dn;
  }
  // translation tables: M2L transposed per offset code
  {
    const int np = C->np;
    const int ncode = (int)(H.offsets.size() / 3);
    C->ncode = ncode;
    std::vector<double> T((size_t)std::max(ncode, 1) * np * np, 0.0), Tt(T.size(), 0.0), tmp(np * np);
    for (int code = 0; code < ncode; ++code) {
      double od[3] = {(double)H.offsets[3 * code], (double)H.offsets[3 * code + 1], (double)H.offsets[3 * code + 2]};
      m2l_matrix_scaled(prm.p, od, tmp.data());
      for (int a = 0; a < np; ++a)
        for (int b = 0; b < np; ++b) {
          T[((size_t)code * np + a) * np + b] = tmp[a * np + b];
          Tt[((size_t)code * np + b) * np + a] = tmp[a * np + b];
        }
    }
    // M2M and L2L run as three 1-D binomial shifts: their coefficients
    // C(n, k) (+-1/4)^(n-k), s = 0 for -1/4, s = 1 for +1/4
    const int P1 = prm.p + 1;
    std::vector<double> sh(2 * (size_t)P1 * P1, 0.0);
    for (int sg = 0; sg < 2; ++sg)
      for (int n = 0; n < P1; ++n)
        for (int k = 0; k <= n; ++k) {
          double c = 1.0;
          for (int i = 1; i <= k; ++i) c = c * (n - k + i) / i;
          sh[((size_t)sg * P1 + n) * P1 + k] = c * std::pow(sg ? 0.25 : -0.25, n - k);
        }
    std::vector<float> sh32(sh.begin(), sh.end());
    std::vector<float> Tt32(Tt.begin(), Tt.end());
    double* dsh;
    float* dsh32;
    bool ok = m.upload(&C->T64, Tt.data(), Tt.size(), st) == cudaSuccess &&
              m.upload(&C->T32, Tt32.data(), Tt32.size(), st) == cudaSuccess &&
              m.upload(&dsh, sh.data(), sh.size(), st) == cudaSuccess &&
              m.upload(&dsh32, sh32.data(), sh32.size(), st) == cudaSuccess;
    C->G.shift64 = dsh;
    C->G.shift32 = dsh32;
    if (!ok) return cleanup(fail(BCFMM_ERR_OOM, "build: device allocation failed (tables)"));
    if (tc_mode) {
      std::vector<int> orders;
      for (int t = 0; t < 3; ++t)
        for (int q : H.task[t].tc_tile_q)
          if (std::find(orders.begin(), orders.end(), q) == orders.end()) orders.push_back(q);
      cudaError_t ce = m2l_tc_prepare_tables(prm.p, ncode, T.data(), nsplit, orders, &C->tc, st);
      if (ce != cudaSuccess) {
        m2l_tc_free_tables(&C->tc);
        return cleanup(fail(BCFMM_ERR_CUDA, std::string("build: tensor tables: ") + cudaGetErrorString(ce)));
      }
    }
    if (prm.precision == BCFMM_FP32) {
      // Taylor-form M2L: D^gamma G(o), |gamma| <= the largest order of any level
      int qt = 0;
      for (int l = 0; l < C->nlevels; ++l) qt = std::max(qt, level_order(prm, l));
      if (qt > 0) {
        const int pitch = m2l_taylor_pitch(qt);
        std::vector<float> g((size_t)std::max(ncode, 1) * pitch, 0.f);
        std::vector<double> gd(nterms_q(qt));
        for (int code = 0; code < ncode; ++code) {
          const double od[3] = {(double)H.offsets[3 * code], (double)H.offsets[3 * code + 1],
                                (double)H.offsets[3 * code + 2]};
          m2l_taylor_coeffs(qt, od, gd.data());
          for (int k = 0; k < nterms_q(qt); ++k) g[(size_t)code * pitch + k] = (float)gd[k];
        }
        // (-1)^{|b|} / b! for the moments, 1 / a! for the locals
        std::vector<float> fac(2 * (size_t)pitch, 0.f);
        MultiIndex M;
        M.init(qt);
        for (int k = 0; k < M.n; ++k) {
          double f = 1.0;
          for (int n = 2; n <= M.a[k]; ++n) f *= n;
          for (int n = 2; n <= M.b[k]; ++n) f *= n;
          for (int n = 2; n <= M.c[k]; ++n) f *= n;
          fac[k] = (float)(((M.a[k] + M.b[k] + M.c[k]) & 1 ? -1.0 : 1.0) / f);
          fac[pitch + k] = (float)(1.0 / f);
        }
        float *dg, *df;
        if (m.upload(&dg, g.data(), g.size(), st) != cudaSuccess || m.upload(&df, fac.data(), fac.size(), st) != cudaSuccess)
          return cleanup(fail(BCFMM_ERR_OOM, "build: device allocation failed (Taylor tables)"));
        C->ty.g = dg;
        C->ty.fac = df;
        C->ty.gpitch = pitch;
        C->ty.q = qt;
      }
    }
  }
  double tn = wall();
  for (int t = 0; t < 3; ++t) {
    int rc = upload_task(C, H, t);
    if (rc != BCFMM_OK) return cleanup(rc);
  }
  C->sec_near_dev = wall() - tn;
  C->reuse = nullptr;
  if (cudaStreamSynchronize(st) != cudaSuccess) return cleanup(fail(BCFMM_ERR_CUDA, "build: stream sync failed"));
  if (prm.timing) {
    C->ev_ok = true;
    for (auto& row : C->ev)
      for (auto& ev : row)
        if (cudaEventCreate(&ev) != cudaSuccess) C->ev_ok = false;
  }
  C->sec_setup = wall() - t0;
  *out = C;
  return BCFMM_OK;
}

extern "C" int bcfmm_build_bc_tree(const double* verts, int64_t nvert, const int32_t* tets, int64_t ntet,
                                   const int32_t* tris, int64_t ntri, const bcfmm_params* prm, void* stream,
                                   bcfmm_ctx** out) {
  if (out) *out = nullptr;
  if (nvert <= 0 || ntet <= 0 || ntri < 0) return fail(BCFMM_ERR_ARG, "build_bc_tree: null mesh arrays or empty mesh");
  const int64_t vo[2] = {0, nvert}, to[2] = {0, ntet}, ro[2] = {0, ntri};
  try {
    return build_impl(verts, vo, tets, to, tris, ro, 1, prm, stream, out);
  } catch (const std::bad_alloc&) {
    return fail(BCFMM_ERR_OOM, "build_bc_tree: host allocation failed");
  } catch (const std::exception& ex) {
    return fail(BCFMM_ERR_ARG, std::string("build_bc_tree: ") + ex.what());
  }
}

extern "C" int bcfmm_build_batch(const double* verts, const int64_t* vert_off, const int32_t* tets,
                                 const int64_t* tet_off, const int32_t* tris, const int64_t* tri_off, int32_t nmesh,
                                 const bcfmm_params* prm, void* stream, bcfmm_ctx** out) {
  try {
    return build_impl(verts, vert_off, tets, tet_off, tris, tri_off, nmesh, prm, stream, out);
  } catch (const std::bad_alloc&) {
    return fail(BCFMM_ERR_OOM, "build_batch: host allocation failed");
  } catch (const std::exception& ex) {
    return fail(BCFMM_ERR_ARG, std::string("build_batch: ") + ex.what());
  }
}

// Host only: boxes and leaves per level of one mesh's octree.
extern "C" int bcfmm_debug_tree_counts(const double* verts, int64_t nvert, const int32_t* tets, int64_t ntet,
                                       const int32_t* tris, int64_t ntri, int32_t leaf_size, int64_t* boxes,
                                       int64_t* leaves, int32_t nlev_cap) {
  if (!verts || !tets || !boxes || !leaves || leaf_size < 1 || leaf_size > 128 || nlev_cap < 1)
    return fail(BCFMM_ERR_ARG, "debug_tree_counts: bad argument");
  try {
    HostSetup H;
    bool me = false;
    const std::string e = setup_mesh(H, verts, nvert, tets, ntet, tris, ntri, &me);
    if (!e.empty()) return fail(me ? BCFMM_ERR_MESH : BCFMM_ERR_ARG, "debug_tree_counts: " + e);
    build_tree(H, leaf_size);
    if (H.nlevels > nlev_cap) return fail(BCFMM_ERR_ARG, "debug_tree_counts: more levels than nlev_cap");
    std::fill(boxes, boxes + nlev_cap, 0);
    std::fill(leaves, leaves + nlev_cap, 0);
    for (const HostBox& B : H.box) {
      boxes[B.level]++;
      if (!B.nchild) leaves[B.level]++;
    }
  } catch (const std::exception& ex) {
    return fail(BCFMM_ERR_ARG, std::string("debug_tree_counts: ") + ex.what());
  }
  return BCFMM_OK;
}

// Host only: the near element pairs of one mesh and task as the build
// finds them (CSR over target elements, sorted source indices).
extern "C" int bcfmm_debug_near_pairs(const double* verts, int64_t nvert, const int32_t* tets, int64_t ntet,
                                      const int32_t* tris, int64_t ntri, double eta_ns, int32_t task, int64_t cap,
                                      int64_t* row_off, int32_t* cols, int64_t* nnz) {
  if (!verts || !tets || !row_off || !nnz || (cap > 0 && !cols) || task < 0 || task > 2 || !(eta_ns > 0))
    return fail(BCFMM_ERR_ARG, "debug_near_pairs: bad argument");
  try {
    HostSetup H;
    bool me = false;
    const std::string e = setup_mesh(H, verts, nvert, tets, ntet, tris, ntri, &me);
    if (!e.empty()) return fail(me ? BCFMM_ERR_MESH : BCFMM_ERR_ARG, "debug_near_pairs: " + e);
    bcfmm_params prm;
    bcfmm_default_params(&prm);
    build_tree(H, prm.leaf_size);
    build_lists(H, prm.eta0);
    find_near_pairs(H, eta_ns);
    const HostTask& T = H.task[task];
    *nnz = (int64_t)T.cor_col.size();
    std::copy(T.cor_off.begin(), T.cor_off.end(), row_off);
    if ((int64_t)T.cor_col.size() > cap)
      return fail(BCFMM_ERR_ARG, "debug_near_pairs: cap too small, need " + std::to_string(T.cor_col.size()));
    std::copy(T.cor_col.begin(), T.cor_col.end(), cols);
  } catch (const std::exception& ex) {
    return fail(BCFMM_ERR_ARG, std::string("debug_near_pairs: ") + ex.what());
  }
  return BCFMM_OK;
}

// Host only: tree and lists as bcfmm_build_batch builds them, then for
// every task and every target leaf the source points of its mesh covered
// by the leaf's merged near-field runs plus the interaction lists of the
// leaf and its ancestors; counts the (leaf, source point) pairs not covered
// exactly once.
extern "C" int bcfmm_debug_list_coverage(const double* verts, const int64_t* vert_off, const int32_t* tets,
                                         const int64_t* tet_off, const int32_t* tris, const int64_t* tri_off,
                                         int32_t nmesh, const bcfmm_params* prm_in, int64_t* out) {
  if (!out || nmesh < 1 || !verts || !vert_off || !tets || !tet_off || !tri_off)
    return fail(BCFMM_ERR_ARG, "debug_list_coverage: null argument");
  bcfmm_params prm;
  bcfmm_default_params(&prm);
  if (prm_in) prm = *prm_in;
  if (prm.leaf_size < 1 || prm.leaf_size > 128 || !(prm.eta0 >= 0.3 && prm.eta0 <= 1.0))
    return fail(BCFMM_ERR_ARG, "debug_list_coverage: bad leaf_size or eta0");
  try {
    std::vector<HostSetup> parts(nmesh);
    for (int m = 0; m < nmesh; ++m) {
      bool me = false;
      const int64_t nt = tet_off[m + 1] - tet_off[m], nf = tri_off[m + 1] - tri_off[m];
      const std::string e = build_host_mesh(parts[m], verts + 3 * vert_off[m], vert_off[m + 1] - vert_off[m],
                                            tets + 4 * tet_off[m], nt, nf > 0 ? tris + 3 * tri_off[m] : nullptr, nf,
                                            prm, false, &me);
      if (!e.empty()) return fail(me ? BCFMM_ERR_MESH : BCFMM_ERR_ARG, "debug_list_coverage: " + e);
    }
    HostSetup H;
    if (nmesh == 1) {
      H = std::move(parts[0]);
      H.mesh_tet_off = {0, tet_off[1]};
      H.mesh_tri_off = {0, tri_off[1]};
    } else {
      merge_setups(parts, H);
    }
    for (int t = 0; t < 3; ++t) {
      const HostTask& T = H.task[t];
      const int sc = T.src_cls, tc = T.tgt_cls;
      const int64_t nsrc = (int64_t)H.perm[sc].size();
      std::vector<int> k_of(H.box.size(), -1);
      for (size_t k = 0; k < T.m2l_tgt.size(); ++k) k_of[T.m2l_tgt[k]] = (int)k;
      const std::vector<int64_t>& toff = tc == 0 ? H.mesh_tet_off : H.mesh_tri_off;
      const std::vector<int64_t>& soff = sc == 0 ? H.mesh_tet_off : H.mesh_tri_off;
      const int nqt = tc == 0 ? 4 : 3, nqs = sc == 0 ? 4 : 3;
      std::vector<int> cnt(nsrc);
      int64_t bad = 0;
      for (size_t i = 0; i < T.p2p_leaf.size(); ++i) {
        const int b = T.p2p_leaf[i];
        std::fill(cnt.begin(), cnt.end(), 0);
        for (int r = T.run_off[i]; r < T.run_off[i + 1]; ++r)
          for (int q = T.runs[2 * r]; q < T.runs[2 * r + 1]; ++q) cnt[q]++;
        for (int a = b; a >= 0; a = H.box[a].parent) {
          if (H.box[a].level < 2) continue;
          const int k = k_of[a];
          if (k < 0) { bad += nsrc; continue; }          // a target's ancestor without a far field
          for (int e = T.vl_off[k]; e < T.vl_off[k + 1]; ++e) {
            const HostBox& C = H.box[T.vl_src[e]];
            for (int q = C.pt0[sc]; q < C.pt1[sc]; ++q) cnt[q]++;
          }
        }
        // the leaf's mesh: from its first target point's element
        const int64_t el = H.perm[tc][H.box[b].pt0[tc]] / nqt;
        const int m = (int)(std::upper_bound(toff.begin(), toff.end(), el) - toff.begin()) - 1;
        const int64_t s0 = nqs * soff[m], s1 = nqs * soff[m + 1];
        for (int64_t q = 0; q < nsrc; ++q) bad += (cnt[q] != ((q >= s0 && q < s1) ? 1 : 0));
      }
      out[t] = bad;
    }
    // tensor-core tiles: the (offset code, source box) entries of each row
    // must be exactly the row's interaction list
    if (prm.q0 > 0)
      for (int l = 0; l < BCFMM_MAX_LEVELS; ++l) prm.p_level[l] = std::max(1, std::min(prm.p, prm.q0 + H.nlevels - 1 - l));
    std::vector<int> box_q(H.box.size());
    for (size_t i = 0; i < H.box.size(); ++i) box_q[i] = level_order(prm, H.box[i].level);
    const int qmax = tc_max_order(2);
    for (int t = 0; t < 3; ++t) {
      build_tc_tiles(H, t, 128, box_q, qmax);
      const HostTask& T = H.task[t];
      std::vector<int> k_of(H.box.size(), -1);
      for (size_t k = 0; k < T.m2l_tgt.size(); ++k) k_of[T.m2l_tgt[k]] = (int)k;
      std::vector<std::vector<std::pair<int, int>>> seen(T.m2l_tgt.size());
      int64_t bad = 0;
      const int ntile = (int)T.tc_tile_off.size() - 1;
      for (int tl = 0; tl < ntile; ++tl)
        for (int r = 0; r < 128; ++r) {
          const int tgt = T.tc_tile_tgt[(size_t)tl * 128 + r];
          for (int e = T.tc_tile_off[tl]; e < T.tc_tile_off[tl + 1]; ++e) {
            const int src = T.tc_ent_src[(size_t)e * 128 + r];
            if (src < 0) continue;
            if (tgt < 0 || k_of[tgt] < 0) { ++bad; continue; }
            seen[k_of[tgt]].push_back({T.tc_ent_code[e], src});
          }
        }
      for (size_t k = 0; k < T.m2l_tgt.size(); ++k) {
        std::vector<std::pair<int, int>> want;
        if (box_q[T.m2l_tgt[k]] <= qmax)        // higher orders: CUDA-core M2L, no tile
          for (int e = T.vl_off[k]; e < T.vl_off[k + 1]; ++e) want.push_back({T.vl_code[e], T.vl_src[e]});
        std::sort(want.begin(), want.end());
        std::sort(seen[k].begin(), seen[k].end());
        if (want != seen[k]) bad += (int64_t)std::max(want.size(), seen[k].size());
      }
      // every row of a tile has the tile's expansion order
      for (int tl = 0; tl < ntile; ++tl)
        for (int r = 0; r < 128; ++r) {
          const int tgt = T.tc_tile_tgt[(size_t)tl * 128 + r];
          if (tgt >= 0 && box_q[tgt] != T.tc_tile_q[tl]) ++bad;
        }
      out[3 + t] = bad;
      // the persistent schedule: every entry of every tile in exactly one
      // unit of its order, every unit exactly once in one CTA's sequence with
      // its first / last flags, split tiles with consecutive partial slots
      int64_t sbad = 0;
      for (int nsm : {1, 7, 152}) {
        std::vector<TcOrderSchedHost> sched;
        m2l_tc_schedule(T.tc_tile_off, T.tc_tile_q, T.tc_ent_src, nsm, 2, prm.tc_unit, sched);
        std::vector<int> ecount(T.tc_ent_code.size(), 0);
        for (const TcOrderSchedHost& O : sched) {
          std::vector<int> useen(O.units.size(), 0);
          int nsl = 0;
          for (const int4& sp : O.splits) nsl += sp.z;
          if (nsl != O.nslot) ++sbad;
          for (size_t u = 0; u < O.units.size(); ++u) {
            const int4 U = O.units[u];
            if (U.x < 0 || U.x >= ntile || T.tc_tile_q[U.x] != O.q) { ++sbad; continue; }
            if (U.y < T.tc_tile_off[U.x] || U.z > T.tc_tile_off[U.x + 1] || U.y >= U.z) ++sbad;
            if (U.w >= 0) {
              bool found = false;
              for (const int4& sp : O.splits)
                if (sp.x == U.x && U.w >= sp.y && U.w < sp.y + sp.z) found = true;
              if (!found) ++sbad;
            } else if (U.y != T.tc_tile_off[U.x] || U.z != T.tc_tile_off[U.x + 1]) {
              ++sbad;                       // an uncut tile's unit covers the whole tile
            }
          }
          if ((int)O.seq_off.size() - 1 > nsm || O.seq_off.front() != 0 || O.seq_off.back() != (int)O.seq_e.size()) ++sbad;
          for (size_t i = 0; i < O.seq_e.size(); ++i) {
            const int u = O.seq_u[i] & ((1 << 29) - 1);
            const bool first = (O.seq_u[i] >> 29) & 1, last = (O.seq_u[i] >> 30) & 1;
            if (u < 0 || u >= (int)O.units.size()) { ++sbad; continue; }
            const int4 U = O.units[u];
            const int e = O.seq_e[i];
            if (e < U.y || e >= U.z || first != (e == U.y) || last != (e == U.z - 1)) ++sbad;
            if (i > 0 && !first && (O.seq_e[i - 1] != e - 1)) ++sbad;
            if (e >= 0 && e < (int)ecount.size()) ecount[e]++;
            if (first) useen[u]++;
          }
          for (int v : useen) sbad += (v != 1);
        }
        for (int v : ecount) sbad += (v != 1);
      }
      out[6 + t] = sbad;
      // the Taylor-form schedule: every list entry of a target of orders
      // 1..kTaylorMaxQ exactly once, in a lane whose chunk is the target's,
      // decoding to the entry's (offset code, source box); every chunk in
      // exactly one lane; every other target in the generic kernel's list
      int64_t ybad = 0;
      std::vector<int> tq(T.m2l_tgt.size());
      for (size_t k = 0; k < tq.size(); ++k) tq[k] = box_q[T.m2l_tgt[k]];
      for (int nsm : {1, 7, 152}) {
        std::vector<TaylorOrderHost> ys;
        std::vector<int> sel;
        int cbits = 0;
        if (!m2l_taylor_schedule(T.m2l_tgt, T.vl_off, T.vl_src, T.vl_code, tq, (int)H.box.size(),
                                 (int)(H.offsets.size() / 3), nsm, ys, sel, &cbits)) {
          ++ybad;
          continue;
        }
        std::vector<std::vector<std::pair<int, int>>> got(T.m2l_tgt.size());
        std::vector<int> in_sel(T.m2l_tgt.size(), 0);
        for (int k : sel) {
          if (k < 0 || k >= (int)in_sel.size()) { ++ybad; continue; }
          in_sel[k]++;
        }
        for (const TaylorOrderHost& O : ys) {
          std::vector<int> ctgt(O.nchunk, -1), cseen(O.nchunk, 0);
          if ((int)O.tchunk.size() != (int)O.tgt.size() + 1 || O.tchunk.back() != O.nchunk) { ++ybad; continue; }
          for (size_t i = 0; i < O.tgt.size(); ++i)
            for (int c = O.tchunk[i]; c < O.tchunk[i + 1]; ++c) ctgt[c] = k_of[O.tgt[i]];
          for (size_t w = 0; w < O.wb.size(); ++w)
            for (int l = 0; l < 32; ++l) {
              const int c = O.lane_chunk[w * 32 + l];
              if (c >= O.nchunk) { ++ybad; continue; }
              if (c >= 0) cseen[c]++;
              for (int j = 0; j < O.wb[w].y; ++j) {
                const uint32_t v = O.pk[(size_t)O.wb[w].x + (size_t)j * 32 + l];
                if (v == ~0u) continue;
                if (c < 0 || ctgt[c] < 0) { ++ybad; continue; }
                got[ctgt[c]].push_back({(int)(v & ((1u << cbits) - 1u)), (int)(v >> cbits)});
              }
            }
          for (int v : cseen) ybad += (v != 1);
        }
        for (size_t k = 0; k < T.m2l_tgt.size(); ++k) {
          const bool taylor = tq[k] >= 1 && tq[k] <= kTaylorMaxQ;
          if (in_sel[k] != (taylor ? 0 : 1)) ++ybad;
          std::vector<std::pair<int, int>> want;
          if (taylor && T.vl_off[k + 1] > T.vl_off[k])
            for (int e = T.vl_off[k]; e < T.vl_off[k + 1]; ++e) want.push_back({T.vl_code[e], T.vl_src[e]});
          std::sort(want.begin(), want.end());
          std::sort(got[k].begin(), got[k].end());
          if (want != got[k]) ybad += (int64_t)std::max(want.size(), got[k].size());
        }
      }
      out[9 + t] = ybad;
    }
    // the packed near field's chunk blocks, cut at a small chunk size (so
    // that small meshes split) and at the library's: every source point of a
    // leaf's list in exactly one of its chunks, none other, a chunk within
    // the size, the leaf's own run whole at the front of chunk 0, split
    // leaves with chunks 0..n-1 on disjoint scratch rows, work non-increasing
    for (int t = 0; t < 3; ++t) {
      const HostTask& T = H.task[t];
      int64_t kbad = 0;
      std::vector<int> idx_of(H.box.size(), -1);
      for (size_t i = 0; i < T.p2p_leaf.size(); ++i) idx_of[T.p2p_leaf[i]] = (int)i;
      for (int64_t chunk : {(int64_t)96, kP2pChunk}) {
        P2pChunks K;
        build_p2p_chunks(H, t, chunk, K);
        const size_t nb = K.leaf.size();
        std::vector<std::vector<int>> blocks_of(T.p2p_leaf.size());
        for (size_t b = 0; b < nb; ++b) {
          const int i = idx_of[K.leaf[b]];
          if (i < 0) { ++kbad; continue; }
          blocks_of[i].push_back((int)b);
        }
        std::vector<int> rowuse(K.rows, 0);
        double prev = 1e300;
        for (size_t b = 0; b < nb; ++b) {
          int64_t ns = 0;
          for (int r = K.run_off[b]; r < K.run_off[b + 1]; ++r) ns += K.runs[2 * r + 1] - K.runs[2 * r];
          const HostBox& B = H.box[K.leaf[b]];
          const double w = (double)ns * (B.pt1[T.tgt_cls] - B.pt0[T.tgt_cls] + 8);
          if (w > prev) ++kbad;
          prev = w;
          if (K.grp[b] >= 0 && ns > std::max<int64_t>(chunk, K.self[b])) ++kbad;
        }
        for (size_t i = 0; i < T.p2p_leaf.size(); ++i) {
          std::vector<std::pair<int, int>> want, got;
          for (int r = T.run_off[i]; r < T.run_off[i + 1]; ++r) want.push_back({T.runs[2 * r], T.runs[2 * r + 1]});
          const std::vector<int>& bl = blocks_of[i];
          const int g = bl.empty() ? -2 : K.grp[bl[0]];
          if (bl.empty() || (g < 0 && bl.size() != 1)) { ++kbad; continue; }
          std::vector<int> seen(bl.size(), 0);
          for (int b : bl) {
            if (K.grp[b] != g) { ++kbad; continue; }
            const int c = g < 0 ? 0 : K.chunk[b];
            if (c < 0 || c >= (int)bl.size() || seen[c]++) { ++kbad; continue; }
            if (g >= 0) {
              if (K.grp_n[g] != (int)bl.size() || K.grp_row[g] + c >= K.rows) ++kbad;
              else rowuse[K.grp_row[g] + c]++;
            }
            // the leaf's own run: whole, first, in chunk 0 only
            if (c == 0) {
              if (K.self[b] != T.self_len[i]) ++kbad;
              if (T.self_len[i] > 0 && (K.run_off[b] == K.run_off[b + 1] || K.runs[2 * K.run_off[b]] != T.runs[2 * T.run_off[i]] ||
                                        K.runs[2 * K.run_off[b] + 1] - K.runs[2 * K.run_off[b]] != T.self_len[i]))
                ++kbad;
            } else if (K.self[b] != 0) {
              ++kbad;
            }
            for (int r = K.run_off[b]; r < K.run_off[b + 1]; ++r) got.push_back({K.runs[2 * r], K.runs[2 * r + 1]});
          }
          // the same points: expand both run lists to point counts
          std::vector<int> cw, cg;
          for (auto& pr : want) for (int q = pr.first; q < pr.second; ++q) cw.push_back(q);
          for (auto& pr : got) for (int q = pr.first; q < pr.second; ++q) cg.push_back(q);
          std::sort(cw.begin(), cw.end());
          std::sort(cg.begin(), cg.end());
          if (cw != cg) kbad += (int64_t)std::max(cw.size(), cg.size());
        }
        for (int r = 0; r < K.rows; ++r) kbad += rowuse[r] != 1;
      }
      out[12 + t] = kbad;
    }
  } catch (const std::exception& ex) {
    return fail(BCFMM_ERR_ARG, std::string("debug_list_coverage: ") + ex.what());
  }
  return BCFMM_OK;
}

extern "C" int bcfmm_build_like(const bcfmm_ctx* base, const bcfmm_params* prm, bcfmm_ctx** out) {
  if (out) *out = nullptr;
  if (!base || !prm || !out) return fail(BCFMM_ERR_ARG, "build_like: null argument");
  if (prm->eta_ns != base->prm.eta_ns || prm->near_n != base->prm.near_n || prm->near_k != base->prm.near_k ||
      prm->near_mode != base->prm.near_mode || prm->double_layer != base->prm.double_layer)
    return fail(BCFMM_ERR_ARG,
                "build_like: eta_ns, near_n, near_k, near_mode and double_layer must match the base context");
  int dev = -1;
  CU(cudaGetDevice(&dev));
  if (dev != base->device) return fail(BCFMM_ERR_STATE, "build_like: the base context's device is not current");
  try {
    return build_impl(base->h_verts.data(), base->h_vo.data(), base->h_tets.data(), base->h_to.data(),
                      base->h_tris.empty() ? nullptr : base->h_tris.data(), base->h_ro.data(), base->nmesh, prm,
                      base->st, out, base);
  } catch (const std::bad_alloc&) {
    return fail(BCFMM_ERR_OOM, "build_like: host allocation failed");
  } catch (const std::exception& ex) {
    return fail(BCFMM_ERR_ARG, std::string("build_like: ") + ex.what());
  }
}

static int ensure_work(bcfmm_ctx* C, int ndp) {
  if (C->work_ndp >= ndp) return BCFMM_OK;
  auto& m = C->mem;
  for (void* p : {(void*)C->W64, (void*)C->mom64, (void*)C->loc64, (void*)C->phi, (void*)C->out_dev, (void*)C->W32,
                  (void*)C->mom32, (void*)C->loc32, (void*)C->tc_partial, (void*)C->tc_momb, (void*)C->ty_momp,
                  (void*)C->ty_partial, (void*)C->W64dl, (void*)C->W32dl})
    if (p) m.release(p);
  C->W64dl = nullptr;
  C->W32dl = nullptr;
  C->tc_partial = nullptr;
  C->tc_momb = nullptr;
  C->ty_momp = C->ty_partial = nullptr;
  const int64_t npmax = std::max(C->npts[0], C->npts[1]);
  const int64_t nel = std::max(C->ntet, C->ntri);
  const size_t nexp = (size_t)C->nbox * ndp * C->G.ms;
  const bool f64 = C->prm.precision == BCFMM_FP64;
  CU(m.alloc(&C->phi, (size_t)ndp * npmax));
  CU(m.alloc(&C->out_dev, (size_t)ndp * nel));
  if (C->prm.double_layer && C->npts[1] > 0) {
    if (f64) CU(m.alloc(&C->W64dl, (size_t)ndp * C->npts[1]));
    else CU(m.alloc(&C->W32dl, (size_t)ndp * C->npts[1]));
  }
  if (f64) {
    CU(m.alloc(&C->W64, (size_t)ndp * npmax));
    CU(m.alloc(&C->mom64, nexp));
    CU(m.alloc(&C->loc64, nexp));
    C->W32 = C->mom32 = C->loc32 = nullptr;
  } else {
    CU(m.alloc(&C->W32, (size_t)ndp * npmax));
    CU(m.alloc(&C->mom32, nexp));
    CU(m.alloc(&C->loc32, nexp));
    C->W64 = C->mom64 = C->loc64 = nullptr;
    if (C->tc.nsplit > 0) {
      CU(m.alloc(&C->tc_partial, std::max<size_t>((size_t)ndp * C->tc_partial_per_dens, 1)));
      // split moments: one row per (box, density, part)
      const int kpitch = m2l_tc_kpitch(C->prm.p);
      CU(m.alloc(&C->tc_momb, (size_t)C->nbox * ndp * C->tc.nsplit * kpitch * 2));
    }
    if (C->ty.g) {
      CU(m.alloc(&C->ty_momp, (size_t)C->nbox * ndp * C->ty.gpitch));
      CU(m.alloc(&C->ty_partial, std::max<size_t>((size_t)ndp * C->ty_partial_per_dens, 1)));
    }
  }
  C->work_ndp = ndp;
  C->work_gen++;
  return BCFMM_OK;
}

extern "C" int bcfmm_set_density(bcfmm_ctx* C, int32_t kind, const double* vals, int32_t ndens, int32_t is_device) {
  if (C && kind == BCFMM_DIPOLE && !vals && ndens == 0) {
    C->ndens[kind] = C->ndp[kind] = 0;     // remove the double-layer density
    return BCFMM_OK;
  }
  if (!C || !vals) return fail(BCFMM_ERR_ARG, "set_density: null argument");
  if (kind != BCFMM_VOLUME && kind != BCFMM_BOUNDARY && kind != BCFMM_DIPOLE)
    return fail(BCFMM_ERR_ARG, "set_density: unknown kind");
  if (kind == BCFMM_DIPOLE && !C->prm.double_layer)
    return fail(BCFMM_ERR_STATE, "set_density: double-layer density needs a context built with double_layer = 1");
  if (ndens < 1 || ndens > 16) return fail(BCFMM_ERR_ARG, "set_density: ndens must be in 1..16");
  const int64_t nel = kind == BCFMM_VOLUME ? C->ntet : C->ntri;
  if (nel == 0) return fail(BCFMM_ERR_ARG, "set_density: the mesh has no elements of this kind");
  const size_t n = (size_t)ndens * nel;
  if (!is_device)
    for (size_t i = 0; i < n; ++i)
      if (!std::isfinite(vals[i])) return fail(BCFMM_ERR_MESH, "set_density: value " + std::to_string(i) + " is not finite");
  if (C->ndens[kind] < ndens) {
    if (C->dens[kind]) C->mem.release(C->dens[kind]);
    C->dens[kind] = nullptr;
    CU(C->mem.alloc(&C->dens[kind], (size_t)16 * nel));
    C->work_gen++;
  }
  CU(cudaMemcpyAsync(C->dens[kind], vals, n * sizeof(double), is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     C->st));
  if (!is_device) CU(cudaStreamSynchronize(C->st));
  C->ndens[kind] = ndens;
  C->ndp[kind] = pad_ndens(ndens);
  return ensure_work(C, C->ndp[kind]);
}

// skip_up: the moments and weights already hold this task's source side;
// skip_far: the local expansions already hold this task's far field (both:
// VtB right after VtV of the same volume density in one graph, VtV's lists
// covering every box with tet or triangle points).
static int eval_impl(bcfmm_ctx* C, int t, double* out, int out_is_device, bool skip_up = false,
                     bool skip_far = false) {
  if (!C) return fail(BCFMM_ERR_ARG, "eval: null context");
  TaskDev& D = C->task[t];
  const DevTaskLists& L = D.L;
  const int kind = L.src_cls;     // class 0 sources: volume density; class 1: boundary density
  if (C->ndens[kind] == 0)
    return fail(BCFMM_ERR_STATE, kind == 0 ? "eval: volume density not set" : "eval: boundary density not set");
  if (!out) return fail(BCFMM_ERR_ARG, "eval: null output");
  const int ndens = C->ndens[kind], ndp = C->ndp[kind];
  // BtV with a double-layer density g: V~ q - K~ g (Algorithm 3)
  const bool dl = t == 2 && C->ndens[BCFMM_DIPOLE] > 0;
  if (dl && C->ndens[BCFMM_DIPOLE] != ndens)
    return fail(BCFMM_ERR_STATE, "eval: the double-layer density's ndens differs from the boundary density's");
  const int rc = ensure_work(C, ndp);
  if (rc != BCFMM_OK) return rc;
  cudaStream_t st = C->st;
  const DevGeom& G = C->G;
  const int64_t nsp = C->npts[L.src_cls], ntp = C->npts[L.tgt_cls];
  const int64_t nsel = kind == 0 ? C->ntet : C->ntri;
  const size_t nexp = (size_t)C->nbox * ndp * C->G.ms;
  const bool f64 = C->prm.precision == BCFMM_FP64;
  const bool tc = C->prm.precision == BCFMM_FP32_BF16X2 || C->prm.precision == BCFMM_FP32_BF16X3;
  const bool tm = C->prm.timing && C->ev_ok;
  cudaEvent_t* ev = C->ev[t];
  double* outd = out_is_device ? out : C->out_dev;
  if (tm) CU(cudaEventRecord(ev[0], st));
  if (f64) {
    if (!skip_up) {
      CU(launch_weights<double>(G, L.src_cls, nsp, C->dens[kind], nsel, ndens, ndp, C->W64, st));
      if (dl) CU(launch_weights<double>(G, 1, nsp, C->dens[BCFMM_DIPOLE], nsel, ndens, ndp, C->W64dl, st));
      CU(cudaMemsetAsync(C->mom64, 0, nexp * sizeof(double), st));
    }
    if (!skip_far) CU(cudaMemsetAsync(C->loc64, 0, nexp * sizeof(double), st));
    if (tm) CU(cudaEventRecord(ev[1], st));
    if (!skip_up) {
      CU(launch_p2m<double>(G, L, C->W64, nsp, ndp, C->mom64, st));
      if (dl) CU(launch_p2m_dl<double>(G, L, C->W64dl, nsp, ndp, C->mom64, st));
      for (int l = C->nlevels - 1; l >= 0; --l) {
        const int n = D.m2m_off[l + 1] - D.m2m_off[l];
        CU(launch_m2m<double>(G, D.m2m_parent + D.m2m_off[l], n, ndp, C->mom64, st));
      }
    }
    if (tm) CU(cudaEventRecord(ev[2], st));
    if (!skip_far) CU(launch_m2l_simt<double>(G, L, C->T64, ndp, C->mom64, C->loc64, st));
    if (tm) CU(cudaEventRecord(ev[3], st));
    for (int l = 3; l < C->nlevels && !skip_far; ++l) {
      const int n = D.l2l_off[l + 1] - D.l2l_off[l];
      CU(launch_l2l<double>(G, D.l2l_child + D.l2l_off[l], n, ndp, C->loc64, st));
    }
    if (tm) CU(cudaEventRecord(ev[4], st));
    CU(launch_p2p_l2p_f64(G, L, C->W64, nsp, ntp, ndp, C->loc64, C->phi, st));
    if (dl) CU(launch_p2p_dl<double>(G, L, C->W64dl, nsp, ntp, ndp, C->phi, st));
  } else {
    if (!skip_up) {
      CU(launch_weights<float>(G, L.src_cls, nsp, C->dens[kind], nsel, ndens, ndp, C->W32, st));
      if (dl) CU(launch_weights<float>(G, 1, nsp, C->dens[BCFMM_DIPOLE], nsel, ndens, ndp, C->W32dl, st));
      CU(cudaMemsetAsync(C->mom32, 0, nexp * sizeof(float), st));
    }
    if (!skip_far) CU(cudaMemsetAsync(C->loc32, 0, nexp * sizeof(float), st));
    if (tm) CU(cudaEventRecord(ev[1], st));
    if (!skip_up) {
      CU(launch_p2m<float>(G, L, C->W32, nsp, ndp, C->mom32, st));
      if (dl) CU(launch_p2m_dl<float>(G, L, C->W32dl, nsp, ndp, C->mom32, st));
      for (int l = C->nlevels - 1; l >= 0; --l) {
        const int n = D.m2m_off[l + 1] - D.m2m_off[l];
        CU(launch_m2m<float>(G, D.m2m_parent + D.m2m_off[l], n, ndp, C->mom32, st));
      }
    }
    if (tm) CU(cudaEventRecord(ev[2], st));
    if (skip_far) {
    } else if (tc) {
      CU(launch_m2l_tc(G, L, D.tcs, C->tc, ndp, C->mom32, C->loc32, C->tc_partial, C->tc_momb, st));
      if (D.tcs.nsimt > 0) CU(launch_m2l_simt<float>(G, L, C->T32, ndp, C->mom32, C->loc32, st, D.tcs.simt_sel, D.tcs.nsimt));
    } else if (C->ty.g) {
      CU(launch_m2l_taylor(G, L, D.tys, C->ty, ndp, C->mom32, C->loc32, C->ty_momp, C->ty_partial, st));
    } else {
      CU(launch_m2l_simt<float>(G, L, C->T32, ndp, C->mom32, C->loc32, st));
    }
    if (tm) CU(cudaEventRecord(ev[3], st));
    for (int l = 3; l < C->nlevels && !skip_far; ++l) {
      const int n = D.l2l_off[l + 1] - D.l2l_off[l];
      CU(launch_l2l<float>(G, D.l2l_child + D.l2l_off[l], n, ndp, C->loc32, st));
    }
    if (tm) CU(cudaEventRecord(ev[4], st));
    CU(launch_p2p_l2p_f32(G, L, C->W32, nsp, ntp, ndp, C->loc32, C->phi, st));
    if (dl) CU(launch_p2p_dl<float>(G, L, C->W32dl, nsp, ntp, ndp, C->phi, st));
  }
  if (tm) CU(cudaEventRecord(ev[5], st));
  CU(launch_elem_sum(G, L, C->phi, ntp, C->dens[kind], ndens, outd, st, dl ? C->dens[BCFMM_DIPOLE] : nullptr));
  if (tm) CU(cudaEventRecord(ev[6], st));
  if (!out_is_device) {
    CU(cudaMemcpyAsync(out, C->out_dev, (size_t)ndens * L.ntgt_el * sizeof(double), cudaMemcpyDeviceToHost, st));
    int herr = 0;
    CU(cudaMemcpyAsync(&herr, C->err, sizeof(int), cudaMemcpyDeviceToHost, st));
    CU(cudaStreamSynchronize(st));
    if (herr) {
      CU(cudaMemsetAsync(C->err, 0, sizeof(int), st));
      return fail(BCFMM_ERR_TIMEOUT, "eval: a bounded device wait expired (tensor-core M2L); results are invalid");
    }
  }
  C->ev_rec[t] = tm;
  return BCFMM_OK;
}

extern "C" int bcfmm_eval_vtv(bcfmm_ctx* C, double* out, int32_t d) { return eval_impl(C, 0, out, d); }
extern "C" int bcfmm_eval_vtb(bcfmm_ctx* C, double* out, int32_t d) { return eval_impl(C, 1, out, d); }
extern "C" int bcfmm_eval_btv(bcfmm_ctx* C, double* out, int32_t d) { return eval_impl(C, 2, out, d); }

// Several tasks through one CUDA graph.  The graph is captured on a
// library-owned stream the first time a (task mask, outputs, density
// sizes, work buffers) combination is seen, and replayed on the context's
// stream afterwards.  VtB right after VtV reuses VtV's upward pass and its
// local expansions (same volume density and source points, so the same
// interaction lists; VtV's far field covers the boxes of both).
extern "C" int bcfmm_eval_graph(bcfmm_ctx* C, int32_t mask, double* out_vtv, double* out_vtb, double* out_btv) {
  if (!C) return fail(BCFMM_ERR_ARG, "eval_graph: null context");
  if (mask <= 0 || mask > 7) return fail(BCFMM_ERR_ARG, "eval_graph: task mask must be a non-empty subset of 1|2|4");
  double* outs[3] = {out_vtv, out_vtb, out_btv};
  for (int t = 0; t < 3; ++t) {
    if (!(mask >> t & 1)) { outs[t] = nullptr; continue; }
    const int kind = C->task[t].L.src_cls;
    if (C->ndens[kind] == 0)
      return fail(BCFMM_ERR_STATE, kind == 0 ? "eval_graph: volume density not set" : "eval_graph: boundary density not set");
    if (!outs[t]) return fail(BCFMM_ERR_ARG, "eval_graph: null output for a task in the mask");
    const int rc = ensure_work(C, C->ndp[kind]);
    if (rc != BCFMM_OK) return rc;
  }
  auto& g = C->graph;
  const bool same = g.exec && g.mask == mask && g.work_gen == C->work_gen && g.ndens[0] == C->ndens[0] &&
                    g.ndens[1] == C->ndens[1] && g.ndens[2] == C->ndens[2] && std::equal(outs, outs + 3, g.out);
  if (!same) {
    if (g.exec) { cudaGraphExecDestroy(g.exec); g.exec = nullptr; }
    if (!C->cap_st) CU(cudaStreamCreateWithFlags(&C->cap_st, cudaStreamNonBlocking));
    cudaStream_t user = C->st;
    const int timing = C->prm.timing;
    C->st = C->cap_st;
    C->prm.timing = 0;
    CU(cudaStreamBeginCapture(C->cap_st, cudaStreamCaptureModeRelaxed));
    int rc = BCFMM_OK;
    for (int t = 0; t < 3 && rc == BCFMM_OK; ++t)
      if (mask >> t & 1) rc = eval_impl(C, t, outs[t], 1, t == 1 && (mask & 1), t == 1 && (mask & 1));
    cudaGraph_t graph = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(C->cap_st, &graph);
    C->st = user;
    C->prm.timing = timing;
    if (rc != BCFMM_OK) { if (graph) cudaGraphDestroy(graph); return rc; }
    if (ce != cudaSuccess) return fail(BCFMM_ERR_CUDA, std::string("eval_graph: capture failed: ") + cudaGetErrorString(ce));
    int nkernel = 0;
    {
      size_t nn = 0;
      if (cudaGraphGetNodes(graph, nullptr, &nn) == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        if (cudaGraphGetNodes(graph, nodes.data(), &nn) == cudaSuccess)
          for (size_t i = 0; i < nn; ++i) {
            cudaGraphNodeType ty;
            if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++nkernel;
          }
      }
    }
    const cudaError_t ie = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) { g.exec = nullptr; return fail(BCFMM_ERR_CUDA, std::string("eval_graph: instantiate: ") + cudaGetErrorString(ie)); }
    g.mask = mask;
    g.work_gen = C->work_gen;
    g.ndens[0] = C->ndens[0];
    g.ndens[1] = C->ndens[1];
    g.ndens[2] = C->ndens[2];
    std::copy(outs, outs + 3, g.out);
    g.nodes = nkernel;
  }
  CU(cudaGraphLaunch(g.exec, C->st));
  C->ev_rec[0] = C->ev_rec[1] = C->ev_rec[2] = false;
  return BCFMM_OK;
}

// One task, one density, no allocation: the tensor-core M2L writes its unit
// partial sums into the library's fixed static device array instead of the
// context's scratch; every other buffer was sized by an earlier
// bcfmm_set_density.  Nothing here calls cudaMalloc, cudaFree or an
// allocating library routine.
extern "C" int bcfmm_eval_noalloc(bcfmm_ctx* C, int32_t task, const double* dens_dev, double* out_dev) {
  if (!C) return fail(BCFMM_ERR_ARG, "eval_noalloc: null context");
  if (task < 0 || task > 2) return fail(BCFMM_ERR_ARG, "eval_noalloc: task must be 0 (VtV), 1 (VtB) or 2 (BtV)");
  if (!dens_dev || !out_dev) return fail(BCFMM_ERR_ARG, "eval_noalloc: null density or output");
  const bool tcp = C->prm.precision == BCFMM_FP32_BF16X2 || C->prm.precision == BCFMM_FP32_BF16X3;
  const bool typ = C->prm.precision == BCFMM_FP32;
  if (!tcp && !typ)
    return fail(BCFMM_ERR_ARG, "eval_noalloc: needs a context built with precision FP32 or a BF16 split");
  TaskDev& D = C->task[task];
  const DevTaskLists& L = D.L;
  const int kind = L.src_cls;
  if (C->work_ndp < 1 || (tcp && C->tc_momb == nullptr) || (typ && C->ty.g && C->ty_momp == nullptr))
    return fail(BCFMM_ERR_STATE, "eval_noalloc: call bcfmm_set_density once first (it sizes the work buffers)");
  int dev = -1;
  CU(cudaGetDevice(&dev));
  if (dev != C->device) return fail(BCFMM_ERR_STATE, "eval_noalloc: the context's device is not the current device");
  float2* partial = nullptr;
  size_t cap = 0;
  CU(m2l_tc_noalloc_scratch(dev, &partial, &cap));
  // tensor cores: float2 unit sums; Taylor form: float chunk sums
  const size_t need = tcp ? D.tcs.partial_per_dens : (D.tys.partial_per_dens + 1) / 2;
  if (need > cap)
    return fail(BCFMM_ERR_ARG, "eval_noalloc: the mesh needs " + std::to_string(need * sizeof(float2)) +
                                   " bytes of M2L scratch, more than the fixed " + std::to_string(cap * sizeof(float2)) +
                                   " bytes (use bcfmm_eval_vtv/vtb/btv)");
  cudaStream_t st = C->st;
  const DevGeom& G = C->G;
  const int ndp = 1;
  const int64_t nsp = C->npts[L.src_cls], ntp = C->npts[L.tgt_cls];
  const int64_t nsel = kind == 0 ? C->ntet : C->ntri;
  const size_t nexp = (size_t)C->nbox * ndp * C->G.ms;
  CU(launch_weights<float>(G, L.src_cls, nsp, dens_dev, nsel, 1, ndp, C->W32, st));
  CU(cudaMemsetAsync(C->mom32, 0, nexp * sizeof(float), st));
  CU(cudaMemsetAsync(C->loc32, 0, nexp * sizeof(float), st));
  CU(launch_p2m<float>(G, L, C->W32, nsp, ndp, C->mom32, st));
  for (int l = C->nlevels - 1; l >= 0; --l) {
    const int n = D.m2m_off[l + 1] - D.m2m_off[l];
    CU(launch_m2m<float>(G, D.m2m_parent + D.m2m_off[l], n, ndp, C->mom32, st));
  }
  if (tcp) {
    CU(launch_m2l_tc(G, L, D.tcs, C->tc, ndp, C->mom32, C->loc32, partial, C->tc_momb, st));
    if (D.tcs.nsimt > 0) CU(launch_m2l_simt<float>(G, L, C->T32, ndp, C->mom32, C->loc32, st, D.tcs.simt_sel, D.tcs.nsimt));
  } else if (C->ty.g) {
    CU(launch_m2l_taylor(G, L, D.tys, C->ty, ndp, C->mom32, C->loc32, C->ty_momp, reinterpret_cast<float*>(partial), st));
  } else {
    CU(launch_m2l_simt<float>(G, L, C->T32, ndp, C->mom32, C->loc32, st));
  }
  for (int l = 3; l < C->nlevels; ++l) {
    const int n = D.l2l_off[l + 1] - D.l2l_off[l];
    CU(launch_l2l<float>(G, D.l2l_child + D.l2l_off[l], n, ndp, C->loc32, st));
  }
  CU(launch_p2p_l2p_f32(G, L, C->W32, nsp, ntp, ndp, C->loc32, C->phi, st));
  CU(launch_elem_sum(G, L, C->phi, ntp, dens_dev, 1, out_dev, st));
  C->ev_rec[task] = false;             // no stage timings recorded by this call
  return BCFMM_OK;
}

extern "C" int bcfmm_direct_sample(bcfmm_ctx* C, int32_t task, const int64_t* targets, int64_t n, double* out) {
  if (!C || !targets || !out || n < 0) return fail(BCFMM_ERR_ARG, "direct_sample: null argument");
  if (task < 0 || task > 2) return fail(BCFMM_ERR_ARG, "direct_sample: task must be 0, 1 or 2");
  if (n > (1 << 20)) return fail(BCFMM_ERR_ARG, "direct_sample: at most 2^20 targets");
  const DevTaskLists& L = C->task[task].L;
  const int kind = L.src_cls;
  if (C->ndens[kind] == 0) return fail(BCFMM_ERR_STATE, "direct_sample: density not set");
  for (int64_t i = 0; i < n; ++i)
    if (targets[i] < 0 || targets[i] >= L.ntgt_el) return fail(BCFMM_ERR_ARG, "direct_sample: target index out of range");
  if (n == 0) return BCFMM_OK;
  const int nd = C->ndens[kind];
  // a target sees the sources of its own mesh only (sorted points are mesh after mesh)
  const std::vector<int64_t>& toff = L.tgt_cls == 0 ? C->mesh_tet_off : C->mesh_tri_off;
  const std::vector<int64_t>& soff = L.src_cls == 0 ? C->mesh_tet_off : C->mesh_tri_off;
  const int nqs = L.src_cls == 0 ? 4 : 3;
  std::vector<int64_t> hbuf(3 * n);
  for (int64_t i = 0; i < n; ++i) {
    const int m = (int)(std::upper_bound(toff.begin(), toff.end(), targets[i]) - toff.begin()) - 1;
    hbuf[i] = targets[i];
    hbuf[n + 2 * i] = nqs * soff[m];
    hbuf[n + 2 * i + 1] = nqs * soff[m + 1];
  }
  int64_t* dt = nullptr;
  double* dout = nullptr;
  CU(cudaMalloc((void**)&dt, 3 * n * sizeof(int64_t)));
  cudaError_t e = cudaMalloc((void**)&dout, (size_t)n * nd * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyAsync(dt, hbuf.data(), 3 * n * sizeof(int64_t), cudaMemcpyHostToDevice, C->st);
  if (e == cudaSuccess) e = launch_direct_sample(C->G, L, dt, dt + n, (int)n, C->dens[kind], nd, dout, C->st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, dout, (size_t)n * nd * sizeof(double), cudaMemcpyDeviceToHost, C->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(C->st);
  cudaFree(dt);
  cudaFree(dout);
  if (e != cudaSuccess) return fail(BCFMM_ERR_CUDA, std::string("direct_sample: ") + cudaGetErrorString(e));
  return BCFMM_OK;
}

extern "C" int64_t bcfmm_mlp_blob_size(void) { return kMlpBlobBytes; }

extern "C" int bcfmm_mlp_dataset(bcfmm_ctx* C, int32_t task, int64_t max_pairs, float* feat, float* qhat, float* chat,
                                 int32_t* bin, int32_t* pairs, int64_t* n_out) {
  if (!C || !feat || !qhat || !chat || !bin || !n_out || max_pairs < 0) return fail(BCFMM_ERR_ARG, "mlp_dataset: null argument");
  if (task < 0 || task > 2) return fail(BCFMM_ERR_ARG, "mlp_dataset: task must be 0, 1 or 2");
  *n_out = 0;
  TaskDev& D = C->task[task];
  const NearGeom& g = D.ng;
  if (!g.ns_list) return fail(BCFMM_ERR_STATE, "mlp_dataset: the context was not built with near_mode 1 or 2");
  const int64_t mcount = std::min(max_pairs, D.n_singular);
  if (mcount == 0) return BCFMM_OK;
  cudaStream_t st = C->st;
  int64_t* sel = nullptr;
  double *Cv = nullptr, *Q = nullptr;
  cudaError_t e = cudaMalloc((void**)&sel, mcount * sizeof(int64_t));
  if (e == cudaSuccess) e = cudaMalloc((void**)&Cv, mcount * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc((void**)&Q, mcount * sizeof(double));
  if (e == cudaSuccess) e = launch_select_strided(g.ns_list, D.n_singular, mcount, sel, st);
  if (e == cudaSuccess)
    e = launch_pair_data(task, sel, mcount, g.row, D.L.cor_col, g.tv, g.sv, feat, qhat, Q, bin, pairs, st);
  if (e == cudaSuccess)
    e = launch_near_rule(task, mcount, sel, g.row, D.L.cor_col, g.tv, g.sv, g.tqp, g.tqw, g.sqp, g.sqw, g.glx, g.glw,
                         C->prm.near_n, C->prm.near_k, 1, Cv, st);
  if (e == cudaSuccess) e = launch_label_ratio(Cv, Q, mcount, chat, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(sel);
  cudaFree(Cv);
  cudaFree(Q);
  if (e != cudaSuccess) return fail(BCFMM_ERR_CUDA, std::string("mlp_dataset: ") + cudaGetErrorString(e));
  *n_out = mcount;
  return BCFMM_OK;
}

extern "C" int bcfmm_mlp_grad(const float* params, const float* feat, const float* qhat, const float* chat, int64_t n,
                              float* grad, float* loss, void* stream) {
  if (!params || !grad || !loss || n < 0 || (n > 0 && (!feat || !qhat || !chat)))
    return fail(BCFMM_ERR_ARG, "mlp_grad: null argument");
  const cudaError_t e = launch_mlp_grad(params, feat, qhat, chat, n, grad, loss, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(BCFMM_ERR_CUDA, std::string("mlp_grad: ") + cudaGetErrorString(e));
  return BCFMM_OK;
}

extern "C" int bcfmm_mlp_adam(float* params, const float* grad, float* m1, float* m2, int32_t step, float lr,
                              float beta1, float beta2, float eps, void* stream) {
  if (!params || !grad || !m1 || !m2 || step < 1) return fail(BCFMM_ERR_ARG, "mlp_adam: bad argument");
  const cudaError_t e = launch_mlp_adam(params, grad, m1, m2, step, lr, beta1, beta2, eps, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(BCFMM_ERR_CUDA, std::string("mlp_adam: ") + cudaGetErrorString(e));
  return BCFMM_OK;
}

extern "C" int bcfmm_mlp_predict(const float* params, const float* feat, const float* qhat, int64_t n, float* out,
                                 void* stream) {
  if (!params || !out || n < 0 || (n > 0 && (!feat || !qhat))) return fail(BCFMM_ERR_ARG, "mlp_predict: null argument");
  const cudaError_t e = launch_mlp_predict(params, feat, qhat, n, out, (cudaStream_t)stream);
  if (e != cudaSuccess) return fail(BCFMM_ERR_CUDA, std::string("mlp_predict: ") + cudaGetErrorString(e));
  return BCFMM_OK;
}

extern "C" int bcfmm_measure_ffma(int32_t device, double* flops) {
  if (!flops) return fail(BCFMM_ERR_ARG, "measure_ffma: null output");
  int cur = -1;
  CU(cudaGetDevice(&cur));
  if (device != cur) CU(cudaSetDevice(device));
  const cudaError_t e = measure_ffma_rate(device, flops);
  if (device != cur) cudaSetDevice(cur);
  if (e != cudaSuccess) return fail(BCFMM_ERR_CUDA, std::string("measure_ffma: ") + cudaGetErrorString(e));
  return BCFMM_OK;
}

extern "C" int bcfmm_debug_expire_wait(bcfmm_ctx* C, int32_t spins) {
  if (!C || spins < 1 || spins > (1 << 20)) return fail(BCFMM_ERR_ARG, "debug_expire_wait: null context or spins not in 1..2^20");
  CU(launch_debug_expire_wait(C->err, spins, C->st));
  return BCFMM_OK;
}

extern "C" int bcfmm_stats(const bcfmm_ctx* C, char* json, size_t cap) {
  if (!C || !json) return fail(BCFMM_ERR_ARG, "stats: null argument");
  std::string s = "{";
  auto kv = [&](const char* k, double v, bool last = false) {
    char b[96];
    snprintf(b, sizeof b, "\"%s\": %.17g%s", k, v, last ? "" : ", ");
    s += b;
  };
  kv("ntet", (double)C->ntet); kv("ntri", (double)C->ntri);
  kv("npts_tet", (double)C->npts[0]); kv("npts_tri", (double)C->npts[1]);
  {
    int herr = 0;
    if (C->err) { cudaMemcpy(&herr, C->err, sizeof(int), cudaMemcpyDeviceToHost); }
    kv("device_error", herr);
  }
  kv("p", C->prm.p); kv("np", C->np); kv("eta0", C->prm.eta0); kv("n_offsets", C->ncode); kv("leaf_size", C->prm.leaf_size); kv("precision", C->prm.precision);
  kv("near_mode", C->prm.near_mode); kv("tc_unit", C->prm.tc_unit);
  kv("graph_kernels", C->graph.exec ? C->graph.nodes : 0); kv("graph_mask", C->graph.exec ? C->graph.mask : 0);
  kv("nbox", C->nbox); kv("nleaf", C->nleaf); kv("nlevels", C->nlevels);
  kv("nmesh", C->nmesh); kv("host_setup_s", C->sec_host);
  kv("setup_s", C->sec_setup); kv("tree_s", C->sec_tree); kv("lists_s", C->sec_lists);
  kv("near_search_s", C->sec_near_host); kv("near_rule_s", C->sec_near_dev);
  const char* names[3] = {"vtv", "vtb", "btv"};
  s += "\"level_order\": [";
  for (int l = 0; l < C->nlevels; ++l) s += std::to_string(level_order(C->prm, l)) + (l + 1 < C->nlevels ? ", " : "");
  s += "], ";
  for (int t = 0; t < 3; ++t) {
    char b[900];
    const TaskDev& D = C->task[t];
    std::string per_q = "[";
    for (int q = 1; q <= kTcMaxQ; ++q) {
      const TcOrderSched& O = D.tcs.ord[q];
      if (O.nunit == 0) continue;
      if (per_q.size() > 1) per_q += ", ";
      per_q += "{\"q\": " + std::to_string(q) + ", \"entries\": " + std::to_string(O.nent) + ", \"rows\": " +
               std::to_string(O.rows) + ", \"units\": " + std::to_string(O.nunit) + ", \"ctas\": " +
               std::to_string(O.ncta) + ", \"split_tiles\": " + std::to_string(O.nsplit_tiles) + "}";
    }
    per_q += "], \"taylor_orders\": [";
    bool first_ty = true;
    for (int q = 1; q <= kTaylorMaxQ; ++q) {
      const TaylorOrderSched& O = D.tys.ord[q];
      if (O.nwarp == 0) continue;
      if (!first_ty) per_q += ", ";
      first_ty = false;
      per_q += "{\"q\": " + std::to_string(q) + ", \"pairs\": " + std::to_string(O.pairs) + ", \"targets\": " +
               std::to_string(O.ntgt) + ", \"chunk\": " + std::to_string(O.chunk) + ", \"chunks\": " +
               std::to_string(O.nchunk) + ", \"warps\": " + std::to_string(O.nwarp) + "}";
    }
    per_q += "], \"m2l_pairs_by_order\": [";
    for (int q = 0; q <= C->prm.p; ++q) per_q += std::to_string(D.m2l_pairs_q[q]) + (q < C->prm.p ? ", " : "");
    per_q += "], \"generic_m2l_targets\": " + std::to_string(C->ty.g ? D.tys.nsimt : (D.tcs.nsimt > 0 ? D.tcs.nsimt : 0));
    per_q += ", \"p2p_sources_per_leaf\": [";
    for (int k = 0; k < 5; ++k) per_q += std::to_string(D.p2p_src_q[k]) + (k < 4 ? ", " : "]");
    snprintf(b, sizeof b,
             "\"%s\": {\"p2p_pairs\": %lld, \"near_boxes\": %lld, \"m2l_pairs\": %lld, \"near_pairs\": %lld, "
             "\"p2p_leaves\": %d, \"m2l_targets\": %d, \"p2m_leaves\": %d, \"tc_entries\": %lld, "
             "\"tc_rows\": %lld, \"tc_mma_flop\": %.17g, "
             "\"near_singular\": %lld, \"near_learned\": %lld, \"near_fp64\": %lld, \"tc_orders\": ",
             names[t], (long long)D.p2p_pairs, (long long)D.near_boxes, (long long)D.m2l_pairs, (long long)D.nnz,
             D.L.n_p2p, D.L.n_m2l, D.L.n_p2m, (long long)D.tc_entries, (long long)D.tc_rows, D.tc_mma_flop,
             (long long)D.n_singular, (long long)D.n_learned,
             (long long)(C->prm.near_mode == 0 ? D.nnz : D.n_fp64));
    s += b;
    s += per_q + "}, ";
  }
  // stages: weights+clear, P2M+M2M, M2L, L2L, L2P+P2P, element sums+corrections
  s += "\"stage_ms\": {";
  for (int t = 0; t < 3; ++t) {
    s += std::string("\"") + names[t] + "\": [";
    for (int i = 0; i < 6; ++i) {
      float ms = -1.f;
      if (C->ev_rec[t] && cudaEventSynchronize(C->ev[t][6]) == cudaSuccess)
        cudaEventElapsedTime(&ms, C->ev[t][i], C->ev[t][i + 1]);
      char b[32];
      snprintf(b, sizeof b, "%.6g%s", ms, i < 5 ? ", " : "");
      s += b;
    }
    s += t < 2 ? "], " : "]";
  }
  s += "}, \"leaves_per_level\": [";
  for (size_t i = 0; i < C->leaves_per_level.size(); ++i) s += std::to_string(C->leaves_per_level[i]) + (i + 1 < C->leaves_per_level.size() ? ", " : "");
  s += "], \"boxes_per_level\": [";
  for (size_t i = 0; i < C->boxes_per_level.size(); ++i) s += std::to_string(C->boxes_per_level[i]) + (i + 1 < C->boxes_per_level.size() ? ", " : "");
  s += "]}";
  if (s.size() + 1 > cap) return fail(BCFMM_ERR_ARG, "stats: buffer too small, need " + std::to_string(s.size() + 1));
  std::memcpy(json, s.c_str(), s.size() + 1);
  return BCFMM_OK;
}

extern "C" void bcfmm_destroy(bcfmm_ctx* C) {
  if (!C) return;
  cudaStreamSynchronize(C->st);
  if (C->ev_ok)
    for (auto& row : C->ev)
      for (auto& ev : row) cudaEventDestroy(ev);
  if (C->graph.exec) cudaGraphExecDestroy(C->graph.exec);
  if (C->cap_st) cudaStreamDestroy(C->cap_st);
  m2l_tc_free_tables(&C->tc);
  C->mem.free_all();
  delete C;
}
