// Device-side declarations shared by the bcfmm translation units.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace bcfmm {

__host__ __device__ __forceinline__ int nterms_q(int q) { return q < 0 ? 0 : (q + 1) * (q + 2) * (q + 3) / 6; }

// Geometry and lists the evaluation kernels read (device pointers).
struct DevGeom {
  int np;                        // nterms(p)
  int ms;                        // row stride of moment / local arrays (np rounded up to 4)
  int p;
  int nbox;
  const int* mi;                 // packed multi-indices a | b << 8 | c << 16, degree-major
  const int* box_q;              // expansion order of each box's level (<= p; Sec. 4.3)
  const double4_32a* box_cs;         // centre xyz, side s
  const int* box_child0;
  const int* box_nchild;
  const int* box_octant;
  const int* box_parent;
  const int2* box_rng[2];        // point range per class
  const double4_32a* pt64[2];        // sorted points: x, y, z, quadrature weight
  const float4* pthi[2];         // float hi parts (x, y, z, weight)
  const float4* ptlo[2];         // float lo parts (x - hi, ...)
  const int* pt_elem[2];         // sorted point -> element
  const double4_32a* tri_nrm;    // unit normal of each triangle (right-hand rule; w unused)
  const double* shift64;         // [2][p+1][p+1] C(n, k) (-+1/4)^(n-k): M2M / L2L 1-D shifts
  const float* shift32;
};

struct DevTaskLists {
  int n_p2p; const int* p2p_leaf; const int* near_off; const int* near_box;
  const int* run_off; const int2* runs; const int* self_len;   // merged source runs per target leaf
  int n_m2l; const int* m2l_tgt; const int* vl_off; const int* vl_src; const uint16_t* vl_code;
  int n_p2m; const int* p2m_leaf;
  int n_l2p; const int* l2p_leaf;
  int64_t ntgt_el, nsrc_el;
  const int64_t* cor_off; const int* cor_col; const double* cor_val;
  const double* cor_val_dl;      // BtV: near-rule corrections of dG/dn_y (same CSR), or null
  const int* elem_pts;           // [ntgt_el][4] sorted positions of the element's points (-1 pad)
  int nq_tgt;                    // 4 (tets) or 3 (triangles)
  int src_cls, tgt_cls;
  // tensor-core M2L tiles: 128 targets of one expansion order and one
  // octant per tile (the entries' source rows live in the schedule)
  int tc_ntile;
  const int* tc_tile_tgt;        // [ntile][128]
  int* err;                      // device error word (bounded waits)
  // the packed FP32 near field's blocks: target leaves whose source lists
  // exceed one chunk are cut into chunks (runs split at chunk boundaries);
  // a chunk block writes its per-target sums to its scratch row and the
  // last chunk of a leaf to finish (ticket counter) adds the rows in chunk
  // order and evaluates L2P
  int sp_n;                      // blocks
  const int* sp_leaf;            // [sp_n] target leaf box
  const int* sp_run_off;         // [sp_n + 1] into sp_runs
  const int2* sp_runs;           // source runs (start, end) of the chunks
  const int* sp_self;            // [sp_n] points of the leaf's own run (chunk 0 of a VtV list), else 0
  const int2* sp_grp;            // [sp_n] (split leaf index or -1, chunk index)
  const int2* grp_info;          // [split leaves] (first scratch row, chunks)
  unsigned* grp_cnt;             // [split leaves] tickets, zero between launches
  float2* sp_scratch;            // [rows][ND][128] (hi, lo) per target
};

// launchers (return cudaGetLastError())
template <typename T>
cudaError_t launch_weights(const DevGeom& G, int cls, int64_t n, const double* dens, int64_t nel, int ndens,
                           int ndp, T* W, cudaStream_t st);
template <typename T>
cudaError_t launch_p2m(const DevGeom& G, const DevTaskLists& L, const T* W, int64_t nsrc_pts, int ndp,
                       T* mom, cudaStream_t st);
template <typename T>
cudaError_t launch_m2m(const DevGeom& G, const int* parents, int n, int ndp, T* mom, cudaStream_t st);
// sel: optional list of indices into L.m2l_tgt (nsel of them); NULL: every target
template <typename T>
cudaError_t launch_m2l_simt(const DevGeom& G, const DevTaskLists& L, const T* Tt, int ndp, const T* mom, T* loc,
                            cudaStream_t st, const int* sel = nullptr, int nsel = 0);
template <typename T>
cudaError_t launch_l2l(const DevGeom& G, const int* children, int n, int ndp, T* loc, cudaStream_t st);
cudaError_t launch_p2p_l2p_f32(const DevGeom& G, const DevTaskLists& L, const float* W, int64_t nsrc_pts,
                               int64_t ntgt_pts, int ndp, const float* loc, double* phi, cudaStream_t st);
cudaError_t launch_p2p_l2p_f64(const DevGeom& G, const DevTaskLists& L, const double* W, int64_t nsrc_pts,
                               int64_t ntgt_pts, int ndp, const double* loc, double* phi, cudaStream_t st);
// dens_dl: BtV double-layer density (subtracts its corrections L.cor_val_dl), or null
cudaError_t launch_elem_sum(const DevGeom& G, const DevTaskLists& L, const double* phi, int64_t ntgt_pts,
                            const double* dens_src, int ndens, double* out, cudaStream_t st,
                            const double* dens_dl = nullptr);
// BtV double layer (Algorithm 3): moments -<gamma_1 (y-c)^b, g> added to mom,
// near field -sum Wg n.(x-y)/(4 pi r^3) subtracted from phi
template <typename T>
cudaError_t launch_p2m_dl(const DevGeom& G, const DevTaskLists& L, const T* W, int64_t nsrc_pts, int ndp, T* mom,
                          cudaStream_t st);
template <typename T>
cudaError_t launch_p2p_dl(const DevGeom& G, const DevTaskLists& L, const T* W, int64_t nsrc_pts, int64_t ntgt_pts,
                          int ndp, double* phi, cudaStream_t st);

// FP32 FMA throughput of the device (flop/s, 2 per FMA), CUDA events
cudaError_t measure_ffma_rate(int device, double* flops);

// FP64 direct evaluation of sampled target elements (out [ndens][n]);
// src_rng [n][2]: sorted source point range of each target's mesh
cudaError_t launch_direct_sample(const DevGeom& G, const DevTaskLists& L, const int64_t* targets, const int64_t* src_rng,
                                 int n, const double* dens, int ndens, double* out, cudaStream_t st);

// setup: near-rule corrections C_ts = N_ts - Q_ts (FP64); task 0 VtV,
// 1 VtB, 2 BtV single layer, 3 BtV double layer (kernel dG/dn_y)
// (sel: optional list of CSR positions; nnz is then its length)
cudaError_t launch_near_rule(int task, int64_t nnz, const int64_t* sel, const int* row, const int* col,
                             const double* tgt_v, const double* src_v,
                             const double* tgt_qp, const double* tgt_qw,
                             const double* src_qp, const double* src_qw,
                             const double* glx, const double* glw, int n, int k, int compact,
                             double* cor_val, cudaStream_t st);

}  // namespace bcfmm
