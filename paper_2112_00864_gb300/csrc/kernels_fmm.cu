// Evaluation kernels of the boundary-concentrated FMM (Sec. 3.3, Algorithms
// 1-3): source weights, moments (P2M), upward pass (M2M), interaction phase
// on CUDA cores (M2L), downward pass (L2L), evaluation fused with the near
// field (L2P + P2P over the extended neighbour list N*), and the Galerkin
// element sums plus near-rule corrections.
//
// Expansions are box-scaled: moments m^b = sum_j W_j ((y_j - c)/s)^b, locals
// phi(x) = sum_a l^a ((x - c)/s)^a, so one M2L table per integer offset
// serves every level (the 1/s factor is applied here).
#include <cstdio>

#include "kernels.cuh"

namespace bcfmm {

constexpr double kInv4Pi = 0.079577471545947667884441881686257;

// ------------------------------------------------------------ weights
// W[d][j] = w_j * dens[d][elem(j)] (d < ndens), zero for ndens <= d < ndp.
template <typename T>
__global__ void k_weights(const double4_32a* __restrict__ pt, const int* __restrict__ elem, int64_t n,
                          const double* __restrict__ dens, int64_t nel, int ndens, int ndp, T* __restrict__ W) {
  int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (j >= n) return;
  double w = pt[j].w;
  int e = elem[j];
  for (int d = 0; d < ndp; ++d) W[(int64_t)d * n + j] = (T)(d < ndens ? w * dens[(int64_t)d * nel + e] : 0.0);
}

template <typename T>
cudaError_t launch_weights(const DevGeom& G, int cls, int64_t n, const double* dens, int64_t nel, int ndens,
                           int ndp, T* W, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_weights<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(G.pt64[cls], G.pt_elem[cls], n, dens, nel, ndens, ndp, W);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- P2M
// One CTA per leaf; thread per coefficient; powers of the scaled offsets
// staged in shared memory for a chunk of 64 points, rows of kPwS = 65
// (threads of one warp read rows of different exponents at the same point:
// an odd stride puts them in different banks).
constexpr int kPwS = 65;
template <typename T>
__global__ void k_p2m(DevGeom G, const int* __restrict__ leaves, int cls, const T* __restrict__ W, int64_t nsp,
                      int ndp, T* __restrict__ mom) {
  extern __shared__ unsigned char smraw[];
  const int P = G.p, np = G.np;
  T* pw = reinterpret_cast<T*>(smraw);               // [3][P+1][64]
  T* ws = pw + 3 * (P + 1) * kPwS;                   // [ndp][64]
  const int leaf = leaves[blockIdx.x];
  const double4_32a cs = G.box_cs[leaf];
  const int2 r = G.box_rng[cls][leaf];
  const double inv_s = 1.0 / cs.w;
  for (int j0 = r.x; j0 < r.y; j0 += 64) {
    const int m = min(64, r.y - j0);
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const double4_32a y = G.pt64[cls][j0 + j];
      const T d[3] = {(T)((y.x - cs.x) * inv_s), (T)((y.y - cs.y) * inv_s), (T)((y.z - cs.z) * inv_s)};
      for (int ax = 0; ax < 3; ++ax) {
        T v = (T)1;
        for (int k = 0; k <= P; ++k) { pw[(ax * (P + 1) + k) * kPwS + j] = v; v *= d[ax]; }
      }
      for (int dd = 0; dd < ndp; ++dd) ws[dd * 64 + j] = W[(int64_t)dd * nsp + j0 + j];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < np; q += blockDim.x) {
      const int mi = G.mi[q];
      const int a = mi & 255, b = (mi >> 8) & 255, c = (mi >> 16) & 255;
      const T* px = pw + (0 * (P + 1) + a) * kPwS;
      const T* py = pw + (1 * (P + 1) + b) * kPwS;
      const T* pz = pw + (2 * (P + 1) + c) * kPwS;
      for (int dd = 0; dd < ndp; ++dd) {
        T acc = 0;
        for (int j = 0; j < m; ++j) acc += ws[dd * 64 + j] * px[j] * py[j] * pz[j];
        mom[((int64_t)leaf * ndp + dd) * G.ms + q] += acc;
      }
    }
  }
}

template <typename T>
cudaError_t launch_p2m(const DevGeom& G, const DevTaskLists& L, const T* W, int64_t nsrc_pts, int ndp,
                       T* mom, cudaStream_t st) {
  if (L.n_p2m == 0) return cudaSuccess;
  size_t sm = sizeof(T) * (3 * (G.p + 1) * kPwS + ndp * 64);
  k_p2m<T><<<L.n_p2m, 128, sm, st>>>(G, L.p2m_leaf, L.src_cls, W, nsrc_pts, ndp, mom);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- M2M
// m_parent[b] = sum_children sum_g M[octant][b][g] m_child[g]; the table is
// stored transposed, Mt[octant][g][b], so threads (b) read it coalesced.
// Shifts between a box and its child in octant o (centre offset sigma s_p/4,
// sigma_i = +-1 by the octant's bits; child side s_p/2), box-scaled:
//   M2M  mhat_p[b] = sum_{g <= b} prod_i C(b_i, g_i) (sigma_i/4)^(b_i - g_i) 2^-|g| mhat_c[g]
//   L2L  lhat_c[a] = 2^-|a| sum_{b >= a} prod_i C(b_i, a_i) (sigma_i/4)^(b_i - a_i) lhat_p[b]
// Both factor into three 1-D binomial shifts, one per axis (the Taylor
// shift of (u + d)^n along each coordinate); every intermediate index stays
// within the total-degree bound (its components lie between those of the
// input and the output), so the passes are exact on the truncated arrays.
// One pass costs about n (p+1)/2 products instead of the dense table's
// n^2 / 2 (n = nterms(p)), and no table is read from memory.

// degree-major position of the multi-index (i, j, k): degree d, then i
// descending, then j descending
__device__ __forceinline__ int midx3(int i, int j, int k) {
  const int d = i + j + k;
  return d * (d + 1) * (d + 2) / 6 + (j + k) * (j + k + 1) / 2 + k;
}

// tab[s][n][k] = C(n, k) (+-1/4)^(n - k), s = 0: -1/4, s = 1: +1/4 (the
// table is built on the host, G.shift64 / G.shift32)
template <typename T>
__device__ __forceinline__ const T* shift_src(const DevGeom& G);
template <>
__device__ __forceinline__ const float* shift_src<float>(const DevGeom& G) { return G.shift32; }
template <>
__device__ __forceinline__ const double* shift_src<double>(const DevGeom& G) { return G.shift64; }
template <typename T>
__device__ void shift_table(const DevGeom& G, T* tab) {
  const T* src = shift_src<T>(G);
  for (int e = threadIdx.x; e < 2 * (G.p + 1) * (G.p + 1); e += blockDim.x) tab[e] = src[e];
}

// one M2M pass along axis ax: out[b] = sum_{g_ax <= b_ax} tab[b_ax][g_ax] in[b with b_ax -> g_ax]
template <typename T>
__device__ __forceinline__ void m2m_pass(const DevGeom& G, int nq, int ax, const T* tb, const T* in, T* out) {
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const int mi = G.mi[q];
    int c[3] = {mi & 255, (mi >> 8) & 255, (mi >> 16) & 255};
    const int n = c[ax];
    const int P1 = G.p + 1;
    T acc = 0;
    for (int k = 0; k <= n; ++k) {
      c[ax] = k;
      acc += tb[n * P1 + k] * in[midx3(c[0], c[1], c[2])];
    }
    out[q] = acc;
  }
}

// one L2L pass along axis ax: out[a] = sum_{b_ax >= a_ax, |b| <= qd} tab[b_ax][a_ax] in[a with a_ax -> b_ax]
template <typename T>
__device__ __forceinline__ void l2l_pass(const DevGeom& G, int nq, int qd, int ax, const T* tb, const T* in, T* out) {
  for (int q = threadIdx.x; q < nq; q += blockDim.x) {
    const int mi = G.mi[q];
    int c[3] = {mi & 255, (mi >> 8) & 255, (mi >> 16) & 255};
    const int a = c[ax], rest = c[0] + c[1] + c[2] - a;
    const int P1 = G.p + 1;
    T acc = 0;
    for (int k = a; k + rest <= qd; ++k) {
      c[ax] = k;
      acc += tb[k * P1 + a] * in[midx3(c[0], c[1], c[2])];
    }
    out[q] = acc;
  }
}

// ---------------------------------------------------------------- M2M
// One CTA per parent box: the children's moments through the three
// passes, summed in shared memory.
template <typename T>
__global__ void k_m2m(DevGeom G, const int* __restrict__ parents, int ndp, T* __restrict__ mom) {
  extern __shared__ unsigned char smraw[];
  const int np = G.np, P1 = G.p + 1;
  T* tab = reinterpret_cast<T*>(smraw);              // [2][P+1][P+1]
  T* va = tab + 2 * P1 * P1;                         // [np]
  T* vb = va + np;                                   // [np]
  T* acc = vb + np;                                  // [np]
  shift_table(G, tab);
  const int P = parents[blockIdx.x];
  const int c0 = G.box_child0[P], nc = G.box_nchild[P];
  for (int d = 0; d < ndp; ++d) {
    for (int q = threadIdx.x; q < np; q += blockDim.x) acc[q] = 0;
    for (int c = 0; c < nc; ++c) {
      const int oc = G.box_octant[c0 + c];
      __syncthreads();
      for (int q = threadIdx.x; q < np; q += blockDim.x) {
        const int mi = G.mi[q];
        const int deg = (mi & 255) + ((mi >> 8) & 255) + ((mi >> 16) & 255);
        va[q] = mom[((int64_t)(c0 + c) * ndp + d) * G.ms + q] / (T)(1 << deg);
      }
      __syncthreads();
      m2m_pass(G, np, 0, tab + ((oc & 1) ? P1 * P1 : 0), va, vb);
      __syncthreads();
      m2m_pass(G, np, 1, tab + ((oc & 2) ? P1 * P1 : 0), vb, va);
      __syncthreads();
      m2m_pass(G, np, 2, tab + ((oc & 4) ? P1 * P1 : 0), va, vb);
      __syncthreads();
      for (int q = threadIdx.x; q < np; q += blockDim.x) acc[q] += vb[q];
    }
    __syncthreads();
    for (int q = threadIdx.x; q < np; q += blockDim.x) mom[((int64_t)P * ndp + d) * G.ms + q] = acc[q];
  }
}

template <typename T>
cudaError_t launch_m2m(const DevGeom& G, const int* parents, int n, int ndp, T* mom, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const size_t sm = sizeof(T) * (2 * (G.p + 1) * (G.p + 1) + 3 * G.np);
  k_m2m<T><<<n, 128, sm, st>>>(G, parents, ndp, mom);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- M2L
// One CTA per target box, thread per row alpha of the local expansion.
// Tt[code][b][a] is the transposed table (coalesced over alpha).  The level
// of the target box has order q <= p (Sec. 4.3): rows |alpha| <= q, and row
// alpha needs only b < nterms(q - |alpha|) (|alpha| + |beta| <= q).
template <typename T, int ND>
__global__ void k_m2l_simt(DevGeom G, DevTaskLists L, const int* __restrict__ sel, const T* __restrict__ Tt, int ndp,
                           const T* __restrict__ mom, T* __restrict__ loc) {
  extern __shared__ unsigned char smraw[];
  T* ms = reinterpret_cast<T*>(smraw);               // [ND][nq]
  const int np = G.np;
  const int ki = sel ? sel[blockIdx.x] : (int)blockIdx.x;   // index into the task's M2L targets
  const int tb = L.m2l_tgt[ki];
  const int q = G.box_q[tb], nq = nterms_q(q);
  const int a = threadIdx.x;
  int K = 0;
  if (a < nq) {
    const int mi = G.mi[a];
    K = nterms_q(q - ((mi & 255) + ((mi >> 8) & 255) + ((mi >> 16) & 255)));
  }
  // products of one translation in T, the sum over the interaction list
  // (~10^3 entries for eta0 = 0.5) in FP64
  double acc[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d) acc[d] = 0.0;
  const int e0 = L.vl_off[ki], e1 = L.vl_off[ki + 1];
  for (int e = e0; e < e1; ++e) {
    const int sb = L.vl_src[e];
    const T* Tc = Tt + (int64_t)L.vl_code[e] * np * np;
    __syncthreads();
    for (int i = threadIdx.x; i < ND * nq; i += blockDim.x) ms[i] = mom[((int64_t)sb * ndp + i / nq) * G.ms + i % nq];
    __syncthreads();
    if (a < nq) {
      T part[ND];
#pragma unroll
      for (int d = 0; d < ND; ++d) part[d] = 0;
      for (int b = 0; b < K; ++b) {
        const T t = Tc[(int64_t)b * np + a];
#pragma unroll
        for (int d = 0; d < ND; ++d) part[d] += t * ms[d * nq + b];
      }
#pragma unroll
      for (int d = 0; d < ND; ++d) acc[d] += (double)part[d];
    }
  }
  if (a < nq) {
    const double inv_s = 1.0 / G.box_cs[tb].w;
#pragma unroll
    for (int d = 0; d < ND; ++d) loc[((int64_t)tb * ndp + d) * G.ms + a] = (T)(acc[d] * inv_s);
  }
}

template <typename T>
cudaError_t launch_m2l_simt(const DevGeom& G, const DevTaskLists& L, const T* Tt, int ndp, const T* mom, T* loc,
                            cudaStream_t st, const int* sel, int nsel) {
  const int n = sel ? nsel : L.n_m2l;
  if (n == 0) return cudaSuccess;
  int threads = ((G.np + 31) / 32) * 32;
  size_t sm = sizeof(T) * ndp * G.np;
  switch (ndp) {
    case 1: k_m2l_simt<T, 1><<<n, threads, sm, st>>>(G, L, sel, Tt, ndp, mom, loc); break;
    case 2: k_m2l_simt<T, 2><<<n, threads, sm, st>>>(G, L, sel, Tt, ndp, mom, loc); break;
    case 4: k_m2l_simt<T, 4><<<n, threads, sm, st>>>(G, L, sel, Tt, ndp, mom, loc); break;
    case 8: k_m2l_simt<T, 8><<<n, threads, sm, st>>>(G, L, sel, Tt, ndp, mom, loc); break;
    case 16: k_m2l_simt<T, 16><<<n, threads, sm, st>>>(G, L, sel, Tt, ndp, mom, loc); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------- L2L
// One CTA per child box.  The parent's expansion has its level's order qp,
// the child's is cut to its own (Sec. 4.3): the passes run over |b| <= qp,
// the child receives |a| <= min(q_child, qp).
template <typename T>
__global__ void k_l2l(DevGeom G, const int* __restrict__ children, int ndp, T* __restrict__ loc) {
  extern __shared__ unsigned char smraw[];
  const int P1 = G.p + 1;
  T* tab = reinterpret_cast<T*>(smraw);              // [2][P+1][P+1]
  T* va = tab + 2 * P1 * P1;                         // [np]
  T* vb = va + G.np;                                 // [np]
  shift_table(G, tab);
  const int C = children[blockIdx.x];
  const int P = G.box_parent[C];
  const int qp = G.box_q[P];
  const int nqc = nterms_q(G.box_q[C]), nqp = nterms_q(qp);
  const int oc = G.box_octant[C];
  for (int d = 0; d < ndp; ++d) {
    __syncthreads();
    for (int q = threadIdx.x; q < nqp; q += blockDim.x) va[q] = loc[((int64_t)P * ndp + d) * G.ms + q];
    __syncthreads();
    l2l_pass(G, nqp, qp, 0, tab + ((oc & 1) ? P1 * P1 : 0), va, vb);
    __syncthreads();
    l2l_pass(G, nqp, qp, 1, tab + ((oc & 2) ? P1 * P1 : 0), vb, va);
    __syncthreads();
    l2l_pass(G, nqp, qp, 2, tab + ((oc & 4) ? P1 * P1 : 0), va, vb);
    __syncthreads();
    // a child of a higher order than its parent gets nothing above |a| = qp
    for (int a = threadIdx.x; a < min(nqc, nqp); a += blockDim.x) {
      const int mi = G.mi[a];
      const int deg = (mi & 255) + ((mi >> 8) & 255) + ((mi >> 16) & 255);
      loc[((int64_t)C * ndp + d) * G.ms + a] += vb[a] / (T)(1 << deg);
    }
  }
}

template <typename T>
cudaError_t launch_l2l(const DevGeom& G, const int* children, int n, int ndp, T* loc, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  const size_t sm = sizeof(T) * (2 * (G.p + 1) * (G.p + 1) + 2 * G.np);
  k_l2l<T><<<n, 128, sm, st>>>(G, children, ndp, loc);
  return cudaGetLastError();
}

// ------------------------------------------------ evaluation + near field
// One CTA (128 threads) per target leaf.  Targets are padded to TP in
// {32, 64, 128}; the 128/TP thread groups split each source tile and are
// reduced at the end.  The sources of N* arrive as merged runs of the sorted
// point array and are streamed through shared memory in tiles that span
// run boundaries.  FP32 coordinates are translated to the target leaf's
// frame with double-float (hi + lo) arithmetic, so differences keep full
// relative accuracy.  Only the leaf's own run (first, VtV) can hold the
// target point itself; tiles overlapping it skip r == 0.  FP32 partial sums
// are folded into FP64 once per tile.
constexpr int kTile = 256;
constexpr int kRunBatch = 256;

__device__ __forceinline__ void split_df(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}

// largest r in [0, n) with pre[r] <= v  (pre[0] = 0 <= v < pre[n])
__device__ __forceinline__ int find_run(const int* pre, int n, int v) {
  int lo = 0, hi = n;
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (pre[mid] <= v) lo = mid; else hi = mid;
  }
  return lo;
}

// prefix sums of the run lengths of one batch (warp 0), starts into rst
__device__ __forceinline__ void scan_runs(const int2* __restrict__ runs, int nr, int* pre, int* rst) {
  if (threadIdx.x < 32) {
    const int lane = threadIdx.x;
    int carry = 0;
    if (lane == 0) pre[0] = 0;
    for (int c = 0; c < nr; c += 32) {
      const int r = c + lane;
      int len = 0;
      if (r < nr) { const int2 rr = runs[r]; len = rr.y - rr.x; rst[r] = rr.x; }
      int x = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) { const int y = __shfl_up_sync(0xffffffffu, x, o); if (lane >= o) x += y; }
      if (r < nr) pre[r + 1] = carry + x;
      carry += __shfl_sync(0xffffffffu, x, 31);
    }
  }
}

template <typename T, int ND>
__device__ __forceinline__ void l2p_and_store(const DevGeom& G, int leaf, int ndp, const T* __restrict__ loc,
                                              double xs, double ys, double zs, const double* near, int64_t pos,
                                              int64_t ntp, double* __restrict__ phi) {
  T far[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d) far[d] = (T)0;
  // L2P: phi_far(x) = sum_a l^a xhat^a, xhat = (x - c)/s (locals of boxes
  // without an interaction list are zero)
  if (loc != nullptr) {
    T px[16], py[16], pz[16];
    px[0] = py[0] = pz[0] = (T)1;
    for (int k = 1; k <= G.p; ++k) { px[k] = px[k - 1] * (T)xs; py[k] = py[k - 1] * (T)ys; pz[k] = pz[k - 1] * (T)zs; }
    const T* lb = loc + (int64_t)leaf * ndp * G.ms;
    const int nq = nterms_q(G.box_q[leaf]);          // the leaf level's order
    for (int q = 0; q < nq; ++q) {
      const int mi = G.mi[q];
      const T mono = px[mi & 255] * py[(mi >> 8) & 255] * pz[(mi >> 16) & 255];
#pragma unroll
      for (int d = 0; d < ND; ++d) far[d] += lb[d * G.ms + q] * mono;
    }
  }
#pragma unroll
  for (int d = 0; d < ND; ++d) phi[(int64_t)d * ntp + pos] = near[d] * kInv4Pi + (double)far[d];
}

// The hardware reciprocal square root (PTX rsqrt.approx.ftz.f32: maximum
// relative error about 2^-22.9, subnormal inputs and results flushed to
// zero).  Squared distances of distinct quadrature points lie far above the
// subnormal range; r^2 = 0 is selected out where it can occur, and the
// padding point's r^2 = inf gives 0.  Without the flush the compiler wraps
// the same instruction in a subnormal rescaling that costs several extra
// instructions per pair.
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__device__ __forceinline__ void two_sum_f(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  lo += (hi - (s - bb)) + (x - bb);
  hi = s;
}

// Two targets per thread (ND <= 2) or one (ND > 2); thread groups split the
// source tile; source tiles are double-buffered (one barrier per tile); the
// per-tile FP32 sums are folded with a compensated (hi + lo) FP32 sum.
template <int ND>
__global__ void __launch_bounds__(128) k_p2p_l2p_f32(DevGeom G, DevTaskLists L, const float* __restrict__ W,
                                                     int64_t nsp, int64_t ntp, int ndp,
                                                     const float* __restrict__ loc, double* __restrict__ phi) {
  constexpr int TPT = ND <= 2 ? 2 : 1;
  constexpr int PPT = kTile / 128;                 // source points loaded per thread per tile
  __shared__ float4 tile[2][kTile];
  __shared__ float tw[2][ND > 1 ? ND - 1 : 1][kTile];
  __shared__ int pre[kRunBatch + 1], rst[kRunBatch];
  __shared__ float2 red[ND][128 * TPT];
  const int b = blockIdx.x;
  const int leaf = L.p2p_leaf[b];
  const int sc = L.src_cls, tc = L.tgt_cls;
  const double4_32a cs = G.box_cs[leaf];
  float chx, clx, chy, cly, chz, clz;
  split_df(cs.x, chx, clx); split_df(cs.y, chy, cly); split_df(cs.z, chz, clz);
  const int2 tr = G.box_rng[tc][leaf];
  const int nt = tr.y - tr.x;
  // TS target slots (TPT targets each) per source group, NG = 128 / TS
  // groups; threads beyond NG * TS only help loading the tiles
  const int TS = (nt + TPT - 1) / TPT;
  const int NG = 128 / TS;
  const int ts = threadIdx.x % TS, gi_raw = threadIdx.x / TS;
  const int gi = gi_raw < NG ? gi_raw : NG;       // NG: idle for the compute
  float xt[TPT], yt[TPT], zt[TPT];
  bool act[TPT];
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int t = ts + u * TS;
    act[u] = t < nt;
    xt[u] = yt[u] = zt[u] = 1e30f;      // padding targets: far away, discarded
    if (act[u]) {
      const float4 h = G.pthi[tc][tr.x + t], l = G.ptlo[tc][tr.x + t];
      xt[u] = (h.x - chx) + (l.x - clx);
      yt[u] = (h.y - chy) + (l.y - cly);
      zt[u] = (h.z - chz) + (l.z - clz);
    }
  }
  float shi[TPT][ND], slo[TPT][ND];
#pragma unroll
  for (int u = 0; u < TPT; ++u)
#pragma unroll
    for (int d = 0; d < ND; ++d) shi[u][d] = slo[u][d] = 0.f;
  const int r0 = L.run_off[b], r1 = L.run_off[b + 1];
  const int self_len = L.self_len[b];
  float4 reg[PPT];
  float regw[PPT][ND > 1 ? ND - 1 : 1];
  for (int rb = r0; rb < r1; rb += kRunBatch) {
    const int nr = min(kRunBatch, r1 - rb);
    __syncthreads();
    scan_runs(L.runs + rb, nr, pre, rst);
    __syncthreads();
    const int total = pre[nr];
    const int ntiles = (total + kTile - 1) / kTile;
    auto load_tile = [&](int t) {
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        const int v = t * kTile + threadIdx.x + q * 128;
        if (v < total) {
          const int r = find_run(pre, nr, v);
          const int src = rst[r] + (v - pre[r]);
          const float4 h = G.pthi[sc][src], l = G.ptlo[sc][src];
          reg[q] = make_float4((h.x - chx) + (l.x - clx), (h.y - chy) + (l.y - cly), (h.z - chz) + (l.z - clz), W[src]);
#pragma unroll
          for (int d = 1; d < ND; ++d) regw[q][d - 1] = W[(int64_t)d * nsp + src];
        }
      }
    };
    auto store_tile = [&](int buf) {
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        const int j = threadIdx.x + q * 128;
        tile[buf][j] = reg[q];
#pragma unroll
        for (int d = 1; d < ND; ++d) tw[buf][d - 1][j] = regw[q][d - 1];
      }
    };
    if (ntiles > 0) {
      load_tile(0);
      store_tile(0);
    }
    __syncthreads();
    for (int t = 0; t < ntiles; ++t) {
      const int cur = t & 1;
      if (t + 1 < ntiles) load_tile(t + 1);      // global loads in flight during the compute
      const int m = min(kTile, total - t * kTile);
      float acc[TPT][ND];
#pragma unroll
      for (int u = 0; u < TPT; ++u)
#pragma unroll
        for (int d = 0; d < ND; ++d) acc[u][d] = 0.f;
      const int jstart = gi_raw < NG ? gi : m;        // idle threads skip the loops
      if (rb == r0 && t * kTile < self_len) {
        for (int j = jstart; j < m; j += NG) {
          const float4 s = tile[cur][j];
#pragma unroll
          for (int u = 0; u < TPT; ++u) {
            const float dx = xt[u] - s.x, dy = yt[u] - s.y, dz = zt[u] - s.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float ri = r2 > 0.f ? rsqrt_ftz(r2) : 0.f;
            acc[u][0] = fmaf(s.w, ri, acc[u][0]);
#pragma unroll
            for (int d = 1; d < ND; ++d) acc[u][d] = fmaf(tw[cur][d - 1][j], ri, acc[u][d]);
          }
        }
      } else {
#pragma unroll 4
        for (int j = jstart; j < m; j += NG) {
          const float4 s = tile[cur][j];
#pragma unroll
          for (int u = 0; u < TPT; ++u) {
            const float dx = xt[u] - s.x, dy = yt[u] - s.y, dz = zt[u] - s.z;
            const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
            const float ri = rsqrt_ftz(r2);
            acc[u][0] = fmaf(s.w, ri, acc[u][0]);
#pragma unroll
            for (int d = 1; d < ND; ++d) acc[u][d] = fmaf(tw[cur][d - 1][j], ri, acc[u][d]);
          }
        }
      }
#pragma unroll
      for (int u = 0; u < TPT; ++u)
#pragma unroll
        for (int d = 0; d < ND; ++d) two_sum_f(shi[u][d], slo[u][d], acc[u][d]);
      if (t + 1 < ntiles) store_tile(cur ^ 1);
      __syncthreads();
    }
  }
#pragma unroll
  for (int u = 0; u < TPT; ++u)
#pragma unroll
    for (int d = 0; d < ND; ++d) red[d][u * 128 + threadIdx.x] = make_float2(shi[u][d], slo[u][d]);
  __syncthreads();
  if (gi_raw == 0) {
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      if (!act[u]) continue;
      double near[ND];
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        float hi = 0.f, lo = 0.f;
        for (int g = 0; g < NG; ++g) {
          const float2 v = red[d][u * 128 + g * TS + ts];
          two_sum_f(hi, lo, v.x);
          lo += v.y;
        }
        near[d] = (double)hi + (double)lo;
      }
      const double inv_s = 1.0 / cs.w;
      l2p_and_store<float, ND>(G, leaf, ndp, loc, xt[u] * inv_s, yt[u] * inv_s, zt[u] * inv_s, near, tr.x + ts + u * TS,
                               ntp, phi);
    }
  }
}



// The packed pair loop over pairs [k0, k1) of a staged tile: per pair and
// target, three packed subtractions (the sources are stored negated), the
// packed r^2 (one multiply, two FMAs), two rsqrt and one packed FMA per
// density.  CHECK: the tile holds the target points themselves (r^2 = 0).
template <int ND, int TPT, bool CHECK>
__device__ __forceinline__ void p2p_pairs_x2(const float4* __restrict__ xy, const float4* __restrict__ zw,
                                             const float2* __restrict__ w2, int k0, int k1, const float2 (&X)[TPT],
                                             const float2 (&Y)[TPT], const float2 (&Z)[TPT], float2 (&acc)[TPT][ND]) {
#pragma unroll 4
  for (int k = k0; k < k1; ++k) {
    const float4 a = xy[k], c = zw[k];
    const float2 nx = make_float2(a.x, a.y), ny = make_float2(a.z, a.w), nz = make_float2(c.x, c.y);
    const float2 w0 = make_float2(c.z, c.w);
    float2 wb = w0;
    if constexpr (ND > 1) wb = w2[k];
#pragma unroll
    for (int u = 0; u < TPT; ++u) {
      const float2 dx = __fadd2_rn(X[u], nx), dy = __fadd2_rn(Y[u], ny), dz = __fadd2_rn(Z[u], nz);
      const float2 r2 = __ffma2_rn(dx, dx, __ffma2_rn(dy, dy, __fmul2_rn(dz, dz)));
      float2 ri;
      if constexpr (CHECK) ri = make_float2(r2.x > 0.f ? rsqrt_ftz(r2.x) : 0.f, r2.y > 0.f ? rsqrt_ftz(r2.y) : 0.f);
      else ri = make_float2(rsqrt_ftz(r2.x), rsqrt_ftz(r2.y));
      acc[u][0] = __ffma2_rn(w0, ri, acc[u][0]);
      if constexpr (ND > 1) acc[u][ND - 1] = __ffma2_rn(wb, ri, acc[u][ND - 1]);
    }
  }
}

// Packed form for ND <= 2: TPT targets per thread (4 for one density, 2
// for two) and source points taken two at a time, every arithmetic
// instruction on a float2 (the two sources of a pair: __fadd2_rn /
// __fmul2_rn / __ffma2_rn), so a target keeps two independent partial sums
// and the instructions issued per point pair nearly halve.  A tile of
// source points is staged pair-interleaved in shared memory, negated and
// relative to the target leaf's centre: xy[k] = (x0, x1, y0, y1), zw[k] =
// (z0, z1, w0, w1) for the pair k = (2k, 2k + 1), so one pair costs two
// 16-byte shared loads.  Each of the NG thread groups takes a contiguous
// range of pairs (odd length, so two groups' loads in one quarter-warp fall
// in different banks) walked with unit stride.  An odd tile is padded with a
// weightless point at -1e30, whose distance overflows to inf (rsqrt 0).  Only
// the pairs that hold the leaf's own points (the first run of a VtV list)
// select r^2 = 0 out.  After the source loop all threads reduce the group
// sums and evaluate L2P, one target each.
constexpr int kTileX2 = 512;     // source points per tile of the packed kernel

template <int ND, int TPT>
__global__ void __launch_bounds__(128) k_p2p_l2p_f32x2(DevGeom G, DevTaskLists L, const float* __restrict__ W,
                                                       int64_t nsp, int64_t ntp, int ndp,
                                                       const float* __restrict__ loc, double* __restrict__ phi) {
  static_assert(ND >= 1 && ND <= 2, "packed P2P serves one or two densities");
  constexpr int kTile = kTileX2;
  constexpr int kPairs = kTile / 2;
  constexpr int PPT = kPairs / 128;                // pairs loaded per thread per tile
  __shared__ float4 sxy[2][kPairs];
  __shared__ float4 szw[2][kPairs];
  __shared__ float2 sw2[ND > 1 ? 2 : 1][ND > 1 ? kPairs : 1];
  __shared__ int pre[kRunBatch + 1], rst[kRunBatch];
  __shared__ float2 red[ND][128 * TPT];
  const int b = blockIdx.x;
  const int leaf = L.sp_leaf[b];
  const int sc = L.src_cls, tc = L.tgt_cls;
  const double4_32a cs = G.box_cs[leaf];
  float chx, clx, chy, cly, chz, clz;
  split_df(cs.x, chx, clx); split_df(cs.y, chy, cly); split_df(cs.z, chz, clz);
  const int2 tr = G.box_rng[tc][leaf];
  const int nt = tr.y - tr.x;
  const int TS = (nt + TPT - 1) / TPT;
  const int NG = 128 / TS;
  const int ts = threadIdx.x % TS, gi_raw = threadIdx.x / TS;
  float2 X[TPT], Y[TPT], Z[TPT];
#pragma unroll
  for (int u = 0; u < TPT; ++u) {
    const int t = ts + u * TS;
    float xt = 1e30f, yt = 1e30f, zt = 1e30f;      // padding targets: far away, discarded
    if (t < nt) {
      const float4 h = G.pthi[tc][tr.x + t], l = G.ptlo[tc][tr.x + t];
      xt = (h.x - chx) + (l.x - clx);
      yt = (h.y - chy) + (l.y - cly);
      zt = (h.z - chz) + (l.z - clz);
    }
    X[u] = make_float2(xt, xt);
    Y[u] = make_float2(yt, yt);
    Z[u] = make_float2(zt, zt);
  }
  float shi[TPT][ND], slo[TPT][ND];
#pragma unroll
  for (int u = 0; u < TPT; ++u)
#pragma unroll
    for (int d = 0; d < ND; ++d) shi[u][d] = slo[u][d] = 0.f;
  const int r0 = L.sp_run_off[b], r1 = L.sp_run_off[b + 1];
  const int self_len = L.sp_self[b];
  float4 rxy[PPT], rzw[PPT];
  float2 rw2[PPT];
  for (int rb = r0; rb < r1; rb += kRunBatch) {
    const int nr = min(kRunBatch, r1 - rb);
    __syncthreads();
    scan_runs(L.sp_runs + rb, nr, pre, rst);
    __syncthreads();
    const int total = pre[nr];
    const int ntiles = (total + kTile - 1) / kTile;
    // source point v of this batch (r: its run), negated, relative to the centre
    auto fetch = [&](int v, int r, float& x, float& y, float& z, float& w, float& w2) {
      const int src = rst[r] + (v - pre[r]);
      const float4 h = G.pthi[sc][src], l = G.ptlo[sc][src];
      x = -((h.x - chx) + (l.x - clx));
      y = -((h.y - chy) + (l.y - cly));
      z = -((h.z - chz) + (l.z - clz));
      w = W[src];
      if constexpr (ND > 1) w2 = W[nsp + src];
    };
    auto load_tile = [&](int t) {
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        const int v0 = t * kTile + 2 * (threadIdx.x + q * 128);
        float x0 = 1e30f, y0 = 1e30f, z0 = 1e30f, w0 = 0.f, u0 = 0.f;   // negated padding points
        float x1 = 1e30f, y1 = 1e30f, z1 = 1e30f, w1 = 0.f, u1 = 0.f;
        if (v0 < total) {
          int r = find_run(pre, nr, v0);
          fetch(v0, r, x0, y0, z0, w0, u0);
          if (v0 + 1 < total) {
            while (r + 1 < nr && pre[r + 1] <= v0 + 1) ++r;
            fetch(v0 + 1, r, x1, y1, z1, w1, u1);
          }
        }
        rxy[q] = make_float4(x0, x1, y0, y1);
        rzw[q] = make_float4(z0, z1, w0, w1);
        rw2[q] = make_float2(u0, u1);
      }
    };
    auto store_tile = [&](int buf) {
#pragma unroll
      for (int q = 0; q < PPT; ++q) {
        const int k = threadIdx.x + q * 128;
        sxy[buf][k] = rxy[q];
        szw[buf][k] = rzw[q];
        if constexpr (ND > 1) sw2[buf][k] = rw2[q];
      }
    };
    if (ntiles > 0) {
      load_tile(0);
      store_tile(0);
    }
    __syncthreads();
    for (int t = 0; t < ntiles; ++t) {
      const int cur = t & 1;
      if (t + 1 < ntiles) load_tile(t + 1);
      const int m = min(kTile, total - t * kTile);
      const int mp = (m + 1) >> 1;
      // group gi_raw's contiguous pair range, odd length
      const int len = ((mp + NG - 1) / NG) | 1;
      const int k0 = gi_raw < NG ? min(gi_raw * len, mp) : mp;
      const int k1 = min(k0 + len, mp);
      // pairs that hold one of the leaf's own points (first run of a VtV list)
      const int ks = rb == r0 ? max(0, min(mp, (self_len - t * kTile + 1) >> 1)) : 0;
      float2 acc[TPT][ND];
#pragma unroll
      for (int u = 0; u < TPT; ++u)
#pragma unroll
        for (int d = 0; d < ND; ++d) acc[u][d] = make_float2(0.f, 0.f);
      const float2* w2 = nullptr;
      if constexpr (ND > 1) w2 = sw2[cur];
      if (k0 < ks) p2p_pairs_x2<ND, TPT, true>(sxy[cur], szw[cur], w2, k0, min(k1, ks), X, Y, Z, acc);
      p2p_pairs_x2<ND, TPT, false>(sxy[cur], szw[cur], w2, max(k0, ks), k1, X, Y, Z, acc);
#pragma unroll
      for (int u = 0; u < TPT; ++u)
#pragma unroll
        for (int d = 0; d < ND; ++d) {
          two_sum_f(shi[u][d], slo[u][d], acc[u][d].x);
          two_sum_f(shi[u][d], slo[u][d], acc[u][d].y);
        }
      if (t + 1 < ntiles) store_tile(cur ^ 1);
      __syncthreads();
    }
  }
#pragma unroll
  for (int u = 0; u < TPT; ++u)
#pragma unroll
    for (int d = 0; d < ND; ++d) red[d][u * 128 + threadIdx.x] = make_float2(shi[u][d], slo[u][d]);
  __syncthreads();
  // every thread: one target, the group sums in group order; a chunk of a
  // split leaf stores them in its scratch row, and the leaf's last chunk
  // to finish adds the rows in chunk order; then L2P
  const int2 grp = L.sp_grp[b];
  __shared__ int last_chunk;
  if (grp.x >= 0) {
    const int2 gi = L.grp_info[grp.x];
    float2* row = L.sp_scratch + (int64_t)(gi.x + grp.y) * ND * 128;
    for (int tt = threadIdx.x; tt < nt; tt += 128) {
      const int u = tt / TS, tsl = tt - u * TS;
#pragma unroll
      for (int d = 0; d < ND; ++d) {
        float hi = 0.f, lo = 0.f;
        for (int g = 0; g < NG; ++g) {
          const float2 v = red[d][u * 128 + g * TS + tsl];
          two_sum_f(hi, lo, v.x);
          lo += v.y;
        }
        __stcg(row + d * 128 + tt, make_float2(hi, lo));
      }
    }
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
      const unsigned ticket = atomicAdd(L.grp_cnt + grp.x, 1u);
      last_chunk = ticket + 1 == (unsigned)gi.y;
      if (last_chunk) L.grp_cnt[grp.x] = 0u;      // ready for the next launch
    }
    __syncthreads();
    if (!last_chunk) return;
    __threadfence();
  }
  const double inv_s = 1.0 / cs.w;
  for (int tt = threadIdx.x; tt < nt; tt += 128) {
    const int u = tt / TS, tsl = tt - u * TS;
    double near[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      float hi = 0.f, lo = 0.f;
      if (grp.x < 0) {
        for (int g = 0; g < NG; ++g) {
          const float2 v = red[d][u * 128 + g * TS + tsl];
          two_sum_f(hi, lo, v.x);
          lo += v.y;
        }
      } else {
        const int2 gi = L.grp_info[grp.x];
        for (int c = 0; c < gi.y; ++c) {
          const float2 v = __ldcg(L.sp_scratch + (int64_t)(gi.x + c) * ND * 128 + d * 128 + tt);
          two_sum_f(hi, lo, v.x);
          lo += v.y;
        }
      }
      near[d] = (double)hi + (double)lo;
    }
    const float4 h = G.pthi[tc][tr.x + tt], l = G.ptlo[tc][tr.x + tt];
    const float xt = (h.x - chx) + (l.x - clx), yt = (h.y - chy) + (l.y - cly), zt = (h.z - chz) + (l.z - clz);
    l2p_and_store<float, ND>(G, leaf, ndp, loc, xt * inv_s, yt * inv_s, zt * inv_s, near, tr.x + tt, ntp, phi);
  }
}

template <int ND>
__global__ void __launch_bounds__(128) k_p2p_l2p_f64(DevGeom G, DevTaskLists L, const double* __restrict__ W,
                                                     int64_t nsp, int64_t ntp, int ndp,
                                                     const double* __restrict__ loc, double* __restrict__ phi) {
  constexpr int TL = kTile / 2;
  __shared__ double4_32a tile[TL];
  __shared__ double tw[ND > 1 ? ND - 1 : 1][TL];
  __shared__ int pre[kRunBatch + 1], rst[kRunBatch];
  __shared__ double red[ND][128];
  const int b = blockIdx.x;
  const int leaf = L.p2p_leaf[b];
  const int sc = L.src_cls, tc = L.tgt_cls;
  const double4_32a cs = G.box_cs[leaf];
  const int2 tr = G.box_rng[tc][leaf];
  const int nt = tr.y - tr.x;
  const int TP = nt <= 8 ? 8 : (nt <= 16 ? 16 : (nt <= 32 ? 32 : (nt <= 64 ? 64 : 128)));
  const int NG = 128 / TP;
  const int ti = threadIdx.x % TP, gi = threadIdx.x / TP;
  const bool active = ti < nt;
  double xt = 0, yt = 0, zt = 0;
  if (active) {
    const double4_32a x = G.pt64[tc][tr.x + ti];
    xt = x.x; yt = x.y; zt = x.z;
  }
  double acc[ND];
#pragma unroll
  for (int d = 0; d < ND; ++d) acc[d] = 0.0;
  const int r0 = L.run_off[b], r1 = L.run_off[b + 1];
  for (int rb = r0; rb < r1; rb += kRunBatch) {
    const int nr = min(kRunBatch, r1 - rb);
    __syncthreads();
    scan_runs(L.runs + rb, nr, pre, rst);
    __syncthreads();
    const int total = pre[nr];
    for (int j0 = 0; j0 < total; j0 += TL) {
      const int m = min(TL, total - j0);
      __syncthreads();
      for (int j = threadIdx.x; j < m; j += 128) {
        const int v = j0 + j;
        const int r = find_run(pre, nr, v);
        const int src = rst[r] + (v - pre[r]);
        const double4_32a y = G.pt64[sc][src];
        tile[j] = make_double4_32a(y.x, y.y, y.z, W[src]);
#pragma unroll
        for (int d = 1; d < ND; ++d) tw[d - 1][j] = W[(int64_t)d * nsp + src];
      }
      __syncthreads();
      if (active) {
        for (int j = gi; j < m; j += NG) {
          const double4_32a s = tile[j];
          const double dx = xt - s.x, dy = yt - s.y, dz = zt - s.z;
          const double r2 = dx * dx + dy * dy + dz * dz;
          const double ri = r2 > 0.0 ? 1.0 / sqrt(r2) : 0.0;
          acc[0] += s.w * ri;
#pragma unroll
          for (int d = 1; d < ND; ++d) acc[d] += tw[d - 1][j] * ri;
        }
      }
    }
  }
#pragma unroll
  for (int d = 0; d < ND; ++d) red[d][threadIdx.x] = acc[d];
  __syncthreads();
  if (gi == 0 && active) {
    double near[ND];
#pragma unroll
    for (int d = 0; d < ND; ++d) {
      double s = 0.0;
      for (int g = 0; g < NG; ++g) s += red[d][g * TP + ti];
      near[d] = s;
    }
    const double inv_s = 1.0 / cs.w;
    l2p_and_store<double, ND>(G, leaf, ndp, loc, (xt - cs.x) * inv_s, (yt - cs.y) * inv_s, (zt - cs.z) * inv_s, near,
                              tr.x + ti, ntp, phi);
  }
}

#define P2P_DISPATCH(KER, ...)                                               \
  switch (ndp) {                                                             \
    case 1: KER<1><<<L.n_p2p, 128, 0, st>>>(__VA_ARGS__); break;             \
    case 2: KER<2><<<L.n_p2p, 128, 0, st>>>(__VA_ARGS__); break;             \
    case 4: KER<4><<<L.n_p2p, 128, 0, st>>>(__VA_ARGS__); break;             \
    case 8: KER<8><<<L.n_p2p, 128, 0, st>>>(__VA_ARGS__); break;             \
    case 16: KER<16><<<L.n_p2p, 128, 0, st>>>(__VA_ARGS__); break;           \
    default: return cudaErrorInvalidValue;                                   \
  }

cudaError_t launch_p2p_l2p_f32(const DevGeom& G, const DevTaskLists& L, const float* W, int64_t nsrc_pts,
                               int64_t ntgt_pts, int ndp, const float* loc, double* phi, cudaStream_t st) {
  if (L.n_p2p == 0) return cudaSuccess;
  switch (ndp) {
    case 1: k_p2p_l2p_f32x2<1, 4><<<L.sp_n, 128, 0, st>>>(G, L, W, nsrc_pts, ntgt_pts, ndp, loc, phi); break;
    case 2: k_p2p_l2p_f32x2<2, 2><<<L.sp_n, 128, 0, st>>>(G, L, W, nsrc_pts, ntgt_pts, ndp, loc, phi); break;
    case 4: k_p2p_l2p_f32<4><<<L.n_p2p, 128, 0, st>>>(G, L, W, nsrc_pts, ntgt_pts, ndp, loc, phi); break;
    case 8: k_p2p_l2p_f32<8><<<L.n_p2p, 128, 0, st>>>(G, L, W, nsrc_pts, ntgt_pts, ndp, loc, phi); break;
    case 16: k_p2p_l2p_f32<16><<<L.n_p2p, 128, 0, st>>>(G, L, W, nsrc_pts, ntgt_pts, ndp, loc, phi); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_p2p_l2p_f64(const DevGeom& G, const DevTaskLists& L, const double* W, int64_t nsrc_pts,
                               int64_t ntgt_pts, int ndp, const double* loc, double* phi, cudaStream_t st) {
  if (L.n_p2p == 0) return cudaSuccess;
  P2P_DISPATCH(k_p2p_l2p_f64, G, L, W, nsrc_pts, ntgt_pts, ndp, loc, phi);
  return cudaGetLastError();
}


// ------------------------------------------- Galerkin sums + corrections
// One warp per target element: u[d][e] = sum_q w_q phi[d][pos_q]
//                                      + sum_k C[k] dens[d][col[k]].
__global__ void k_elem_sum(DevGeom G, DevTaskLists L, const double* __restrict__ phi, int64_t ntp,
                           const double* __restrict__ dens, int ndens, const double* __restrict__ dens_dl,
                           double* __restrict__ out) {
  const int64_t e = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= L.ntgt_el) return;
  const int tc = L.tgt_cls;
  for (int d = 0; d < ndens; ++d) {
    double s = 0.0;
    if (lane < L.nq_tgt) {
      const int pos = L.elem_pts[e * 4 + lane];
      s = G.pt64[tc][pos].w * phi[(int64_t)d * ntp + pos];
    }
    const int64_t k0 = L.cor_off[e], k1 = L.cor_off[e + 1];
#pragma unroll 4
    for (int64_t k = k0 + lane; k < k1; k += 32) s += L.cor_val[k] * dens[(int64_t)d * L.nsrc_el + L.cor_col[k]];
    // BtV double layer: - (N - Q) of dG/dn_y times g
    if (dens_dl)
      for (int64_t k = k0 + lane; k < k1; k += 32) s -= L.cor_val_dl[k] * dens_dl[(int64_t)d * L.nsrc_el + L.cor_col[k]];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[(int64_t)d * L.ntgt_el + e] = s;
  }
}

cudaError_t launch_elem_sum(const DevGeom& G, const DevTaskLists& L, const double* phi, int64_t ntgt_pts,
                            const double* dens_src, int ndens, double* out, cudaStream_t st, const double* dens_dl) {
  if (L.ntgt_el == 0) return cudaSuccess;
  if (dens_dl && !L.cor_val_dl) return cudaErrorInvalidValue;
  const int64_t threads = L.ntgt_el * 32;
  k_elem_sum<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(G, L, phi, ntgt_pts, dens_src, ndens, dens_dl, out);
  return cudaGetLastError();
}

// ------------------------------------------------- double layer (BtV)
// Moments of the double-layer density g (Algorithm 3: m^b includes
// - <gamma_1 (y - c)^b, g>; this pass adds that term).  Box-scaled, with
// u = (y - c)/s: n . grad_y (u^b) = (1/s) sum_i n_i b_i u^(b - e_i), so
// mhat^b -= (Wg_j / s) sum_i n_i b_i u_j^(b - e_i), Wg_j = w_j g(elem j),
// n the unit normal of point j's triangle.
template <typename T>
__global__ void k_p2m_dl(DevGeom G, const int* __restrict__ leaves, const T* __restrict__ W, int64_t nsp, int ndp,
                         T* __restrict__ mom) {
  extern __shared__ unsigned char smraw[];
  const int P = G.p, np = G.np;
  T* pw = reinterpret_cast<T*>(smraw);               // [3][P+1][64]
  T* wn = pw + 3 * (P + 1) * kPwS;                   // [ndp][3][64]: Wg n_i / s
  const int leaf = leaves[blockIdx.x];
  const double4_32a cs = G.box_cs[leaf];
  const int2 r = G.box_rng[1][leaf];
  const double inv_s = 1.0 / cs.w;
  for (int j0 = r.x; j0 < r.y; j0 += 64) {
    const int m = min(64, r.y - j0);
    __syncthreads();
    for (int j = threadIdx.x; j < m; j += blockDim.x) {
      const double4_32a y = G.pt64[1][j0 + j];
      const T d[3] = {(T)((y.x - cs.x) * inv_s), (T)((y.y - cs.y) * inv_s), (T)((y.z - cs.z) * inv_s)};
      for (int ax = 0; ax < 3; ++ax) {
        T v = (T)1;
        for (int k = 0; k <= P; ++k) { pw[(ax * (P + 1) + k) * kPwS + j] = v; v *= d[ax]; }
      }
      const double4_32a nr = G.tri_nrm[G.pt_elem[1][j0 + j]];
      for (int dd = 0; dd < ndp; ++dd) {
        const double wg = (double)W[(int64_t)dd * nsp + j0 + j] * inv_s;
        wn[(dd * 3 + 0) * 64 + j] = (T)(wg * nr.x);
        wn[(dd * 3 + 1) * 64 + j] = (T)(wg * nr.y);
        wn[(dd * 3 + 2) * 64 + j] = (T)(wg * nr.z);
      }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < np; q += blockDim.x) {
      const int mi = G.mi[q];
      const int a = mi & 255, b = (mi >> 8) & 255, c = (mi >> 16) & 255;
      const T* px = pw + (0 * (P + 1)) * kPwS;
      const T* py = pw + (1 * (P + 1)) * kPwS;
      const T* pz = pw + (2 * (P + 1)) * kPwS;
      for (int dd = 0; dd < ndp; ++dd) {
        const T* wx = wn + (dd * 3 + 0) * 64;
        const T* wy = wn + (dd * 3 + 1) * 64;
        const T* wz = wn + (dd * 3 + 2) * 64;
        T acc = 0;
        for (int j = 0; j < m; ++j) {
          T g = 0;
          if (a) g += (T)a * wx[j] * px[(a - 1) * kPwS + j] * py[b * kPwS + j] * pz[c * kPwS + j];
          if (b) g += (T)b * wy[j] * px[a * kPwS + j] * py[(b - 1) * kPwS + j] * pz[c * kPwS + j];
          if (c) g += (T)c * wz[j] * px[a * kPwS + j] * py[b * kPwS + j] * pz[(c - 1) * kPwS + j];
          acc += g;
        }
        mom[((int64_t)leaf * ndp + dd) * G.ms + q] -= acc;
      }
    }
  }
}

template <typename T>
cudaError_t launch_p2m_dl(const DevGeom& G, const DevTaskLists& L, const T* W, int64_t nsrc_pts, int ndp, T* mom,
                          cudaStream_t st) {
  if (L.n_p2m == 0) return cudaSuccess;
  const size_t sm = sizeof(T) * (3 * (G.p + 1) * kPwS + 3 * ndp * 64);
  k_p2m_dl<T><<<L.n_p2m, 128, sm, st>>>(G, L.p2m_leaf, W, nsrc_pts, ndp, mom);
  return cudaGetLastError();
}

// Near field of the double layer over the extended neighbour list:
// phi(x) -= (1/4pi) sum_j Wg_j n_j.(x - y_j) / |x - y_j|^3 for the leaf's
// target points, one CTA per target leaf, one target point per thread
// (chunks of 128 target points); sources stream through shared memory.
// FP32: leaf-frame double-float coordinates as in the single-layer pass,
// tile sums folded into FP64; FP64: plain.
template <typename T>
__global__ void __launch_bounds__(128) k_p2p_dl(DevGeom G, DevTaskLists L, const T* __restrict__ W, int64_t nsp,
                                                int64_t ntp, int ndp, double* __restrict__ phi) {
  constexpr int kT = 128;
  __shared__ T sx[kT], sy[kT], sz[kT], snx[kT], sny[kT], snz[kT];
  __shared__ int pre[kRunBatch + 1], rst[kRunBatch];
  const int b = blockIdx.x;
  const int leaf = L.p2p_leaf[b];
  const int tc = L.tgt_cls;
  const double4_32a cs = G.box_cs[leaf];
  float chx, clx, chy, cly, chz, clz;
  split_df(cs.x, chx, clx); split_df(cs.y, chy, cly); split_df(cs.z, chz, clz);
  const int2 tr = G.box_rng[tc][leaf];
  const int nt = tr.y - tr.x;
  const int r0 = L.run_off[b], r1 = L.run_off[b + 1];
  for (int t0 = 0; t0 < nt; t0 += kT) {
  const int t = t0 + threadIdx.x;
  const bool act = t < nt;
  T xt = 0, yt = 0, zt = 0;
  if (act) {
    if (sizeof(T) == 4) {
      const float4 h = G.pthi[tc][tr.x + t], l = G.ptlo[tc][tr.x + t];
      xt = (T)((h.x - chx) + (l.x - clx));
      yt = (T)((h.y - chy) + (l.y - cly));
      zt = (T)((h.z - chz) + (l.z - clz));
    } else {
      const double4_32a x = G.pt64[tc][tr.x + t];
      xt = (T)(x.x - cs.x); yt = (T)(x.y - cs.y); zt = (T)(x.z - cs.z);
    }
  }
  for (int d = 0; d < ndp; ++d) {
    double total = 0.0;
    for (int rb = r0; rb < r1; rb += kRunBatch) {
      const int nr = min(kRunBatch, r1 - rb);
      __syncthreads();
      scan_runs(L.runs + rb, nr, pre, rst);
      __syncthreads();
      const int cnt = pre[nr];
      for (int v0 = 0; v0 < cnt; v0 += kT) {
        const int m = min(kT, cnt - v0);
        __syncthreads();
        if (threadIdx.x < m) {
          const int v = v0 + threadIdx.x;
          const int rr = find_run(pre, nr, v);
          const int src = rst[rr] + (v - pre[rr]);
          T px, py, pz;
          if (sizeof(T) == 4) {
            const float4 h = G.pthi[1][src], l = G.ptlo[1][src];
            px = (T)((h.x - chx) + (l.x - clx));
            py = (T)((h.y - chy) + (l.y - cly));
            pz = (T)((h.z - chz) + (l.z - clz));
          } else {
            const double4_32a y = G.pt64[1][src];
            px = (T)(y.x - cs.x); py = (T)(y.y - cs.y); pz = (T)(y.z - cs.z);
          }
          const double4_32a nr3 = G.tri_nrm[G.pt_elem[1][src]];
          const T wg = W[(int64_t)d * nsp + src];
          sx[threadIdx.x] = px; sy[threadIdx.x] = py; sz[threadIdx.x] = pz;
          snx[threadIdx.x] = wg * (T)nr3.x; sny[threadIdx.x] = wg * (T)nr3.y; snz[threadIdx.x] = wg * (T)nr3.z;
        }
        __syncthreads();
        if (act) {
          T acc = 0;
          for (int j = 0; j < m; ++j) {
            const T dx = xt - sx[j], dy = yt - sy[j], dz = zt - sz[j];
            const T r2 = dx * dx + dy * dy + dz * dz;
            if (r2 > (T)0) {
              const T ri = (sizeof(T) == 4) ? (T)rsqrt_ftz((float)r2) : (T)(1.0 / sqrt((double)r2));
              acc += (snx[j] * dx + sny[j] * dy + snz[j] * dz) * ri * ri * ri;
            }
          }
          total += (double)acc;
        }
      }
    }
    if (act) phi[(int64_t)d * ntp + tr.x + t] -= total * kInv4Pi;
  }
  }
}

template <typename T>
cudaError_t launch_p2p_dl(const DevGeom& G, const DevTaskLists& L, const T* W, int64_t nsrc_pts, int64_t ntgt_pts,
                          int ndp, double* phi, cudaStream_t st) {
  if (L.n_p2p == 0) return cudaSuccess;
  k_p2p_dl<T><<<L.n_p2p, 128, 0, st>>>(G, L, W, nsrc_pts, ntgt_pts, ndp, phi);
  return cudaGetLastError();
}

template cudaError_t launch_p2m_dl<float>(const DevGeom&, const DevTaskLists&, const float*, int64_t, int, float*, cudaStream_t);
template cudaError_t launch_p2m_dl<double>(const DevGeom&, const DevTaskLists&, const double*, int64_t, int, double*, cudaStream_t);
template cudaError_t launch_p2p_dl<float>(const DevGeom&, const DevTaskLists&, const float*, int64_t, int64_t, int, double*, cudaStream_t);
template cudaError_t launch_p2p_dl<double>(const DevGeom&, const DevTaskLists&, const double*, int64_t, int64_t, int, double*, cudaStream_t);

template cudaError_t launch_weights<float>(const DevGeom&, int, int64_t, const double*, int64_t, int, int, float*, cudaStream_t);
template cudaError_t launch_weights<double>(const DevGeom&, int, int64_t, const double*, int64_t, int, int, double*, cudaStream_t);
template cudaError_t launch_p2m<float>(const DevGeom&, const DevTaskLists&, const float*, int64_t, int, float*, cudaStream_t);
template cudaError_t launch_p2m<double>(const DevGeom&, const DevTaskLists&, const double*, int64_t, int, double*, cudaStream_t);
template cudaError_t launch_m2m<float>(const DevGeom&, const int*, int, int, float*, cudaStream_t);
template cudaError_t launch_m2m<double>(const DevGeom&, const int*, int, int, double*, cudaStream_t);
template cudaError_t launch_m2l_simt<float>(const DevGeom&, const DevTaskLists&, const float*, int, const float*, float*, cudaStream_t, const int*, int);
template cudaError_t launch_m2l_simt<double>(const DevGeom&, const DevTaskLists&, const double*, int, const double*, double*, cudaStream_t, const int*, int);
template cudaError_t launch_l2l<float>(const DevGeom&, const int*, int, int, float*, cudaStream_t);
template cudaError_t launch_l2l<double>(const DevGeom&, const int*, int, int, double*, cudaStream_t);

}  // namespace bcfmm
