// Learned correction of near-singular element pairs (near pairs whose
// closures are apart).  The near field of Sec. 3.3 treats every near pair
// with an accurate rule; here a small network predicts, from the pair's
// relative geometry, corrections dw_ij of the product rule's 4 x 4 (or
// 4 x 3) weights:  C_ts ~ sum_ij dw_ij q_ij,  q_ij = W_i W_j / (4 pi r_ij).
//
//   features  the source vertices in the affine frame of the target,
//             centred at the target centroid (12 numbers; both vertex
//             orders canonical: by distance to the other element's centroid)
//   network   12 -> 64 -> 64 -> 16, exact GELU, BF16 weights, FP32 math
//   loss      (sum_ij dw_ij qhat_ij - chat)^2, qhat = q / Q, chat = C / Q,
//             Q = sum_ij q_ij (the pair's product-rule value)
//
// Parameter vector (FP32, 6032): W1[64][12] b1[64] W2[64][64] b2[64]
// W3[16][64] b3[16].  Training keeps FP32 master weights and runs the
// forward and backward passes on their BF16 roundings.
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "mlp.cuh"

namespace bcfmm {

constexpr double kInv4PiM = 0.079577471545947667884441881686257;
constexpr int kMlpThreads = 128;

__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ float gelu(float z) { return 0.5f * z * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu_d(float z) {
  return 0.5f * (1.0f + erff(z * 0.70710678118654752f)) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// ------------------------------------------------------------ geometry
struct D3 { double x, y, z; };
__device__ __forceinline__ D3 dsub(D3 a, D3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double ddot(D3 a, D3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ D3 dcross(D3 a, D3 b) { return {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x}; }

__device__ void load_elem(const double* V, int64_t e, int nv, D3* v) {
  for (int i = 0; i < nv; ++i) v[i] = {V[(e * nv + i) * 3], V[(e * nv + i) * 3 + 1], V[(e * nv + i) * 3 + 2]};
}

__device__ D3 centroid(const D3* v, int nv) {
  D3 c = {0, 0, 0};
  for (int i = 0; i < nv; ++i) { c.x += v[i].x; c.y += v[i].y; c.z += v[i].z; }
  return {c.x / nv, c.y / nv, c.z / nv};
}

__device__ double radius(const D3* v, int nv, D3 c) {
  double r = 0;
  for (int i = 0; i < nv; ++i) { D3 d = dsub(v[i], c); r = fmax(r, sqrt(ddot(d, d))); }
  return r;
}

// Lower bound of the distance between two convex elements (separating
// axes: face normals of both and cross products of edge pairs).  The true
// distance is at least the largest projected gap over any axis.
__device__ double sat_gap(const D3* a, int na, const D3* b, int nb) {
  const int tet_e[6][2] = {{0, 1}, {0, 2}, {0, 3}, {1, 2}, {1, 3}, {2, 3}};
  const int tri_e[3][2] = {{0, 1}, {1, 2}, {0, 2}};
  const int tet_f[4][3] = {{1, 2, 3}, {0, 2, 3}, {0, 1, 3}, {0, 1, 2}};
  double best = -1e300;
  auto test = [&](D3 u) {
    const double l2 = ddot(u, u);
    if (!(l2 > 0)) return;
    const double s = 1.0 / sqrt(l2);
    double amin = 1e300, amax = -1e300, bmin = 1e300, bmax = -1e300;
    for (int i = 0; i < na; ++i) { const double p = ddot(a[i], u) * s; amin = fmin(amin, p); amax = fmax(amax, p); }
    for (int i = 0; i < nb; ++i) { const double p = ddot(b[i], u) * s; bmin = fmin(bmin, p); bmax = fmax(bmax, p); }
    best = fmax(best, fmax(bmin - amax, amin - bmax));
  };
  const int nfa = na == 4 ? 4 : 1, nfb = nb == 4 ? 4 : 1;
  for (int f = 0; f < nfa; ++f) {
    const int* F = na == 4 ? tet_f[f] : tet_f[3];
    test(dcross(dsub(a[F[1]], a[F[0]]), dsub(a[F[2]], a[F[0]])));
  }
  for (int f = 0; f < nfb; ++f) {
    const int* F = nb == 4 ? tet_f[f] : tet_f[3];
    test(dcross(dsub(b[F[1]], b[F[0]]), dsub(b[F[2]], b[F[0]])));
  }
  const int nea = na == 4 ? 6 : 3, neb = nb == 4 ? 6 : 3;
  for (int i = 0; i < nea; ++i) {
    const int* E = na == 4 ? tet_e[i] : tri_e[i];
    const D3 ea = dsub(a[E[1]], a[E[0]]);
    for (int j = 0; j < neb; ++j) {
      const int* G = nb == 4 ? tet_e[j] : tri_e[j];
      const D3 u = dcross(ea, dsub(b[G[1]], b[G[0]]));
      if (ddot(u, u) > 1e-24 * ddot(ea, ea) * ddot(ea, ea)) test(u);
    }
  }
  return best;
}

// calibration bin of a near-singular pair: centroid distance over the
// radius sum (8 bins on [0,1)) x gap lower bound over the radius sum
// (4 bins: [0,.05) [.05,.15) [.15,.3) [.3,inf))
__device__ int pair_bin(double dist_ratio, double gap_ratio) {
  const int a = min(kMlpBinsEta - 1, max(0, (int)(dist_ratio * kMlpBinsEta)));
  const int b = gap_ratio < 0.05 ? 0 : (gap_ratio < 0.15 ? 1 : (gap_ratio < 0.3 ? 2 : 3));
  return a * kMlpBinsGap + b;
}

// Features, normalised product-rule terms and Q of one pair.
//   tgt (nvt vertices), src (nvs vertices); quadrature point k of an
//   element carries the largest barycentric weight at vertex k.
__device__ void pair_features(const D3* tv_in, int nvt, double tvol, const D3* sv_in, int nvs, double svol,
                              float* feat, float* qhat, double* Q) {
  const D3 ct = centroid(tv_in, nvt), cs = centroid(sv_in, nvs);
  // canonical vertex orders: by distance to the other element's centroid
  int pt[4] = {0, 1, 2, 3}, ps[4] = {0, 1, 2, 3};
  double dt[4], ds[4];
  // (squared distances rounded as written, no fused multiply-add: equal
  // distances of symmetric configurations stay exactly equal, so ties keep
  // the input order on every machine)
  auto d2 = [](D3 d) { return __dadd_rn(__dadd_rn(__dmul_rn(d.x, d.x), __dmul_rn(d.y, d.y)), __dmul_rn(d.z, d.z)); };
  for (int i = 0; i < nvt; ++i) dt[i] = d2(dsub(tv_in[i], cs));
  for (int i = 0; i < nvs; ++i) ds[i] = d2(dsub(sv_in[i], ct));
  for (int i = 1; i < nvt; ++i)
    for (int j = i; j > 0 && dt[pt[j]] < dt[pt[j - 1]]; --j) { int t = pt[j]; pt[j] = pt[j - 1]; pt[j - 1] = t; }
  for (int i = 1; i < nvs; ++i)
    for (int j = i; j > 0 && ds[ps[j]] < ds[ps[j - 1]]; --j) { int t = ps[j]; ps[j] = ps[j - 1]; ps[j - 1] = t; }
  D3 tv[4], sv[4];
  for (int i = 0; i < nvt; ++i) tv[i] = tv_in[pt[i]];
  for (int i = 0; i < nvs; ++i) sv[i] = sv_in[ps[i]];
  // target frame columns a0, a1, a2
  D3 a0 = dsub(tv[1], tv[0]), a1 = dsub(tv[2], tv[0]), a2;
  if (nvt == 4) {
    a2 = dsub(tv[3], tv[0]);
  } else {
    D3 n = dcross(a0, a1);
    const double nn = sqrt(ddot(n, n));
    const double s = sqrt(nn) / nn;                // unit normal times sqrt(2 area)
    n = {n.x * s, n.y * s, n.z * s};
    if (ddot(n, dsub(cs, ct)) < 0) n = {-n.x, -n.y, -n.z};
    a2 = n;
  }
  // inverse of [a0 a1 a2] by cofactors
  const D3 c0 = dcross(a1, a2), c1 = dcross(a2, a0), c2 = dcross(a0, a1);
  const double det = ddot(a0, c0);
  const double id = 1.0 / det;
  for (int k = 0; k < 4; ++k) {
    if (k < nvs) {
      const D3 r = dsub(sv[k], ct);
      feat[3 * k] = (float)(ddot(c0, r) * id);
      feat[3 * k + 1] = (float)(ddot(c1, r) * id);
      feat[3 * k + 2] = (float)(ddot(c2, r) * id);
    } else {
      feat[3 * k] = feat[3 * k + 1] = feat[3 * k + 2] = 0.f;
    }
  }
  // quadrature points in the canonical orders and the product-rule terms
  const double ta = (5.0 + 3.0 * sqrt(5.0)) / 20.0, tb = (5.0 - sqrt(5.0)) / 20.0;
  D3 xq[4], yq[4];
  for (int q = 0; q < nvt; ++q) {
    D3 s = {0, 0, 0};
    for (int i = 0; i < nvt; ++i) {
      const double w = nvt == 4 ? (i == q ? ta : tb) : (i == q ? 2.0 / 3.0 : 1.0 / 6.0);
      s.x += w * tv[i].x; s.y += w * tv[i].y; s.z += w * tv[i].z;
    }
    xq[q] = s;
  }
  for (int q = 0; q < nvs; ++q) {
    D3 s = {0, 0, 0};
    for (int i = 0; i < nvs; ++i) {
      const double w = nvs == 4 ? (i == q ? ta : tb) : (i == q ? 2.0 / 3.0 : 1.0 / 6.0);
      s.x += w * sv[i].x; s.y += w * sv[i].y; s.z += w * sv[i].z;
    }
    yq[q] = s;
  }
  const double wt = tvol / nvt, ws = svol / nvs;
  double q[16], sum = 0.0;
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double v = 0.0;
      if (i < nvt && j < nvs) {
        const D3 d = dsub(xq[i], yq[j]);
        const double r = sqrt(ddot(d, d));
        v = r > 0 ? wt * ws * kInv4PiM / r : 0.0;
      }
      q[4 * i + j] = v;
      sum += v;
    }
  *Q = sum;
  for (int k = 0; k < 16; ++k) qhat[k] = (float)(q[k] / sum);
}

__device__ double elem_size(const D3* v, int nv) {
  const D3 n = dcross(dsub(v[1], v[0]), dsub(v[2], v[0]));
  if (nv == 3) return 0.5 * sqrt(ddot(n, n));
  return fabs(ddot(n, dsub(v[3], v[0]))) / 6.0;
}

// ------------------------------------------------------------ network
// forward on BF16-rounded weights held in shared memory (FP32 storage)
__device__ float mlp_forward(const float* __restrict__ P, const float* x, const float* qhat, float* z1, float* z2) {
  float h1[kMlpH];
  for (int j = 0; j < kMlpH; ++j) {
    float s = P[kOffB1 + j];
#pragma unroll
    for (int k = 0; k < kMlpIn; ++k) s = fmaf(P[kOffW1 + j * kMlpIn + k], x[k], s);
    z1[j] = s;
    h1[j] = gelu(s);
  }
  float pred = 0.f;
  float h2[kMlpH];
  for (int j = 0; j < kMlpH; ++j) {
    float s = P[kOffB2 + j];
    for (int k = 0; k < kMlpH; ++k) s = fmaf(P[kOffW2 + j * kMlpH + k], h1[k], s);
    z2[j] = s;
    h2[j] = gelu(s);
  }
  for (int o = 0; o < kMlpOut; ++o) {
    float s = P[kOffB3 + o];
    for (int k = 0; k < kMlpH; ++k) s = fmaf(P[kOffW3 + o * kMlpH + k], h2[k], s);
    pred = fmaf(s, qhat[o], pred);
  }
  return pred;
}

__device__ void load_params_bf16(const float* __restrict__ src, float* dst) {
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) dst[i] = bf16r(src[i]);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Mean loss and its gradient over n pairs (grad and loss accumulated with
// atomics; the caller zeroes them).  One pair per thread.  Weight
// gradients are outer-product sums over the pairs of a warp: the warp
// stages its 32 rows of the two factors in shared memory and every lane
// forms whole dot products over the 32 pairs (no per-parameter shuffles).
constexpr int kStage = 65;                              // padded row of a staged factor
constexpr int kGradSmem = (2 * kMlpParams + (kMlpThreads / 32) * 2 * 32 * kStage) * 4;

__device__ __forceinline__ void warp_outer(const float* A, int na, const float* B, int nb, float* G, int lane) {
  for (int idx = lane; idx < na * nb; idx += 32) {
    const int a = idx / nb, b = idx - a * nb;
    float s = 0.f;
#pragma unroll 8
    for (int p = 0; p < 32; ++p) s = fmaf(A[p * kStage + a], B[p * kStage + b], s);
    atomicAdd(&G[idx], s);
  }
}

__device__ __forceinline__ void warp_colsum(const float* A, int na, float* G, int lane) {
  for (int a = lane; a < na; a += 32) {
    float s = 0.f;
    for (int p = 0; p < 32; ++p) s += A[p * kStage + a];
    atomicAdd(&G[a], s);
  }
}

__global__ void __launch_bounds__(kMlpThreads) k_mlp_grad(const float* __restrict__ params,
                                                          const float* __restrict__ feat,
                                                          const float* __restrict__ qhat,
                                                          const float* __restrict__ chat, int64_t n, float inv_n,
                                                          float* __restrict__ grad, float* __restrict__ loss) {
  extern __shared__ float sm[];
  float* P = sm;
  float* Gs = sm + kMlpParams;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  float* A = sm + 2 * kMlpParams + warp * 2 * 32 * kStage;
  float* B = A + 32 * kStage;
  load_params_bf16(params, P);
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) Gs[i] = 0.f;
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const bool live = i < n;
  float x[kMlpIn], qh[kMlpOut], z1[kMlpH], z2[kMlpH];
  for (int k = 0; k < kMlpIn; ++k) x[k] = live ? feat[i * kMlpIn + k] : 0.f;
  for (int k = 0; k < kMlpOut; ++k) qh[k] = live ? qhat[i * kMlpOut + k] : 0.f;
  const float pred = mlp_forward(P, x, qh, z1, z2);
  const float e = live ? pred - chat[i] : 0.f;
  const float dpred = 2.f * e * inv_n;
  {
    const float l = warp_sum(e * e * inv_n);
    if (lane == 0) atomicAdd(loss, l);
  }
  float* ra = A + lane * kStage;
  float* rb = B + lane * kStage;
  // layer 3: dy_o = dpred qhat_o;  dW3 = dy h2^T, db3 = dy
  for (int o = 0; o < kMlpOut; ++o) ra[o] = dpred * qh[o];
  for (int k = 0; k < kMlpH; ++k) rb[k] = gelu(z2[k]);
  __syncwarp();
  warp_outer(A, kMlpOut, B, kMlpH, Gs + kOffW3, lane);
  warp_colsum(A, kMlpOut, Gs + kOffB3, lane);
  float dz2[kMlpH];
  for (int k = 0; k < kMlpH; ++k) {
    float s = 0.f;
    for (int o = 0; o < kMlpOut; ++o) s = fmaf(P[kOffW3 + o * kMlpH + k], ra[o], s);
    dz2[k] = s * gelu_d(z2[k]);
  }
  __syncwarp();
  // layer 2: dW2 = dz2 h1^T, db2 = dz2
  for (int k = 0; k < kMlpH; ++k) { ra[k] = dz2[k]; rb[k] = gelu(z1[k]); }
  __syncwarp();
  warp_outer(A, kMlpH, B, kMlpH, Gs + kOffW2, lane);
  warp_colsum(A, kMlpH, Gs + kOffB2, lane);
  float dz1[kMlpH];
  for (int m = 0; m < kMlpH; ++m) {
    float s = 0.f;
    for (int k = 0; k < kMlpH; ++k) s = fmaf(P[kOffW2 + k * kMlpH + m], ra[k], s);
    dz1[m] = s * gelu_d(z1[m]);
  }
  __syncwarp();
  // layer 1: dW1 = dz1 x^T, db1 = dz1
  for (int m = 0; m < kMlpH; ++m) ra[m] = dz1[m];
  for (int k = 0; k < kMlpIn; ++k) rb[k] = x[k];
  __syncwarp();
  warp_outer(A, kMlpH, B, kMlpIn, Gs + kOffW1, lane);
  warp_colsum(A, kMlpH, Gs + kOffB1, lane);
  __syncthreads();
  for (int p = threadIdx.x; p < kMlpParams; p += blockDim.x) atomicAdd(&grad[p], Gs[p]);
}

__global__ void k_mlp_adam(float* __restrict__ params, const float* __restrict__ grad, float* __restrict__ m1,
                           float* __restrict__ m2, float lr, float b1, float b2, float eps, float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  const float g = grad[i];
  const float a = b1 * m1[i] + (1.f - b1) * g;
  const float b = b2 * m2[i] + (1.f - b2) * g * g;
  m1[i] = a;
  m2[i] = b;
  params[i] -= lr * (a * c1) / (sqrtf(b * c2) + eps);
}

__global__ void __launch_bounds__(kMlpThreads) k_mlp_predict(const float* __restrict__ params,
                                                             const float* __restrict__ feat,
                                                             const float* __restrict__ qhat, int64_t n,
                                                             float* __restrict__ out) {
  __shared__ float P[kMlpParams];
  load_params_bf16(params, P);
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  float x[kMlpIn], qh[kMlpOut], z1[kMlpH], z2[kMlpH];
  for (int k = 0; k < kMlpIn; ++k) x[k] = feat[i * kMlpIn + k];
  for (int k = 0; k < kMlpOut; ++k) qh[k] = qhat[i * kMlpOut + k];
  out[i] = mlp_forward(P, x, qh, z1, z2);
}

// ------------------------------------------------------- setup passes
// Classify every near pair k (CSR position): touching (gap bound <= 1e-9
// of the radius sum) -> FP64 near rule; near-singular -> appended to the
// near-singular list and, by mode, to the learned list (its bin's
// calibrated error <= tol), the FP64 list (bin rejected), or nowhere
// (mode 2: product rule only).
__global__ void k_near_classify(int task, int64_t nnz, const int* __restrict__ row, const int* __restrict__ col,
                                const double* __restrict__ tgt_v, const double* __restrict__ src_v, int mode,
                                const float* __restrict__ eps_tab, float tol, int64_t* __restrict__ lists,
                                unsigned long long* __restrict__ counts, int64_t cap) {
  const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (k >= nnz) return;
  const int nvt = task == 1 ? 3 : 4, nvs = task == 2 ? 3 : 4;
  D3 tv[4], sv[4];
  load_elem(tgt_v, row[k], nvt, tv);
  load_elem(src_v, col[k], nvs, sv);
  const D3 ct = centroid(tv, nvt), cs = centroid(sv, nvs);
  const double rs = radius(tv, nvt, ct) + radius(sv, nvs, cs);
  const double gap = sat_gap(tv, nvt, sv, nvs);
  int cls;                                   // 0 FP64 list, 1 learned list, 2 none
  if (gap <= 1e-9 * rs) {
    cls = 0;
  } else {
    const unsigned long long s = atomicAdd(&counts[3], 1ull);
    if ((int64_t)s < cap) lists[3 * cap + s] = k;
    if (mode == 2) {
      cls = 2;
    } else {
      const D3 d = dsub(ct, cs);
      const int b = pair_bin(sqrt(ddot(d, d)) / rs, gap / rs);
      cls = (eps_tab != nullptr && eps_tab[b] <= tol) ? 1 : 0;
    }
  }
  if (cls < 2) {
    const unsigned long long s = atomicAdd(&counts[cls], 1ull);
    if ((int64_t)s < cap) lists[cls * cap + s] = k;
  }
}

// Fused learned correction of the pairs in sel[0..n): geometry, features,
// network (BF16 weights in shared memory, FP32 accumulation) and the
// contraction with the product-rule terms; writes C_ts = Q sum dw qhat.
__global__ void __launch_bounds__(kMlpThreads) k_near_mlp(int task, const int64_t* __restrict__ sel, int64_t n,
                                                          const int* __restrict__ row, const int* __restrict__ col,
                                                          const double* __restrict__ tgt_v,
                                                          const double* __restrict__ src_v,
                                                          const float* __restrict__ params,
                                                          double* __restrict__ cor_val) {
  __shared__ float P[kMlpParams];
  load_params_bf16(params, P);
  __syncthreads();
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t k = sel[i];
  const int nvt = task == 1 ? 3 : 4, nvs = task == 2 ? 3 : 4;
  D3 tv[4], sv[4];
  load_elem(tgt_v, row[k], nvt, tv);
  load_elem(src_v, col[k], nvs, sv);
  float x[kMlpIn], qh[kMlpOut], z1[kMlpH], z2[kMlpH];
  double Q;
  pair_features(tv, nvt, elem_size(tv, nvt), sv, nvs, elem_size(sv, nvs), x, qh, &Q);
  cor_val[k] = Q * (double)mlp_forward(P, x, qh, z1, z2);
}

// Training / validation data of the pairs sel[0..n): features, qhat, Q,
// calibration bin (labels come from the FP64 near rule separately).
__global__ void k_pair_data(int task, const int64_t* __restrict__ sel, int64_t n, const int* __restrict__ row,
                            const int* __restrict__ col, const double* __restrict__ tgt_v,
                            const double* __restrict__ src_v, float* __restrict__ feat, float* __restrict__ qhat,
                            double* __restrict__ Q, int* __restrict__ bin, int* __restrict__ pairs) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t k = sel[i];
  if (pairs) { pairs[2 * i] = row[k]; pairs[2 * i + 1] = col[k]; }
  const int nvt = task == 1 ? 3 : 4, nvs = task == 2 ? 3 : 4;
  D3 tv[4], sv[4];
  load_elem(tgt_v, row[k], nvt, tv);
  load_elem(src_v, col[k], nvs, sv);
  pair_features(tv, nvt, elem_size(tv, nvt), sv, nvs, elem_size(sv, nvs), feat + i * kMlpIn, qhat + i * kMlpOut, &Q[i]);
  const D3 ct = centroid(tv, nvt), cs = centroid(sv, nvs);
  const double rs = radius(tv, nvt, ct) + radius(sv, nvs, cs);
  const D3 d = dsub(ct, cs);
  bin[i] = pair_bin(sqrt(ddot(d, d)) / rs, sat_gap(tv, nvt, sv, nvs) / rs);
}

__global__ void k_select_strided(const int64_t* __restrict__ list, int64_t n_list, int64_t m, int64_t* __restrict__ sel) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < m) sel[i] = list[(int64_t)((double)i * (double)n_list / (double)m)];
}

__global__ void k_label_ratio(const double* __restrict__ C, const double* __restrict__ Q, int64_t n,
                              float* __restrict__ chat) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) chat[i] = (float)(C[i] / Q[i]);
}

// ------------------------------------------------------------ launchers
cudaError_t launch_mlp_grad(const float* params, const float* feat, const float* qhat, const float* chat, int64_t n,
                            float* grad, float* loss, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(grad, 0, kMlpParams * sizeof(float), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(loss, 0, sizeof(float), st);
  if (e != cudaSuccess || n == 0) return e;
  e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize, kGradSmem);
  if (e != cudaSuccess) return e;
  k_mlp_grad<<<(unsigned)((n + kMlpThreads - 1) / kMlpThreads), kMlpThreads, kGradSmem, st>>>(
      params, feat, qhat, chat, n, 1.0f / (float)n, grad, loss);
  return cudaGetLastError();
}

cudaError_t launch_mlp_adam(float* params, const float* grad, float* m1, float* m2, int step, float lr, float b1,
                            float b2, float eps, cudaStream_t st) {
  const float c1 = 1.0f / (1.0f - powf(b1, (float)step)), c2 = 1.0f / (1.0f - powf(b2, (float)step));
  k_mlp_adam<<<(kMlpParams + 255) / 256, 256, 0, st>>>(params, grad, m1, m2, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t launch_mlp_predict(const float* params, const float* feat, const float* qhat, int64_t n, float* out,
                               cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_mlp_predict<<<(unsigned)((n + kMlpThreads - 1) / kMlpThreads), kMlpThreads, 0, st>>>(params, feat, qhat, n, out);
  return cudaGetLastError();
}

cudaError_t launch_near_classify(int task, int64_t nnz, const int* row, const int* col, const double* tgt_v,
                                 const double* src_v, int mode, const float* eps_tab, float tol, int64_t* lists,
                                 unsigned long long* counts, int64_t cap, cudaStream_t st) {
  if (nnz == 0) return cudaSuccess;
  k_near_classify<<<(unsigned)((nnz + 127) / 128), 128, 0, st>>>(task, nnz, row, col, tgt_v, src_v, mode, eps_tab, tol,
                                                                 lists, counts, cap);
  return cudaGetLastError();
}

cudaError_t launch_near_mlp(int task, const int64_t* sel, int64_t n, const int* row, const int* col,
                            const double* tgt_v, const double* src_v, const float* params, double* cor_val,
                            cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_near_mlp<<<(unsigned)((n + kMlpThreads - 1) / kMlpThreads), kMlpThreads, 0, st>>>(task, sel, n, row, col, tgt_v,
                                                                                    src_v, params, cor_val);
  return cudaGetLastError();
}

cudaError_t launch_select_strided(const int64_t* list, int64_t n_list, int64_t m, int64_t* sel, cudaStream_t st) {
  if (m == 0) return cudaSuccess;
  k_select_strided<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(list, n_list, m, sel);
  return cudaGetLastError();
}

cudaError_t launch_label_ratio(const double* C, const double* Q, int64_t n, float* chat, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_label_ratio<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(C, Q, n, chat);
  return cudaGetLastError();
}

cudaError_t launch_pair_data(int task, const int64_t* sel, int64_t n, const int* row, const int* col,
                             const double* tgt_v, const double* src_v, float* feat, float* qhat, double* Q, int* bin,
                             int* pairs, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_pair_data<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(task, sel, n, row, col, tgt_v, src_v, feat, qhat, Q, bin,
                                                           pairs);
  return cudaGetLastError();
}

}  // namespace bcfmm
