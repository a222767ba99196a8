// Auxiliary device passes: the FP64 direct evaluation of sampled target
// elements (the discrete operator summed pair by pair, no expansions),
// which the library uses to measure the error of a fast configuration.
#include <algorithm>

#include "kernels.cuh"

namespace bcfmm {

constexpr double kInv4PiA = 0.079577471545947667884441881686257;
constexpr int kDirectThreads = 256;

// One block per sampled target element e: sum over every source point y_j
// of e's mesh (sorted positions src_rng[2i] .. src_rng[2i+1]) of
// W_j f(elem(y_j)) w_i / (4 pi |x_i - y_j|) over the element's points x_i
// (r = 0 skipped, as in the near-field pass), then e's near corrections.
__global__ void __launch_bounds__(kDirectThreads) k_direct_sample(DevGeom G, DevTaskLists L,
                                                                   const int64_t* __restrict__ targets,
                                                                   const int64_t* __restrict__ src_rng,
                                                                   const double* __restrict__ dens, int ndens, int n,
                                                                   double* __restrict__ out) {
  const int64_t e = targets[blockIdx.x];
  const int sc = L.src_cls, tc = L.tgt_cls;
  double4_32a tp[4];
  const int nq = L.nq_tgt;
  for (int q = 0; q < 4; ++q) {
    const int pos = q < nq ? L.elem_pts[4 * e + q] : -1;
    tp[q] = pos >= 0 ? G.pt64[tc][pos] : make_double4_32a(0, 0, 0, 0);
  }
  double acc[16];
  for (int d = 0; d < 16; ++d) acc[d] = 0.0;
  const int64_t j0 = src_rng[2 * blockIdx.x], j1 = src_rng[2 * blockIdx.x + 1];
  for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
    const double4_32a y = G.pt64[sc][j];
    double g = 0.0;
    for (int q = 0; q < nq; ++q) {
      const double dx = tp[q].x - y.x, dy = tp[q].y - y.y, dz = tp[q].z - y.z;
      const double r2 = dx * dx + dy * dy + dz * dz;
      if (r2 > 0.0) g += tp[q].w / sqrt(r2);
    }
    g *= y.w;
    const int se = G.pt_elem[sc][j];
    for (int d = 0; d < ndens; ++d) acc[d] += g * dens[(int64_t)d * L.nsrc_el + se];
  }
  __shared__ double red[kDirectThreads / 32][16];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int d = 0; d < ndens; ++d) {
    double v = acc[d];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) red[warp][d] = v;
  }
  __syncthreads();
  if (threadIdx.x < ndens) {
    const int d = threadIdx.x;
    double v = 0.0;
    for (int w = 0; w < kDirectThreads / 32; ++w) v += red[w][d];
    v *= kInv4PiA;
    for (int64_t k = L.cor_off[e]; k < L.cor_off[e + 1]; ++k) v += L.cor_val[k] * dens[(int64_t)d * L.nsrc_el + L.cor_col[k]];
    out[(int64_t)d * n + blockIdx.x] = v;
  }
}

cudaError_t launch_direct_sample(const DevGeom& G, const DevTaskLists& L, const int64_t* targets, const int64_t* src_rng,
                                 int n, const double* dens, int ndens, double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (ndens < 1 || ndens > 16) return cudaErrorInvalidValue;
  k_direct_sample<<<n, kDirectThreads, 0, st>>>(G, L, targets, src_rng, dens, ndens, n, out);
  return cudaGetLastError();
}

// FP32 FMA throughput probe: every thread runs 8 independent FMA chains
// (enough to cover the pipe latency) for `iters` steps; the result is
// stored so that nothing is eliminated.
__global__ void __launch_bounds__(256) k_ffma_rate(int iters, float a, float b, float* __restrict__ out) {
  float x[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) x[i] = (float)(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

cudaError_t measure_ffma_rate(int device, double* flops) {
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDeviceProperties(&prop, device);
  if (e != cudaSuccess) return e;
  const int blocks = prop.multiProcessorCount * 8, threads = 256, iters = 1 << 14;
  float* out = nullptr;
  cudaEvent_t t0 = nullptr, t1 = nullptr;
  e = cudaMalloc(&out, sizeof(float) * blocks * threads);
  if (e == cudaSuccess) e = cudaEventCreate(&t0);
  if (e == cudaSuccess) e = cudaEventCreate(&t1);
  float best = 1e30f;
  for (int rep = 0; rep < 4 && e == cudaSuccess; ++rep) {
    // a < 1 keeps the chains finite; rep 0 is the warm-up
    k_ffma_rate<<<blocks, threads>>>(iters, 0.999f, 1e-3f, out);
    e = cudaEventRecord(t0);
    k_ffma_rate<<<blocks, threads>>>(iters, 0.999f, 1e-3f, out);
    if (e == cudaSuccess) e = cudaEventRecord(t1);
    if (e == cudaSuccess) e = cudaEventSynchronize(t1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, t0, t1);
    if (e == cudaSuccess && rep > 0) best = std::min(best, ms);
  }
  if (e == cudaSuccess) *flops = 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3);
  if (t0) cudaEventDestroy(t0);
  if (t1) cudaEventDestroy(t1);
  if (out) cudaFree(out);
  return e;
}

}  // namespace bcfmm
