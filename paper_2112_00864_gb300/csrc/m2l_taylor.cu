// CUDA-core M2L in the Taylor-coefficient form (Sec. 3.3): prescaled
// moments, per-offset derivative coefficients, register-blocked contraction
// over gamma = a + b, chunk sums reduced per target (compensated FP32).
#include <algorithm>
#include <numeric>
#include <utility>

#include "m2l_taylor.cuh"

namespace bcfmm {
namespace {

// degree-major multi-index position: degree d = i + j + k, then i
// descending, then j descending (the order of the expansion arrays)
__host__ __device__ constexpr int mi_idx(int i, int j, int k) {
  return (i + j + k) * (i + j + k + 1) * (i + j + k + 2) / 6 + (j + k) * (j + k + 1) / 2 + k;
}

// The (a, b, gamma = a + b) triples of order Q in contraction order: gamma
// degree-major, then a by components; built at compile time, so that the
// unrolled kernel indexes its register arrays with constants.
__host__ __device__ constexpr int taylor_nterms(int q) {
  int n = 0;
  for (int gi = 0; gi <= q; ++gi)
    for (int gj = 0; gj <= q - gi; ++gj)
      for (int gk = 0; gk <= q - gi - gj; ++gk) n += (gi + 1) * (gj + 1) * (gk + 1);
  return n;
}
template <int Q>
struct TaylorTerms {
  static constexpr int N = taylor_nterms(Q);
  int a[N], b[N], g[N];
  __host__ __device__ constexpr TaylorTerms() : a{}, b{}, g{} {
    int n = 0;
    for (int gi = 0; gi <= Q; ++gi)
      for (int gj = 0; gj <= Q - gi; ++gj)
        for (int gk = 0; gk <= Q - gi - gj; ++gk)
          for (int ai = 0; ai <= gi; ++ai)
            for (int aj = 0; aj <= gj; ++aj)
              for (int ak = 0; ak <= gk; ++ak) {
                a[n] = mi_idx(ai, aj, ak);
                b[n] = mi_idx(gi - ai, gj - aj, gk - ak);
                g[n] = mi_idx(gi, gj, gk);
                ++n;
              }
  }
};
template <int Q>
struct TaylorTab {
  static constexpr TaylorTerms<Q> v{};
};
template <int Q, int I>
struct TaylorTerm {
  static constexpr int a = TaylorTab<Q>::v.a[I], b = TaylorTab<Q>::v.b[I], g = TaylorTab<Q>::v.g[I];
};
template <int Q, int... I>
__device__ __forceinline__ void taylor_contract(float* acc, const float* m, const float* g,
                                                std::integer_sequence<int, I...>) {
  ((acc[TaylorTerm<Q, I>::a] = fmaf(g[TaylorTerm<Q, I>::g], m[TaylorTerm<Q, I>::b], acc[TaylorTerm<Q, I>::a])), ...);
}

__device__ __forceinline__ void two_sum(float& hi, float& lo, float x) {
  const float t = hi + x;
  const float b = t - hi;
  lo += (hi - (t - b)) + (x - b);
  hi = t;
}

// m'[row][b] = m[row][b] * fac[b], fac[b] = (-1)^{|b|} / b!  (b < nq; zero up to the pitch)
__global__ void k_taylor_prescale(const float* __restrict__ mom, int64_t nrow, int ms, int nq, int pitch,
                                  const float* __restrict__ fac, float* __restrict__ momp) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nrow * pitch) return;
  const int64_t row = i / pitch;
  const int b = (int)(i % pitch);
  momp[i] = b < nq ? mom[row * ms + b] * fac[b] : 0.f;
}

// 32-byte read-only load (eight floats; the address is 32-byte aligned)
__device__ __forceinline__ void ldg8(const float* p, float* v) {
  asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=f"(v[0]), "=f"(v[1]), "=f"(v[2]), "=f"(v[3]), "=f"(v[4]), "=f"(v[5]), "=f"(v[6]), "=f"(v[7])
      : "l"(p));
}

struct TaylorArgs {
  const int2* wb;
  const int* lane_chunk;
  const uint32_t* pk;
  int nwarp, cbits, ndp, pitch;
  const float* momp;   // [nbox * ndp][pitch]
  const float* g;      // [ncode][pitch]
  float* partial;      // [nchunk][ndp][nq]
};

// one lane = one chunk: sum over its entries of lambda'_a = sum_b g[a+b] m'_b
template <int Q>
__global__ void __launch_bounds__(128) k_m2l_taylor(TaylorArgs A) {
  constexpr int NQ = (Q + 1) * (Q + 2) * (Q + 3) / 6;
  // 32-byte loads up to order 6; 16-byte loads above (fewer live registers)
  constexpr int W = Q <= 6 ? 8 : 4;
  constexpr int NV = (NQ + W - 1) / W;
  const int w = blockIdx.x * 4 + (threadIdx.x >> 5), lane = threadIdx.x & 31, d = blockIdx.y;
  if (w >= A.nwarp) return;
  const int2 wb = A.wb[w];
  const uint32_t cmask = (1u << A.cbits) - 1u;
  const uint32_t* pk = A.pk + wb.x + lane;
  float acc[NQ];
#pragma unroll
  for (int a = 0; a < NQ; ++a) acc[a] = 0.f;
  uint32_t nxt = wb.y > 0 ? __ldg(pk) : ~0u;
  for (int j = 0; j < wb.y; ++j) {
    const uint32_t cur = nxt;
    if (j + 1 < wb.y) nxt = __ldg(pk + 32 * (j + 1));
    if (cur == ~0u) continue;
    const float* mr = A.momp + ((int64_t)(cur >> A.cbits) * A.ndp + d) * A.pitch;
    const float* gr = A.g + (int64_t)(cur & cmask) * A.pitch;
    float m[NV * W], g[NV * W];
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      if constexpr (W == 8) {
        ldg8(mr + 8 * v, m + 8 * v);
        ldg8(gr + 8 * v, g + 8 * v);
      } else {
        const float4 x = __ldg(reinterpret_cast<const float4*>(mr) + v);
        const float4 y = __ldg(reinterpret_cast<const float4*>(gr) + v);
        m[4 * v] = x.x; m[4 * v + 1] = x.y; m[4 * v + 2] = x.z; m[4 * v + 3] = x.w;
        g[4 * v] = y.x; g[4 * v + 1] = y.y; g[4 * v + 2] = y.z; g[4 * v + 3] = y.w;
      }
    }
    // every (a, b) with |a + b| <= Q
    taylor_contract<Q>(acc, m, g, std::make_integer_sequence<int, taylor_nterms(Q)>{});
  }
  const int c = A.lane_chunk[w * 32 + lane];
  if (c < 0) return;
  float* o = A.partial + ((int64_t)c * A.ndp + d) * NQ;
#pragma unroll
  for (int a = 0; a < NQ; ++a) o[a] = acc[a];
}

// loc[t][d][a] = post[a] / s_t * (sum over the target's chunks, in chunk
// order, compensated), post[a] = 1 / a!; one thread per (target, d, a)
__global__ void __launch_bounds__(128) k_m2l_taylor_reduce(int ntgt, const int* __restrict__ tgt,
                                                          const int* __restrict__ tchunk,
                                                          const float* __restrict__ partial, int nq, int ndp, int ms,
                                                          const float* __restrict__ post,
                                                          const double4_32a* __restrict__ box_cs,
                                                          float* __restrict__ loc) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  const int per = ndp * nq;
  if (i >= (int64_t)ntgt * per) return;
  const int t = (int)(i / per), r = (int)(i % per), d = r / nq, a = r % nq;
  const int tb = tgt[t], c0 = tchunk[t], c1 = tchunk[t + 1];
  float hi = 0.f, lo = 0.f;
  const float* pp = partial + (int64_t)d * nq + a;
#pragma unroll 4
  for (int c = c0; c < c1; ++c) two_sum(hi, lo, __ldg(pp + (int64_t)c * per));
  loc[((int64_t)tb * ndp + d) * ms + a] = (hi + lo) * post[a] / (float)box_cs[tb].w;
}

// Orders above the register-blocked range (any q <= p): one CTA per target,
// the entry's g row and prescaled moment row staged in shared memory, one
// thread per output a (strided), the multi-index of a + b computed from the
// components; FP32 products per entry, compensated FP32 sum over the list.
template <int ND>
__global__ void __launch_bounds__(128) k_m2l_taylor_wide(DevGeom G, DevTaskLists L, const int* __restrict__ sel,
                                                        const float* __restrict__ g, int pitch,
                                                        const float* __restrict__ momp, const float* __restrict__ post,
                                                        float* __restrict__ loc) {
  constexpr int ndp = ND;
  extern __shared__ float wsm[];
  const int ki = sel[blockIdx.x];
  const int tb = L.m2l_tgt[ki];
  const int q = G.box_q[tb], nq = nterms_q(q);
  float* sg = wsm;                       // [nq] the entry's g row
  float* smv = sg + pitch;               // [ndp][nq] its prescaled moment rows
  int* smi = reinterpret_cast<int*>(smv + (size_t)ndp * pitch);   // [nq] packed multi-indices
  for (int i = threadIdx.x; i < nq; i += blockDim.x) smi[i] = G.mi[i];
  constexpr int kMaxPer = 4;             // outputs per thread: nq <= 4 * 128 (q <= 12)
  constexpr int kMaxD = ND;
  float hi[kMaxPer][kMaxD], lo[kMaxPer][kMaxD];
#pragma unroll
  for (int u = 0; u < kMaxPer; ++u)
#pragma unroll
    for (int d = 0; d < kMaxD; ++d) hi[u][d] = lo[u][d] = 0.f;
  const int e0 = L.vl_off[ki], e1 = L.vl_off[ki + 1];
  for (int e = e0; e < e1; ++e) {
    const int sb = L.vl_src[e];
    const float* gr = g + (int64_t)L.vl_code[e] * pitch;
    __syncthreads();
    for (int i = threadIdx.x; i < nq; i += blockDim.x) sg[i] = gr[i];
    for (int i = threadIdx.x; i < ndp * nq; i += blockDim.x)
      smv[(i / nq) * pitch + i % nq] = momp[((int64_t)sb * ndp + i / nq) * pitch + i % nq];
    __syncthreads();
#pragma unroll
    for (int u = 0; u < kMaxPer; ++u) {
      const int a = threadIdx.x + u * 128;
      if (a >= nq) break;
      const int ma = smi[a];
      const int ai = ma & 255, aj = (ma >> 8) & 255, ak = (ma >> 16) & 255;
      const int kb = nterms_q(q - ai - aj - ak);
      float part[kMaxD];
#pragma unroll
      for (int d = 0; d < kMaxD; ++d) part[d] = 0.f;
      for (int b = 0; b < kb; ++b) {
        const int mb = smi[b];
        const int gi = ai + (mb & 255), gj = aj + ((mb >> 8) & 255), gk = ak + ((mb >> 16) & 255);
        const int dg = gi + gj + gk;
        const float gv = sg[dg * (dg + 1) * (dg + 2) / 6 + (gj + gk) * (gj + gk + 1) / 2 + gk];
#pragma unroll
        for (int d = 0; d < kMaxD; ++d) part[d] = fmaf(gv, smv[d * pitch + b], part[d]);
      }
#pragma unroll
      for (int d = 0; d < kMaxD; ++d) two_sum(hi[u][d], lo[u][d], part[d]);
    }
  }
  const float inv_s = 1.0f / (float)G.box_cs[tb].w;
#pragma unroll
  for (int u = 0; u < kMaxPer; ++u) {
    const int a = threadIdx.x + u * 128;
    if (a >= nq) break;
    for (int d = 0; d < ndp; ++d) loc[((int64_t)tb * ndp + d) * G.ms + a] = (hi[u][d] + lo[u][d]) * post[a] * inv_s;
  }
}

template <int Q>
cudaError_t launch_order(const TaylorOrderSched& O, const TaylorTaskSched& S, const TaylorTables& tab, const DevGeom& G,
                         int ndp, const float* momp, float* loc, float* partial, cudaStream_t st) {
  constexpr int NQ = (Q + 1) * (Q + 2) * (Q + 3) / 6;
  TaylorArgs A;
  A.wb = O.wb;
  A.lane_chunk = O.lane_chunk;
  A.pk = O.pk;
  A.nwarp = O.nwarp;
  A.cbits = S.cbits;
  A.ndp = ndp;
  A.pitch = tab.gpitch;
  A.momp = momp;
  A.g = tab.g;
  A.partial = partial;
  k_m2l_taylor<Q><<<dim3((unsigned)((O.nwarp + 3) / 4), (unsigned)ndp), 128, 0, st>>>(A);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t n = (int64_t)O.ntgt * ndp * NQ;
  k_m2l_taylor_reduce<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(O.ntgt, O.tgt, O.tchunk, partial, NQ, ndp, G.ms,
                                                                   tab.fac + tab.gpitch, G.box_cs, loc);
  return cudaGetLastError();
}

}  // namespace

int m2l_taylor_pitch(int q) { return (nterms_q(q) + 7) / 8 * 8; }

bool m2l_taylor_schedule(const std::vector<int>& m2l_tgt, const std::vector<int>& vl_off,
                         const std::vector<int>& vl_src, const std::vector<uint16_t>& vl_code,
                         const std::vector<int>& target_q, int nbox, int ncode, int nsm,
                         std::vector<TaylorOrderHost>& out, std::vector<int>& sel, int* cbits) {
  out.clear();
  sel.clear();
  int cb = 1;
  while ((1 << cb) < std::max(ncode, 2)) ++cb;
  *cbits = cb;
  if ((int64_t)std::max(nbox, 1) << cb >= (int64_t)0xFFFFFFFFu) return false;
  const int nt = (int)m2l_tgt.size();
  for (int k = 0; k < nt; ++k)
    if (target_q[k] < 1 || target_q[k] > kTaylorMaxQ) sel.push_back(k);
  for (int q = 1; q <= kTaylorMaxQ; ++q) {
    TaylorOrderHost O;
    O.q = q;
    std::vector<int> ks;
    for (int k = 0; k < nt; ++k)
      if (target_q[k] == q && vl_off[k + 1] > vl_off[k]) {
        ks.push_back(k);
        O.pairs += vl_off[k + 1] - vl_off[k];
      }
    if (ks.empty()) continue;
    // chunk length: about 48 warps of work per SM, at most 32 entries (the
    // FP32 sum of a chunk stays short), at least 8 (partial-sum traffic)
    O.chunk = (int)std::min<int64_t>(32, std::max<int64_t>(8, (O.pairs + 1536LL * nsm - 1) / (1536LL * nsm)));
    std::vector<int2> ch;   // (first entry, length)
    O.tchunk.assign(1, 0);
    for (int k : ks) {
      const int a = vl_off[k], n = vl_off[k + 1] - a;
      const int nc = (n + O.chunk - 1) / O.chunk;
      for (int i = 0; i < nc; ++i) {
        const int b0 = a + (int)((int64_t)n * i / nc), b1 = a + (int)((int64_t)n * (i + 1) / nc);
        ch.push_back(make_int2(b0, b1 - b0));
      }
      O.tgt.push_back(m2l_tgt[k]);
      O.tchunk.push_back((int)ch.size());
    }
    O.nchunk = (int)ch.size();
    std::vector<int> ord(ch.size());
    std::iota(ord.begin(), ord.end(), 0);
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return ch[x].y > ch[y].y; });
    const int nwarp = (O.nchunk + 31) / 32;
    O.lane_chunk.assign((size_t)nwarp * 32, -1);
    for (int w = 0; w < nwarp; ++w) {
      const int len = ch[ord[(size_t)w * 32]].y;
      O.wb.push_back(make_int2((int)O.pk.size(), len));
      const size_t base = O.pk.size();
      O.pk.resize(base + (size_t)len * 32, ~0u);
      for (int l = 0; l < 32 && w * 32 + l < O.nchunk; ++l) {
        const int c = ord[(size_t)w * 32 + l];
        O.lane_chunk[(size_t)w * 32 + l] = c;
        for (int j = 0; j < ch[c].y; ++j) {
          const int e = ch[c].x + j;
          O.pk[base + (size_t)j * 32 + l] = ((uint32_t)vl_src[e] << cb) | (uint32_t)vl_code[e];
        }
      }
    }
    if (O.pk.size() >= (size_t)INT32_MAX) return false;
    out.push_back(std::move(O));
  }
  return true;
}

cudaError_t launch_m2l_taylor(const DevGeom& G, const DevTaskLists& L, const TaylorTaskSched& S,
                              const TaylorTables& tab, int ndp, const float* mom, float* loc, float* momp,
                              float* partial, cudaStream_t st) {
  int qtop = 0;
  for (int q = 1; q <= kTaylorMaxQ; ++q)
    if (S.ord[q].nwarp > 0) qtop = q;
  if (qtop == 0 && S.nsimt == 0) return cudaSuccess;
  if (qtop > tab.q || tab.gpitch != m2l_taylor_pitch(tab.q) || ndp > 16 || tab.q > 12) return cudaErrorInvalidValue;
  {
    const int64_t nrow = (int64_t)G.nbox * ndp;
    const int64_t n = nrow * tab.gpitch;
    k_taylor_prescale<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(mom, nrow, G.ms, nterms_q(tab.q), tab.gpitch,
                                                                   tab.fac, momp);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (S.nsimt > 0) {
    const size_t sm = sizeof(float) * (size_t)(1 + ndp) * tab.gpitch + sizeof(int) * tab.gpitch;
    const float* post = tab.fac + tab.gpitch;
    switch (ndp) {
      case 1: k_m2l_taylor_wide<1><<<S.nsimt, 128, sm, st>>>(G, L, S.simt_sel, tab.g, tab.gpitch, momp, post, loc); break;
      case 2: k_m2l_taylor_wide<2><<<S.nsimt, 128, sm, st>>>(G, L, S.simt_sel, tab.g, tab.gpitch, momp, post, loc); break;
      case 4: k_m2l_taylor_wide<4><<<S.nsimt, 128, sm, st>>>(G, L, S.simt_sel, tab.g, tab.gpitch, momp, post, loc); break;
      case 8: k_m2l_taylor_wide<8><<<S.nsimt, 128, sm, st>>>(G, L, S.simt_sel, tab.g, tab.gpitch, momp, post, loc); break;
      case 16: k_m2l_taylor_wide<16><<<S.nsimt, 128, sm, st>>>(G, L, S.simt_sel, tab.g, tab.gpitch, momp, post, loc); break;
      default: return cudaErrorInvalidValue;
    }
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  for (int q = 1; q <= kTaylorMaxQ; ++q) {
    const TaylorOrderSched& O = S.ord[q];
    if (O.nwarp == 0) continue;
    cudaError_t e = cudaSuccess;
    switch (q) {
      case 1: e = launch_order<1>(O, S, tab, G, ndp, momp, loc, partial, st); break;
      case 2: e = launch_order<2>(O, S, tab, G, ndp, momp, loc, partial, st); break;
      case 3: e = launch_order<3>(O, S, tab, G, ndp, momp, loc, partial, st); break;
      case 4: e = launch_order<4>(O, S, tab, G, ndp, momp, loc, partial, st); break;
      case 5: e = launch_order<5>(O, S, tab, G, ndp, momp, loc, partial, st); break;
      case 6: e = launch_order<6>(O, S, tab, G, ndp, momp, loc, partial, st); break;
      case 7: e = launch_order<7>(O, S, tab, G, ndp, momp, loc, partial, st); break;
      default: e = cudaErrorInvalidValue;
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace bcfmm
