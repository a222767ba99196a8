// Interaction phase (M2L, Sec. 3.3) on the 5th-generation tensor cores.
//
// For one tile of 128 target boxes (same level, same octant in the parent)
// and one density, the kernel walks the interaction offsets o present in the
// tile.  Per offset it forms
//   A[r][b] = m_{src(r,o)}^b           (128 rows: targets; K: moment index b)
//   B[a][b] = T_o[a][b]                (N: local index a)
// and accumulates D = A B^T in TMEM (tcgen05.mma, kind::f16, BF16 operands,
// FP32 accumulation): D[r][a] = sum_b T_o[a][b] m^b = lambda_r^a * s.
// FP32 operands are split into BF16 parts (hi + lo, or hi + mid + lo) and the
// partial products that carry the significant bits are summed
// (x2: hh + hl + lh; x3: hh + hm + mh + hl + lh + mm).
// T_o[a][b] vanishes unless |a| + |b| <= p, so the N range is cut into
// chunks whose K extent shrinks with the degree of a.
// D lives in one of two TMEM windows; every kFlush offsets the finished
// window is added into a compensated running sum SH + SL (TwoSum, also in
// TMEM) while the next window accumulates, so the sum over the ~10^3 offsets
// of a box never runs through one long FP32 chain.
//
// Shared-memory operands use the K-major, no-swizzle canonical layout: core
// matrices of 8 rows x 16 bytes; LBO = 128 B (next core along K), SBO =
// (K extent / 8) * 128 B (next group of 8 rows).
#include <cuda_bf16.h>

#include <cstdint>
#include <cstring>
#include <vector>

#include "internal.h"
#include "m2l_tc.cuh"

namespace bcfmm {

namespace {

constexpr int kTileM = 128;
constexpr int kFlush = 4;           // offsets per TMEM accumulation window
constexpr long kSpinLimit = 1L << 22;

struct Chunk {
  int n0, n, ksteps;    // N range [n0, n0+n), K extent = 16 * ksteps
  int boff;             // byte offset of the chunk inside one B part
};

struct TcPlan {
  int p = 0, np = 0, kpad = 0, npad = 0, nchunk = 0, nsplit = 0;
  Chunk ch[16];
  int bpart_bytes = 0;  // one BF16 part of one offset's B (all chunks)
  int apart_bytes = 0;  // one BF16 part of A (128 rows x kpad)
  int stage_bytes = 0;
  int smem_bytes = 0;
  int tmem_cols = 0;
};

struct TcArgs {
  TcPlan P;
  const int* tile_tgt;       // [ntile][128] target box (-1 pad)
  const int* tile_off;       // [ntile+1] entry range
  const int* ent_code;       // [nent] offset code
  const int* ent_src;        // [nent][128] source box (-1: none)
  const uint8_t* bparts;     // [ncode][nsplit][bpart_bytes]
  const float* mom;          // [nbox][ndp][np]
  float* loc;                // [nbox][ndp][np]
  const double4_32a* box_cs;
  int ndp;
  int* err;
};

int host_nterms(int p) { return p < 0 ? 0 : (p + 1) * (p + 2) * (p + 3) / 6; }

TcPlan make_plan(int p, int nsplit) {
  TcPlan P;
  P.p = p;
  P.np = host_nterms(p);
  P.kpad = (P.np + 15) / 16 * 16;
  P.npad = P.kpad;
  P.nsplit = nsplit;
  MultiIndex M;
  M.init(p);
  auto ksteps_at = [&](int n0) {
    if (n0 >= P.np) return 1;
    const int deg = M.a[n0] + M.b[n0] + M.c[n0];
    return (host_nterms(p - deg) + 15) / 16;
  };
  int boff = 0;
  for (int n0 = 0; n0 < P.npad; n0 += 16) {
    const int ks = ksteps_at(n0);
    if (P.nchunk > 0 && P.ch[P.nchunk - 1].ksteps == ks && P.ch[P.nchunk - 1].n + 16 <= 256) {
      P.ch[P.nchunk - 1].n += 16;
    } else {
      P.ch[P.nchunk] = {n0, 16, ks, 0};
      P.nchunk++;
    }
  }
  for (int c = 0; c < P.nchunk; ++c) {
    P.ch[c].boff = boff;
    boff += P.ch[c].n * P.ch[c].ksteps * 16 * 2;
  }
  P.bpart_bytes = boff;
  P.apart_bytes = kTileM * P.kpad * 2;
  P.stage_bytes = nsplit * (P.apart_bytes + P.bpart_bytes);
  P.smem_bytes = 2 * P.stage_bytes + 1024 + 64;   // + alignment slack, barriers, TMEM address
  int cols = 32;
  while (cols < P.npad) cols <<= 1;
  P.tmem_cols = cols;
  return P;
}

// byte offset of element (row r, col k) in a K-major no-swizzle operand
// whose K extent is kext
inline int canon_off(int r, int k, int kext) { return (r >> 3) * (kext / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2; }

__host__ __device__ inline void split_parts(float x, int nsplit, __nv_bfloat16* out) {
  const __nv_bfloat16 h = __float2bfloat16_rn(x);
  const float r1 = x - __bfloat162float(h);
  out[0] = h;
  if (nsplit == 2) {
    out[1] = __float2bfloat16_rn(r1);
  } else {
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    out[1] = m;
    out[2] = __float2bfloat16_rn(r1 - __bfloat162float(m));
  }
}

// ------------------------------------------------------------- PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

// bounded wait: sets *err and returns false when the phase never completes
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  for (long i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(err, 1);
  return false;
}

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);   // version 1, no swizzle
}

// kind::f16 instruction descriptor: D f32, A/B bf16, both K-major, M = 128
__device__ __forceinline__ uint32_t idesc_bf16(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
}

__device__ __forceinline__ void umma(uint32_t tmem_d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void umma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// --------------------------------------------------------------- kernel
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float* v) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          taddr),
      "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])), "r"(__float_as_uint(v[3])),
      "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])), "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])),
      "r"(__float_as_uint(v[8])), "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
      "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])), "r"(__float_as_uint(v[15]))
      : "memory");
}

// TMEM columns: two window accumulators and the compensated running sum
constexpr uint32_t kColD0 = 0, kColD1 = 128, kColSH = 256, kColSL = 384;
constexpr int kThreads = 256;       // row r = tid % 128, half h = tid / 128
constexpr int kMaxB16 = 8;          // uint4 of B per thread (prefetched)

// Adds window accumulator D into the running sum (SH + SL) with TwoSum, for
// this thread's 32-lane quarter and column half.
template <int NPAD>
__device__ __forceinline__ void drain(uint32_t tq, uint32_t dcol, int h, bool first) {
#pragma unroll
  for (int c = 0; c < NPAD / 2; c += 16) {
    const uint32_t col = (uint32_t)(h * (NPAD / 2) + c);
    float d[16], sh[16], sl[16];
    tmem_ld16(tq + dcol + col, d);
    if (first) {
#pragma unroll
      for (int i = 0; i < 16; ++i) { sh[i] = d[i]; sl[i] = 0.f; }
    } else {
      tmem_ld16(tq + kColSH + col, sh);
      tmem_ld16(tq + kColSL + col, sl);
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const float s = sh[i] + d[i];
        const float bb = s - sh[i];
        const float e = (sh[i] - (s - bb)) + (d[i] - bb);
        sh[i] = s;
        sl[i] += e;
      }
    }
    tmem_st16(tq + kColSH + col, sh);
    tmem_st16(tq + kColSL + col, sl);
  }
  asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

template <int NSPLIT, int NPAD>
__global__ void __launch_bounds__(kThreads, 1) k_m2l_tc(TcArgs args) {
  extern __shared__ __align__(1024) uint8_t smraw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const TcPlan& P = args.P;
  uint8_t* stage[2] = {sm, sm + P.stage_bytes};
  uint64_t* bars = (uint64_t*)(sm + 2 * P.stage_bytes);          // [2] MMA-completion barriers
  uint32_t* tmem_holder = (uint32_t*)(bars + 2);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = tid & (kTileM - 1), h = tid >> 7;
  const int tile = blockIdx.x, d = blockIdx.y;
  const int e0 = args.tile_off[tile], e1 = args.tile_off[tile + 1];
  const int nent = e1 - e0;
  const int row_tgt = args.tile_tgt[tile * kTileM + row];
  constexpr int KH4 = NPAD / 8;     // float4 per half row (K extent = NPAD)
  const int np = P.np, ms = (np + 3) & ~3;

  if (tid == 0) {
    mbar_init(smem_u32(&bars[0]), 1);
    mbar_init(smem_u32(&bars[1]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_holder;
  const uint32_t tq = tmem + ((uint32_t)((warp & 3) * 32) << 16);   // this warp's lane quarter

  const uint32_t sbo_a = (uint32_t)(P.kpad / 8) * 128u;
  const int row_off = (row >> 3) * (int)sbo_a + (row & 7) * 16;
  const int k0 = h * (NPAD / 2);
  const int n16 = NSPLIT * P.bpart_bytes / 16;

  // prefetch registers: this thread's half row of moments and its share of
  // B for the next offset; the source index two offsets ahead
  float4 rb[KH4];
  uint4 bb[kMaxB16];
  int src_next = nent > 0 ? args.ent_src[(int64_t)e0 * kTileM + row] : -1;
  int src_next2 = nent > 1 ? args.ent_src[(int64_t)(e0 + 1) * kTileM + row] : -1;
  auto load_entry = [&](int g) {
    const int e = e0 + g;
    const int src = src_next;
    src_next = src_next2;
    src_next2 = (g + 2 < nent) ? args.ent_src[(int64_t)(e + 2) * kTileM + row] : -1;
    const float4* mrow = reinterpret_cast<const float4*>(args.mom + ((int64_t)(src < 0 ? 0 : src) * args.ndp + d) * ms);
#pragma unroll
    for (int i = 0; i < KH4; ++i) {
      const int k = k0 + 4 * i;
      rb[i] = (src >= 0 && k < ms) ? __ldg(mrow + k / 4) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const uint4* srcb = reinterpret_cast<const uint4*>(args.bparts + (int64_t)args.ent_code[e] * NSPLIT * P.bpart_bytes);
#pragma unroll
    for (int i = 0; i < kMaxB16; ++i) {
      const int q = tid + i * kThreads;
      if (q < n16) bb[i] = __ldg(srcb + q);
    }
  };

  bool ok = true;
  int win = 0;                       // window index of code g
  if (nent > 0) load_entry(0);
  for (int g = 0; g < nent && ok; ++g) {
    const int s = g & 1;
    uint8_t* st = stage[s];
    const bool win_first = (g % kFlush) == 0;
    win = g / kFlush;
    // A: split this thread's half row into BF16 parts (canonical K-major layout)
#pragma unroll
    for (int jj = 0; jj < KH4 / 2; ++jj) {
      const float4 lo4 = rb[2 * jj], hi4 = rb[2 * jj + 1];
      const float x[8] = {lo4.x, lo4.y, lo4.z, lo4.w, hi4.x, hi4.y, hi4.z, hi4.w};
      __nv_bfloat16 part[NSPLIT][8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        __nv_bfloat16 pp[3];
        split_parts(x[q], NSPLIT, pp);
#pragma unroll
        for (int t = 0; t < NSPLIT; ++t) part[t][q] = pp[t];
      }
      const int j = (k0 >> 3) + jj;
#pragma unroll
      for (int t = 0; t < NSPLIT; ++t)
        *reinterpret_cast<uint4*>(st + t * P.apart_bytes + row_off + j * 128) = *reinterpret_cast<const uint4*>(part[t]);
    }
    // B: the pre-laid-out parts of T_o
    {
      uint4* dstb = reinterpret_cast<uint4*>(st + NSPLIT * P.apart_bytes);
#pragma unroll
      for (int i = 0; i < kMaxB16; ++i) {
        const int q = tid + i * kThreads;
        if (q < n16) dstb[q] = bb[i];
      }
    }
    if (g + 1 < nent) load_entry(g + 1);      // in flight while the MMAs run
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t dbase = tmem + ((win & 1) ? kColD1 : kColD0);
      const uint32_t abase = smem_u32(st), bbase = smem_u32(st + NSPLIT * P.apart_bytes);
      const int npr = NSPLIT == 2 ? 3 : 6;
      const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
      for (int pr = 0; pr < npr; ++pr) {
        for (int c = 0; c < P.nchunk; ++c) {
          const Chunk& C = P.ch[c];
          const uint32_t sbo_b = (uint32_t)C.ksteps * 2u * 128u;
          const uint32_t idesc = idesc_bf16(C.n);
          for (int ks = 0; ks < C.ksteps; ++ks) {
            const uint64_t ad = sdesc(abase + pa[pr] * P.apart_bytes + ks * 256, 128, sbo_a);
            const uint64_t bd = sdesc(bbase + pb[pr] * P.bpart_bytes + C.boff + ks * 256, 128, sbo_b);
            const uint32_t acc = (win_first && pr == 0 && ks == 0) ? 0u : 1u;
            umma(dbase + (uint32_t)C.n0, ad, bd, idesc, acc);
          }
        }
      }
      umma_commit(smem_u32(&bars[s]));
    }
    // the MMAs of code g - 1 must finish before stage s^1 is rewritten
    if (g >= 1) {
      ok = __syncthreads_and(mbar_wait(smem_u32(&bars[s ^ 1]), ((g - 1) >> 1) & 1, args.err));
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      if (win_first) drain<NPAD>(tq, ((win - 1) & 1) ? kColD1 : kColD0, h, win == 1);
    }
  }
  if (ok && nent > 0) {
    const int g = nent - 1;
    ok = __syncthreads_and(mbar_wait(smem_u32(&bars[g & 1]), (g >> 1) & 1, args.err));
    if (ok) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      drain<NPAD>(tq, ((g / kFlush) & 1) ? kColD1 : kColD0, h, g / kFlush == 0);
    }
  }
  // read the running sums (collective per warp), store the real rows
  if (ok) {
    const float inv_s = row_tgt >= 0 ? (float)(1.0 / args.box_cs[row_tgt].w) : 0.f;
    float* out = args.loc + ((int64_t)(row_tgt < 0 ? 0 : row_tgt) * args.ndp + d) * ms;
#pragma unroll
    for (int c = 0; c < NPAD / 2; c += 16) {
      const int col = h * (NPAD / 2) + c;
      float sh[16], sl[16];
      if (nent > 0) {
        tmem_ld16(tq + kColSH + (uint32_t)col, sh);
        tmem_ld16(tq + kColSL + (uint32_t)col, sl);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) sh[i] = sl[i] = 0.f;
      }
      if (row_tgt >= 0) {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (col + i < np) out[col + i] = (sh[i] + sl[i]) * inv_s;
      }
    }
  }
  // after a wait gave up, give the tensor pipe a bounded grace period
  if (!ok) {
    for (int s = 0; s < 2; ++s)
      for (long i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(smem_u32(&bars[s]), 0) || mbar_try_wait(smem_u32(&bars[s]), 1)) break;
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}


}  // namespace

bool m2l_tc_supported(int p, int nsplit) {
  return p >= 1 && p <= kTcMaxP && (nsplit == 2 || nsplit == 3) && make_plan(p, nsplit).smem_bytes <= 227 * 1024;
}

cudaError_t m2l_tc_prepare_tables(int p, int ncode, const double* T, int nsplit, M2LTensorTables* out, cudaStream_t st) {
  if (!m2l_tc_supported(p, nsplit)) return cudaErrorInvalidValue;
  TcPlan P = make_plan(p, nsplit);
  if (P.smem_bytes > 227 * 1024) return cudaErrorInvalidValue;
  const int np = P.np;
  std::vector<uint8_t> host((size_t)std::max(ncode, 1) * nsplit * P.bpart_bytes, 0);
  for (int code = 0; code < ncode; ++code) {
    const double* Tc = T + (size_t)code * np * np;
    for (int c = 0; c < P.nchunk; ++c) {
      const Chunk& C = P.ch[c];
      const int kext = 16 * C.ksteps;
      for (int r = 0; r < C.n; ++r)
        for (int k = 0; k < kext; ++k) {
          const int a = C.n0 + r;
          const float x = (a < np && k < np) ? (float)Tc[(size_t)a * np + k] : 0.f;
          __nv_bfloat16 parts[3];
          split_parts(x, nsplit, parts);
          for (int t = 0; t < nsplit; ++t) {
            uint8_t* base = host.data() + ((size_t)code * nsplit + t) * P.bpart_bytes + C.boff;
            std::memcpy(base + canon_off(r, k, kext), &parts[t], 2);
          }
        }
    }
  }
  void* dev = nullptr;
  cudaError_t e = cudaMalloc(&dev, host.size());
  if (e != cudaSuccess) return e;
  e = cudaMemcpyAsync(dev, host.data(), host.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) { cudaFree(dev); return e; }
  e = cudaStreamSynchronize(st);
  out->tab = dev;
  out->p = p;
  out->nsplit = nsplit;
  return e;
}

void m2l_tc_free_tables(M2LTensorTables* t) {
  if (t && t->tab) cudaFree(t->tab);
  if (t) t->tab = nullptr;
}

template <int NSPLIT, int NPAD>
static cudaError_t launch_impl(const TcArgs& a, int ntile, int ndp, cudaStream_t st) {
  auto ker = k_m2l_tc<NSPLIT, NPAD>;
  cudaError_t e = cudaFuncSetAttribute(ker, cudaFuncAttributeMaxDynamicSharedMemorySize, a.P.smem_bytes);
  if (e != cudaSuccess) return e;
  ker<<<dim3(ntile, ndp), kThreads, a.P.smem_bytes, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_m2l_tc(const DevGeom& G, const DevTaskLists& L, const M2LTensorTables& tab, int ndp,
                          const float* mom, float* loc, cudaStream_t st) {
  if (L.tc_ntile == 0) return cudaSuccess;
  TcArgs a;
  a.P = make_plan(tab.p, tab.nsplit);
  a.tile_tgt = L.tc_tile_tgt;
  a.tile_off = L.tc_tile_off;
  a.ent_code = L.tc_ent_code;
  a.ent_src = L.tc_ent_src;
  a.bparts = (const uint8_t*)tab.tab;
  a.mom = mom;
  a.loc = loc;
  a.box_cs = G.box_cs;
  a.ndp = ndp;
  a.err = L.err;
  const int npad = a.P.npad;
  if (tab.nsplit == 2) {
    switch (npad) {
      case 16: return launch_impl<2, 16>(a, L.tc_ntile, ndp, st);
      case 32: return launch_impl<2, 32>(a, L.tc_ntile, ndp, st);
      case 48: return launch_impl<2, 48>(a, L.tc_ntile, ndp, st);
      case 64: return launch_impl<2, 64>(a, L.tc_ntile, ndp, st);
      case 96: return launch_impl<2, 96>(a, L.tc_ntile, ndp, st);
      case 128: return launch_impl<2, 128>(a, L.tc_ntile, ndp, st);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (npad) {
    case 16: return launch_impl<3, 16>(a, L.tc_ntile, ndp, st);
    case 32: return launch_impl<3, 32>(a, L.tc_ntile, ndp, st);
    case 48: return launch_impl<3, 48>(a, L.tc_ntile, ndp, st);
    case 64: return launch_impl<3, 64>(a, L.tc_ntile, ndp, st);
    case 96: return launch_impl<3, 96>(a, L.tc_ntile, ndp, st);
    default: return cudaErrorInvalidValue;
  }
}

int m2l_tc_smem_bytes(int p, int nsplit) { return make_plan(p, nsplit).smem_bytes; }

}  // namespace bcfmm
