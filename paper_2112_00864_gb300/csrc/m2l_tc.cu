// Interaction phase (M2L, Sec. 3.3) on the 5th-generation tensor cores.
//
// Work unit = (tile of 128 target boxes of one level and one octant in the
// parent, a range of the interaction offsets o present in the tile, one
// density).  Per offset the unit forms
//   A[r][b] = m_{src(r,o)}^b          (M = 128 rows: targets; K: moment index b)
//   B[a][b] = T_o[a][b]               (N: local index a)
// and accumulates D = A B^T in TMEM (tcgen05.mma, kind::f16, BF16 operands,
// FP32 accumulation): D[r][a] = sum_b T_o[a][b] m^b = lambda_r^a s.
// FP32 operands are split into BF16 parts (hi + lo, or hi + mid + lo) and the
// partial products that carry the significant bits are summed
// (x2: hh + hl + lh; x3: hh + hm + mh + hl + lh + mm).  The moments are split
// once per evaluation (k_split_moments); T_o is split at setup.
// T_o[a][b] vanishes unless |a| + |b| <= p; when shared memory is short the
// N range is cut into chunks whose K extent shrinks with the degree of a.
//
// Warp roles: warp 0 (one lane) issues the MMAs; warps 1-8 fill an NS-stage
// shared-memory ring: A rows by cp.async (16-byte pieces straight into the
// operand layout), B by one cp.async.bulk per offset.  A stage is marked
// full NS-1 offsets after its copies were issued, so NS-1 offsets of memory
// latency overlap the MMAs.  D alternates between two TMEM windows of kFlush
// offsets; a finished window is added into a compensated running sum SH + SL
// (TwoSum, in TMEM) one window later, so the ~10^3-term sum of a box never
// runs through one long FP32 chain.  Each unit writes its (SH, SL) partial;
// k_m2l_unit_reduce adds the partials of a tile in a fixed order
// (deterministic) and applies the 1/s scaling.
//
// Shared-memory operands use the K-major, no-swizzle canonical layout: core
// matrices of 8 rows x 16 bytes; LBO = 128 B (next core along K), SBO =
// (K extent / 8) * 128 B (next group of 8 rows).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"
#include "m2l_tc.cuh"

namespace bcfmm {

namespace {

constexpr int kTileM = 128;
constexpr int kFlush = 4;                 // offsets per TMEM accumulation window
constexpr long kSpinLimit = 1L << 22;     // bounded waits (then error flag)
constexpr int kProducers = 256;           // warps 1..8
constexpr int kThreads = 32 + kProducers;
constexpr int kMaxMma = 256;              // entries of the MMA table
constexpr int kSmemLimit = 227 * 1024;

struct Chunk {
  int n0, n, ksteps;    // N range [n0, n0+n), K extent = 16 * ksteps
  int boff;             // byte offset of the chunk inside one B part
};

struct TcPlan {
  int p = 0, np = 0, kpad = 0, npad = 0, nchunk = 0, nsplit = 0, nstage = 0, nmma = 0;
  Chunk ch[16];
  int bpart_bytes = 0;  // one BF16 part of one offset's B (all chunks)
  int apart_bytes = 0;  // one BF16 part of A (128 rows x kpad)
  int stage_bytes = 0;
  int smem_bytes = 0;
};

struct TcArgs {
  TcPlan P;
  const int* ent_code;       // [nent] offset code
  const int* ent_src;        // [nent][128] source box (-1: none)
  const int4* units;         // [nunit] (tile, first entry, end entry, -)
  const uint8_t* bparts;     // [ncode][nsplit][bpart_bytes]
  const __nv_bfloat16* momb; // [nbox * ndp][nsplit][kpad] split moments
  float2* partial;           // [ndp][nunit][npad][128] (SH, SL)
  int nunit;
  int ndp;
  int* err;
};

int host_nterms(int p) { return p < 0 ? 0 : (p + 1) * (p + 2) * (p + 3) / 6; }

TcPlan make_plan_impl(int p, int nsplit, bool dense) {
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
  int boff = 0, kssum = 0;
  for (int n0 = 0; n0 < P.npad; n0 += 16) {
    const int ks = dense ? P.kpad / 16 : ksteps_at(n0);
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
    kssum += P.ch[c].ksteps;
  }
  P.nmma = (nsplit == 2 ? 3 : 6) * kssum;
  P.bpart_bytes = boff;
  P.apart_bytes = kTileM * P.kpad * 2;
  P.stage_bytes = nsplit * (P.apart_bytes + P.bpart_bytes);
  const int fixed = 1024 + 16 * kMaxMma + 256;     // alignment slack, MMA table, barriers + TMEM address
  P.nstage = std::min(4, (kSmemLimit - fixed) / std::max(P.stage_bytes, 1));
  P.smem_bytes = P.nstage * P.stage_bytes + fixed;
  return P;
}

// Each tcgen05.mma costs a roughly fixed issue time (measured ~70 cycles of
// the tc pipe) whatever its N, so the N range is one dense chunk with the
// full K extent (fewest instructions, padded MACs) unless its B operand
// leaves fewer than two pipeline stages; then the chunked form is used.
TcPlan make_plan(int p, int nsplit) {
  const TcPlan dense = make_plan_impl(p, nsplit, true);
  return dense.nstage >= 2 ? dense : make_plan_impl(p, nsplit, false);
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

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
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
__device__ __forceinline__ bool mbar_wait_n(uint32_t bar, uint32_t parity, int* err, long limit) {
  for (long i = 0; i < limit; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  atomicExch(err, 1);
  return false;
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err) {
  return mbar_wait_n(bar, parity, err, kSpinLimit);
}

// Test of the expiry path: one thread waits, through the same bounded
// wait, on an mbarrier whose single expected arrival never comes.
__global__ void k_debug_expire_wait(int* err, long limit) {
  __shared__ __align__(8) unsigned long long bar;
  const uint32_t b = smem_u32(&bar);
  mbar_init(b, 1);
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  mbar_wait_n(b, 0, err, limit);
}

// 1-D bulk copy global -> shared, completion counted on the mbarrier
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);   // version 1, no swizzle
}

// kind::f16 instruction descriptor: D f32, A/B bf16, both K-major, M = 128
__host__ __device__ __forceinline__ uint32_t idesc_bf16(int n) {
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

__device__ __forceinline__ void two_sum(float& hi, float& lo, float x) {
  const float s = hi + x;
  const float bb = s - hi;
  const float e = (hi - (s - bb)) + (x - bb);
  hi = s;
  lo += e;
}

// TMEM columns: two window accumulators and the compensated running sum
constexpr uint32_t kColD0 = 0, kColD1 = 128, kColSH = 256, kColSL = 384;

// ------------------------------------------------ moment split (per eval)
// momb[row][t][k] = part t of mom[row][k] (k < np), zero for np <= k < kpad
template <int NSPLIT>
__global__ void k_split_moments(const float* __restrict__ mom, int64_t nrow, int np, int ms, int kpad,
                                __nv_bfloat16* __restrict__ momb) {
  const int ng = kpad / 8;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= nrow * ng) return;
  const int64_t row = i / ng;
  const int j = (int)(i % ng);
  __nv_bfloat16 part[NSPLIT][8];
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const int k = 8 * j + q;
    const float x = k < np ? mom[row * ms + k] : 0.f;
    __nv_bfloat16 pp[3];
    split_parts(x, NSPLIT, pp);
#pragma unroll
    for (int t = 0; t < NSPLIT; ++t) part[t][q] = pp[t];
  }
#pragma unroll
  for (int t = 0; t < NSPLIT; ++t)
    *reinterpret_cast<uint4*>(momb + (row * NSPLIT + t) * kpad + 8 * j) = *reinterpret_cast<const uint4*>(part[t]);
}

// --------------------------------------------------------------- kernel
template <int NSPLIT, int NPAD, int NS>
__global__ void __launch_bounds__(kThreads, 1) k_m2l_tc(TcArgs args) {
  extern __shared__ __align__(1024) uint8_t smraw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const TcPlan& P = args.P;
  uint4* mtab = (uint4*)(sm + NS * P.stage_bytes);                 // MMA table
  uint64_t* full = (uint64_t*)(mtab + kMaxMma);                    // A rows landed (256 arrivals)
  uint64_t* bfull = full + NS;                                     // B landed (1 arrival + bytes)
  uint64_t* empty = bfull + NS;                                    // MMAs done with the stage
  uint64_t* windone = empty + NS;
  uint64_t* drained = windone + 2;
  uint32_t* tmem_holder = (uint32_t*)(drained + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int4 U = args.units[blockIdx.x];
  const int e0 = U.y, nent = U.z - U.y;
  const int d = blockIdx.y;

  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(smem_u32(&full[s]), kProducers);
      mbar_init(smem_u32(&bfull[s]), 1);
      mbar_init(smem_u32(&empty[s]), 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(smem_u32(&windone[b]), 1);
      mbar_init(smem_u32(&drained[b]), kProducers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    // MMA table, independent of the stage: A offset, B offset,
    // (first-of-chunk flag << 31 | SBO_B << 8 | D column), instruction descriptor
    int j = 0;
    const int npr = NSPLIT == 2 ? 3 : 6;
    const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
    for (int pr = 0; pr < npr; ++pr)
      for (int c = 0; c < P.nchunk; ++c)
        for (int ks = 0; ks < P.ch[c].ksteps; ++ks) {
          const uint32_t aoff = (uint32_t)(pa[pr] * P.apart_bytes + ks * 256);
          const uint32_t boff = (uint32_t)(NSPLIT * P.apart_bytes + pb[pr] * P.bpart_bytes + P.ch[c].boff + ks * 256);
          const uint32_t sbo_b = (uint32_t)P.ch[c].ksteps * 256u;
          const uint32_t first = (pr == 0 && ks == 0) ? 1u : 0u;
          mtab[j++] = make_uint4(aoff, boff, (first << 31) | (sbo_b << 8) | (uint32_t)P.ch[c].n0, idesc_bf16(P.ch[c].n));
        }
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
  const uint32_t sbo_a = (uint32_t)(P.kpad / 8) * 128u;

  if (warp == 0) {
    // ------------------------------------------------------ MMA issuer
    if (lane == 0) {
      bool ok = true;
      for (int g = 0; g < nent && ok; ++g) {
        const int s = g % NS, k = g / NS, w = g / kFlush, b = w & 1;
        const bool wfirst = (g % kFlush) == 0;
        if (wfirst && w >= 2) ok = mbar_wait(smem_u32(&drained[b]), ((w - 2) >> 1) & 1, args.err);
        if (ok) ok = mbar_wait(smem_u32(&full[s]), k & 1, args.err);
        if (ok) ok = mbar_wait(smem_u32(&bfull[s]), k & 1, args.err);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t base = smem_u32(sm + s * P.stage_bytes);
        const uint32_t dcol = tmem + (b ? kColD1 : kColD0);
        for (int j = 0; j < P.nmma; ++j) {
          const uint4 t = mtab[j];
          const uint64_t ad = sdesc(base + t.x, 128, sbo_a);
          const uint64_t bd = sdesc(base + t.y, 128, (t.z >> 8) & 0x7FFFFFu);
          const uint32_t acc = (wfirst && (t.z >> 31)) ? 0u : 1u;
          umma(dcol + (t.z & 0xFFu), ad, bd, t.w, acc);
        }
        umma_commit(smem_u32(&empty[s]));
        if ((g % kFlush) == kFlush - 1 || g == nent - 1) umma_commit(smem_u32(&windone[b]));
      }
    }
    __syncwarp();
  } else {
    // ---------------------------------------------- producers / drainers
    const int pidx = tid - 32, row = pidx & (kTileM - 1), h = pidx >> 7;
    constexpr int KG = NPAD / 16;     // 16-byte K groups per half row
    const int j0 = h * KG;
    const int row_off = (row >> 3) * (int)sbo_a + (row & 7) * 16;
    const uint32_t bbytes = (uint32_t)(NSPLIT * P.bpart_bytes);
    // drain mapping: TMEM lane quarter = warp % 4; the 16-column groups of
    // the window alternate between the two warps of a quarter (dh)
    const uint32_t tq = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const int dh = (warp - 1) >> 2;
    const int64_t rstride = (int64_t)NSPLIT * P.kpad;    // bf16 per split-moment row
    int src_cur = nent > 0 ? args.ent_src[(int64_t)e0 * kTileM + row] : -1;
    int src_nxt = nent > 1 ? args.ent_src[(int64_t)(e0 + 1) * kTileM + row] : -1;
    int code_cur = nent > 0 ? args.ent_code[e0] : 0;
    int code_nxt = nent > 1 ? args.ent_code[e0 + 1] : 0;
    bool ok = true;
    int next_drain = 0;                  // windows drained so far
    auto drain_window = [&](int wd) {    // add window wd into (SH, SL)
      bool r = mbar_wait(smem_u32(&windone[wd & 1]), (wd >> 1) & 1, args.err);
      if (!r) return false;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int gi = dh; gi < NPAD / 16; gi += 2) {      // 16-column groups, alternating halves
        const uint32_t col = (uint32_t)(gi * 16);
        float dv[16], sh[16], sl[16];
        tmem_ld16(tq + ((wd & 1) ? kColD1 : kColD0) + col, dv);
        if (wd == 0) {
#pragma unroll
          for (int i = 0; i < 16; ++i) { sh[i] = dv[i]; sl[i] = 0.f; }
        } else {
          tmem_ld16(tq + kColSH + col, sh);
          tmem_ld16(tq + kColSL + col, sl);
#pragma unroll
          for (int i = 0; i < 16; ++i) two_sum(sh[i], sl[i], dv[i]);
        }
        tmem_st16(tq + kColSH + col, sh);
        tmem_st16(tq + kColSL + col, sl);
      }
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&drained[wd & 1]));
      return true;
    };
    // entry c's rows are marked full; a finished window is drained one
    // window later (the MMAs have had a window's time to complete)
    auto mark_full = [&](int c) {
      mbar_arrive(smem_u32(&full[c % NS]));
      if ((c + 1) % kFlush == 0 && (c + 1) / kFlush >= 2) {
        const int wd = (c + 1) / kFlush - 2;
        if (wd == next_drain) { ok = drain_window(wd); ++next_drain; }
      }
    };
    for (int g = 0; g < nent && ok; ++g) {
      const int s = g % NS;
      if (g >= NS) ok = mbar_wait(smem_u32(&empty[s]), ((g / NS) - 1) & 1, args.err);
      if (!ok) break;
      uint8_t* st = sm + s * P.stage_bytes;
      const int e = e0 + g;
      if (pidx == 0) {
        mbar_arrive_tx(smem_u32(&bfull[s]), bbytes);
        bulk_g2s(smem_u32(st + NSPLIT * P.apart_bytes), args.bparts + (int64_t)code_cur * bbytes, bbytes,
                 smem_u32(&bfull[s]));
      }
      code_cur = code_nxt;
      code_nxt = (g + 2 < nent) ? args.ent_code[e + 2] : 0;
      const int src = src_cur;
      src_cur = src_nxt;
      src_nxt = (g + 2 < nent) ? args.ent_src[(int64_t)(e + 2) * kTileM + row] : -1;
      if (src >= 0) {
        const __nv_bfloat16* mrow = args.momb + ((int64_t)src * args.ndp + d) * rstride;
#pragma unroll
        for (int t = 0; t < NSPLIT; ++t)
#pragma unroll
          for (int jj = 0; jj < KG; ++jj)
            cp16(smem_u32(st + t * P.apart_bytes + row_off + (j0 + jj) * 128), mrow + t * P.kpad + 8 * (j0 + jj));
      } else {
#pragma unroll
        for (int t = 0; t < NSPLIT; ++t)
#pragma unroll
          for (int jj = 0; jj < KG; ++jj)
            *reinterpret_cast<uint4*>(st + t * P.apart_bytes + row_off + (j0 + jj) * 128) = make_uint4(0, 0, 0, 0);
      }
      cp_commit();
      const int c = g - (NS - 1);
      if (c >= 0) {
        cp_wait<NS - 1>();                         // entry c's copies have landed
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mark_full(c);
      }
    }
    if (ok && nent > 0) {
      cp_wait<0>();
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      for (int c = std::max(0, nent - (NS - 1)); c < nent && ok; ++c) mark_full(c);
    }
    // remaining windows, the last one straight into this unit's partial
    float2* out = args.partial + ((int64_t)d * args.nunit + blockIdx.x) * NPAD * kTileM;
    const int prow = (warp & 3) * 32 + lane;
    const int W = nent > 0 ? (nent - 1) / kFlush : -1;
    while (ok && next_drain < W) { ok = drain_window(next_drain); ++next_drain; }
    if (ok && nent > 0) {
      ok = mbar_wait(smem_u32(&windone[W & 1]), (W >> 1) & 1, args.err);
      if (ok) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
        for (int gi = dh; gi < NPAD / 16; gi += 2) {
          const uint32_t col = (uint32_t)(gi * 16);
          float dv[16], sh[16], sl[16];
          tmem_ld16(tq + ((W & 1) ? kColD1 : kColD0) + col, dv);
          if (W == 0) {
#pragma unroll
            for (int i = 0; i < 16; ++i) { sh[i] = dv[i]; sl[i] = 0.f; }
          } else {
            tmem_ld16(tq + kColSH + col, sh);
            tmem_ld16(tq + kColSL + col, sl);
#pragma unroll
            for (int i = 0; i < 16; ++i) two_sum(sh[i], sl[i], dv[i]);
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) out[(int64_t)(col + i) * kTileM + prow] = make_float2(sh[i], sl[i]);
        }
      }
    } else if (ok) {
      for (int gi = dh; gi < NPAD / 16; gi += 2)
        for (int i = 0; i < 16; ++i) out[(int64_t)(gi * 16 + i) * kTileM + prow] = make_float2(0.f, 0.f);
    }
    if (!ok) cp_wait<0>();               // no copy may land after the CTA exits
  }
  // free TMEM once every MMA has completed (all windows were waited on, or
  // a bounded wait gave up; then allow a bounded grace period)
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    if (lane == 0 && nent > 0) {
      const int W = (nent - 1) / kFlush;
      for (long i = 0; i < kSpinLimit; ++i)
        if (mbar_try_wait(smem_u32(&windone[W & 1]), (W >> 1) & 1)) break;
      // bulk copies in flight complete on bfull; wait for the last phase of each stage
      for (int s = 0; s < NS && s < nent; ++s) {
        const int last_use = (nent - 1 - s) / NS;     // uses of stage s: g = s, s+NS, ...
        for (long i = 0; i < kSpinLimit; ++i)
          if (mbar_try_wait(smem_u32(&bfull[s]), last_use & 1)) break;
      }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// lambda[tgt][a] = (sum over the tile's units of SH + SL) / s, in unit order
template <int NPAD>
__global__ void __launch_bounds__(kTileM) k_m2l_unit_reduce(const int* __restrict__ tile_tgt,
                                                          const int* __restrict__ tile_unit_off,
                                                          const float2* __restrict__ partial, int nunit, int ndp,
                                                          int np, int ms, const double4_32a* __restrict__ box_cs,
                                                          float* __restrict__ loc) {
  const int tile = blockIdx.x, d = blockIdx.y, row = threadIdx.x;
  const int tgt = tile_tgt[tile * kTileM + row];
  if (tgt < 0) return;
  const int u0 = tile_unit_off[tile], u1 = tile_unit_off[tile + 1];
  const float inv_s = (float)(1.0 / box_cs[tgt].w);
  float* out = loc + ((int64_t)tgt * ndp + d) * ms;
  for (int a = 0; a < np; ++a) {
    float hi = 0.f, lo = 0.f;
    for (int u = u0; u < u1; ++u) {
      const float2 v = partial[(((int64_t)d * nunit + u) * NPAD + a) * kTileM + row];
      two_sum(hi, lo, v.x);
      lo += v.y;
    }
    out[a] = (hi + lo) * inv_s;
  }
}

}  // namespace

bool m2l_tc_supported(int p, int nsplit) {
  if (p < 1 || p > kTcMaxP || (nsplit != 2 && nsplit != 3)) return false;
  const TcPlan P = make_plan(p, nsplit);
  return P.nstage >= 2 && P.nmma <= kMaxMma;
}

cudaError_t m2l_tc_prepare_tables(int p, int ncode, const double* T, int nsplit, M2LTensorTables* out, cudaStream_t st) {
  if (!m2l_tc_supported(p, nsplit)) return cudaErrorInvalidValue;
  TcPlan P = make_plan(p, nsplit);
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
  out->npad = P.npad;
  out->kpad = P.kpad;
  return e;
}

void m2l_tc_free_tables(M2LTensorTables* t) {
  if (t && t->tab) cudaFree(t->tab);
  if (t) t->tab = nullptr;
}

template <int NSPLIT, int NPAD, int NS>
static cudaError_t launch_impl(const TcArgs& a, int ndp, cudaStream_t st) {
  auto ker = k_m2l_tc<NSPLIT, NPAD, NS>;
  cudaError_t e = cudaFuncSetAttribute(ker, cudaFuncAttributeMaxDynamicSharedMemorySize, a.P.smem_bytes);
  if (e != cudaSuccess) return e;
  ker<<<dim3(a.nunit, ndp), kThreads, a.P.smem_bytes, st>>>(a);
  return cudaGetLastError();
}

template <int NSPLIT, int NPAD>
static cudaError_t launch_ns(const TcArgs& a, int ndp, cudaStream_t st) {
  switch (a.P.nstage) {
    case 2: return launch_impl<NSPLIT, NPAD, 2>(a, ndp, st);
    case 3: return launch_impl<NSPLIT, NPAD, 3>(a, ndp, st);
    default: return launch_impl<NSPLIT, NPAD, 4>(a, ndp, st);
  }
}

template <int NPAD>
static cudaError_t launch_reduce(const DevGeom& G, const DevTaskLists& L, const float2* partial, int ndp, float* loc,
                                 cudaStream_t st) {
  k_m2l_unit_reduce<NPAD><<<dim3(L.tc_ntile, ndp), kTileM, 0, st>>>(L.tc_tile_tgt, L.tc_tile_unit_off, partial,
                                                                  L.tc_nunit, ndp, G.np, G.ms, G.box_cs, loc);
  return cudaGetLastError();
}

cudaError_t launch_m2l_tc(const DevGeom& G, const DevTaskLists& L, const M2LTensorTables& tab, int ndp,
                          const float* mom, float* loc, float2* partial, void* momb, cudaStream_t st) {
  if (L.tc_nunit == 0) return cudaSuccess;
  TcArgs a;
  a.P = make_plan(tab.p, tab.nsplit);
  // split the moments of every box once
  {
    const int64_t nrow = (int64_t)G.nbox * ndp;
    const int64_t nthr = nrow * (a.P.kpad / 8);
    const unsigned nblk = (unsigned)((nthr + 255) / 256);
    if (tab.nsplit == 2)
      k_split_moments<2><<<nblk, 256, 0, st>>>(mom, nrow, G.np, G.ms, a.P.kpad, (__nv_bfloat16*)momb);
    else
      k_split_moments<3><<<nblk, 256, 0, st>>>(mom, nrow, G.np, G.ms, a.P.kpad, (__nv_bfloat16*)momb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  a.ent_code = L.tc_ent_code;
  a.ent_src = L.tc_ent_src;
  a.units = L.tc_units;
  a.bparts = (const uint8_t*)tab.tab;
  a.momb = (const __nv_bfloat16*)momb;
  a.partial = partial;
  a.nunit = L.tc_nunit;
  a.ndp = ndp;
  a.err = L.err;
  cudaError_t e = cudaErrorInvalidValue;
  if (tab.nsplit == 2) {
    switch (a.P.npad) {
      case 16: e = launch_ns<2, 16>(a, ndp, st); break;
      case 32: e = launch_ns<2, 32>(a, ndp, st); break;
      case 48: e = launch_ns<2, 48>(a, ndp, st); break;
      case 64: e = launch_ns<2, 64>(a, ndp, st); break;
      case 96: e = launch_ns<2, 96>(a, ndp, st); break;
      case 128: e = launch_ns<2, 128>(a, ndp, st); break;
      default: break;
    }
  } else {
    switch (a.P.npad) {
      case 16: e = launch_ns<3, 16>(a, ndp, st); break;
      case 32: e = launch_ns<3, 32>(a, ndp, st); break;
      case 48: e = launch_ns<3, 48>(a, ndp, st); break;
      case 64: e = launch_ns<3, 64>(a, ndp, st); break;
      case 96: e = launch_ns<3, 96>(a, ndp, st); break;
      default: break;
    }
  }
  if (e != cudaSuccess) return e;
  switch (a.P.npad) {
    case 16: return launch_reduce<16>(G, L, partial, ndp, loc, st);
    case 32: return launch_reduce<32>(G, L, partial, ndp, loc, st);
    case 48: return launch_reduce<48>(G, L, partial, ndp, loc, st);
    case 64: return launch_reduce<64>(G, L, partial, ndp, loc, st);
    case 96: return launch_reduce<96>(G, L, partial, ndp, loc, st);
    case 128: return launch_reduce<128>(G, L, partial, ndp, loc, st);
    default: return cudaErrorInvalidValue;
  }
}

int m2l_tc_smem_bytes(int p, int nsplit) { return make_plan(p, nsplit).smem_bytes; }
int m2l_tc_npad(int p) { return make_plan(p, 2).npad; }

// ------------------------------------------------ fixed scratch (no alloc)
// Unit partial sums for bcfmm_eval_noalloc: a file-scope device array, so
// that entry point needs no cudaMalloc.  Every device that loads this
// library holds it (64 MiB) until the process exits.  Calls that use it
// and overlap on the GPU race on it; each unit writes all of its entries
// before the reduce reads them, so nothing needs clearing between calls.
static __device__ __align__(256) float2 g_noalloc_partial[kNoAllocPartialElems];

namespace {
std::mutex g_noalloc_mu;
float2* g_noalloc_ptr[kNoAllocMaxDevices] = {};
}  // namespace

cudaError_t m2l_tc_noalloc_scratch(int device, float2** ptr, size_t* elems) {
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (device < 0 || device >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
  if (g_noalloc_ptr[device] == nullptr) {
    // host code only knows a stand-in for the array: ask the runtime for
    // its device address, once per device, with that device current
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partial);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[device] = static_cast<float2*>(p);
  }
  *ptr = g_noalloc_ptr[device];
  *elems = kNoAllocPartialElems;
  return cudaSuccess;
}

cudaError_t launch_debug_expire_wait(int* err, long limit, cudaStream_t st) {
  k_debug_expire_wait<<<1, 1, 0, st>>>(err, limit);
  return cudaGetLastError();
}

}  // namespace bcfmm
