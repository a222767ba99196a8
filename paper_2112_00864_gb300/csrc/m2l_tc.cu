// Interaction phase (M2L, Sec. 3.3) on the 5th-generation tensor cores.
//
// Entry = (tile of 128 target boxes whose level has expansion order q, one
// interaction offset o present in the tile).  Per entry the MMAs form
//   A[r][b] = m_{src(r,o)}^b          (M = 128 rows: targets; K: moment index b)
//   B[a][b] = T_o[a][b]               (N: local index a)
// and D = A B^T in TMEM (tcgen05.mma, kind::f16, BF16 operands, FP32
// accumulation): D[r][a] = sum_b T_o[a][b] m^b = lambda_r^a s.  T_o is
// nonzero only for |a| + |b| <= q.  FP32 operands are split into BF16 parts
// (hi + lo, or hi + mid + lo) and the partial products that carry the
// significant bits are summed (x2: hh + hl + lh; x3: hh + hm + mh + hl + lh + mm).
// The parts of B are stacked along N, so one MMA forms A_hi times every
// B part (orders <= 5; at order 6 the parts are separate MMAs), into
// separate column regions of the accumulator that the drain adds.
//
// Accuracy of the accumulation.  Each tcgen05.mma adds its 16 products to
// the accumulator in one step whose rounding is relative to the
// accumulator's magnitude, so every entry starts in a fresh TMEM buffer and
// issues its small terms first: the cross products, then hi*hi with the K
// blocks in descending degree (the degree-0 moments, which carry most of
// the value, come last).  A finished entry is added into a compensated
// running sum SH + SL (TwoSum, in TMEM) of its unit by the drain warps.
//
// Data movement.  The 128 A rows of an entry are gathered by cp.async
// (16-byte pieces straight into the operand layout) from the split moments
// (k_split_moments, once per evaluation); rows without a source are zero.
// B comes from a compact table that holds only the nonzeros of T_o (the
// triangle |a| + |b| <= q), loaded into registers and stored value by value
// to its place in a B buffer whose zero pattern is written once at kernel
// start.  The producers form G groups; group j takes entries j, j + G, ...
// and finishes each one on its own (copies landed, B stored, proxy fence,
// arrival), so an entry's fence never waits for another entry's copies and
// G entries are loading at any time.  The source row of every (entry, row)
// is stored in the CTA's walking order: a producer reads its rows' box
// indices with no indirection.
//
// Warp roles (416 threads, one CTA per SM, persistent): warp 0 allocates
// TMEM and one lane issues the MMAs; warps 1-8 are the producer groups,
// filling NA stages of A and NB B buffers; warps 9-12 drain ND TMEM D
// buffers (warp w reads TMEM lanes 32 (w % 4) .. + 31: one target row per
// thread).  Every wait on an mbarrier is bounded; on expiry the device error
// word is set and the CTA winds down (copies drained, MMAs completed, TMEM
// freed).
//
// Work: units (tile, entry range) of one order are dealt to persistent CTAs
// on the host (longest first to the least loaded CTA); each CTA walks its
// own sequence of (entry, unit) items, once per density.  A unit covering
// its whole tile writes lambda (times 1/s) straight into the local
// expansions; the units of a tile that was cut write (SH, SL) partials that
// k_m2l_unit_reduce adds in unit order (deterministic).
//
// Shared-memory operands use the K-major, no-swizzle canonical layout: core
// matrices of 8 rows x 16 bytes; LBO = 128 B (next core along K), SBO =
// (K extent / 8) * 128 B (next group of 8 rows).  The split parts of B are
// consecutive row blocks of one operand (each padded to brows rows).
#include <cuda_bf16.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <queue>
#include <vector>

#include "internal.h"
#include "m2l_tc.cuh"

namespace bcfmm {
namespace {

constexpr int kTileM = 128;
constexpr long kSpinLimit = 1L << 22;     // bounded waits (then error flag)
constexpr int kProducers = 256;           // warps 1..8
constexpr int kDrainers = 128;            // warps 9..12
constexpr int kThreads = 32 + kProducers + kDrainers;
constexpr int kSmemLimit = 227 * 1024;
constexpr int kMaxStages = 6;             // A stages
constexpr int kMaxB = 4;                  // B buffers (one per producer group)
constexpr int kMaxD = 4;                  // TMEM D buffers
constexpr int kMaxChunkRounds = 4;        // B chunks per producer thread (group of 64: nchunk <= 256)
constexpr int kFirst = 1 << 29, kLast = 1 << 30, kUnitMask = kFirst - 1;

struct Plan {
  int q = 0, np = 0, kpad = 0, npad = 0, kst = 0, nsplit = 0;
  int nnz = 0, nchunk = 0;                // nonzeros of T_o, 16-byte chunks of 8 per part
  bool fused = false;                     // B parts stacked along N: one MMA per A part and K step
  int brows = 0;                          // rows of one B part (>= npad) = TMEM columns between D regions
  int dwidth = 0, nd = 0, shcol = 0, slcol = 0;
  int apart = 0, bpart = 0, sa = 0, sb = 0;
  int na = 0, nb = 0, ng = 0, smem = 0;   // A stages, B buffers, producer groups
};

int host_nterms(int p) { return p < 0 ? 0 : (p + 1) * (p + 2) * (p + 3) / 6; }

int count_nnz(int q) {
  int n = 0;
  for (int d = 0; d <= q; ++d) n += (d + 1) * (d + 2) / 2 * host_nterms(q - d);
  return n;
}

Plan make_plan(int q, int nsplit) {
  Plan P;
  P.q = q;
  P.nsplit = nsplit;
  P.np = host_nterms(q);
  P.kpad = (P.np + 15) / 16 * 16;
  P.npad = P.kpad;
  P.kst = P.kpad / 16;
  P.nnz = count_nnz(q);
  P.nchunk = (P.nnz + 7) / 8;
  // stacked B parts (each padded to brows rows, so that every TMEM region
  // starts on a 32-column boundary) when two D buffers of nsplit regions plus
  // the running sum fit the 512 columns
  P.brows = (P.npad + 31) / 32 * 32;
  P.fused = 2 * nsplit * P.brows + 2 * P.brows <= 512 && nsplit * P.brows <= 256;
  if (!P.fused) P.brows = P.npad;
  P.dwidth = (P.fused ? nsplit : 1) * P.brows;
  P.nd = std::min(kMaxD, (512 - 2 * P.brows) / P.dwidth);
  P.shcol = P.nd * P.dwidth;
  P.slcol = P.shcol + P.brows;
  P.apart = kTileM * P.kpad * 2;
  P.bpart = P.brows * P.kpad * 2;
  P.sa = nsplit * P.apart;
  P.sb = nsplit * P.bpart;
  // producer groups: G groups with one B buffer each and at least G A
  // stages.  A group then only ever waits for the phase right after the one
  // it last saw complete on any barrier, which the parity form of the wait
  // requires (two phases ahead it would read an old phase as done).
  const int fixed = 1024 + 512;           // alignment slack, barriers + TMEM address
  for (int ng = 4; ng >= 2 && P.na == 0; ng -= 2)
    for (int na = kMaxStages; na >= ng; --na)
      if (na * P.sa + ng * P.sb + fixed <= kSmemLimit) {
        P.na = na;
        P.nb = ng;
        P.ng = ng;
        break;
      }
  // at least half the shared memory: one CTA per SM, so that no second CTA
  // waits for the 512 TMEM columns
  P.smem = std::max(P.na * P.sa + P.nb * P.sb + fixed, kSmemLimit / 2 + 1024);
  return P;
}

struct TcArgs {
  Plan P;
  const int* seq_src;          // [items][128]
  const int* seq_code;         // [items]
  const int* seq_u;            // [items]
  const int* seq_off;          // [ncta + 1]
  const int4* units;
  const int* tile_tgt;
  const uint4* comp;           // [ncode][nsplit][nchunk]
  const int* nz_ab;            // [nchunk * 8]
  const __nv_bfloat16* momb;   // [(nbox * ndp) * nsplit][kpitch]
  int kpitch;
  const double4_32a* box_cs;
  float* loc;
  int ms;
  float2* partial;             // [ndp][nslot][npad][128] (SH, SL)
  int nslot;
  int ndp;
  int* err;
};

// byte offset of element (row r, col k) in a K-major no-swizzle operand
// whose K extent is kext
__host__ __device__ inline int canon_off(int r, int k, int kext) {
  return (r >> 3) * (kext / 8) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

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

__device__ __forceinline__ void cp16(uint32_t dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// shared-memory matrix descriptor: K-major, no swizzle
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

#define BCFMM_LD16(A, R)                                                                                        \
  asm volatile(                                                                                                 \
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];" \
      : "=r"(R[0]), "=r"(R[1]), "=r"(R[2]), "=r"(R[3]), "=r"(R[4]), "=r"(R[5]), "=r"(R[6]), "=r"(R[7]),         \
        "=r"(R[8]), "=r"(R[9]), "=r"(R[10]), "=r"(R[11]), "=r"(R[12]), "=r"(R[13]), "=r"(R[14]), "=r"(R[15])    \
      : "r"(A))
// makes the registers of a load depend on the preceding wait (asm volatile
// statements keep their order), so no use is scheduled before it
#define BCFMM_DEP16(R)                                                                                          \
  asm volatile("" : "+r"(R[0]), "+r"(R[1]), "+r"(R[2]), "+r"(R[3]), "+r"(R[4]), "+r"(R[5]), "+r"(R[6]),        \
               "+r"(R[7]), "+r"(R[8]), "+r"(R[9]), "+r"(R[10]), "+r"(R[11]), "+r"(R[12]), "+r"(R[13]),          \
               "+r"(R[14]), "+r"(R[15]))

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

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

// ------------------------------------------------ moment split (per eval)
// momb[row * NSPLIT + t][k] = part t of mom[row][k] (k < np), zero up to kpitch
template <int NSPLIT>
__global__ void k_split_moments(const float* __restrict__ mom, int64_t nrow, int np, int ms, int kpitch,
                                __nv_bfloat16* __restrict__ momb) {
  const int ng = kpitch / 8;
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
    *reinterpret_cast<uint4*>(momb + (row * NSPLIT + t) * kpitch + 8 * j) = *reinterpret_cast<const uint4*>(part[t]);
}

// --------------------------------------------------------------- kernel
template <int NSPLIT>
__global__ void __launch_bounds__(kThreads, 1) k_m2l_tc(TcArgs args) {
  extern __shared__ __align__(1024) uint8_t smraw[];
  uint8_t* sm = (uint8_t*)(((uintptr_t)smraw + 1023) & ~(uintptr_t)1023);
  const Plan& P = args.P;
  uint8_t* sA = sm;
  uint8_t* sB = sm + P.na * P.sa;
  uint64_t* full = (uint64_t*)(sB + P.nb * P.sb);   // stage ready: A landed, B stored (one group's arrivals)
  uint64_t* aempty = full + kMaxStages;             // MMAs done with an A stage
  uint64_t* bempty = aempty + kMaxStages;           // MMAs done with a B buffer
  uint64_t* dfull = bempty + kMaxB;                 // entry's D buffer complete
  uint64_t* dempty = dfull + kMaxD;                 // D buffer drained (128 arrivals)
  uint32_t* tmem_holder = (uint32_t*)(dempty + kMaxD);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int i0 = args.seq_off[blockIdx.x], len = args.seq_off[blockIdx.x + 1] - i0;
  const int total = len * args.ndp;
  const int gsize = kProducers / P.ng;              // threads of one producer group

  if (tid == 0) {
    for (int s = 0; s < P.na; ++s) {
      mbar_init(smem_u32(&full[s]), gsize);
      mbar_init(smem_u32(&aempty[s]), 1);
    }
    for (int b = 0; b < P.nb; ++b) mbar_init(smem_u32(&bempty[b]), 1);
    for (int b = 0; b < P.nd; ++b) {
      mbar_init(smem_u32(&dfull[b]), 1);
      mbar_init(smem_u32(&dempty[b]), kDrainers);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_holder)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  } else if (warp <= 8) {
    // zero pattern of the B buffers: only the triangle's nonzeros are
    // written per entry, everything else stays zero
    const uint4 z = make_uint4(0, 0, 0, 0);
    for (int i = tid - 32; i < P.nb * P.sb / 16; i += kProducers) reinterpret_cast<uint4*>(sB)[i] = z;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_holder;
  const uint32_t sbo = (uint32_t)P.kpad * 16u;

  if (warp == 0) {
    // ------------------------------------------------------ MMA issuer
    if (lane == 0) {
      int last = -1;
      bool ok = true;
      for (int g = 0; g < total && ok; ++g) {
        const int s = g % P.na, b = g % P.nb, db = g % P.nd;
        if (g >= P.nd) ok = mbar_wait(smem_u32(&dempty[db]), ((g / P.nd) - 1) & 1, args.err);
        if (ok) ok = mbar_wait(smem_u32(&full[s]), (g / P.na) & 1, args.err);
        if (!ok) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t abase = smem_u32(sA + s * P.sa), bbase = smem_u32(sB + b * P.sb);
        const uint32_t dcol = tmem + (uint32_t)(db * P.dwidth);
        auto ad = [&](int t, int ks) { return sdesc(abase + (uint32_t)(t * P.apart + ks * 256), 128, sbo); };
        auto bd = [&](int t, int ks) { return sdesc(bbase + (uint32_t)(t * P.bpart + ks * 256), 128, sbo); };
        if (P.fused) {
          // regions of D (brows columns each): hh; the next-order terms;
          // (x3) the last.  A part t meets B parts 0 ..
          // nsplit-1-t (stacked along N).  The first MMA (the top K block
          // of A_hi against every B part) starts every region fresh.
          const int ktop = P.kst - 1;
          umma(dcol, ad(0, ktop), bd(0, ktop), idesc_bf16(NSPLIT * P.brows), 0u);
          for (int t = NSPLIT - 1; t >= 1; --t)
            for (int ks = 0; ks < P.kst; ++ks)
              umma(dcol + (uint32_t)(t * P.brows), ad(t, ks), bd(0, ks), idesc_bf16((NSPLIT - t) * P.brows), 1u);
          for (int ks = ktop - 1; ks >= 0; --ks) umma(dcol, ad(0, ks), bd(0, ks), idesc_bf16(NSPLIT * P.brows), 1u);
        } else {
          // one region: the cross products, then hi*hi with K descending
          const uint32_t id = idesc_bf16(P.npad);
          uint32_t acc = 0;
          for (int ks = 0; ks < P.kst; ++ks) {
            umma(dcol, ad(0, ks), bd(1, ks), id, acc);
            acc = 1;
            umma(dcol, ad(1, ks), bd(0, ks), id, 1u);
          }
          for (int ks = P.kst - 1; ks >= 0; --ks) umma(dcol, ad(0, ks), bd(0, ks), id, 1u);
        }
        umma_commit(smem_u32(&aempty[s]));
        umma_commit(smem_u32(&bempty[b]));
        umma_commit(smem_u32(&dfull[db]));
        last = g;
      }
      // no MMA may still run when TMEM is freed (bounded grace period)
      if (last >= 0)
        for (long i = 0; i < kSpinLimit; ++i)
          if (mbar_try_wait(smem_u32(&dfull[last % P.nd]), (last / P.nd) & 1)) break;
    }
    __syncwarp();
  } else if (warp <= 8) {
    // --------------------------------------------- producer groups (A, B)
    const int pidx = tid - 32, grp = pidx / gsize, gt = pidx % gsize;
    const int rpt = kTileM / gsize;              // rows per thread (1 or 2)
    const int KG = P.kpad / 8;                   // 16-byte K groups per row
    const int64_t rstride = (int64_t)NSPLIT * args.kpitch;
    const int nrounds = (P.nchunk + gsize - 1) / gsize;   // <= kMaxChunkRounds
    // B byte offsets (inside one part) of this thread's chunks' 8 nonzeros
    uint32_t noff[kMaxChunkRounds][4];
#pragma unroll
    for (int j = 0; j < kMaxChunkRounds; ++j)
#pragma unroll
      for (int i = 0; i < 4; ++i) noff[j][i] = 0xFFFFFFFFu;
    for (int j = 0; j < nrounds; ++j) {
      const int c = gt + j * gsize;
      if (c >= P.nchunk) continue;
      for (int i = 0; i < 8; ++i) {
        const int ab = args.nz_ab[c * 8 + i];
        const uint32_t o = ab < 0 ? 0xFFFFu : (uint32_t)canon_off(ab & 0xFFFF, ab >> 16, P.kpad);
        noff[j][i >> 1] = (noff[j][i >> 1] & ~(0xFFFFu << (16 * (i & 1)))) | (o << (16 * (i & 1)));
      }
    }
    bool ok = true;
    for (int g = grp; g < total && ok; g += P.ng) {
      const int s = g % P.na, b = g % P.nb;      // b == grp: this group's own B buffer
      const int k = i0 + g % len, d = g / len;
      // the entry's source rows and B chunks (loads in flight while waiting)
      int src[2] = {-1, -1};
#pragma unroll
      for (int u = 0; u < 2; ++u)
        if (u < rpt) src[u] = args.seq_src[(int64_t)k * kTileM + gt + u * gsize];
      const uint4* cw = args.comp + (int64_t)args.seq_code[k] * NSPLIT * P.nchunk;
      uint4 wv[NSPLIT][kMaxChunkRounds];
#pragma unroll
      for (int t = 0; t < NSPLIT; ++t)
#pragma unroll
        for (int j = 0; j < kMaxChunkRounds; ++j)
          if (j < nrounds && gt + j * gsize < P.nchunk) wv[t][j] = __ldg(cw + t * P.nchunk + gt + j * gsize);
      if (g >= P.na) ok = mbar_wait(smem_u32(&aempty[s]), ((g / P.na) - 1) & 1, args.err);
      if (!ok) break;
      // A rows
      uint8_t* st = sA + s * P.sa;
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (u >= rpt) break;
        const int row = gt + u * gsize;
        const int rowoff = (row >> 3) * (P.kpad * 16) + (row & 7) * 16;
        if (src[u] >= 0) {
          const __nv_bfloat16* mrow = args.momb + ((int64_t)src[u] * args.ndp + d) * rstride;
#pragma unroll
          for (int t = 0; t < NSPLIT; ++t)
            for (int jj = 0; jj < KG; ++jj)
              cp16(smem_u32(st + t * P.apart + rowoff + jj * 128), mrow + t * args.kpitch + 8 * jj);
        } else {
#pragma unroll
          for (int t = 0; t < NSPLIT; ++t)
            for (int jj = 0; jj < KG; ++jj)
              *reinterpret_cast<uint4*>(st + t * P.apart + rowoff + jj * 128) = make_uint4(0, 0, 0, 0);
        }
      }
      cp_commit();
      // B: its buffer's previous user (this group's previous entry) must be done
      if (g >= P.nb) ok = mbar_wait(smem_u32(&bempty[b]), ((g / P.nb) - 1) & 1, args.err);
      if (!ok) break;
      uint8_t* bb = sB + b * P.sb;
#pragma unroll
      for (int t = 0; t < NSPLIT; ++t)
#pragma unroll
        for (int j = 0; j < kMaxChunkRounds; ++j) {
          if (j >= nrounds || gt + j * gsize >= P.nchunk) continue;
          const uint32_t w[4] = {wv[t][j].x, wv[t][j].y, wv[t][j].z, wv[t][j].w};
#pragma unroll
          for (int i = 0; i < 8; ++i) {
            const uint32_t o = (noff[j][i >> 1] >> (16 * (i & 1))) & 0xFFFFu;
            if (o != 0xFFFFu) *reinterpret_cast<uint16_t*>(bb + t * P.bpart + o) = (uint16_t)(w[i >> 1] >> (16 * (i & 1)));
          }
        }
      cp_wait_all();                             // this thread's rows of the entry have landed
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_arrive(smem_u32(&full[s]));
    }
    cp_wait_all();                               // no copy may land after the CTA exits
  } else {
    // ------------------------------------------------------- drainers
    const int qd = warp & 3, row = qd * 32 + lane;
    const uint32_t tq = tmem + ((uint32_t)(qd * 32) << 16);
    const int ngrp = P.npad / 16;
    const int nreg = P.fused ? NSPLIT : 1;
    for (int g = 0; g < total; ++g) {
      const int k = i0 + g % len, d = g / len, db = g % P.nd;
      const int uf = args.seq_u[k];
      const bool first = (uf & kFirst) != 0, last = (uf & kLast) != 0;
      // one lane polls; the warp stays converged for the aligned TMEM accesses
      int okw = 1;
      if (lane == 0) okw = mbar_wait(smem_u32(&dfull[db]), (g / P.nd) & 1, args.err) ? 1 : 0;
      okw = __shfl_sync(0xffffffffu, okw, 0);
      if (!okw) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      float* lout = nullptr;
      float2* pout = nullptr;
      float inv_s = 0.f;
      if (last) {
        const int4 U = args.units[uf & kUnitMask];
        if (U.w < 0) {
          const int tgt = args.tile_tgt[U.x * kTileM + row];
          if (tgt >= 0) {
            lout = args.loc + ((int64_t)tgt * args.ndp + d) * args.ms;
            inv_s = (float)(1.0 / args.box_cs[tgt].w);
          }
        } else {
          pout = args.partial + ((int64_t)d * args.nslot + U.w) * P.npad * kTileM + row;
        }
      }
      const uint32_t dcol = tq + (uint32_t)(db * P.dwidth);
      for (int gi = 0; gi < ngrp; ++gi) {
        const uint32_t col = (uint32_t)(gi * 16);
        uint32_t r0[16], r1[16], r2[16], rh[16], rl[16];
        BCFMM_LD16(dcol + col, r0);
        if (nreg > 1) BCFMM_LD16(dcol + (uint32_t)P.brows + col, r1);
        if (nreg > 2) BCFMM_LD16(dcol + (uint32_t)(2 * P.brows) + col, r2);
        if (!first) {
          BCFMM_LD16(tq + (uint32_t)P.shcol + col, rh);
          BCFMM_LD16(tq + (uint32_t)P.slcol + col, rl);
        }
        tmem_wait_ld();
        BCFMM_DEP16(r0);
        if (nreg > 1) BCFMM_DEP16(r1);
        if (nreg > 2) BCFMM_DEP16(r2);
        if (!first) {
          BCFMM_DEP16(rh);
          BCFMM_DEP16(rl);
        }
        float sh[16], sl[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          // the entry's value: smaller regions first
          float v = 0.f;
          if (nreg > 2) v = __uint_as_float(r2[i]);
          if (nreg > 1) v += __uint_as_float(r1[i]);
          v += __uint_as_float(r0[i]);
          if (first) {
            sh[i] = v;
            sl[i] = 0.f;
          } else {
            sh[i] = __uint_as_float(rh[i]);
            sl[i] = __uint_as_float(rl[i]);
            two_sum(sh[i], sl[i], v);
          }
        }
        if (!last) {
          tmem_st16(tq + (uint32_t)P.shcol + col, sh);
          tmem_st16(tq + (uint32_t)P.slcol + col, sl);
        } else if (lout) {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if ((int)col + i < P.np) lout[col + i] = (sh[i] + sl[i]) * inv_s;
        } else if (pout) {
#pragma unroll
          for (int i = 0; i < 16; ++i) pout[(int64_t)(col + i) * kTileM] = make_float2(sh[i], sl[i]);
        }
      }
      if (!last) asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(smem_u32(&dempty[db]));
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// lambda[tgt][a] = (sum over the tile's units of SH + SL) / s, in unit order
__global__ void __launch_bounds__(kTileM) k_m2l_unit_reduce(const int4* __restrict__ splits,
                                                          const int* __restrict__ tile_tgt,
                                                          const float2* __restrict__ partial, int nslot, int npad,
                                                          int ndp, int np, int ms,
                                                          const double4_32a* __restrict__ box_cs,
                                                          float* __restrict__ loc) {
  const int4 S = splits[blockIdx.x];
  const int d = blockIdx.y, row = threadIdx.x;
  const int tgt = tile_tgt[S.x * kTileM + row];
  if (tgt < 0) return;
  const float inv_s = (float)(1.0 / box_cs[tgt].w);
  float* out = loc + ((int64_t)tgt * ndp + d) * ms;
  for (int a = 0; a < np; ++a) {
    float hi = 0.f, lo = 0.f;
    for (int u = 0; u < S.z; ++u) {
      const float2 v = partial[(((int64_t)d * nslot + S.y + u) * npad + a) * kTileM + row];
      two_sum(hi, lo, v.x);
      lo += v.y;
    }
    out[a] = (hi + lo) * inv_s;
  }
}

}  // namespace

bool m2l_tc_supported(int q, int nsplit) {
  if (q < 1 || (nsplit != 2 && nsplit != 3) || q > tc_max_order(nsplit)) return false;
  const Plan P = make_plan(q, nsplit);
  const int gsize = kProducers / P.ng;
  return P.nd >= 2 && P.na >= 2 && (P.nchunk + gsize - 1) / gsize <= kMaxChunkRounds;
}

int m2l_tc_npad(int q) { return make_plan(q, 2).npad; }

int m2l_tc_kpitch(int p) { return (host_nterms(p) + 15) / 16 * 16; }

void m2l_tc_schedule(const std::vector<int>& tile_off, const std::vector<int>& tile_q, const std::vector<int>& ent_src,
                     int nsm, int nsplit, int unit_entries, std::vector<TcOrderSchedHost>& out) {
  out.clear();
  const int ntile = (int)tile_q.size();
  for (int q = 1; q <= kTcMaxQ; ++q) {
    std::vector<int> tiles;
    int64_t E = 0;
    for (int tl = 0; tl < ntile; ++tl)
      if (tile_q[tl] == q && tile_off[tl + 1] > tile_off[tl]) {
        tiles.push_back(tl);
        E += tile_off[tl + 1] - tile_off[tl];
      }
    if (tiles.empty()) continue;
    TcOrderSchedHost O;
    O.q = q;
    O.nent = E;
    for (int tl : tiles)
      for (int64_t i = (int64_t)tile_off[tl] * kTileM; i < (int64_t)tile_off[tl + 1] * kTileM; ++i) O.rows += ent_src[i] >= 0;
    // entries per unit: about three units per SM (load balance), so that
    // small launches spread over the GPU and large tiles are cut
    const int U = unit_entries > 0 ? unit_entries
                                   : (int)std::max<int64_t>(8, (E + 3 * (int64_t)nsm - 1) / (3 * (int64_t)nsm));
    for (int tl : tiles) {
      const int a = tile_off[tl], b = tile_off[tl + 1], n = b - a;
      const int k = (n + U - 1) / U;
      const int per = (n + k - 1) / k;
      if (k == 1) {
        O.units.push_back(make_int4(tl, a, b, -1));
      } else {
        O.splits.push_back(make_int4(tl, O.nslot, k, 0));
        for (int x = a, u = 0; x < b; x += per, ++u) O.units.push_back(make_int4(tl, x, std::min(b, x + per), O.nslot + u));
        O.nslot += k;
      }
    }
    // longest unit first to the least loaded CTA
    const int nu = (int)O.units.size();
    const int ncta = std::min(nsm, nu);
    std::vector<int> ord(nu);
    for (int i = 0; i < nu; ++i) ord[i] = i;
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) {
      return O.units[x].z - O.units[x].y > O.units[y].z - O.units[y].y;
    });
    using LoadCta = std::pair<int64_t, int>;
    std::priority_queue<LoadCta, std::vector<LoadCta>, std::greater<LoadCta>> pq;
    for (int c = 0; c < ncta; ++c) pq.push({0, c});
    std::vector<std::vector<int>> lists(ncta);
    for (int u : ord) {
      auto [ld, c] = pq.top();
      pq.pop();
      lists[c].push_back(u);
      pq.push({ld + O.units[u].z - O.units[u].y, c});
    }
    O.seq_off.assign(1, 0);
    for (int c = 0; c < ncta; ++c) {
      for (int u : lists[c]) {
        const int4 Un = O.units[u];
        for (int e = Un.y; e < Un.z; ++e) {
          O.seq_e.push_back(e);
          O.seq_u.push_back(u | (e == Un.y ? kFirst : 0) | (e == Un.z - 1 ? kLast : 0));
        }
      }
      O.seq_off.push_back((int)O.seq_e.size());
    }
    out.push_back(std::move(O));
  }
}

cudaError_t m2l_tc_prepare_tables(int p, int ncode, const double* T, int nsplit, const std::vector<int>& orders,
                                  M2LTensorTables* out, cudaStream_t st) {
  out->p = p;
  out->nsplit = nsplit;
  out->ncode = ncode;
  const int np = host_nterms(p);
  MultiIndex M;
  M.init(p);
  for (int q : orders) {
    if (!m2l_tc_supported(q, nsplit) || q > p || out->used[q]) continue;
    const Plan P = make_plan(q, nsplit);
    // nonzeros of the order-q triangle |a| + |b| <= q, row by row
    std::vector<int> ab;
    for (int a = 0; a < P.np; ++a) {
      const int da = M.a[a] + M.b[a] + M.c[a];
      for (int b = 0; b < host_nterms(q - da); ++b) ab.push_back(a | (b << 16));
    }
    ab.resize((size_t)P.nchunk * 8, -1);
    // [code][part][chunk]: 8 BF16 values per 16-byte chunk
    std::vector<uint16_t> comp((size_t)std::max(ncode, 1) * nsplit * P.nchunk * 8, 0);
    for (int code = 0; code < ncode; ++code)
      for (int n = 0; n < P.nnz; ++n) {
        const int a = ab[n] & 0xFFFF, b = ab[n] >> 16;
        __nv_bfloat16 parts[3];
        split_parts((float)T[((size_t)code * np + a) * np + b], nsplit, parts);
        for (int t = 0; t < nsplit; ++t)
          std::memcpy(&comp[(((size_t)code * nsplit + t) * P.nchunk) * 8 + n], &parts[t], 2);
      }
    void *dcomp = nullptr, *dab = nullptr;
    cudaError_t e = cudaMalloc(&dcomp, comp.size() * 2);
    if (e != cudaSuccess) return e;
    out->owned.push_back(dcomp);
    e = cudaMalloc(&dab, ab.size() * 4);
    if (e != cudaSuccess) return e;
    out->owned.push_back(dab);
    e = cudaMemcpyAsync(dcomp, comp.data(), comp.size() * 2, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dab, ab.data(), ab.size() * 4, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    out->used[q] = true;
    out->ord[q].nchunk = P.nchunk;
    out->ord[q].comp = static_cast<const uint4*>(dcomp);
    out->ord[q].nz_ab = static_cast<const int*>(dab);
  }
  return cudaSuccess;
}

void m2l_tc_free_tables(M2LTensorTables* t) {
  if (!t) return;
  for (void* p : t->owned) cudaFree(p);
  t->owned.clear();
  for (int q = 0; q <= kTcMaxQ; ++q) { t->used[q] = false; t->ord[q] = TcOrderTables(); }
}

cudaError_t launch_m2l_tc(const DevGeom& G, const DevTaskLists& L, const TcTaskSched& S, const M2LTensorTables& tab,
                          int ndp, const float* mom, float* loc, float2* partial, void* momb, cudaStream_t st) {
  bool any = false;
  for (int q = 1; q <= kTcMaxQ; ++q) any = any || S.ord[q].nunit > 0;
  if (!any) return cudaSuccess;
  const int nsplit = tab.nsplit;
  const int kpitch = m2l_tc_kpitch(G.p);
  // split the moments of every box once (order p: every level's order fits)
  {
    const int64_t nrow = (int64_t)G.nbox * ndp;
    const int64_t nthr = nrow * (kpitch / 8);
    const unsigned nblk = (unsigned)((nthr + 255) / 256);
    if (nsplit == 2)
      k_split_moments<2><<<nblk, 256, 0, st>>>(mom, nrow, G.np, G.ms, kpitch, (__nv_bfloat16*)momb);
    else
      k_split_moments<3><<<nblk, 256, 0, st>>>(mom, nrow, G.np, G.ms, kpitch, (__nv_bfloat16*)momb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  for (int q = 1; q <= kTcMaxQ; ++q) {
    const TcOrderSched& O = S.ord[q];
    if (O.nunit == 0) continue;
    if (!tab.used[q]) return cudaErrorInvalidValue;
    TcArgs a;
    a.P = make_plan(q, nsplit);
    if (a.P.na < 2 || a.P.nd < 2 || (a.P.nchunk + kProducers / a.P.ng - 1) / (kProducers / a.P.ng) > kMaxChunkRounds)
      return cudaErrorInvalidValue;
    a.seq_src = O.seq_src;
    a.seq_code = O.seq_code;
    a.seq_u = O.seq_u;
    a.seq_off = O.seq_off;
    a.units = O.units;
    a.tile_tgt = L.tc_tile_tgt;
    a.comp = tab.ord[q].comp;
    a.nz_ab = tab.ord[q].nz_ab;
    a.momb = (const __nv_bfloat16*)momb;
    a.kpitch = kpitch;
    a.box_cs = G.box_cs;
    a.loc = loc;
    a.ms = G.ms;
    a.partial = partial;
    a.nslot = O.nslot;
    a.ndp = ndp;
    a.err = L.err;
    cudaError_t e;
    if (nsplit == 2) {
      e = cudaFuncSetAttribute(k_m2l_tc<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, a.P.smem);
      if (e == cudaSuccess) k_m2l_tc<2><<<O.ncta, kThreads, a.P.smem, st>>>(a);
    } else {
      e = cudaFuncSetAttribute(k_m2l_tc<3>, cudaFuncAttributeMaxDynamicSharedMemorySize, a.P.smem);
      if (e == cudaSuccess) k_m2l_tc<3><<<O.ncta, kThreads, a.P.smem, st>>>(a);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (O.nsplit_tiles > 0) {
      k_m2l_unit_reduce<<<dim3(O.nsplit_tiles, ndp), kTileM, 0, st>>>(O.splits, L.tc_tile_tgt, partial, O.nslot,
                                                                       a.P.npad, ndp, a.P.np, G.ms, G.box_cs, loc);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

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

