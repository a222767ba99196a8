// CUDA-core M2L of the boundary-concentrated FMM in the Taylor-coefficient
// form (FP32 products, compensated sums over work chunks).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "kernels.cuh"

namespace bcfmm {

// Largest order handled by the register-blocked kernel (higher orders, up
// to 12, go to a one-CTA-per-target kernel in the same Taylor form).
constexpr int kTaylorMaxQ = 7;

// The expansion coefficients of Sec. 3.3,
//   lambda^a = sum_{|b| <= q - |a|} D^{a+b} G(o) / (a! b!) (-1)^{|b|} m^b,
// depend on the offset o only through the derivatives D^gamma G(o),
// |gamma| <= q: with prescaled moments m'_b = (-1)^{|b|} m^b / b! and
// g_o[gamma] = D^gamma G(o) = D^gamma (1/r)(o) / (4 pi),
//   lambda^a = (1/a!) sum_b g_o[a + b] m'_b,
// so one offset needs nterms(q) numbers instead of an nterms(q)^2 matrix,
// and the product costs one FMA per (a, b) with |a| + |b| <= q.  (Box-
// scaled expansions: o is the integer offset in units of the box side s,
// and the stored local is lambda / s.)
//
// Work of one order: the interaction list of every target of that order is
// cut into chunks of at most `chunk` entries; the chunks, longest first, are
// dealt 32 to a warp (one per lane), and the lane's entries are interleaved
// with its warp's others (entry j of lane l at pk[first + 32 j + l]) so that
// every index load is one coalesced line.  A chunk's FP32 sum goes to its
// own partial slot; a second kernel adds a target's slots in chunk order
// (compensated FP32 sum, deterministic) and stores the local expansion.
struct TaylorOrderSched {
  int q = 0, nwarp = 0, nchunk = 0, ntgt = 0, chunk = 0;
  int64_t pairs = 0;
  const int2* wb = nullptr;          // [nwarp] (first pk index, entries per lane)
  const int* lane_chunk = nullptr;   // [nwarp * 32] chunk of each lane (-1: none)
  const uint32_t* pk = nullptr;      // source box << cbits | offset code; ~0u: no entry
  const int* tgt = nullptr;          // [ntgt] target boxes
  const int* tchunk = nullptr;       // [ntgt + 1] chunk range of each target
};
struct TaylorTaskSched {
  TaylorOrderSched ord[kTaylorMaxQ + 1];   // index = order q (nwarp 0: none)
  int cbits = 0;                           // bits of the offset code in pk
  size_t partial_per_dens = 0;             // floats of chunk partial sums per density
  const int* simt_sel = nullptr;           // targets (indices into the task's list) of
  int nsimt = 0;                           // higher orders: one CTA per target
};

// Host side of one order's schedule (built at setup, uploaded by the caller).
struct TaylorOrderHost {
  int q = 0, nchunk = 0, chunk = 0;
  int64_t pairs = 0;
  std::vector<int2> wb;
  std::vector<int> lane_chunk, tgt, tchunk;
  std::vector<uint32_t> pk;
};
// target_q[k]: order of the task's k-th M2L target.  Orders 1..kTaylorMaxQ
// are scheduled; `sel` receives the targets of every other order.  Returns
// false when box and code indices do not fit the 32-bit packing.
bool m2l_taylor_schedule(const std::vector<int>& m2l_tgt, const std::vector<int>& vl_off,
                         const std::vector<int>& vl_src, const std::vector<uint16_t>& vl_code,
                         const std::vector<int>& target_q, int nbox, int ncode, int nsm,
                         std::vector<TaylorOrderHost>& out, std::vector<int>& sel, int* cbits);

// Offset coefficients g_o (FP32, [ncode][gpitch], |gamma| <= q) and the
// multi-index factors fac[0..gpitch) = (-1)^{|b|} / b! (moments),
// fac[gpitch..2 gpitch) = 1 / a! (locals).
struct TaylorTables {
  const float* g = nullptr;
  const float* fac = nullptr;
  int gpitch = 0, q = 0;
};
// row pitch (floats, a multiple of 8: rows are read as 32-byte pieces) of
// the prescaled moments and of g for order q
int m2l_taylor_pitch(int q);

// Scratch (device memory owned by the caller):
//   momp:    nbox * ndp * m2l_taylor_pitch(tab.q) floats (prescaled moments)
//   partial: ndp * S.partial_per_dens floats (chunk sums)
// tab.q must be the largest order of any target (the wide kernel reads the
// g rows and moments up to it); targets in S.simt_sel use the wide kernel.
cudaError_t launch_m2l_taylor(const DevGeom& G, const DevTaskLists& L, const TaylorTaskSched& S,
                              const TaylorTables& tab, int ndp, const float* mom, float* loc, float* momp,
                              float* partial, cudaStream_t st);

}  // namespace bcfmm
