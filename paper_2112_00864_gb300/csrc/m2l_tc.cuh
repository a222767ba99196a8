// Tensor-core (tcgen05) M2L of the boundary-concentrated FMM.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <vector>

#include "kernels.cuh"

namespace bcfmm {

constexpr int kTcMaxQ = 6;     // largest order on the tensor cores with the 2-term split
constexpr int kTcMaxQ3 = 5;    // with the 3-term split
inline int tc_max_order(int nsplit) { return nsplit == 3 ? kTcMaxQ3 : kTcMaxQ; }

// Device tables of the tensor-core M2L for one expansion order q: the
// nonzero entries (|alpha| + |beta| <= q) of every offset's box-scaled
// translation matrix, split into BF16 parts, plus where each nonzero goes
// in the MMA's B operand.
struct TcOrderTables {
  int nchunk = 0;                  // 16-byte chunks of 8 nonzeros per part
  const uint4* comp = nullptr;     // [ncode][nsplit][nchunk]
  const int* nz_ab = nullptr;      // [nchunk * 8] alpha | beta << 16 (multi-index positions; -1 pad)
};
struct M2LTensorTables {
  int p = 0, nsplit = 0, ncode = 0;
  bool used[kTcMaxQ + 1] = {};
  TcOrderTables ord[kTcMaxQ + 1];  // index = order q
  std::vector<void*> owned;        // device allocations
};

// Work of one order: units = (tile, entry range), dealt to persistent CTAs
// (longest first to the least loaded); every CTA walks its own sequence of
// (entry, unit) items.  A tile cut into several units writes per-unit
// partial sums that k_m2l_unit_reduce adds in unit order.
struct TcOrderSched {
  int q = 0, ncta = 0, nunit = 0, nslot = 0, nsplit_tiles = 0;
  int64_t nent = 0, rows = 0;      // (tile, offset) entries, filled rows (box pairs)
  const int4* units = nullptr;     // [nunit] (tile, first entry, end entry, partial slot or -1)
  const int* seq_src = nullptr;    // [items][128] source box of every row of the item's entry (-1: none)
  const int* seq_code = nullptr;   // [items] offset code of the item's entry
  const int* seq_u = nullptr;      // [items] unit | first-of-unit << 29 | last-of-unit << 30
  const int* seq_off = nullptr;    // [ncta + 1]
  const int4* splits = nullptr;    // [nsplit_tiles] (tile, first slot, slots, -)
};
struct TcTaskSched {
  TcOrderSched ord[kTcMaxQ + 1];   // index = order q (nunit 0: no tiles of that order)
  size_t partial_per_dens = 0;     // float2 elements of partial sums per density
  const int* simt_sel = nullptr;   // M2L targets (indices into the task's list) whose order the
  int nsimt = 0;                   // tensor cores do not take: CUDA-core M2L
};

// Host side of the schedule (built at setup, uploaded by the caller).
struct TcOrderSchedHost {
  int q = 0, nslot = 0;
  int64_t nent = 0, rows = 0;
  std::vector<int4> units, splits;
  std::vector<int> seq_e, seq_u, seq_off;
};
// tile_off [ntile+1] entry ranges, tile_q [ntile] orders, ent_src [nent][128].
// unit_entries > 0 fixes the entries per unit; 0 chooses it per order so
// that every SM gets about three units' worth of work.
void m2l_tc_schedule(const std::vector<int>& tile_off, const std::vector<int>& tile_q, const std::vector<int>& ent_src,
                     int nsm, int nsplit, int unit_entries, std::vector<TcOrderSchedHost>& out);

bool m2l_tc_supported(int q, int nsplit);
int m2l_tc_npad(int q);
// columns of a split-moment row (the K extent of order p, a multiple of 16)
int m2l_tc_kpitch(int p);
// Tables for every order in `orders` (T: [ncode][np][np] FP64 at order p).
cudaError_t m2l_tc_prepare_tables(int p, int ncode, const double* T, int nsplit, const std::vector<int>& orders,
                                  M2LTensorTables* out, cudaStream_t st);
void m2l_tc_free_tables(M2LTensorTables* t);

// Scratch (device memory owned by the caller):
//   partial: ndp * sched.partial_per_dens float2 (unit partial sums)
//   momb:    nbox * ndp * nsplit * kpitch BF16 (split moments)
cudaError_t launch_m2l_tc(const DevGeom& G, const DevTaskLists& L, const TcTaskSched& S, const M2LTensorTables& tab,
                          int ndp, const float* mom, float* loc, float2* partial, void* momb, cudaStream_t st);
// one bounded mbarrier wait that expires (sets *err); test of the error path
cudaError_t launch_debug_expire_wait(int* err, long limit, cudaStream_t st);

// Fixed device scratch for the unit partial sums of bcfmm_eval_noalloc
// (float2 elements); the address is looked up once per device.
constexpr size_t kNoAllocPartialElems = size_t(8) << 20;   // 64 MiB
constexpr int kNoAllocMaxDevices = 64;
cudaError_t m2l_tc_noalloc_scratch(int device, float2** ptr, size_t* elems);

}  // namespace bcfmm
