// Tensor-core (tcgen05) M2L of the boundary-concentrated FMM.
#pragma once
#include <cuda_runtime.h>

#include "kernels.cuh"

namespace bcfmm {

constexpr int kTcMaxP = 7;

// Device tables of the tensor-core M2L (BF16 split parts of the box-scaled
// translation matrices, one per offset code).
struct M2LTensorTables {
  void* tab = nullptr;   // bf16 parts, layout private to m2l_tc.cu
  int p = 0, nsplit = 0, npad = 0, kpad = 0;
};

bool m2l_tc_supported(int p, int nsplit);
int m2l_tc_smem_bytes(int p, int nsplit);
cudaError_t m2l_tc_prepare_tables(int p, int ncode, const double* T /*[ncode][np][np]*/, int nsplit, M2LTensorTables* out,
                                  cudaStream_t st);
// Scratch (device memory owned by the caller):
//   partial: ndp * L.tc_nunit * npad * 128 float2 (unit partial sums)
//   momb:    nbox * ndp * nsplit * kpad BF16 (split moments)
cudaError_t launch_m2l_tc(const DevGeom& G, const DevTaskLists& L, const M2LTensorTables& tab, int ndp,
                          const float* mom, float* loc, float2* partial, void* momb, cudaStream_t st);
int m2l_tc_npad(int p);
// one bounded mbarrier wait that expires (sets *err); test of the error path
cudaError_t launch_debug_expire_wait(int* err, long limit, cudaStream_t st);

// Fixed device scratch for the unit partial sums of bcfmm_eval_noalloc
// (float2 elements); the address is looked up once per device.
constexpr size_t kNoAllocPartialElems = size_t(8) << 20;   // 64 MiB
constexpr int kNoAllocMaxDevices = 64;
cudaError_t m2l_tc_noalloc_scratch(int device, float2** ptr, size_t* elems);
void m2l_tc_free_tables(M2LTensorTables* t);

}  // namespace bcfmm
