// Learned near-singular correction: network shape, parameter layout,
// calibration bins and launchers (see mlp.cu).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace bcfmm {

constexpr int kMlpIn = 12, kMlpH = 64, kMlpOut = 16;
constexpr int kOffW1 = 0;
constexpr int kOffB1 = kOffW1 + kMlpH * kMlpIn;
constexpr int kOffW2 = kOffB1 + kMlpH;
constexpr int kOffB2 = kOffW2 + kMlpH * kMlpH;
constexpr int kOffW3 = kOffB2 + kMlpH;
constexpr int kOffB3 = kOffW3 + kMlpOut * kMlpH;
constexpr int kMlpParams = kOffB3 + kMlpOut;          // 6032
constexpr int kMlpBinsEta = 8, kMlpBinsGap = 4, kMlpBins = kMlpBinsEta * kMlpBinsGap;

cudaError_t launch_mlp_grad(const float* params, const float* feat, const float* qhat, const float* chat, int64_t n,
                            float* grad, float* loss, cudaStream_t st);
cudaError_t launch_mlp_adam(float* params, const float* grad, float* m1, float* m2, int step, float lr, float b1,
                            float b2, float eps, cudaStream_t st);
cudaError_t launch_mlp_predict(const float* params, const float* feat, const float* qhat, int64_t n, float* out,
                               cudaStream_t st);
// lists: [4][cap] (0 FP64 rule, 1 learned, 2 unused, 3 every near-singular pair); counts [4]
cudaError_t launch_near_classify(int task, int64_t nnz, const int* row, const int* col, const double* tgt_v,
                                 const double* src_v, int mode, const float* eps_tab, float tol, int64_t* lists,
                                 unsigned long long* counts, int64_t cap, cudaStream_t st);
cudaError_t launch_near_mlp(int task, const int64_t* sel, int64_t n, const int* row, const int* col,
                            const double* tgt_v, const double* src_v, const float* params, double* cor_val,
                            cudaStream_t st);
cudaError_t launch_pair_data(int task, const int64_t* sel, int64_t n, const int* row, const int* col,
                             const double* tgt_v, const double* src_v, float* feat, float* qhat, double* Q, int* bin,
                             int* pairs, cudaStream_t st);

cudaError_t launch_select_strided(const int64_t* list, int64_t n_list, int64_t m, int64_t* sel, cudaStream_t st);
cudaError_t launch_label_ratio(const double* C, const double* Q, int64_t n, float* chat, cudaStream_t st);

}  // namespace bcfmm
