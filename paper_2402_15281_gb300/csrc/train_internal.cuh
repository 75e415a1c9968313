// train_internal.cuh -- shared declarations of the training kernels.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>

namespace svm {

constexpr int kEpiFwd = 0, kEpiDgrad = 1, kEpiWgrad = 2;

// Arguments of one training GEMM D[M][N] = A[M][K] B[N][K]^T (bfloat16).
struct GemmArgs {
    int n_mt, n_nt, n_ks;           // tiles along M (128), N (256), K splits
    int k_len;                      // K elements per split (multiple of 64)
    int k_last;                     // K elements of the last split (multiple of 64; 0: k_len)
    long long ld_rows;              // row stride of the row-major [M][.] operands and outputs
    const float* bias;              // FWD: [N]
    const __nv_bfloat16* d_in;      // DGRAD: D = act'(z) of the previous layer
    float* dw;                      // WGRAD: FP32 partials [n_ks][M][N]
    long long split_stride;         // WGRAD: elements between the partials of two splits
    unsigned int* err;              // bounded-wait error word
};

int train_gemm_bm();
int train_gemm_bn();
int train_gemm_bk();
int train_make_map(void* map, const void* base, long long rows, long long cols, int box_rows);
int train_make_store_map(void* map, const void* base, long long rows, long long cols, int fp32);
// smap0 / smap1: tensor maps of the outputs (FWD: D, H; DGRAD: G; WGRAD: the
// FP32 partials as [n_ks * M][N])
void launch_train_gemm(int epi, int act, const void* amap, const void* bmap, const void* smap0, const void* smap1,
                       const GemmArgs& g, int n_sms, cudaStream_t s);

}  // namespace svm
