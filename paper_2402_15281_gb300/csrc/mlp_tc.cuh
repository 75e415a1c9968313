// mlp_tc.cuh -- host interface of the tcgen05 tensor-core network kernel.
#pragma once
#include "svm.h"
#include "svm_internal.cuh"

namespace svm {

// Per-model state of the tensor-core path (TMA descriptors of the weights).
struct TcModel {
    bool ready = false;
    int prec = 0;                       // SVM_BF16 or SVM_FP8_E4M3
    int act = 0;                        // SVM_RELU or SVM_SILU
    int arch = 0;                       // SVM_ARCH_MLP or SVM_ARCH_BLOCKS
    alignas(64) unsigned char wmap[128];  // CUtensorMap of the hidden weights
    alignas(64) unsigned char w1map[128]; // CUtensorMap of the padded x-weights (the plain network's
                                          // layer 1; the blocks' jump inputs)
};

int tc_tile_rows();                                    // pairs per tile
size_t tc_workspace_bytes(int n_motions);              // extra workspace per call
int tc_prepare(TcModel& t, const svm_model_desc& d, const DevWeights& w);
void tc_release(TcModel& t);
int tc_launch(TcModel& t, const CallArgs& a, const DevWeights& w, int n_tiles, void* ws, int n_sms,
              cudaStream_t s);
// The block architecture (width 512, BF16, ReLU) on the tensor cores: wh is the
// blocks' h-weights, [n_hidden * 512][512] bfloat16 (outputs x inputs), followed
// by the padded x-weights, [n_hidden * 512][16] bfloat16 (the initial layer's in
// the place of block 1, then the blocks' jump x-weights), on the device.
int tc_block_prepare(TcModel& t, const svm_model_desc& d, const void* wh);
int tc_block_launch(const TcModel& t, const CallArgs& a, const DevWeights& w, int n_tiles, int grid, cudaStream_t s);

}  // namespace svm
