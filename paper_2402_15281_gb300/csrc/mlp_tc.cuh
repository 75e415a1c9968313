// mlp_tc.cuh -- host interface of the tcgen05 tensor-core network kernel.
#pragma once
#include "svm.h"
#include "svm_internal.cuh"

namespace svm {

constexpr int kTcMaxHidden = 8;

// Small per-layer constants of the tensor-core path, passed to the kernel as
// a __grid_constant__ parameter (constant bank): every lane of a warp reads
// the same bias entry at the same time, a broadcast from the constant cache.
struct TcConst {
    float bh[kTcMaxHidden][256];   // hidden-layer biases
    float wout[256];               // output-layer weights
    float bout;
    float wscale[kTcMaxHidden];    // FP8 weight scales
    float ascale[kTcMaxHidden];    // FP8 activation scales (input of hidden layer l)
};

// Per-model state of the tensor-core path (TMA descriptors of the weights).
struct TcModel {
    bool ready = false;
    int prec = 0;                       // SVM_BF16 or SVM_FP8_E4M3
    int act = 0;                        // SVM_RELU or SVM_SILU
    alignas(64) unsigned char wmap[128];  // CUtensorMap of the hidden weights
    alignas(64) unsigned char w1map[128]; // CUtensorMap of the padded layer-1 x-weights
    TcConst kc{};
};

int tc_tile_rows();                                    // pairs per tile
size_t tc_workspace_bytes(int n_motions);              // extra workspace per call
// used: the model's weights in blob order (after rounding); wscale, ascale:
// n_hidden FP8 scales (ignored for BF16).
int tc_prepare(TcModel& t, const svm_model_desc& d, const DevWeights& w, const float* used, const float* wscale,
               const float* ascale);
void tc_set_act_scales(TcModel& t, const float* ascale, int n);
void tc_release(TcModel& t);
int tc_launch(TcModel& t, const CallArgs& a, const DevWeights& w, int n_tiles, void* ws, int n_sms,
              cudaStream_t s);

}  // namespace svm
