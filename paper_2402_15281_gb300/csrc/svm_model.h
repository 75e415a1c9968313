// svm_model.h -- the model object behind the opaque svm_model handle (host).
#pragma once
#include <cmath>
#include <string>
#include <vector>

#include "svm.h"
#include "svm_internal.cuh"
#include "mlp_tc.cuh"

// The model owns its device weights, a workspace that grows on demand, a
// pinned staging buffer for the per-call host arrays and the events that
// guard them.
struct svm_model {
    int device = 0;
    int n_sms = 0;
    int cc_major = 0, cc_minor = 0;
    svm_model_desc desc{};
    svm::RobotParams rp{};
    bool has_weights = false;
    float tau = INFINITY;
    std::vector<float> used;          // weights as used, blob order
    std::vector<float> ascales;       // FP8 activation scales
    std::vector<float> bh_host;       // hidden biases [L][W] (for the FP8 scaled copy)
    void* search_dev = nullptr;       // motion search: device result records
    void* search_host = nullptr;      // and their pinned host copy
    size_t search_cap = 0;            // records each holds
    void* d_weights = nullptr;        // one allocation for all weight arrays
    svm::DevWeights dw{};
    svm::TcModel tc{};                     // tensor-core path state (BF16 / FP8)
    void* ws = nullptr;               // workspace
    size_t ws_bytes = 0;
    void* pinned = nullptr;           // host staging for per-call arrays
    size_t pinned_bytes = 0;
    cudaEvent_t staging_done = nullptr;
    bool prof = false;
    bool prof_valid = false;
    cudaEvent_t ev[5] = {};
    unsigned int* calib_amax = nullptr;   // set only on a calibration model
    unsigned int* gate_out = nullptr;     // during svm_calibrate_gate: [2] max key and count
    float gate_cut = 0.0f;                // during svm_calibrate_gate: margin + band
    int test_stalls = 0;                   // check calls left to run with the test stall
    int tie_cap = 0;                       // tie-list entries per call (0 = all); a test hook
    std::string last_error;
};

// Per-motion bias floats of the prologue: c_m (plain MLP), or the initial
// layer's and every block's c (W each) and the final layer's scalar (blocks).
inline int cbias_stride(const svm_model_desc& d)
{
    // blocks: padded to a multiple of 4 floats, so every motion's row starts 16-byte aligned (the
    // tensor-core block kernel reads two adjacent columns' biases as one 8-byte load)
    return d.arch == SVM_ARCH_BLOCKS ? ((d.n_hidden + 1) * d.width + 1 + 3) / 4 * 4 : d.width;
}

// Segments per path of a check call's flags (1: every motion stands alone).
inline int path_len_of(uint32_t flags)
{
    return (flags & SVM_PATHS3) ? 3 : (flags & SVM_PATHS2) ? 2 : 1;
}

