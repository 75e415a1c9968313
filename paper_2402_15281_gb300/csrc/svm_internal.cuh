// svm_internal.cuh -- device-side data layout shared by the kernels of libsvm.
//
// HBM layout of one check call (all owned by the model's workspace):
//   q0, q1        [M][6] double     motion end configurations
//   pbeg, pend    [M] int64         point range of motion m in the point array
//   tile_off      [M+1] int32       prefix of MLP tiles (one motion per tile)
//   pair_off      [M+1] int64       prefix of point counts: motion m's flagged
//                                   indices live at idx[pair_off[m] ...]
//   caps          [M][N+1][7] Capsule   FP32 capsule table (from FP64 FK)
//   cbias         [M][W] float      per-motion first-layer bias c_m
//   st            [M] MotionState   counters and running minima
//   idx           [sum P_m] uint32  flagged point indices (compaction)
//   chunk_off     [M+1] int32       verifier work prefix (written on device)
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

namespace svm {

// A named NVTX range on the host timeline for the life of a scope: profilers
// (ncu --nvtx) attribute the kernels launched inside it to the call or phase.
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

constexpr int kDof = 6;
constexpr int kCaps = 7;
constexpr int kInDim = 15;
constexpr int kMaxSteps = 900;        // capsule table of one motion fits in shared memory
constexpr float kAmbiguousBand = 4e-6f;
constexpr int kTieCap = 16384;        // pairs per call whose verdict is re-decided in FP64

// A (motion, point) pair whose FP32 distance fell within kAmbiguousBand of the
// margin; the verifier defers it to the FP64 tie kernel.
struct TiePair {
    int m;
    int pad;
    long long p;
};
inline size_t tie_list_bytes() { return (size_t)kTieCap * sizeof(TiePair); }

// One capsule at one sample: a = start point, r = radius; e = b - a and
// inv_ee = 1 / |e|^2 (0 for a zero-length axis, which makes it a sphere).
struct __align__(16) Capsule {
    float4 a_r;    // a.x, a.y, a.z, r
    float4 e_inv;  // e.x, e.y, e.z, inv_ee
};

// Per-motion device state, reset by the prologue of every call.
struct MotionState {
    unsigned int n_flagged;     // compaction counter (append position)
    int collided;               // 0 / 1, set by the verifier
    unsigned int dmin_key;      // ordered encoding of the exact minimum
    unsigned int dhat_key;      // ordered encoding of the network minimum
    unsigned int n_verified;
    int witness_point;
    int witness_step;
    unsigned int n_ambiguous;
    unsigned long long probe_key;   // (float_key(f) << 32) | point index of the motion's
                                    // smallest flagged prediction; ~0 if none
    unsigned int inexact;           // 1 if a pair of this motion at the margin found the tie
                                    // list full and was decided in FP32
    unsigned int pad;
};

// Order-preserving float <-> uint32 map: unsigned comparison of keys equals
// float comparison of values (for non-NaN values).
__device__ __forceinline__ unsigned int float_key(float f) {
    unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(unsigned int k) {
    unsigned int u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
    return __uint_as_float(u);
}

// Robot geometry (FP64 kinematics; FP32 radii for the capsule tables, FP64
// radii for the re-check of pairs at the margin).
struct RobotParams {
    double d[kDof], a[kDof], ca[kDof], sa[kDof], th0[kDof];
    double tool_len;
    float radius[kCaps];
    double radius64[kCaps];
};

// Everything a kernel of one call needs, passed by value.
struct CallArgs {
    int M;              // motions
    int N;              // steps (N+1 samples)
    int W;              // network width
    int L;              // hidden layers
    int act;            // 0 relu, 1 silu
    int arch;           // 0 plain MLP, 1 block architecture
    int cb_stride;      // per-motion bias floats: W (arch 0), (L + 1) W + 1 rounded up to a multiple of 4 (arch 1)
    uint32_t flags;
    float margin;
    float gate;         // margin + tau
    const double* q0;
    const double* q1;
    const long long* pbeg;
    const long long* pend;
    const int* tile_off;
    const long long* pair_off;
    const float4* points;
    Capsule* caps;
    float* cbias;
    MotionState* st;
    unsigned int* idx;
    int* chunk_off;
    float* f_out;       // optional per-pair network output (eval mode)
    long long f_stride; // row stride of f_out (points per motion row)
    int path_len;       // segments per path: 1 (single motions), 2 or 3
    unsigned int* dev_err;  // per-call error word: nonzero if a bounded wait expired
    unsigned int* amax;     // optional [L]: bit patterns of max |input of hidden layer l| (calibration)
    int test_stall;         // test hook: CTA 0 withholds its first layer-0 hand-over, so that
                            // the MMA warp's bounded wait expires (tensor-core path)
    RobotParams rp;         // robot (FP64 re-check of pairs at the margin)
    double* fk64;           // [M][N+1][8][3]: joint origins o_0..o_6 and tool axis of every sample, FP64
    unsigned int* tie_count;    // pairs appended to tie_list (reset by the prologue)
    TiePair* tie_list;          // [kTieCap] pairs deferred to the FP64 tie kernel
    int tie_cap;                // list entries used, 1..kTieCap (0 = kTieCap); lowered by a test hook
};

// Entries of the tie list a call may use.
__device__ __forceinline__ unsigned tie_capacity(const CallArgs& A) {
    return (A.tie_cap > 0 && A.tie_cap < kTieCap) ? (unsigned)A.tie_cap : (unsigned)kTieCap;
}

// Model weights on the device.  FP32 copies are always present; the layer-1
// and output weights hold the values of the model precision (BF16-rounded in
// the BF16 and FP8 modes).
struct DevWeights {
    const float* w1x;     // [W][3]    layer-1 weights of x, y, z
    const float* w1q;     // [W][12]   layer-1 weights of q0, q1
    const float* b1;      // [W]
    const float* wT;      // [L][W in][W out]  hidden weights, transposed (FP32 path)
    const float* bh;      // [L][W]
    const float* wout;    // [W]
    float bout;
    const void* wq;       // [L][W out][W in] BF16 or E4M3 hidden weights (tensor path)
    const void* w1pad;    // [W][64] BF16 layer-1 x-weights for the tensor path: row o is
                          // (w_ox, w_oy, w_oz, w_ox, w_oy, w_oz, 0, ...), applied to
                          // (x_hi, y_hi, z_hi, x_lo, y_lo, z_lo, 0, ...)
    const float* wscale;  // [L] per-layer weight scale (FP8), else 1
    const float* ascale;  // [L] per-layer activation scale (FP8), else 1
    const float* bhs;     // FP8: [L][W] hidden biases divided by the next layer's
                          // activation scale (b_l / ascale[l], l < L-1)
    // block architecture (arch 1): L blocks
    const float* blk_wx;  // [L][W][3]   jump weights of x, y, z (block 1: zero)
    const float* blk_wq;  // [L+1][W][12] weights of q0, q1: initial layer, then blocks
    const float* blk_b;   // [L+1][W]    biases: initial layer, then blocks
    const float* blk_s;   // [L][W]      folded BatchNorm scale gamma / sqrt(var + eps)
    const float* blk_t;   // [L][W]      folded BatchNorm shift beta - mean * scale
    const float* blk_pk;  // [L][W/2][4] per column pair (c, c+1) of block l: s_c, s_c+1, t_c, t_c+1 --
                          // one 16-byte load in the tensor-core block kernel's epilogue
    const float* out_wx;  // [3]         final-layer weights of x, y, z
    const float* out_wq;  // [12]        final-layer weights of q0, q1
};

__device__ __forceinline__ float act_fn(float z, int act) {
    return act == 0 ? fmaxf(z, 0.0f) : z / (1.0f + __expf(-z));
}

// Motion index of tile t: the last m with tile_off[m] <= t.
__device__ __forceinline__ int find_segment(const int* off, int n, int t) {
    int lo = 0, hi = n;   // invariant: off[lo] <= t < off[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= t) lo = mid; else hi = mid;
    }
    return lo;
}

// Squared distances from x to the 7 capsule axes, minimised over samples.
__device__ __forceinline__ void scan_samples(const Capsule* cs, int n_samples, float3 x, float (&mn)[kCaps])
{
    #pragma unroll
    for (int j = 0; j < kCaps; ++j) mn[j] = __int_as_float(0x7f800000);
    for (int k = 0; k < n_samples; ++k) {
        #pragma unroll
        for (int j = 0; j < kCaps; ++j) {
            const float4 ar = cs[k * kCaps + j].a_r;
            const float4 ei = cs[k * kCaps + j].e_inv;
            const float wx = x.x - ar.x, wy = x.y - ar.y, wz = x.z - ar.z;
            const float t = __saturatef(fmaf(wz, ei.z, fmaf(wy, ei.y, wx * ei.x)) * ei.w);
            const float dx = fmaf(-t, ei.x, wx), dy = fmaf(-t, ei.y, wy), dz = fmaf(-t, ei.z, wz);
            mn[j] = fminf(mn[j], fmaf(dz, dz, fmaf(dy, dy, dx * dx)));
        }
    }
}

__device__ __forceinline__ float capsule_min(const float (&mn)[kCaps], const Capsule* cs)
{
    float d = __int_as_float(0x7f800000);
    #pragma unroll
    for (int j = 0; j < kCaps; ++j) d = fminf(d, sqrtf(mn[j]) - cs[j].a_r.w);
    return d;
}

// ---------------------------------------------------------------- launches
void launch_prologue(const CallArgs& a, const DevWeights& w, cudaStream_t s);
void launch_mlp_fp32(const CallArgs& a, const DevWeights& w, int n_tiles, int bm, cudaStream_t s);
int  mlp_fp32_tile_rows();                                  // pairs per tile (64)
// Pairs per tile of the FP32 path for a call that has `tiles_small` tiles of
// 16 pairs: 16 when those fit in one wave on n_sms SMs, else 64.
int  mlp_fp32_tile_rows(long long tiles_small, int n_sms);
int  mlp_fp32_small_tile_rows();                            // 16
// Verifier launch shape: points each thread checks per chunk (1, 2 or 4) and
// resident CTAs per SM (0 = as many as shared memory allows, at most 8).
struct VerifyConfig {
    int points_per_thread = 2;
    int ctas_per_sm = 0;
};
void launch_verify(const CallArgs& a, int range_mode, int strict_pass, cudaStream_t s, int n_sms);
void launch_verify_cfg(const CallArgs& a, int range_mode, int strict_pass, cudaStream_t s, int n_sms,
                       const VerifyConfig& cfg);
void launch_ties(const CallArgs& a, cudaStream_t s, int n_sms);
void launch_finalize(const CallArgs& a, void* results, cudaStream_t s);
void launch_label(const CallArgs& a, float* delta, long long stride, cudaStream_t s);
// out[0] = ordered key of max (f - delta) over pairs with delta <= near_cut (atomicMax; 0 if
// none), out[1] += their count; out must be zeroed by the caller before the first launch.
void launch_gate_overestimate(const CallArgs& a, const float* f, long long stride, float near_cut,
                              unsigned int* out, cudaStream_t s);
void launch_quantize_bf16(const float* in, uint16_t* out, long long n, cudaStream_t s);
void launch_round_bf16(float* inout, long long n, cudaStream_t s);
void launch_quantize_e4m3(const float* in, uint8_t* out, float* deq, long long n, float scale, cudaStream_t s);
void launch_transpose(const float* in, float* out, int rows, int cols, int batches, cudaStream_t s);

}  // namespace svm

namespace svm {
void launch_prologue_fk(const CallArgs& a, const RobotParams& rp, const DevWeights& w, cudaStream_t s);
}  // namespace svm
