// mlp_tc.cu -- the network f(x, q0, q1) of Sec. IV-A on the 5th-generation
// tensor cores (tcgen05): BF16 or FP8 E4M3 operands, FP32 accumulation in
// tensor memory, fused with the gate and the compaction of flagged pairs.
//
// Persistent kernel, one CTA per SM, 18 warps:
//   warp 0       TMA producer: streams the weights, one 128-byte K-slice x
//                256 output rows (32 KB) per stage, into a ring of shared-
//                memory stages (128B swizzle, the K-major B operand);
//   warp 1       allocates the 512 TMEM columns and issues tcgen05.mma
//                (M = 128 pairs, N = 256 outputs) from one thread;
//   warps 2-9    epilogue of tile slot 0, warps 10-17 epilogue of slot 1;
//                two warps per TMEM lane quarter, each owning 128 columns.
// A CTA runs two tiles of 128 pairs at a time (slots 0 and 1 use TMEM
// columns [0,256) and [256,512)): while the tensor core computes a layer of
// one slot, the other slot's epilogue drains its accumulator -- TMEM ->
// registers (tcgen05.ld) -> bias, activation, rounding -> the next layer's A
// operand in shared memory (128B swizzle, K-major).
//
// Layer 1: the network input is [x; q0; q1]; W1 [x; q0; q1] + b1 splits into
// W1x x + c_m, with c_m from the prologue.  W1x x runs as one K = 16 BF16 MMA
// on (x_hi, y_hi, z_hi, x_lo, y_lo, z_lo), x = x_hi + x_lo in two bfloat16
// parts (x to about 2^-17 relative), against the BF16 layer-1 weights
// repeated twice; c_m is the bias of its epilogue.  Hidden layers are
// K = 256 MMAs.  The output layer W -> 1 is an FP32 dot product on the last
// accumulator, reduced over the two column halves through shared memory.
// Then the gate f <= margin + tau, a warp ballot and one atomicAdd per warp
// append the flagged point indices to the motion's list, and the motion's
// minimum prediction (Eq. 6) is kept with an atomic minimum.
//
// FP8: hidden weights and activations are E4M3 with per-layer scales; the
// accumulator is rescaled by s_w * s_a before the bias.  Both slots consume
// every weight stage (REUSE = 2), so each weight byte is read once per pair
// of tiles.  BF16: a 128 KB layer does not fit twice, so each slot streams it.
//
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the waiter
// sets the call's error word and an abort flag, every role leaves its loop,
// the MMA issuer and the producer wait (bounded) for their own operations in
// flight, and the TMEM is freed before the CTA exits.
#include <mutex>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include "mlp_tc.cuh"
#include "tc_ptx.cuh"

namespace svm {

namespace {

constexpr int TM = 128;                    // pairs per tile = MMA M
constexpr int WN = 256;                    // network width = MMA N = hidden K
constexpr int NUM_EPI_WARPS = 16;
constexpr int NUM_WARPS = 2 + NUM_EPI_WARPS;
constexpr int NUM_THREADS = NUM_WARPS * 32;
constexpr int EPI_PER_SLOT = NUM_EPI_WARPS / 2;
constexpr int HALF_COLS = WN / 2;
constexpr int STAGE_BYTES = 32768;         // one 128-byte K-slice x 256 rows
constexpr int KBLOCK_BYTES = TM * 128;     // one 128-byte K-block of a 128-row tile

// kind::f16 instruction descriptor: D f32 (bit 4), A and B bf16 (bits 7-9,
// 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t IDESC_BF16 = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(WN >> 3) << 17) |
                                ((uint32_t)(TM >> 4) << 24);
// kind::f8f6f4: D f32, A and B e4m3 (format code 0).
constexpr uint32_t IDESC_E4M3 = (1u << 4) | ((uint32_t)(WN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);

template <int PREC>
struct Cfg;
template <>
struct Cfg<SVM_BF16> {
    static constexpr int ELEM = 2;
    static constexpr int SLICE_K = 64;                   // elements per 128-byte row
    static constexpr int SLICES = WN / SLICE_K;          // 4 per hidden layer
    static constexpr int MMAS = 4;                       // K = 16 each
    static constexpr int STAGES = 3;
    static constexpr int REUSE = 1;
};
template <>
struct Cfg<SVM_FP8_E4M3> {
    static constexpr int ELEM = 1;
    static constexpr int SLICE_K = 128;
    static constexpr int SLICES = WN / SLICE_K;          // 2 per hidden layer
    static constexpr int MMAS = 4;                       // K = 32 each
    static constexpr int STAGES = 4;
    static constexpr int REUSE = 2;
};

// FP8 keeps its hidden biases (already divided by the next activation
// scale), the output layer's bias and the output weights in shared memory,
// read as broadcast 16-byte loads; BF16 has no room left and broadcasts them
// from registers with shuffles.
constexpr int MAX_HIDDEN = 16;
template <int PREC>
__host__ __device__ constexpr int bias_smem_bytes()
{
    return PREC == SVM_FP8_E4M3 ? (MAX_HIDDEN + 1) * WN * 4 : 0;
}

template <int PREC>
struct Smem {
    static constexpr int ACT_BYTES = TM * WN * Cfg<PREC>::ELEM;
    static constexpr int ACT0 = 0;
    static constexpr int W0 = 2 * ACT_BYTES;
    static constexpr int RED = W0 + Cfg<PREC>::STAGES * STAGE_BYTES;   // 2 x 128 floats
    static constexpr int BARS = RED + 2 * TM * 4;
    static constexpr int N_BARS = 2 * Cfg<PREC>::STAGES + 5;
    static constexpr int MISC = BARS + 8 * N_BARS;
    // [L-1 hidden][W], [output bias][W], [w_out][W]; 16-byte loads need 16-byte alignment
    static constexpr int BIAS = (MISC + 16 + 127) / 128 * 128;
    static constexpr int TOTAL = BIAS + bias_smem_bytes<PREC>();
    static constexpr int DYN = TOTAL + 1024;      // slack for 1024-byte alignment
};
static_assert(Smem<SVM_BF16>::DYN <= 232448, "shared memory budget");
static_assert(Smem<SVM_FP8_E4M3>::BIAS % 16 == 0, "bias table alignment");
static_assert(Smem<SVM_FP8_E4M3>::DYN <= 232448, "shared memory budget");

// ------------------------------------------------------------ PTX wrappers

using namespace ptx;

template <int ACT>
__device__ __forceinline__ float act_t(float z)
{
    if constexpr (ACT == SVM_RELU) return fmaxf(z, 0.0f);
    else return z / (1.0f + __expf(-z));
}

// Address of 16-byte chunk `c` (0..7) of K-block `kb` in row `r` of a tile
// stored K-major with the 128B swizzle (the layout the MMA descriptor reads).
__device__ __forceinline__ uint32_t act_chunk_addr(uint32_t base, int kb, int r, int c)
{
    return base + kb * KBLOCK_BYTES + r * 128 + ((c ^ (r & 7)) << 4);
}

// z = v * scale + bias for 32 columns, activation, rounding, and store as
// columns o0..o0+31 of row r of the next layer's A operand.
template <int PREC, int ACT>
__device__ __forceinline__ void epilogue32(uint32_t base, int r, int o0, float (&v)[32], const float* bias,
                                           float scale, float inv_next)
{
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 b4 = __ldg(reinterpret_cast<const float4*>(bias + o0 + 4 * q));
        v[4 * q + 0] = fmaf(v[4 * q + 0], scale, b4.x);
        v[4 * q + 1] = fmaf(v[4 * q + 1], scale, b4.y);
        v[4 * q + 2] = fmaf(v[4 * q + 2], scale, b4.z);
        v[4 * q + 3] = fmaf(v[4 * q + 3], scale, b4.w);
    }
    if constexpr (PREC == SVM_BF16) {
        constexpr bool RELU = ACT == SVM_RELU;
        if constexpr (!RELU) {
#pragma unroll
            for (int i = 0; i < 32; ++i) v[i] = act_t<ACT>(v[i]);
        }
        const int kb = o0 >> 6, c0 = (o0 & 63) >> 3;
#pragma unroll
        for (int c = 0; c < 4; ++c)
            st_shared_v4(act_chunk_addr(base, kb, r, c0 + c), pack_bf16<RELU>(v[8 * c + 0], v[8 * c + 1]),
                         pack_bf16<RELU>(v[8 * c + 2], v[8 * c + 3]), pack_bf16<RELU>(v[8 * c + 4], v[8 * c + 5]),
                         pack_bf16<RELU>(v[8 * c + 6], v[8 * c + 7]));
    } else {
#pragma unroll
        for (int i = 0; i < 32; ++i) v[i] = act_t<ACT>(v[i]) * inv_next;
        const int kb = o0 >> 7, c0 = (o0 & 127) >> 4;
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const float* g = v + 16 * c;
            st_shared_v4(act_chunk_addr(base, kb, r, c0 + c), pack_e4m3x4(g[0], g[1], g[2], g[3]),
                         pack_e4m3x4(g[4], g[5], g[6], g[7]), pack_e4m3x4(g[8], g[9], g[10], g[11]),
                         pack_e4m3x4(g[12], g[13], g[14], g[15]));
        }
    }
}

// 16-byte global load that does not allocate in L1
__device__ __forceinline__ float4 ld_stream_f4(const float4* p)
{
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

// ---- packed FP32 pairs (sm_100+): two values per instruction
__device__ __forceinline__ uint64_t f2(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
// max(v, 0) of both halves rounded to bfloat16, low half first
__device__ __forceinline__ uint32_t relu_bf16x2(uint64_t v)
{
    uint32_t d;
    asm("{\n .reg .f32 lo, hi;\n mov.b64 {lo, hi}, %1;\n cvt.rn.relu.bf16x2.f32 %0, hi, lo;\n}" : "=r"(d) : "l"(v));
    return d;
}
// max(v, 0) of both halves rounded to E4M3 (saturating), low byte first
__device__ __forceinline__ uint32_t relu_e4m3x2(uint64_t v)
{
    uint16_t d;
    asm("{\n .reg .f32 lo, hi;\n mov.b64 {lo, hi}, %1;\n cvt.rn.satfinite.relu.e4m3x2.f32 %0, hi, lo;\n}"
        : "=h"(d)
        : "l"(v));
    return d;
}

// Epilogue of 32 columns (o0..o0+31) of row r with ReLU, packed arithmetic:
//   BF16:        h = relu(acc + b)                  -> bfloat16
//   FP8 hidden:  h = relu(acc * c + b)  with c = s_w s_a / s_next and b
//                already divided by s_next          -> E4M3
//   FP8 layer 0: h = relu((acc + b) * c), c = 1 / s_next
// The 32 biases of the chunk are held one per lane (lane i holds the bias of
// column o0 + i) and broadcast by shuffles: no memory access on the path from
// the accumulator to the stores.
template <int PREC, bool LAYER0>
__device__ __forceinline__ void epilogue32_relu_lane(uint32_t base, int r, int o0, const float (&v)[32], float bl,
                                                     float c)
{
    const uint64_t c2 = f2(c, c);
    uint32_t out[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        const uint64_t a = f2(v[2 * q], v[2 * q + 1]);
        const uint64_t b = f2(__shfl_sync(0xffffffffu, bl, 2 * q), __shfl_sync(0xffffffffu, bl, 2 * q + 1));
        uint64_t z;
        if constexpr (PREC == SVM_BF16) {
            z = f2_add(a, b);
            out[q] = relu_bf16x2(z);
        } else {
            if constexpr (LAYER0) z = f2_mul(f2_add(a, b), c2);
            else z = f2_fma(a, c2, b);
            out[q] = relu_e4m3x2(z);
        }
    }
    if constexpr (PREC == SVM_BF16) {
        const int kb = o0 >> 6, c0 = (o0 & 63) >> 3;
#pragma unroll
        for (int k = 0; k < 4; ++k)
            st_shared_v4(act_chunk_addr(base, kb, r, c0 + k), out[4 * k + 0], out[4 * k + 1], out[4 * k + 2],
                         out[4 * k + 3]);
    } else {
        uint32_t w[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) w[k] = (out[2 * k] & 0xFFFFu) | (out[2 * k + 1] << 16);
        const int kb = o0 >> 7, c0 = (o0 & 127) >> 4;
        st_shared_v4(act_chunk_addr(base, kb, r, c0), w[0], w[1], w[2], w[3]);
        st_shared_v4(act_chunk_addr(base, kb, r, c0 + 1), w[4], w[5], w[6], w[7]);
    }
}

__device__ __forceinline__ float4 ld_shared_f4(uint32_t addr)
{
    float4 v;
    asm volatile("ld.shared.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(addr));
    return v;
}

// FP8 hidden layer with the 32 biases (divided by the next activation scale)
// read from shared memory at `brow` (broadcast loads): h = relu(acc * c + b).
__device__ __forceinline__ void epilogue32_relu_e4m3_sm(uint32_t base, int r, int o0, const float (&v)[32],
                                                        uint32_t brow, float c)
{
    const uint64_t c2 = f2(c, c);
    uint32_t out[16];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const float4 b4 = ld_shared_f4(brow + 16 * q);
        out[2 * q + 0] = relu_e4m3x2(f2_fma(f2(v[4 * q + 0], v[4 * q + 1]), c2, f2(b4.x, b4.y)));
        out[2 * q + 1] = relu_e4m3x2(f2_fma(f2(v[4 * q + 2], v[4 * q + 3]), c2, f2(b4.z, b4.w)));
    }
    uint32_t w[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) w[k] = (out[2 * k] & 0xFFFFu) | (out[2 * k + 1] << 16);
    const int kb = o0 >> 7, c0 = (o0 & 127) >> 4;
    st_shared_v4(act_chunk_addr(base, kb, r, c0), w[0], w[1], w[2], w[3]);
    st_shared_v4(act_chunk_addr(base, kb, r, c0 + 1), w[4], w[5], w[6], w[7]);
}

// BF16 ReLU epilogue of 32 columns (o0..o0+31) of a warp's 32 rows, read in
// the accumulator-fragment shape of tmem_ld_frag32: thread t owns columns
// 8 g + 2 (t % 4), +1 of each 8-column group g, so it needs two biases per
// group (two shuffles from bl, lane i holding the bias of column o0 + i)
// where the row-per-lane shape needs all 32; h = relu(acc + b) rounded to
// bfloat16 pairs, stored as the next layer's A operand (128B swizzle,
// K-major) by four stmatrix.x4, one per (16-row block, 8-row half): lane l
// addresses row l % 8 of the matrix of group l / 8.
__device__ __forceinline__ void epilogue32_bf16_frag(uint32_t base, int quarter, int lane, int o0,
                                                     const float (&v)[32], float bl)
{
    const int c2 = 2 * (lane & 3);
    uint32_t pk[16];                                   // [16-row block][8-row half][group]
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const uint64_t b = f2(__shfl_sync(0xffffffffu, bl, 8 * g + c2), __shfl_sync(0xffffffffu, bl, 8 * g + c2 + 1));
#pragma unroll
        for (int rb = 0; rb < 2; ++rb)
#pragma unroll
            for (int rh = 0; rh < 2; ++rh) {
                const int i = 16 * rb + 4 * g + 2 * rh;
                pk[8 * rb + 4 * rh + g] = relu_bf16x2(f2_add(f2(v[i], v[i + 1]), b));
            }
    }
    const int i = lane & 7, g = lane >> 3;   // row within the matrix (= row & 7), group of the matrix
    const uint32_t cpart =
        base + (uint32_t)((o0 >> 6) * KBLOCK_BYTES) + ((uint32_t)((((o0 & 63) >> 3) + g) ^ i) << 4);
#pragma unroll
    for (int rb = 0; rb < 2; ++rb)
#pragma unroll
        for (int rh = 0; rh < 2; ++rh) {
            const int r = quarter * 32 + 16 * rb + 8 * rh + i;
            stmatrix_x4(cpart + (uint32_t)(r * 128), pk[8 * rb + 4 * rh + 0], pk[8 * rb + 4 * rh + 1],
                        pk[8 * rb + 4 * rh + 2], pk[8 * rb + 4 * rh + 3]);
        }
}

// FP8 ReLU epilogue of 32 columns (o0..o0+31) of a warp's 32 rows in the
// accumulator-fragment shape (thread t: columns 8 g + 2 (t % 4), +1 of rows
// t / 4 and t / 4 + 8 of each 16-row block), stored with stmatrix.  Two E4M3
// values are one 16-bit element, so the columns of each 16-column block are
// stored in the order pi(j) = 4 ((j & 7) >> 1) + 2 (j >> 3) + (j & 1): thread
// t's pairs from groups 2p and 2p + 1 become the 4 adjacent bytes 4 (t % 4) ..
// of 16-byte chunk p, which is the element pair stmatrix takes from it.  The
// next layer's weights hold their K columns in the same order (host), so the
// products are unchanged.  Layer 0: h = relu((acc + b) c), b one per lane
// (lane i: column o0 + i); hidden: h = relu(acc c + b), b from the
// shared-memory table at brow (column o0 first).
template <bool LAYER0>
__device__ __forceinline__ void epilogue32_e4m3_frag(uint32_t base, int quarter, int lane, int o0, const float (&v)[32],
                                                     float bl, uint32_t brow, float c)
{
    const int c2 = 2 * (lane & 3);
    const uint64_t cc = f2(c, c);
    uint32_t pk[8];                                    // [16-row block][8-row half][16-column block]
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        uint32_t e16[2][4];                            // [group 2p, 2p + 1][16-row block, 8-row half]
#pragma unroll
        for (int gg = 0; gg < 2; ++gg) {
            const int g = 2 * p + gg;
            uint64_t b;
            if constexpr (LAYER0) {
                b = f2(__shfl_sync(0xffffffffu, bl, 8 * g + c2), __shfl_sync(0xffffffffu, bl, 8 * g + c2 + 1));
            } else {
                uint64_t t;
                asm volatile("ld.shared.b64 %0, [%1];" : "=l"(t) : "r"(brow + (uint32_t)((8 * g + c2) * 4)));
                b = t;
            }
#pragma unroll
            for (int rb = 0; rb < 2; ++rb)
#pragma unroll
                for (int rh = 0; rh < 2; ++rh) {
                    const int i = 16 * rb + 4 * g + 2 * rh;
                    const uint64_t a = f2(v[i], v[i + 1]);
                    const uint64_t z = LAYER0 ? f2_mul(f2_add(a, b), cc) : f2_fma(a, cc, b);
                    e16[gg][2 * rb + rh] = relu_e4m3x2(z);
                }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) pk[2 * k + p] = (e16[0][k] & 0xFFFFu) | (e16[1][k] << 16);
    }
    // stmatrix k (16-row block rb): lane l addresses row l % 8 of matrix l / 8 = (8-row half, 16-column block)
    const int i = lane & 7, j = lane >> 3, rh = j >> 1, p = j & 1;
    const int kb = o0 >> 7, c16 = ((o0 & 127) >> 4) + p;
#pragma unroll
    for (int rb = 0; rb < 2; ++rb) {
        const int r = quarter * 32 + 16 * rb + 8 * rh + i;
        stmatrix_x4(act_chunk_addr(base, kb, r, c16), pk[4 * rb + 0], pk[4 * rb + 1], pk[4 * rb + 2], pk[4 * rb + 3]);
    }
}

// ------------------------------------------------------------------ kernel

template <int PREC, int ACT>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    mlp_tc_kernel(const __grid_constant__ CUtensorMap wmap, const __grid_constant__ CUtensorMap w1map, CallArgs A,
                  DevWeights Wt, int n_tiles)
{
    using C = Cfg<PREC>;
    using SM = Smem<PREC>;
    extern __shared__ __align__(1024) unsigned char dsm_raw[];
    unsigned char* dsm =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(dsm);
    const uint32_t w_base = sbase + SM::W0;
    const uint32_t bar0 = sbase + SM::BARS;
    float* red = reinterpret_cast<float*>(dsm + SM::RED);
    auto act_base = [&](int s) { return sbase + SM::ACT0 + (uint32_t)(s * SM::ACT_BYTES); };
    auto full_bar = [&](int s) { return bar0 + 8 * s; };
    auto empty_bar = [&](int s) { return bar0 + 8 * (C::STAGES + s); };
    auto accf_bar = [&](int s) { return bar0 + 8 * (2 * C::STAGES + s); };
    auto epid_bar = [&](int s) { return bar0 + 8 * (2 * C::STAGES + 2 + s); };
    const uint32_t drain_bar = bar0 + 8 * (2 * C::STAGES + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(dsm + SM::MISC);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(dsm + SM::MISC + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_mine =
        n_tiles > (int)blockIdx.x ? (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    const int n_pairs = (n_mine + 1) >> 1;
    const int n_layers = A.L + 1;             // layer 0 = the x part of layer 1, then L hidden layers

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(accf_bar(s), 1);
            mbar_init(epid_bar(s), EPI_PER_SLOT);
        }
        mbar_init(drain_bar, 1);
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "r"(512)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if constexpr (bias_smem_bytes<PREC>() > 0) {
        // rows 0..L-2: hidden biases / next activation scale; row L-1: the
        // output layer's bias; row L: w_out
        float4* dst = reinterpret_cast<float4*>(dsm + SM::BIAS);
        const int L = A.L, q = WN / 4;
        for (int i = threadIdx.x; i < (L + 1) * q; i += blockDim.x) {
            const int row = i / q, c4 = i % q;
            const float* src = row < L - 1 ? Wt.bhs + (long long)row * WN
                                            : (row == L - 1 ? Wt.bh + (long long)(L - 1) * WN : Wt.wout);
            dst[i] = __ldg(reinterpret_cast<const float4*>(src) + c4);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&wmap)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&w1map)) : "memory");
            int stage = 0;
            uint32_t phase = 0;
            uint32_t armed = 0;            // bit s: stage s has been loaded at least once
            uint32_t armed_par = 0;        // bit s: parity of its last load
            bool ok = true;
            // the weight slices of one block (layer l), in MMA order
            auto load_layer = [&](int l) {
                const int slices = l == 0 ? 1 : C::SLICES;
                for (int kk = 0; kk < slices; ++kk) {
                    if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, A.dev_err)) { ok = false; return; }
                    mbar_arrive_tx(full_bar(stage), STAGE_BYTES);
                    if (l == 0) tma_load_2d(w_base + stage * STAGE_BYTES, &w1map, 0, 0, full_bar(stage));
                    else tma_load_2d(w_base + stage * STAGE_BYTES, &wmap, kk * C::SLICE_K, (l - 1) * WN,
                                     full_bar(stage));
                    armed |= 1u << stage;
                    armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
                    if (++stage == C::STAGES) { stage = 0; phase ^= 1u; }
                }
            };
            // lockstep: layer l of slot 0, then of slot 1; with REUSE = 2 both
            // slots consume one copy of the layer's slices
            for (int j = 0; j < n_pairs && ok; ++j)
                for (int l = 0; l < n_layers && ok; ++l)
                    for (int s = 0; s < (C::REUSE == 2 ? 1 : min(2, n_mine - 2 * j)) && ok; ++s) load_layer(l);
            // wait (bounded) for every copy this thread started
            for (int s = 0; s < C::STAGES; ++s)
                if (armed & (1u << s)) {
                    const uint32_t par = (armed_par >> s) & 1u;
                    const uint64_t t0 = globaltimer();
                    while (!mbar_try(full_bar(s), par) && globaltimer() - t0 < kTimeoutNs) {
                    }
                }
        }
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        // The whole warp runs the loop (warp-uniform control flow); one
        // elected lane issues each MMA and commit.  Descriptors are built
        // once: advancing K by 32 bytes inside a swizzle atom adds 2 to the
        // start-address field, a 128-byte K-block of the activations adds
        // KBLOCK_BYTES >> 4.
        const uint64_t a_desc0 = sdesc(act_base(0)), a_desc1 = sdesc(act_base(1));
        const uint64_t b_desc0 = sdesc(w_base);
        constexpr uint32_t IDESC = PREC == SVM_BF16 ? IDESC_BF16 : IDESC_E4M3;
        int stage = 0;
        uint32_t phase = 0;
        uint32_t epi_phase0 = 0u, epi_phase1 = 0u;
        bool ok = true;
        // one block: layer l of the tile in slot s.  first/last: whether this
        // block is the first / last consumer of the layer's weight stages.
        auto mma_block = [&](int s, int l, bool first, bool last) {
            uint32_t& ep = s == 0 ? epi_phase0 : epi_phase1;
            if (!mbar_wait_warp(epid_bar(s), ep, abort_flag, A.dev_err)) { ok = false; return; }
            ep ^= 1u;
            tc_fence_after();
            const uint32_t d_tmem = tmem_base + (uint32_t)(s * WN);
            const int slices = l == 0 ? 1 : C::SLICES;
            for (int kk = 0; kk < slices; ++kk) {
                if (first) {
                    if (!mbar_wait_warp(full_bar(stage), phase, abort_flag, A.dev_err)) { ok = false; return; }
                    tc_fence_after();
                }
                const uint64_t ad = (s == 0 ? a_desc0 : a_desc1) + (uint64_t)(kk * (KBLOCK_BYTES >> 4));
                const uint64_t bd = b_desc0 + (uint64_t)(stage * (STAGE_BYTES >> 4));
                if (l == 0) {
                    mma_f16_warp(d_tmem, ad, bd, IDESC_BF16, 0u);
                } else {
#pragma unroll
                    for (int k = 0; k < C::MMAS; ++k) {
                        if constexpr (PREC == SVM_BF16)
                            mma_f16_warp(d_tmem, ad + 2 * k, bd + 2 * k, IDESC, (kk | k) != 0 ? 1u : 0u);
                        else
                            mma_f8f6f4_warp(d_tmem, ad + 2 * k, bd + 2 * k, IDESC, (kk | k) != 0 ? 1u : 0u);
                    }
                }
                if (last) mma_commit_warp(empty_bar(stage));
                if (++stage == C::STAGES) { stage = 0; phase ^= 1u; }
            }
            mma_commit_warp(accf_bar(s));
        };
        {
            // lockstep: layer l of slot 0, then of slot 1 (on the same weight
            // stages when REUSE = 2).  Tried: staggering the slots by two
            // layers so that no two short layer-0 blocks meet -- slower.
            for (int j = 0; j < n_pairs && ok; ++j) {
                const int nslots = min(2, n_mine - 2 * j);
                for (int l = 0; l < n_layers && ok; ++l) {
                    const int layer_stage = stage;
                    const uint32_t layer_phase = phase;
                    for (int s = 0; s < nslots && ok; ++s) {
                        if (C::REUSE == 2) {
                            stage = layer_stage;
                            phase = layer_phase;
                            mma_block(s, l, s == 0, s == nslots - 1);
                        } else {
                            mma_block(s, l, true, true);
                        }
                    }
                }
            }
        }
        // every MMA issued by this warp has completed before TMEM is freed
        mma_commit_warp(drain_bar);
        const uint64_t t0 = globaltimer();
        while (!mbar_try(drain_bar, 0u) && globaltimer() - t0 < kTimeoutNs) {
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue warps
        // BF16 ReLU reads the accumulator in the fragment shape (two biases per thread and
        // 8-column group, stmatrix stores); FP8 and SiLU keep the row-per-lane shape
        constexpr bool kFrag = PREC == SVM_BF16 && ACT == SVM_RELU;
        constexpr bool kFrag8 = PREC == SVM_FP8_E4M3 && ACT == SVM_RELU;   // hidden stores only
        const int ew = warp - 2;
        const int s = ew / EPI_PER_SLOT;           // tile slot
        const int half = (ew % EPI_PER_SLOT) / 4;  // column half [half*128, half*128+128)
        const int quarter = warp & 3;              // TMEM lane quarter this warp may access
        const int r = quarter * 32 + lane;         // row of the tile = TMEM lane
        const int col0 = half * HALF_COLS;
        const uint32_t abase = act_base(s);
        const uint32_t t_row = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(s * WN + col0);
        float* red_s = red + s * TM;
        uint32_t acc_phase = 0;
        bool ok = true;
        // tile i of this CTA: its motion, this lane's point, whether it exists
        auto tile_info = [&](int i, int& m, long long& p, bool& valid) {
            const int t = (int)blockIdx.x + i * (int)gridDim.x;
            m = find_segment(A.tile_off, A.M, t);
            p = A.pbeg[m] + (long long)(t - A.tile_off[m]) * TM + r;
            valid = p < A.pend[m];
        };
        // streamed once per tile: kept out of L1 so that the bias vectors stay there
        auto load_x = [&](long long p, bool valid) {
            return valid ? ld_stream_f4(A.points + p) : make_float4(0.f, 0.f, 0.f, 0.f);
        };
        // A operand of layer 0 (column half 0 writes it): (x_hi, y_hi, z_hi,
        // x_lo, y_lo, z_lo, 0, ...); then every warp of the slot arrives
        auto stage_x = [&](float4 x) {
            if (half == 0) {
                // hi parts are the nearest bfloat16; the differences are exact in FP32
                const float xl = x.x - __bfloat162float(__float2bfloat16_rn(x.x));
                const float yl = x.y - __bfloat162float(__float2bfloat16_rn(x.y));
                const float zl = x.z - __bfloat162float(__float2bfloat16_rn(x.z));
                st_shared_v4(act_chunk_addr(abase, 0, r, 0), pack_bf16<false>(x.x, x.y), pack_bf16<false>(x.z, xl),
                             pack_bf16<false>(yl, zl), 0u);
                st_shared_v4(act_chunk_addr(abase, 0, r, 1), 0u, 0u, 0u, 0u);
                fence_async_smem();
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(epid_bar(s));
        };
        // gate and compaction of a finished tile (column half 0): flag f <= margin + tau,
        // append the flagged points to the motion's list, keep the minimum prediction
        bool pend = false, pvalid = false;
        float pf = 0.0f;
        int pm = 0;
        long long pp = 0;
        // In two parts: gate() reserves the list space (the atomic is left in
        // flight), gate_store() -- one layer later -- writes the indices.
        unsigned pmask = 0, pbase = 0;
        bool pstore = false;
        auto gate = [&]() {
            pend = false;
            if (A.f_out != nullptr && pvalid) A.f_out[(long long)pm * A.f_stride + (pp - A.pbeg[pm])] = pf;
            const bool flag = pvalid && pf <= A.gate;
            pmask = __ballot_sync(0xffffffffu, flag);
            pbase = 0;
            if (lane == 0 && pmask) pbase = atomicAdd(&A.st[pm].n_flagged, (unsigned)__popc(pmask));
            pstore = true;
            float fm = pvalid ? pf : __int_as_float(0x7f800000);
#pragma unroll
            for (int sh = 16; sh > 0; sh >>= 1) fm = fminf(fm, __shfl_xor_sync(0xffffffffu, fm, sh));
            if (lane == 0 && fm < __int_as_float(0x7f800000)) atomicMin(&A.st[pm].dhat_key, float_key(fm));
            if (fm <= A.gate) {        // the warp's smallest prediction is flagged: a probe candidate
                const unsigned who = __ballot_sync(0xffffffffu, pvalid && pf == fm);
                const unsigned pi = __shfl_sync(0xffffffffu, (unsigned)pp, __ffs(who) - 1);
                if (lane == 0) atomicMin(&A.st[pm].probe_key, ((unsigned long long)float_key(fm) << 32) | pi);
            }
        };
        auto gate_store = [&]() {
            pstore = false;
            const unsigned base = __shfl_sync(0xffffffffu, pbase, 0);
            if ((pmask >> lane) & 1u)
                A.idx[A.pair_off[pm] + base + __popc(pmask & ((1u << lane) - 1u))] = (unsigned)pp;
        };
        int m = 0;
        long long p = 0;
        bool valid = false;
        if (s < n_mine) {
            tile_info(s, m, p, valid);
            if (!(A.test_stall && blockIdx.x == 0 && s == 0)) stage_x(load_x(p, valid));
        }
        for (int i = s; i < n_mine && ok; i += 2) {
            // the slot's next tile: looked up, and its points loaded, during the
            // output layer of this one; staged as soon as the output is reduced
            const bool has_next = i + 2 < n_mine;
            int nm = 0;
            long long np = 0;
            bool nvalid = false;
            float4 nx = make_float4(0.f, 0.f, 0.f, 0.f);
            // ---- layers
            for (int l = 0; l < n_layers; ++l) {
                const float* bias = l == 0 ? A.cbias + (long long)m * WN : Wt.bh + (long long)(l - 1) * WN;
                // ReLU hidden layers: the 128 biases of this warp's columns, one
                // per lane per 32-column chunk, loaded before the accumulator wait
                // (the output layer also takes its output weights the same way)
                // (FP8 layers after the first read them from the shared-memory table)
                constexpr bool kSmemBias = bias_smem_bytes<PREC>() > 0 && ACT == SVM_RELU;
                const bool sm_bias = kSmemBias && l > 0;
                const uint32_t sb = smem_u32(dsm + SM::BIAS);
                float bl0 = 0.0f, bl1 = 0.0f, bl2 = 0.0f, bl3 = 0.0f;
                float wl0 = 0.0f, wl1 = 0.0f, wl2 = 0.0f, wl3 = 0.0f;
                if (ACT == SVM_RELU && !sm_bias) {
                    const float* bsrc =
                        (PREC == SVM_FP8_E4M3 && l > 0 && l + 1 < n_layers) ? Wt.bhs + (long long)(l - 1) * WN : bias;
                    bl0 = __ldg(bsrc + col0 + lane);
                    bl1 = __ldg(bsrc + col0 + 32 + lane);
                    bl2 = __ldg(bsrc + col0 + 64 + lane);
                    bl3 = __ldg(bsrc + col0 + 96 + lane);
                    if (l + 1 == n_layers) {
                        wl0 = __ldg(Wt.wout + col0 + lane);
                        wl1 = __ldg(Wt.wout + col0 + 32 + lane);
                        wl2 = __ldg(Wt.wout + col0 + 64 + lane);
                        wl3 = __ldg(Wt.wout + col0 + 96 + lane);
                    }
                }
                if (l == 1 && pend) {         // the previous tile's gate, after this tile's layer 0
                    gate();
                    if (n_layers < 3) gate_store();
                }
                if (l == 2 && pstore) gate_store();
                if (l + 1 == n_layers && has_next) {
                    tile_info(i + 2, nm, np, nvalid);
                    if (half == 0) nx = load_x(np, nvalid);
                }
                if (!mbar_wait(accf_bar(s), acc_phase, abort_flag, A.dev_err)) { ok = false; break; }
                acc_phase ^= 1u;
                tc_fence_after();
                const float scale =
                    (PREC == SVM_FP8_E4M3 && l > 0) ? __ldg(Wt.wscale + l - 1) * __ldg(Wt.ascale + l - 1) : 1.0f;
                if (l + 1 < n_layers) {
                    const float inv_next = PREC == SVM_FP8_E4M3 ? 1.0f / __ldg(Wt.ascale + l) : 1.0f;
#pragma unroll 1
                    for (int o0 = 0; o0 < HALF_COLS; o0 += 32) {
                        float v[32];
                        if constexpr (kFrag) {
                            tmem_ld_frag32(t_row + (uint32_t)o0, v);
                            epilogue32_bf16_frag(abase, quarter, lane, col0 + o0, v, bl0);
                            bl0 = bl1;
                            bl1 = bl2;
                            bl2 = bl3;
                            continue;
                        }
                        if constexpr (kFrag8) {
                            tmem_ld_frag32(t_row + (uint32_t)o0, v);
                            if (l == 0)
                                epilogue32_e4m3_frag<true>(abase, quarter, lane, col0 + o0, v, bl0, 0u, inv_next);
                            else
                                epilogue32_e4m3_frag<false>(abase, quarter, lane, col0 + o0, v, 0.0f,
                                                            sb + (uint32_t)(((l - 1) * WN + col0 + o0) * 4),
                                                            scale * inv_next);
                            bl0 = bl1;
                            bl1 = bl2;
                            bl2 = bl3;
                            continue;
                        }
                        tmem_ld32(t_row + (uint32_t)o0, v);
                        if constexpr (ACT == SVM_RELU) {
                            if (PREC == SVM_FP8_E4M3 && l == 0)
                                epilogue32_relu_lane<PREC, true>(abase, r, col0 + o0, v, bl0, inv_next);
                            else if (sm_bias)
                                epilogue32_relu_e4m3_sm(abase, r, col0 + o0, v,
                                                        sb + (uint32_t)(((l - 1) * WN + col0 + o0) * 4),
                                                        scale * inv_next);
                            else if (PREC == SVM_FP8_E4M3)
                                epilogue32_relu_lane<PREC, false>(abase, r, col0 + o0, v, bl0, scale * inv_next);
                            else
                                epilogue32_relu_lane<PREC, false>(abase, r, col0 + o0, v, bl0, 1.0f);
                            bl0 = bl1;
                            bl1 = bl2;
                            bl2 = bl3;
                        } else {
                            epilogue32<PREC, ACT>(abase, r, col0 + o0, v, bias, scale, inv_next);
                        }
                    }
                    fence_async_smem();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(epid_bar(s));
                } else {
                    float f = 0.0f;
                    uint64_t f2acc = f2(0.0f, 0.0f);
                    const uint64_t s2 = f2(scale, scale);
                    if constexpr (kFrag) {
                        // fragment shape: partial dot products of the thread's four rows, summed over the
                        // four threads of a row, then handed to the row-per-lane layout of the gate
                        const int c2 = 2 * (lane & 3);
                        uint64_t acc4[4] = {f2acc, f2acc, f2acc, f2acc};
#pragma unroll 1
                        for (int o0 = 0; o0 < HALF_COLS; o0 += 32) {
                            float v[32];
                            tmem_ld_frag32(t_row + (uint32_t)o0, v);
#pragma unroll
                            for (int g = 0; g < 4; ++g) {
                                const uint64_t b = f2(__shfl_sync(0xffffffffu, bl0, 8 * g + c2),
                                                      __shfl_sync(0xffffffffu, bl0, 8 * g + c2 + 1));
                                const uint64_t w = f2(__shfl_sync(0xffffffffu, wl0, 8 * g + c2),
                                                      __shfl_sync(0xffffffffu, wl0, 8 * g + c2 + 1));
#pragma unroll
                                for (int k = 0; k < 4; ++k) {
                                    const int i = 16 * (k >> 1) + 4 * g + 2 * (k & 1);
                                    float zl, zh;
                                    asm("mov.b64 {%0, %1}, %2;" : "=f"(zl), "=f"(zh) : "l"(f2_add(f2(v[i], v[i + 1]), b)));
                                    acc4[k] = f2_fma(w, f2(fmaxf(zl, 0.0f), fmaxf(zh, 0.0f)), acc4[k]);
                                }
                            }
                            bl0 = bl1;
                            bl1 = bl2;
                            bl2 = bl3;
                            wl0 = wl1;
                            wl1 = wl2;
                            wl2 = wl3;
                        }
                        // every TMEM read of this tile is done: hand the slot and the next tile's layer-0
                        // operand over now, before the reductions and the gate
                        tc_fence_before();
                        if (has_next) stage_x(nx);
                        float sk[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            float lo, hi;
                            asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc4[k]));
                            sk[k] = lo + hi;
                            sk[k] += __shfl_xor_sync(0xffffffffu, sk[k], 1);
                            sk[k] += __shfl_xor_sync(0xffffffffu, sk[k], 2);
                        }
                        // row 16 rb + 8 rh + t / 4 of the warp is in sk[2 rb + rh] of threads 4 (t / 4) ..;
                        // lane L takes row L: k = L / 8 from thread 4 (L % 8)
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const float x = __shfl_sync(0xffffffffu, sk[k], 4 * (lane & 7));
                            if ((lane >> 3) == k) f = x;
                        }
                    }
#pragma unroll 1
                    for (int o0 = 0; o0 < (kFrag ? 0 : HALF_COLS); o0 += 32) {
                        float v[32];
                        tmem_ld32(t_row + (uint32_t)o0, v);
                        if (sm_bias) {
                            const uint32_t brow = sb + (uint32_t)(((A.L - 1) * WN + col0 + o0) * 4);
                            const uint32_t wrow = sb + (uint32_t)((A.L * WN + col0 + o0) * 4);
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const float4 b4 = ld_shared_f4(brow + 16 * q), w4 = ld_shared_f4(wrow + 16 * q);
                                const uint64_t z0 = f2_fma(f2(v[4 * q + 0], v[4 * q + 1]), s2, f2(b4.x, b4.y));
                                const uint64_t z1 = f2_fma(f2(v[4 * q + 2], v[4 * q + 3]), s2, f2(b4.z, b4.w));
                                float z0l, z0h, z1l, z1h;
                                asm("mov.b64 {%0, %1}, %2;" : "=f"(z0l), "=f"(z0h) : "l"(z0));
                                asm("mov.b64 {%0, %1}, %2;" : "=f"(z1l), "=f"(z1h) : "l"(z1));
                                f2acc = f2_fma(f2(w4.x, w4.y), f2(fmaxf(z0l, 0.0f), fmaxf(z0h, 0.0f)), f2acc);
                                f2acc = f2_fma(f2(w4.z, w4.w), f2(fmaxf(z1l, 0.0f), fmaxf(z1h, 0.0f)), f2acc);
                            }
                            continue;
                        }
                        if constexpr (ACT == SVM_RELU) {
#pragma unroll
                            for (int q = 0; q < 16; ++q) {
                                const uint64_t b = f2(__shfl_sync(0xffffffffu, bl0, 2 * q),
                                                      __shfl_sync(0xffffffffu, bl0, 2 * q + 1));
                                const uint64_t w = f2(__shfl_sync(0xffffffffu, wl0, 2 * q),
                                                      __shfl_sync(0xffffffffu, wl0, 2 * q + 1));
                                const uint64_t z = f2_fma(f2(v[2 * q], v[2 * q + 1]), s2, b);
                                float zl, zh;
                                asm("mov.b64 {%0, %1}, %2;" : "=f"(zl), "=f"(zh) : "l"(z));
                                f2acc = f2_fma(w, f2(fmaxf(zl, 0.0f), fmaxf(zh, 0.0f)), f2acc);
                            }
                            bl0 = bl1;
                            bl1 = bl2;
                            bl2 = bl3;
                            wl0 = wl1;
                            wl1 = wl2;
                            wl2 = wl3;
                        } else {
#pragma unroll
                            for (int q = 0; q < 8; ++q) {
                                const float4 b4 = __ldg(reinterpret_cast<const float4*>(bias + col0 + o0 + 4 * q));
                                const float4 w4 = __ldg(reinterpret_cast<const float4*>(Wt.wout + col0 + o0 + 4 * q));
                                f = fmaf(w4.x, act_t<ACT>(fmaf(v[4 * q + 0], scale, b4.x)), f);
                                f = fmaf(w4.y, act_t<ACT>(fmaf(v[4 * q + 1], scale, b4.y)), f);
                                f = fmaf(w4.z, act_t<ACT>(fmaf(v[4 * q + 2], scale, b4.z)), f);
                                f = fmaf(w4.w, act_t<ACT>(fmaf(v[4 * q + 3], scale, b4.w)), f);
                            }
                        }
                    }
                    if constexpr (!kFrag) {
                        // every TMEM read of this tile is done: hand the slot and the next tile's
                        // layer-0 operand over before the reductions and the gate
                        tc_fence_before();
                        if (has_next) stage_x(nx);
                    }
                    {
                        float lo, hi;
                        asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(f2acc));
                        f += lo + hi;
                    }
                    // the two column halves of a row meet in shared memory
                    if (half == 1) red_s[r] = f;
                    named_sync(1 + s, 32 * EPI_PER_SLOT);
                    if (half == 0) f += red_s[r] + Wt.bout;
                    // FP8: the gate of this tile waits until the next tile's layer-0
                    // epilogue is done (its atomics would delay that epilogue; FP8's
                    // short MMA blocks leave no slack for them).  Measured slower
                    // for BF16, which gates at once.
                    constexpr bool kDeferGate = PREC == SVM_FP8_E4M3;
                    if (half == 0) {
                        pend = true;
                        pf = f;
                        pm = m;
                        pp = p;
                        pvalid = valid;
                        if (!has_next || !kDeferGate) {
                            gate();
                            gate_store();
                        }
                    }
                }
            }
            m = nm;
            p = np;
            valid = nvalid;
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
    }
}

using EncodeFn = PFN_cuTensorMapEncodeTiled_v12000;

EncodeFn get_encode()
{
    static EncodeFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    }
    return fn;
}

template <int PREC, int ACT>
void launch_t(const TcModel& t, const CallArgs& a, const DevWeights& w, int n_tiles, int grid, cudaStream_t s)
{
    int dev = 0;
    cudaGetDevice(&dev);
    static std::once_flag done[64];            // once per device, safe across host threads
    if (dev >= 0 && dev < 64)
        std::call_once(done[dev], [] {
            cudaFuncSetAttribute(mlp_tc_kernel<PREC, ACT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 Smem<PREC>::DYN);
        });
    const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(t.wmap);
    const CUtensorMap* map1 = reinterpret_cast<const CUtensorMap*>(t.w1map);
    mlp_tc_kernel<PREC, ACT><<<grid, NUM_THREADS, Smem<PREC>::DYN, s>>>(*map, *map1, a, w, n_tiles);
}

CUresult encode_2d(EncodeFn enc, CUtensorMap* map, CUtensorMapDataType dt, const void* gaddr, uint64_t inner,
                   uint64_t rows, uint64_t row_bytes, uint32_t box_inner, uint32_t box_rows)
{
    const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)row_bytes};
    const cuuint32_t box[2] = {box_inner, box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return enc(map, dt, 2, const_cast<void*>(gaddr), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
               CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

}  // namespace

int tc_tile_rows() { return TM; }

size_t tc_workspace_bytes(int) { return 256; }

int tc_prepare(TcModel& t, const svm_model_desc& d, const DevWeights& w)
{
    t.ready = false;
    t.prec = d.prec;
    t.act = d.act;
    t.arch = SVM_ARCH_MLP;
    EncodeFn enc = get_encode();
    if (!enc || d.width != WN || !w.wq || !w.w1pad) return -1;
    const int elem = d.prec == SVM_BF16 ? 2 : 1;
    const CUtensorMapDataType dt = d.prec == SVM_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8;
    if (encode_2d(enc, reinterpret_cast<CUtensorMap*>(t.wmap), dt, w.wq, WN, (uint64_t)WN * d.n_hidden, WN * elem,
                  128 / elem, WN) != CUDA_SUCCESS)
        return -2;
    if (encode_2d(enc, reinterpret_cast<CUtensorMap*>(t.w1map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, w.w1pad, 64, WN, 128,
                  64, WN) != CUDA_SUCCESS)
        return -3;
    t.ready = true;
    return 0;
}

void tc_release(TcModel& t) { t.ready = false; }

int tc_launch(TcModel& t, const CallArgs& a, const DevWeights& w, int n_tiles, void* ws, int n_sms, cudaStream_t s)
{
    (void)ws;
    if (!t.ready) return -1;
    if (n_tiles <= 0) return 0;
    const int grid = n_tiles < n_sms ? n_tiles : n_sms;
    if (t.arch == SVM_ARCH_BLOCKS) return tc_block_launch(t, a, w, n_tiles, grid, s);
    if (t.prec == SVM_BF16) {
        if (t.act == SVM_RELU) launch_t<SVM_BF16, SVM_RELU>(t, a, w, n_tiles, grid, s);
        else launch_t<SVM_BF16, SVM_SILU>(t, a, w, n_tiles, grid, s);
    } else {
        if (t.act == SVM_RELU) launch_t<SVM_FP8_E4M3, SVM_RELU>(t, a, w, n_tiles, grid, s);
        else launch_t<SVM_FP8_E4M3, SVM_SILU>(t, a, w, n_tiles, grid, s);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace svm
