// mlp_tc_block.cu -- the block architecture of Sec. IV-A (Fig. 2) on the
// 5th-generation tensor cores: BF16 operands, FP32 accumulation in tensor
// memory, width 512, fused with the gate and the compaction of flagged pairs.
//
// Network (u = [x; q0; q1]):
//   h_0 = W_0 u + b_0                                   initial linear layer
//   block l = 1..L:  z_l = W_l v_l + b_l,  v_1 = h_0,  v_l = [h_{l-1}; u]
//                    (the jump connection from the second block on)
//                    h_l = BN_l(relu(z_l)) + h_{l-1}    (skip connection)
//   f = w_f [h_L; u] + b_f                              final layer
// BatchNorm at inference is folded into a per-channel scale s_l and shift t_l
// at load.  Every layer's q-part and bias is a per-motion constant c_{l,m}
// (the prologue), the h-parts are 128 x 512 x 512 tcgen05 GEMMs (two N = 256
// halves), and the jump x-part of blocks 2..L (K = 3) is one more K = 16 MMA
// per half on (x_hi, y_hi, z_hi, x_mid, .., z_lo, 0, ...), x = x_hi + x_mid +
// x_lo in three bfloat16 parts (x to about 2^-24 relative), against the
// block's bfloat16 x-weights repeated three times.  The initial layer is such
// an MMA too: a layer 0 of x entries only, whose epilogue adds c_0 and rounds
// h_0.  At a tile change each column half of the last block is handed to the
// next tile's layer 0 as soon as it is read, and the finished tile's
// reduction and gate follow the next tile's layer-0 epilogue, beside the next
// tile's first block.
//
// Persistent kernel, one CTA per SM, 18 warps:
//   warp 0       producer: weight slices of 64 K x 256 output rows (32 KB,
//                128B swizzle, K-major B operand) by TMA into a 3-stage ring;
//                for layer 0 and blocks 2..L, ahead of each half's slices, an x
//                entry: the half's x-weights (256 rows x 16 K, 32B swizzle) by
//                TMA and the tile's (x_hi, .., z_lo) rows, written by the warp's
//                32 lanes into the same stage (the A operand, 32B swizzle);
//   warp 1       allocates the 512 TMEM columns and issues tcgen05.mma (one
//                elected lane, warp-uniform loop): per layer and N = 256 half
//                the x entry's MMA, then (blocks) 8 K-slices of 4 MMAs (K = 16);
//   warps 2-17   epilogue: warp w reads TMEM lane quarter w % 4 and owns 64
//                columns of each column half, 64 * ((w - 2) / 4) onwards.
// One 128-pair tile is in flight per CTA: its 512-wide FP32 accumulator fills
// the TMEM, and the layer's input -- a 128 x 512 bfloat16 tile in shared
// memory (K-major, 128B swizzle), which is also its skip term -- is updated in
// place by the epilogue.  The epilogue works in two column halves, each taken
// by all 16 warps: a block issues [output half 0 x input half 0], [half 0 x
// input half 1], [half 1 x input half 0], then commits -- output half 0 is
// final and input half 0 has been read by both halves, so the epilogue of
// columns 0-255 runs while the last quarter [half 1 x input half 1] computes;
// the next block's first quarter needs only that half of its input, and its
// second quarter the other half.
// The epilogue reads the accumulator in the 16x256b fragment shape (thread t:
// two adjacent columns of two rows per 8-column group), reads the skip term
// with ldmatrix and writes the new activation with stmatrix.  The final layer
// sums per-thread partial dot products over the four threads of a row, the
// four column quarters of a row meet in shared memory, and the gate, ballot
// compaction and per-motion minima follow as in mlp_tc.cu.
//
// Every mbarrier wait is bounded (2 s); on expiry the waiter sets the call's
// error word and the CTA's abort flag, every role leaves its loop, and the
// TMEM is freed before the CTA exits (the records then carry status 1).
#include <mutex>
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "mlp_tc.cuh"
#include "tc_ptx.cuh"

namespace svm {

namespace {

using namespace ptx;

constexpr int TM = 128;                      // pairs per tile = MMA M
constexpr int WB = 512;                      // network width
constexpr int NH = 256;                      // MMA N: one half of the width
constexpr int BK = 64;                       // K elements per weight slice (128 bytes)
constexpr int KSL = WB / BK;                 // 8 slices per half and block
constexpr int STAGES = 3;
constexpr int STAGE_BYTES = NH * 128;        // 32 KB
constexpr int XW_BYTES = NH * 32;            // x entry: the half's x-weights, 256 rows x 32 bytes
constexpr int XT_OFF = XW_BYTES;             // x entry: the tile's x rows, 128 x 32 bytes, after them
constexpr int KBLOCK_BYTES = TM * 128;       // one 128-byte K-block of the activation tile
constexpr int ACT_BYTES = TM * WB * 2;       // 128 KB
constexpr int NUM_EPI_WARPS = 16;
constexpr int NUM_THREADS = (2 + NUM_EPI_WARPS) * 32;
constexpr int OFF_W = ACT_BYTES;
constexpr int OFF_RED = OFF_W + STAGES * STAGE_BYTES;       // [3][TM] floats: column quarters 1-3
constexpr int OFF_BAR = OFF_RED + 3 * TM * 4;
constexpr int N_BARS = 2 * STAGES + 5;
constexpr int OFF_MISC = OFF_BAR + 8 * N_BARS;
constexpr int SMEM_DYN = OFF_MISC + 16 + 1024;              // slack for 1024-byte alignment
static_assert(SMEM_DYN <= 232448, "shared memory budget");
// kind::f16: D f32, A and B bf16, both K-major, N >> 3 at bit 17, M >> 4 at bit 24
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NH >> 3) << 17) |
                           ((uint32_t)(TM >> 4) << 24);

__device__ __forceinline__ uint64_t f2(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void f2_split(uint64_t v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ uint64_t f2_relu(uint64_t v)
{
    float lo, hi;
    f2_split(v, lo, hi);
    return f2(fmaxf(lo, 0.0f), fmaxf(hi, 0.0f));
}
// both halves rounded to bfloat16, low half first
__device__ __forceinline__ uint32_t bf16x2(uint64_t v)
{
    uint32_t d;
    asm("{\n .reg .f32 lo, hi;\n mov.b64 {lo, hi}, %1;\n cvt.rn.bf16x2.f32 %0, hi, lo;\n}" : "=r"(d) : "l"(v));
    return d;
}
__device__ __forceinline__ uint64_t bf16x2_to_f2(uint32_t w)
{
    return f2(__uint_as_float(w << 16), __uint_as_float(w & 0xFFFF0000u));
}
__device__ __forceinline__ float2 ldg2(const float* p) { return __ldg(reinterpret_cast<const float2*>(p)); }

__device__ __forceinline__ float4 ld_stream_f4(const float4* p)
{
    float4 v;
    asm volatile("ld.global.nc.L1::no_allocate.v4.f32 {%0,%1,%2,%3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p));
    return v;
}

// Shared-memory matrix descriptor of a K-major operand with 32-byte rows (K =
// 16 bfloat16) in the 32B swizzle: 8-row groups 256 bytes apart (SBO).
__device__ __forceinline__ uint64_t sdesc32(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // LBO (unused: one swizzle atom spans the MMA's K)
    d |= (uint64_t)(256 >> 4) << 32;        // SBO
    d |= (uint64_t)1 << 46;                 // version
    d |= (uint64_t)6 << 61;                 // SWIZZLE_32B
    return d;
}

// Byte offset of 16-byte chunk c (0, 1) of row r in a tile of 32-byte rows,
// 32B swizzle (the layout TMA writes and the descriptor above reads): the
// chunk index flips with bit 2 of the row.
__device__ __forceinline__ uint32_t swz32(int r, int c) { return (uint32_t)(r * 32 + ((c ^ ((r >> 2) & 1)) << 4)); }

// Shared-memory address of row `row`, 16-byte chunk of column c8 * 8, of the
// activation tile (K-major, 128B swizzle: the layout the MMA descriptor reads).
__device__ __forceinline__ uint32_t act_addr(uint32_t base, int row, int c8)
{
    return base + (uint32_t)((c8 >> 3) * KBLOCK_BYTES + row * 128 + (((c8 & 7) ^ (row & 7)) << 4));
}

// The per-column constants of a 32-column chunk from c0, one load per lane
// (taken before the wait for the accumulator, so that they arrive while the
// MMAs run): lanes 0-15 hold column pair c0 + 2 (lane % 16)'s record (s, s',
// t, t') in ka and, for the final layer, its output weights in kb; lanes 16-31
// hold its per-motion constants (c, c') in ka.xy.
__device__ __forceinline__ void chunk_consts(int lane, int c0, const float* cl, const float* crec, const float* wf,
                                             bool last, float4& ka, float2& kb)
{
    const int c = c0 + 2 * (lane & 15);
    kb = make_float2(0.f, 0.f);
    if (lane < 16) {
        ka = __ldg(reinterpret_cast<const float4*>(crec + 2 * c));
        if (last) kb = ldg2(wf + c);
    } else {
        const float2 b = ldg2(cl + c);
        ka = make_float4(b.x, b.y, 0.f, 0.f);
    }
}

template <bool LAST>
__device__ __forceinline__ void block_chunk(uint32_t abase, uint32_t t_addr, int q, int lane, int c0, float4 ka,
                                            float2 kb, uint64_t (&acc4)[4])
{
    float v[32];
    tmem_ld_frag32(t_addr, v);
    const int i8 = lane & 7, j = lane >> 3;
    uint32_t pk[16];                                  // [row block k][group g]
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        // this thread's columns c0 + 8 g + 2 (lane % 4) and the next: pair pi of the chunk
        const int pi = 4 * g + (lane & 3);
        // the skip term: the block's input at the same rows and columns
        uint32_t hp[4];
        ldmatrix_x4(act_addr(abase, q * 32 + 16 * (j >> 1) + 8 * (j & 1) + i8, (c0 + 8 * g) >> 3), hp[0], hp[1],
                    hp[2], hp[3]);
        const uint64_t s2 = f2(__shfl_sync(0xffffffffu, ka.x, pi), __shfl_sync(0xffffffffu, ka.y, pi));
        const uint64_t t2 = f2(__shfl_sync(0xffffffffu, ka.z, pi), __shfl_sync(0xffffffffu, ka.w, pi));
        const uint64_t b2 = f2(__shfl_sync(0xffffffffu, ka.x, 16 + pi), __shfl_sync(0xffffffffu, ka.y, 16 + pi));
        uint64_t w2 = 0;
        if constexpr (LAST) w2 = f2(__shfl_sync(0xffffffffu, kb.x, pi), __shfl_sync(0xffffffffu, kb.y, pi));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int vi = 16 * (k >> 1) + 4 * g + 2 * (k & 1);
            const uint64_t z = f2_add(f2(v[vi], v[vi + 1]), b2);
            const uint64_t h = f2_add(f2_fma(f2_relu(z), s2, t2), bf16x2_to_f2(hp[k]));
            if constexpr (LAST) acc4[k] = f2_fma(w2, h, acc4[k]);
            else pk[4 * k + g] = bf16x2(h);
        }
    }
    if constexpr (!LAST) {
#pragma unroll
        for (int k = 0; k < 4; ++k)
            stmatrix_x4(act_addr(abase, q * 32 + 16 * (k >> 1) + 8 * (k & 1) + i8, (c0 >> 3) + j), pk[4 * k + 0],
                        pk[4 * k + 1], pk[4 * k + 2], pk[4 * k + 3]);
    }
}

// h_0 = W_0x x + c_0 (no activation) for the warp's 32 rows and the 32 columns
// from c0: the accumulator holds W_0x x (the tile's layer-0 x entry); c_0 of
// column pair i of the chunk is in lane base + i (kc = (c, c')).  Rounded to
// bfloat16, it is the first block's input.
__device__ __forceinline__ void h0_chunk(uint32_t abase, uint32_t t_addr, int q, int lane, int c0, float2 kc, int base)
{
    float v[32];
    tmem_ld_frag32(t_addr, v);
    const int i8 = lane & 7, j = lane >> 3;
    uint32_t pk[16];
#pragma unroll
    for (int g = 0; g < 4; ++g) {
        const int pi = base + 4 * g + (lane & 3);
        const uint64_t b2 = f2(__shfl_sync(0xffffffffu, kc.x, pi), __shfl_sync(0xffffffffu, kc.y, pi));
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int vi = 16 * (k >> 1) + 4 * g + 2 * (k & 1);
            pk[4 * k + g] = bf16x2(f2_add(f2(v[vi], v[vi + 1]), b2));
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
        stmatrix_x4(act_addr(abase, q * 32 + 16 * (k >> 1) + 8 * (k & 1) + i8, (c0 >> 3) + j), pk[4 * k + 0],
                    pk[4 * k + 1], pk[4 * k + 2], pk[4 * k + 3]);
}

__global__ void __launch_bounds__(NUM_THREADS, 1)
    mlp_tc_block_kernel(const __grid_constant__ CUtensorMap wmap, const __grid_constant__ CUtensorMap xmap, CallArgs A,
                        DevWeights Wt, int n_tiles)
{
    extern __shared__ __align__(1024) unsigned char dsm_raw[];
    unsigned char* dsm =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(dsm);
    const uint32_t abase = sbase;
    const uint32_t w_base = sbase + OFF_W;
    const uint32_t bar0 = sbase + OFF_BAR;
    float* red = reinterpret_cast<float*>(dsm + OFF_RED);
    auto full_bar = [&](int s) { return bar0 + 8 * s; };
    auto empty_bar = [&](int s) { return bar0 + 8 * (STAGES + s); };
    // acc_bar(0): the first output half is final and the first input half consumed by both halves;
    // acc_bar(1): the whole block (layer 0: acc_bar(e) after the x entry of half e).
    // epi_bar(e), 16 warps: column half e of the next input written; ahead of a tile's layer 0, the
    // half's TMEM and input columns free (after the previous tile's last block, or at the start)
    auto acc_bar = [&](int e) { return bar0 + 8 * (2 * STAGES + e); };
    auto epi_bar = [&](int e) { return bar0 + 8 * (2 * STAGES + 2 + e); };
    const uint32_t drain_bar = bar0 + 8 * (2 * STAGES + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(dsm + OFF_MISC);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(dsm + OFF_MISC + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_mine =
        n_tiles > (int)blockIdx.x ? (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    const int L = A.L;

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int e = 0; e < 2; ++e) {
            mbar_init(acc_bar(e), 1);
            mbar_init(epi_bar(e), NUM_EPI_WARPS);
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
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ producer (whole warp; lane 0 issues the copies)
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&wmap)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&xmap)) : "memory");
        }
        int stage = 0;
        uint32_t phase = 0, armed = 0, armed_par = 0;
        bool ok = true;
        auto advance = [&]() {
            armed |= 1u << stage;
            armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
            if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        };
        for (int i = 0; i < n_mine && ok; ++i) {
            // the tile's x rows lane + 32 j in three bfloat16 parts, x = x_hi + x_mid + x_lo (each part
            // the nearest bfloat16 of what the previous ones leave, the remainders exact in FP32; x to
            // about 2^-24 relative), as pairs (x_hi, y_hi), (z_hi, x_mid), (y_mid, z_mid), (x_lo, y_lo),
            // (z_lo, 0)
            uint32_t xw[4][5];
            {
                const int t = (int)blockIdx.x + i * (int)gridDim.x;
                const int m = find_segment(A.tile_off, A.M, t);
                const long long p0 = A.pbeg[m] + (long long)(t - A.tile_off[m]) * TM, pe = A.pend[m];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const long long p = p0 + lane + 32 * j;
                    const float4 x = p < pe ? ld_stream_f4(A.points + p) : make_float4(0.f, 0.f, 0.f, 0.f);
                    float hi[3], mid[3], lo[3];
                    const float xs[3] = {x.x, x.y, x.z};
#pragma unroll
                    for (int c = 0; c < 3; ++c) {
                        hi[c] = __bfloat162float(__float2bfloat16_rn(xs[c]));
                        const float r1 = xs[c] - hi[c];
                        mid[c] = __bfloat162float(__float2bfloat16_rn(r1));
                        lo[c] = r1 - mid[c];
                    }
                    xw[j][0] = pack_bf16<false>(hi[0], hi[1]);
                    xw[j][1] = pack_bf16<false>(hi[2], mid[0]);
                    xw[j][2] = pack_bf16<false>(mid[1], mid[2]);
                    xw[j][3] = pack_bf16<false>(lo[0], lo[1]);
                    xw[j][4] = pack_bf16<false>(lo[2], 0.0f);
                }
            }
            // layer l = 0 is the initial layer: an x entry per half and nothing else; blocks 2..L
            // have an x entry ahead of each half's slices; block 1 has none (its x-weight rows hold the
            // initial layer's)
            for (int l = 0; l <= L && ok; ++l)
                for (int h = 0; h < 2 && ok; ++h) {
                    if (l != 1) {
                        // x entry: the x rows (generic stores, then the proxy fence), then the x-weights
                        if (!mbar_wait_warp(empty_bar(stage), phase ^ 1u, abort_flag, A.dev_err)) { ok = false; break; }
                        const uint32_t sb = w_base + stage * STAGE_BYTES;
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const int r = lane + 32 * j;
                            st_shared_v4(sb + XT_OFF + swz32(r, 0), xw[j][0], xw[j][1], xw[j][2], xw[j][3]);
                            st_shared_v4(sb + XT_OFF + swz32(r, 1), xw[j][4], 0u, 0u, 0u);
                        }
                        fence_async_smem();
                        __syncwarp();
                        if (lane == 0) {
                            mbar_arrive_tx(full_bar(stage), XW_BYTES);
                            tma_load_2d(sb, &xmap, 0, (l == 0 ? 0 : (l - 1) * WB) + h * NH, full_bar(stage));
                        }
                        advance();
                    }
                    for (int kk = 0; kk < (l == 0 ? 0 : KSL); ++kk) {
                        if (!mbar_wait_warp(empty_bar(stage), phase ^ 1u, abort_flag, A.dev_err)) { ok = false; break; }
                        if (lane == 0) {
                            mbar_arrive_tx(full_bar(stage), STAGE_BYTES);
                            tma_load_2d(w_base + stage * STAGE_BYTES, &wmap, kk * BK, (l - 1) * WB + h * NH,
                                        full_bar(stage));
                        }
                        advance();
                    }
                }
        }
        // wait (bounded) for every copy this warp started
        if (lane == 0)
            for (int s = 0; s < STAGES; ++s)
                if (armed & (1u << s)) {
                    const uint32_t par = (armed_par >> s) & 1u;
                    const uint64_t t0 = globaltimer();
                    while (!mbar_try(full_bar(s), par) && globaltimer() - t0 < kTimeoutNs) {
                    }
                }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------ MMA issuer
        // Per block: [N-half 0: x entry, K 0-3] (needs input half 0), [N-half 0, K 4-7] (needs input
        // half 1), [N-half 1: x entry, K 0-3], commit acc_bar(0), [N-half 1, K 4-7], commit acc_bar(1);
        // block 1 has no x entries.  The epilogue of output half 0 then overlaps the last quarter of the
        // block's MMAs, and the next block's first quarter waits only for it.
        const uint64_t a_desc0 = sdesc(abase), b_desc0 = sdesc(w_base);
        int stage = 0;
        uint32_t phase = 0, ep0 = 0, ep1 = 0;
        bool ok = true;
        // the x entry of half h: D = x rows x x-weights (overwrites the half's accumulator)
        auto x_entry = [&](int h) {
            if (!mbar_wait_warp(full_bar(stage), phase, abort_flag, A.dev_err)) { ok = false; return; }
            tc_fence_after();
            const uint32_t sb = w_base + stage * STAGE_BYTES;
            mma_f16_warp(tmem_base + (uint32_t)(h * NH), sdesc32(sb + XT_OFF), sdesc32(sb), IDESC, 0u);
            mma_commit_warp(empty_bar(stage));
            if (++stage == STAGES) { stage = 0; phase ^= 1u; }
        };
        auto quarter_block = [&](int h, int k0, bool accumulate) {
            const uint32_t d_tmem = tmem_base + (uint32_t)(h * NH);
            for (int kk = k0; kk < k0 + KSL / 2; ++kk) {
                if (!mbar_wait_warp(full_bar(stage), phase, abort_flag, A.dev_err)) { ok = false; return; }
                tc_fence_after();
                const uint64_t ad = a_desc0 + (uint64_t)(kk * (KBLOCK_BYTES >> 4));
                const uint64_t bd = b_desc0 + (uint64_t)(stage * (STAGE_BYTES >> 4));
#pragma unroll
                for (int k = 0; k < 4; ++k)
                    mma_f16_warp(d_tmem, ad + 2 * k, bd + 2 * k, IDESC, (accumulate || (kk | k) != 0) ? 1u : 0u);
                mma_commit_warp(empty_bar(stage));
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
        };
        for (int i = 0; i < n_mine && ok; ++i)
            for (int l = 0; l <= L && ok; ++l) {
                if (l == 0) {
                    // the initial layer's x-part, one x entry per half, each half once its TMEM and its
                    // input columns are free
                    for (int h = 0; h < 2 && ok; ++h) {
                        if (!mbar_wait_warp(epi_bar(h), h == 0 ? ep0 : ep1, abort_flag, A.dev_err)) { ok = false; break; }
                        if (h == 0) ep0 ^= 1u;
                        else ep1 ^= 1u;
                        tc_fence_after();
                        x_entry(h);
                        if (ok) mma_commit_warp(acc_bar(h));
                    }
                    continue;
                }
                const bool xe = l >= 2;
                if (!mbar_wait_warp(epi_bar(0), ep0, abort_flag, A.dev_err)) { ok = false; break; }
                ep0 ^= 1u;
                tc_fence_after();
                if (xe) x_entry(0);
                if (ok) quarter_block(0, 0, xe);
                if (!ok) break;
                if (!mbar_wait_warp(epi_bar(1), ep1, abort_flag, A.dev_err)) { ok = false; break; }
                ep1 ^= 1u;
                tc_fence_after();
                quarter_block(0, KSL / 2, true);
                if (ok && xe) x_entry(1);
                if (ok) quarter_block(1, 0, xe);
                if (ok) mma_commit_warp(acc_bar(0));
                if (ok) quarter_block(1, KSL / 2, true);
                if (ok) mma_commit_warp(acc_bar(1));
            }
        // every MMA issued by this warp has completed before TMEM is freed
        mma_commit_warp(drain_bar);
        const uint64_t t0 = globaltimer();
        while (!mbar_try(drain_bar, 0u) && globaltimer() - t0 < kTimeoutNs) {
        }
        __syncwarp();
    } else {
        // ------------------------------------------------ epilogue warps
        const int q = warp & 3;                      // TMEM lane quarter: rows 32 q ..
        const int cq = (warp - 2) >> 2;              // columns 64 cq .. of each column half
        const int r = q * 32 + lane;                 // this lane's row (gate, reduction)
        const uint32_t t_row = tmem_base + ((uint32_t)(q * 32) << 16);
        const int cbs = A.cb_stride;
        uint32_t acc_phase = 0;
        bool ok = true;
        // tile i of this CTA: motion, first point, end of the motion's range
        auto tile_of = [&](int i, int& m, long long& p0, long long& pe) {
            const int t = (int)blockIdx.x + i * (int)gridDim.x;
            m = find_segment(A.tile_off, A.M, t);
            p0 = A.pbeg[m] + (long long)(t - A.tile_off[m]) * TM;
            pe = A.pend[m];
        };
        // layer 0 of the tile of motion m_: h_0 = (W_0x x from the accumulator) + c_0, per column half, then
        // the half's arrival.  c_0 of the warp's 64 columns of a half: one pair per lane.
        auto l0_pass = [&](int m_) {
            const float* c0m = A.cbias + (long long)m_ * cbs;
            for (int e = 0; e < 2 && ok; ++e) {
                const int c0 = e * NH + 64 * cq;
                const float2 kc = ldg2(c0m + c0 + 2 * lane);
                if (!mbar_wait(acc_bar(e), acc_phase, abort_flag, A.dev_err)) { ok = false; break; }
                tc_fence_after();
                h0_chunk(abase, t_row + (uint32_t)c0, q, lane, c0, kc, 0);
                h0_chunk(abase, t_row + (uint32_t)(c0 + 32), q, lane, c0 + 32, kc, 16);
                fence_async_smem();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(epi_bar(e));
            }
            acc_phase ^= 1u;
        };
        int m = 0;
        long long p0 = 0, pe = 0;
        if (n_mine > 0) {
            tile_of(0, m, p0, pe);
            // the TMEM and the input tile are free: the first tile's layer 0 may start
            if (!(A.test_stall && blockIdx.x == 0) && lane == 0) {
                mbar_arrive(epi_bar(0));
                mbar_arrive(epi_bar(1));
            }
            l0_pass(m);
        }
        for (int i = 0; i < n_mine && ok; ++i) {
            const bool has_next = i + 1 < n_mine;
            const float* cm = A.cbias + (long long)m * cbs;
            for (int l = 1; l <= L && ok; ++l) {
                const float* cl = cm + (long long)l * WB;
                const float* crec = Wt.blk_pk + (long long)(l - 1) * WB * 2;   // [W/2][4] of block l
                uint64_t acc4[4] = {0ull, 0ull, 0ull, 0ull};
                // column half e: its accumulator is final (and for e = 0 input half 0 read by both MMA
                // halves); the next block's input half e, or on the last block the final layer's partial
                // sums; then the half is handed over (on the last block to the next tile's layer 0)
                for (int e = 0; e < 2 && ok; ++e) {
                    const int c0 = e * NH + 64 * cq;
                    float4 ka0, ka1;
                    float2 kb0, kb1;
                    chunk_consts(lane, c0, cl, crec, Wt.wout, l == L, ka0, kb0);
                    chunk_consts(lane, c0 + 32, cl, crec, Wt.wout, l == L, ka1, kb1);
                    if (!mbar_wait(acc_bar(e), acc_phase, abort_flag, A.dev_err)) { ok = false; break; }
                    tc_fence_after();
                    if (l < L) {
                        block_chunk<false>(abase, t_row + (uint32_t)c0, q, lane, c0, ka0, kb0, acc4);
                        block_chunk<false>(abase, t_row + (uint32_t)(c0 + 32), q, lane, c0 + 32, ka1, kb1, acc4);
                    } else {
                        block_chunk<true>(abase, t_row + (uint32_t)c0, q, lane, c0, ka0, kb0, acc4);
                        block_chunk<true>(abase, t_row + (uint32_t)(c0 + 32), q, lane, c0 + 32, ka1, kb1, acc4);
                    }
                    if (l < L || has_next) {
                        fence_async_smem();
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(epi_bar(e));
                    }
                }
                acc_phase ^= 1u;
                if (l < L || !ok) continue;
                // ---- the final layer
                float sk[4];
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    float lo, hi;
                    f2_split(acc4[k], lo, hi);
                    sk[k] = lo + hi;
                    sk[k] += __shfl_xor_sync(0xffffffffu, sk[k], 1);
                    sk[k] += __shfl_xor_sync(0xffffffffu, sk[k], 2);
                }
                // row 16 (k >> 1) + 8 (k & 1) + t / 4 of the quarter is in sk[k] of thread 4 (t / 4) ..:
                // lane L takes row L, k = L / 8, from thread 4 (L % 8)
                float f = 0.0f;
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float v = __shfl_sync(0xffffffffu, sk[k], 4 * (lane & 7));
                    if ((lane >> 3) == k) f = v;
                }
                // the next tile's layer 0 first (its MMAs ran meanwhile), so that this tile's reduction and
                // gate overlap the next tile's first block
                int nm = 0;
                long long np0 = 0, npe = 0;
                if (has_next) {
                    tile_of(i + 1, nm, np0, npe);
                    l0_pass(nm);
                    if (!ok) break;
                }
                // the four column quarters of a row meet in shared memory
                if (cq > 0) red[(cq - 1) * TM + r] = f;
                named_sync(1 + q, 128);
                if (cq == 0) {
                    const long long p = p0 + r;
                    const bool valid = p < pe;
                    const float4 xr = valid ? ld_stream_f4(A.points + p) : make_float4(0.f, 0.f, 0.f, 0.f);
                    f += red[r] + red[TM + r] + red[2 * TM + r];
                    f = fmaf(__ldg(Wt.out_wx + 2), xr.z, fmaf(__ldg(Wt.out_wx + 1), xr.y, fmaf(__ldg(Wt.out_wx), xr.x, f)));
                    f += __ldg(cm + (long long)(L + 1) * WB);
                    // gate, compaction, per-motion minima (as in mlp_tc.cu)
                    if (A.f_out != nullptr && valid) A.f_out[(long long)m * A.f_stride + (p - A.pbeg[m])] = f;
                    const bool flag = valid && f <= A.gate;
                    const unsigned mask = __ballot_sync(0xffffffffu, flag);
                    unsigned base = 0;
                    if (lane == 0 && mask) base = atomicAdd(&A.st[m].n_flagged, (unsigned)__popc(mask));
                    base = __shfl_sync(0xffffffffu, base, 0);
                    if (flag) A.idx[A.pair_off[m] + base + __popc(mask & ((1u << lane) - 1u))] = (unsigned)p;
                    float fm = valid ? f : __int_as_float(0x7f800000);
#pragma unroll
                    for (int sh = 16; sh > 0; sh >>= 1) fm = fminf(fm, __shfl_xor_sync(0xffffffffu, fm, sh));
                    if (lane == 0 && fm < __int_as_float(0x7f800000)) atomicMin(&A.st[m].dhat_key, float_key(fm));
                    if (fm <= A.gate) {
                        const unsigned who = __ballot_sync(0xffffffffu, valid && f == fm);
                        const unsigned pi = __shfl_sync(0xffffffffu, (unsigned)p, __ffs(who) - 1);
                        if (lane == 0) atomicMin(&A.st[m].probe_key, ((unsigned long long)float_key(fm) << 32) | pi);
                    }
                }
                // the reduction buffer is read before any warp of the quarter can write the next tile's sums
                named_sync(5 + q, 128);
                if (has_next) {
                    m = nm;
                    p0 = np0;
                    pe = npe;
                }
            }
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

EncodeFn encode_fn()
{
    static EncodeFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) ==
                cudaSuccess &&
            qr == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeFn>(p);
    }
    return fn;
}

}  // namespace

int tc_block_prepare(TcModel& t, const svm_model_desc& d, const void* wh)
{
    t.ready = false;
    t.prec = d.prec;
    t.act = d.act;
    t.arch = SVM_ARCH_BLOCKS;
    EncodeFn enc = encode_fn();
    if (!enc || d.width != WB || d.prec != SVM_BF16 || d.act != SVM_RELU || !wh) return -1;
    // the blocks' h-weights, [L * 512 rows (outputs)][512 (inputs, K)] bfloat16
    const cuuint64_t dims[2] = {(cuuint64_t)WB, (cuuint64_t)WB * d.n_hidden};
    const cuuint64_t strides[1] = {(cuuint64_t)WB * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)NH};
    const cuuint32_t estr[2] = {1, 1};
    if (enc(reinterpret_cast<CUtensorMap*>(t.wmap), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(wh), dims,
            strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return -2;
    // their padded jump x-weights after them, [L * 512 rows][16] bfloat16: boxes of 256 rows x 32 bytes
    const void* wx = static_cast<const char*>(wh) + (size_t)d.n_hidden * WB * WB * 2;
    const cuuint64_t xdims[2] = {16, (cuuint64_t)WB * d.n_hidden};
    const cuuint64_t xstrides[1] = {32};
    const cuuint32_t xbox[2] = {16, (cuuint32_t)NH};
    if (enc(reinterpret_cast<CUtensorMap*>(t.w1map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(wx), xdims,
            xstrides, xbox, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return -2;
    t.ready = true;
    return 0;
}

int tc_block_launch(const TcModel& t, const CallArgs& a, const DevWeights& w, int n_tiles, int grid, cudaStream_t s)
{
    if (!t.ready || t.arch != SVM_ARCH_BLOCKS) return -1;
    if (n_tiles <= 0) return 0;
    int dev = 0;
    cudaGetDevice(&dev);
    static std::once_flag done[64];            // once per device, safe across host threads
    if (dev >= 0 && dev < 64)
        std::call_once(done[dev], [] {
            cudaFuncSetAttribute(mlp_tc_block_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_DYN);
        });
    if (grid > n_tiles) grid = n_tiles;
    mlp_tc_block_kernel<<<grid, NUM_THREADS, SMEM_DYN, s>>>(*reinterpret_cast<const CUtensorMap*>(t.wmap),
                                                             *reinterpret_cast<const CUtensorMap*>(t.w1map), a, w,
                                                             n_tiles);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace svm
