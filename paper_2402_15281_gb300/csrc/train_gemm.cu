// train_gemm.cu -- BF16 tcgen05 GEMM of the training step, D = A B^T with A
// [M][K] and B [N][K] both K-major (row-major, K contiguous) in global memory,
// FP32 accumulation in TMEM, and three fused epilogues:
//
//   FWD    hidden layer forward, rows = samples:  z = acc + b, h = act(z),
//          d = act'(z); writes H [M][N] (the next layer's A) and D [M][N]
//          (bfloat16, both rounded once from the FP32 z).  ReLU writes only
//          H: its d is [h > 0] of the stored h.
//   DGRAD  input gradient, rows = samples:  g = acc * d_prev; writes G [M][N]
//          (bfloat16).  ReLU reads H_prev and multiplies by [h_prev > 0], the
//          same factor as its D (0 or 1).
//   WGRAD  weight gradient dW = G^T H over a slice of the batch (split-K):
//          stores the FP32 partial of split s into dW + s * M * N ([M][N]);
//          the splits are summed afterwards in a fixed order, so the result
//          does not depend on the order in which CTAs finish.  G and H are
//          read as stored, [batch][features], as MN-major operands: per stage
//          64 x 64 boxes (64 features of 64 batch rows, 128B swizzle), the
//          descriptor's LBO the 8 KB between boxes along M / N and SBO the
//          1 KB between 8-row groups along K (the K = batch step of one MMA
//          is 16 rows, 2 KB); the instruction descriptor marks A and B
//          MN-major.
//
// Persistent kernel, one CTA per SM, 10 warps: warp 0 streams A and B tiles
// (128 x 64 and 256 x 64 bfloat16, 128B swizzle) with TMA into a 4-stage
// ring; warp 1 issues tcgen05.mma (M = 128, N = 256, K = 16; warp-uniform
// loop, one elected lane) into one of two
// TMEM accumulators; warps 2-9 drain the other accumulator (two warps per TMEM
// lane quarter, 128 columns each), so the epilogue of one tile overlaps the
// MMAs of the next.  Outputs leave by TMA: a warp writes its 32-row block
// (64 bfloat16 or 32 FP32 columns, 128 bytes a row) into its own 4 KB buffer
// in the 128-byte-swizzled layout -- row-per-lane 16-byte stores free of bank
// conflicts -- and one lane issues a tensor store of the box, so no global
// store passes through the load/store unit.  The D input of DGRAD (ReLU: the
// previous layer's H) is read
// with coalesced 16-byte loads (eight lanes per 128-byte row) one block
// ahead, and transposed to a row per lane through the same buffer.
// All mbarrier waits are bounded (see tc_ptx.cuh).
#include <mutex>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include "tc_ptx.cuh"
#include "train_internal.cuh"

namespace svm {

namespace {

using namespace ptx;

constexpr int BM = 128, BN = 256, BK = 64;
constexpr int STAGES = 4;
constexpr int A_BYTES = BM * BK * 2;
constexpr int B_BYTES = BN * BK * 2;
constexpr int STAGE_BYTES = A_BYTES + B_BYTES;
constexpr int EPI_WARPS = 8;
constexpr int THREADS = (2 + EPI_WARPS) * 32;
constexpr int BUF_BYTES = 32 * 128;                   // a warp's output box: 32 rows x 128 bytes
constexpr int OFF_BUF = STAGES * STAGE_BYTES;          // 1024-byte aligned (the swizzle period)
constexpr int OFF_BIAS = OFF_BUF + EPI_WARPS * BUF_BYTES;     // FWD: the CTA's 256 bias values
constexpr int OFF_BAR = OFF_BIAS + BN * 4;
constexpr int N_BARS = 2 * STAGES + 5;
constexpr int OFF_MISC = OFF_BAR + 8 * N_BARS;
constexpr int SMEM_DYN = OFF_MISC + 16 + 1024;
static_assert(SMEM_DYN <= 232448, "shared memory budget");
constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(BN >> 3) << 17) |
                           ((uint32_t)(BM >> 4) << 24);
// the same with A and B MN-major (bits 15 and 16)
constexpr uint32_t IDESC_MN = IDESC | (1u << 15) | (1u << 16);
constexpr int MN_BOX_BYTES = 64 * BK * 2;                 // one 64-feature x 64-row box

// Shared-memory descriptor of an MN-major operand, 128B swizzle: LBO = bytes
// between 64-element boxes along M / N, SBO = bytes between 8-row groups along K.
__device__ __forceinline__ uint64_t sdesc_mn(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)(MN_BOX_BYTES >> 4) << 16;   // LBO
    d |= (uint64_t)(1024 >> 4) << 32;           // SBO
    d |= (uint64_t)1 << 46;                     // version
    d |= (uint64_t)2 << 61;                     // SWIZZLE_128B
    return d;
}

__device__ __forceinline__ uint32_t bf2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

// h = act(z) and d = act'(z).  SiLU: with s = 1 / (1 + e^-z) (fast
// reciprocal, within a few ulp of the division), h = z s and d = s (1 + z (1 - s)).
// ReLU: d = 1 where the bfloat16 z is positive, else 0.
template <int ACT>
__device__ __forceinline__ void act_hd(float z, float& h, float& d)
{
    if constexpr (ACT == 0) {
        h = fmaxf(z, 0.0f);
        d = __bfloat162float(__float2bfloat16_rn(z)) > 0.0f ? 1.0f : 0.0f;
    } else {
        const float s = __fdividef(1.0f, 1.0f + __expf(-z));
        h = z * s;
        d = s * (1.0f + z * (1.0f - s));
    }
}

// Byte offset of 16-byte piece j of row r in a 128-byte-swizzled box (the
// layout TMA reads for CU_TENSOR_MAP_SWIZZLE_128B with 128-byte rows).
__device__ __forceinline__ int swz(int r, int j) { return r * 128 + ((j ^ (r & 7)) << 4); }

__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, uint32_t src, int x, int y)
{
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group [%0, {%1, %2}], [%3];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(src)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <int EPI, int ACT>
__global__ void __launch_bounds__(THREADS, 1)
    train_gemm_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap,
                      const __grid_constant__ CUtensorMap smap0, const __grid_constant__ CUtensorMap smap1, GemmArgs g)
{
    extern __shared__ __align__(1024) unsigned char dsm_raw[];
    unsigned char* dsm =
        reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(dsm);
    const uint32_t bar0 = sbase + OFF_BAR;
    auto full_bar = [&](int s) { return bar0 + 8 * s; };
    auto empty_bar = [&](int s) { return bar0 + 8 * (STAGES + s); };
    auto accf_bar = [&](int b) { return bar0 + 8 * (2 * STAGES + b); };
    auto acce_bar = [&](int b) { return bar0 + 8 * (2 * STAGES + 2 + b); };
    const uint32_t drain_bar = bar0 + 8 * (2 * STAGES + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(dsm + OFF_MISC);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(dsm + OFF_MISC + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_units = g.n_ks * g.n_mt * g.n_nt;
    const int n_mine =
        n_units > (int)blockIdx.x ? (n_units - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    // K slices of split ks: k_len, the last split k_last (the splits of WGRAD cover the batch exactly)
    const int k_last = g.k_last > 0 ? g.k_last : g.k_len;
    auto k_slices_of = [&](int ks) { return (ks == g.n_ks - 1 ? k_last : g.k_len) / BK; };

    if (threadIdx.x == 0) {
        for (int s = 0; s < STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(accf_bar(b), 1);
            mbar_init(acce_bar(b), EPI_WARPS);
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

    auto unit_coords = [&](int i, int& ks, int& mt, int& nt) {
        const int u = (int)blockIdx.x + i * (int)gridDim.x;
        nt = u % g.n_nt;
        mt = (u / g.n_nt) % g.n_mt;
        ks = u / (g.n_nt * g.n_mt);
    };

    if (warp == 0) {
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&amap)) : "memory");
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&bmap)) : "memory");
            int stage = 0;
            uint32_t phase = 0, armed = 0, armed_par = 0;
            bool ok = true;
            for (int i = 0; i < n_mine && ok; ++i) {
                int ks, mt, nt;
                unit_coords(i, ks, mt, nt);
                const int k0 = ks * g.k_len;
                const int k_slices = k_slices_of(ks);
                for (int kk = 0; kk < k_slices; ++kk) {
                    if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, g.err)) { ok = false; break; }
                    mbar_arrive_tx(full_bar(stage), STAGE_BYTES);
                    const uint32_t dst = sbase + stage * STAGE_BYTES;
                    if constexpr (EPI == kEpiWgrad) {
                        // MN-major: boxes of 64 features x 64 batch rows, consecutive along M / N
                        for (int j = 0; j < BM / 64; ++j)
                            tma_load_2d(dst + j * MN_BOX_BYTES, &amap, mt * BM + 64 * j, k0 + kk * BK, full_bar(stage));
                        for (int j = 0; j < BN / 64; ++j)
                            tma_load_2d(dst + A_BYTES + j * MN_BOX_BYTES, &bmap, nt * BN + 64 * j, k0 + kk * BK,
                                        full_bar(stage));
                    } else {
                        tma_load_2d(dst, &amap, k0 + kk * BK, mt * BM, full_bar(stage));
                        tma_load_2d(dst + A_BYTES, &bmap, k0 + kk * BK, nt * BN, full_bar(stage));
                    }
                    armed |= 1u << stage;
                    armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
                    if (++stage == STAGES) { stage = 0; phase ^= 1u; }
                }
            }
            for (int s = 0; s < STAGES; ++s)
                if (armed & (1u << s)) {
                    const uint32_t par = (armed_par >> s) & 1u;
                    const uint64_t t0 = globaltimer();
                    while (!mbar_try(full_bar(s), par) && globaltimer() - t0 < kTimeoutNs) {
                    }
                }
        }
    } else if (warp == 1) {
        // warp-uniform issue loop, one elected lane issues; descriptors advance
        // by adding to the start-address field (32 B within a swizzle atom)
        int stage = 0;
        uint32_t phase = 0;
        uint32_t acce_phase0 = 0u, acce_phase1 = 0u;
        constexpr bool MN = EPI == kEpiWgrad;
        const uint64_t a_desc0 = MN ? sdesc_mn(sbase) : sdesc(sbase);
        const uint64_t b_desc0 = MN ? sdesc_mn(sbase + A_BYTES) : sdesc(sbase + A_BYTES);
        // one MMA step of K = 16: 32 bytes along a K-major row, 16 rows (2 KB) of an MN-major box
        constexpr uint64_t kstep = MN ? (16 * 128) >> 4 : 2;
        bool ok = true;
        for (int i = 0; i < n_mine && ok; ++i) {
            const int b = i & 1;
            uint32_t& ap = b == 0 ? acce_phase0 : acce_phase1;
            if (!mbar_wait_warp(acce_bar(b), ap ^ 1u, abort_flag, g.err)) { ok = false; break; }
            ap ^= 1u;
            tc_fence_after();
            const uint32_t d_tmem = tmem_base + (uint32_t)(b * BN);
            int ks, mt, nt;
            unit_coords(i, ks, mt, nt);
            const int k_slices = k_slices_of(ks);
            for (int kk = 0; kk < k_slices; ++kk) {
                if (!mbar_wait_warp(full_bar(stage), phase, abort_flag, g.err)) { ok = false; break; }
                tc_fence_after();
                const uint64_t ad = a_desc0 + (uint64_t)(stage * (STAGE_BYTES >> 4));
                const uint64_t bd = b_desc0 + (uint64_t)(stage * (STAGE_BYTES >> 4));
#pragma unroll
                for (int k = 0; k < BK / 16; ++k)
                    mma_f16_warp(d_tmem, ad + kstep * k, bd + kstep * k, MN ? IDESC_MN : IDESC, (kk | k) != 0 ? 1u : 0u);
                mma_commit_warp(empty_bar(stage));
                if (++stage == STAGES) { stage = 0; phase ^= 1u; }
            }
            if (ok) mma_commit_warp(accf_bar(b));
        }
        mma_commit_warp(drain_bar);
        const uint64_t t0 = globaltimer();
        while (!mbar_try(drain_bar, 0u) && globaltimer() - t0 < kTimeoutNs) {
        }
        __syncwarp();
    } else {
        const int ew = warp - 2;
        const int quarter = warp & 3;
        const int half = ew >> 2;
        unsigned char* buf = dsm + OFF_BUF + ew * BUF_BYTES;
        const uint32_t buf_s = smem_u32(buf);
        uint32_t accf_phase[2] = {0u, 0u};
        // the buffer is free once the previous tensor store has read it
        auto wait_buf = [&]() {
            if (lane == 0) bulk_wait_read();
            __syncwarp();
        };
        // the lanes' shared-memory writes, then one lane stores the box at (x, y)
        auto store_box = [&](const CUtensorMap* map, int x, int y) {
            fence_async_smem();
            __syncwarp();
            if (lane == 0) {
                tma_store_2d(map, buf_s, x, y);
                bulk_commit();
            }
        };
        // DGRAD: the D block (32 rows x 64 columns) of (unit, chunk), loaded one
        // chunk ahead; lane l holds piece l % 8 of rows l / 8 + 4 j
        uint4 dr[8];
        auto load_d = [&](int i, int c) {
            int ks, mt, nt;
            unit_coords(i, ks, mt, nt);
            const __nv_bfloat16* src =
                g.d_in + ((long long)mt * BM + quarter * 32) * g.ld_rows + nt * BN + half * 128 + c * 64;
#pragma unroll
            for (int j = 0; j < 8; ++j)
                dr[j] = __ldg(reinterpret_cast<const uint4*>(src + ((lane >> 3) + 4 * j) * g.ld_rows + (lane & 7) * 8));
        };
        if constexpr (EPI == kEpiDgrad) {
            if (n_mine > 0) load_d(0, 0);
        }
        // FWD: when every unit of this CTA has the same N tile (grid a multiple of
        // the N tiles), its 256 bias values are staged once in shared memory
        const float* bias_s = reinterpret_cast<const float*>(dsm + OFF_BIAS);
        const bool bias_staged = EPI == kEpiFwd && (int)gridDim.x % g.n_nt == 0;
        if (bias_staged) {
            const int nt0 = (int)blockIdx.x % g.n_nt;
            reinterpret_cast<float*>(dsm + OFF_BIAS)[ew * 32 + lane] = g.bias[nt0 * BN + ew * 32 + lane];
            asm volatile("bar.sync 1, %0;" ::"n"(EPI_WARPS * 32) : "memory");
        }
        for (int i = 0; i < n_mine; ++i) {
            const int b = i & 1;
            if (!mbar_wait(accf_bar(b), accf_phase[b], abort_flag, g.err)) break;
            accf_phase[b] ^= 1u;
            tc_fence_after();
            int ks, mt, nt;
            unit_coords(i, ks, mt, nt);
            const int m0 = mt * BM + quarter * 32;                     // first row of this warp
            const uint32_t t_row = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * BN + half * 128);
            if constexpr (EPI == kEpiWgrad) {
#pragma unroll 1
                for (int c = 0; c < 4; ++c) {
                    float v[32];
                    tmem_ld32(t_row + (uint32_t)(c * 32), v);
                    wait_buf();
#pragma unroll
                    for (int j = 0; j < 8; ++j)
                        *reinterpret_cast<float4*>(buf + swz(lane, j)) =
                            make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
                    store_box(&smap0, nt * BN + half * 128 + c * 32, ks * g.n_mt * BM + m0);
                }
            } else {
#pragma unroll 1
                for (int c = 0; c < 2; ++c) {
                    const int n0 = nt * BN + half * 128 + c * 64;
                    float v[64];
                    if constexpr (EPI == kEpiFwd) {
                        tmem_ld32(t_row + (uint32_t)(c * 64), *reinterpret_cast<float(*)[32]>(v));
                        tmem_ld32(t_row + (uint32_t)(c * 64 + 32), *reinterpret_cast<float(*)[32]>(v + 32));
#pragma unroll
                        for (int q = 0; q < 16; ++q) {
                            const float4 b4 = bias_staged
                                                  ? *reinterpret_cast<const float4*>(bias_s + half * 128 + c * 64 + 4 * q)
                                                  : __ldg(reinterpret_cast<const float4*>(g.bias + n0 + 4 * q));
                            v[4 * q + 0] += b4.x;
                            v[4 * q + 1] += b4.y;
                            v[4 * q + 2] += b4.z;
                            v[4 * q + 3] += b4.w;
                        }
                        if constexpr (ACT == 0) {
                            // ReLU: h = max(z, 0) only
#pragma unroll
                            for (int e = 0; e < 64; ++e) v[e] = fmaxf(v[e], 0.0f);
                        } else {
                            // D box from z, with h = act(z) left in v
                            wait_buf();
#pragma unroll
                            for (int j = 0; j < 8; ++j) {
                                float d[8];
#pragma unroll
                                for (int e = 0; e < 8; ++e) act_hd<ACT>(v[8 * j + e], v[8 * j + e], d[e]);
                                *reinterpret_cast<uint4*>(buf + swz(lane, j)) =
                                    make_uint4(bf2(d[0], d[1]), bf2(d[2], d[3]), bf2(d[4], d[5]), bf2(d[6], d[7]));
                            }
                            store_box(&smap0, n0, m0);                  // D
                        }
                        wait_buf();
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            *reinterpret_cast<uint4*>(buf + swz(lane, j)) =
                                make_uint4(bf2(v[8 * j], v[8 * j + 1]), bf2(v[8 * j + 2], v[8 * j + 3]),
                                           bf2(v[8 * j + 4], v[8 * j + 5]), bf2(v[8 * j + 6], v[8 * j + 7]));
                        store_box(&smap1, n0, m0);                      // H
                    } else {
                        wait_buf();
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            *reinterpret_cast<uint4*>(buf + swz((lane >> 3) + 4 * j, lane & 7)) = dr[j];
                        __syncwarp();
                        // the next D block is in flight while this one is used
                        if (c + 1 < 2) load_d(i, c + 1);
                        else if (i + 1 < n_mine) load_d(i + 1, 0);
                        // from here each lane reads and rewrites only its own row: g in place of d
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            float u[32];
                            tmem_ld32(t_row + (uint32_t)(c * 64 + hh * 32), u);
#pragma unroll
                            for (int jj = 0; jj < 4; ++jj) {
                                const int j = hh * 4 + jj;
                                const uint4 dv = *reinterpret_cast<const uint4*>(buf + swz(lane, j));
                                float* w = u + 8 * jj;
                                const float dd[8] = {bf_lo(dv.x), bf_hi(dv.x), bf_lo(dv.y), bf_hi(dv.y),
                                                     bf_lo(dv.z), bf_hi(dv.z), bf_lo(dv.w), bf_hi(dv.w)};
#pragma unroll
                                for (int e = 0; e < 8; ++e) w[e] *= ACT == 0 ? (dd[e] > 0.0f ? 1.0f : 0.0f) : dd[e];
                                *reinterpret_cast<uint4*>(buf + swz(lane, j)) =
                                    make_uint4(bf2(w[0], w[1]), bf2(w[2], w[3]), bf2(w[4], w[5]), bf2(w[6], w[7]));
                            }
                        }
                        store_box(&smap0, n0, m0);                      // G
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce_bar(b));
        }
        // the tensor stores have completed before the CTA ends
        if (lane == 0) bulk_wait_all();
        __syncwarp();
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
    }
}

template <int EPI, int ACT>
void launch_t(const CUtensorMap& a, const CUtensorMap& b, const CUtensorMap& s0, const CUtensorMap& s1,
              const GemmArgs& g, int grid, cudaStream_t s)
{
    int dev = 0;
    cudaGetDevice(&dev);
    static std::once_flag done[64];            // once per device, safe across host threads
    if (dev >= 0 && dev < 64)
        std::call_once(done[dev], [] {
            cudaFuncSetAttribute(train_gemm_kernel<EPI, ACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_DYN);
        });
    train_gemm_kernel<EPI, ACT><<<grid, THREADS, SMEM_DYN, s>>>(a, b, s0, s1, g);
}

}  // namespace

int train_gemm_bm() { return BM; }
int train_gemm_bn() { return BN; }
int train_gemm_bk() { return BK; }

// Tensor map of a row-major bfloat16 matrix [rows][cols] read in boxes of
// box_rows x 64 columns with the 128-byte swizzle.
int train_make_map(void* map, const void* base, long long rows, long long cols, int box_rows)
{
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    if (!enc) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return -1;
        enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    const cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(reinterpret_cast<CUtensorMap*>(map), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                           const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -2;
}

void launch_train_gemm(int epi, int act, const void* amap, const void* bmap, const void* smap0, const void* smap1,
                       const GemmArgs& g, int n_sms, cudaStream_t s)
{
    const int units = g.n_ks * g.n_mt * g.n_nt;
    if (units <= 0) return;
    const int grid = units < n_sms ? units : n_sms;
    const CUtensorMap& a = *reinterpret_cast<const CUtensorMap*>(amap);
    const CUtensorMap& b = *reinterpret_cast<const CUtensorMap*>(bmap);
    const CUtensorMap& s0 = *reinterpret_cast<const CUtensorMap*>(smap0);
    const CUtensorMap& s1 = *reinterpret_cast<const CUtensorMap*>(smap1 ? smap1 : smap0);
    if (epi == kEpiFwd) {
        if (act == 0) launch_t<kEpiFwd, 0>(a, b, s0, s1, g, grid, s); else launch_t<kEpiFwd, 1>(a, b, s0, s1, g, grid, s);
    } else if (epi == kEpiDgrad) {
        if (act == 0) launch_t<kEpiDgrad, 0>(a, b, s0, s1, g, grid, s);
        else launch_t<kEpiDgrad, 1>(a, b, s0, s1, g, grid, s);
    } else {
        launch_t<kEpiWgrad, 0>(a, b, s0, s1, g, grid, s);
    }
}

// Tensor map of a row-major [rows][cols] matrix written in boxes of 32 rows x
// 128 bytes (64 bfloat16 or 32 FP32 columns), 128-byte swizzle.
int train_make_store_map(void* map, const void* base, long long rows, long long cols, int fp32)
{
    static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
    if (!enc) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess)
            return -1;
        enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    const int es = fp32 ? 4 : 2;
    const cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)cols * es};
    const cuuint32_t box[2] = {(cuuint32_t)(128 / es), 32};
    const cuuint32_t estr[2] = {1, 1};
    const CUresult r = enc(reinterpret_cast<CUtensorMap*>(map),
                           fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                           const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_NONE,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? 0 : -2;
}

}  // namespace svm
