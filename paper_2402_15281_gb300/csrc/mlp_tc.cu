// mlp_tc.cu -- the network f(x, q0, q1) of Sec. IV-A on the 5th-generation
// tensor cores (tcgen05), BF16 or FP8 E4M3 operands with FP32 accumulation
// in tensor memory, fused with the gate and the compaction of flagged pairs.
//
// Persistent kernel, one CTA per SM, 10 warps:
//   warp 0      TMA producer: streams the hidden-layer weights, one 128-byte
//               wide K-slice (256 output rows) per stage, into a ring of
//               shared-memory stages (128B swizzle, K-major B operand);
//   warp 1      allocates the 512 TMEM columns and issues tcgen05.mma
//               (M = 128 pairs, N = 256 outputs) from one thread;
//   warps 2-5   epilogue of tile slot 0, warps 6-9 epilogue of slot 1.
// Each CTA takes tiles of 128 pairs of one motion and runs two of them at a
// time (slots 0 and 1, TMEM columns [0,256) and [256,512)), so that while the
// tensor core works on one slot's layer, the other slot's epilogue drains its
// accumulator: TMEM -> registers (tcgen05.ld) -> bias, activation, rounding
// -> the next layer's A operand in shared memory (128B swizzle, K-major).
//
// Layer 1 uses the split W1 [x; q0; q1] + b1 = W1x x + c_m: the epilogue warps
// compute it in FP32 from the point and the per-motion bias c_m.  The output
// layer W -> 1 is a dot product on the last accumulator in FP32.  Then the
// gate f <= margin + tau, a warp ballot and one atomicAdd per warp append the
// flagged point indices to the motion's list, and the motion's minimum
// prediction (Eq. 6) is kept with an atomic minimum.
//
// FP8: hidden weights and activations are E4M3 with per-layer scales; the
// accumulator is rescaled by s_w * s_a before the bias.  Both slots share
// every weight stage (REUSE = 2), so each weight byte is read once per pair
// of tiles.  BF16: the 128 KB layer does not fit twice, each slot streams it.
//
// Every mbarrier wait is bounded (2 s of %globaltimer); on expiry the waiter
// sets the call's error word and an abort flag, all roles leave their loops,
// the MMA issuer and the producer wait (bounded) for their own operations in
// flight, and the TMEM is freed before the CTA exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cudaTypedefs.h>

#include "mlp_tc.cuh"

namespace svm {

namespace {

constexpr int TM = 128;                    // pairs per tile = MMA M
constexpr int WN = 256;                    // network width = MMA N = hidden K
constexpr int NUM_WARPS = 10;
constexpr int NUM_THREADS = NUM_WARPS * 32;
constexpr int STAGE_BYTES = 32768;         // one 128-byte K-slice x 256 rows
constexpr int KBLOCK_BYTES = TM * 128;     // one 128-byte K-block of a 128-row tile
constexpr unsigned long long kTimeoutNs = 2000000000ull;
constexpr unsigned kErrTimeout = 1u;

template <int PREC>
struct Cfg;
template <>
struct Cfg<SVM_BF16> {
    static constexpr int ELEM = 2;
    static constexpr int SLICE_K = 64;                   // elements per 128-byte row
    static constexpr int SLICES = WN / SLICE_K;          // 4 per layer
    static constexpr int MMA_K = 16;
    static constexpr int MMAS = SLICE_K / MMA_K;         // 4 per slice
    static constexpr int STAGES = 3;
    static constexpr int REUSE = 1;
    // kind::f16: D f32 (bit 4), A bf16 (bits 7-9 = 1), B bf16 (bits 10-12 = 1),
    // both K-major, N >> 3 at bit 17, M >> 4 at bit 24
    static constexpr uint32_t IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(WN >> 3) << 17) |
                                      ((uint32_t)(TM >> 4) << 24);
};
template <>
struct Cfg<SVM_FP8_E4M3> {
    static constexpr int ELEM = 1;
    static constexpr int SLICE_K = 128;
    static constexpr int SLICES = WN / SLICE_K;          // 2 per layer
    static constexpr int MMA_K = 32;
    static constexpr int MMAS = SLICE_K / MMA_K;         // 4 per slice
    static constexpr int STAGES = 5;
    static constexpr int REUSE = 2;
    // kind::f8f6f4: D f32, A e4m3 (0), B e4m3 (0)
    static constexpr uint32_t IDESC = (1u << 4) | ((uint32_t)(WN >> 3) << 17) | ((uint32_t)(TM >> 4) << 24);
};

template <int PREC>
struct Smem {
    static constexpr int ACT_BYTES = TM * WN * Cfg<PREC>::ELEM;
    static constexpr int ACT0 = 0;
    static constexpr int W0 = 2 * ACT_BYTES;
    static constexpr int BARS = W0 + Cfg<PREC>::STAGES * STAGE_BYTES;
    static constexpr int N_BARS = 2 * Cfg<PREC>::STAGES + 5;
    static constexpr int MISC = BARS + 8 * N_BARS;
    static constexpr int TOTAL = MISC + 16;
    static constexpr int DYN = TOTAL + 1024;      // slack for 1024-byte alignment
};

// ------------------------------------------------------------ PTX wrappers

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ uint64_t globaltimer()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(bar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}" ::"r"(bar),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for the phase of `parity` to complete.  On expiry: record the
// error, raise the CTA's abort flag, return false.  Also returns false as
// soon as another role has aborted.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort_flag, unsigned* err)
{
    if (mbar_try(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    for (uint32_t it = 1;; ++it) {
        if (mbar_try(bar, parity)) return true;
        if ((it & 63u) == 0) {
            if (*abort_flag) return false;
            if (globaltimer() - t0 > kTimeoutNs) {
                atomicOr(err, kErrTimeout);
                *abort_flag = 1;
                return false;
            }
        }
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int c0, int c1, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// Shared-memory matrix descriptor: K-major operand, 128B swizzle, 8-row
// groups 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;                 // LBO (unused with 128B swizzle, K-major)
    d |= (uint64_t)(1024 >> 4) << 32;       // SBO
    d |= (uint64_t)1 << 46;                 // version
    d |= (uint64_t)2 << 61;                 // SWIZZLE_128B
    return d;
}

template <int PREC>
__device__ __forceinline__ void mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    if constexpr (PREC == SVM_BF16) {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(Cfg<PREC>::IDESC), "r"(accumulate)
            : "memory");
    } else {
        asm volatile(
            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
            " tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
            "l"(adesc), "l"(bdesc), "r"(Cfg<PREC>::IDESC), "r"(accumulate)
            : "memory");
    }
}

__device__ __forceinline__ void mma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 lanes x 32 consecutive FP32 columns of TMEM into 32 registers per thread.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d)
                 : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ uint32_t pack_e4m3x4(float a, float b, float c, float d)
{
    const uint32_t lo = __nv_cvt_float2_to_fp8x2(make_float2(a, b), __NV_SATFINITE, __NV_E4M3);
    const uint32_t hi = __nv_cvt_float2_to_fp8x2(make_float2(c, d), __NV_SATFINITE, __NV_E4M3);
    return (lo & 0xFFFFu) | (hi << 16);
}

// Address of 16-byte chunk `c` (0..7) of K-block `kb` in row `r` of a tile
// stored K-major with the 128B swizzle (the layout the MMA descriptor reads).
__device__ __forceinline__ uint32_t act_chunk_addr(uint32_t base, int kb, int r, int c)
{
    return base + kb * KBLOCK_BYTES + r * 128 + ((c ^ (r & 7)) << 4);
}

// Store 32 activations (columns o0..o0+31 of the next layer's input) of row r.
template <int PREC>
__device__ __forceinline__ void store_act32(uint32_t base, int r, int o0, const float (&h)[32], float inv_scale)
{
    if constexpr (PREC == SVM_BF16) {
        const int kb = o0 >> 6, c0 = (o0 & 63) >> 3;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            st_shared_v4(act_chunk_addr(base, kb, r, c0 + q), pack_bf16(h[8 * q + 0], h[8 * q + 1]),
                         pack_bf16(h[8 * q + 2], h[8 * q + 3]), pack_bf16(h[8 * q + 4], h[8 * q + 5]),
                         pack_bf16(h[8 * q + 6], h[8 * q + 7]));
    } else {
        const int kb = o0 >> 7, c0 = (o0 & 127) >> 4;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const float* g = h + 16 * q;
            st_shared_v4(act_chunk_addr(base, kb, r, c0 + q),
                         pack_e4m3x4(g[0] * inv_scale, g[1] * inv_scale, g[2] * inv_scale, g[3] * inv_scale),
                         pack_e4m3x4(g[4] * inv_scale, g[5] * inv_scale, g[6] * inv_scale, g[7] * inv_scale),
                         pack_e4m3x4(g[8] * inv_scale, g[9] * inv_scale, g[10] * inv_scale, g[11] * inv_scale),
                         pack_e4m3x4(g[12] * inv_scale, g[13] * inv_scale, g[14] * inv_scale, g[15] * inv_scale));
        }
    }
}

// ------------------------------------------------------------------ kernel

template <int PREC>
__global__ void __launch_bounds__(NUM_THREADS, 1)
    mlp_tc_kernel(const __grid_constant__ CUtensorMap wmap, CallArgs A, DevWeights Wt, int n_tiles)
{
    using C = Cfg<PREC>;
    using SM = Smem<PREC>;
    extern __shared__ __align__(1024) unsigned char dsm_raw[];
    unsigned char* dsm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
    const uint32_t sbase = smem_u32(dsm);
    const uint32_t act_base[2] = {sbase + SM::ACT0, sbase + SM::ACT0 + SM::ACT_BYTES};
    const uint32_t w_base = sbase + SM::W0;
    const uint32_t bar0 = sbase + SM::BARS;
    auto full_bar = [&](int s) { return bar0 + 8 * s; };
    auto empty_bar = [&](int s) { return bar0 + 8 * (C::STAGES + s); };
    auto accf_bar = [&](int s) { return bar0 + 8 * (2 * C::STAGES + s); };
    auto epid_bar = [&](int s) { return bar0 + 8 * (2 * C::STAGES + 2 + s); };
    const uint32_t drain_bar = bar0 + 8 * (2 * C::STAGES + 4);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(dsm + SM::MISC);
    volatile int* abort_flag = reinterpret_cast<volatile int*>(dsm + SM::MISC + 4);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int n_mine = n_tiles > (int)blockIdx.x ? (n_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
    const int n_pairs = (n_mine + 1) >> 1;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(full_bar(s), 1);
            mbar_init(empty_bar(s), 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(accf_bar(s), 1);
            mbar_init(epid_bar(s), 4);
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
        // ------------------------------------------------ TMA producer
        if (lane == 0) {
            asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&wmap)) : "memory");
            int stage = 0;
            uint32_t phase = 0;
            uint32_t armed = 0;            // bit s: stage s has been loaded at least once
            uint32_t armed_par = 0;        // bit s: parity of its last load
            bool ok = true;
            for (int j = 0; j < n_pairs && ok; ++j) {
                const int nslots = min(2, n_mine - 2 * j);
                for (int l = 0; l < A.L && ok; ++l) {
                    const int passes = C::REUSE == 2 ? 1 : nslots;
                    for (int s = 0; s < passes && ok; ++s)
                        for (int kk = 0; kk < C::SLICES; ++kk) {
                            if (!mbar_wait(empty_bar(stage), phase ^ 1u, abort_flag, A.dev_err)) { ok = false; break; }
                            mbar_arrive_tx(full_bar(stage), STAGE_BYTES);
                            tma_load_2d(w_base + stage * STAGE_BYTES, &wmap, kk * C::SLICE_K, l * WN, full_bar(stage));
                            armed |= 1u << stage;
                            armed_par = (armed_par & ~(1u << stage)) | (phase << stage);
                            if (++stage == C::STAGES) { stage = 0; phase ^= 1u; }
                        }
                }
            }
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
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            uint32_t epi_phase[2] = {0u, 0u};
            bool ok = true;
            for (int j = 0; j < n_pairs && ok; ++j) {
                const int nslots = min(2, n_mine - 2 * j);
                for (int l = 0; l < A.L && ok; ++l) {
                    const int layer_stage = stage;
                    const uint32_t layer_phase = phase;
                    for (int s = 0; s < nslots && ok; ++s) {
                        if (!mbar_wait(epid_bar(s), epi_phase[s], abort_flag, A.dev_err)) { ok = false; break; }
                        epi_phase[s] ^= 1u;
                        tc_fence_after();
                        if (C::REUSE == 2) { stage = layer_stage; phase = layer_phase; }
                        const uint32_t d_tmem = tmem_base + (uint32_t)(s * WN);
                        for (int kk = 0; kk < C::SLICES; ++kk) {
                            const bool first_use = C::REUSE == 1 || s == 0;
                            if (first_use) {
                                if (!mbar_wait(full_bar(stage), phase, abort_flag, A.dev_err)) { ok = false; break; }
                                tc_fence_after();
                            }
                            const uint32_t a0 = act_base[s] + kk * KBLOCK_BYTES;
                            const uint32_t b0 = w_base + stage * STAGE_BYTES;
#pragma unroll
                            for (int k = 0; k < C::MMAS; ++k)
                                mma<PREC>(d_tmem, sdesc(a0 + k * 32), sdesc(b0 + k * 32), (kk | k) != 0 ? 1u : 0u);
                            const bool last_use = C::REUSE == 1 || s == nslots - 1;
                            if (last_use) mma_commit(empty_bar(stage));
                            if (++stage == C::STAGES) { stage = 0; phase ^= 1u; }
                        }
                        if (ok) mma_commit(accf_bar(s));
                    }
                }
            }
            // every MMA issued by this thread has completed before TMEM is freed
            mma_commit(drain_bar);
            const uint64_t t0 = globaltimer();
            while (!mbar_try(drain_bar, 0u) && globaltimer() - t0 < kTimeoutNs) {
            }
        }
    } else {
        // ------------------------------------------------ epilogue warps
        const int ew = warp - 2;
        const int s = ew >> 2;                 // tile slot
        const int quarter = warp & 3;          // TMEM lane quarter this warp may access
        const int r = quarter * 32 + lane;     // row of the tile = TMEM lane
        const uint32_t t_row = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(s * WN);
        uint32_t acc_phase = 0;
        bool ok = true;
        for (int i = s; i < n_mine && ok; i += 2) {
            const int t = (int)blockIdx.x + i * (int)gridDim.x;
            const int m = find_segment(A.tile_off, A.M, t);
            const long long p = A.pbeg[m] + (long long)(t - A.tile_off[m]) * TM + r;
            const bool valid = p < A.pend[m];
            const float4 x = valid ? __ldg(A.points + p) : make_float4(0.f, 0.f, 0.f, 0.f);
            // ---- layer 1 in FP32: act(W1x x + c_m)
            {
                const float* cb = A.cbias + (long long)m * WN;
                const float inv0 = PREC == SVM_FP8_E4M3 ? 1.0f / __ldg(Wt.ascale) : 1.0f;
#pragma unroll 1
                for (int o0 = 0; o0 < WN; o0 += 32) {
                    float h[32];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const float4 w0 = __ldg(reinterpret_cast<const float4*>(Wt.w1x + (o0 + 4 * q) * 3));
                        const float4 w1 = __ldg(reinterpret_cast<const float4*>(Wt.w1x + (o0 + 4 * q) * 3 + 4));
                        const float4 w2 = __ldg(reinterpret_cast<const float4*>(Wt.w1x + (o0 + 4 * q) * 3 + 8));
                        const float4 c4 = __ldg(reinterpret_cast<const float4*>(cb + o0 + 4 * q));
                        h[4 * q + 0] = act_fn(fmaf(w0.z, x.z, fmaf(w0.y, x.y, fmaf(w0.x, x.x, c4.x))), A.act);
                        h[4 * q + 1] = act_fn(fmaf(w1.y, x.z, fmaf(w1.x, x.y, fmaf(w0.w, x.x, c4.y))), A.act);
                        h[4 * q + 2] = act_fn(fmaf(w2.x, x.z, fmaf(w1.w, x.y, fmaf(w1.z, x.x, c4.z))), A.act);
                        h[4 * q + 3] = act_fn(fmaf(w2.w, x.z, fmaf(w2.z, x.y, fmaf(w2.y, x.x, c4.w))), A.act);
                    }
                    store_act32<PREC>(act_base[s], r, o0, h, inv0);
                }
                fence_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(epid_bar(s));
            }
            // ---- hidden layers
            for (int l = 0; l < A.L; ++l) {
                if (!mbar_wait(accf_bar(s), acc_phase, abort_flag, A.dev_err)) { ok = false; break; }
                acc_phase ^= 1u;
                tc_fence_after();
                const float* bl = Wt.bh + (long long)l * WN;
                const float scale = PREC == SVM_FP8_E4M3 ? __ldg(Wt.wscale + l) * __ldg(Wt.ascale + l) : 1.0f;
                if (l + 1 < A.L) {
                    const float inv_next = PREC == SVM_FP8_E4M3 ? 1.0f / __ldg(Wt.ascale + l + 1) : 1.0f;
#pragma unroll 1
                    for (int o0 = 0; o0 < WN; o0 += 32) {
                        float v[32];
                        tmem_ld32(t_row + (uint32_t)o0, v);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const float4 b4 = __ldg(reinterpret_cast<const float4*>(bl + o0 + 4 * q));
                            v[4 * q + 0] = act_fn(fmaf(v[4 * q + 0], scale, b4.x), A.act);
                            v[4 * q + 1] = act_fn(fmaf(v[4 * q + 1], scale, b4.y), A.act);
                            v[4 * q + 2] = act_fn(fmaf(v[4 * q + 2], scale, b4.z), A.act);
                            v[4 * q + 3] = act_fn(fmaf(v[4 * q + 3], scale, b4.w), A.act);
                        }
                        store_act32<PREC>(act_base[s], r, o0, v, inv_next);
                    }
                    fence_async_smem();
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) mbar_arrive(epid_bar(s));
                } else {
                    float f = 0.0f;
#pragma unroll 1
                    for (int o0 = 0; o0 < WN; o0 += 32) {
                        float v[32];
                        tmem_ld32(t_row + (uint32_t)o0, v);
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const float4 b4 = __ldg(reinterpret_cast<const float4*>(bl + o0 + 4 * q));
                            const float4 w4 = __ldg(reinterpret_cast<const float4*>(Wt.wout + o0 + 4 * q));
                            f = fmaf(w4.x, act_fn(fmaf(v[4 * q + 0], scale, b4.x), A.act), f);
                            f = fmaf(w4.y, act_fn(fmaf(v[4 * q + 1], scale, b4.y), A.act), f);
                            f = fmaf(w4.z, act_fn(fmaf(v[4 * q + 2], scale, b4.z), A.act), f);
                            f = fmaf(w4.w, act_fn(fmaf(v[4 * q + 3], scale, b4.w), A.act), f);
                        }
                    }
                    tc_fence_before();
                    f += Wt.bout;
                    // gate, compaction, running minimum (one warp = 32 rows)
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

template <int PREC>
void configure(int dev)
{
    static bool done[64] = {};
    if (dev >= 0 && dev < 64 && !done[dev]) {
        cudaFuncSetAttribute(mlp_tc_kernel<PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize, Smem<PREC>::DYN);
        done[dev] = true;
    }
}

}  // namespace

int tc_tile_rows() { return TM; }

size_t tc_workspace_bytes(int) { return 256; }

int tc_prepare(TcModel& t, const svm_model_desc& d, const DevWeights& w)
{
    t.ready = false;
    t.prec = d.prec;
    EncodeFn enc = get_encode();
    if (!enc || d.width != WN) return -1;
    const int elem = d.prec == SVM_BF16 ? 2 : 1;
    const cuuint64_t dims[2] = {(cuuint64_t)WN, (cuuint64_t)WN * (cuuint64_t)d.n_hidden};
    const cuuint64_t strides[1] = {(cuuint64_t)WN * elem};
    const cuuint32_t box[2] = {(cuuint32_t)(128 / elem), (cuuint32_t)WN};
    const cuuint32_t estr[2] = {1, 1};
    CUtensorMap* map = reinterpret_cast<CUtensorMap*>(t.wmap);
    const CUresult r = enc(map, d.prec == SVM_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_UINT8, 2,
                           const_cast<void*>(w.wq), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return -2;
    t.ready = true;
    return 0;
}

void tc_release(TcModel& t) { t.ready = false; }

int tc_launch(TcModel& t, const CallArgs& a, const DevWeights& w, int n_tiles, void* ws, int n_sms, cudaStream_t s)
{
    (void)ws;
    if (!t.ready) return -1;
    if (n_tiles <= 0) return 0;
    int dev = 0;
    cudaGetDevice(&dev);
    const int grid = n_tiles < n_sms ? n_tiles : n_sms;
    const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(t.wmap);
    if (t.prec == SVM_BF16) {
        configure<SVM_BF16>(dev);
        mlp_tc_kernel<SVM_BF16><<<grid, NUM_THREADS, Smem<SVM_BF16>::DYN, s>>>(*map, a, w, n_tiles);
    } else {
        configure<SVM_FP8_E4M3>(dev);
        mlp_tc_kernel<SVM_FP8_E4M3><<<grid, NUM_THREADS, Smem<SVM_FP8_E4M3>::DYN, s>>>(*map, a, w, n_tiles);
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}

}  // namespace svm
