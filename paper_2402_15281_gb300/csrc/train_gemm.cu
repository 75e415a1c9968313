// train_gemm.cu -- BF16 tcgen05 GEMM of the training step, D = A B^T with A
// [M][K] and B [N][K] both K-major (row-major, K contiguous) in global memory,
// FP32 accumulation in TMEM, and three fused epilogues:
//
//   FWD    hidden layer forward, rows = samples:  z = acc + b, h = act(z);
//          writes H [M][N] (the next layer's A) and Z [M][N] (for act')
//          (bfloat16).
//   DGRAD  input gradient, rows = samples:  g = acc * act'(z_prev);
//          writes G [M][N] (bfloat16).
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
// MMAs of the next.  A warp's 32 x 32 blocks of bfloat16 outputs (and of
// the Z input of DGRAD) pass through a padded 32-row tile in shared memory:
// the accumulator gives a warp one row per lane, while global memory is
// written (and read) as 64-byte row segments, four lanes per row and eight
// rows per instruction -- full sectors and a quarter of the L1 wavefronts of
// row-per-lane accesses.
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
constexpr int TP_STRIDE = 80;                         // bytes per staging row (64 + 16 padding)
constexpr int TP_BYTES = 32 * TP_STRIDE;
constexpr int OFF_TP = STAGES * STAGE_BYTES;
constexpr int OFF_BAR = OFF_TP + EPI_WARPS * TP_BYTES;
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

__device__ __forceinline__ void st_global_v4(void* p, uint32_t a, uint32_t b, uint32_t c, uint32_t d)
{
    asm volatile("st.global.v4.b32 [%0], {%1, %2, %3, %4};" ::"l"(p), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}

__device__ __forceinline__ uint32_t bf2(float lo, float hi)
{
    const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<const uint32_t*>(&v);
}

__device__ __forceinline__ float bf_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf_hi(uint32_t w) { return __uint_as_float(w & 0xFFFF0000u); }

template <int ACT>
__device__ __forceinline__ float act_fwd(float z)
{
    if constexpr (ACT == 0) return fmaxf(z, 0.0f);
    else return __fdividef(z, 1.0f + __expf(-z));   // fast reciprocal: within a few ulp of the division
}

template <int ACT>
__device__ __forceinline__ float act_grad(float z)
{
    if constexpr (ACT == 0) return z > 0.0f ? 1.0f : 0.0f;
    else {
        const float s = __fdividef(1.0f, 1.0f + __expf(-z));
        return s * (1.0f + z * (1.0f - s));
    }
}

// The staging tile of a warp: 32 rows of 32 bfloat16 (64 bytes) at a
// stride of 80 bytes, so row-per-lane 16-byte accesses are free of bank
// conflicts.  stage_row: lane = row, v = its 32 values.
__device__ __forceinline__ void stage_row(unsigned char* tp, int lane, const float (&v)[32])
{
    uint4* d = reinterpret_cast<uint4*>(tp + lane * TP_STRIDE);
#pragma unroll
    for (int q = 0; q < 4; ++q)
        d[q] = make_uint4(bf2(v[8 * q], v[8 * q + 1]), bf2(v[8 * q + 2], v[8 * q + 3]), bf2(v[8 * q + 4], v[8 * q + 5]),
                          bf2(v[8 * q + 6], v[8 * q + 7]));
}

// Staged 32 x 32 block -> global rows (dst = element [row 0][col 0], row
// stride ld): lane l writes 16-byte piece l % 4 of rows l / 4 + 8 j.
__device__ __forceinline__ void flush_rows(const unsigned char* tp, int lane, __nv_bfloat16* dst, long long ld)
{
    const int piece = lane & 3;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int r = (lane >> 2) + 8 * j;
        const uint4 w = *reinterpret_cast<const uint4*>(tp + r * TP_STRIDE + piece * 16);
        st_global_v4(dst + r * ld + piece * 8, w.x, w.y, w.z, w.w);
    }
}

// Global 32 x 32 block -> registers in the same coalesced pattern.
__device__ __forceinline__ void load_rows(const __nv_bfloat16* src, long long ld, int lane, uint4 (&w)[4])
{
    const int piece = lane & 3;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int r = (lane >> 2) + 8 * j;
        w[j] = __ldg(reinterpret_cast<const uint4*>(src + r * ld + piece * 8));
    }
}

__device__ __forceinline__ void stage_loaded(unsigned char* tp, int lane, const uint4 (&w)[4])
{
    const int piece = lane & 3;
#pragma unroll
    for (int j = 0; j < 4; ++j) *reinterpret_cast<uint4*>(tp + ((lane >> 2) + 8 * j) * TP_STRIDE + piece * 16) = w[j];
}

template <int EPI, int ACT>
__global__ void __launch_bounds__(THREADS, 1)
    train_gemm_kernel(const __grid_constant__ CUtensorMap amap, const __grid_constant__ CUtensorMap bmap, GemmArgs g)
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
    const int k_slices = g.k_len / BK;

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
        const int row = quarter * 32 + lane;
        unsigned char* tp = dsm + OFF_TP + ew * TP_BYTES;
        uint32_t accf_phase[2] = {0u, 0u};
        // DGRAD: the Z block of (unit, chunk), loaded one chunk ahead
        uint4 zr[4];
        auto z_block = [&](int i, int c) {
            int ks, mt, nt;
            unit_coords(i, ks, mt, nt);
            return g.z_in + ((long long)mt * BM + quarter * 32) * g.ld_rows + nt * BN + half * 128 + c * 32;
        };
        if constexpr (EPI == kEpiDgrad) {
            if (n_mine > 0) load_rows(z_block(0, 0), g.ld_rows, lane, zr);
        }
        for (int i = 0; i < n_mine; ++i) {
            const int b = i & 1;
            if (!mbar_wait(accf_bar(b), accf_phase[b], abort_flag, g.err)) break;
            accf_phase[b] ^= 1u;
            tc_fence_after();
            int ks, mt, nt;
            unit_coords(i, ks, mt, nt);
            const long long m = (long long)mt * BM + row;              // output row
            const long long m0 = (long long)mt * BM + quarter * 32;    // first row of this warp
            const uint32_t t_row = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(b * BN + half * 128);
#pragma unroll 1
            for (int c = 0; c < 4; ++c) {
                const int n0 = nt * BN + half * 128 + c * 32;
                float v[32];
                if constexpr (EPI == kEpiFwd) {
                    float4 b4[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) b4[q] = __ldg(reinterpret_cast<const float4*>(g.bias + n0 + 4 * q));
                    tmem_ld32(t_row + (uint32_t)(c * 32), v);
                    float z[32];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        z[4 * q + 0] = v[4 * q + 0] + b4[q].x;
                        z[4 * q + 1] = v[4 * q + 1] + b4[q].y;
                        z[4 * q + 2] = v[4 * q + 2] + b4[q].z;
                        z[4 * q + 3] = v[4 * q + 3] + b4[q].w;
                    }
#pragma unroll
                    for (int q = 0; q < 32; ++q) v[q] = act_fwd<ACT>(z[q]);
                    stage_row(tp, lane, z);
                    __syncwarp();
                    flush_rows(tp, lane, g.z_out + m0 * g.ld_rows + n0, g.ld_rows);
                    __syncwarp();
                    stage_row(tp, lane, v);
                    __syncwarp();
                    flush_rows(tp, lane, g.h_out + m0 * g.ld_rows + n0, g.ld_rows);
                    __syncwarp();
                } else if constexpr (EPI == kEpiDgrad) {
                    stage_loaded(tp, lane, zr);
                    // the next chunk's Z block is in flight while this one is used
                    if (c + 1 < 4) load_rows(z_block(i, c + 1), g.ld_rows, lane, zr);
                    else if (i + 1 < n_mine) load_rows(z_block(i + 1, 0), g.ld_rows, lane, zr);
                    tmem_ld32(t_row + (uint32_t)(c * 32), v);
                    __syncwarp();
                    const uint4* zp = reinterpret_cast<const uint4*>(tp + lane * TP_STRIDE);
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const uint4 w = zp[q];
                        v[8 * q + 0] *= act_grad<ACT>(bf_lo(w.x));
                        v[8 * q + 1] *= act_grad<ACT>(bf_hi(w.x));
                        v[8 * q + 2] *= act_grad<ACT>(bf_lo(w.y));
                        v[8 * q + 3] *= act_grad<ACT>(bf_hi(w.y));
                        v[8 * q + 4] *= act_grad<ACT>(bf_lo(w.z));
                        v[8 * q + 5] *= act_grad<ACT>(bf_hi(w.z));
                        v[8 * q + 6] *= act_grad<ACT>(bf_lo(w.w));
                        v[8 * q + 7] *= act_grad<ACT>(bf_hi(w.w));
                    }
                    __syncwarp();
                    stage_row(tp, lane, v);
                    __syncwarp();
                    flush_rows(tp, lane, g.h_out + m0 * g.ld_rows + n0, g.ld_rows);
                    __syncwarp();
                } else {
                    tmem_ld32(t_row + (uint32_t)(c * 32), v);
                    float4* dst = reinterpret_cast<float4*>(g.dw + (long long)ks * g.split_stride + m * g.ld_rows + n0);
#pragma unroll
                    for (int q = 0; q < 8; ++q) dst[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(acce_bar(b));
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base), "r"(512) : "memory");
    }
}

template <int EPI, int ACT>
void launch_t(const CUtensorMap& a, const CUtensorMap& b, const GemmArgs& g, int grid, cudaStream_t s)
{
    int dev = 0;
    cudaGetDevice(&dev);
    static std::once_flag done[64];            // once per device, safe across host threads
    if (dev >= 0 && dev < 64)
        std::call_once(done[dev], [] {
            cudaFuncSetAttribute(train_gemm_kernel<EPI, ACT>, cudaFuncAttributeMaxDynamicSharedMemorySize, SMEM_DYN);
        });
    train_gemm_kernel<EPI, ACT><<<grid, THREADS, SMEM_DYN, s>>>(a, b, g);
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

void launch_train_gemm(int epi, int act, const void* amap, const void* bmap, const GemmArgs& g, int n_sms,
                       cudaStream_t s)
{
    const int units = g.n_ks * g.n_mt * g.n_nt;
    if (units <= 0) return;
    const int grid = units < n_sms ? units : n_sms;
    const CUtensorMap& a = *reinterpret_cast<const CUtensorMap*>(amap);
    const CUtensorMap& b = *reinterpret_cast<const CUtensorMap*>(bmap);
    if (epi == kEpiFwd) {
        if (act == 0) launch_t<kEpiFwd, 0>(a, b, g, grid, s); else launch_t<kEpiFwd, 1>(a, b, g, grid, s);
    } else if (epi == kEpiDgrad) {
        if (act == 0) launch_t<kEpiDgrad, 0>(a, b, g, grid, s); else launch_t<kEpiDgrad, 1>(a, b, g, grid, s);
    } else {
        launch_t<kEpiWgrad, 0>(a, b, g, grid, s);
    }
}

}  // namespace svm
