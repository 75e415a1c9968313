// train.cu -- training of the swept-volume network on the GPU (C ABI
// svm_train_*): data generation with the exact geometric check as labeller,
// and BF16 forward / backward / Adam steps.
//
// Data (Sec. IV-C: tuples (x, q0, q1, delta)): for each motion, points drawn
// with a counter-based SplitMix64 stream (seed, motion, point) -- 70 % near
// the robot's swept surface (a random sample k, capsule j, position along its
// axis, unit direction, and radial offset r_j + U[-0.1, 0.1] m), 30 % uniform
// in a box (default the workspace cube [-0.75,0.75]^2 x [0,1.5]; see
// svm_train_set_box) -- labelled with the exact
// sampled swept-volume distance (the verifier's arithmetic, no gate).
// Samples are stored grouped by motion; a batch takes every n_batch-th sample
// from a per-epoch random offset, so each batch mixes all motions.
//
// Step (loss: mean |f - delta|, the error the paper reports as MAE):
//   layer 1 (15 -> W) in FP32 on CUDA cores, hidden layers as BF16 tcgen05
//   GEMMs (train_gemm.cu), each layer storing h = act(z) and d = act'(z)
//   (bfloat16, rounded once from the FP32 z) for the backward pass; output
//   layer, loss and its gradient on CUDA cores;
//   backward: per hidden layer a split-K weight-gradient GEMM (reading G and
//   H as stored, [batch][features], as MN-major operands) and an input-
//   gradient GEMM, bias gradients by column sums, layer-1 gradient on CUDA
//   cores; then Adam (lr, betas (0.9, 0.999), eps 1e-8, as in Sec. V) on FP32
//   master weights, which also refreshes the BF16 copies W and W^T.
//   Every sum over the batch is formed from per-block (or per-split)
//   partials reduced in a fixed order -- no floating-point atomics -- so a
//   step, an epoch and a resumed run are bitwise reproducible.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include "svm.h"
#include "svm_internal.cuh"
#include "train_internal.cuh"

using namespace svm;

namespace {

// cp.async of 4 or 8 bytes into shared memory (data in flight without
// holding registers), its group commit and wait.
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem)
{
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit_group() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait_group() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// ------------------------------------------------------------ SplitMix64

__device__ __forceinline__ unsigned long long sm_fin(unsigned long long z)
{
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27; z *= 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double sm_u01(unsigned long long base, unsigned long long i)
{
    return (double)(sm_fin(base + (i + 1ull) * 0x9E3779B97F4A7C15ull) >> 11) * 0x1.0p-53;
}

// The box of the uniformly drawn training points.
struct SampleBox {
    double lo[3], hi[3];
};

// One training point of motion m, local index j, and its exact label.
__global__ void __launch_bounds__(256) sample_kernel(const Capsule* caps, int N, int spm, unsigned long long seed,
                                                     SampleBox box, float4* X, int* MID)
{
    extern __shared__ __align__(16) unsigned char smem[];
    Capsule* cs = reinterpret_cast<Capsule*>(smem);
    const int m = blockIdx.x;
    const int ns = N + 1;
    const float4* src = reinterpret_cast<const float4*>(caps + (long long)m * ns * kCaps);
    for (int i = threadIdx.x; i < ns * kCaps * 2; i += blockDim.x) reinterpret_cast<float4*>(cs)[i] = src[i];
    __syncthreads();
    const unsigned long long base =
        sm_fin((seed * 0x9E3779B97F4A7C15ull) ^ ((unsigned long long)m * 0xD1B54A32D192ED03ull));
    for (int j = threadIdx.x; j < spm; j += blockDim.x) {
        const unsigned long long c = (unsigned long long)j * 8ull;
        const double u0 = sm_u01(base, c);
        float3 p;
        if (u0 < 0.7) {
            const int k = min((int)(sm_u01(base, c + 1) * ns), ns - 1);
            const int cj = min((int)(sm_u01(base, c + 2) * kCaps), kCaps - 1);
            const float t = (float)sm_u01(base, c + 3);
            const float zc = (float)(2.0 * sm_u01(base, c + 4) - 1.0);
            const float ph = (float)(6.283185307179586 * sm_u01(base, c + 5));
            const float off = (float)(-0.1 + 0.2 * sm_u01(base, c + 6));
            const Capsule& q = cs[k * kCaps + cj];
            const float rxy = sqrtf(fmaxf(0.0f, 1.0f - zc * zc));
            float sp, cp;
            sincosf(ph, &sp, &cp);
            const float rad = q.a_r.w + off;
            p.x = q.a_r.x + t * q.e_inv.x + rad * rxy * cp;
            p.y = q.a_r.y + t * q.e_inv.y + rad * rxy * sp;
            p.z = q.a_r.z + t * q.e_inv.z + rad * zc;
        } else {
            p.x = (float)(box.lo[0] + (box.hi[0] - box.lo[0]) * sm_u01(base, c + 1));
            p.y = (float)(box.lo[1] + (box.hi[1] - box.lo[1]) * sm_u01(base, c + 2));
            p.z = (float)(box.lo[2] + (box.hi[2] - box.lo[2]) * sm_u01(base, c + 3));
        }
        float mn[kCaps];
        scan_samples(cs, ns, p, mn);
        const long long s = (long long)m * spm + j;
        X[s] = make_float4(p.x, p.y, p.z, capsule_min(mn, cs));
        MID[s] = m;
    }
}

// ------------------------------------------------------------ layer 1 and head

struct StepArgs {
    int W, B, act;
    long long base, stride;           // sample of batch row r: base + r * stride
    const float4* X;
    const int* MID;
    const double* q0;
    const double* q1;
    const float* P;                   // FP32 master parameters (blob order)
    float* Gr;                        // FP32 gradient (blob order)
    float* loss;                      // per-block partial sums of |f - delta|
    float* part;                      // per-block partial gradients
    long long off_w1, off_b1, off_out;
};

// h = act(z) and d = act'(z), the values the step stores (bfloat16) for the
// forward and backward passes.  SiLU: with s = 1 / (1 + e^-z) (fast
// reciprocal, within a few ulp of the division), h = z s and d = s (1 + z (1 -
// s)).  ReLU: d = 1 where the bfloat16 z is positive, else 0.
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

// Packed FP32 pairs (sm_100+): each half is rounded as the scalar operation
// would round it, so pairing changes no result bit.
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
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

__device__ __forceinline__ void input_row(const StepArgs& a, int r, float (&in)[15], float& delta)
{
    const long long s = a.base + (long long)r * a.stride;
    const float4 x = a.X[s];
    const int m = a.MID[s];
    in[0] = x.x; in[1] = x.y; in[2] = x.z;
    for (int i = 0; i < 6; ++i) {
        in[3 + i] = (float)a.q0[m * 6 + i];
        in[9 + i] = (float)a.q1[m * 6 + i];
    }
    delta = x.w;
}

// Layer 1 forward: a block takes 64 samples; thread t owns features 2t and
// 2t + 1 (blockDim = W / 2) with their 15 weights and bias in registers, and
// for each sample forms z = b + sum_k w_k in_k (fused multiply-adds in the
// order k = 0..14), h = act(z) and d = act'(z), storing the feature pair of
// D0 and H0 as one bfloat16x2 word each (a warp writes 128 contiguous bytes of
// a row).  ReLU stores no D0: d = [h > 0] of the stored bfloat16 h (rounding
// is monotone, so h > 0 exactly where the bfloat16 z is positive).  Two samples go through one packed multiply-add (fma.rn.f32x2, the
// inputs of samples 2p and 2p + 1 interleaved in shared memory).
constexpr int kL1Rows = 64;

template <int ACT>
__global__ void __launch_bounds__(256) layer1_fwd_kernel(StepArgs a, __nv_bfloat16* D0, __nv_bfloat16* H0)
{
    __shared__ __align__(16) float2 ins[kL1Rows / 2][16];     // [sample pair][k] = (in_2p[k], in_2p+1[k])
    const int r0 = blockIdx.x * kL1Rows;
    for (int i = threadIdx.x; i < kL1Rows; i += blockDim.x) {
        float in[15], delta;
        input_row(a, r0 + i, in, delta);
        float* dst = reinterpret_cast<float*>(ins[i >> 1]) + (i & 1);
#pragma unroll
        for (int k = 0; k < 15; ++k) dst[2 * k] = in[k];
        dst[30] = 0.0f;
    }
    const int o = 2 * threadIdx.x;
    uint64_t wa[15], wb[15];
#pragma unroll
    for (int k = 0; k < 15; ++k) {
        const float x = a.P[a.off_w1 + (long long)o * 15 + k], y = a.P[a.off_w1 + (long long)(o + 1) * 15 + k];
        wa[k] = f2(x, x);
        wb[k] = f2(y, y);
    }
    const float ba = a.P[a.off_b1 + o], bb = a.P[a.off_b1 + o + 1];
    const uint64_t ba2 = f2(ba, ba), bb2 = f2(bb, bb);
    __syncthreads();
#pragma unroll 2
    for (int p = 0; p < kL1Rows / 2; ++p) {
        const ulonglong2* x2 = reinterpret_cast<const ulonglong2*>(ins[p]);
        uint64_t in2[16];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const ulonglong2 v = x2[q];
            in2[2 * q] = v.x;
            in2[2 * q + 1] = v.y;
        }
        uint64_t za = ba2, zb = bb2;          // (sample 2p, sample 2p + 1) of features o and o + 1
#pragma unroll
        for (int k = 0; k < 15; ++k) {
            za = f2_fma(wa[k], in2[k], za);
            zb = f2_fma(wb[k], in2[k], zb);
        }
        float z[2][2];
        f2_split(za, z[0][0], z[1][0]);
        f2_split(zb, z[0][1], z[1][1]);
#pragma unroll
        for (int e = 0; e < 2; ++e) {
            const long long at = (long long)(r0 + 2 * p + e) * a.W + o;
            float ha, hb, da, db;
            act_hd<ACT>(z[e][0], ha, da);
            act_hd<ACT>(z[e][1], hb, db);
            if constexpr (ACT != 0) *reinterpret_cast<__nv_bfloat162*>(D0 + at) = __floats2bfloat162_rn(da, db);
            *reinterpret_cast<__nv_bfloat162*>(H0 + at) = __floats2bfloat162_rn(ha, hb);
        }
    }
}

// Output layer, loss and its gradient for 32 samples per block (128 threads):
// f = w_out . h_L + b_out, e = f - delta; the block's sum of |e| goes to
// loss[b]; with eval == 0 also df = sign(e)/B, G_L = (df w_out) d_L (d = act'(z)) and
// the block's partial gradients of w_out and b_out to part[b][0..W].
// Arithmetic order, fixed (the step is bitwise reproducible): f is four
// chains, chain w summing the features of the 32-wide chunks w, w + 4, ...
// in ascending order by fused multiply-adds, then ((f_0 + f_1) + f_2) + f_3
// + b_out; the sums over the block's 32 samples (|e|, df, df h) are the
// butterfly x_l += x_{l ^ s}, s = 16, 8, 4, 2, 1, read at lane 0 (for df h
// written as the same tree over registers).  The 32 rows of H_L are staged in
// shared memory with coalesced 16-byte loads; each row is padded by 16 bytes,
// so the row-per-lane reads of the chains are free of bank conflicts.  D_L is
// read where G_L is formed, a feature pair per lane (coalesced); ReLU takes
// d = [h > 0] from the staged H_L instead (DL unused).
constexpr int kHeadPad = 8;   // bfloat16 elements of padding per staged row

size_t head_smem_bytes(int W) { return (size_t)32 * (W + kHeadPad) * sizeof(__nv_bfloat16); }

template <int ACT>
__global__ void __launch_bounds__(128) head_kernel(StepArgs a, const __nv_bfloat16* HL, const __nv_bfloat16* DL,
                                                   __nv_bfloat16* GL, int eval)
{
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ float part[4][32];
    __shared__ float dfs[32];
    const int W = a.W, ld = W + kHeadPad;
    __nv_bfloat16* hs = reinterpret_cast<__nv_bfloat16*>(smem);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long row0 = (long long)blockIdx.x * 32;
    {
        const int per_row = W / 8, n = 32 * per_row;     // 16-byte pieces
        const uint4* gh = reinterpret_cast<const uint4*>(HL + row0 * W);
        for (int i0 = threadIdx.x; i0 < n; i0 += 16 * 128) {
            uint4 vh[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int i = i0 + u * 128;
                if (i < n) vh[u] = gh[i];
            }
#pragma unroll
            for (int u = 0; u < 16; ++u) {
                const int i = i0 + u * 128;
                if (i < n) {
                    const int rr = i / per_row, cc = i % per_row;
                    *reinterpret_cast<uint4*>(hs + rr * ld + cc * 8) = vh[u];
                }
            }
        }
    }
    __syncthreads();
    const float* wo = a.P + a.off_out;
    float f = 0.0f;
    for (int c = warp; c < W / 32; c += 4) {
        const uint4* p = reinterpret_cast<const uint4*>(hs + lane * ld + c * 32);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 w4 = p[q];
            const uint32_t ws[4] = {w4.x, w4.y, w4.z, w4.w};
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                f = fmaf(wo[c * 32 + 8 * q + 2 * i], __uint_as_float(ws[i] << 16), f);
                f = fmaf(wo[c * 32 + 8 * q + 2 * i + 1], __uint_as_float(ws[i] & 0xFFFF0000u), f);
            }
        }
    }
    part[warp][lane] = f;
    __syncthreads();
    if (warp == 0) {
        const long long s = a.base + (row0 + lane) * a.stride;
        const float delta = a.X[s].w;
        const float fr = part[0][lane] + part[1][lane] + part[2][lane] + part[3][lane] + wo[W];
        const float e = fr - delta;
        float ae = fabsf(e);
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) ae += __shfl_xor_sync(0xffffffffu, ae, sh);
        if (lane == 0) a.loss[blockIdx.x] = ae;
        const float df = (e > 0.0f ? 1.0f : (e < 0.0f ? -1.0f : 0.0f)) / (float)a.B;
        float dsum = df;
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) dsum += __shfl_xor_sync(0xffffffffu, dsum, sh);
        if (!eval && lane == 0) a.part[(long long)blockIdx.x * (W + 1) + W] = dsum;
        dfs[lane] = df;
    }
    if (eval) return;
    __syncthreads();
    float* pb = a.part + (long long)blockIdx.x * (W + 1);
    for (int o = 2 * threadIdx.x; o < W; o += 2 * 128) {
        const float wa = wo[o], wb = wo[o + 1];
        float xa[32], xb[32];
#pragma unroll
        for (int r = 0; r < 32; ++r) {
            const float df = dfs[r];
            const uint32_t h2 = *reinterpret_cast<const uint32_t*>(hs + r * ld + o);
            xa[r] = df * __uint_as_float(h2 << 16);
            xb[r] = df * __uint_as_float(h2 & 0xFFFF0000u);
            float da, db;
            if constexpr (ACT == 0) {
                da = __uint_as_float(h2 << 16) > 0.0f ? 1.0f : 0.0f;
                db = __uint_as_float(h2 & 0xFFFF0000u) > 0.0f ? 1.0f : 0.0f;
            } else {
                const uint32_t d2 = __ldg(reinterpret_cast<const unsigned int*>(DL + (row0 + r) * W + o));
                da = __uint_as_float(d2 << 16);
                db = __uint_as_float(d2 & 0xFFFF0000u);
            }
            const float ga = df * wa * da;
            const float gb = df * wb * db;
            *reinterpret_cast<__nv_bfloat162*>(GL + (row0 + r) * W + o) = __floats2bfloat162_rn(ga, gb);
        }
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) {
#pragma unroll
            for (int l = 0; l < sh; ++l) {
                xa[l] += xa[l + sh];
                xb[l] += xb[l + sh];
            }
        }
        pb[o] = xa[0];
        pb[o + 1] = xb[0];
    }
}

// Layer-1 gradients of 256 samples per block row (blockIdx.x) and 256
// features per block column (blockIdx.y); thread t owns features n, n + 1:
// part[b][n * 15 + k] = sum_r G0[r][n] in_r[k], part[b][15 W + n] = sum_r
// G0[r][n] -- the layout of W1 and b1 in the parameter vector -- each sum a
// chain of fused multiply-adds over the block's samples in ascending order
// (two chains per packed fma.rn.f32x2).  The G0 words reach shared memory by
// cp.async, 16 samples per group and two groups in flight, so the loads do
// not wait on the arithmetic.
__global__ void __launch_bounds__(128) layer1_bwd_kernel(StepArgs a, const __nv_bfloat16* G0)
{
    __shared__ __align__(16) float ins[256][16];
    __shared__ uint32_t ring[2][16][128];
    const int r0 = blockIdx.x * 256;
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        float in[15], delta;
        input_row(a, r0 + i, in, delta);
#pragma unroll
        for (int k = 0; k < 15; ++k) ins[i][k] = in[k];
        ins[i][15] = 1.0f;
    }
    __syncthreads();
    const int n = blockIdx.y * 256 + 2 * threadIdx.x;
    // (acc[k], acc[k + 1]) of features n and n + 1 as packed pairs
    uint64_t acc0[8], acc1[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) acc0[k] = acc1[k] = 0ull;
    // G0[r0 + b][n, n + 1] for 16 samples per group, two groups in flight
    const uint32_t* g = reinterpret_cast<const uint32_t*>(G0 + (long long)r0 * a.W + n);
    const int ldw = a.W / 2;
    auto issue = [&](int grp) {
        uint32_t* dst = &ring[grp & 1][0][threadIdx.x];
#pragma unroll
        for (int u = 0; u < 16; ++u) cp_async_small<4>(dst + u * 128, g + (long long)(grp * 16 + u) * ldw);
        cp_async_commit_group();
    };
    issue(0);
    for (int grp = 0; grp < 16; ++grp) {
        if (grp + 1 < 16) {
            issue(grp + 1);
            cp_async_wait_group<1>();
        } else {
            cp_async_wait_group<0>();
        }
#pragma unroll
        for (int u = 0; u < 16; ++u) {
            const uint32_t gv = ring[grp & 1][u][threadIdx.x];
            const float g0 = __uint_as_float(gv << 16), g1 = __uint_as_float(gv & 0xFFFF0000u);
            const uint64_t g00 = f2(g0, g0), g11 = f2(g1, g1);
            const ulonglong2* x2 = reinterpret_cast<const ulonglong2*>(ins[grp * 16 + u]);
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const ulonglong2 x = x2[q];            // (in[4q], in[4q+1]), (in[4q+2], in[4q+3])
                acc0[2 * q] = f2_fma(g00, x.x, acc0[2 * q]);
                acc0[2 * q + 1] = f2_fma(g00, x.y, acc0[2 * q + 1]);
                acc1[2 * q] = f2_fma(g11, x.x, acc1[2 * q]);
                acc1[2 * q + 1] = f2_fma(g11, x.y, acc1[2 * q + 1]);
            }
        }
    }
    float* pb = a.part + (long long)blockIdx.x * a.W * 16;
    float s0[16], s1[16];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        f2_split(acc0[k], s0[2 * k], s0[2 * k + 1]);
        f2_split(acc1[k], s1[2 * k], s1[2 * k + 1]);
    }
#pragma unroll
    for (int k = 0; k < 15; ++k) {
        pb[(long long)n * 15 + k] = s0[k];
        pb[(long long)(n + 1) * 15 + k] = s1[k];
    }
    pb[15LL * a.W + n] = s0[15];
    pb[15LL * a.W + n + 1] = s1[15];
}

// Bias gradients db[n] += sum over the batch of G[b][n] (G row-major [B][W]),
// in a fixed order, so a step is deterministic: 256 chains per column (chain
// t sums rows t, t + 256, ... in order), then per group of 32 chains the
// butterfly x_l += x_{l ^ s} (s = 16, 8, 4, 2, 1) read at lane 0, then the 8
// group results in order.  Part 1 runs the chains: thread (t, q) of a block
// sums columns 4q..4q+3 of its rows, a warp covering 128 contiguous columns
// of one row (full sectors), and writes chain[t][n]; its rows reach shared
// memory by cp.async, 32 per group with two groups in flight, so enough bytes
// are in flight to stream G at the memory's rate.  Part 2 (one warp per
// column) forms the tree.
constexpr int kCsDepth = 32;   // rows per cp.async group of the chains

constexpr int kCsThreads = 128;   // 4 chains x 32 column quads per block

size_t colsum_smem_bytes() { return (size_t)2 * kCsDepth * kCsThreads * sizeof(uint2); }

__global__ void __launch_bounds__(kCsThreads) colsum_chains_kernel(const __nv_bfloat16* G, long long B, int W,
                                                                  float* chain)
{
    extern __shared__ __align__(16) uint2 cs_ring[];              // [2][kCsDepth][kCsThreads]
    const int q = blockIdx.x * 32 + (threadIdx.x & 31);          // column quad
    const int t = blockIdx.y * (kCsThreads / 32) + (threadIdx.x >> 5);   // chain (row class), 0..255
    const int n0 = 4 * q;
    const long long rows = (B - t + 255) / 256;                   // rows t, t + 256, ... below B
    const long long ng = (rows + kCsDepth - 1) / kCsDepth;
    const __nv_bfloat16* src = G + (long long)t * W + n0;
    const long long step = 256LL * W;
    auto issue = [&](long long grp) {
        uint2* dst = cs_ring + (grp & 1) * kCsDepth * kCsThreads + threadIdx.x;
        const long long r0 = grp * kCsDepth;
#pragma unroll 8
        for (int u = 0; u < kCsDepth; ++u)
            if (r0 + u < rows) cp_async_small<8>(dst + u * kCsThreads, src + (r0 + u) * step);
        cp_async_commit_group();
    };
    float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    if (ng > 0) issue(0);
    for (long long grp = 0; grp < ng; ++grp) {
        if (grp + 1 < ng) {
            issue(grp + 1);
            cp_async_wait_group<1>();
        } else {
            cp_async_wait_group<0>();
        }
        const uint2* buf = cs_ring + (grp & 1) * kCsDepth * kCsThreads + threadIdx.x;
        const int cnt = (int)min((long long)kCsDepth, rows - grp * kCsDepth);
#pragma unroll 8
        for (int u = 0; u < cnt; ++u) {
            const uint2 w = buf[u * kCsThreads];
            s[0] += __uint_as_float(w.x << 16);
            s[1] += __uint_as_float(w.x & 0xFFFF0000u);
            s[2] += __uint_as_float(w.y << 16);
            s[3] += __uint_as_float(w.y & 0xFFFF0000u);
        }
    }
    *reinterpret_cast<float4*>(chain + (long long)t * W + n0) = make_float4(s[0], s[1], s[2], s[3]);
}

__global__ void __launch_bounds__(256) colsum_tree_kernel(const float* chain, int W, float* db)
{
    const int n = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
    if (n >= W) return;
    float total = 0.0f;
    for (int w = 0; w < 8; ++w) {
        float x = chain[(long long)(32 * w + lane) * W + n];
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) x += __shfl_xor_sync(0xffffffffu, x, sh);
        total += x;
    }
    if (lane == 0) db[n] += total;
}

// dst[j] += sum_{p < P} part[p * n + j] for long sums (P in the hundreds to
// thousands): a block takes TJ outputs and stages tiles of 8192 / TJ partials
// x TJ outputs (32 KB) in shared memory, each thread issuing its 32 loads
// before storing them; thread j then adds its column in the order p = 0, 1,
// ... (the order of reduce_kernel).
template <int TJ>
__global__ void __launch_bounds__(256) reduce_long_kernel(const float* part, int P, long long n, float* dst)
{
    constexpr int TP = 8192 / TJ, PASS = 256 / TJ, PER = TP / PASS;
    __shared__ float tile[TP * TJ];
    const long long j0 = (long long)blockIdx.x * TJ;
    const int jj = threadIdx.x % TJ, pr = threadIdx.x / TJ;
    const bool col_ok = j0 + jj < n;
    float s = 0.0f;
    for (int p0 = 0; p0 < P; p0 += TP) {
        float v[PER];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int p = p0 + u * PASS + pr;
            v[u] = (col_ok && p < P) ? part[(long long)p * n + j0 + jj] : 0.0f;
        }
#pragma unroll
        for (int u = 0; u < PER; ++u) tile[(u * PASS + pr) * TJ + jj] = v[u];
        __syncthreads();
        if (threadIdx.x < TJ) {
            const int lim = min(TP, P - p0);
            int pp = 0;
            for (; pp + 16 <= lim; pp += 16) {       // 16 reads issued before their adds
                float v[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) v[u] = tile[(pp + u) * TJ + threadIdx.x];
#pragma unroll
                for (int u = 0; u < 16; ++u) s += v[u];
            }
            for (; pp < lim; ++pp) s += tile[pp * TJ + threadIdx.x];
        }
        __syncthreads();
    }
    if (threadIdx.x < TJ && j0 + threadIdx.x < n) dst[j0 + threadIdx.x] += s;
}
constexpr int kRedCols = 4;        // the output-layer gradient (2 048 partials of W + 1 sums)
constexpr int kRedColsL1 = 8;      // the layer-1 gradient (256 partials of 16 W sums)

// dst[j] += sum_{p < P} part[p * n + j], summed in the order p = 0, 1, ...;
// the loads of 8 partials are issued before their adds (same order of the adds).
__global__ void reduce_kernel(const float* part, int P, long long n, float* dst)
{
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < n; j += (long long)gridDim.x * blockDim.x) {
        float s = 0.0f;
        int p = 0;
        for (; p + 8 <= P; p += 8) {
            float v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = part[(long long)(p + u) * n + j];
#pragma unroll
            for (int u = 0; u < 8; ++u) s += v[u];
        }
        for (; p < P; ++p) s += part[(long long)p * n + j];
        dst[j] += s;
    }
}

// dst[0] += sum_{p < P} part[p] in the order p = 0, 1, ... (the order of
// reduce_kernel), by one warp: 32 partials per coalesced load, added
// in order through shuffles.  It needs no shared memory, so it can share SMs
// with a running GEMM.
__global__ void reduce_scalar_kernel(const float* part, int P, float* dst)
{
    const int lane = threadIdx.x & 31;
    float s = 0.0f;
    for (int p0 = 0; p0 < P; p0 += 32) {
        const float v = p0 + lane < P ? part[p0 + lane] : 0.0f;
        const int lim = min(32, P - p0);
        for (int j = 0; j < lim; ++j) s += __shfl_sync(0xffffffffu, v, j);
    }
    if (lane == 0) dst[0] += s;
}

// Adam on the FP32 master parameters (two kernels); refreshes the BF16 copies
// of the hidden weights (W [out][in] and W^T [in][out]).
__device__ __forceinline__ float adam_update(float* P, const float* G, float* Mo, float* Vo, long long i, float lr,
                                             float b1, float b2, float eps, float c1, float c2)
{
    const float g = G[i];
    const float m = b1 * Mo[i] + (1.0f - b1) * g;
    const float v = b2 * Vo[i] + (1.0f - b2) * g * g;
    Mo[i] = m;
    Vo[i] = v;
    const float p = P[i] - lr * (m / c1) / (sqrtf(v / c2) + eps);
    P[i] = p;
    return p;
}

// The hidden-layer weight matrices, one 32 x 32 tile (outputs o0.., inputs
// k0..) of layer blockIdx.z per block: coalesced reads and writes of the FP32
// state and of W (bfloat16), and W^T written through a shared-memory tile.
__global__ void __launch_bounds__(256) adam_hidden_kernel(float* P, const float* G, float* Mo, float* Vo, float lr,
                                                          float b1, float b2, float eps, float c1, float c2, int W,
                                                          long long off_h, __nv_bfloat16* wb, __nv_bfloat16* wbt)
{
    __shared__ __nv_bfloat16 tile[32][34];
    const int l = blockIdx.z, o0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const long long base = off_h + (long long)l * ((long long)W * W + W);
    const long long lw = (long long)l * W * W;
#pragma unroll
    for (int r = ty; r < 32; r += 8) {
        const long long w = (long long)(o0 + r) * W + k0 + tx;
        const float p = adam_update(P, G, Mo, Vo, base + w, lr, b1, b2, eps, c1, c2);
        const __nv_bfloat16 pb = __float2bfloat16_rn(p);
        wb[lw + w] = pb;
        tile[r][tx] = pb;
    }
    __syncthreads();
#pragma unroll
    for (int r = ty; r < 32; r += 8) wbt[lw + (long long)(k0 + r) * W + o0 + tx] = tile[tx][r];
}

// Every other parameter: layer 1 (weights and bias), the hidden biases, the
// output layer.
__global__ void adam_rest_kernel(float* P, const float* G, float* Mo, float* Vo, float lr, float b1, float b2, float eps,
                                 float c1, float c2, int W, int L, long long off_h, long long off_out)
{
    const long long n = off_h + (long long)L * W + W + 1;
    for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n; t += (long long)gridDim.x * blockDim.x) {
        long long i;
        if (t < off_h) {
            i = t;
        } else if (t < off_h + (long long)L * W) {
            const long long u = t - off_h, l = u / W;
            i = off_h + l * ((long long)W * W + W) + (long long)W * W + (u - l * W);
        } else {
            i = off_out + (t - off_h - (long long)L * W);
        }
        adam_update(P, G, Mo, Vo, i, lr, b1, b2, eps, c1, c2);
    }
}

__global__ void refresh_bf16_kernel(const float* P, int W, int L, long long off_h, __nv_bfloat16* wb,
                                    __nv_bfloat16* wbt)
{
    const long long total = (long long)L * W * W;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long l = i / ((long long)W * W), w = i % ((long long)W * W);
        const long long o = w / W, k = w % W;
        const __nv_bfloat16 pb = __float2bfloat16_rn(P[off_h + l * ((long long)W * W + W) + w]);
        wb[i] = pb;
        wbt[l * W * W + k * W + o] = pb;
    }
}

int grid_for(long long n) { long long g = (n + 255) / 256; return (int)(g > 8192 ? 8192 : (g < 1 ? 1 : g)); }

struct Map { alignas(64) unsigned char b[128]; };

}  // namespace

struct svm_trainer {
    int device = 0, n_sms = 0;
    svm_model_desc desc{};
    RobotParams rp{};
    int W = 0, L = 0, act = 0, B = 0;
    // weight-gradient split of the batch: wg_ks splits of wg_klen rows, the last wg_klast
    int wg_ks = 1, wg_klen = 0, wg_klast = 0;
    long long np = 0, off_w1 = 0, off_b1 = 0, off_h = 0, off_out = 0;
    long long step = 0;
    float* P = nullptr; float* Gr = nullptr; float* Mo = nullptr; float* Vo = nullptr;
    float* loss = nullptr;            // per-block loss partials (B / 32)
    float* loss_sum = nullptr;        // batch-summed losses of the current call
    float* part = nullptr;            // per-block partials of the head and of layer 1
    long long part_n = 0;
    float* kpart[2] = {nullptr, nullptr};   // split-K weight-gradient partials, alternating by layer
    float* chain[2] = {nullptr, nullptr};   // bias-gradient chains [256][W], alternating by layer
    // the second stream: per layer, the split-K reduction and the bias-sum tree run
    // beside the next GEMMs (no shared memory, so they share SMs with them)
    cudaStream_t side = nullptr;
    std::vector<cudaEvent_t> ev_w, ev_c, ev_s;   // per layer: partials ready, chains ready, side done
    cudaEvent_t ev_head = nullptr, ev_side = nullptr;
    // an epoch replays one captured step (gradient reset, forward, backward) on
    // the stream `main`, with the batch's sample offset patched into the three
    // kernels that read samples (layer 1 forward, head, layer 1 backward)
    cudaStream_t main = nullptr;
    cudaGraph_t step_graph = nullptr;
    cudaGraphExec_t step_exec = nullptr;
    cudaGraphNode_t node_l1f = nullptr, node_head = nullptr, node_l1b = nullptr;
    unsigned int* err = nullptr;
    __nv_bfloat16* wb = nullptr; __nv_bfloat16* wbt = nullptr;
    std::vector<__nv_bfloat16*> H, D, G;             // per layer 0..L, [B][W]; D = act'(z)
    // A operands of the forward and input-gradient GEMMs (K-major, 128-row boxes) and the MN-major
    // operands of the weight-gradient GEMM (64 x 64 boxes)
    std::vector<Map> mapH, mapG, mapHmn, mapGmn, mapW, mapWT, mapDst, mapHst, mapGst;
    Map mapPst[2];
    // data
    float4* X = nullptr; int* MID = nullptr; double* q0 = nullptr; double* q1 = nullptr;
    int n_motions = 0; long long n_samples = 0;
    double box_lo[3] = {-0.75, -0.75, 0.0}, box_hi[3] = {0.75, 0.75, 1.5};   // uniform training points
    std::vector<void*> allocs;
    std::string last_error;
};

namespace {

svm_status tfail(svm_trainer* t, svm_status s, const std::string& msg)
{
    if (t) t->last_error = msg;
    return s;
}

#define TCK(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return tfail(t, SVM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));   \
    } while (0)

template <class T>
svm_status talloc(svm_trainer* t, T** p, size_t bytes)
{
    void* q = nullptr;
    if (cudaMalloc(&q, bytes) != cudaSuccess) {
        cudaGetLastError();
        return tfail(t, SVM_E_OOM, "trainer allocation failed");
    }
    t->allocs.push_back(q);
    *p = static_cast<T*>(q);
    return SVM_OK;
}

void free_data(svm_trainer* t)
{
    for (void* p : {(void*)t->X, (void*)t->MID, (void*)t->q0, (void*)t->q1})
        if (p) {
            cudaFree(p);
            for (auto& a : t->allocs)
                if (a == p) a = nullptr;
        }
    t->X = nullptr; t->MID = nullptr; t->q0 = nullptr; t->q1 = nullptr;
    t->n_motions = 0; t->n_samples = 0;
}

struct DevGuard {
    int prev = -1;
    explicit DevGuard(int d) { if (cudaGetDevice(&prev) != cudaSuccess) prev = -1; if (prev != d) cudaSetDevice(d); }
    ~DevGuard() { int c = -1; if (prev >= 0 && cudaGetDevice(&c) == cudaSuccess && c != prev) cudaSetDevice(prev); }
};

StepArgs step_args(svm_trainer* t, long long base, long long stride)
{
    StepArgs a{};
    a.W = t->W; a.B = t->B; a.act = t->act;
    a.base = base; a.stride = stride;
    a.X = t->X; a.MID = t->MID; a.q0 = t->q0; a.q1 = t->q1;
    a.P = t->P; a.Gr = t->Gr; a.loss = t->loss; a.part = t->part;
    a.off_w1 = t->off_w1; a.off_b1 = t->off_b1; a.off_out = t->off_out;
    return a;
}

// Forward over one batch; with grad, also the backward pass into Gr.
svm_status run_batch(svm_trainer* t, long long base, long long stride, bool grad, cudaStream_t s)
{
    const int W = t->W, L = t->L, B = t->B;
    const StepArgs a = step_args(t, base, stride);
    if (t->act == 0) layer1_fwd_kernel<0><<<B / kL1Rows, W / 2, 0, s>>>(a, t->D[0], t->H[0]);
    else layer1_fwd_kernel<1><<<B / kL1Rows, W / 2, 0, s>>>(a, t->D[0], t->H[0]);
    for (int l = 1; l <= L; ++l) {
        GemmArgs g{};
        g.n_mt = B / 128; g.n_nt = W / 256; g.n_ks = 1; g.k_len = W;
        g.ld_rows = W;
        g.bias = t->P + t->off_h + (long long)(l - 1) * ((long long)W * W + W) + (long long)W * W;
        g.err = t->err;
        // ReLU stores no D (its first store map is unused)
        const unsigned char* dmap = t->act == 0 ? t->mapHst[l].b : t->mapDst[l].b;
        launch_train_gemm(kEpiFwd, t->act, t->mapH[l - 1].b, t->mapW[l - 1].b, dmap, t->mapHst[l].b, g, t->n_sms, s);
    }
    const size_t head_smem = head_smem_bytes(W);
    if (t->act == 0) head_kernel<0><<<B / 32, 128, head_smem, s>>>(a, t->H[L], t->D[L], t->G[L], grad ? 0 : 1);
    else head_kernel<1><<<B / 32, 128, head_smem, s>>>(a, t->H[L], t->D[L], t->G[L], grad ? 0 : 1);
    if (!grad) {
        reduce_scalar_kernel<<<1, 32, 0, s>>>(t->loss, B / 32, t->loss_sum);
        return SVM_OK;
    }
    cudaStream_t s2 = t->side;
    cudaEventRecord(t->ev_head, s);
    cudaStreamWaitEvent(s2, t->ev_head, 0);
    reduce_scalar_kernel<<<1, 32, 0, s2>>>(t->loss, B / 32, t->loss_sum);
    reduce_long_kernel<kRedCols><<<(W + 1 + kRedCols - 1) / kRedCols, 256, 0, s>>>(t->part, B / 32, W + 1, t->Gr + t->off_out);
    for (int l = L; l >= 1; --l) {
        const long long woff = t->off_h + (long long)(l - 1) * ((long long)W * W + W);
        const int buf = l & 1;
        // the buffers of layer l + 2 are free once the side stream has reduced them
        if (l + 2 <= L) cudaStreamWaitEvent(s, t->ev_s[l + 2], 0);
        GemmArgs g{};
        g.n_mt = W / 128; g.n_nt = W / 256; g.n_ks = t->wg_ks; g.k_len = t->wg_klen; g.k_last = t->wg_klast;
        g.ld_rows = W; g.dw = t->kpart[buf]; g.split_stride = (long long)W * W; g.err = t->err;
        launch_train_gemm(kEpiWgrad, 0, t->mapGmn[l].b, t->mapHmn[l - 1].b, t->mapPst[buf].b, nullptr, g, t->n_sms, s);
        cudaEventRecord(t->ev_w[l], s);
        colsum_chains_kernel<<<dim3(W / 128, 256 / (kCsThreads / 32)), kCsThreads, colsum_smem_bytes(), s>>>(t->G[l], B, W,
                                                                                                        t->chain[buf]);
        cudaEventRecord(t->ev_c[l], s);
        cudaStreamWaitEvent(s2, t->ev_w[l], 0);
        reduce_kernel<<<grid_for((long long)W * W), 256, 0, s2>>>(t->kpart[buf], g.n_ks, (long long)W * W, t->Gr + woff);
        cudaStreamWaitEvent(s2, t->ev_c[l], 0);
        colsum_tree_kernel<<<W / 8, 256, 0, s2>>>(t->chain[buf], W, t->Gr + woff + (long long)W * W);
        cudaEventRecord(t->ev_s[l], s2);
        GemmArgs d{};
        d.n_mt = B / 128; d.n_nt = W / 256; d.n_ks = 1; d.k_len = W;
        d.ld_rows = W; d.d_in = t->act == 0 ? t->H[l - 1] : t->D[l - 1];   // ReLU: d = [h > 0]
        d.err = t->err;
        launch_train_gemm(kEpiDgrad, t->act, t->mapG[l].b, t->mapWT[l - 1].b, t->mapGst[l - 1].b, nullptr, d, t->n_sms,
                          s);
    }
    layer1_bwd_kernel<<<dim3(B / 256, W / 256), 128, 0, s>>>(a, t->G[0]);
    reduce_long_kernel<kRedColsL1><<<W * 16 / kRedColsL1, 256, 0, s>>>(t->part, B / 256, (long long)W * 16, t->Gr + t->off_w1);
    // the step ends when the side stream's sums are in the gradient too
    cudaEventRecord(t->ev_side, s2);
    cudaStreamWaitEvent(s, t->ev_side, 0);
    return SVM_OK;
}

}  // namespace

extern "C" {

const char* svm_train_last_error(const svm_trainer* t) { return t ? t->last_error.c_str() : "null trainer"; }

svm_status svm_train_create(const svm_model_desc* desc, int device, int32_t batch, svm_trainer** out)
{
    svm_trainer* t = nullptr;
    if (!desc || !out) return SVM_E_INVALID;
    *out = nullptr;
    const svm_model_desc& d = *desc;
    if (!(d.width == 256 || d.width == 512) || d.n_hidden < 1 || d.n_hidden > 16) return SVM_E_UNSUPPORTED;
    if (d.arch != SVM_ARCH_MLP) return SVM_E_UNSUPPORTED;
    if (d.act != SVM_RELU && d.act != SVM_SILU) return SVM_E_INVALID;
    if (batch < 256 || batch % 256 != 0) return SVM_E_INVALID;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) return SVM_E_INVALID;
    int maj = 0, min_ = 0;
    cudaDeviceGetAttribute(&maj, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&min_, cudaDevAttrComputeCapabilityMinor, device);
    if (!(maj == 10 && min_ == 3)) return SVM_E_UNSUPPORTED;
    t = new svm_trainer();
    DevGuard gd(device);
    t->device = device;
    t->desc = d;
    cudaDeviceGetAttribute(&t->n_sms, cudaDevAttrMultiProcessorCount, device);
    // the head stages 32 rows of H_L: 33 KB at width 512
    cudaFuncSetAttribute(head_kernel<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)head_smem_bytes(512));
    cudaFuncSetAttribute(head_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)head_smem_bytes(512));
    cudaFuncSetAttribute(colsum_chains_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)colsum_smem_bytes());
    for (int j = 0; j < 6; ++j) {
        t->rp.d[j] = d.dh[j][0]; t->rp.a[j] = d.dh[j][1];
        t->rp.ca[j] = std::cos(d.dh[j][2]); t->rp.sa[j] = std::sin(d.dh[j][2]); t->rp.th0[j] = d.dh[j][3];
    }
    t->rp.tool_len = d.tool_len;
    for (int j = 0; j < 7; ++j) {
        t->rp.radius[j] = (float)d.radius[j];
        t->rp.radius64[j] = d.radius[j];
    }
    t->W = d.width; t->L = d.n_hidden; t->act = d.act; t->B = batch;
    const long long W = t->W, L = t->L, B = t->B;
    t->off_w1 = 0; t->off_b1 = W * 15; t->off_h = W * 16;
    t->off_out = t->off_h + L * (W * W + W);
    t->np = t->off_out + W + 1;
    svm_status st;
    auto fail_free = [&](svm_status s) { svm_train_destroy(t); return s; };
    if ((st = talloc(t, &t->P, t->np * 4)) != SVM_OK) return fail_free(st);
    if ((st = talloc(t, &t->Gr, t->np * 4)) != SVM_OK) return fail_free(st);
    if ((st = talloc(t, &t->Mo, t->np * 4)) != SVM_OK) return fail_free(st);
    if ((st = talloc(t, &t->Vo, t->np * 4)) != SVM_OK) return fail_free(st);
    if ((st = talloc(t, &t->loss, (B / 32) * 4)) != SVM_OK) return fail_free(st);
    if ((st = talloc(t, &t->loss_sum, 256)) != SVM_OK) return fail_free(st);
    {
        // The weight-gradient GEMM has (W / 128) (W / 256) output tiles and cuts the batch into splits of
        // 2048 rows (smaller batches: one split).  Where tiles x splits is more than one unit per SM (a
        // second, partial wave), it takes fewer, longer splits instead -- multiples of 64 rows, about one
        // unit per SM, the last split the remainder -- which also means fewer partials to sum; elsewhere
        // more splits would only add partial traffic.  Each split's FP32 partial is summed afterwards
        // in split order.
        const long long tiles = (W / 128) * (W / 256);
        long long kl = B >= 2048 ? 2048 : B;
        long long ks = B / kl;
        if (tiles * ks > t->n_sms) {
            const long long target = std::max<long long>(1, t->n_sms / tiles);
            kl = (B + target - 1) / target;
            kl = (kl + 63) / 64 * 64;
            ks = (B + kl - 1) / kl;
        }
        t->wg_klen = (int)kl;
        t->wg_ks = (int)ks;
        t->wg_klast = (int)(B - (ks - 1) * kl);
        t->part_n = std::max((B / 32) * (W + 1), (B / 256) * W * 16);
        for (int b = 0; b < 2; ++b) {
            if ((st = talloc(t, &t->kpart[b], (long long)t->wg_ks * W * W * 4)) != SVM_OK) return fail_free(st);
            if ((st = talloc(t, &t->chain[b], 256LL * W * 4)) != SVM_OK) return fail_free(st);
        }
    }
    if ((st = talloc(t, &t->part, t->part_n * 4)) != SVM_OK) return fail_free(st);
    if (cudaStreamCreateWithFlags(&t->side, cudaStreamNonBlocking) != cudaSuccess) return fail_free(SVM_E_CUDA);
    // blocking: it orders with the default stream the other trainer calls use
    if (cudaStreamCreate(&t->main) != cudaSuccess) return fail_free(SVM_E_CUDA);
    t->ev_w.assign(L + 1, nullptr); t->ev_c.assign(L + 1, nullptr); t->ev_s.assign(L + 1, nullptr);
    for (int l = 0; l <= L; ++l)
        for (auto* v : {&t->ev_w, &t->ev_c, &t->ev_s})
            if (cudaEventCreateWithFlags(&(*v)[l], cudaEventDisableTiming) != cudaSuccess) return fail_free(SVM_E_CUDA);
    if (cudaEventCreateWithFlags(&t->ev_head, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&t->ev_side, cudaEventDisableTiming) != cudaSuccess)
        return fail_free(SVM_E_CUDA);
    if ((st = talloc(t, &t->err, 256)) != SVM_OK) return fail_free(st);
    if ((st = talloc(t, &t->wb, L * W * W * 2)) != SVM_OK) return fail_free(st);
    if ((st = talloc(t, &t->wbt, L * W * W * 2)) != SVM_OK) return fail_free(st);
    t->H.resize(L + 1); t->D.assign(L + 1, nullptr); t->G.resize(L + 1);
    for (int l = 0; l <= L; ++l)
        for (auto* v : {&t->H, &t->D, &t->G})
            if ((v != &t->D || t->act != 0) && (st = talloc(t, &(*v)[l], B * W * 2)) != SVM_OK) return fail_free(st);
    cudaMemset(t->P, 0, t->np * 4);
    cudaMemset(t->Mo, 0, t->np * 4);
    cudaMemset(t->Vo, 0, t->np * 4);
    cudaMemset(t->err, 0, 4);
    t->mapH.resize(L + 1); t->mapG.resize(L + 1); t->mapHmn.resize(L + 1); t->mapGmn.resize(L + 1);
    t->mapW.resize(L); t->mapWT.resize(L);
    t->mapDst.resize(L + 1); t->mapHst.resize(L + 1); t->mapGst.resize(L + 1);
    int bad = 0;
    for (int l = 0; l <= L; ++l) {
        if (t->act != 0) bad |= train_make_store_map(t->mapDst[l].b, t->D[l], B, W, 0);  // outputs of FWD and DGRAD
        bad |= train_make_store_map(t->mapHst[l].b, t->H[l], B, W, 0);
        bad |= train_make_store_map(t->mapGst[l].b, t->G[l], B, W, 0);
        bad |= train_make_map(t->mapH[l].b, t->H[l], B, W, 128);       // A of FWD
        bad |= train_make_map(t->mapG[l].b, t->G[l], B, W, 128);       // A of DGRAD
        bad |= train_make_map(t->mapHmn[l].b, t->H[l], B, W, 64);      // B of WGRAD (MN-major)
        bad |= train_make_map(t->mapGmn[l].b, t->G[l], B, W, 64);      // A of WGRAD (MN-major)
    }
    for (int l = 0; l < L; ++l) {
        bad |= train_make_map(t->mapW[l].b, t->wb + (long long)l * W * W, W, W, 256);    // B of FWD
        bad |= train_make_map(t->mapWT[l].b, t->wbt + (long long)l * W * W, W, W, 256);  // B of DGRAD
    }
    {
        // the weight-gradient partials, [splits * W][W] FP32
        for (int b = 0; b < 2; ++b)
            bad |= train_make_store_map(t->mapPst[b].b, t->kpart[b], (long long)t->wg_ks * W, W, 1);
    }
    if (bad) return fail_free(SVM_E_CUDA);
    if (cudaDeviceSynchronize() != cudaSuccess) return fail_free(SVM_E_CUDA);
    *out = t;
    return SVM_OK;
}

svm_status svm_train_destroy(svm_trainer* t)
{
    if (!t) return SVM_E_INVALID;
    {
        DevGuard gd(t->device);
        cudaDeviceSynchronize();
        for (void* p : t->allocs)
            if (p) cudaFree(p);
        for (auto* v : {&t->ev_w, &t->ev_c, &t->ev_s})
            for (cudaEvent_t e : *v)
                if (e) cudaEventDestroy(e);
        if (t->ev_head) cudaEventDestroy(t->ev_head);
        if (t->ev_side) cudaEventDestroy(t->ev_side);
        if (t->side) cudaStreamDestroy(t->side);
        if (t->step_exec) cudaGraphExecDestroy(t->step_exec);
        if (t->step_graph) cudaGraphDestroy(t->step_graph);
        if (t->main) cudaStreamDestroy(t->main);
    }
    delete t;
    return SVM_OK;
}

svm_status svm_train_set_weights(svm_trainer* t, const void* blob, size_t bytes)
{
    if (!t || !blob) return SVM_E_INVALID;
    const unsigned char* p = static_cast<const unsigned char*>(blob);
    auto rd32 = [&](size_t off) { uint32_t v; std::memcpy(&v, p + off, 4); return v; };
    if (bytes < 28 || std::memcmp(p, "SVMW", 4) != 0 || rd32(4) != 1) return tfail(t, SVM_E_WEIGHTS, "bad blob header");
    if ((int)rd32(8) != t->L + 2 || rd32(12) != 15 || (int)rd32(16) != t->W || (int)rd32(20) != t->act)
        return tfail(t, SVM_E_WEIGHTS, "blob does not match the trainer");
    std::vector<float> P(t->np);
    size_t off = 28;
    long long pos = 0;
    for (int l = 0; l < t->L + 2; ++l) {
        if (off + 8 > bytes) return tfail(t, SVM_E_WEIGHTS, "truncated blob");
        const uint32_t o = rd32(off), i = rd32(off + 4);
        off += 8;
        const size_t nb = ((size_t)o * i + o) * 4;
        if ((long long)(pos + (long long)o * i + o) > t->np || off + nb > bytes) return tfail(t, SVM_E_WEIGHTS, "bad layer");
        std::memcpy(P.data() + pos, p + off, nb);
        off += nb;
        pos += (long long)o * i + o;
    }
    if (pos != t->np || off != bytes) return tfail(t, SVM_E_WEIGHTS, "blob size mismatch");
    DevGuard gd(t->device);
    TCK(cudaMemcpy(t->P, P.data(), t->np * 4, cudaMemcpyHostToDevice));
    TCK(cudaMemset(t->Mo, 0, t->np * 4));
    TCK(cudaMemset(t->Vo, 0, t->np * 4));
    t->step = 0;
    refresh_bf16_kernel<<<grid_for((long long)t->L * t->W * t->W), 256>>>(t->P, t->W, t->L, t->off_h, t->wb, t->wbt);
    TCK(cudaGetLastError());
    TCK(cudaDeviceSynchronize());
    return SVM_OK;
}

svm_status svm_train_get_weights(svm_trainer* t, void* blob, size_t cap, size_t* needed)
{
    if (!t) return SVM_E_INVALID;
    const size_t need = 28 + (size_t)(t->L + 2) * 8 + (size_t)t->np * 4;
    if (needed) *needed = need;
    if (!blob) return SVM_OK;
    if (cap < need) return tfail(t, SVM_E_INVALID, "buffer too small");
    std::vector<float> P(t->np);
    DevGuard gd(t->device);
    TCK(cudaDeviceSynchronize());
    TCK(cudaMemcpy(P.data(), t->P, t->np * 4, cudaMemcpyDeviceToHost));
    unsigned char* o = static_cast<unsigned char*>(blob);
    std::memcpy(o, "SVMW", 4);
    const uint32_t hdr[5] = {1u, (uint32_t)(t->L + 2), 15u, (uint32_t)t->W, (uint32_t)t->act};
    std::memcpy(o + 4, hdr, 20);
    const float tau = INFINITY;
    std::memcpy(o + 24, &tau, 4);
    size_t off = 28;
    long long pos = 0;
    for (int l = 0; l < t->L + 2; ++l) {
        const uint32_t out = l == t->L + 1 ? 1u : (uint32_t)t->W;
        const uint32_t in = l == 0 ? 15u : (uint32_t)t->W;
        std::memcpy(o + off, &out, 4);
        std::memcpy(o + off + 4, &in, 4);
        off += 8;
        const size_t nb = ((size_t)out * in + out) * 4;
        std::memcpy(o + off, P.data() + pos, nb);
        off += nb;
        pos += (long long)out * in + out;
    }
    return SVM_OK;
}

svm_status svm_train_make_data(svm_trainer* t, const double* q0, const double* q1, int32_t n_motions,
                               int32_t samples_per_motion, int32_t steps, uint64_t seed)
{
    if (!t || !q0 || !q1 || n_motions < 1 || samples_per_motion < 1 || steps < 1 || steps > kMaxSteps)
        return tfail(t, SVM_E_INVALID, "bad data arguments");
    for (long long i = 0; i < (long long)n_motions * 6; ++i)
        if (!std::isfinite(q0[i]) || !std::isfinite(q1[i])) return tfail(t, SVM_E_INVALID, "non-finite joint angle");
    DevGuard gd(t->device);
    TCK(cudaDeviceSynchronize());
    free_data(t);
    const long long S = (long long)n_motions * samples_per_motion;
    svm_status st;
    if ((st = talloc(t, &t->X, S * 16)) != SVM_OK) return st;
    if ((st = talloc(t, &t->MID, S * 4)) != SVM_OK) return st;
    if ((st = talloc(t, &t->q0, (size_t)n_motions * 48)) != SVM_OK) return st;
    if ((st = talloc(t, &t->q1, (size_t)n_motions * 48)) != SVM_OK) return st;
    TCK(cudaMemcpy(t->q0, q0, (size_t)n_motions * 48, cudaMemcpyHostToDevice));
    TCK(cudaMemcpy(t->q1, q1, (size_t)n_motions * 48, cudaMemcpyHostToDevice));
    Capsule* caps = nullptr;
    MotionState* stt = nullptr;
    TCK(cudaMalloc(&caps, (size_t)n_motions * (steps + 1) * kCaps * sizeof(Capsule)));
    TCK(cudaMalloc(&stt, (size_t)n_motions * sizeof(MotionState)));
    CallArgs a{};
    a.M = n_motions; a.N = steps; a.W = t->W; a.q0 = t->q0; a.q1 = t->q1; a.caps = caps; a.st = stt;
    DevWeights dw{};
    launch_prologue_fk(a, t->rp, dw, 0);
    const size_t smem = (size_t)(steps + 1) * kCaps * sizeof(Capsule);
    cudaFuncSetAttribute(sample_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (kMaxSteps + 1) * kCaps * (int)sizeof(Capsule));
    SampleBox box;
    for (int q = 0; q < 3; ++q) {
        box.lo[q] = t->box_lo[q];
        box.hi[q] = t->box_hi[q];
    }
    sample_kernel<<<n_motions, 256, smem, 0>>>(caps, steps, samples_per_motion, (unsigned long long)seed, box, t->X,
                                               t->MID);
    const cudaError_t e = cudaDeviceSynchronize();
    cudaFree(caps);
    cudaFree(stt);
    if (e != cudaSuccess) return tfail(t, SVM_E_CUDA, std::string("data generation: ") + cudaGetErrorString(e));
    t->n_motions = n_motions;
    t->n_samples = S;
    return SVM_OK;
}

svm_status svm_train_set_box(svm_trainer* t, const double* lo, const double* hi)
{
    if (!t || !lo || !hi) return SVM_E_INVALID;
    for (int q = 0; q < 3; ++q)
        if (!std::isfinite(lo[q]) || !std::isfinite(hi[q]) || !(hi[q] > lo[q]))
            return tfail(t, SVM_E_INVALID, "box needs finite lo < hi");
    for (int q = 0; q < 3; ++q) {
        t->box_lo[q] = lo[q];
        t->box_hi[q] = hi[q];
    }
    return SVM_OK;
}

svm_status svm_train_set_samples(svm_trainer* t, const double* q0, const double* q1, int32_t n_motions,
                                 const float* x4, const int32_t* motion, int64_t n)
{
    if (!t || !q0 || !q1 || !x4 || !motion || n_motions < 1 || n < 1) return tfail(t, SVM_E_INVALID, "bad samples");
    for (long long i = 0; i < n; ++i)
        if (motion[i] < 0 || motion[i] >= n_motions) return tfail(t, SVM_E_INVALID, "motion index out of range");
    DevGuard gd(t->device);
    TCK(cudaDeviceSynchronize());
    free_data(t);
    svm_status st;
    if ((st = talloc(t, &t->X, n * 16)) != SVM_OK) return st;
    if ((st = talloc(t, &t->MID, n * 4)) != SVM_OK) return st;
    if ((st = talloc(t, &t->q0, (size_t)n_motions * 48)) != SVM_OK) return st;
    if ((st = talloc(t, &t->q1, (size_t)n_motions * 48)) != SVM_OK) return st;
    TCK(cudaMemcpy(t->X, x4, n * 16, cudaMemcpyHostToDevice));
    TCK(cudaMemcpy(t->MID, motion, n * 4, cudaMemcpyHostToDevice));
    TCK(cudaMemcpy(t->q0, q0, (size_t)n_motions * 48, cudaMemcpyHostToDevice));
    TCK(cudaMemcpy(t->q1, q1, (size_t)n_motions * 48, cudaMemcpyHostToDevice));
    t->n_motions = n_motions;
    t->n_samples = n;
    return SVM_OK;
}

svm_status svm_train_copy_samples(svm_trainer* t, float* x4_out, int32_t* motion_out, int64_t n)
{
    if (!t || n < 0 || n > t->n_samples) return tfail(t, SVM_E_INVALID, "bad copy");
    DevGuard gd(t->device);
    TCK(cudaDeviceSynchronize());
    if (x4_out) TCK(cudaMemcpy(x4_out, t->X, n * 16, cudaMemcpyDeviceToHost));
    if (motion_out) TCK(cudaMemcpy(motion_out, t->MID, n * 4, cudaMemcpyDeviceToHost));
    return SVM_OK;
}

svm_status svm_train_gradient(svm_trainer* t, int64_t sample_begin, float* grad_out, float* loss_out)
{
    if (!t || !grad_out) return SVM_E_INVALID;
    if (sample_begin < 0 || sample_begin + t->B > t->n_samples) return tfail(t, SVM_E_INVALID, "batch out of range");
    DevGuard gd(t->device);
    TCK(cudaMemset(t->Gr, 0, t->np * 4));
    TCK(cudaMemset(t->loss_sum, 0, 4));
    svm_status st = run_batch(t, sample_begin, 1, true, 0);
    if (st != SVM_OK) return st;
    TCK(cudaGetLastError());
    TCK(cudaDeviceSynchronize());
    TCK(cudaMemcpy(grad_out, t->Gr, t->np * 4, cudaMemcpyDeviceToHost));
    float l = 0;
    TCK(cudaMemcpy(&l, t->loss_sum, 4, cudaMemcpyDeviceToHost));
    if (loss_out) *loss_out = l / (float)t->B;
    unsigned e = 0;
    TCK(cudaMemcpy(&e, t->err, 4, cudaMemcpyDeviceToHost));
    if (e) return tfail(t, SVM_E_TIMEOUT, "a bounded device wait expired");
    return SVM_OK;
}

svm_status adam_on(svm_trainer* t, float lr, cudaStream_t s);

svm_status svm_train_adam(svm_trainer* t, float lr)
{
    if (!t || !(lr > 0)) return SVM_E_INVALID;
    DevGuard gd(t->device);
    return adam_on(t, lr, 0);
}

svm_status adam_on(svm_trainer* t, float lr, cudaStream_t s)
{
    t->step += 1;
    const double b1 = 0.9, b2 = 0.999;
    const float c1 = (float)(1.0 - std::pow(b1, (double)t->step)), c2 = (float)(1.0 - std::pow(b2, (double)t->step));
    adam_hidden_kernel<<<dim3(t->W / 32, t->W / 32, t->L), 256, 0, s>>>(t->P, t->Gr, t->Mo, t->Vo, lr, (float)b1,
                                                                         (float)b2, 1e-8f, c1, c2, t->W, t->off_h, t->wb,
                                                                         t->wbt);
    adam_rest_kernel<<<grid_for(t->off_h + (long long)t->L * t->W + t->W + 1), 256, 0, s>>>(
        t->P, t->Gr, t->Mo, t->Vo, lr, (float)b1, (float)b2, 1e-8f, c1, c2, t->W, t->L, t->off_h, t->off_out);
    TCK(cudaGetLastError());
    return SVM_OK;
}

// Captures one training step (gradient reset and run_batch) on t->main as a
// graph and finds the kernel nodes that take the batch's sample offset.
svm_status capture_step(svm_trainer* t, long long base, long long stride)
{
    cudaGraph_t g = nullptr;
    TCK(cudaStreamBeginCapture(t->main, cudaStreamCaptureModeThreadLocal));
    cudaMemsetAsync(t->Gr, 0, t->np * 4, t->main);
    const svm_status st = run_batch(t, base, stride, true, t->main);
    const cudaError_t ce = cudaStreamEndCapture(t->main, &g);
    if (st != SVM_OK || ce != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return st != SVM_OK ? st : tfail(t, SVM_E_CUDA, "training step capture failed");
    }
    size_t n = 0;
    TCK(cudaGraphGetNodes(g, nullptr, &n));
    std::vector<cudaGraphNode_t> nodes(n);
    TCK(cudaGraphGetNodes(g, nodes.data(), &n));
    const void* f_l1f = t->act == 0 ? (const void*)layer1_fwd_kernel<0> : (const void*)layer1_fwd_kernel<1>;
    const void* f_head = t->act == 0 ? (const void*)head_kernel<0> : (const void*)head_kernel<1>;
    const void* f_l1b = (const void*)layer1_bwd_kernel;
    for (cudaGraphNode_t nd : nodes) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nd, &ty) != cudaSuccess || ty != cudaGraphNodeTypeKernel) continue;
        cudaKernelNodeParams kp{};
        if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) continue;
        if (kp.func == f_l1f) t->node_l1f = nd;
        else if (kp.func == f_head) t->node_head = nd;
        else if (kp.func == f_l1b) t->node_l1b = nd;
    }
    cudaGraphExec_t ex = nullptr;
    if (!t->node_l1f || !t->node_head || !t->node_l1b || cudaGraphInstantiate(&ex, g, 0) != cudaSuccess) {
        cudaGraphDestroy(g);
        t->node_l1f = t->node_head = t->node_l1b = nullptr;
        return tfail(t, SVM_E_CUDA, "training step graph setup failed");
    }
    t->step_graph = g;
    t->step_exec = ex;
    return SVM_OK;
}

// Replays the captured step for the batch at `base`.
svm_status replay_step(svm_trainer* t, long long base, long long stride)
{
    StepArgs a = step_args(t, base, stride);
    auto patch = [&](cudaGraphNode_t nd, void** args) {
        cudaKernelNodeParams kp{};
        if (cudaGraphKernelNodeGetParams(nd, &kp) != cudaSuccess) return false;
        kp.kernelParams = args;
        kp.extra = nullptr;
        return cudaGraphExecKernelNodeSetParams(t->step_exec, nd, &kp) == cudaSuccess;
    };
    const int W = t->W, L = t->L;
    (void)W;
    __nv_bfloat16 *d0 = t->D[0], *h0 = t->H[0], *hl = t->H[L], *dl = t->D[L], *gl = t->G[L], *g0 = t->G[0];
    int eval = 0;
    void* a_l1f[] = {&a, &d0, &h0};
    void* a_head[] = {&a, &hl, &dl, &gl, &eval};
    void* a_l1b[] = {&a, &g0};
    if (!patch(t->node_l1f, a_l1f) || !patch(t->node_head, a_head) || !patch(t->node_l1b, a_l1b))
        return tfail(t, SVM_E_CUDA, "training step graph update failed");
    TCK(cudaGraphLaunch(t->step_exec, t->main));
    return SVM_OK;
}

svm_status svm_train_epoch(svm_trainer* t, int64_t sample_begin, int64_t sample_end, float lr, uint64_t shuffle_seed,
                           float* mean_loss)
{
    const Range call_range("svm_train_epoch");
    if (!t || !(lr > 0)) return SVM_E_INVALID;
    const long long S = sample_end - sample_begin;
    if (sample_begin < 0 || sample_end > t->n_samples || S < t->B) return tfail(t, SVM_E_INVALID, "bad sample range");
    const long long nb = S / t->B;                    // batches per epoch; batch i takes offset perm[i]
    std::vector<long long> perm(nb);
    for (long long i = 0; i < nb; ++i) perm[i] = i;
    std::mt19937_64 rng(shuffle_seed);
    std::shuffle(perm.begin(), perm.end(), rng);
    DevGuard gd(t->device);
    TCK(cudaMemset(t->loss_sum, 0, 4));
    for (long long i = 0; i < nb; ++i) {
        const long long base = sample_begin + perm[i];
        svm_status st = SVM_OK;
        if (i == 0 || !t->step_exec) {
            // eager (the first batch also makes every one-time kernel setting)
            TCK(cudaMemsetAsync(t->Gr, 0, t->np * 4, t->main));
            st = run_batch(t, base, nb, true, t->main);
            if (st == SVM_OK && i == 0 && !t->step_exec) st = capture_step(t, base, nb);
        } else {
            st = replay_step(t, base, nb);
        }
        if (st != SVM_OK) return st;
        st = adam_on(t, lr, t->main);
        if (st != SVM_OK) return st;
    }
    TCK(cudaGetLastError());
    TCK(cudaDeviceSynchronize());
    float l = 0;
    TCK(cudaMemcpy(&l, t->loss_sum, 4, cudaMemcpyDeviceToHost));
    if (mean_loss) *mean_loss = l / (float)(nb * t->B);
    unsigned e = 0;
    TCK(cudaMemcpy(&e, t->err, 4, cudaMemcpyDeviceToHost));
    if (e) return tfail(t, SVM_E_TIMEOUT, "a bounded device wait expired");
    return SVM_OK;
}

svm_status svm_train_evaluate(svm_trainer* t, int64_t sample_begin, int64_t sample_end, float* mae)
{
    if (!t || !mae) return SVM_E_INVALID;
    const long long S = sample_end - sample_begin;
    if (sample_begin < 0 || sample_end > t->n_samples || S < t->B) return tfail(t, SVM_E_INVALID, "bad sample range");
    const long long nb = S / t->B;
    DevGuard gd(t->device);
    TCK(cudaMemset(t->loss_sum, 0, 4));
    for (long long i = 0; i < nb; ++i) {
        svm_status st = run_batch(t, sample_begin + i * t->B, 1, false, 0);
        if (st != SVM_OK) return st;
    }
    TCK(cudaGetLastError());
    TCK(cudaDeviceSynchronize());
    float l = 0;
    TCK(cudaMemcpy(&l, t->loss_sum, 4, cudaMemcpyDeviceToHost));
    *mae = l / (float)(nb * t->B);
    return SVM_OK;
}

svm_status svm_train_state(svm_trainer* t, float* params, float* m1, float* m2, int64_t* step, int64_t n)
{
    if (!t || n != t->np) return tfail(t, SVM_E_INVALID, "state size mismatch");
    DevGuard gd(t->device);
    TCK(cudaDeviceSynchronize());
    if (params) TCK(cudaMemcpy(params, t->P, n * 4, cudaMemcpyDeviceToHost));
    if (m1) TCK(cudaMemcpy(m1, t->Mo, n * 4, cudaMemcpyDeviceToHost));
    if (m2) TCK(cudaMemcpy(m2, t->Vo, n * 4, cudaMemcpyDeviceToHost));
    if (step) *step = t->step;
    return SVM_OK;
}

svm_status svm_train_restore(svm_trainer* t, const float* params, const float* m1, const float* m2, int64_t step,
                             int64_t n)
{
    if (!t || n != t->np || !params || !m1 || !m2 || step < 0) return tfail(t, SVM_E_INVALID, "state size mismatch");
    DevGuard gd(t->device);
    TCK(cudaDeviceSynchronize());
    TCK(cudaMemcpy(t->P, params, n * 4, cudaMemcpyHostToDevice));
    TCK(cudaMemcpy(t->Mo, m1, n * 4, cudaMemcpyHostToDevice));
    TCK(cudaMemcpy(t->Vo, m2, n * 4, cudaMemcpyHostToDevice));
    t->step = step;
    refresh_bf16_kernel<<<grid_for((long long)t->L * t->W * t->W), 256>>>(t->P, t->W, t->L, t->off_h, t->wb, t->wbt);
    TCK(cudaGetLastError());
    TCK(cudaDeviceSynchronize());
    return SVM_OK;
}

int64_t svm_train_param_count(const svm_trainer* t) { return t ? t->np : 0; }

}  // extern "C"
