// mlp_fp32.cu -- the plain FP32 path of the network f(x, q0, q1) (Sec. IV-A)
// on CUDA cores, fused with the gate and the compaction of flagged pairs.
//
// One CTA takes a tile of 64 pairs of one motion (at width 1024 in two passes
// of 32 pairs, so that the activations fit in shared memory), or of 16 pairs
// when all 16-pair tiles of the call fit in one wave on the SMs (a call of few
// pairs: the time is then the network's depth on one SM, and smaller tiles
// spread it over more SMs).  Layer 1 uses the split
// W1 [x; q0; q1] + b1 = W1x x + c_m (c_m from the prologue); the hidden
// layers are register-blocked SIMT GEMMs over activations kept in shared
// memory, with the transposed weights streamed through a double-buffered
// shared-memory ring (cp.async); the output layer is a dot product reduced
// with warp shuffles.  Then f <= gate flags a pair (Algorithm 1 checks the
// motions whose prediction is under the margin), a warp ballot counts the
// flags and one atomicAdd per warp reserves their slots in the motion's index
// list, and the motion's minimum prediction d^(X, m) of Eq. 6 is kept with
// an atomic minimum.
#include <mutex>
#include "svm_internal.cuh"

namespace svm {

namespace {

constexpr int BM_LARGE = 64;  // pairs per tile
constexpr int BM_SMALL = 16;  // pairs per tile of small calls
constexpr int NT = 256;       // threads: 16 row groups x 16 column groups
constexpr int HPAD = 4;       // row padding of the activation tile (floats)

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// W: network width.  KC: hidden-weight rows per pipeline stage.  BLOCK: the
// block architecture (initial layer without activation; per block
// h = s * relu(W h + Wx x + c_{m,l}) + t + h, the jump input's q-part folded
// into c_{m,l} by the prologue, BatchNorm folded into s and t; final layer
// w_f . h + w_fx . x + c_{m,f}).
template <int W, int KC, bool BLOCK, int BM>
__global__ void __launch_bounds__(NT, 1) mlp_fp32_kernel(CallArgs A, DevWeights Wt)
{
    constexpr int CPT = W / 16;          // columns per thread
    constexpr int CG = CPT / 4;          // float4 column groups per thread
    constexpr int HS = W + HPAD;         // activation row stride
    constexpr int BMP = (W > 512 && BM > 32) ? 32 : BM;   // pairs per pass
    constexpr int RPT = BMP / 16;        // rows per thread
    constexpr int NPASS = BM / BMP;
    extern __shared__ __align__(16) float smem[];
    float* H = smem;                     // [BMP][HS] activations of the pass, row-major
    float* WS = smem + BMP * HS;         // [2][KC][W] transposed weight stages
    __shared__ float f_s[BM];
    __shared__ float4 x_s[BM];           // the tile's points (block architecture)

    const int tid = threadIdx.x;
    const int ty = tid >> 4, tx = tid & 15;
    const int tile = blockIdx.x;
    const int m = find_segment(A.tile_off, A.M, tile);
    const long long p0 = A.pbeg[m] + (long long)(tile - A.tile_off[m]) * BM;
    const long long pe = A.pend[m];
    const float* cb = A.cbias + (long long)m * A.cb_stride;

    // stage loader: flat chunk g = layer * (W/KC) + kc
    constexpr int CHUNKS_PER_LAYER = W / KC;
    const int total_chunks = A.L * CHUNKS_PER_LAYER;
    auto load_chunk = [&](int g, int buf) {
        const int l = g / CHUNKS_PER_LAYER, kc = g % CHUNKS_PER_LAYER;
        const float* src = Wt.wT + ((long long)l * W + kc * KC) * W;
        float* dst = WS + buf * KC * W;
        #pragma unroll
        for (int i = tid; i < KC * W / 4; i += NT) cp_async16(dst + i * 4, src + i * 4);
        cp_async_commit();
    };
    for (int pass = 0; pass < NPASS; ++pass) {
        const int r0 = pass * BMP;           // first tile row of this pass
        if (pass > 0) __syncthreads();       // the previous pass is done with H and WS
        if (total_chunks > 0) load_chunk(0, 0);

        // ---- layer 1: h = act(W1x x + c_m)
        {
            float4 xr[RPT];
            #pragma unroll
            for (int r = 0; r < RPT; ++r) {
                const long long p = p0 + r0 + ty * RPT + r;
                xr[r] = p < pe ? __ldg(A.points + p) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
            #pragma unroll
            for (int c = 0; c < CG; ++c) {
                #pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int o = tx * 4 + 64 * c + i;
                    const float w0 = __ldg(Wt.w1x + o * 3 + 0), w1 = __ldg(Wt.w1x + o * 3 + 1),
                                w2 = __ldg(Wt.w1x + o * 3 + 2), bo = __ldg(cb + o);
                    #pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        const float z = fmaf(w2, xr[r].z, fmaf(w1, xr[r].y, fmaf(w0, xr[r].x, bo)));
                        H[(ty * RPT + r) * HS + o] = BLOCK ? z : act_fn(z, A.act);
                    }
                }
            }
            if (BLOCK && tx == 0) {
                #pragma unroll
                for (int r = 0; r < RPT; ++r) x_s[r0 + ty * RPT + r] = xr[r];
            }
        }
        // calibration: the largest magnitude entering each hidden layer (valid rows only)
        auto record_amax = [&](int layer) {
            float mx = 0.0f;
            for (int r = 0; r < RPT; ++r) {
                if (p0 + r0 + ty * RPT + r >= pe) continue;
                for (int c = 0; c < CG; ++c)
                    for (int i = 0; i < 4; ++i) mx = fmaxf(mx, fabsf(H[(ty * RPT + r) * HS + tx * 4 + 64 * c + i]));
            }
            #pragma unroll
            for (int s = 16; s > 0; s >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, s));
            if ((tid & 31) == 0) atomicMax(A.amax + layer, __float_as_uint(mx));
        };
        if (A.amax != nullptr && A.L > 0) { __syncthreads(); record_amax(0); }

        float acc[RPT][CPT];
        float fpart[RPT];
        #pragma unroll
        for (int r = 0; r < RPT; ++r) fpart[r] = 0.f;
        int g = 0;
        for (int l = 0; l < A.L; ++l) {
            #pragma unroll
            for (int r = 0; r < RPT; ++r)
                #pragma unroll
                for (int j = 0; j < CPT; ++j) acc[r][j] = 0.f;

            for (int kc = 0; kc < CHUNKS_PER_LAYER; ++kc, ++g) {
                if (g + 1 < total_chunks) { load_chunk(g + 1, (g + 1) & 1); cp_async_wait<1>(); }
                else cp_async_wait<0>();
                __syncthreads();
                const float* ws = WS + (g & 1) * KC * W;
                #pragma unroll 2
                for (int k4 = 0; k4 < KC; k4 += 4) {
                    float4 a4[RPT];
                    #pragma unroll
                    for (int r = 0; r < RPT; ++r)
                        a4[r] = *reinterpret_cast<const float4*>(H + (ty * RPT + r) * HS + kc * KC + k4);
                    #pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        float av[RPT];
                        #pragma unroll
                        for (int r = 0; r < RPT; ++r)
                            av[r] = kk == 0 ? a4[r].x : kk == 1 ? a4[r].y : kk == 2 ? a4[r].z : a4[r].w;
                        #pragma unroll
                        for (int c = 0; c < CG; ++c) {
                            const float4 b = *reinterpret_cast<const float4*>(ws + (k4 + kk) * W + tx * 4 + 64 * c);
                            #pragma unroll
                            for (int r = 0; r < RPT; ++r) {
                                acc[r][c * 4 + 0] = fmaf(av[r], b.x, acc[r][c * 4 + 0]);
                                acc[r][c * 4 + 1] = fmaf(av[r], b.y, acc[r][c * 4 + 1]);
                                acc[r][c * 4 + 2] = fmaf(av[r], b.z, acc[r][c * 4 + 2]);
                                acc[r][c * 4 + 3] = fmaf(av[r], b.w, acc[r][c * 4 + 3]);
                            }
                        }
                    }
                }
                __syncthreads();   // stage (g & 1) and H reads done
            }

            if constexpr (BLOCK) {
                // z = W h + Wx x + c_{m,l}; h <- s relu(z) + t + h (own elements, after the GEMM's reads)
                const float* cl = cb + (long long)(l + 1) * W;
                const float* wxl = Wt.blk_wx + (long long)l * W * 3;
                const float* sl = Wt.blk_s + (long long)l * W;
                const float* tl = Wt.blk_t + (long long)l * W;
                const bool last = l + 1 == A.L;
                #pragma unroll
                for (int c = 0; c < CG; ++c)
                    #pragma unroll
                    for (int i = 0; i < 4; ++i) {
                        const int o = tx * 4 + 64 * c + i;
                        const float w0 = __ldg(wxl + o * 3 + 0), w1 = __ldg(wxl + o * 3 + 1), w2 = __ldg(wxl + o * 3 + 2);
                        const float co = __ldg(cl + o), so = __ldg(sl + o), to = __ldg(tl + o);
                        const float wo = last ? __ldg(Wt.wout + o) : 0.0f;
                        #pragma unroll
                        for (int r = 0; r < RPT; ++r) {
                            const float4 x = x_s[r0 + ty * RPT + r];
                            const float z = fmaf(w2, x.z, fmaf(w1, x.y, fmaf(w0, x.x, acc[r][c * 4 + i] + co)));
                            float* hp = H + (ty * RPT + r) * HS + o;
                            const float h = fmaf(so, fmaxf(z, 0.0f), to) + *hp;
                            if (last) fpart[r] = fmaf(wo, h, fpart[r]);
                            else *hp = h;
                        }
                    }
                if (!last) __syncthreads();
                continue;
            }
            const float* bl = Wt.bh + (long long)l * W;
            if (l + 1 < A.L) {
                // epilogue: bias + activation back into the activation tile
                #pragma unroll
                for (int c = 0; c < CG; ++c) {
                    const int o = tx * 4 + 64 * c;
                    const float4 bb = __ldg(reinterpret_cast<const float4*>(bl + o));
                    #pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        float4 h;
                        h.x = act_fn(acc[r][c * 4 + 0] + bb.x, A.act);
                        h.y = act_fn(acc[r][c * 4 + 1] + bb.y, A.act);
                        h.z = act_fn(acc[r][c * 4 + 2] + bb.z, A.act);
                        h.w = act_fn(acc[r][c * 4 + 3] + bb.w, A.act);
                        *reinterpret_cast<float4*>(H + (ty * RPT + r) * HS + o) = h;
                    }
                }
                __syncthreads();
                if (A.amax != nullptr) record_amax(l + 1);
            } else {
                // last hidden layer: fold the output layer into the epilogue
                #pragma unroll
                for (int c = 0; c < CG; ++c) {
                    const int o = tx * 4 + 64 * c;
                    const float4 bb = __ldg(reinterpret_cast<const float4*>(bl + o));
                    const float4 wo = __ldg(reinterpret_cast<const float4*>(Wt.wout + o));
                    #pragma unroll
                    for (int r = 0; r < RPT; ++r) {
                        fpart[r] = fmaf(wo.x, act_fn(acc[r][c * 4 + 0] + bb.x, A.act), fpart[r]);
                        fpart[r] = fmaf(wo.y, act_fn(acc[r][c * 4 + 1] + bb.y, A.act), fpart[r]);
                        fpart[r] = fmaf(wo.z, act_fn(acc[r][c * 4 + 2] + bb.z, A.act), fpart[r]);
                        fpart[r] = fmaf(wo.w, act_fn(acc[r][c * 4 + 3] + bb.w, A.act), fpart[r]);
                    }
                }
            }
        }
        if (A.L == 0) {
            // no hidden layer: output directly from the layer-1 activations
            __syncthreads();
            #pragma unroll
            for (int c = 0; c < CG; ++c)
                #pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int o = tx * 4 + 64 * c + i;
                    #pragma unroll
                    for (int r = 0; r < RPT; ++r) fpart[r] = fmaf(__ldg(Wt.wout + o), H[(ty * RPT + r) * HS + o], fpart[r]);
                }
        }

        // reduce the output dot over the 16 column groups (one half-warp)
        #pragma unroll
        for (int r = 0; r < RPT; ++r) {
            float v = fpart[r];
            v += __shfl_xor_sync(0xffffffffu, v, 8);
            v += __shfl_xor_sync(0xffffffffu, v, 4);
            v += __shfl_xor_sync(0xffffffffu, v, 2);
            v += __shfl_xor_sync(0xffffffffu, v, 1);
            if (tx == 0) {
                if constexpr (BLOCK) {
                    const float4 x = x_s[r0 + ty * RPT + r];
                    const float* ow = Wt.out_wx;
                    f_s[r0 + ty * RPT + r] = v + fmaf(__ldg(ow + 2), x.z, fmaf(__ldg(ow + 1), x.y,
                                                                        fmaf(__ldg(ow), x.x, cb[(long long)(A.L + 1) * W])));
                } else {
                    f_s[r0 + ty * RPT + r] = v + Wt.bout;
                }
            }
        }
    }   // passes
    __syncthreads();

    // gate + compaction + running minimum (whole warps, one pair per lane)
    if (tid < (BM + 31) / 32 * 32) {
        const long long p = p0 + tid;
        const bool valid = tid < BM && p < pe;
        const float f = tid < BM ? f_s[tid] : __int_as_float(0x7f800000);
        if (A.f_out != nullptr && valid)
            A.f_out[(long long)m * A.f_stride + (p - A.pbeg[m])] = f;
        const bool flag = valid && f <= A.gate;
        const unsigned mask = __ballot_sync(0xffffffffu, flag);
        const int lane = tid & 31;
        unsigned base = 0;
        if (lane == 0 && mask) base = atomicAdd(&A.st[m].n_flagged, (unsigned)__popc(mask));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (flag) {
            const unsigned slot = base + __popc(mask & ((1u << lane) - 1u));
            A.idx[A.pair_off[m] + slot] = (unsigned)p;
        }
        float fm = valid ? f : __int_as_float(0x7f800000);
        #pragma unroll
        for (int s = 16; s > 0; s >>= 1) fm = fminf(fm, __shfl_xor_sync(0xffffffffu, fm, s));
        if (lane == 0 && fm < __int_as_float(0x7f800000)) atomicMin(&A.st[m].dhat_key, float_key(fm));
        if (fm <= A.gate) {            // the warp's smallest prediction is flagged: a probe candidate
            const unsigned who = __ballot_sync(0xffffffffu, valid && f == fm);
            const unsigned pi = __shfl_sync(0xffffffffu, (unsigned)p, __ffs(who) - 1);
            if (lane == 0) atomicMin(&A.st[m].probe_key, ((unsigned long long)float_key(fm) << 32) | pi);
        }
    }
}

template <int W, int KC, bool BLOCK, int BM>
void launch_wb(const CallArgs& a, const DevWeights& w, int n_tiles, cudaStream_t s)
{
    constexpr int BMP = (W > 512 && BM > 32) ? 32 : BM;
    const size_t smem = (size_t)(BMP * (W + HPAD) + 2 * KC * W) * sizeof(float);
    int dev = 0;
    cudaGetDevice(&dev);
    static std::once_flag configured[64];      // once per device, safe across host threads
    if (dev >= 0 && dev < 64)
        std::call_once(configured[dev], [smem] {
            cudaFuncSetAttribute(mlp_fp32_kernel<W, KC, BLOCK, BM>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
        });
    mlp_fp32_kernel<W, KC, BLOCK, BM><<<n_tiles, NT, smem, s>>>(a, w);
}

template <int W, int KC>
void launch_w(const CallArgs& a, const DevWeights& w, int n_tiles, int bm, cudaStream_t s)
{
    if (bm == BM_SMALL) {
        if (a.arch == 1) launch_wb<W, KC, true, BM_SMALL>(a, w, n_tiles, s);
        else launch_wb<W, KC, false, BM_SMALL>(a, w, n_tiles, s);
    } else {
        if (a.arch == 1) launch_wb<W, KC, true, BM_LARGE>(a, w, n_tiles, s);
        else launch_wb<W, KC, false, BM_LARGE>(a, w, n_tiles, s);
    }
}

}  // namespace

// A 16-pair tile takes 0.5-0.65 of a 64-pair tile's time (measured), so 16-pair
// tiles win only when they all run in one wave.
int mlp_fp32_tile_rows(long long tiles_small, int n_sms)
{
    return tiles_small <= (long long)n_sms ? BM_SMALL : BM_LARGE;
}

int mlp_fp32_small_tile_rows() { return BM_SMALL; }

int mlp_fp32_tile_rows() { return BM_LARGE; }

void launch_mlp_fp32(const CallArgs& a, const DevWeights& w, int n_tiles, int bm, cudaStream_t s)
{
    if (n_tiles <= 0) return;
    switch (a.W) {
        case 64: launch_w<64, 32>(a, w, n_tiles, bm, s); break;
        case 128: launch_w<128, 32>(a, w, n_tiles, bm, s); break;
        case 256: launch_w<256, 32>(a, w, n_tiles, bm, s); break;
        case 512: launch_w<512, 16>(a, w, n_tiles, bm, s); break;
        case 1024: launch_w<1024, 8>(a, w, n_tiles, bm, s); break;
        default: break;
    }
}

}  // namespace svm
