// verify.cu -- the exact geometric check of flagged pairs and the verdicts.
//
// For a point x and motion m the checked distance is the sampled swept-volume
// distance  min_{k=0..N} min_{j<7} ( |x - seg_{m,k,j}| - r_j ),  the minimum
// over the robot's capsules at the N+1 samples of the motion (Eqs. 1, 3-4 with
// the union over s taken on the samples; the geometric checker of Sec. IV-B
// discretises the motion in the same way).  Since r_j does not depend on k,
// each thread keeps, per capsule j, the minimum squared axis distance over k
// and takes 7 square roots at the end.
//
// Work: persistent CTAs walk a list of chunks (256 points of one motion).
// The motion's capsule table is staged in shared memory as packed pairs of
// capsules and read as broadcasts, and the distance tests run on FP32 pairs
// (sub/mul/fma.rn.f32x2: two capsules per instruction, the same roundings as
// the scalar expressions); points are read as float4.  A motion that has collided stops
// its remaining chunks (early exit), as Algorithm 1 needs only the verdict.
#include <mutex>
#include "svm_internal.cuh"

namespace svm {

namespace {

constexpr int VT = 256;   // threads per CTA = points per chunk

// chunk_off[m + 1] - chunk_off[m] = chunks of `chunk` points of motion m;
// one CTA scans the M motions.
__global__ void plan_kernel(CallArgs A, int range_mode, int chunk)
{
    __shared__ int carry;
    __shared__ int warp_sums[32];
    if (threadIdx.x == 0) { carry = 0; A.chunk_off[0] = 0; }
    __syncthreads();
    for (int base = 0; base < A.M; base += blockDim.x) {
        const int m = base + threadIdx.x;
        int c = 0;
        if (m < A.M) {
            const long long n = range_mode ? (A.pend[m] - A.pbeg[m]) : (long long)A.st[m].n_flagged;
            c = (int)((n + chunk - 1) / chunk);
        }
        // block inclusive scan
        int v = c;
        const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
        #pragma unroll
        for (int s = 1; s < 32; s <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, v, s);
            if (lane >= s) v += t;
        }
        if (lane == 31) warp_sums[wid] = v;
        __syncthreads();
        if (wid == 0) {
            int w = lane < (int)(blockDim.x >> 5) ? warp_sums[lane] : 0;
            #pragma unroll
            for (int s = 1; s < 32; s <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, w, s);
                if (lane >= s) w += t;
            }
            warp_sums[lane] = w;
        }
        __syncthreads();
        const int incl = v + (wid > 0 ? warp_sums[wid - 1] : 0) + carry;
        if (m < A.M) A.chunk_off[m + 1] = incl;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = incl;
        __syncthreads();
    }
}

// First sample k at which x is within `margin` of the robot (witness).
__device__ int witness_sample(const Capsule* cs, int n_samples, float3 x, float margin)
{
    for (int k = 0; k < n_samples; ++k) {
        float mn[kCaps];
        scan_samples(cs + k * kCaps, 1, x, mn);
        if (capsule_min(mn, cs + k * kCaps) <= margin) return k;
    }
    return n_samples - 1;
}

// Distance of x to capsule j at sample k of motion m in FP64 (Eqs. 1, 3-5),
// from the prologue's FP64 joint origins and tool axis:
// t = clamp(((x - a) . e) / |e|^2, 0, 1) (0 for a degenerate axis), then
// |x - (a + t e)| - r.
__device__ double capsule_distance64(const CallArgs& A, int m, int k, int j, const double (&x)[3])
{
    const double* f = A.fk64 + ((long long)m * (A.N + 1) + k) * 24;
    double a[3], e[3];
    for (int i = 0; i < 3; ++i) {
        a[i] = f[j * 3 + i];
        e[i] = j < kDof ? f[(j + 1) * 3 + i] - a[i] : f[21 + i];
    }
    const double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    const double we = (x[0] - a[0]) * e[0] + (x[1] - a[1]) * e[1] + (x[2] - a[2]) * e[2];
    double t = ee > 0.0 ? we / ee : 0.0;
    t = t < 0.0 ? 0.0 : (t > 1.0 ? 1.0 : t);
    const double dx = x[0] - (a[0] + t * e[0]), dy = x[1] - (a[1] + t * e[1]), dz = x[2] - (a[2] + t * e[2]);
    return sqrt(dx * dx + dy * dy + dz * dz) - A.rp.radius64[j];
}

// The same distance in FP32 from the capsule table, with the verifier's
// roundings (its minimum over all (k, j) is the verifier's distance).
__device__ __forceinline__ float capsule_distance32(const Capsule& c, float3 x)
{
    const float wx = x.x - c.a_r.x, wy = x.y - c.a_r.y, wz = x.z - c.a_r.z;
    const float t = __saturatef(fmaf(wz, c.e_inv.z, fmaf(wy, c.e_inv.y, wx * c.e_inv.x)) * c.e_inv.w);
    const float dx = fmaf(-t, c.e_inv.x, wx), dy = fmaf(-t, c.e_inv.y, wy), dz = fmaf(-t, c.e_inv.z, wz);
    return sqrtf(fmaf(dz, dz, fmaf(dy, dy, dx * dx))) - c.a_r.w;
}

// ---- packed FP32 pairs: two capsules per instruction
__device__ __forceinline__ uint64_t pk(float lo, float hi)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(uint64_t v, float& lo, float& hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ uint64_t p_sub(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t p_mul(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ uint64_t p_fma(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// The capsule table of one motion in the form the verifier reads: for sample
// k and capsule pair p (capsules 2p and 2p+1; pair 3 repeats capsule 6),
// seven packed pairs (a_x, a_y, a_z, -e_x, -e_y, -e_z, -1/|e|^2).  With the
// negated axis the test below computes exactly the scalar expressions
//   t = sat((w . e) / |e|^2),  d = w - t e,  |d|^2   (w = x - a),
// two capsules per instruction: w.(-e) = -(w.e) and fma(t, -e, w) =
// fma(-t, e, w) bit for bit.  Same size as the Capsule table (224 B per sample).
// (A field-major layout read with 16-byte loads was measured slower: it holds
// the whole sample in registers.)
constexpr int kPairs = 4;
struct CapPair {
    uint64_t ax, ay, az, nex, ney, nez, nei;
};
static_assert(sizeof(CapPair) * kPairs == sizeof(Capsule) * kCaps, "packed table size");

// One chunk = VT * PPT points of one motion; thread t checks points
// t, t + VT, ..., so each capsule read from shared memory serves PPT points.
template <int RANGE, int PPT>
__global__ void __launch_bounds__(VT) verify_kernel(CallArgs A, int strict_pass)
{
    extern __shared__ __align__(16) unsigned char vsm[];
    CapPair* cp = reinterpret_cast<CapPair*>(vsm);
    __shared__ float s_r[kCaps];
    __shared__ int s_m;
    __shared__ int s_skip;
    __shared__ unsigned s_nver, s_namb;
    __shared__ unsigned s_dkey;

    const int n_samples = A.N + 1;
    const int total = A.chunk_off[A.M];
    const bool early = !(A.flags & 2u);
    int cur_m = -1;

    for (int c = blockIdx.x; c < total; c += gridDim.x) {
        if (threadIdx.x == 0) {
            const int m = find_segment(A.chunk_off, A.M, c);
            s_m = m;
            const int path_head = (m / A.path_len) * A.path_len;
            int skip = 0;
            if (early && *(volatile int*)&A.st[path_head].collided) skip = 1;
            // second pass of strict mode: only motions still without a collision
            if (strict_pass && *(volatile int*)&A.st[m].collided) skip = 1;
            s_skip = skip;
            s_nver = 0;
            s_namb = 0;
            s_dkey = 0xffffffffu;
        }
        __syncthreads();
        const int m = s_m;
        if (s_skip) { __syncthreads(); continue; }
        const Capsule* mcaps = A.caps + (long long)m * n_samples * kCaps;
        if (m != cur_m) {
            for (int i = threadIdx.x; i < n_samples * kPairs; i += VT) {
                const int k = i / kPairs, pr = i % kPairs;
                const Capsule c0 = mcaps[k * kCaps + 2 * pr], c1 = mcaps[k * kCaps + min(2 * pr + 1, kCaps - 1)];
                CapPair q;
                q.ax = pk(c0.a_r.x, c1.a_r.x);
                q.ay = pk(c0.a_r.y, c1.a_r.y);
                q.az = pk(c0.a_r.z, c1.a_r.z);
                q.nex = pk(-c0.e_inv.x, -c1.e_inv.x);
                q.ney = pk(-c0.e_inv.y, -c1.e_inv.y);
                q.nez = pk(-c0.e_inv.z, -c1.e_inv.z);
                q.nei = pk(-c0.e_inv.w, -c1.e_inv.w);
                cp[i] = q;
            }
            if (threadIdx.x < kCaps) s_r[threadIdx.x] = mcaps[threadIdx.x].a_r.w;
            cur_m = m;
            __syncthreads();
        }
        const long long base = (long long)(c - A.chunk_off[m]) * VT * PPT + threadIdx.x;
        const long long n = RANGE ? (A.pend[m] - A.pbeg[m]) : (long long)A.st[m].n_flagged;
        float3 x[PPT];
        long long pidx[PPT];
        bool valid[PPT];
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            const long long local = base + (long long)j * VT;
            valid[j] = local < n;
            pidx[j] = 0;
            x[j] = make_float3(0.f, 0.f, 0.f);
            if (valid[j]) {
                pidx[j] = RANGE ? A.pbeg[m] + local : (long long)A.idx[A.pair_off[m] + local];
                const float4 x4 = __ldg(A.points + pidx[j]);
                x[j] = make_float3(x4.x, x4.y, x4.z);
            }
        }
        // per point and capsule: minimum squared axis distance over the samples
        float mn[PPT][2 * kPairs];
        uint64_t X[PPT], Y[PPT], Z[PPT];
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            X[j] = pk(x[j].x, x[j].x);
            Y[j] = pk(x[j].y, x[j].y);
            Z[j] = pk(x[j].z, x[j].z);
#pragma unroll
            for (int q = 0; q < 2 * kPairs; ++q) mn[j][q] = __int_as_float(0x7f800000);
        }
        for (int k = 0; k < n_samples; ++k) {
#pragma unroll
            for (int pr = 0; pr < kPairs; ++pr) {
                const CapPair q = cp[k * kPairs + pr];
                float ni0, ni1;
                upk(q.nei, ni0, ni1);
#pragma unroll
                for (int j = 0; j < PPT; ++j) {
                    const uint64_t wx = p_sub(X[j], q.ax), wy = p_sub(Y[j], q.ay), wz = p_sub(Z[j], q.az);
                    float nd0, nd1;       // -(w . e) for the two capsules
                    upk(p_fma(wz, q.nez, p_fma(wy, q.ney, p_mul(wx, q.nex))), nd0, nd1);
                    const uint64_t t = pk(__saturatef(nd0 * ni0), __saturatef(nd1 * ni1));
                    const uint64_t dx = p_fma(t, q.nex, wx), dy = p_fma(t, q.ney, wy), dz = p_fma(t, q.nez, wz);
                    float d0, d1;
                    upk(p_fma(dz, dz, p_fma(dy, dy, p_mul(dx, dx))), d0, d1);
                    mn[j][2 * pr] = fminf(mn[j][2 * pr], d0);
                    mn[j][2 * pr + 1] = fminf(mn[j][2 * pr + 1], d1);
                }
            }
        }
#pragma unroll
        for (int j = 0; j < PPT; ++j) {
            if (!valid[j]) continue;
            float d = __int_as_float(0x7f800000);
#pragma unroll
            for (int q = 0; q < kCaps; ++q) d = fminf(d, sqrtf(mn[j][q]) - s_r[q]);
            atomicAdd(&s_nver, 1u);
            // within the FP32 error band of the margin: the FP64 tie kernel decides
            // (if the tie list is full, the FP32 verdict stands and the record says so)
            if (fabsf(d - A.margin) < kAmbiguousBand) {
                atomicAdd(&s_namb, 1u);
                const unsigned slot = atomicAdd(A.tie_count, 1u);
                if (slot < tie_capacity(A)) {
                    A.tie_list[slot] = TiePair{m, 0, pidx[j]};
                    continue;
                }
                atomicExch(&A.st[m].inexact, 1u);
            }
            atomicMin(&s_dkey, float_key(d));
            if (d <= A.margin) {
                const int path_head = (m / A.path_len) * A.path_len;
                if (atomicCAS(&A.st[m].collided, 0, 1) == 0) {
                    A.st[m].witness_point = (int)pidx[j];
                    A.st[m].witness_step = witness_sample(mcaps, n_samples, x[j], A.margin);
                }
                if (path_head != m) atomicExch(&A.st[path_head].collided, 1);
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (s_nver) atomicAdd(&A.st[m].n_verified, s_nver);
            if (s_namb) atomicAdd(&A.st[m].n_ambiguous, s_namb);
            if (s_dkey != 0xffffffffu) atomicMin(&A.st[m].dmin_key, s_dkey);
        }
        __syncthreads();
    }
}

// Exact distance of every pair, no gate and no early exit (labels).
__global__ void __launch_bounds__(VT) label_kernel(CallArgs A, float* delta, long long stride)
{
    extern __shared__ __align__(16) unsigned char vsm[];
    Capsule* cs = reinterpret_cast<Capsule*>(vsm);
    const int m = blockIdx.y;
    const int n_samples = A.N + 1;
    const float4* src = reinterpret_cast<const float4*>(A.caps + (long long)m * n_samples * kCaps);
    float4* dst = reinterpret_cast<float4*>(cs);
    for (int i = threadIdx.x; i < n_samples * kCaps * 2; i += VT) dst[i] = __ldg(src + i);
    __syncthreads();
    const long long n = A.pend[m] - A.pbeg[m];
    for (long long local = (long long)blockIdx.x * VT + threadIdx.x; local < n; local += (long long)gridDim.x * VT) {
        const float4 x4 = __ldg(A.points + A.pbeg[m] + local);
        float mn[kCaps];
        scan_samples(cs, n_samples, make_float3(x4.x, x4.y, x4.z), mn);
        delta[(long long)m * stride + local] = capsule_min(mn, cs);
    }
}

// Gate calibration (the margin widened by the measured error of the network):
// the largest overestimate f - delta over the pairs that can collide, delta <=
// near_cut, where f is the network output of the pair (row stride `stride`)
// and delta its exact distance, computed with the label kernel's arithmetic
// (bit for bit the value svm_label_pairs writes; it is never stored).  out[0]
// takes the ordered key of the maximum by atomicMax (0 if no pair qualifies),
// out[1] counts the qualifying pairs; a maximum does not depend on the order
// of the updates, so the result is deterministic.
__global__ void __launch_bounds__(VT) gate_overestimate_kernel(CallArgs A, const float* f, long long stride,
                                                             float near_cut, unsigned int* out)
{
    extern __shared__ __align__(16) unsigned char vsm[];
    Capsule* cs = reinterpret_cast<Capsule*>(vsm);
    const int m = blockIdx.y;
    const int n_samples = A.N + 1;
    const float4* src = reinterpret_cast<const float4*>(A.caps + (long long)m * n_samples * kCaps);
    float4* dst = reinterpret_cast<float4*>(cs);
    for (int i = threadIdx.x; i < n_samples * kCaps * 2; i += VT) dst[i] = __ldg(src + i);
    __syncthreads();
    const long long n = A.pend[m] - A.pbeg[m];
    unsigned int best = 0u, cnt = 0u;
    for (long long local = (long long)blockIdx.x * VT + threadIdx.x; local < n; local += (long long)gridDim.x * VT) {
        const float4 x4 = __ldg(A.points + A.pbeg[m] + local);
        float mn[kCaps];
        scan_samples(cs, n_samples, make_float3(x4.x, x4.y, x4.z), mn);
        const float delta = capsule_min(mn, cs);
        if (delta <= near_cut) {
            best = max(best, float_key(__ldg(f + (long long)m * stride + local) - delta));
            ++cnt;
        }
    }
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        best = max(best, __shfl_xor_sync(0xffffffffu, best, o));
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0 && cnt) {
        atomicMax(out, best);
        atomicAdd(out + 1, cnt);
    }
}

// FP64 decision of the pairs the verifier deferred (FP32 distance within
// kAmbiguousBand of the margin).  One warp per pair, consecutive pairs on
// different CTAs (FP64 throughput is per SM).  The lanes first take the FP32
// distance of every (sample, capsule) item and its minimum lo; FP64 is then
// spent only on items within 4 kAmbiguousBand of lo.  With an FP32 error below
// 2 kAmbiguousBand per item, an item above that cut can neither be the FP64
// minimum nor lie within the margin (the pair's lo is within kAmbiguousBand of
// it), so the result equals the FP64 check of all items.  Collision iff the
// FP64 distance <= margin; the pair's distance enters d_min rounded to FP32
// (rounding is monotone, so a collision never reports d_min above the margin);
// the witness is the first colliding sample.
__global__ void __launch_bounds__(256) tie_kernel(CallArgs A)
{
    const unsigned n = min(*A.tie_count, tie_capacity(A));
    const int lane = threadIdx.x & 31;
    const unsigned n_warps = gridDim.x * (blockDim.x >> 5);
    const int n_items = (A.N + 1) * kCaps;
    for (unsigned i = blockIdx.x + gridDim.x * (threadIdx.x >> 5); i < n; i += n_warps) {
        const TiePair tp = A.tie_list[i];
        const float4 x4 = __ldg(A.points + tp.p);
        const float3 xf = make_float3(x4.x, x4.y, x4.z);
        const double x[3] = {(double)x4.x, (double)x4.y, (double)x4.z};
        const Capsule* cs = A.caps + (long long)tp.m * n_items;
        float lo = __int_as_float(0x7f800000);
        for (int it = lane; it < n_items; it += 32) lo = fminf(lo, capsule_distance32(cs[it], xf));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        const float cut = lo + 4.0f * kAmbiguousBand;
        const double margin = (double)A.margin;
        double best = 1.0 / 0.0;
        int first = 0x7fffffff;
        for (int it = lane; it < n_items; it += 32) {
            if (capsule_distance32(cs[it], xf) > cut) continue;
            const int k = it / kCaps;
            const double dk = capsule_distance64(A, tp.m, k, it - k * kCaps, x);
            best = fmin(best, dk);
            if (dk <= margin && k < first) first = k;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            best = fmin(best, __shfl_xor_sync(0xffffffffu, best, o));
            first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
        }
        if (lane == 0) {
            MotionState& st = A.st[tp.m];
            atomicMin(&st.dmin_key, float_key((float)best));
            if (best <= margin) {
                if (atomicCAS(&st.collided, 0, 1) == 0) {
                    st.witness_point = (int)tp.p;
                    st.witness_step = first;
                }
                const int path_head = (tp.m / A.path_len) * A.path_len;
                if (path_head != tp.m) atomicExch(&A.st[path_head].collided, 1);
            }
        }
    }
}

// Early exit first: before the flagged lists are checked, each motion's
// point of smallest prediction (recorded by the network kernel's gate) is
// checked alone, one warp per motion.  A collision found there (outside the
// margin's FP32 band, which is left to the main pass and the tie kernel)
// marks the motion -- and its path -- as colliding, so the main pass skips
// every chunk of it; otherwise the point is checked again in the main pass,
// which counts it.  The order follows Algorithm 1's use of the prediction to
// choose what to check first, inside one motion.
__global__ void __launch_bounds__(256) probe_kernel(CallArgs A)
{
    const int lane = threadIdx.x & 31;
    const int m = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    if (m >= A.M) return;
    const unsigned long long key = A.st[m].probe_key;
    const int path_head = (m / A.path_len) * A.path_len;
    if (key == ~0ull || *(volatile int*)&A.st[path_head].collided) return;
    const unsigned p = (unsigned)(key & 0xffffffffull);
    const float4 x4 = __ldg(A.points + p);
    const float3 xf = make_float3(x4.x, x4.y, x4.z);
    const int n_items = (A.N + 1) * kCaps;
    const Capsule* cs = A.caps + (long long)m * n_items;
    float d = __int_as_float(0x7f800000);
    int first = 0x7fffffff;
    for (int it = lane; it < n_items; it += 32) {
        const float di = capsule_distance32(cs[it], xf);
        d = fminf(d, di);
        if (di <= A.margin && it / kCaps < first) first = it / kCaps;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        d = fminf(d, __shfl_xor_sync(0xffffffffu, d, o));
        first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
    }
    if (lane != 0 || !(d <= A.margin) || fabsf(d - A.margin) < kAmbiguousBand) return;
    MotionState& st = A.st[m];
    atomicAdd(&st.n_verified, 1u);
    atomicMin(&st.dmin_key, float_key(d));
    if (atomicCAS(&st.collided, 0, 1) == 0) {
        st.witness_point = (int)p;
        st.witness_step = first;
    }
    if (path_head != m) atomicExch(&A.st[path_head].collided, 1);
}

struct ResultRec {
    uint8_t collision, early_exit;
    uint16_t status;
    float d_min, dhat_min;
    uint32_t n_flagged, n_verified;
    int32_t witness_point, witness_step;
    uint32_t n_ambiguous;
};
static_assert(sizeof(ResultRec) == 32, "result record is 32 bytes");

__global__ void finalize_kernel(CallArgs A, ResultRec* out)
{
    const int n_out = A.M / A.path_len;
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_out) return;
    const int seg = A.path_len;
    ResultRec o;
    o.collision = 0;
    o.early_exit = 0;
    o.status = (A.dev_err != nullptr && *A.dev_err != 0u) ? 1 : 0;
    unsigned dk = 0xffffffffu, hk = 0xffffffffu;
    o.n_flagged = 0;
    o.n_verified = 0;
    o.witness_point = -1;
    o.witness_step = -1;
    o.n_ambiguous = 0;
    bool inexact = false;
    for (int s = 0; s < seg; ++s) {
        const MotionState st = A.st[r * seg + s];
        inexact = inexact || st.inexact != 0u;
        dk = min(dk, st.dmin_key);
        hk = min(hk, st.dhat_key);
        o.n_flagged += st.n_flagged;
        o.n_verified += st.n_verified;
        o.n_ambiguous += st.n_ambiguous;
        if (st.collided && st.witness_point >= 0 && o.witness_point < 0) {
            o.witness_point = st.witness_point;
            o.witness_step = s * (A.N + 1) + st.witness_step;
        }
        if (st.collided) o.collision = 1;
    }
    const bool early = !(A.flags & 2u);
    o.early_exit = (early && o.collision) ? 1 : 0;
    o.d_min = key_float(dk);
    o.dhat_min = key_float(hk);
    if (o.status == 0 && inexact) o.status = 2;
    out[r] = o;
}

}  // namespace

namespace {
// The capsule table of one motion can exceed the default 48 KB of dynamic
// shared memory; raise the limit once per device for the kernels that stage it.
// The kernels' shared-memory limits, set once per device; call_once makes the
// first calls from several host threads on one device safe.
std::once_flag g_smem_once[64];

void configure_smem_now()
{
    const int mx = (kMaxSteps + 1) * kCaps * (int)sizeof(Capsule);
    cudaFuncSetAttribute(verify_kernel<0, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(verify_kernel<1, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(verify_kernel<0, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(verify_kernel<1, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(verify_kernel<0, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(verify_kernel<1, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(label_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
    cudaFuncSetAttribute(gate_overestimate_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, mx);
}

void configure_smem()
{
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return;
    std::call_once(g_smem_once[dev], configure_smem_now);
}
}  // namespace

void launch_verify_cfg(const CallArgs& a, int range_mode, int strict_pass, cudaStream_t s, int n_sms,
                       const VerifyConfig& cfg)
{
    if (a.M <= 0) return;
    configure_smem();
    const int ppt = (cfg.points_per_thread == 1 || cfg.points_per_thread == 4) ? cfg.points_per_thread : 2;
    if (!range_mode && !strict_pass && !(a.flags & 2u)) probe_kernel<<<(a.M + 7) / 8, 256, 0, s>>>(a);
    plan_kernel<<<1, 1024, 0, s>>>(a, range_mode, VT * ppt);
    const size_t smem = (size_t)(a.N + 1) * kCaps * sizeof(Capsule);
    // enough resident CTAs to fill the GPU: shared memory bounds CTAs per SM
    int per_sm = (int)((200 * 1024) / (smem + 2048));
    if (per_sm < 1) per_sm = 1;
    if (per_sm > 8) per_sm = 8;
    if (cfg.ctas_per_sm > 0 && cfg.ctas_per_sm < per_sm) per_sm = cfg.ctas_per_sm;
    const int grid = n_sms * per_sm;
    if (ppt == 1) {
        if (range_mode) verify_kernel<1, 1><<<grid, VT, smem, s>>>(a, strict_pass);
        else verify_kernel<0, 1><<<grid, VT, smem, s>>>(a, strict_pass);
    } else if (ppt == 2) {
        if (range_mode) verify_kernel<1, 2><<<grid, VT, smem, s>>>(a, strict_pass);
        else verify_kernel<0, 2><<<grid, VT, smem, s>>>(a, strict_pass);
    } else {
        if (range_mode) verify_kernel<1, 4><<<grid, VT, smem, s>>>(a, strict_pass);
        else verify_kernel<0, 4><<<grid, VT, smem, s>>>(a, strict_pass);
    }
}

void launch_verify(const CallArgs& a, int range_mode, int strict_pass, cudaStream_t s, int n_sms)
{
    launch_verify_cfg(a, range_mode, strict_pass, s, n_sms, VerifyConfig{});
}

void launch_label(const CallArgs& a, float* delta, long long stride, cudaStream_t s)
{
    if (a.M <= 0) return;
    configure_smem();
    const size_t smem = (size_t)(a.N + 1) * kCaps * sizeof(Capsule);
    const int gx = 64;
    label_kernel<<<dim3(gx, a.M), VT, smem, s>>>(a, delta, stride);
}

void launch_gate_overestimate(const CallArgs& a, const float* f, long long stride, float near_cut,
                              unsigned int* out, cudaStream_t s)
{
    if (a.M <= 0) return;
    configure_smem();
    const size_t smem = (size_t)(a.N + 1) * kCaps * sizeof(Capsule);
    const int gx = 64;
    gate_overestimate_kernel<<<dim3(gx, a.M), VT, smem, s>>>(a, f, stride, near_cut, out);
}

void launch_ties(const CallArgs& a, cudaStream_t s, int n_sms)
{
    if (a.M > 0 && a.tie_count) tie_kernel<<<n_sms, 256, 0, s>>>(a);
}

void launch_finalize(const CallArgs& a, void* results, cudaStream_t s)
{
    const int n_out = a.M / a.path_len;
    if (n_out <= 0) return;
    finalize_kernel<<<(n_out + 127) / 128, 128, 0, s>>>(a, reinterpret_cast<ResultRec*>(results));
}

}  // namespace svm
