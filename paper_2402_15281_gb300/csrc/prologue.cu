// prologue.cu -- per-motion set-up of a check call.
//
// (a) Forward kinematics of every sample q_k = ((N-k) q0 + k q1) / N of the
//     linear joint motion (Eq. 2 with s = k/N; the paper discretises motions
//     by joint interpolation, Sec. IV-C), in FP64 -- the only FP64 arithmetic
//     on the GPU -- and the 7 capsules of the robot at that sample, cast once
//     to FP32 for the verifier; the FP64 joint origins and tool axis are kept
//     for the FP64 decision of pairs at the margin.
// (b) The per-motion part of the first network layer.  The input of the
//     network is [x, q0, q1] (Sec. IV-A), so W1 [x; q0; q1] + b1 splits into
//     W1x x + c_m with c_m = W1q [q0; q1] + b1, computed here once per motion
//     instead of once per pair.
// (c) Reset of the per-motion counters and minima, and of the call's tie list.
#include "svm_internal.cuh"

namespace svm {

constexpr int kProThreads = 256;   // samples per round of the FK chains

__global__ void __launch_bounds__(kProThreads) prologue_kernel(CallArgs A, RobotParams R, DevWeights Wt)
{
    const int m = blockIdx.x;
    const double* q0 = A.q0 + m * kDof;
    const double* q1 = A.q1 + m * kDof;
    const int N = A.N;
    // sin and cos of every joint angle of the round's samples, computed by all
    // threads in parallel before the per-sample chains use them
    __shared__ double sc[kProThreads][kDof][2];

    // (a) one thread per sample, kProThreads samples per round
    for (int k0 = 0; k0 <= N; k0 += kProThreads) {
        const int nk = min(kProThreads, N + 1 - k0);
        for (int idx = threadIdx.x; idx < nk * kDof; idx += blockDim.x) {
            const int kk = idx / kDof, j = idx - kk * kDof, k = k0 + kk;
            const double qk = ((double)(N - k) * q0[j] + (double)k * q1[j]) / (double)N;
            sincos(qk + R.th0[j], &sc[kk][j][0], &sc[kk][j][1]);
        }
        __syncthreads();
        const int k = k0 + threadIdx.x;
        if (threadIdx.x < nk) {
        double Rm[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1};
        double p[3] = {0, 0, 0};
        double o[kDof + 1][3];
        o[0][0] = o[0][1] = o[0][2] = 0.0;
        for (int j = 0; j < kDof; ++j) {
            const double st = sc[threadIdx.x][j][0], ct = sc[threadIdx.x][j][1];
            const double ca = R.ca[j], sa = R.sa[j];
            // link transform rotation columns and translation (standard DH)
            const double c0[3] = {ct, st, 0.0};
            const double c1[3] = {-st * ca, ct * ca, sa};
            const double c2[3] = {st * sa, -ct * sa, ca};
            const double t[3] = {R.a[j] * ct, R.a[j] * st, R.d[j]};
            double Rn[9], pn[3];
            for (int r = 0; r < 3; ++r) {
                const double r0 = Rm[r * 3 + 0], r1 = Rm[r * 3 + 1], r2 = Rm[r * 3 + 2];
                Rn[r * 3 + 0] = r0 * c0[0] + r1 * c0[1] + r2 * c0[2];
                Rn[r * 3 + 1] = r0 * c1[0] + r1 * c1[1] + r2 * c1[2];
                Rn[r * 3 + 2] = r0 * c2[0] + r1 * c2[1] + r2 * c2[2];
                pn[r] = r0 * t[0] + r1 * t[1] + r2 * t[2] + p[r];
            }
            for (int i = 0; i < 9; ++i) Rm[i] = Rn[i];
            for (int i = 0; i < 3; ++i) { p[i] = pn[i]; o[j + 1][i] = pn[i]; }
        }
        Capsule* out = A.caps + ((long long)m * (N + 1) + k) * kCaps;
        if (A.fk64 != nullptr) {
            double* f = A.fk64 + ((long long)m * (N + 1) + k) * 24;
            for (int j = 0; j <= kDof; ++j)
                for (int i = 0; i < 3; ++i) f[j * 3 + i] = o[j][i];
            for (int i = 0; i < 3; ++i) f[21 + i] = R.tool_len * Rm[i * 3 + 2];
        }
        for (int j = 0; j < kCaps; ++j) {
            double a3[3], e3[3];
            for (int i = 0; i < 3; ++i) {
                a3[i] = o[j < kDof ? j : kDof][i];
                e3[i] = j < kDof ? o[j + 1][i] - o[j][i] : R.tool_len * Rm[i * 3 + 2];
            }
            const double ee = e3[0] * e3[0] + e3[1] * e3[1] + e3[2] * e3[2];
            Capsule c;
            c.a_r = make_float4((float)a3[0], (float)a3[1], (float)a3[2], R.radius[j]);
            c.e_inv = make_float4((float)e3[0], (float)e3[1], (float)e3[2],
                                  ee > 0.0 ? (float)(1.0 / ee) : 0.0f);
            out[j] = c;
        }
        }
        __syncthreads();
    }

    // (b) c_m = W1q [q0; q1] + b1, q cast to FP32 once.  Block architecture:
    //     the same for the initial layer and for every block (its q-weights
    //     and bias; block 1 has no jump input), then the final layer's scalar.
    if (A.cbias != nullptr) {
        float qf[12];
        for (int i = 0; i < kDof; ++i) { qf[i] = (float)q0[i]; qf[kDof + i] = (float)q1[i]; }
        float* cm = A.cbias + (long long)m * A.cb_stride;
        if (A.arch == 0) {
            for (int o = threadIdx.x; o < A.W; o += blockDim.x) {
                float s = Wt.b1[o];
                const float* wr = Wt.w1q + o * 12;
                #pragma unroll
                for (int i = 0; i < 12; ++i) s = fmaf(wr[i], qf[i], s);
                cm[o] = s;
            }
        } else {
            const int n = (A.L + 1) * A.W;
            for (int k = threadIdx.x; k <= n; k += blockDim.x) {
                const float* wr = k < n ? Wt.blk_wq + (long long)k * 12 : Wt.out_wq;
                float s = k < n ? Wt.blk_b[k] : Wt.bout;
                #pragma unroll
                for (int i = 0; i < 12; ++i) s = fmaf(wr[i], qf[i], s);
                cm[k] = s;
            }
        }
    }

    // (c) counters
    if (threadIdx.x == 0) {
        MotionState z;
        z.n_flagged = 0;
        z.collided = 0;
        z.dmin_key = float_key(__int_as_float(0x7f800000));
        z.dhat_key = float_key(__int_as_float(0x7f800000));
        z.n_verified = 0;
        z.witness_point = -1;
        z.witness_step = -1;
        z.n_ambiguous = 0;
        z.probe_key = ~0ull;
        z.inexact = 0;
        z.pad = 0;
        A.st[m] = z;
        if (m == 0 && A.tie_count) *A.tie_count = 0;
    }
}

void launch_prologue_fk(const CallArgs& a, const RobotParams& rp, const DevWeights& w, cudaStream_t s)
{
    if (a.M > 0) prologue_kernel<<<a.M, kProThreads, 0, s>>>(a, rp, w);
}

}  // namespace svm
