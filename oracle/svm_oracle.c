/*
 * svm_oracle.c -- plain FP64 CPU oracle for the neural implicit swept-volume
 * collision check (Joho, Schwinn, Safronov, "Neural Implicit Swept Volume
 * Models for Fast Collision Detection", arXiv 2402.15281).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct
 * statement of what the GPU path computes.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark load it.  It shares no code,
 * header, table or helper with the CUDA library: it is written from the
 * paper's definitions, in double precision, with no blocking or fusion.
 *
 * Parts and the passages they follow:
 *   orc_fk, orc_capsules      robot pose V_R(q) of Sec. III; the arm is a
 *                             standard-DH 6R chain of 7 capsules (the paper's
 *                             KUKA meshes are not available).
 *   orc_point_capsule         signed distance d(x, V) of Eq. 1 for one capsule.
 *   orc_robot_sdf             d(x, V_R(q)) for the union of the capsules.
 *   orc_swept_sdf             f_d(x, m) of Eq. 1 with V_S(m) of Eqs. 3-4, the
 *                             union over s taken on the N+1 samples of the
 *                             linear joint motion c(m, s) of Eq. 2, as the
 *                             paper's data generation discretises it (Sec. IV-C).
 *   orc_gcc_motion            d(X, m) of Eq. 5: exact minimum over the cloud.
 *   orc_mlp_forward           the network f_theta(x, q0, q1) (Sec. IV-A), as a
 *                             plain MLP: 15 -> W, L hidden W -> W, W -> 1.
 *   orc_check_motions         the margin-gated combined check: network
 *                             minimum d^(X, m) of Eq. 6, gate, exact check of
 *                             the flagged points, verdict "free iff > eps_S"
 *                             (Sec. IV-B, Algorithm 1).
 *   orc_mlp_loss_grad         L1 training loss and its gradient (backprop).
 *   orc_mlp_loss_grad_bf16    the same backpropagation with bfloat16 rounding
 *                             of the hidden weights in their products and of
 *                             H = act(z), D = act'(z) (both of the unrounded
 *                             pre-activation) and each hidden layer's
 *                             gradient G (the values a BF16 training step
 *                             stores).
 *   orc_adam_step             Adam update with bias correction (Sec. V).
 *   orc_round_bf16,
 *   orc_round_e4m3            the quantisers that define the BF16 and FP8
 *                             E4M3 weights (round to nearest, ties to even).
 *   orc_splitmix64_u01,
 *   orc_training_points       the counter-based sampler of training points.
 *
 * Conventions: all arrays are row-major; q is 6 joint angles (rad); points
 * are (n, 3) doubles; distances are in metres, positive outside the robot.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>
#include <stdlib.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define DOF 6
#define NCAPS 7

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ---------------------------------------------------------------- FK ---- */

static void mat4_identity(double M[16])
{
    memset(M, 0, 16 * sizeof(double));
    M[0] = M[5] = M[10] = M[15] = 1.0;
}

static void mat4_mul(const double A[16], const double B[16], double C[16])
{
    double R[16];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double s = 0.0;
            for (int k = 0; k < 4; ++k) s += A[i * 4 + k] * B[k * 4 + j];
            R[i * 4 + j] = s;
        }
    memcpy(C, R, sizeof R);
}

static void rot_z(double th, double M[16])
{
    mat4_identity(M);
    M[0] = cos(th); M[1] = -sin(th);
    M[4] = sin(th); M[5] = cos(th);
}

static void rot_x(double al, double M[16])
{
    mat4_identity(M);
    M[5] = cos(al); M[6] = -sin(al);
    M[9] = sin(al); M[10] = cos(al);
}

static void trans(double x, double y, double z, double M[16])
{
    mat4_identity(M);
    M[3] = x; M[7] = y; M[11] = z;
}

/* Frames T_0..T_6 of the standard Denavit-Hartenberg chain:
 *   T_0 = I,  T_j = T_{j-1} Rz(q_j + theta_j) Tz(d_j) Tx(a_j) Rx(alpha_j).
 * dh is (6, 4): d, a, alpha, theta offset.  T is (7, 16). */
void orc_fk(const double *dh, const double *q, double *T)
{
    double M[16], E[16];
    mat4_identity(M);
    memcpy(T, M, sizeof M);
    for (int j = 0; j < DOF; ++j) {
        const double d = dh[j * 4 + 0], a = dh[j * 4 + 1];
        const double alpha = dh[j * 4 + 2], th0 = dh[j * 4 + 3];
        rot_z(q[j] + th0, E);       mat4_mul(M, E, M);
        trans(0.0, 0.0, d, E);      mat4_mul(M, E, M);
        trans(a, 0.0, 0.0, E);      mat4_mul(M, E, M);
        rot_x(alpha, E);            mat4_mul(M, E, M);
        memcpy(T + 16 * (j + 1), M, sizeof M);
    }
}

/* The 7 capsule axes of the robot at q.  Capsule j < 6 joins the origins of
 * frames j and j+1; capsule 6 starts at the origin of frame 6 and runs
 * tool_len along that frame's z axis.  a, b are (7, 3). */
void orc_capsules(const double *dh, double tool_len, const double *q, double *a, double *b)
{
    double T[7 * 16];
    orc_fk(dh, q, T);
    for (int j = 0; j < 6; ++j)
        for (int c = 0; c < 3; ++c) {
            a[j * 3 + c] = T[16 * j + 4 * c + 3];
            b[j * 3 + c] = T[16 * (j + 1) + 4 * c + 3];
        }
    for (int c = 0; c < 3; ++c) {
        a[18 + c] = T[16 * 6 + 4 * c + 3];
        b[18 + c] = T[16 * 6 + 4 * c + 3] + tool_len * T[16 * 6 + 4 * c + 2];
    }
}

/* ------------------------------------------------------- distances ---- */

/* Signed distance from x to the capsule of axis a-b and radius r: distance to
 * the closest point of the segment, minus r.  A zero-length axis is a sphere. */
double orc_point_capsule(const double *x, const double *a, const double *b, double r)
{
    double e[3], w[3];
    for (int c = 0; c < 3; ++c) { e[c] = b[c] - a[c]; w[c] = x[c] - a[c]; }
    const double ee = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
    double t = 0.0;
    if (ee > 0.0) {
        t = (w[0] * e[0] + w[1] * e[1] + w[2] * e[2]) / ee;
        if (t < 0.0) t = 0.0;
        if (t > 1.0) t = 1.0;
    }
    double s = 0.0;
    for (int c = 0; c < 3; ++c) {
        const double p = a[c] + t * e[c];
        s += (x[c] - p) * (x[c] - p);
    }
    return sqrt(s) - r;
}

/* Signed distance to the robot at pose (a, b): the minimum over its capsules
 * (exact outside the union, a lower bound of the depth inside). */
static double robot_sdf_caps(const double *x, const double *a, const double *b, const double *radius)
{
    double best = INFINITY;
    for (int j = 0; j < NCAPS; ++j) {
        const double d = orc_point_capsule(x, a + 3 * j, b + 3 * j, radius[j]);
        if (d < best) best = d;
    }
    return best;
}

double orc_robot_sdf(const double *dh, double tool_len, const double *radius,
                     const double *q, const double *x)
{
    double a[NCAPS * 3], b[NCAPS * 3];
    orc_capsules(dh, tool_len, q, a, b);
    return robot_sdf_caps(x, a, b, radius);
}

/* Joint configuration at sample k of N of the linear motion q0 -> q1 (Eq. 2
 * with s = k / N), written as ((N - k) q0 + k q1) / N. */
static void motion_sample(const double *q0, const double *q1, int k, int N, double *qk)
{
    for (int i = 0; i < DOF; ++i)
        qk[i] = ((double)(N - k) * q0[i] + (double)k * q1[i]) / (double)N;
}

/* Capsules of the N+1 sampled poses of one motion: (N+1, 7, 3) each. */
static void motion_capsules(const double *dh, double tool_len, const double *q0,
                            const double *q1, int N, double *A, double *B)
{
    double qk[DOF];
    for (int k = 0; k <= N; ++k) {
        motion_sample(q0, q1, k, N, qk);
        orc_capsules(dh, tool_len, qk, A + k * NCAPS * 3, B + k * NCAPS * 3);
    }
}

/* Ground-truth swept-volume SDF: min over the N+1 sampled poses of the robot
 * SDF (Eqs. 1, 3, 4, with the union over s sampled).  N = 0 means the static
 * robot at q0. */
double orc_swept_sdf(const double *dh, double tool_len, const double *radius,
                     const double *q0, const double *q1, int N, const double *x)
{
    if (N <= 0) return orc_robot_sdf(dh, tool_len, radius, q0, x);
    double qk[DOF], best = INFINITY;
    for (int k = 0; k <= N; ++k) {
        motion_sample(q0, q1, k, N, qk);
        const double d = orc_robot_sdf(dh, tool_len, radius, qk, x);
        if (d < best) best = d;
    }
    return best;
}

/* delta[m][i] = swept SDF of point i for motion m, for all M x n pairs. */
void orc_swept_sdf_batch(const double *dh, double tool_len, const double *radius,
                         const double *q0, const double *q1, int M, int N,
                         const double *pts, long n, double *delta)
{
    for (int m = 0; m < M; ++m) {
        const int K = N > 0 ? N : 0;
        double A[(K + 1) * NCAPS * 3], B[(K + 1) * NCAPS * 3];
        if (N > 0) {
            motion_capsules(dh, tool_len, q0 + m * DOF, q1 + m * DOF, N, A, B);
        } else {
            orc_capsules(dh, tool_len, q0 + m * DOF, A, B);
        }
        #pragma omp parallel for schedule(static)
        for (long i = 0; i < n; ++i) {
            double best = INFINITY;
            for (int k = 0; k <= K; ++k) {
                const double d = robot_sdf_caps(pts + 3 * i, A + k * NCAPS * 3, B + k * NCAPS * 3, radius);
                if (d < best) best = d;
            }
            delta[(long)m * n + i] = best;
        }
    }
}

/* d(X, m) of Eq. 5 for every motion: the exact minimum over the whole cloud,
 * and the collision verdict "collision iff d <= eps" (free iff d > eps_S). */
void orc_gcc_motion(const double *dh, double tool_len, const double *radius,
                    const double *q0, const double *q1, int M, int N,
                    const double *pts, long n, double eps, double *dmin, int32_t *collision)
{
    for (int m = 0; m < M; ++m) {
        double A[(N + 1) * NCAPS * 3], B[(N + 1) * NCAPS * 3];
        motion_capsules(dh, tool_len, q0 + m * DOF, q1 + m * DOF, N, A, B);
        double best = INFINITY;
        #pragma omp parallel for schedule(static) reduction(min:best)
        for (long i = 0; i < n; ++i) {
            for (int k = 0; k <= N; ++k) {
                const double d = robot_sdf_caps(pts + 3 * i, A + k * NCAPS * 3, B + k * NCAPS * 3, radius);
                if (d < best) best = d;
            }
        }
        dmin[m] = best;
        collision[m] = best <= eps;
    }
}

/* ------------------------------------------------------------- MLP ---- */

/* Parameter layout (shared by forward, backward and Adam): for each layer
 * l = 0 .. L+1 in order, W_l (out x in, row-major) then b_l (out).  Layer 0
 * is 15 -> W, layers 1..L are W -> W, layer L+1 is W -> 1.  Input columns are
 * [x, y, z, q0_1..q0_6, q1_1..q1_6]. */
long orc_param_count(int width, int n_hidden)
{
    return (long)width * 15 + width + (long)n_hidden * ((long)width * width + width) + width + 1;
}

static double act_f(double z, int act)
{
    if (act == 0) return z > 0.0 ? z : 0.0;          /* ReLU */
    return z / (1.0 + exp(-z));                        /* SiLU */
}

static double act_df(double z, int act)
{
    if (act == 0) return z > 0.0 ? 1.0 : 0.0;
    const double s = 1.0 / (1.0 + exp(-z));
    return s * (1.0 + z * (1.0 - s));
}

/* One input row through the network; h holds (L+1) x W activations and z the
 * matching pre-activations (both may be NULL-free scratch of that size). */
static double mlp_row(const double *P, int width, int n_hidden, int act,
                      const double *in, double *z, double *h)
{
    const double *W = P, *b = P + (long)width * 15;
    for (int o = 0; o < width; ++o) {
        double s = b[o];
        for (int i = 0; i < 15; ++i) s += W[(long)o * 15 + i] * in[i];
        z[o] = s;
        h[o] = act_f(s, act);
    }
    const double *p = b + width;
    for (int l = 1; l <= n_hidden; ++l) {
        const double *Wl = p, *bl = p + (long)width * width;
        const double *hp = h + (long)(l - 1) * width;
        for (int o = 0; o < width; ++o) {
            double s = bl[o];
            for (int i = 0; i < width; ++i) s += Wl[(long)o * width + i] * hp[i];
            z[(long)l * width + o] = s;
            h[(long)l * width + o] = act_f(s, act);
        }
        p = bl + width;
    }
    const double *hl = h + (long)n_hidden * width;
    double f = p[width];
    for (int i = 0; i < width; ++i) f += p[i] * hl[i];
    return f;
}

/* f_theta for n input rows of 15 values each. */
void orc_mlp_forward(const double *P, int width, int n_hidden, int act,
                     const double *inputs, long n, double *out)
{
    #pragma omp parallel
    {
        double z[(n_hidden + 1) * width], h[(n_hidden + 1) * width];
        #pragma omp for schedule(static)
        for (long r = 0; r < n; ++r)
            out[r] = mlp_row(P, width, n_hidden, act, inputs + 15 * r, z, h);
    }
}

/* f_theta for every (motion, point) pair: out[m][i]. */
void orc_mlp_pairs(const double *P, int width, int n_hidden, int act,
                   const double *q0, const double *q1, int M,
                   const double *pts, long n, double *out)
{
    #pragma omp parallel
    {
        double z[(n_hidden + 1) * width], h[(n_hidden + 1) * width], in[15];
        #pragma omp for schedule(static) collapse(2)
        for (int m = 0; m < M; ++m)
            for (long i = 0; i < n; ++i) {
                for (int c = 0; c < 3; ++c) in[c] = pts[3 * i + c];
                for (int c = 0; c < DOF; ++c) {
                    in[3 + c] = q0[m * DOF + c];
                    in[9 + c] = q1[m * DOF + c];
                }
                out[(long)m * n + i] = mlp_row(P, width, n_hidden, act, in, z, h);
            }
    }
}

/* The network as a reduced-precision model evaluates it: the input of every
 * hidden layer is rounded to the model's activation format before the layer
 * (fmt 1: nearest-even bfloat16; fmt 2: FP8 E4M3 as e4m3(h / s_l) * s_l with
 * the per-layer scale s_l), everything else in double.  fmt 0 is the plain
 * network.  out[m][i] for all pairs, like orc_mlp_pairs. */
float orc_round_bf16(float v);
double orc_round_e4m3(double v);

/* One input row through the network with the input of hidden layer l
 * rounded to format fmts[l] (0 none, 1 bfloat16, 2 E4M3 with scale
 * scales[l]); h and z hold width doubles each. */
static double mlp_row_rounded(const double *P, int width, int n_hidden, int act, const int32_t *fmts,
                              const double *scales, const double *in, double *h, double *z)
{
    const double *W = P, *b = P + (long)width * 15;
    for (int o = 0; o < width; ++o) {
        double s = b[o];
        for (int k = 0; k < 15; ++k) s += W[(long)o * 15 + k] * in[k];
        h[o] = act_f(s, act);
    }
    const double *p = b + width;
    for (int l = 0; l < n_hidden; ++l) {
        for (int k = 0; k < width; ++k) {
            if (fmts[l] == 1) h[k] = (double)orc_round_bf16((float)h[k]);
            if (fmts[l] == 2) h[k] = orc_round_e4m3(h[k] / scales[l]) * scales[l];
        }
        const double *Wl = p, *bl = p + (long)width * width;
        for (int o = 0; o < width; ++o) {
            double s = bl[o];
            for (int k = 0; k < width; ++k) s += Wl[(long)o * width + k] * h[k];
            z[o] = act_f(s, act);
        }
        memcpy(h, z, sizeof(double) * (size_t)width);
        p = bl + width;
    }
    double f = p[width];
    for (int k = 0; k < width; ++k) f += p[k] * h[k];
    return f;
}

/* Every (motion, point) pair with the input of each hidden layer rounded to
 * the activation format of the network's precision, as the tensor-core path
 * stores it (fmt 1: nearest-even bfloat16; fmt 2: FP8 E4M3 as
 * e4m3(h / s_l) * s_l with the per-layer scale s_l), everything else in
 * double.  fmt 0 is the plain network.  out[m][i] for all pairs, like
 * orc_mlp_pairs. */
void orc_mlp_pairs_rounded(const double *P, int width, int n_hidden, int act, int fmt,
                           const double *scales, const double *q0, const double *q1, int M,
                           const double *pts, long n, double *out)
{
    int32_t fmts[n_hidden > 0 ? n_hidden : 1];
    for (int l = 0; l < n_hidden; ++l) fmts[l] = fmt;
    #pragma omp parallel
    {
        double h[width], z[width];
        #pragma omp for schedule(static) collapse(2)
        for (int m = 0; m < M; ++m)
            for (long i = 0; i < n; ++i) {
                double in[15];
                for (int c = 0; c < 3; ++c) in[c] = pts[3 * i + c];
                for (int c = 0; c < DOF; ++c) {
                    in[3 + c] = q0[m * DOF + c];
                    in[9 + c] = q1[m * DOF + c];
                }
                out[(long)m * n + i] = mlp_row_rounded(P, width, n_hidden, act, fmts, scales, in, h, z);
            }
    }
}

/* Given input rows (n x 15), the network with a separate activation format
 * per hidden layer (fmts[l], as above): separates the contribution of each
 * layer's rounding to the error of a precision. */
void orc_mlp_forward_rounded(const double *P, int width, int n_hidden, int act, const int32_t *fmts,
                             const double *scales, const double *inputs, long n, double *out)
{
    #pragma omp parallel
    {
        double h[width], z[width];
        #pragma omp for schedule(static)
        for (long i = 0; i < n; ++i)
            out[i] = mlp_row_rounded(P, width, n_hidden, act, fmts, scales, inputs + 15 * i, h, z);
    }
}

/* Mean L1 loss (1/n) sum |f - delta| and its gradient w.r.t. every parameter
 * (written into G, same layout as P).  Backpropagation of the plain MLP. */
double orc_mlp_loss_grad(const double *P, int width, int n_hidden, int act,
                         const double *inputs, const double *target, long n, double *G)
{
    const long np = orc_param_count(width, n_hidden);
    memset(G, 0, np * sizeof(double));
    double loss = 0.0;
    double z[(n_hidden + 1) * width], h[(n_hidden + 1) * width];
    double g[width], gp[width];
    for (long r = 0; r < n; ++r) {
        const double *in = inputs + 15 * r;
        const double f = mlp_row(P, width, n_hidden, act, in, z, h);
        const double diff = f - target[r];
        loss += fabs(diff);
        const double df = (diff > 0.0 ? 1.0 : (diff < 0.0 ? -1.0 : 0.0)) / (double)n;
        /* output layer */
        const long off_out = np - (width + 1);
        const double *Wo = P + off_out;
        const double *hl = h + (long)n_hidden * width;
        for (int i = 0; i < width; ++i) {
            G[off_out + i] += df * hl[i];
            g[i] = df * Wo[i] * act_df(z[(long)n_hidden * width + i], act);   /* dL/dz_L */
        }
        G[off_out + width] += df;
        /* hidden layers, from the top down */
        for (int l = n_hidden; l >= 1; --l) {
            const long off = (long)width * 15 + width + (long)(l - 1) * ((long)width * width + width);
            const double *Wl = P + off;
            const double *hp = h + (long)(l - 1) * width;
            for (int o = 0; o < width; ++o) {
                for (int i = 0; i < width; ++i) G[off + (long)o * width + i] += g[o] * hp[i];
                G[off + (long)width * width + o] += g[o];
            }
            for (int i = 0; i < width; ++i) {
                double s = 0.0;
                for (int o = 0; o < width; ++o) s += Wl[(long)o * width + i] * g[o];
                gp[i] = s * act_df(z[(long)(l - 1) * width + i], act);
            }
            memcpy(g, gp, sizeof g);
        }
        /* input layer */
        for (int o = 0; o < width; ++o) {
            for (int i = 0; i < 15; ++i) G[(long)o * 15 + i] += g[o] * in[i];
            G[(long)width * 15 + o] += g[o];
        }
    }
    return loss / (double)n;
}

/* orc_mlp_loss_grad with the values rounded to nearest-even bfloat16 where a
 * BF16 training step stores them, everything else in double: the hidden
 * weights inside the hidden layers' products, every layer's pre-activation
 * Z_l and activation H_l = bf16(act(z_l)) (act of the unrounded z_l; layer 1
 * included), the output layer's gradient G_L = bf16(df w_out act'(Z_L)) and
 * every lower layer's G_{l-1} = bf16((W_l^T G_l) act'(Z_{l-1})), act' taken
 * at the rounded Z.  The input layer, the output layer's weights and every
 * bias stay unrounded.  It separates the arithmetic of a BF16 trainer from
 * the rounding that the format itself brings. */
static double rbf(double v) { return (double)orc_round_bf16((float)v); }

double orc_mlp_loss_grad_bf16(const double *P, int width, int n_hidden, int act,
                              const double *inputs, const double *target, long n, double *G)
{
    const long np = orc_param_count(width, n_hidden);
    memset(G, 0, np * sizeof(double));
    const long hs = (long)width * width + width;           /* one hidden layer: W then b */
    const long off_h = (long)width * 15 + width;
    const long off_out = np - (width + 1);
    double *Wr = malloc(sizeof(double) * (size_t)(n_hidden > 0 ? n_hidden : 1) * width * width);
    for (int l = 0; l < n_hidden; ++l)
        for (long i = 0; i < (long)width * width; ++i) Wr[l * (long)width * width + i] = rbf(P[off_h + l * hs + i]);
    double loss = 0.0;
    double *D = malloc(sizeof(double) * (size_t)(n_hidden + 1) * width);
    double *H = malloc(sizeof(double) * (size_t)(n_hidden + 1) * width);
    double *g = malloc(sizeof(double) * (size_t)width), *gp = malloc(sizeof(double) * (size_t)width);
    for (long r = 0; r < n; ++r) {
        const double *in = inputs + 15 * r;
        for (int o = 0; o < width; ++o) {
            double s = P[(long)width * 15 + o];
            for (int k = 0; k < 15; ++k) s += P[(long)o * 15 + k] * in[k];
            D[o] = rbf(act_df(s, act));
            H[o] = rbf(act_f(s, act));
        }
        for (int l = 1; l <= n_hidden; ++l) {
            const double *Wl = Wr + (long)(l - 1) * width * width, *bl = P + off_h + (l - 1) * hs + (long)width * width;
            for (int o = 0; o < width; ++o) {
                double s = 0.0;
                for (int i = 0; i < width; ++i) s += Wl[(long)o * width + i] * H[(long)(l - 1) * width + i];
                s += bl[o];
                D[(long)l * width + o] = rbf(act_df(s, act));
                H[(long)l * width + o] = rbf(act_f(s, act));
            }
        }
        const double *Wo = P + off_out, *hl = H + (long)n_hidden * width, *dl = D + (long)n_hidden * width;
        double f = Wo[width];
        for (int i = 0; i < width; ++i) f += Wo[i] * hl[i];
        const double diff = f - target[r];
        loss += fabs(diff);
        const double df = (diff > 0.0 ? 1.0 : (diff < 0.0 ? -1.0 : 0.0)) / (double)n;
        for (int i = 0; i < width; ++i) {
            G[off_out + i] += df * hl[i];
            g[i] = rbf(df * Wo[i] * dl[i]);
        }
        G[off_out + width] += df;
        for (int l = n_hidden; l >= 1; --l) {
            const long off = off_h + (l - 1) * hs;
            const double *Wl = Wr + (long)(l - 1) * width * width;
            const double *hp = H + (long)(l - 1) * width, *dp = D + (long)(l - 1) * width;
            for (int o = 0; o < width; ++o) {
                for (int i = 0; i < width; ++i) G[off + (long)o * width + i] += g[o] * hp[i];
                G[off + (long)width * width + o] += g[o];
            }
            for (int i = 0; i < width; ++i) {
                double s = 0.0;
                for (int o = 0; o < width; ++o) s += Wl[(long)o * width + i] * g[o];
                gp[i] = rbf(s * dp[i]);
            }
            memcpy(g, gp, sizeof(double) * (size_t)width);
        }
        for (int o = 0; o < width; ++o) {
            for (int k = 0; k < 15; ++k) G[(long)o * 15 + k] += g[o] * in[k];
            G[(long)width * 15 + o] += g[o];
        }
    }
    free(Wr); free(D); free(H); free(g); free(gp);
    return loss / (double)n;
}

/* One Adam step (Kingma and Ba) with bias correction, t = step count >= 1:
 * m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 * p -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps). */
void orc_adam_step(double *P, const double *G, double *Mo, double *Vo, long n, long t,
                   double lr, double b1, double b2, double eps)
{
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (long i = 0; i < n; ++i) {
        Mo[i] = b1 * Mo[i] + (1.0 - b1) * G[i];
        Vo[i] = b2 * Vo[i] + (1.0 - b2) * G[i] * G[i];
        P[i] -= lr * (Mo[i] / c1) / (sqrt(Vo[i] / c2) + eps);
    }
}

/* ------------------------------------------------ combined check ---- */

/* The margin-gated check of Sec. IV-B for each motion m:
 *   f_i     = f_theta(x_i, q0_m, q1_m) for every point;
 *   dhat_m  = min_i f_i                                 (Eq. 6);
 *   flagged = { i : f_i <= gate }   (gate = eps + tau; ties are flagged);
 *   verdict = collision iff some flagged i has delta_N(x_i, m) <= eps;
 *   dmin_m  = min over flagged i of delta_N (+inf when none is flagged).
 * With strict != 0, a motion with no flagged collision has all of its points
 * checked exactly (a free verdict is always confirmed by the exact check, as
 * in Algorithm 1), and dmin then covers every point.
 * f (M x n) may be given (precomputed network outputs) or NULL. */
void orc_check_motions(const double *P, int width, int n_hidden, int act,
                       const double *dh, double tool_len, const double *radius,
                       const double *q0, const double *q1, int M, int N,
                       const double *pts, long n, double eps, double gate, int strict,
                       const double *f_in, int32_t *collision, double *dmin,
                       double *dhat, int64_t *n_flagged)
{
    double in[15];
    (void)in;
    for (int m = 0; m < M; ++m) {
        double A[(N + 1) * NCAPS * 3], B[(N + 1) * NCAPS * 3];
        motion_capsules(dh, tool_len, q0 + m * DOF, q1 + m * DOF, N, A, B);
        double fmin = INFINITY, best = INFINITY, best_all = INFINITY;
        long nf = 0;
        #pragma omp parallel reduction(min:fmin,best,best_all) reduction(+:nf)
        {
            double z[(n_hidden + 1) * width], h[(n_hidden + 1) * width], row[15];
            #pragma omp for schedule(static)
            for (long i = 0; i < n; ++i) {
                double f;
                if (f_in) {
                    f = f_in[(long)m * n + i];
                } else {
                    for (int c = 0; c < 3; ++c) row[c] = pts[3 * i + c];
                    for (int c = 0; c < DOF; ++c) {
                        row[3 + c] = q0[m * DOF + c];
                        row[9 + c] = q1[m * DOF + c];
                    }
                    f = mlp_row(P, width, n_hidden, act, row, z, h);
                }
                if (f < fmin) fmin = f;
                const int flag = f <= gate;
                if (flag || strict) {
                    double d = INFINITY;
                    for (int k = 0; k <= N; ++k) {
                        const double dk = robot_sdf_caps(pts + 3 * i, A + k * NCAPS * 3, B + k * NCAPS * 3, radius);
                        if (dk < d) d = dk;
                    }
                    if (flag) { ++nf; if (d < best) best = d; }
                    if (d < best_all) best_all = d;
                }
            }
        }
        int coll = best <= eps;
        double dm = best;
        if (strict && !coll) {
            coll = best_all <= eps;
            dm = best_all;
        }
        collision[m] = coll;
        dmin[m] = dm;
        dhat[m] = fmin;
        n_flagged[m] = nf;
    }
}

/* ------------------------------------------------------ quantisers ---- */

/* Round a float to the nearest bfloat16 (8-bit exponent, 7 stored mantissa
 * bits), ties to even, and return it as a float.  Finite inputs only. */
float orc_round_bf16(float v)
{
    uint32_t u;
    memcpy(&u, &v, 4);
    const uint32_t lower = u & 0xFFFFu;
    uint32_t upper = u >> 16;
    if (lower > 0x8000u || (lower == 0x8000u && (upper & 1u))) upper += 1u;
    u = upper << 16;
    float r;
    memcpy(&r, &u, 4);
    return r;
}

void orc_round_bf16_array(float *v, long n)
{
    for (long i = 0; i < n; ++i) v[i] = orc_round_bf16(v[i]);
}

/* Round to the nearest FP8 E4M3 value (OCP FP8: bias 7, 3 mantissa bits,
 * largest finite 448, smallest normal 2^-6, subnormal step 2^-9), ties to
 * even, saturating to +-448.  The value is returned as a double. */
double orc_round_e4m3(double v)
{
    const double av = fabs(v);
    if (av == 0.0) return v;
    int e;
    frexp(av, &e);                 /* av = f * 2^e, f in [0.5, 1) -> exponent e-1 */
    int ex = e - 1;
    if (ex < -6) ex = -6;          /* subnormal range shares the 2^-6 quantum */
    const double quantum = ldexp(1.0, ex - 3);
    double r = nearbyint(av / quantum) * quantum;   /* default mode: ties to even */
    if (r > 448.0) r = 448.0;
    return v < 0.0 ? -r : r;
}

/* Per-tensor FP8 scale of a weight matrix: s = max|w| / 448 in float (a zero
 * matrix gets s = 1).  q holds the dequantised values e4m3(w / s) * s. */
float orc_quantize_e4m3(const float *w, long n, float *q)
{
    float mx = 0.0f;
    for (long i = 0; i < n; ++i) {
        const float a = fabsf(w[i]);
        if (a > mx) mx = a;
    }
    const float s = mx > 0.0f ? mx / 448.0f : 1.0f;
    for (long i = 0; i < n; ++i) {
        const float t = w[i] / s;
        q[i] = (float)(orc_round_e4m3((double)t) * (double)s);
    }
    return s;
}

/* -------------------------------------------------- training sampler ---- */

/* SplitMix64 (Steele, Lea, Flood 2014): value i of stream (seed, stream) is
 * fin(base + (i + 1) * gamma) mod 2^64, base = fin(seed*gamma ^ stream*c). */
static uint64_t sm_fin(uint64_t z)
{
    z ^= z >> 30; z *= 0xBF58476D1CE4E5B9ull;
    z ^= z >> 27; z *= 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

double orc_splitmix64_u01(uint64_t seed, uint64_t stream, uint64_t i)
{
    const uint64_t gamma = 0x9E3779B97F4A7C15ull;
    const uint64_t base = sm_fin((seed * gamma) ^ (stream * 0xD1B54A32D192ED03ull));
    const uint64_t u = sm_fin(base + (i + 1) * gamma);
    return (double)(u >> 11) * 0x1.0p-53;
}

/* Training points of one motion m (samples_per_motion of them), the recipe of
 * the data generator (Sec. IV-C adapted to capsules): draws u_0..u_6 of the
 * SplitMix64 stream (seed, m) at counters 8j..8j+6; with u_0 < 0.7 a point
 * near capsule c = floor(7 u_2) of sample k = floor((N+1) u_1):
 * a + u_3 (b - a) + (r_c + off) d, with d = (sqrt(1 - z^2) cos phi,
 * sqrt(1 - z^2) sin phi, z), z = 2 u_4 - 1, phi = 2 pi u_5,
 * off = -0.1 + 0.2 u_6; otherwise uniform in the box [lo, hi] from u_1..u_3
 * (lo + (hi - lo) u per axis).  Each point gets its exact sampled
 * swept-volume distance.
 * out is (spm, 4): x, y, z, delta. */
void orc_training_points_region(const double *dh, double tool_len, const double *radius, const double *q0,
                                const double *q1, int N, uint64_t seed, int m, int spm, const double *lo,
                                const double *hi, double *out)
{
    double A[(N + 1) * NCAPS * 3], Bx[(N + 1) * NCAPS * 3];
    motion_capsules(dh, tool_len, q0, q1, N, A, Bx);
    #pragma omp parallel for schedule(static)
    for (int j = 0; j < spm; ++j) {
        const uint64_t c = (uint64_t)j * 8u;
        double u[7];
        for (int i = 0; i < 7; ++i) u[i] = orc_splitmix64_u01(seed, (uint64_t)m, c + (uint64_t)i);
        double p[3];
        if (u[0] < 0.7) {
            int k = (int)(u[1] * (N + 1));
            if (k > N) k = N;
            int cj = (int)(u[2] * NCAPS);
            if (cj > NCAPS - 1) cj = NCAPS - 1;
            const double *a = A + (k * NCAPS + cj) * 3, *b = Bx + (k * NCAPS + cj) * 3;
            const double z = 2.0 * u[4] - 1.0, phi = 2.0 * 3.141592653589793 * u[5];
            const double off = -0.1 + 0.2 * u[6];
            const double rxy = sqrt(fmax(0.0, 1.0 - z * z));
            const double d[3] = {rxy * cos(phi), rxy * sin(phi), z};
            for (int q = 0; q < 3; ++q) p[q] = a[q] + u[3] * (b[q] - a[q]) + (radius[cj] + off) * d[q];
        } else {
            for (int q = 0; q < 3; ++q) p[q] = lo[q] + (hi[q] - lo[q]) * u[1 + q];
        }
        double best = INFINITY;
        for (int k = 0; k <= N; ++k) {
            const double dd = robot_sdf_caps(p, A + k * NCAPS * 3, Bx + k * NCAPS * 3, radius);
            if (dd < best) best = dd;
        }
        for (int q = 0; q < 3; ++q) out[4 * j + q] = p[q];
        out[4 * j + 3] = best;
    }
}

/* The same with the uniform points in the default box [-0.75,0.75]^2 x [0,1.5]. */
void orc_training_points(const double *dh, double tool_len, const double *radius, const double *q0,
                         const double *q1, int N, uint64_t seed, int m, int spm, double *out)
{
    const double lo[3] = {-0.75, -0.75, 0.0}, hi[3] = {0.75, 0.75, 1.5};
    orc_training_points_region(dh, tool_len, radius, q0, q1, N, seed, m, spm, lo, hi, out);
}
