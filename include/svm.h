/*
 * svm.h -- C ABI of libsvm: GPU collision checking of joint-space motions
 * against a point cloud with a neural implicit swept-volume model and an
 * exact geometric verifier.
 *
 * Method: Joho, Schwinn, Safronov, "Neural Implicit Swept Volume Models for
 * Fast Collision Detection" (arXiv 2402.15281).
 *   - the network f(x, q0, q1) approximates the signed distance of a point x
 *     to the volume swept by the robot on the linear joint motion q0 -> q1
 *     (Sec. III, Eqs. 1-4; network of Sec. IV-A);
 *   - the minimum of the network over the cloud is the proxy d^(X, m) of
 *     Eq. 6, the exact minimum d(X, m) of Eq. 5 is the geometric check, and a
 *     motion is free iff d(X, m) > eps_S (Sec. IV-B, Algorithm 1).
 * The library fuses both: the network flags the pairs whose prediction is
 * under a gate g = margin + tau, and only those are checked exactly, so the
 * verdict of a motion is decided by the geometric check.
 *
 * Conventions for every entry point:
 *   - All calls return svm_status; no exception or abort crosses the ABI.
 *     svm_last_error() gives a text for the last failing call on a model.
 *   - Device pointers are CUDA global-memory addresses on the model's device.
 *     The caller owns them; the library never frees them.  Host pointers are
 *     read (or written) before the call returns.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is enqueued asynchronously on it; device results are
 *     valid after the stream is synchronised.
 *   - Points are float4 records (x, y, z, w) in metres, w ignored, 16-byte
 *     aligned.  Joint angles are radians, 6 per configuration, row-major.
 *   - A model is not thread safe: calls on one model must not overlap in
 *     host threads; calls on one model are serialised in stream order.
 *   - Profiling: the check, evaluation, labelling, search, plan-launch and
 *     training-epoch calls each push an NVTX range named after the call; a
 *     check call also names its phases (prologue, network, verify, finalize),
 *     so that `ncu --nvtx` can select kernels by call and phase.
 *   - The environment variable SVM_WORKSPACE_LIMIT (decimal bytes), when set,
 *     caps the device workspace a model allocates for its check, evaluation
 *     and labelling calls: a call that needs more returns SVM_E_OOM before it
 *     allocates anything (this is how the out-of-memory path is tested).
 */
#ifndef SVM_H
#define SVM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SVM_OK = 0,
    SVM_E_INVALID = 1,      /* bad argument: size, pointer, NaN, layout        */
    SVM_E_CUDA = 2,         /* a CUDA runtime or launch error                   */
    SVM_E_OOM = 3,          /* device workspace could not be allocated          */
    SVM_E_TIMEOUT = 4,      /* a bounded device wait expired (sticky per model) */
    SVM_E_WEIGHTS = 5,      /* malformed weight blob or no weights loaded       */
    SVM_E_UNSUPPORTED = 6   /* valid but not supported on this device/config    */
} svm_status;

typedef enum { SVM_FP32 = 0, SVM_BF16 = 1, SVM_FP8_E4M3 = 2 } svm_precision;
typedef enum { SVM_RELU = 0, SVM_SILU = 1 } svm_act;

/* Robot and network description; copied by svm_create_model.
 * Robot: standard Denavit-Hartenberg chain of 6 revolute joints,
 *   T_j = T_{j-1} Rz(q_j + theta_j) Tz(d_j) Tx(a_j) Rx(alpha_j), T_0 = I,
 * dh[j] = {d_j, a_j, alpha_j, theta_j}.  Its geometry is 7 capsules: capsule
 * j < 6 joins the origins of frames j and j+1, capsule 6 runs tool_len along
 * the z axis of frame 6; radius[j] is capsule j's radius.
 * Network (arch SVM_ARCH_MLP): input [x, y, z, q0_1..q0_6, q1_1..q1_6] ->
 * width (act) -> n_hidden x (width -> width, act) -> 1.  The BF16 and FP8
 * tensor-core path needs width 256 and 1 <= n_hidden <= 16; the FP32 path
 * takes width 64, 128, 256, 512 or 1024 and 0 <= n_hidden <= 16.
 * Network (arch SVM_ARCH_BLOCKS, the block architecture of Sec. IV-A):
 * an initial linear layer 15 -> width, n_hidden blocks (linear -> ReLU ->
 * BatchNorm at inference, plus the block input; from the second block on the
 * linear layer also reads the network input, the jump connection), and a
 * final layer [h; input] -> 1.  FP32 path only, ReLU, width 64..1024,
 * 1 <= n_hidden <= 16; BatchNorm is folded into a per-channel scale and
 * shift at load. */
typedef struct {
    double dh[6][4];
    double radius[7];
    double tool_len;
    int32_t width;
    int32_t n_hidden;   /* hidden layers (SVM_ARCH_MLP) or blocks (SVM_ARCH_BLOCKS) */
    int32_t act;        /* svm_act       */
    int32_t prec;       /* svm_precision */
    int32_t arch;       /* SVM_ARCH_MLP (0) or SVM_ARCH_BLOCKS (1) */
} svm_model_desc;

#define SVM_ARCH_MLP    0
#define SVM_ARCH_BLOCKS 1

/* Per-motion (or per-path) result, 32 bytes, written to device memory. */
typedef struct {
    uint8_t collision;      /* 1 iff some checked point has distance <= margin */
    uint8_t early_exit;     /* 1 if checking stopped at the first collision     */
    uint16_t status;        /* 0 = valid; 1 = a bounded device wait expired during
                               the call and this record is not valid; 2 = valid
                               except that a checked pair of this motion (or
                               path) whose FP32 distance lay within 4e-6 m of
                               the margin found the call's list of such pairs
                               full (16 384) and was decided in FP32, so its
                               verdict and d_min may differ from the FP64
                               decision                                        */
    float d_min;            /* minimum exact distance over the checked points;
                               +inf if none was checked; on early exit the first
                               value found <= margin                            */
    float dhat_min;         /* minimum network prediction over all points (Eq. 6);
                               +inf when the network was not run                */
    uint32_t n_flagged;     /* points whose prediction was <= the gate          */
    uint32_t n_verified;    /* points checked exactly                           */
    int32_t witness_point;  /* index of a colliding point, -1 if none           */
    int32_t witness_step;   /* a sample k in [0, steps] where it collides, -1 if
                               none; for paths: segment * (steps + 1) + k       */
    uint32_t n_ambiguous;   /* checked points whose FP32 distance lies within
                               4e-6 m of the margin; their verdict and distance
                               are recomputed in FP64 (the first 16384 such
                               pairs of a call; beyond that the FP32 decision
                               stands and the record carries status 2)        */
} svm_result;

typedef struct svm_model svm_model;

/* Flags of the check calls. */
#define SVM_STRICT        1u  /* a motion without a flagged collision has every
                                 point checked exactly: "free" is then always
                                 confirmed by the geometric check (Algorithm 1)  */
#define SVM_NO_EARLY_EXIT 2u  /* check every flagged point (exact d_min)         */
#define SVM_VERIFY_ALL    4u  /* skip the network; check every pair exactly (the
                                 geometric check alone, GCC_0 of Sec. V-B)       */
#define SVM_PATHS3        8u  /* motions 3p, 3p+1, 3p+2 are the segments of path
                                 p; one result per path (collision = OR), and a
                                 path stops at its first colliding segment      */
#define SVM_PATHS2       32u  /* as SVM_PATHS3 with paths of two segments
                                 (motions 2p, 2p+1); n_motions % 2 == 0        */
#define SVM_PREDICT_ONLY 16u  /* run the network only: dhat_min (Eq. 6) per
                                 motion, no exact check (collision = 0, d_min =
                                 +inf); not with SVM_VERIFY_ALL or SVM_STRICT;
                                 svm_check_motions / svm_check_batch only       */

const char* svm_status_string(svm_status s);
const char* svm_last_error(const svm_model* m);

/* Create a model on CUDA device `device`.  Checks the description (finite
 * DH values, radii >= 0, width/n_hidden/prec supported on this device).
 * *out receives the handle; free it with svm_destroy_model. */
svm_status svm_create_model(const svm_model_desc* desc, int device, svm_model** out);
svm_status svm_destroy_model(svm_model* m);

/* Load network weights from a little-endian blob:
 *   char magic[4] = "SVMW"; uint32 version = 1; uint32 n_layers;
 *   uint32 in_dim = 15; uint32 width; uint32 act; float tau;
 *   then for each layer: uint32 out, uint32 in, float W[out][in] (row-major),
 *   float b[out].
 * Layers must be 15 -> width, n_hidden x (width -> width), width -> 1 as in
 * the description.  The weights are rounded to the model precision on the
 * device: BF16 rounds every weight to nearest-even bfloat16; FP8 rounds the
 * hidden weights to E4M3 (nearest-even, saturating) with the per-layer scale
 * s = max|W| / 448 (float) and the other layers to BF16.  Biases stay FP32.
 * tau sets the gate offset (see svm_set_gate).  Returns SVM_E_WEIGHTS on a
 * malformed blob.
 * SVM_ARCH_BLOCKS models take version 2:
 *   char magic[4] = "SVMW"; uint32 version = 2; uint32 n_blocks;
 *   uint32 in_dim = 15; uint32 width; uint32 act = 0; float tau; float bn_eps;
 *   initial layer: uint32 width, uint32 15, float W[width][15], float b[width];
 *   block l = 1..n_blocks: uint32 width, uint32 in (width for l = 1, width + 15
 *   after: [h; x, q0, q1]), float W[width][in], b[width], gamma[width],
 *   beta[width], running_mean[width], running_var[width];
 *   final layer: uint32 1, uint32 width + 15, float W[width + 15], float b. */
svm_status svm_load_weights(svm_model* m, const void* blob, size_t bytes);

/* Copy the weights as the model uses them (after rounding, dequantised to
 * float) into host memory, in the blob's layer order (W then b per layer).
 * `count` is the capacity of `out` in floats; the required count is written
 * to *needed (may be NULL). */
svm_status svm_export_weights(const svm_model* m, float* out, size_t count, size_t* needed);

/* Test hook for the failure path of the bounded device waits: the next
 * n_calls check calls of this tensor-core model run with CTA 0 withholding
 * its first layer-0 hand-over, so that its MMA warp's wait expires after
 * 2 s; every role of that CTA leaves its loop, waits (bounded) for its own
 * operations in flight and frees its TMEM, the other CTAs finish, and every
 * record of the call carries status 1.  Later calls are unaffected.  The
 * call itself returns SVM_OK (the failure is reported in the records).
 * SVM_E_UNSUPPORTED for FP32 models (no device waits). */
svm_status svm_test_expire_wait(svm_model* m, int32_t n_calls);

/* Test hook for the tie-list overflow path: later calls of this model keep
 * at most `cap` pairs at the margin (1..16384) for the FP64 decision, so that
 * a small case overflows the list; 0 restores the full list.  Records of
 * motions with a pair beyond the cap carry status 2. */
svm_status svm_test_set_tie_cap(svm_model* m, int32_t cap);

/* Gate offset tau >= 0 (metres): a pair is checked exactly iff its network
 * prediction f <= margin + tau.  tau = +inf checks every pair. */
svm_status svm_set_gate(svm_model* m, float tau);

/* FP8 only: per-hidden-layer activation scales (n_hidden values > 0); the
 * input of hidden layer l is stored as e4m3(h / scale[l]). */
svm_status svm_set_act_scales(svm_model* m, const float* scales, int32_t n);

/* FP8 only: choose the activation scales from data.  The network is run in
 * FP32 on the model's rounded weights over every (motion, point) pair given
 * (host q0/q1, device points), recording the largest magnitude entering each
 * hidden layer; scale[l] = headroom * max[l] / 448 (headroom >= 1 keeps
 * unseen larger activations below the E4M3 saturation).  Sets the scales and
 * writes them to scales_out (n_hidden floats, may be NULL).  Synchronous;
 * allocates temporary device memory. */
svm_status svm_calibrate_act_scales(svm_model* m, const double* q0, const double* q1, int32_t n_motions,
                                    const float* points_dev, int64_t n_points, float headroom,
                                    float* scales_out);

/* Gate calibration: the margin widened by the measured error of the network
 * (Sec. IV-B gates the exact check with the network's prediction; here the
 * gate is g = margin + tau).  Over every (motion, point) pair given (host
 * q0/q1, n_motions x 6; device points), with f the network output in the
 * model's own precision and delta the exact sampled distance at `steps`
 * steps (the values svm_eval_pairs and svm_label_pairs would write):
 *   over = max (f - delta) over the pairs with delta <= margin + band
 *          (the pairs that can collide; margin + band rounded to float),
 *   tau  = max(0, safety * over), or 0 when no pair is that close.
 * Sets the model's gate to tau (svm_set_gate) and writes tau, over (-inf if
 * no pair qualifies) and the number of qualifying pairs to the host outputs
 * (each may be NULL).  The calibration motions should be separate from the
 * motions to be checked and drawn like them; the gate is an empirical bound,
 * not a guarantee (SVM_STRICT confirms free verdicts regardless).
 *   band >= 0, safety >= 1, margin >= 0, steps as in svm_check_motions;
 *   n_motions * n_points < 2^32.
 * The network outputs are formed in chunks of motions in a temporary buffer
 * of at most 2^26 floats (cudaMalloc, freed before return); delta is never
 * stored.  Synchronous on `stream`.  SVM_E_WEIGHTS without weights. */
svm_status svm_calibrate_gate(svm_model* m, const double* q0, const double* q1, int32_t n_motions,
                              const float* points_dev, int64_t n_points, float margin, int32_t steps, float band,
                              float safety, float* tau_out, float* overestimate_out, int64_t* n_near_out,
                              void* stream);

/* Check n_motions linear motions q0[m] -> q1[m] against one point cloud.
 *   q0, q1       host, n_motions x 6 doubles, finite.
 *   points_dev   device, n_points float4 records.
 *   margin       eps_S >= 0 in metres: collision iff distance <= margin.
 *   steps        N >= 1: the motion is sampled at q_k = ((N-k) q0 + k q1) / N,
 *                k = 0..N, and each sample is checked exactly.
 *   results_dev  device, n_motions svm_result records (n_motions / 3 with
 *                SVM_PATHS3, which needs n_motions % 3 == 0; n_motions / 2
 *                with SVM_PATHS2).
 * The model's workspace grows on demand (cudaMalloc; SVM_E_OOM on failure). */
svm_status svm_check_motions(svm_model* m, const double* q0, const double* q1,
                             int32_t n_motions, const float* points_dev, int64_t n_points,
                             float margin, int32_t steps, uint32_t flags,
                             svm_result* results_dev, void* stream);

/* Batched form over several scenes in one launch sequence.  Scene s owns the
 * points [scene_offsets[s], scene_offsets[s+1]) of points_dev; motion m is
 * checked against scene motion_scene[m].  scene_offsets (n_scenes + 1 int64)
 * and motion_scene (n_motions int32) are host arrays. */
svm_status svm_check_batch(svm_model* m, const double* q0, const double* q1,
                           int32_t n_motions, const int32_t* motion_scene,
                           const float* points_dev, const int64_t* scene_offsets,
                           int32_t n_scenes, float margin, int32_t steps, uint32_t flags,
                           svm_result* results_dev, void* stream);

/* ------------------------------------------------------------ motion search
 * Algorithm 1 (Sec. IV-B): find a collision-free motion among n_motions
 * candidates with the network as a proxy.  d_hat(X, m) = min over the cloud of
 * f(x, m) (Eq. 6) is computed for every motion in one network launch.  First
 * loop: the motions with d_hat > margin, in the given order, are checked
 * exactly (the geometric check of every point, free iff every distance >
 * margin, Eq. 5); the first free one is returned.  Otherwise, second loop: the
 * remaining motions sorted by decreasing d_hat (ties in the given order) are
 * checked exactly until one is free.  With SVM_SEARCH_GCC0 the network is not
 * used and every motion is checked exactly in the given order (GCC_0 of
 * Sec. V-B).
 *   wave    exact checks run `wave` candidates per launch (1 reproduces the
 *           sequential algorithm; more trades extra checks for fewer round
 *           trips); the result is the same for every wave.
 * With SVM_SEARCH_SORTED only the second loop runs: every candidate is
 * checked in decreasing d_hat (the bin-picking use of Sec. V-C, where the
 * network predicts no free motion).  With SVM_SEARCH_PATHS2 / _PATHS3 the
 * candidates are paths of 2 / 3 consecutive segments (n_motions a multiple
 * of that): a path's d_hat is the minimum over its segments and its exact
 * check that of SVM_PATHS2 / SVM_PATHS3 (free iff every segment is free);
 * `motion` then indexes paths.
 * Synchronous on `stream` (it reads results back to decide); q0/q1 host,
 * points device; out is a host struct.  Allocates its result buffers on the
 * first call (cudaMalloc / cudaMallocHost), then reuses them. */
#define SVM_SEARCH_GCC0   1u
#define SVM_SEARCH_SORTED 2u
#define SVM_SEARCH_PATHS2 4u
#define SVM_SEARCH_PATHS3 8u

typedef struct {
    int32_t motion;       /* index of the free motion found, -1 if none          */
    int32_t loop;         /* 1 or 2: the loop that found it; 0 if none            */
    float delta;          /* its exact distance d(X, m) (min over the cloud), m   */
    float delta_hat;      /* its d_hat(X, m); +inf under SVM_SEARCH_GCC0          */
    int32_t n_exact;      /* exact checks the sequential algorithm makes          */
    int32_t n_exact_run;  /* exact checks run (n_exact rounded up to whole waves) */
    int32_t n_nn;         /* segments evaluated by the network launch (n_motions) */
    int32_t n_nn_seq;     /* network evaluations (segments) the sequential first
                             loop makes: up to the returned candidate, all if
                             the second loop runs                               */
} svm_search_result;

svm_status svm_search_free_motion(svm_model* m, const double* q0, const double* q1, int32_t n_motions,
                                  const float* points_dev, int64_t n_points, float margin, int32_t steps,
                                  int32_t wave, uint32_t flags, svm_search_result* out, void* stream);

/* ------------------------------------------------------------ prepared batches
 * A plan holds a fixed batch (motions, their scenes, margin, steps, flags)
 * validated and uploaded once, with its own workspace (cudaMalloc at
 * creation).  svm_plan_launch then only enqueues the kernels of one check
 * (no host synchronisation, no allocation): it may be captured in a CUDA
 * graph.  Results as in svm_check_batch; the model must outlive the plan.
 * Weights or gate changed after creation apply to later launches, except
 * that an instantiated graph keeps the gate it was captured with. */
typedef struct svm_plan svm_plan;
svm_status svm_plan_create(svm_model* m, const double* q0, const double* q1, int32_t n_motions,
                           const int32_t* motion_scene, const int64_t* scene_offsets, int32_t n_scenes,
                           float margin, int32_t steps, uint32_t flags, svm_plan** out);
/* Waits for the device, then frees the plan's workspace and graph. */
svm_status svm_plan_destroy(svm_plan* p);
/* One check of the plan's batch on `stream`: points_dev holds the scenes'
 * clouds concatenated as described by scene_offsets at creation (float4,
 * 16-byte aligned, device); results_dev receives one record per motion (or
 * per path), device, caller-owned.  SVM_E_INVALID for null or misaligned
 * buffers; enqueue errors as SVM_E_CUDA. */
svm_status svm_plan_launch(svm_plan* p, const float* points_dev, svm_result* results_dev, void* stream);
/* Replay the plan as a CUDA graph on `stream` (a created stream, not the
 * default one).  The first call, and any call with other points or results
 * pointers, runs one plain launch and captures the graph for the next calls. */
svm_status svm_plan_graph_launch(svm_plan* p, const float* points_dev, svm_result* results_dev, void* stream);
/* Verifier launch shape: points per thread (1, 2 or 4: one shared-memory read
 * of a capsule serves that many points) and CTAs per SM (0 = all that fit). */
svm_status svm_plan_set_verify_shape(svm_plan* p, int32_t points_per_thread, int32_t ctas_per_sm);
/* Persistent grid of the tensor-core network kernel: ctas CTAs (1..number of
 * SMs; 0 = one per SM, the default).  No effect on FP32 models. */
svm_status svm_plan_set_network_grid(svm_plan* p, int32_t ctas);
/* Time the launch shapes on the plan's data (one warm-up and 3 timed
 * launches each, CUDA events, synchronous) and keep the fastest: first the
 * network kernel's grid (tensor-core models: all SMs, 15/16, 7/8, 3/4 and
 * 1/2 of them), then, at that grid, the verifier's 9 shapes.  Writes a JSON
 * report {"network_candidates": [...], "candidates": [...], "best": {...}}
 * of all timings and the choice to `report` (may be NULL); the choice can be
 * re-applied later with svm_plan_set_network_grid and
 * svm_plan_set_verify_shape. */
svm_status svm_plan_autotune(svm_plan* p, const float* points_dev, svm_result* results_dev, void* stream,
                             char* report, size_t capacity);

/* Network output for every (motion, point) pair: f_dev[m * n_points + i] =
 * f(x_i, q0_m, q1_m) in the model precision (device, n_motions x n_points
 * floats).  Same kernels as the check, with the output stored. */
svm_status svm_eval_pairs(svm_model* m, const double* q0, const double* q1, int32_t n_motions,
                          const float* points_dev, int64_t n_points, float* f_dev, void* stream);

/* Exact sampled swept-volume distance (the verifier without gate or early
 * exit) for every pair: delta_dev[m * n_points + i] = min over k = 0..steps
 * and the 7 capsules of (distance to the capsule axis - radius). */
svm_status svm_label_pairs(svm_model* m, const double* q0, const double* q1, int32_t n_motions,
                           const float* points_dev, int64_t n_points, int32_t steps,
                           float* delta_dev, void* stream);

/* Allocation-free variant of svm_check_motions, for callers that cannot
 * allocate device memory while they check motions: a real-time control loop
 * whose memory is fixed at start-up (an allocation there can stall, or fail
 * when the device is full), or a process whose device memory is owned by
 * another framework's allocator, which may already hold all of it.  The paper
 * has no counterpart; this is an interface of this library only.
 *   - Allocates nothing: no cudaMalloc, cudaFree, pinned host memory or
 *     allocating library call.  Its scratch is one fixed 32 MiB array in
 *     device memory that the library declares at file scope; every GPU that
 *     loads the library holds it until the process exits.
 *   - q0_dev, q1_dev are DEVICE (or managed) arrays, n_motions x 6 doubles,
 *     8-byte aligned, on the model's device (checked: SVM_E_INVALID
 *     otherwise); their values must be finite (not checked).  The other
 *     arguments and the results are as in svm_check_motions.
 *   - A call needs about 4 bytes per motion-point pair plus, per motion,
 *     (steps + 1) * 416 bytes (the FP32 capsule table and the FP64 kinematics
 *     kept for pairs at the margin) and about 1.3 KB, plus 256 KB for the
 *     list of pairs at the margin; a call needing more than the
 *     32 MiB is rejected with SVM_E_INVALID and a message naming the sizes
 *     (e.g. 64 motions x 100 000 points fit, 64 x 200 000 do not).
 *   - The first call on a device looks up the scratch array's device address
 *     (cudaGetSymbolAddress) and keeps it for the life of the process; make
 *     that first call before any stream capture.  A cudaDeviceReset (or any
 *     other teardown of the device's primary context) invalidates the kept
 *     address: do not call this entry point on that device afterwards.
 *   - Every call, from every model on that device, shares the one array and
 *     finds the previous call's contents in it; the call re-initialises what
 *     it needs.  Calls whose kernels overlap on the GPU (different streams
 *     without ordering) race on the array and give wrong results. */
svm_status svm_check_motions_noalloc(svm_model* m, const double* q0_dev, const double* q1_dev,
                                     int32_t n_motions, const float* points_dev, int64_t n_points,
                                     float margin, int32_t steps, uint32_t flags,
                                     svm_result* results_dev, void* stream);

/* ---------------------------------------------------------------- training
 * The network is trained on the GPU on tuples (x, q0, q1, delta) (Sec. IV-C)
 * whose labels come from the exact geometric check, with mean absolute error
 * as the loss (the paper reports MAE) and Adam (betas 0.9 / 0.999, eps 1e-8,
 * Sec. V).  Hidden layers run as BF16 tensor-core GEMMs with FP32
 * accumulation and FP32 master weights; layer 1 and the output layer in FP32.
 * A trainer owns its parameters, Adam moments, activations for one batch and
 * its data; calls are synchronous (they return after the GPU work). */
typedef struct svm_trainer svm_trainer;

/* width 256 or 512, n_hidden 1..16, act ReLU or SiLU; batch a multiple of
 * 256 (>= 256).  Parameters start at zero: load initial weights with
 * svm_train_set_weights.  Needs a GPU of compute capability 10.3. */
svm_status svm_train_create(const svm_model_desc* desc, int device, int32_t batch, svm_trainer** out);
/* Waits for the device, then frees everything the trainer owns. */
svm_status svm_train_destroy(svm_trainer* t);
/* Text of the last failing call on the trainer. */
const char* svm_train_last_error(const svm_trainer* t);
/* Number of parameters in blob order (weights and biases of every layer). */
int64_t svm_train_param_count(const svm_trainer* t);

/* Weights in the blob format of svm_load_weights (tau ignored).  Setting
 * weights resets the Adam moments and the step count. */
svm_status svm_train_set_weights(svm_trainer* t, const void* blob, size_t bytes);
/* The current FP32 master weights as a blob (tau = +inf): *needed receives
 * its size; with blob = NULL only the size is returned; SVM_E_INVALID if
 * capacity is smaller than that.  Synchronous. */
svm_status svm_train_get_weights(svm_trainer* t, void* blob, size_t capacity, size_t* needed);

/* The box of the uniformly drawn training points for later svm_train_make_data
 * calls (lo, hi: 3 doubles each, lo < hi): cover the volume where the
 * checked points will lie. */
svm_status svm_train_set_box(svm_trainer* t, const double* lo, const double* hi);

/* Generate n_motions * samples_per_motion labelled samples on the GPU for
 * the host motions q0, q1 (n_motions x 6): for motion m and local index j the
 * SplitMix64 stream (seed, m) gives draws u_0..u_6 at counters 8j..8j+6;
 * with u_0 < 0.7 the point is near capsule floor(u_2 * 7) at sample
 * floor(u_1 * (steps + 1)): a + u_3 e + (r + off) d with d the unit vector of
 * (z = 2 u_4 - 1, phi = 2 pi u_5) and off = -0.1 + 0.2 u_6; otherwise it is
 * uniform in the sampling box (default [-0.75,0.75]^2 x [0,1.5]; coordinate
 * q is lo_q + (hi_q - lo_q) u_{1+q}).  The label is the exact
 * sampled swept-volume distance with `steps` steps.  Sample s = m *
 * samples_per_motion + j. */
svm_status svm_train_make_data(svm_trainer* t, const double* q0, const double* q1, int32_t n_motions,
                               int32_t samples_per_motion, int32_t steps, uint64_t seed);
/* Explicit samples: x4 (n x 4 floats: x, y, z, delta) and motion indices. */
svm_status svm_train_set_samples(svm_trainer* t, const double* q0, const double* q1, int32_t n_motions,
                                 const float* x4, const int32_t* motion, int64_t n);
/* Copy the first n samples to the host (either output may be NULL):
 * x4_out n x 4 floats (x, y, z, delta), motion_out n motion indices;
 * SVM_E_INVALID if n exceeds the samples held.  Synchronous. */
svm_status svm_train_copy_samples(svm_trainer* t, float* x4_out, int32_t* motion_out, int64_t n);

/* Loss and gradient (blob order, param_count floats, host) of the batch of
 * samples [sample_begin, sample_begin + batch); no update. */
svm_status svm_train_gradient(svm_trainer* t, int64_t sample_begin, float* grad_out, float* loss_out);
/* One Adam step with the gradient held by the trainer. */
svm_status svm_train_adam(svm_trainer* t, float lr);
/* One epoch over the samples [begin, end): floor((end-begin)/batch) batches,
 * batch i holding the samples begin + o_i + r * n_batches (r < batch) with a
 * random permutation o of the batch offsets drawn from shuffle_seed. */
svm_status svm_train_epoch(svm_trainer* t, int64_t sample_begin, int64_t sample_end, float lr,
                           uint64_t shuffle_seed, float* mean_loss);
/* Mean absolute error over the whole batches of [begin, end). */
svm_status svm_train_evaluate(svm_trainer* t, int64_t sample_begin, int64_t sample_end, float* mae);
/* Checkpoint: parameters, Adam moments (param_count floats each) and step. */
svm_status svm_train_state(svm_trainer* t, float* params, float* m1, float* m2, int64_t* step, int64_t n);
/* The inverse of svm_train_state (n must equal svm_train_param_count); a
 * restored trainer continues bit for bit as the one the state was taken
 * from. */
svm_status svm_train_restore(svm_trainer* t, const float* params, const float* m1, const float* m2, int64_t step,
                             int64_t n);

/* Phase timing.  With profiling on, every check call records CUDA events on
 * its stream between its phases; svm_profile_read waits for the last call to
 * finish and writes n <= 4 durations in milliseconds: ms[0] the per-call
 * copy + prologue (FK, per-motion bias), ms[1] the network kernel (gate and
 * compaction included), ms[2] the verifier (both passes in strict mode),
 * ms[3] the finalize kernel.  Not part of the computation; off by default. */
svm_status svm_profile_enable(svm_model* m, int on);
svm_status svm_profile_read(svm_model* m, float* ms, int32_t n);

#ifdef __cplusplus
}
#endif

#endif /* SVM_H */
