// plan.cu -- prepared batches (svm_plan_*): the arrays of a fixed batch of
// motions over one or more scenes are validated and uploaded once, with the
// plan's own workspace; a launch then only enqueues the kernels of a check
// call (no host synchronisation, no allocation), so it can be captured in a
// CUDA graph and replayed.  An autotuner times the launch shapes on the
// plan's own data and keeps the fastest: the persistent grid of the
// tensor-core network kernel (CTAs, one per SM at most), then the verifier's
// points per thread and CTAs per SM.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "svm_model.h"

using namespace svm;

struct svm_plan {
    svm_model* m = nullptr;
    int M = 0, N = 0, S = 0;
    uint32_t flags = 0;
    float margin = 0.0f;
    int bm = 0, n_tiles = 0;
    long long P_total = 0;
    void* ws = nullptr;
    size_t o_q0 = 0, o_q1 = 0, o_pbeg = 0, o_pend = 0, o_toff = 0, o_poff = 0;
    size_t o_caps = 0, o_fk64 = 0, o_cbias = 0, o_st = 0, o_idx = 0, o_chunk = 0, o_err = 0, o_tie = 0, total = 0;
    VerifyConfig vcfg{};
    int net_grid = 0;                 // CTAs of the tensor-core network kernel (0 = one per SM)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const void* g_points = nullptr;
    void* g_results = nullptr;
};

namespace {

size_t al256(size_t x) { return (x + 255) & ~size_t(255); }

svm_status pfail(svm_model* m, svm_status s, const std::string& msg)
{
    if (m) m->last_error = msg;
    return s;
}

struct Guard {
    int prev = -1;
    explicit Guard(int d) { if (cudaGetDevice(&prev) != cudaSuccess) prev = -1; if (prev != d) cudaSetDevice(d); }
    ~Guard() { int c = -1; if (prev >= 0 && cudaGetDevice(&c) == cudaSuccess && c != prev) cudaSetDevice(prev); }
};

void drop_graph(svm_plan* p)
{
    if (p->exec) cudaGraphExecDestroy(p->exec);
    if (p->graph) cudaGraphDestroy(p->graph);
    p->exec = nullptr;
    p->graph = nullptr;
    p->g_points = nullptr;
    p->g_results = nullptr;
}

CallArgs plan_args(svm_plan* p, const float* points)
{
    svm_model* m = p->m;
    char* ws = static_cast<char*>(p->ws);
    CallArgs a{};
    a.M = p->M;
    a.N = p->N;
    a.W = m->desc.width;
    a.L = m->desc.n_hidden;
    a.act = m->desc.act;
    a.arch = m->desc.arch;
    a.rp = m->rp;
    a.cb_stride = cbias_stride(m->desc);
    a.flags = p->flags;
    a.margin = p->margin;
    a.gate = p->margin + m->tau;
    a.q0 = reinterpret_cast<const double*>(ws + p->o_q0);
    a.q1 = reinterpret_cast<const double*>(ws + p->o_q1);
    a.pbeg = reinterpret_cast<const long long*>(ws + p->o_pbeg);
    a.pend = reinterpret_cast<const long long*>(ws + p->o_pend);
    a.tile_off = reinterpret_cast<const int*>(ws + p->o_toff);
    a.pair_off = reinterpret_cast<const long long*>(ws + p->o_poff);
    a.points = reinterpret_cast<const float4*>(points);
    a.caps = reinterpret_cast<Capsule*>(ws + p->o_caps);
    a.fk64 = reinterpret_cast<double*>(ws + p->o_fk64);
    a.cbias = (p->flags & SVM_VERIFY_ALL) ? nullptr : reinterpret_cast<float*>(ws + p->o_cbias);
    a.st = reinterpret_cast<MotionState*>(ws + p->o_st);
    a.idx = reinterpret_cast<unsigned*>(ws + p->o_idx);
    a.chunk_off = reinterpret_cast<int*>(ws + p->o_chunk);
    a.f_out = nullptr;
    a.f_stride = 0;
    a.path_len = path_len_of(p->flags);
    a.dev_err = reinterpret_cast<unsigned int*>(ws + p->o_err);
    a.tie_count = reinterpret_cast<unsigned int*>(ws + p->o_tie);
    a.tie_list = reinterpret_cast<TiePair*>(ws + p->o_tie + 256);
    a.amax = nullptr;
    return a;
}

// Enqueue the kernels of one check of the plan's batch.
svm_status enqueue(svm_plan* p, const float* points, svm_result* results, cudaStream_t s)
{
    svm_model* m = p->m;
    CallArgs a = plan_args(p, points);
    cudaError_t e = cudaMemsetAsync(a.dev_err, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return pfail(m, SVM_E_CUDA, cudaGetErrorString(e));
    launch_prologue_fk(a, m->rp, m->dw, s);
    if (!(p->flags & SVM_VERIFY_ALL)) {
        if (m->desc.prec != SVM_FP32) {
            const int grid = p->net_grid > 0 && p->net_grid < m->n_sms ? p->net_grid : m->n_sms;
            if (tc_launch(m->tc, a, m->dw, p->n_tiles, nullptr, grid, s) != 0)
                return pfail(m, SVM_E_CUDA, "tensor-core launch failed");
        } else {
            launch_mlp_fp32(a, m->dw, p->n_tiles, p->bm, s);
        }
        launch_verify_cfg(a, 0, 0, s, m->n_sms, p->vcfg);
        if (p->flags & SVM_STRICT) launch_verify_cfg(a, 1, 1, s, m->n_sms, p->vcfg);
    } else {
        launch_verify_cfg(a, 1, 0, s, m->n_sms, p->vcfg);
    }
    launch_ties(a, s, m->n_sms);
    launch_finalize(a, results, s);
    e = cudaGetLastError();
    if (e != cudaSuccess) return pfail(m, SVM_E_CUDA, cudaGetErrorString(e));
    return SVM_OK;
}

}  // namespace

extern "C" {

svm_status svm_plan_create(svm_model* m, const double* q0, const double* q1, int32_t n_motions,
                           const int32_t* motion_scene, const int64_t* scene_offsets, int32_t n_scenes,
                           float margin, int32_t steps, uint32_t flags, svm_plan** out)
{
    if (!m || !out) return SVM_E_INVALID;
    *out = nullptr;
    const int M = n_motions;
    if (M < 1 || !q0 || !q1 || !motion_scene || !scene_offsets || n_scenes < 1)
        return pfail(m, SVM_E_INVALID, "plan needs motions, scenes and their offsets");
    if (!m->has_weights && !(flags & SVM_VERIFY_ALL)) return pfail(m, SVM_E_WEIGHTS, "no weights loaded");
    if (!(margin >= 0) || !std::isfinite(margin)) return pfail(m, SVM_E_INVALID, "margin must be finite and >= 0");
    if (steps < 1 || steps > kMaxSteps) return pfail(m, SVM_E_INVALID, "steps out of range");
    if (flags & ~(SVM_STRICT | SVM_NO_EARLY_EXIT | SVM_VERIFY_ALL | SVM_PATHS3 | SVM_PATHS2))
        return pfail(m, SVM_E_INVALID, "unknown flag");
    if ((flags & SVM_PATHS3) && (flags & SVM_PATHS2)) return pfail(m, SVM_E_INVALID, "SVM_PATHS2 with SVM_PATHS3");
    if (M % path_len_of(flags) != 0) return pfail(m, SVM_E_INVALID, "n_motions is not a multiple of the path length");
    if (scene_offsets[0] != 0) return pfail(m, SVM_E_INVALID, "scene_offsets[0] must be 0");
    for (int s = 0; s < n_scenes; ++s)
        if (scene_offsets[s + 1] < scene_offsets[s]) return pfail(m, SVM_E_INVALID, "scene offsets decrease");
    if (scene_offsets[n_scenes] > (int64_t)0xffffffffLL) return pfail(m, SVM_E_INVALID, "too many points");
    for (long long i = 0; i < (long long)M * 6; ++i)
        if (!std::isfinite(q0[i]) || !std::isfinite(q1[i])) return pfail(m, SVM_E_INVALID, "non-finite joint angle");
    for (int i = 0; i < M; ++i)
        if (motion_scene[i] < 0 || motion_scene[i] >= n_scenes) return pfail(m, SVM_E_INVALID, "motion scene out of range");

    svm_plan* p = new svm_plan();
    p->m = m;
    p->M = M;
    p->N = steps;
    p->S = n_scenes;
    p->flags = flags;
    p->margin = margin;
    p->bm = m->desc.prec != SVM_FP32 ? tc_tile_rows() : mlp_fp32_tile_rows();
    if (m->desc.prec == SVM_FP32) {
        const long long sb = mlp_fp32_small_tile_rows();
        long long small = 0;
        for (int i = 0; i < M; ++i) {
            const long long n = scene_offsets[motion_scene[i] + 1] - scene_offsets[motion_scene[i]];
            small += (n + sb - 1) / sb;
        }
        p->bm = mlp_fp32_tile_rows(small, m->n_sms);
    }
    std::vector<long long> pbeg(M), pend(M), poff(M + 1);
    std::vector<int> toff(M + 1);
    toff[0] = 0;
    poff[0] = 0;
    for (int i = 0; i < M; ++i) {
        const int s = motion_scene[i];
        pbeg[i] = scene_offsets[s];
        pend[i] = scene_offsets[s + 1];
        const long long n = pend[i] - pbeg[i];
        const long long t = toff[i] + (n + p->bm - 1) / p->bm;
        if (t > 0x7fffffffLL) { delete p; return pfail(m, SVM_E_INVALID, "too many tiles"); }
        toff[i + 1] = (int)t;
        poff[i + 1] = poff[i] + n;
    }
    p->n_tiles = toff[M];
    p->P_total = poff[M];
    size_t at = 0;
    p->o_q0 = at; at = al256(at + (size_t)M * 48);
    p->o_q1 = at; at = al256(at + (size_t)M * 48);
    p->o_pbeg = at; at = al256(at + (size_t)M * 8);
    p->o_pend = at; at = al256(at + (size_t)M * 8);
    p->o_toff = at; at = al256(at + (size_t)(M + 1) * 4);
    p->o_poff = at; at = al256(at + (size_t)(M + 1) * 8);
    const size_t header = at;
    p->o_caps = at; at = al256(at + (size_t)M * (steps + 1) * kCaps * sizeof(Capsule));
    p->o_fk64 = at; at = al256(at + (size_t)M * (steps + 1) * 24 * sizeof(double));
    p->o_cbias = at; at = al256(at + (size_t)M * cbias_stride(m->desc) * 4);
    p->o_st = at; at = al256(at + (size_t)M * sizeof(MotionState));
    p->o_idx = at; at = al256(at + (size_t)std::max<long long>(1, p->P_total) * 4);
    p->o_chunk = at; at = al256(at + (size_t)(M + 1) * 4);
    p->o_err = at; at = al256(at + 4);
    p->o_tie = at; at = al256(at + 256 + tie_list_bytes());
    p->total = at;
    Guard g(m->device);
    if (cudaMalloc(&p->ws, p->total) != cudaSuccess) {
        cudaGetLastError();
        delete p;
        return pfail(m, SVM_E_OOM, "plan workspace allocation failed");
    }
    std::vector<char> h(header, 0);
    std::memcpy(h.data() + p->o_q0, q0, (size_t)M * 48);
    std::memcpy(h.data() + p->o_q1, q1, (size_t)M * 48);
    std::memcpy(h.data() + p->o_pbeg, pbeg.data(), (size_t)M * 8);
    std::memcpy(h.data() + p->o_pend, pend.data(), (size_t)M * 8);
    std::memcpy(h.data() + p->o_toff, toff.data(), (size_t)(M + 1) * 4);
    std::memcpy(h.data() + p->o_poff, poff.data(), (size_t)(M + 1) * 8);
    const cudaError_t e = cudaMemcpy(p->ws, h.data(), header, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(p->ws);
        delete p;
        return pfail(m, SVM_E_CUDA, cudaGetErrorString(e));
    }
    *out = p;
    return SVM_OK;
}

svm_status svm_plan_destroy(svm_plan* p)
{
    if (!p) return SVM_E_INVALID;
    {
        Guard g(p->m->device);
        cudaDeviceSynchronize();
        drop_graph(p);
        if (p->ws) cudaFree(p->ws);
    }
    delete p;
    return SVM_OK;
}

svm_status svm_plan_launch(svm_plan* p, const float* points_dev, svm_result* results_dev, void* stream)
{
    const Range call_range("svm_plan_launch");
    if (!p || !results_dev) return SVM_E_INVALID;
    if (p->P_total > 0 && (!points_dev || reinterpret_cast<uintptr_t>(points_dev) % 16))
        return pfail(p->m, SVM_E_INVALID, "points missing or not 16-byte aligned");
    Guard g(p->m->device);
    return enqueue(p, points_dev, results_dev, static_cast<cudaStream_t>(stream));
}

svm_status svm_plan_graph_launch(svm_plan* p, const float* points_dev, svm_result* results_dev, void* stream)
{
    const Range call_range("svm_plan_graph_launch");
    if (!p || !results_dev) return SVM_E_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (s == nullptr || s == cudaStreamLegacy || s == cudaStreamPerThread)
        return pfail(p->m, SVM_E_INVALID, "graph launch needs a created (non-default) stream");
    if (p->P_total > 0 && (!points_dev || reinterpret_cast<uintptr_t>(points_dev) % 16))
        return pfail(p->m, SVM_E_INVALID, "points missing or not 16-byte aligned");
    Guard g(p->m->device);
    if (!p->exec || p->g_points != points_dev || p->g_results != results_dev) {
        drop_graph(p);
        // one plain launch first: it sets the kernels' shared-memory limits outside the capture
        svm_status st = enqueue(p, points_dev, results_dev, s);
        if (st != SVM_OK) return st;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return pfail(p->m, SVM_E_CUDA, cudaGetErrorString(e));
        st = enqueue(p, points_dev, results_dev, s);
        cudaGraph_t graph = nullptr;
        e = cudaStreamEndCapture(s, &graph);
        if (st != SVM_OK) { if (graph) cudaGraphDestroy(graph); return st; }
        if (e != cudaSuccess) return pfail(p->m, SVM_E_CUDA, cudaGetErrorString(e));
        e = cudaGraphInstantiate(&p->exec, graph, 0);
        if (e != cudaSuccess) { cudaGraphDestroy(graph); return pfail(p->m, SVM_E_CUDA, cudaGetErrorString(e)); }
        p->graph = graph;
        p->g_points = points_dev;
        p->g_results = results_dev;
        return SVM_OK;     // the plain launch above already produced this call's results
    }
    const cudaError_t e = cudaGraphLaunch(p->exec, s);
    if (e != cudaSuccess) return pfail(p->m, SVM_E_CUDA, cudaGetErrorString(e));
    return SVM_OK;
}

svm_status svm_plan_set_verify_shape(svm_plan* p, int32_t points_per_thread, int32_t ctas_per_sm)
{
    if (!p) return SVM_E_INVALID;
    if (!(points_per_thread == 1 || points_per_thread == 2 || points_per_thread == 4) || ctas_per_sm < 0 ||
        ctas_per_sm > 8)
        return pfail(p->m, SVM_E_INVALID, "points_per_thread must be 1, 2 or 4 and ctas_per_sm 0..8");
    p->vcfg.points_per_thread = points_per_thread;
    p->vcfg.ctas_per_sm = ctas_per_sm;
    Guard g(p->m->device);
    cudaDeviceSynchronize();
    drop_graph(p);
    return SVM_OK;
}

svm_status svm_plan_set_network_grid(svm_plan* p, int32_t ctas)
{
    if (!p) return SVM_E_INVALID;
    if (ctas < 0 || ctas > p->m->n_sms) return pfail(p->m, SVM_E_INVALID, "ctas must be 0..number of SMs");
    p->net_grid = ctas;
    Guard g(p->m->device);
    cudaDeviceSynchronize();
    drop_graph(p);
    return SVM_OK;
}

svm_status svm_plan_autotune(svm_plan* p, const float* points_dev, svm_result* results_dev, void* stream,
                             char* report, size_t capacity)
{
    if (!p || !results_dev) return SVM_E_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    Guard g(p->m->device);
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return pfail(p->m, SVM_E_CUDA, "event creation failed");
    svm_status st = SVM_OK;
    // mean time of 3 launches after one warm-up launch, CUDA events on the plan's stream
    auto time_launch = [&](float& ms) {
        st = enqueue(p, points_dev, results_dev, s);
        if (st != SVM_OK) return false;
        cudaEventRecord(e0, s);
        const int reps = 3;
        for (int r = 0; r < reps && st == SVM_OK; ++r) st = enqueue(p, points_dev, results_dev, s);
        cudaEventRecord(e1, s);
        if (st != SVM_OK) return false;
        if (cudaEventSynchronize(e1) != cudaSuccess) { st = pfail(p->m, SVM_E_CUDA, "autotune timing failed"); return false; }
        cudaEventElapsedTime(&ms, e0, e1);
        ms /= reps;
        return true;
    };
    std::string rep = "{\"network_candidates\": [";
    char buf[192];
    // 1. the network kernel's persistent grid (tensor-core models run the network)
    const bool net = p->m->desc.prec != SVM_FP32 && !(p->flags & SVM_VERIFY_ALL);
    const int n_sms = p->m->n_sms;
    int best_grid = p->net_grid;
    if (net) {
        const int grids[5] = {n_sms, n_sms - n_sms / 16, n_sms - n_sms / 8, (3 * n_sms) / 4, n_sms / 2};
        float best = INFINITY;
        for (int i = 0; i < 5 && st == SVM_OK; ++i) {
            p->net_grid = grids[i];
            float ms = 0.0f;
            if (!time_launch(ms)) break;
            std::snprintf(buf, sizeof buf, "%s{\"grid\": %d, \"ms\": %.4f}", i ? ", " : "", grids[i], ms);
            rep += buf;
            if (ms < best) { best = ms; best_grid = grids[i]; }
        }
    }
    p->net_grid = best_grid;
    // 2. the verifier's shape at that grid
    const int ppts[3] = {1, 2, 4};
    const int ctas[3] = {0, 4, 2};
    float best = INFINITY;
    VerifyConfig best_cfg = p->vcfg;
    rep += "], \"candidates\": [";
    bool first = true;
    for (int a = 0; a < 3 && st == SVM_OK; ++a)
        for (int b = 0; b < 3 && st == SVM_OK; ++b) {
            p->vcfg.points_per_thread = ppts[a];
            p->vcfg.ctas_per_sm = ctas[b];
            float ms = 0.0f;
            if (!time_launch(ms)) break;
            std::snprintf(buf, sizeof buf, "%s{\"points_per_thread\": %d, \"ctas_per_sm\": %d, \"ms\": %.4f}",
                          first ? "" : ", ", ppts[a], ctas[b], ms);
            rep += buf;
            first = false;
            if (ms < best) { best = ms; best_cfg = p->vcfg; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    p->vcfg = best_cfg;
    drop_graph(p);
    if (st != SVM_OK) return st;
    std::snprintf(buf, sizeof buf,
                  "], \"best\": {\"network_grid\": %d, \"points_per_thread\": %d, \"ctas_per_sm\": %d, "
                  "\"ms\": %.4f}}",
                  p->net_grid > 0 ? p->net_grid : n_sms, best_cfg.points_per_thread, best_cfg.ctas_per_sm, best);
    rep += buf;
    if (report && capacity > 0) {
        const size_t n = std::min(capacity - 1, rep.size());
        std::memcpy(report, rep.data(), n);
        report[n] = 0;
    }
    return SVM_OK;
}

}  // extern "C"
