// svm_api.cu -- host side of libsvm: the C ABI declared in include/svm.h.
//
// The model owns its device weights, a workspace that grows on demand, a
// pinned staging buffer for the per-call host arrays and the events that
// guard them.  A check call validates its arguments on the host, copies the
// small per-motion arrays (q0, q1, point ranges, tile prefix) in one
// host-to-device copy, and enqueues the kernels on the caller's stream:
// prologue (FK + per-motion bias) -> fused network + gate + compaction ->
// verifier (-> strict second pass) -> finalize.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "svm.h"
#include "svm_internal.cuh"
#include "mlp_tc.cuh"
#include "svm_model.h"

using namespace svm;


namespace {

const char* kStatusText[] = {"ok", "invalid argument", "CUDA error", "out of device memory",
                             "device wait timed out", "bad or missing weights", "unsupported"};

svm_status fail(svm_model* m, svm_status s, const std::string& msg)
{
    if (m) m->last_error = msg;
    return s;
}

#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(m, SVM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// SVM_WORKSPACE_LIMIT (decimal bytes), when set, caps the device workspace a
// model may allocate for its calls; 0 when unset or malformed.
size_t workspace_limit()
{
    const char* s = std::getenv("SVM_WORKSPACE_LIMIT");
    if (!s || !*s) return 0;
    char* end = nullptr;
    const unsigned long long v = std::strtoull(s, &end, 10);
    return (end && *end == 0) ? (size_t)v : 0;
}

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

long long layer_count(const svm_model_desc& d) { return (long long)d.n_hidden + 2; }

// Offsets of the layers in the flat blob-order parameter vector.
struct Layout {
    long long w1, b1, wh0, out_w, out_b, total;
    long long hidden_stride;   // W*W + W
};
Layout layout_of(const svm_model_desc& d)
{
    Layout L{};
    const long long W = d.width;
    L.w1 = 0;
    L.b1 = W * kInDim;
    L.wh0 = L.b1 + W;
    L.hidden_stride = W * W + W;
    L.out_w = L.wh0 + (long long)d.n_hidden * L.hidden_stride;
    L.out_b = L.out_w + W;
    L.total = L.out_b + 1;
    return L;
}

bool finite_all(const double* p, long long n)
{
    for (long long i = 0; i < n; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// FP8: hidden biases divided by the activation scale of the layer they feed
// (b_l / ascale[l] for hidden layers l < L-1, 0-based), the form the packed
// epilogue adds after its single rescaling multiply.
svm_status upload_scaled_biases(svm_model* m)
{
    const long long W = m->desc.width, L = m->desc.n_hidden;
    if (!m->dw.bhs || (long long)m->bh_host.size() != L * W) return SVM_OK;
    std::vector<float> bhs(L * W, 0.0f);
    for (long long l = 0; l + 1 < L; ++l)
        for (long long o = 0; o < W; ++o) bhs[l * W + o] = m->bh_host[l * W + o] / m->ascales[l + 1];
    const cudaError_t e = cudaMemcpy(const_cast<float*>(m->dw.bhs), bhs.data(), L * W * 4, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return fail(m, SVM_E_CUDA, std::string("bias upload: ") + cudaGetErrorString(e));
    return SVM_OK;
}

// Version-2 blob of the block architecture: parse, fold BatchNorm into a
// per-channel scale and shift, and upload the FP32 layouts the FP32 kernel
// and the prologue read.
svm_status load_block_weights(svm_model* m, const unsigned char* p, size_t bytes)
{
    const svm_model_desc& d = m->desc;
    auto rd32 = [&](size_t off) { uint32_t v; std::memcpy(&v, p + off, 4); return v; };
    if (bytes < 32) return fail(m, SVM_E_WEIGHTS, "truncated blob");
    const uint32_t nb = rd32(8), in_dim = rd32(12), width = rd32(16), act = rd32(20);
    float tau, bn_eps;
    std::memcpy(&tau, p + 24, 4);
    std::memcpy(&bn_eps, p + 28, 4);
    if ((int)nb != d.n_hidden || in_dim != (uint32_t)kInDim || width != (uint32_t)d.width || act != SVM_RELU)
        return fail(m, SVM_E_WEIGHTS, "blob does not match the model description");
    if (!(bn_eps >= 0.0f) || !std::isfinite(bn_eps)) return fail(m, SVM_E_WEIGHTS, "bad BatchNorm epsilon");
    const long long W = d.width, L = d.n_hidden, J = W + kInDim;
    size_t off = 32;
    std::vector<float> all;   // every float of the blob in order (the export)
    auto take = [&](uint32_t want_o, uint32_t want_i, size_t n_extra, std::vector<float>& dst) -> bool {
        if (off + 8 > bytes) return false;
        if (rd32(off) != want_o || rd32(off + 4) != want_i) return false;
        off += 8;
        const size_t n = (size_t)want_o * want_i + n_extra;
        if (off + n * 4 > bytes) return false;
        dst.resize(n);
        std::memcpy(dst.data(), p + off, n * 4);
        off += n * 4;
        all.insert(all.end(), dst.begin(), dst.end());
        return true;
    };
    std::vector<float> init, fin;
    std::vector<std::vector<float>> blk(L);
    if (!take((uint32_t)W, (uint32_t)kInDim, W, init)) return fail(m, SVM_E_WEIGHTS, "initial layer shape or size");
    for (long long l = 0; l < L; ++l)
        if (!take((uint32_t)W, (uint32_t)(l == 0 ? W : J), 5 * W, blk[l]))
            return fail(m, SVM_E_WEIGHTS, "block shape or size");
    if (!take(1u, (uint32_t)J, 1, fin)) return fail(m, SVM_E_WEIGHTS, "final layer shape or size");
    if (off != bytes) return fail(m, SVM_E_WEIGHTS, "trailing bytes in blob");
    for (float v : all)
        if (!std::isfinite(v)) return fail(m, SVM_E_WEIGHTS, "non-finite weight");
    const bool bf16 = d.prec == SVM_BF16;
    if (bf16) {
        // BF16 model: every weight matrix rounded to nearest-even bfloat16 (biases and BatchNorm
        // statistics stay FP32); the export then holds the rounded values
        auto rnd = [](float v) {
            uint32_t u;
            std::memcpy(&u, &v, 4);
            u += 0x7FFFu + ((u >> 16) & 1u);
            u &= 0xFFFF0000u;
            float r;
            std::memcpy(&r, &u, 4);
            return r;
        };
        for (long long i = 0; i < W * kInDim; ++i) init[i] = rnd(init[i]);
        for (long long l = 0; l < L; ++l)
            for (long long i = 0; i < W * (l == 0 ? W : J); ++i) blk[l][i] = rnd(blk[l][i]);
        for (long long i = 0; i < J; ++i) fin[i] = rnd(fin[i]);
        all.clear();
        all.insert(all.end(), init.begin(), init.end());
        for (long long l = 0; l < L; ++l) all.insert(all.end(), blk[l].begin(), blk[l].end());
        all.insert(all.end(), fin.begin(), fin.end());
    }

    std::vector<float> w1x(W * 3), wT(L * W * W), wout(W), blk_wx(L * W * 3, 0.0f), blk_wq((L + 1) * W * 12),
        blk_b((L + 1) * W), blk_s(L * W), blk_t(L * W), out_wx(3), out_wq(12);
    for (long long o = 0; o < W; ++o) {
        for (int c = 0; c < 3; ++c) w1x[o * 3 + c] = init[o * kInDim + c];
        for (int c = 0; c < 12; ++c) blk_wq[o * 12 + c] = init[o * kInDim + 3 + c];
        blk_b[o] = init[W * kInDim + o];
    }
    for (long long l = 0; l < L; ++l) {
        const long long in = l == 0 ? W : J;
        const float* Wl = blk[l].data();
        const float* bl = Wl + W * in;
        const float *gamma = bl + W, *beta = bl + 2 * W, *mean = bl + 3 * W, *var = bl + 4 * W;
        for (long long o = 0; o < W; ++o) {
            for (long long i = 0; i < W; ++i) wT[(l * W + i) * W + o] = Wl[o * in + i];
            if (l > 0) {
                for (int c = 0; c < 3; ++c) blk_wx[(l * W + o) * 3 + c] = Wl[o * in + W + c];
                for (int c = 0; c < 12; ++c) blk_wq[((l + 1) * W + o) * 12 + c] = Wl[o * in + W + 3 + c];
            } else {
                for (int c = 0; c < 12; ++c) blk_wq[((l + 1) * W + o) * 12 + c] = 0.0f;
            }
            blk_b[(l + 1) * W + o] = bl[o];
            const double sc = (double)gamma[o] / std::sqrt((double)var[o] + (double)bn_eps);
            blk_s[l * W + o] = (float)sc;
            blk_t[l * W + o] = (float)((double)beta[o] - (double)mean[o] * sc);
        }
    }
    for (long long o = 0; o < W; ++o) wout[o] = fin[o];
    for (int c = 0; c < 3; ++c) out_wx[c] = fin[W + c];
    for (int c = 0; c < 12; ++c) out_wq[c] = fin[W + 3 + c];
    const float bout = fin[J];
    // BF16: the blocks' weights for the tensor cores (K-major B operands, bfloat16): the h-weights,
    // [L][W outputs][W inputs], then the x-weights padded to K = 16, [L][W outputs][16] with row
    // (w_x, w_y, w_z) three times, then zeros, applied to (x_hi, y_hi, z_hi, x_mid, .., z_lo, 0, ...):
    // block l's jump x-weights, and in the place of block 1 (which has no jump input) the initial
    // layer's.  The weights are BF16-rounded above, so the upper half of each FP32 word is the exact value.
    std::vector<uint16_t> wh;
    if (bf16) {
        auto hi16 = [](float v) {
            uint32_t u;
            std::memcpy(&u, &v, 4);
            return (uint16_t)(u >> 16);
        };
        wh.assign((size_t)L * W * W + (size_t)L * W * 16, 0);
        for (long long l = 0; l < L; ++l) {
            const long long in = l == 0 ? W : J;
            for (long long o = 0; o < W; ++o) {
                for (long long i = 0; i < W; ++i) wh[((size_t)l * W + o) * W + i] = hi16(blk[l][o * in + i]);
                uint16_t* xr = &wh[(size_t)L * W * W + ((size_t)l * W + o) * 16];
                for (int c = 0; c < 3; ++c)
                    xr[c] = xr[3 + c] = xr[6 + c] =
                        hi16(l == 0 ? w1x[o * 3 + c] : blk_wx[((size_t)l * W + o) * 3 + c]);
            }
        }
    }

    // the block kernel's per-column-pair record (see DevWeights::blk_pk)
    std::vector<float> blk_pk;
    if (d.arch == SVM_ARCH_BLOCKS && W % 2 == 0) {
        blk_pk.assign((size_t)L * (W / 2) * 4, 0.0f);
        for (int l = 0; l < L; ++l)
            for (int c = 0; c < W; c += 2) {
                float* r = &blk_pk[((size_t)l * (W / 2) + c / 2) * 4];
                r[0] = blk_s[l * W + c];
                r[1] = blk_s[l * W + c + 1];
                r[2] = blk_t[l * W + c];
                r[3] = blk_t[l * W + c + 1];
            }
    }
    DeviceGuard g(m->device);
    CK(cudaDeviceSynchronize());
    size_t total = 0;
    const std::vector<const std::vector<float>*> parts = {&w1x, &wT, &wout, &blk_wx, &blk_wq, &blk_b, &blk_s,
                                                          &blk_t, &out_wx, &out_wq, &blk_pk};
    for (auto* v : parts) total += align256(std::max<size_t>(1, v->size()) * 4);
    const size_t wh_at = total;
    total += align256(wh.size() * 2);
    if (m->d_weights) { cudaFree(m->d_weights); m->d_weights = nullptr; }
    if (cudaMalloc(&m->d_weights, total) != cudaSuccess) return fail(m, SVM_E_OOM, "weights allocation failed");
    char* base = static_cast<char*>(m->d_weights);
    size_t at = 0;
    std::vector<const float*> dev;
    for (auto* v : parts) {
        if (!v->empty()) CK(cudaMemcpy(base + at, v->data(), v->size() * 4, cudaMemcpyHostToDevice));
        dev.push_back(reinterpret_cast<const float*>(base + at));
        at += align256(std::max<size_t>(1, v->size()) * 4);
    }
    DevWeights& dw = m->dw;
    dw = DevWeights{};
    dw.w1x = dev[0];
    dw.wT = dev[1];
    dw.wout = dev[2];
    dw.blk_wx = dev[3];
    dw.blk_wq = dev[4];
    dw.blk_b = dev[5];
    dw.blk_s = dev[6];
    dw.blk_t = dev[7];
    dw.out_wx = dev[8];
    dw.out_wq = dev[9];
    dw.blk_pk = dev[10];
    dw.bout = bout;
    if (bf16) {
        CK(cudaMemcpy(base + wh_at, wh.data(), wh.size() * 2, cudaMemcpyHostToDevice));
        dw.wq = base + wh_at;
        if (tc_block_prepare(m->tc, d, dw.wq) != 0) return fail(m, SVM_E_UNSUPPORTED, "tensor-core block setup failed");
    }
    m->used = all;
    m->tau = std::isfinite(tau) && tau >= 0 ? tau : INFINITY;
    m->has_weights = true;
    return SVM_OK;
}

}  // namespace

extern "C" {

const char* svm_status_string(svm_status s)
{
    const int i = (int)s;
    return (i >= 0 && i <= 6) ? kStatusText[i] : "unknown status";
}

const char* svm_last_error(const svm_model* m) { return m ? m->last_error.c_str() : "null model"; }

svm_status svm_create_model(const svm_model_desc* desc, int device, svm_model** out)
{
    svm_model* m = nullptr;
    if (!desc || !out) return SVM_E_INVALID;
    *out = nullptr;
    const svm_model_desc& d = *desc;
    for (int j = 0; j < 6; ++j)
        if (!finite_all(d.dh[j], 4)) return SVM_E_INVALID;
    for (int j = 0; j < 7; ++j)
        if (!std::isfinite(d.radius[j])) return SVM_E_INVALID;
    if (!std::isfinite(d.tool_len) || d.tool_len < 0) return SVM_E_INVALID;
    if (d.act != SVM_RELU && d.act != SVM_SILU) return SVM_E_INVALID;
    if (d.prec < SVM_FP32 || d.prec > SVM_FP8_E4M3) return SVM_E_INVALID;
    if (d.n_hidden < 0 || d.n_hidden > 16) return SVM_E_INVALID;
    if (d.arch != SVM_ARCH_MLP && d.arch != SVM_ARCH_BLOCKS) return SVM_E_INVALID;
    if (d.arch == SVM_ARCH_BLOCKS && (d.act != SVM_RELU || d.n_hidden < 1)) return SVM_E_UNSUPPORTED;
    // the block architecture runs in FP32 (SIMT) or, at width 512, in BF16 on the tensor cores
    if (d.arch == SVM_ARCH_BLOCKS && d.prec != SVM_FP32 && !(d.prec == SVM_BF16 && d.width == 512))
        return SVM_E_UNSUPPORTED;
    if (d.arch == SVM_ARCH_BLOCKS && d.prec == SVM_BF16) {
        // checked above
    } else if (d.prec == SVM_FP32) {
        if (!(d.width == 64 || d.width == 128 || d.width == 256 || d.width == 512 || d.width == 1024))
            return SVM_E_UNSUPPORTED;
    } else {
        if (d.width != 256 || d.n_hidden < 1) return SVM_E_UNSUPPORTED;
    }
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) return SVM_E_INVALID;
    m = new svm_model();
    m->device = device;
    m->desc = d;
    DeviceGuard g(device);
    cudaDeviceGetAttribute(&m->n_sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&m->cc_major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&m->cc_minor, cudaDevAttrComputeCapabilityMinor, device);
    if (d.prec != SVM_FP32 && !(m->cc_major == 10 && m->cc_minor == 3)) {
        delete m;
        return SVM_E_UNSUPPORTED;
    }
    for (int j = 0; j < 6; ++j) {
        m->rp.d[j] = d.dh[j][0];
        m->rp.a[j] = d.dh[j][1];
        m->rp.ca[j] = std::cos(d.dh[j][2]);
        m->rp.sa[j] = std::sin(d.dh[j][2]);
        m->rp.th0[j] = d.dh[j][3];
    }
    m->rp.tool_len = d.tool_len;
    for (int j = 0; j < 7; ++j) {
        m->rp.radius[j] = (float)d.radius[j];
        m->rp.radius64[j] = d.radius[j];
    }
    if (cudaEventCreateWithFlags(&m->staging_done, cudaEventDisableTiming) != cudaSuccess) {
        delete m;
        return SVM_E_CUDA;
    }
    m->ascales.assign(d.n_hidden, 1.0f);
    *out = m;
    return SVM_OK;
}

svm_status svm_destroy_model(svm_model* m)
{
    if (!m) return SVM_E_INVALID;
    {
        DeviceGuard g(m->device);
        cudaDeviceSynchronize();
        tc_release(m->tc);
        if (m->d_weights) cudaFree(m->d_weights);
        if (m->ws) cudaFree(m->ws);
        if (m->pinned) cudaFreeHost(m->pinned);
        if (m->search_dev) cudaFree(m->search_dev);
        if (m->search_host) cudaFreeHost(m->search_host);
        if (m->staging_done) cudaEventDestroy(m->staging_done);
        for (auto& e : m->ev)
            if (e) cudaEventDestroy(e);
    }
    delete m;
    return SVM_OK;
}

svm_status svm_test_expire_wait(svm_model* m, int32_t n_calls)
{
    if (!m || n_calls < 0) return SVM_E_INVALID;
    if (m->desc.prec == SVM_FP32) return fail(m, SVM_E_UNSUPPORTED, "the FP32 path has no device waits");
    m->test_stalls = n_calls;
    return SVM_OK;
}

svm_status svm_test_set_tie_cap(svm_model* m, int32_t cap)
{
    if (!m || cap < 0 || cap > kTieCap) return SVM_E_INVALID;
    m->tie_cap = cap;
    return SVM_OK;
}

svm_status svm_set_gate(svm_model* m, float tau)
{
    if (!m) return SVM_E_INVALID;
    if (std::isnan(tau) || tau < 0) return fail(m, SVM_E_INVALID, "tau must be >= 0");
    m->tau = tau;
    return SVM_OK;
}

svm_status svm_set_act_scales(svm_model* m, const float* scales, int32_t n)
{
    if (!m || !scales) return SVM_E_INVALID;
    if (n != m->desc.n_hidden) return fail(m, SVM_E_INVALID, "need one activation scale per hidden layer");
    for (int i = 0; i < n; ++i)
        if (!(scales[i] > 0) || !std::isfinite(scales[i])) return fail(m, SVM_E_INVALID, "scale must be finite and > 0");
    m->ascales.assign(scales, scales + n);
    if (m->has_weights && m->dw.ascale) {
        DeviceGuard g(m->device);
        CK(cudaMemcpy(const_cast<float*>(m->dw.ascale), scales, n * sizeof(float), cudaMemcpyHostToDevice));
        const svm_status st = upload_scaled_biases(m);
        if (st != SVM_OK) return st;
    }
    return SVM_OK;
}

svm_status svm_load_weights(svm_model* m, const void* blob, size_t bytes)
{
    if (!m || !blob) return SVM_E_INVALID;
    const svm_model_desc& d = m->desc;
    const unsigned char* p = static_cast<const unsigned char*>(blob);
    auto rd32 = [&](size_t off) { uint32_t v; std::memcpy(&v, p + off, 4); return v; };
    if (bytes < 28 || std::memcmp(p, "SVMW", 4) != 0) return fail(m, SVM_E_WEIGHTS, "bad magic");
    if (d.arch == SVM_ARCH_BLOCKS) {
        if (rd32(4) != 2) return fail(m, SVM_E_WEIGHTS, "block models take blob version 2");
        return load_block_weights(m, p, bytes);
    }
    if (rd32(4) != 1) return fail(m, SVM_E_WEIGHTS, "unsupported blob version");
    const uint32_t n_layers = rd32(8), in_dim = rd32(12), width = rd32(16), act = rd32(20);
    float tau;
    std::memcpy(&tau, p + 24, 4);
    if ((long long)n_layers != layer_count(d) || in_dim != (uint32_t)kInDim || width != (uint32_t)d.width ||
        act != (uint32_t)d.act)
        return fail(m, SVM_E_WEIGHTS, "blob does not match the model description");
    const Layout Lo = layout_of(d);
    std::vector<float> orig(Lo.total);
    size_t off = 28;
    long long pos = 0;
    for (uint32_t l = 0; l < n_layers; ++l) {
        if (off + 8 > bytes) return fail(m, SVM_E_WEIGHTS, "truncated blob");
        const uint32_t o = rd32(off), i = rd32(off + 4);
        off += 8;
        const uint32_t want_o = (l + 1 == n_layers) ? 1u : width;
        const uint32_t want_i = (l == 0) ? (uint32_t)kInDim : width;
        if (o != want_o || i != want_i) return fail(m, SVM_E_WEIGHTS, "layer shape mismatch");
        const size_t nb = ((size_t)o * i + o) * 4;
        if (off + nb > bytes) return fail(m, SVM_E_WEIGHTS, "truncated blob");
        std::memcpy(orig.data() + pos, p + off, nb);
        off += nb;
        pos += (long long)o * i + o;
    }
    if (off != bytes) return fail(m, SVM_E_WEIGHTS, "trailing bytes in blob");
    for (float v : orig)
        if (!std::isfinite(v)) return fail(m, SVM_E_WEIGHTS, "non-finite weight");

    DeviceGuard g(m->device);
    CK(cudaDeviceSynchronize());
    const long long W = d.width, L = d.n_hidden;
    // 1) rounding to the model precision on the device
    std::vector<uint8_t> e4(L * W * W);
    std::vector<float> wscale(L, 1.0f);
    {
        float* tmp = nullptr;
        uint8_t* tq = nullptr;
        CK(cudaMalloc(&tmp, Lo.total * sizeof(float)));
        CK(cudaMalloc(&tq, (size_t)std::max<long long>(1, L * W * W)));
        CK(cudaMemcpy(tmp, orig.data(), Lo.total * sizeof(float), cudaMemcpyHostToDevice));
        if (d.prec == SVM_BF16 || d.prec == SVM_FP8_E4M3) {
            launch_round_bf16(tmp + Lo.w1, W * kInDim, 0);
            launch_round_bf16(tmp + Lo.out_w, W, 0);
        }
        for (long long l = 0; l < L; ++l) {
            float* wl = tmp + Lo.wh0 + l * Lo.hidden_stride;
            if (d.prec == SVM_BF16) launch_round_bf16(wl, W * W, 0);
            if (d.prec == SVM_FP8_E4M3) {
                float mx = 0.f;
                const float* hw = orig.data() + Lo.wh0 + l * Lo.hidden_stride;
                for (long long i = 0; i < W * W; ++i) mx = std::max(mx, std::fabs(hw[i]));
                const float s = mx > 0.f ? mx / 448.0f : 1.0f;
                wscale[l] = s;
                launch_quantize_e4m3(wl, tq + l * W * W, wl, W * W, s, 0);
            }
        }
        CK(cudaGetLastError());
        m->used.resize(Lo.total);
        CK(cudaMemcpy(m->used.data(), tmp, Lo.total * sizeof(float), cudaMemcpyDeviceToHost));
        if (d.prec == SVM_FP8_E4M3) CK(cudaMemcpy(e4.data(), tq, L * W * W, cudaMemcpyDeviceToHost));
        cudaFree(tmp);
        cudaFree(tq);
    }
    // 2) device layouts of the used values
    const std::vector<float>& u = m->used;
    std::vector<float> w1x(W * 3), w1q(W * 12), b1(W), wT(L * W * W), bh(L * W), wout(W);
    for (long long o = 0; o < W; ++o) {
        for (int c = 0; c < 3; ++c) w1x[o * 3 + c] = u[Lo.w1 + o * kInDim + c];
        for (int c = 0; c < 12; ++c) w1q[o * 12 + c] = u[Lo.w1 + o * kInDim + 3 + c];
        b1[o] = u[Lo.b1 + o];
        wout[o] = u[Lo.out_w + o];
    }
    for (long long l = 0; l < L; ++l) {
        const float* wl = u.data() + Lo.wh0 + l * Lo.hidden_stride;
        for (long long o = 0; o < W; ++o)
            for (long long i = 0; i < W; ++i) wT[(l * W + i) * W + o] = wl[o * W + i];
        for (long long o = 0; o < W; ++o) bh[l * W + o] = wl[W * W + o];
    }
    // hidden weights for the tensor-core path, [L][W out][W in]
    std::vector<uint16_t> bf(d.prec == SVM_BF16 ? L * W * W : 0);
    if (d.prec == SVM_BF16)
        for (long long l = 0; l < L; ++l) {
            const float* wl = u.data() + Lo.wh0 + l * Lo.hidden_stride;
            for (long long i = 0; i < W * W; ++i) {
                uint32_t bits;
                std::memcpy(&bits, wl + i, 4);
                bf[l * W * W + i] = (uint16_t)(bits >> 16);   // exact: value is a bfloat16
            }
        }
    // layer-1 x-weights for the tensor path (values already bfloat16 in these modes)
    std::vector<uint16_t> w1pad(d.prec != SVM_FP32 ? W * 64 : 0, 0);
    if (d.prec != SVM_FP32)
        for (long long o = 0; o < W; ++o)
            for (int c = 0; c < 3; ++c) {
                uint32_t bits;
                std::memcpy(&bits, &w1x[o * 3 + c], 4);
                w1pad[o * 64 + c] = w1pad[o * 64 + 3 + c] = (uint16_t)(bits >> 16);
            }
    const size_t n_w1pad = align256(std::max<long long>(1, (long long)w1pad.size() * 2));
    const size_t n_w1x = align256(W * 3 * 4), n_w1q = align256(W * 12 * 4), n_b1 = align256(W * 4),
                 n_wT = align256(L * W * W * 4), n_bh = align256(std::max<long long>(1, L * W) * 4),
                 n_wout = align256(W * 4), n_wq = align256(std::max<long long>(1, L * W * W * 2)),
                 n_sc = align256(std::max<long long>(1, L) * 4);
    const size_t total = n_w1x + n_w1q + n_b1 + n_wT + n_bh + n_wout + n_wq + 2 * n_sc + n_w1pad + n_bh;
    if (m->d_weights) { cudaFree(m->d_weights); m->d_weights = nullptr; }
    if (cudaMalloc(&m->d_weights, total) != cudaSuccess) return fail(m, SVM_E_OOM, "weights allocation failed");
    char* base = static_cast<char*>(m->d_weights);
    size_t at = 0;
    auto put = [&](const void* src, size_t nbytes, size_t slot) {
        void* dst = base + at;
        if (nbytes) cudaMemcpy(dst, src, nbytes, cudaMemcpyHostToDevice);
        at += slot;
        return dst;
    };
    DevWeights& dw = m->dw;
    dw.w1x = (const float*)put(w1x.data(), W * 3 * 4, n_w1x);
    dw.w1q = (const float*)put(w1q.data(), W * 12 * 4, n_w1q);
    dw.b1 = (const float*)put(b1.data(), W * 4, n_b1);
    dw.wT = (const float*)put(wT.data(), L * W * W * 4, n_wT);
    dw.bh = (const float*)put(bh.data(), L * W * 4, n_bh);
    dw.wout = (const float*)put(wout.data(), W * 4, n_wout);
    if (d.prec == SVM_FP8_E4M3 && d.act == SVM_RELU) {
        // The FP8 ReLU kernel stores each activation's 16-column blocks in the order
        // pi(j) = 4 ((j & 7) >> 1) + 2 (j >> 3) + (j & 1) (its fragment-shape stores); the hidden
        // weights take their K columns in the same order, so every product is unchanged.
        std::vector<uint8_t> e4p(e4.size());
        for (long long row = 0; row < L * W; ++row)
            for (long long k = 0; k < W; ++k) {
                const int j = (int)(k & 15);
                const long long pk = (k & ~15LL) + 4 * ((j & 7) >> 1) + 2 * (j >> 3) + (j & 1);
                e4p[row * W + pk] = e4[row * W + k];
            }
        e4.swap(e4p);
    }
    if (d.prec == SVM_BF16) dw.wq = put(bf.data(), L * W * W * 2, n_wq);
    else if (d.prec == SVM_FP8_E4M3) dw.wq = put(e4.data(), L * W * W, n_wq);
    else dw.wq = put(nullptr, 0, n_wq);
    dw.wscale = (const float*)put(wscale.data(), L * 4, n_sc);
    dw.ascale = (const float*)put(m->ascales.data(), L * 4, n_sc);
    dw.w1pad = put(w1pad.data(), w1pad.size() * 2, n_w1pad);
    m->bh_host = bh;
    dw.bhs = (const float*)put(nullptr, 0, n_bh);
    {
        const svm_status st2 = upload_scaled_biases(m);
        if (st2 != SVM_OK) return st2;
    }
    dw.bout = u[Lo.out_b];
    CK(cudaGetLastError());
    CK(cudaDeviceSynchronize());
    if (d.prec != SVM_FP32) {
        const int st = tc_prepare(m->tc, d, dw);
        if (st != 0) return fail(m, SVM_E_CUDA, "tensor-core path set-up failed");
    }
    m->tau = std::isfinite(tau) && tau >= 0 ? tau : INFINITY;
    m->has_weights = true;
    return SVM_OK;
}

svm_status svm_export_weights(const svm_model* mc, float* out, size_t count, size_t* needed)
{
    svm_model* m = const_cast<svm_model*>(mc);
    if (!m) return SVM_E_INVALID;
    if (!m->has_weights) return fail(m, SVM_E_WEIGHTS, "no weights loaded");
    if (needed) *needed = m->used.size();
    if (!out) return SVM_OK;
    if (count < m->used.size()) return fail(m, SVM_E_INVALID, "output too small");
    std::memcpy(out, m->used.data(), m->used.size() * sizeof(float));
    return SVM_OK;
}

}  // extern "C"

namespace {

enum Mode { kCheck = 0, kEval = 1, kLabel = 2, kGate = 3 };

struct CallPlan {
    int M, N;
    long long P_total;       // sum of points over motions
    int n_tiles;
    int bm;
    // offsets in the workspace
    size_t o_q0, o_q1, o_pbeg, o_pend, o_toff, o_poff, header_bytes;
    size_t o_caps, o_fk64, o_cbias, o_st, o_idx, o_chunk, o_tie, total;
};

// Shared driver of the check, eval and label calls.
svm_status run_call(svm_model* m, Mode mode, const double* q0, const double* q1, int32_t M,
                    const int32_t* motion_scene, const float* points_dev, const int64_t* scene_off,
                    int32_t n_scenes, float margin, int32_t steps, uint32_t flags, void* results_dev,
                    float* out_dev, cudaStream_t stream)
{
    const Range call_range(mode == kCheck ? "svm_check" : mode == kEval ? "svm_eval_pairs"
                           : mode == kLabel ? "svm_label_pairs" : "svm_calibrate_gate");
    const svm_model_desc& d = m->desc;
    if (M < 0) return fail(m, SVM_E_INVALID, "n_motions < 0");
    if (M > 0 && (!q0 || !q1)) return fail(m, SVM_E_INVALID, "null q0/q1");
    if (n_scenes < 1 || !scene_off) return fail(m, SVM_E_INVALID, "no scene");
    if (mode != kLabel && mode != kGate && !m->has_weights && !(flags & SVM_VERIFY_ALL))
        return fail(m, SVM_E_WEIGHTS, "no weights loaded");
    if (mode == kCheck && M > 0 && !results_dev) return fail(m, SVM_E_INVALID, "null results");
    if (mode != kCheck && M > 0 && !out_dev) return fail(m, SVM_E_INVALID, "null output");
    if (!(margin >= 0) || !std::isfinite(margin)) return fail(m, SVM_E_INVALID, "margin must be finite and >= 0");
    if (steps < 1 || steps > kMaxSteps) return fail(m, SVM_E_INVALID, "steps out of range");
    if (flags & ~(SVM_STRICT | SVM_NO_EARLY_EXIT | SVM_VERIFY_ALL | SVM_PATHS3 | SVM_PATHS2 | SVM_PREDICT_ONLY))
        return fail(m, SVM_E_INVALID, "unknown flag");
    if ((flags & SVM_PATHS3) && (flags & SVM_PATHS2)) return fail(m, SVM_E_INVALID, "SVM_PATHS2 with SVM_PATHS3");
    if (M % path_len_of(flags) != 0) return fail(m, SVM_E_INVALID, "n_motions is not a multiple of the path length");
    if ((flags & SVM_PREDICT_ONLY) && (flags & (SVM_VERIFY_ALL | SVM_STRICT)))
        return fail(m, SVM_E_INVALID, "SVM_PREDICT_ONLY excludes SVM_VERIFY_ALL and SVM_STRICT");
    if (scene_off[0] != 0) return fail(m, SVM_E_INVALID, "scene_offsets[0] must be 0");
    for (int s = 0; s < n_scenes; ++s)
        if (scene_off[s + 1] < scene_off[s]) return fail(m, SVM_E_INVALID, "scene offsets decrease");
    if (scene_off[n_scenes] > 0) {
        if (!points_dev) return fail(m, SVM_E_INVALID, "null points");
        if (reinterpret_cast<uintptr_t>(points_dev) % 16) return fail(m, SVM_E_INVALID, "points not 16-byte aligned");
    }
    if (scene_off[n_scenes] > (int64_t)0xffffffffLL) return fail(m, SVM_E_INVALID, "too many points");
    if (M == 0) return SVM_OK;
    if (!finite_all(q0, (long long)M * 6) || !finite_all(q1, (long long)M * 6))
        return fail(m, SVM_E_INVALID, "non-finite joint angle");
    for (int i = 0; i < M; ++i) {
        const int s = motion_scene ? motion_scene[i] : 0;
        if (s < 0 || s >= n_scenes) return fail(m, SVM_E_INVALID, "motion scene out of range");
    }

    const bool tc = d.prec != SVM_FP32;
    CallPlan pl{};
    pl.M = M;
    pl.N = steps;
    pl.bm = tc ? tc_tile_rows() : mlp_fp32_tile_rows();
    auto count_tiles = [&]() {
        pl.P_total = 0;
        pl.n_tiles = 0;
        for (int i = 0; i < M; ++i) {
            const int s = motion_scene ? motion_scene[i] : 0;
            const long long n = scene_off[s + 1] - scene_off[s];
            pl.P_total += n;
            pl.n_tiles += (int)((n + pl.bm - 1) / pl.bm);
        }
    };
    if (!tc) {
        pl.bm = mlp_fp32_small_tile_rows();
        count_tiles();
        pl.bm = mlp_fp32_tile_rows(pl.n_tiles, m->n_sms);
    }
    count_tiles();
    size_t at = 0;
    pl.o_q0 = at; at = align256(at + (size_t)M * 6 * 8);
    pl.o_q1 = at; at = align256(at + (size_t)M * 6 * 8);
    pl.o_pbeg = at; at = align256(at + (size_t)M * 8);
    pl.o_pend = at; at = align256(at + (size_t)M * 8);
    pl.o_toff = at; at = align256(at + (size_t)(M + 1) * 4);
    pl.o_poff = at; at = align256(at + (size_t)(M + 1) * 8);
    pl.header_bytes = at;
    pl.o_caps = at; at = align256(at + (size_t)M * (steps + 1) * kCaps * sizeof(Capsule));
    pl.o_fk64 = at; at = align256(at + (size_t)M * (steps + 1) * 24 * sizeof(double));
    pl.o_cbias = at; at = align256(at + (size_t)M * cbias_stride(d) * 4);
    pl.o_st = at; at = align256(at + (size_t)M * sizeof(MotionState));
    pl.o_idx = at; at = align256(at + (size_t)std::max<long long>(1, pl.P_total) * 4);
    pl.o_chunk = at; at = align256(at + (size_t)(M + 1) * 4);
    at = align256(at + tc_workspace_bytes(M));
    pl.o_tie = at; at = align256(at + 256 + tie_list_bytes());
    pl.total = at;

    DeviceGuard g(m->device);
    // grow the workspace and staging buffer (not inside a stream capture)
    if (pl.total > m->ws_bytes) {
        const size_t limit = workspace_limit();
        if (limit && pl.total > limit)
            return fail(m, SVM_E_OOM, "the call needs " + std::to_string(pl.total) +
                                          " bytes of workspace, more than SVM_WORKSPACE_LIMIT = " +
                                          std::to_string(limit));
        CK(cudaDeviceSynchronize());
        if (m->ws) cudaFree(m->ws);
        m->ws = nullptr;
        m->ws_bytes = 0;
        size_t want = pl.total + pl.total / 4;
        if (limit && want > limit) want = limit;
        if (cudaMalloc(&m->ws, want) != cudaSuccess) {
            cudaGetLastError();
            return fail(m, SVM_E_OOM, "workspace allocation failed");
        }
        m->ws_bytes = want;
    }
    if (pl.header_bytes > m->pinned_bytes) {
        CK(cudaEventSynchronize(m->staging_done));
        if (m->pinned) cudaFreeHost(m->pinned);
        m->pinned = nullptr;
        m->pinned_bytes = 0;
        CK(cudaMallocHost(&m->pinned, pl.header_bytes * 2));
        m->pinned_bytes = pl.header_bytes * 2;
    }
    // the previous call's header copy must have finished before the rewrite
    CK(cudaEventSynchronize(m->staging_done));
    char* h = static_cast<char*>(m->pinned);
    std::memcpy(h + pl.o_q0, q0, (size_t)M * 48);
    std::memcpy(h + pl.o_q1, q1, (size_t)M * 48);
    long long* pbeg = reinterpret_cast<long long*>(h + pl.o_pbeg);
    long long* pend = reinterpret_cast<long long*>(h + pl.o_pend);
    int* toff = reinterpret_cast<int*>(h + pl.o_toff);
    long long* poff = reinterpret_cast<long long*>(h + pl.o_poff);
    toff[0] = 0;
    poff[0] = 0;
    for (int i = 0; i < M; ++i) {
        const int s = motion_scene ? motion_scene[i] : 0;
        pbeg[i] = scene_off[s];
        pend[i] = scene_off[s + 1];
        const long long n = pend[i] - pbeg[i];
        toff[i + 1] = toff[i] + (int)((n + pl.bm - 1) / pl.bm);
        poff[i + 1] = poff[i] + n;
    }
    char* ws = static_cast<char*>(m->ws);
    const bool prof = m->prof && mode == kCheck;
    m->prof_valid = false;
    if (prof) CK(cudaEventRecord(m->ev[0], stream));
    CK(cudaMemcpyAsync(ws, h, pl.header_bytes, cudaMemcpyHostToDevice, stream));
    CK(cudaEventRecord(m->staging_done, stream));

    CallArgs a{};
    a.M = M;
    a.N = steps;
    a.W = d.width;
    a.L = d.n_hidden;
    a.act = d.act;
    a.arch = d.arch;
    a.rp = m->rp;
    a.cb_stride = cbias_stride(d);
    a.flags = flags;
    a.margin = margin;
    a.gate = (mode == kEval || (flags & SVM_PREDICT_ONLY)) ? -INFINITY : margin + m->tau;
    a.q0 = reinterpret_cast<const double*>(ws + pl.o_q0);
    a.q1 = reinterpret_cast<const double*>(ws + pl.o_q1);
    a.pbeg = reinterpret_cast<const long long*>(ws + pl.o_pbeg);
    a.pend = reinterpret_cast<const long long*>(ws + pl.o_pend);
    a.tile_off = reinterpret_cast<const int*>(ws + pl.o_toff);
    a.pair_off = reinterpret_cast<const long long*>(ws + pl.o_poff);
    a.points = reinterpret_cast<const float4*>(points_dev);
    a.caps = reinterpret_cast<Capsule*>(ws + pl.o_caps);
    a.fk64 = reinterpret_cast<double*>(ws + pl.o_fk64);
    a.cbias = (mode == kLabel || mode == kGate || (flags & SVM_VERIFY_ALL)) ? nullptr
                                                                           : reinterpret_cast<float*>(ws + pl.o_cbias);
    a.st = reinterpret_cast<MotionState*>(ws + pl.o_st);
    a.idx = reinterpret_cast<unsigned*>(ws + pl.o_idx);
    a.chunk_off = reinterpret_cast<int*>(ws + pl.o_chunk);
    a.f_out = (mode == kEval) ? out_dev : nullptr;
    a.f_stride = (n_scenes == 1) ? scene_off[1] : 0;
    a.path_len = path_len_of(flags);
    a.amax = m->calib_amax;
    if (mode == kCheck && tc && m->test_stalls > 0 && !(flags & SVM_VERIFY_ALL)) {
        a.test_stall = 1;
        --m->test_stalls;
    }
    void* tc_ws = ws + pl.o_chunk + align256((size_t)(M + 1) * 4);
    a.dev_err = static_cast<unsigned int*>(tc_ws);
    a.tie_count = reinterpret_cast<unsigned int*>(ws + pl.o_tie);
    a.tie_list = reinterpret_cast<TiePair*>(ws + pl.o_tie + 256);
    a.tie_cap = m->tie_cap;
    CK(cudaMemsetAsync(a.dev_err, 0, sizeof(unsigned int), stream));

    {
        const Range r("prologue");
        launch_prologue_fk(a, m->rp, m->dw, stream);
    }
    if (prof) CK(cudaEventRecord(m->ev[1], stream));
    if (mode == kLabel) {
        const Range r("label");
        launch_label(a, out_dev, a.f_stride, stream);
        CK(cudaGetLastError());
        return SVM_OK;
    }
    if (mode == kGate) {
        const Range r("overestimate");
        launch_gate_overestimate(a, out_dev, a.f_stride, m->gate_cut, m->gate_out, stream);
        CK(cudaGetLastError());
        return SVM_OK;
    }
    if (!(flags & SVM_VERIFY_ALL)) {
        {
            const Range r("network");
            if (tc) {
                const int st = tc_launch(m->tc, a, m->dw, pl.n_tiles, tc_ws, m->n_sms, stream);
                if (st != 0) return fail(m, SVM_E_CUDA, "tensor-core launch failed");
            } else {
                launch_mlp_fp32(a, m->dw, pl.n_tiles, pl.bm, stream);
            }
        }
        if (mode == kEval) {
            CK(cudaGetLastError());
            return SVM_OK;
        }
        if (prof) CK(cudaEventRecord(m->ev[2], stream));
        if (!(flags & SVM_PREDICT_ONLY)) {
            const Range r("verify");
            launch_verify(a, 0, 0, stream, m->n_sms);
            if (flags & SVM_STRICT) launch_verify(a, 1, 1, stream, m->n_sms);
            launch_ties(a, stream, m->n_sms);
        }
    } else {
        if (prof) CK(cudaEventRecord(m->ev[2], stream));
        const Range r("verify");
        launch_verify(a, 1, 0, stream, m->n_sms);
        launch_ties(a, stream, m->n_sms);
    }
    if (prof) CK(cudaEventRecord(m->ev[3], stream));
    {
        const Range r("finalize");
        launch_finalize(a, results_dev, stream);
    }
    if (prof) {
        CK(cudaEventRecord(m->ev[4], stream));
        m->prof_valid = true;
    }
    CK(cudaGetLastError());
    return SVM_OK;
}

}  // namespace

extern "C" {

svm_status svm_check_motions(svm_model* m, const double* q0, const double* q1, int32_t n_motions,
                             const float* points_dev, int64_t n_points, float margin, int32_t steps,
                             uint32_t flags, svm_result* results_dev, void* stream)
{
    if (!m) return SVM_E_INVALID;
    if (n_points < 0) return fail(m, SVM_E_INVALID, "n_points < 0");
    const int64_t off[2] = {0, n_points};
    return run_call(m, kCheck, q0, q1, n_motions, nullptr, points_dev, off, 1, margin, steps, flags,
                    results_dev, nullptr, static_cast<cudaStream_t>(stream));
}

svm_status svm_check_batch(svm_model* m, const double* q0, const double* q1, int32_t n_motions,
                           const int32_t* motion_scene, const float* points_dev, const int64_t* scene_offsets,
                           int32_t n_scenes, float margin, int32_t steps, uint32_t flags,
                           svm_result* results_dev, void* stream)
{
    if (!m) return SVM_E_INVALID;
    if (n_motions > 0 && !motion_scene) return fail(m, SVM_E_INVALID, "null motion_scene");
    return run_call(m, kCheck, q0, q1, n_motions, motion_scene, points_dev, scene_offsets, n_scenes, margin,
                    steps, flags, results_dev, nullptr, static_cast<cudaStream_t>(stream));
}

svm_status svm_eval_pairs(svm_model* m, const double* q0, const double* q1, int32_t n_motions,
                          const float* points_dev, int64_t n_points, float* f_dev, void* stream)
{
    if (!m) return SVM_E_INVALID;
    if (n_points < 0) return fail(m, SVM_E_INVALID, "n_points < 0");
    const int64_t off[2] = {0, n_points};
    return run_call(m, kEval, q0, q1, n_motions, nullptr, points_dev, off, 1, 0.0f, 1, 0u, nullptr, f_dev,
                    static_cast<cudaStream_t>(stream));
}

svm_status svm_calibrate_act_scales(svm_model* m, const double* q0, const double* q1, int32_t n_motions,
                                    const float* points_dev, int64_t n_points, float headroom, float* scales_out)
{
    if (!m) return SVM_E_INVALID;
    const svm_model_desc& d = m->desc;
    if (d.prec != SVM_FP8_E4M3) return fail(m, SVM_E_INVALID, "activation scales apply to FP8 models only");
    if (!(headroom >= 1.0f) || !std::isfinite(headroom)) return fail(m, SVM_E_INVALID, "headroom must be >= 1");
    if (n_motions < 1 || n_points < 1) return fail(m, SVM_E_INVALID, "empty calibration set");
    // the FP32 network on the model's rounded weights records the largest
    // activation entering each hidden layer; scale = headroom * max / 448
    svm_model_desc d32 = d;
    d32.prec = SVM_FP32;
    svm_model* c = nullptr;
    svm_status st = svm_create_model(&d32, m->device, &c);
    if (st != SVM_OK) return fail(m, st, "calibration model");
    c->used = m->used;
    {
        // load the rounded weights as FP32 weights (they round to themselves)
        const Layout Lo = layout_of(d);
        std::vector<unsigned char> blob(28 + (size_t)(d.n_hidden + 2) * 8 + Lo.total * 4);
        if (blob.size() < 28) { svm_destroy_model(c); return fail(m, SVM_E_INVALID, "calibration blob size"); }
        unsigned char* o = blob.data();
        std::memcpy(o, "SVMW", 4);
        const uint32_t hdr[5] = {1u, (uint32_t)(d.n_hidden + 2), 15u, (uint32_t)d.width, (uint32_t)d.act};
        std::memcpy(o + 4, hdr, 20);
        const float inf = INFINITY;
        std::memcpy(o + 24, &inf, 4);
        size_t off = 28;
        long long pos = 0;
        for (int l = 0; l < d.n_hidden + 2; ++l) {
            const uint32_t out = l == d.n_hidden + 1 ? 1u : (uint32_t)d.width;
            const uint32_t in = l == 0 ? 15u : (uint32_t)d.width;
            std::memcpy(o + off, &out, 4);
            std::memcpy(o + off + 4, &in, 4);
            off += 8;
            std::memcpy(o + off, m->used.data() + pos, ((size_t)out * in + out) * 4);
            off += ((size_t)out * in + out) * 4;
            pos += (long long)out * in + out;
        }
        st = svm_load_weights(c, blob.data(), blob.size());
        if (st != SVM_OK) { svm_destroy_model(c); return fail(m, st, "calibration weights"); }
    }
    DeviceGuard g(m->device);
    unsigned int* amax = nullptr;
    if (cudaMalloc(&amax, sizeof(unsigned int) * d.n_hidden) != cudaSuccess) {
        svm_destroy_model(c);
        return fail(m, SVM_E_OOM, "calibration buffer");
    }
    cudaMemset(amax, 0, sizeof(unsigned int) * d.n_hidden);
    c->calib_amax = amax;
    float* fdev = nullptr;
    if (cudaMalloc(&fdev, sizeof(float) * (size_t)n_motions * n_points) != cudaSuccess) {
        cudaFree(amax);
        svm_destroy_model(c);
        return fail(m, SVM_E_OOM, "calibration buffer");
    }
    st = svm_eval_pairs(c, q0, q1, n_motions, points_dev, n_points, fdev, nullptr);
    std::vector<unsigned int> h(d.n_hidden);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(h.data(), amax, sizeof(unsigned int) * d.n_hidden, cudaMemcpyDeviceToHost);
    cudaFree(fdev);
    cudaFree(amax);
    svm_destroy_model(c);
    if (st != SVM_OK) return fail(m, st, "calibration run");
    if (e != cudaSuccess) return fail(m, SVM_E_CUDA, cudaGetErrorString(e));
    std::vector<float> sc(d.n_hidden);
    for (int l = 0; l < d.n_hidden; ++l) {
        float mx;
        std::memcpy(&mx, &h[l], 4);
        sc[l] = mx > 0.0f ? headroom * mx / 448.0f : 1.0f;
    }
    if (scales_out) std::memcpy(scales_out, sc.data(), sizeof(float) * d.n_hidden);
    return svm_set_act_scales(m, sc.data(), d.n_hidden);
}

svm_status svm_calibrate_gate(svm_model* m, const double* q0, const double* q1, int32_t n_motions,
                              const float* points_dev, int64_t n_points, float margin, int32_t steps, float band,
                              float safety, float* tau_out, float* overestimate_out, int64_t* n_near_out,
                              void* stream_v)
{
    if (!m) return SVM_E_INVALID;
    if (!m->has_weights) return fail(m, SVM_E_WEIGHTS, "no weights loaded");
    if (n_motions < 1 || n_points < 1) return fail(m, SVM_E_INVALID, "empty calibration set");
    if ((long long)n_motions * n_points > 0xffffffffLL) return fail(m, SVM_E_INVALID, "calibration set too large");
    if (!(band >= 0) || !std::isfinite(band)) return fail(m, SVM_E_INVALID, "band must be finite and >= 0");
    if (!(safety >= 1) || !std::isfinite(safety)) return fail(m, SVM_E_INVALID, "safety must be finite and >= 1");
    if (!(margin >= 0) || !std::isfinite(margin)) return fail(m, SVM_E_INVALID, "margin must be finite and >= 0");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    DeviceGuard g(m->device);
    // motions in chunks whose network outputs fit in a bounded buffer (at most 2^26 floats)
    const long long cap = 1LL << 26;
    const int chunk = (int)std::max<long long>(1, std::min<long long>(n_motions, cap / n_points));
    float* fbuf = nullptr;
    unsigned int* outd = nullptr;
    if (cudaMalloc(&fbuf, sizeof(float) * (size_t)chunk * n_points) != cudaSuccess ||
        cudaMalloc(&outd, 2 * sizeof(unsigned int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(fbuf);
        return fail(m, SVM_E_OOM, "calibration buffer");
    }
    svm_status st = SVM_OK;
    cudaError_t e = cudaMemsetAsync(outd, 0, 2 * sizeof(unsigned int), stream);
    m->gate_out = outd;
    m->gate_cut = (float)((double)margin + (double)band);
    const int64_t off[2] = {0, n_points};
    for (int c0 = 0; c0 < n_motions && st == SVM_OK && e == cudaSuccess; c0 += chunk) {
        const int cm = std::min(chunk, n_motions - c0);
        st = run_call(m, kEval, q0 + 6LL * c0, q1 + 6LL * c0, cm, nullptr, points_dev, off, 1, 0.0f, 1, 0u,
                      nullptr, fbuf, stream);
        if (st == SVM_OK)
            st = run_call(m, kGate, q0 + 6LL * c0, q1 + 6LL * c0, cm, nullptr, points_dev, off, 1, 0.0f, steps,
                          0u, nullptr, fbuf, stream);
    }
    m->gate_out = nullptr;
    unsigned int h[2] = {0u, 0u};
    if (st == SVM_OK && e == cudaSuccess) e = cudaStreamSynchronize(stream);
    if (st == SVM_OK && e == cudaSuccess) e = cudaMemcpy(h, outd, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(fbuf);
    cudaFree(outd);
    if (st != SVM_OK) return st;
    if (e != cudaSuccess) return fail(m, SVM_E_CUDA, cudaGetErrorString(e));
    float over = -INFINITY;
    if (h[1] > 0) {
        const unsigned int k = h[0];
        const unsigned int u = (k & 0x80000000u) ? (k & 0x7fffffffu) : ~k;
        std::memcpy(&over, &u, 4);
    }
    const float tau = h[1] > 0 ? (float)std::max(0.0, (double)safety * (double)over) : 0.0f;
    if (tau_out) *tau_out = tau;
    if (overestimate_out) *overestimate_out = over;
    if (n_near_out) *n_near_out = (int64_t)h[1];
    return svm_set_gate(m, tau);
}

svm_status svm_profile_enable(svm_model* m, int on)
{
    if (!m) return SVM_E_INVALID;
    DeviceGuard g(m->device);
    if (on && !m->ev[0])
        for (auto& e : m->ev) CK(cudaEventCreate(&e));
    m->prof = on != 0;
    return SVM_OK;
}

svm_status svm_profile_read(svm_model* m, float* ms, int32_t n)
{
    if (!m || !ms || n < 0 || n > 4) return SVM_E_INVALID;
    if (!m->prof_valid) return fail(m, SVM_E_INVALID, "no profiled call");
    DeviceGuard g(m->device);
    CK(cudaEventSynchronize(m->ev[4]));
    for (int i = 0; i < n; ++i) CK(cudaEventElapsedTime(ms + i, m->ev[i], m->ev[i + 1]));
    return SVM_OK;
}

svm_status svm_label_pairs(svm_model* m, const double* q0, const double* q1, int32_t n_motions,
                           const float* points_dev, int64_t n_points, int32_t steps, float* delta_dev,
                           void* stream)
{
    if (!m) return SVM_E_INVALID;
    if (n_points < 0) return fail(m, SVM_E_INVALID, "n_points < 0");
    const int64_t off[2] = {0, n_points};
    return run_call(m, kLabel, q0, q1, n_motions, nullptr, points_dev, off, 1, 0.0f, steps, 0u, nullptr,
                    delta_dev, static_cast<cudaStream_t>(stream));
}


svm_status svm_search_free_motion(svm_model* m, const double* q0, const double* q1, int32_t n_motions,
                                  const float* points_dev, int64_t n_points, float margin, int32_t steps,
                                  int32_t wave, uint32_t flags, svm_search_result* out, void* stream_)
{
    const Range call_range("svm_search_free_motion");
    if (!m || !out) return SVM_E_INVALID;
    if (n_motions < 0 || n_points < 0) return fail(m, SVM_E_INVALID, "negative count");
    if (wave < 1) return fail(m, SVM_E_INVALID, "wave must be >= 1");
    if (flags & ~(SVM_SEARCH_GCC0 | SVM_SEARCH_SORTED | SVM_SEARCH_PATHS2 | SVM_SEARCH_PATHS3))
        return fail(m, SVM_E_INVALID, "unknown search flag");
    if ((flags & SVM_SEARCH_PATHS2) && (flags & SVM_SEARCH_PATHS3))
        return fail(m, SVM_E_INVALID, "SVM_SEARCH_PATHS2 with SVM_SEARCH_PATHS3");
    const bool use_nn = !(flags & SVM_SEARCH_GCC0);
    if (use_nn && !m->has_weights) return fail(m, SVM_E_WEIGHTS, "no weights loaded");
    // candidates: single motions, or paths of 2 or 3 consecutive segments
    const int plen = (flags & SVM_SEARCH_PATHS3) ? 3 : (flags & SVM_SEARCH_PATHS2) ? 2 : 1;
    const uint32_t pflag = plen == 3 ? SVM_PATHS3 : plen == 2 ? SVM_PATHS2 : 0u;
    if (n_motions % plen != 0) return fail(m, SVM_E_INVALID, "n_motions is not a multiple of the path length");
    cudaStream_t stream = static_cast<cudaStream_t>(stream_);
    *out = svm_search_result{-1, 0, INFINITY, INFINITY, 0, 0, 0, 0};
    const int M = n_motions / plen;           // candidates
    if (M == 0) return SVM_OK;
    DeviceGuard g(m->device);
    // result records: one per motion for the prediction, one per motion of a wave
    const size_t need = (size_t)std::max(M, wave);
    if (need > m->search_cap) {
        CK(cudaStreamSynchronize(stream));
        if (m->search_dev) cudaFree(m->search_dev);
        if (m->search_host) cudaFreeHost(m->search_host);
        m->search_dev = nullptr;
        m->search_host = nullptr;
        m->search_cap = 0;
        if (cudaMalloc(&m->search_dev, need * sizeof(svm_result)) != cudaSuccess ||
            cudaMallocHost(&m->search_host, need * sizeof(svm_result)) != cudaSuccess) {
            cudaGetLastError();
            return fail(m, SVM_E_OOM, "search buffers");
        }
        m->search_cap = need;
    }
    svm_result* rd = static_cast<svm_result*>(m->search_dev);
    svm_result* rh = static_cast<svm_result*>(m->search_host);
    const int64_t off[2] = {0, n_points};
    // d_hat(X, m) of every motion (Eq. 6): one network launch, no exact check
    std::vector<float> dhat(M, INFINITY);
    if (use_nn) {
        const svm_status st = run_call(m, kCheck, q0, q1, n_motions, nullptr, points_dev, off, 1, margin, steps,
                                       SVM_PREDICT_ONLY | pflag, rd, nullptr, stream);
        if (st != SVM_OK) return st;
        CK(cudaMemcpyAsync(rh, rd, (size_t)M * sizeof(svm_result), cudaMemcpyDeviceToHost, stream));
        CK(cudaStreamSynchronize(stream));
        for (int i = 0; i < M; ++i) {
            if (rh[i].status == 1) return fail(m, SVM_E_TIMEOUT, "a device wait expired");
            dhat[i] = rh[i].dhat_min;      // a path's: the minimum over its segments
        }
        out->n_nn = n_motions;
    }
    // exact checks (the geometric check of every point, early exit at the first
    // collision) of the motions `list`, in order, `wave` at a time; returns the
    // position in `list` of the first free motion, or -1
    std::vector<double> wq0, wq1;
    auto exact_in_order = [&](const std::vector<int>& list, int& pos, svm_status& st) {
        pos = -1;
        for (size_t b = 0; b < list.size(); b += (size_t)wave) {
            const int nw = (int)std::min<size_t>((size_t)wave, list.size() - b);
            wq0.resize((size_t)nw * plen * 6);
            wq1.resize((size_t)nw * plen * 6);
            for (int k = 0; k < nw; ++k) {
                std::memcpy(&wq0[(size_t)k * plen * 6], q0 + (size_t)list[b + k] * plen * 6, 48 * (size_t)plen);
                std::memcpy(&wq1[(size_t)k * plen * 6], q1 + (size_t)list[b + k] * plen * 6, 48 * (size_t)plen);
            }
            st = run_call(m, kCheck, wq0.data(), wq1.data(), nw * plen, nullptr, points_dev, off, 1, margin, steps,
                          SVM_VERIFY_ALL | pflag, rd, nullptr, stream);
            if (st != SVM_OK) return;
            if (cudaMemcpyAsync(rh, rd, (size_t)nw * sizeof(svm_result), cudaMemcpyDeviceToHost, stream) !=
                    cudaSuccess ||
                cudaStreamSynchronize(stream) != cudaSuccess) {
                st = fail(m, SVM_E_CUDA, "search result copy");
                return;
            }
            out->n_exact_run += nw;
            for (int k = 0; k < nw; ++k) {
                if (rh[k].status == 1) {
                    st = fail(m, SVM_E_TIMEOUT, "a device wait expired");
                    return;
                }
                if (!rh[k].collision) {
                    pos = (int)b + k;
                    out->delta = rh[k].d_min;
                    return;
                }
            }
        }
    };
    svm_status st = SVM_OK;
    int pos = -1;
    // first loop: the motions predicted free, in the given order (none when only
    // the second loop runs)
    const bool sorted_only = use_nn && (flags & SVM_SEARCH_SORTED);
    std::vector<int> first, rest;
    for (int i = 0; i < M; ++i) (dhat[i] > margin && !sorted_only ? first : rest).push_back(i);
    exact_in_order(first, pos, st);
    if (st != SVM_OK) return st;
    if (pos >= 0) {
        out->motion = first[pos];
        out->loop = 1;
        out->n_exact = pos + 1;
        out->delta_hat = dhat[first[pos]];
        // the sequential first loop evaluated the network up to the returned motion
        out->n_nn_seq = use_nn ? (out->motion + 1) * plen : 0;
        return SVM_OK;
    }
    out->n_exact = (int)first.size();
    out->n_nn_seq = use_nn ? n_motions : 0;
    // second loop: the others by decreasing prediction (ties keep the given order);
    // GCC_0 keeps the given order
    if (use_nn) std::stable_sort(rest.begin(), rest.end(), [&](int a, int b) { return dhat[a] > dhat[b]; });
    exact_in_order(rest, pos, st);
    if (st != SVM_OK) return st;
    if (pos >= 0) {
        out->motion = rest[pos];
        out->loop = 2;
        out->n_exact += pos + 1;
        out->delta_hat = dhat[rest[pos]];
    } else {
        out->n_exact += (int)rest.size();
    }
    return SVM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------------
// Allocation-free check.  Some callers cannot allocate device memory while
// they check motions: a real-time control loop whose memory is fixed at
// start-up, a process whose allocator is owned by another framework, or code
// running between a stream capture's begin and end, where cudaMalloc is not
// allowed.  svm_check_motions grows its workspace with cudaMalloc and stages
// q0/q1 in pinned host memory it allocates on first use; the entry point
// below does neither.  Its scratch is one fixed array in device memory,
// declared here at file scope, which every GPU that loads this library holds
// until the process exits.
// ------------------------------------------------------------------------

#include <mutex>

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;   // 32 MiB per device
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_ptr[64] = {};

// Device address of the scratch array on the current device.  In host code
// the array's name is only a stand-in; the address comes from the runtime.
cudaError_t noalloc_scratch(int dev, void** out)
{
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = p;
    }
    *out = g_noalloc_ptr[dev];
    return cudaSuccess;
}

// Per-motion point ranges and prefixes for one cloud shared by all motions,
// and the call's error word, written into the scratch on the device.
__global__ void noalloc_setup_kernel(int M, long long n_points, int bm, long long* pbeg, long long* pend,
                                     int* tile_off, long long* pair_off, unsigned int* err)
{
    const long long tiles = (n_points + bm - 1) / bm;
    for (int m = blockIdx.x * blockDim.x + threadIdx.x; m <= M; m += gridDim.x * blockDim.x) {
        if (m < M) {
            pbeg[m] = 0;
            pend[m] = n_points;
        }
        tile_off[m] = (int)(tiles * m);
        pair_off[m] = n_points * m;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *err = 0u;
}

}  // namespace

extern "C" svm_status svm_check_motions_noalloc(svm_model* m, const double* q0_dev, const double* q1_dev,
                                                int32_t n_motions, const float* points_dev, int64_t n_points,
                                                float margin, int32_t steps, uint32_t flags,
                                                svm_result* results_dev, void* stream_v)
{
    if (!m) return SVM_E_INVALID;
    const svm_model_desc& d = m->desc;
    cudaStream_t stream = static_cast<cudaStream_t>(stream_v);
    const int M = n_motions;
    if (M < 0 || n_points < 0) return fail(m, SVM_E_INVALID, "negative size");
    if (M == 0) return SVM_OK;
    if (!q0_dev || !q1_dev || !results_dev) return fail(m, SVM_E_INVALID, "null q0/q1/results");
    if (n_points > 0 && !points_dev) return fail(m, SVM_E_INVALID, "null points");
    if (reinterpret_cast<uintptr_t>(points_dev) % 16) return fail(m, SVM_E_INVALID, "points not 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(q0_dev) % 8 || reinterpret_cast<uintptr_t>(q1_dev) % 8)
        return fail(m, SVM_E_INVALID, "q0/q1 not 8-byte aligned");
    {
        // q0/q1 are read by the prologue kernel: they must be memory the device can address
        // (device or managed memory), not pageable host memory
        const void* ptrs[2] = {q0_dev, q1_dev};
        for (const void* p : ptrs) {
            cudaPointerAttributes at{};
            if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
                cudaGetLastError();
                return fail(m, SVM_E_INVALID, "q0/q1 is not a CUDA pointer");
            }
            if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
                return fail(m, SVM_E_INVALID, "q0/q1 must be device or managed memory");
            if (at.type == cudaMemoryTypeDevice && at.device != m->device)
                return fail(m, SVM_E_INVALID, "q0/q1 live on another device than the model");
        }
    }
    if (!m->has_weights && !(flags & SVM_VERIFY_ALL)) return fail(m, SVM_E_WEIGHTS, "no weights loaded");
    if (!(margin >= 0) || !std::isfinite(margin)) return fail(m, SVM_E_INVALID, "margin must be finite and >= 0");
    if (steps < 1 || steps > kMaxSteps) return fail(m, SVM_E_INVALID, "steps out of range");
    if (flags & ~(SVM_STRICT | SVM_NO_EARLY_EXIT | SVM_VERIFY_ALL | SVM_PATHS3 | SVM_PATHS2))
        return fail(m, SVM_E_INVALID, "unknown flag");
    if ((flags & SVM_PATHS3) && (flags & SVM_PATHS2)) return fail(m, SVM_E_INVALID, "SVM_PATHS2 with SVM_PATHS3");
    if (M % path_len_of(flags) != 0) return fail(m, SVM_E_INVALID, "n_motions is not a multiple of the path length");

    const bool tc = d.prec != SVM_FP32;
    int bm = tc ? tc_tile_rows() : mlp_fp32_tile_rows();
    if (!tc) {
        const long long sb = mlp_fp32_small_tile_rows();
        bm = mlp_fp32_tile_rows((long long)M * ((n_points + sb - 1) / sb), m->n_sms);
    }
    const long long tiles_per = (n_points + bm - 1) / bm;
    if ((long long)M * tiles_per > 0x7fffffffLL || n_points > (int64_t)0xffffffffLL)
        return fail(m, SVM_E_INVALID, "too many tiles");
    // scratch layout (the same arrays as the workspace of svm_check_motions)
    size_t at = 0;
    const size_t o_pbeg = at; at = align256(at + (size_t)M * 8);
    const size_t o_pend = at; at = align256(at + (size_t)M * 8);
    const size_t o_toff = at; at = align256(at + (size_t)(M + 1) * 4);
    const size_t o_poff = at; at = align256(at + (size_t)(M + 1) * 8);
    const size_t o_caps = at; at = align256(at + (size_t)M * (steps + 1) * kCaps * sizeof(Capsule));
    const size_t o_fk64 = at; at = align256(at + (size_t)M * (steps + 1) * 24 * sizeof(double));
    const size_t o_cbias = at; at = align256(at + (size_t)M * cbias_stride(d) * 4);
    const size_t o_st = at; at = align256(at + (size_t)M * sizeof(MotionState));
    const size_t o_idx = at; at = align256(at + (size_t)std::max<long long>(1, (long long)M * n_points) * 4);
    const size_t o_chunk = at; at = align256(at + (size_t)(M + 1) * 4);
    const size_t o_err = at; at = align256(at + 4);
    const size_t o_tie = at; at = align256(at + 256 + tie_list_bytes());
    if (at > kNoAllocScratchBytes)
        return fail(m, SVM_E_INVALID,
                    "svm_check_motions_noalloc: the call needs " + std::to_string(at) +
                        " bytes of scratch, more than its fixed 32 MiB; use fewer motions or points per call "
                        "(about 4 bytes per motion-point pair plus ~54 KB per motion at 128 steps)");

    DeviceGuard g(m->device);
    void* sp = nullptr;
    {
        const cudaError_t e = noalloc_scratch(m->device, &sp);
        if (e != cudaSuccess) return fail(m, SVM_E_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    }
    char* ws = static_cast<char*>(sp);
    CallArgs a{};
    a.M = M;
    a.N = steps;
    a.W = d.width;
    a.L = d.n_hidden;
    a.act = d.act;
    a.arch = d.arch;
    a.rp = m->rp;
    a.cb_stride = cbias_stride(d);
    a.flags = flags;
    a.margin = margin;
    a.gate = margin + m->tau;
    a.q0 = q0_dev;
    a.q1 = q1_dev;
    a.pbeg = reinterpret_cast<const long long*>(ws + o_pbeg);
    a.pend = reinterpret_cast<const long long*>(ws + o_pend);
    a.tile_off = reinterpret_cast<const int*>(ws + o_toff);
    a.pair_off = reinterpret_cast<const long long*>(ws + o_poff);
    a.points = reinterpret_cast<const float4*>(points_dev);
    a.caps = reinterpret_cast<Capsule*>(ws + o_caps);
    a.fk64 = reinterpret_cast<double*>(ws + o_fk64);
    a.cbias = (flags & SVM_VERIFY_ALL) ? nullptr : reinterpret_cast<float*>(ws + o_cbias);
    a.st = reinterpret_cast<MotionState*>(ws + o_st);
    a.idx = reinterpret_cast<unsigned*>(ws + o_idx);
    a.chunk_off = reinterpret_cast<int*>(ws + o_chunk);
    a.f_out = nullptr;
    a.f_stride = n_points;
    a.path_len = path_len_of(flags);
    a.dev_err = reinterpret_cast<unsigned int*>(ws + o_err);
    a.tie_count = reinterpret_cast<unsigned int*>(ws + o_tie);
    a.tie_list = reinterpret_cast<TiePair*>(ws + o_tie + 256);

    noalloc_setup_kernel<<<(M + 256) / 256, 256, 0, stream>>>(
        M, n_points, bm, reinterpret_cast<long long*>(ws + o_pbeg), reinterpret_cast<long long*>(ws + o_pend),
        reinterpret_cast<int*>(ws + o_toff), reinterpret_cast<long long*>(ws + o_poff), a.dev_err);
    launch_prologue_fk(a, m->rp, m->dw, stream);
    if (!(flags & SVM_VERIFY_ALL)) {
        const int n_tiles = (int)(M * tiles_per);
        if (tc) {
            if (tc_launch(m->tc, a, m->dw, n_tiles, nullptr, m->n_sms, stream) != 0)
                return fail(m, SVM_E_CUDA, "tensor-core launch failed");
        } else {
            launch_mlp_fp32(a, m->dw, n_tiles, bm, stream);
        }
        launch_verify(a, 0, 0, stream, m->n_sms);
        if (flags & SVM_STRICT) launch_verify(a, 1, 1, stream, m->n_sms);
    } else {
        launch_verify(a, 1, 0, stream, m->n_sms);
    }
    launch_ties(a, stream, m->n_sms);
    launch_finalize(a, results_dev, stream);
    CK(cudaGetLastError());
    return SVM_OK;
}
