// weights.cu -- device-side rounding of the network weights to the model
// precision, done once at load time with the GPU's own conversions:
// bfloat16 round-to-nearest-even (cvt.rn.bf16.f32) and FP8 E4M3
// round-to-nearest-even with saturation (cvt.rn.satfinite.e4m3x2.f32).
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include "svm_internal.cuh"

namespace svm {

namespace {

__global__ void quantize_bf16_kernel(const float* in, uint16_t* out, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const __nv_bfloat16 b = __float2bfloat16_rn(in[i]);
        out[i] = *reinterpret_cast<const uint16_t*>(&b);
    }
}

__global__ void round_bf16_kernel(float* v, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        v[i] = __bfloat162float(__float2bfloat16_rn(v[i]));
}

// q = e4m3(w / scale), deq = float(q) * scale
__global__ void quantize_e4m3_kernel(const float* in, uint8_t* out, float* deq, long long n, float scale)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        const float t = in[i] / scale;
        const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(t, __NV_SATFINITE, __NV_E4M3);
        out[i] = q;
        const __half_raw hr = __nv_cvt_fp8_to_halfraw(q, __NV_E4M3);
        deq[i] = __half2float(__half(hr)) * scale;
    }
}

// out[b][c][r] = in[b][r][c]
__global__ void transpose_kernel(const float* in, float* out, int rows, int cols)
{
    __shared__ float t[32][33];
    const long long b = blockIdx.z;
    const float* src = in + b * rows * cols;
    float* dst = out + b * rows * cols;
    const int c0 = blockIdx.x * 32, r0 = blockIdx.y * 32;
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int r = r0 + i, c = c0 + threadIdx.x;
        if (r < rows && c < cols) t[i][threadIdx.x] = src[(long long)r * cols + c];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += blockDim.y) {
        const int c = c0 + i, r = r0 + threadIdx.x;
        if (r < rows && c < cols) dst[(long long)c * rows + r] = t[threadIdx.x][i];
    }
}

int grid_for(long long n) {
    long long g = (n + 255) / 256;
    return (int)(g > 4096 ? 4096 : (g < 1 ? 1 : g));
}

}  // namespace

void launch_quantize_bf16(const float* in, uint16_t* out, long long n, cudaStream_t s)
{
    if (n > 0) quantize_bf16_kernel<<<grid_for(n), 256, 0, s>>>(in, out, n);
}

void launch_round_bf16(float* inout, long long n, cudaStream_t s)
{
    if (n > 0) round_bf16_kernel<<<grid_for(n), 256, 0, s>>>(inout, n);
}

void launch_quantize_e4m3(const float* in, uint8_t* out, float* deq, long long n, float scale, cudaStream_t s)
{
    if (n > 0) quantize_e4m3_kernel<<<grid_for(n), 256, 0, s>>>(in, out, deq, n, scale);
}

void launch_transpose(const float* in, float* out, int rows, int cols, int batches, cudaStream_t s)
{
    if (rows <= 0 || cols <= 0 || batches <= 0) return;
    dim3 grid((cols + 31) / 32, (rows + 31) / 32, batches);
    transpose_kernel<<<grid, dim3(32, 8), 0, s>>>(in, out, rows, cols);
}

}  // namespace svm
