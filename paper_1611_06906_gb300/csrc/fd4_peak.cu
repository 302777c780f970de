// FP32 FMA rate of the GPU, measured (no counterpart in the paper): the
// denominator of the ALU-bound kernels' fractions (the Gaussian-derivative
// strips are bound by FP32 FMA issue).  Every thread runs 8 independent FMA
// chains (scalar form) or 4 chains of packed pairs (two FP32 lanes per
// instruction); the grid fills every SM with 2048 threads.
#include "fd4_internal.h"

namespace fd4 {
namespace {

constexpr int kPeakIters = 4096;

__global__ void __launch_bounds__(256) k_fma_scalar(float *out, float a, float b)
{
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (float)(threadIdx.x + i);
#pragma unroll 4
    for (int it = 0; it < kPeakIters; ++it) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == 1.2345f) out[blockIdx.x] = s;  // keeps the chains alive
}

__global__ void __launch_bounds__(256) k_fma_pair(float *out, float a, float b)
{
    float2 x[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) x[i] = make_float2((float)(threadIdx.x + i), (float)(threadIdx.x - i));
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll 4
    for (int it = 0; it < kPeakIters; ++it) {
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = __ffma2_rn(x[i], a2, b2);
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) s += x[i].x + x[i].y;
    if (s == 1.2345f) out[blockIdx.x] = s;
}

}  // namespace
}  // namespace fd4

extern "C" int fd4_measure_fma_rate(void *d_scratch, size_t scratch_bytes, double *scalar_tfma, double *pair_tfma,
                                    fd4_stream_t stream)
{
    using namespace fd4;
    if (!d_scratch || !scalar_tfma || !pair_tfma) return FD4_ERR_BAD_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FD4_ERR_CUDA;
    const int blocks = sms * 8;  // 8 blocks of 256 threads per SM
    if (scratch_bytes < sizeof(float) * (size_t)blocks) return FD4_ERR_WS_TOO_SMALL;
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess) return FD4_ERR_CUDA;
    if (cudaEventCreate(&e1) != cudaSuccess) {
        cudaEventDestroy(e0);
        return FD4_ERR_CUDA;
    }
    const double fmas = (double)blocks * 256.0 * 8.0 * kPeakIters;  // both kernels: 8 FMAs per thread-iteration
    int rc = FD4_OK;
    for (int form = 0; form < 2 && rc == FD4_OK; ++form) {
        float best = 0.0f;
        for (int rep = 0; rep < 4 && rc == FD4_OK; ++rep) {  // the first launch warms up
            if (cudaEventRecord(e0, st) != cudaSuccess) rc = FD4_ERR_CUDA;
            if (form == 0) k_fma_scalar<<<blocks, 256, 0, st>>>((float *)d_scratch, 0.999f, 1e-3f);
            else k_fma_pair<<<blocks, 256, 0, st>>>((float *)d_scratch, 0.999f, 1e-3f);
            if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) rc = FD4_ERR_CUDA;
            float ms = 0.0f;
            if (rc == FD4_OK && cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) rc = FD4_ERR_CUDA;
            if (rep > 0 && (best == 0.0f || ms < best)) best = ms;
        }
        if (rc == FD4_OK) *(form == 0 ? scalar_tfma : pair_tfma) = fmas / (best * 1e-3) / 1e12;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return rc;
}
