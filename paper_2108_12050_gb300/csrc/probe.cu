// FP32 FFMA throughput probe: the denominator of the fused kernel's
// roofline (one FFMA counted as one operation).  Each thread runs eight
// independent FMA chains on registers; the grid covers every SM several
// times over.  Timed with CUDA events on the caller's stream.
#include "internal.h"

namespace mhfd {

namespace {

constexpr int kIters = 4096;

__global__ void __launch_bounds__(256) ffma_probe(float *out, float a, float b) {
    float x0 = threadIdx.x * 1e-7f, x1 = x0 + 1e-3f, x2 = x0 + 2e-3f, x3 = x0 + 3e-3f;
    float x4 = x0 + 4e-3f, x5 = x0 + 5e-3f, x6 = x0 + 6e-3f, x7 = x0 + 7e-3f;
#pragma unroll 16
    for (int i = 0; i < kIters; ++i) {
        x0 = fmaf(x0, a, b);
        x1 = fmaf(x1, a, b);
        x2 = fmaf(x2, a, b);
        x3 = fmaf(x3, a, b);
        x4 = fmaf(x4, a, b);
        x5 = fmaf(x5, a, b);
        x6 = fmaf(x6, a, b);
        x7 = fmaf(x7, a, b);
    }
    const float r = ((x0 + x1) + (x2 + x3)) + ((x4 + x5) + (x6 + x7));
    if (r == 1234.5f) out[blockIdx.x] = r;  // keeps the chains alive
}

}  // namespace

int probe_ffma(cudaStream_t s, double *ops_per_s) {
    int dev = 0, sms = 0;
    MHFD_CUDA(cudaGetDevice(&dev));
    MHFD_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    float *out = nullptr;
    MHFD_CUDA(cudaMalloc(&out, sizeof(float) * 4096));
    const int grid = sms * 8 * 4;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    for (int w = 0; w < 3; ++w) ffma_probe<<<grid, 256, 0, s>>>(out, 0.999f, 1e-6f);
    float best = 1e30f;
    for (int r = 0; r < 5; ++r) {
        cudaEventRecord(e0, s);
        ffma_probe<<<grid, 256, 0, s>>>(out, 0.999f, 1e-6f);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    MHFD_CUDA(cudaGetLastError());
    const double ops = (double)grid * 256.0 * kIters * 8.0;
    *ops_per_s = ops / (best * 1e-3);
    return MHFD_OK;
}

}  // namespace mhfd
