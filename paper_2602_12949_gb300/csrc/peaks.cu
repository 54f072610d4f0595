// Peak-rate probe for the roofline of the plain FP32 path: independent FP32 FMA chains on
// every thread, nothing else in the loop.  A diagnostic with no counterpart in the paper.
#include "niv_internal.cuh"

namespace {

constexpr int kChains = 8;  // independent chains per thread, enough to cover the FMA latency

__global__ void __launch_bounds__(256) peak_ffma_kernel(float* __restrict__ out, int iters, float a, float b) {
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c) * 1e-3f;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    if (s == 12345.678f) out[blockIdx.x] = s;  // keeps the chains live; practically never stores
}

}  // namespace

extern "C" int niv_peak_ffma(float* out, int32_t blocks, int32_t iters, niv_stream stream) {
    if (!out || blocks < 1 || iters < 1) return niv_fail(NIV_ERR_ARG, "out is NULL or blocks / iters < 1");
    peak_ffma_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(out, iters, 0.999999f, 1e-6f);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}
