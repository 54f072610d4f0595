// Peak-rate probe for the roofline of the plain FP32 path: independent FP32 FMA chains on
// every thread, nothing else in the loop.  A measurement aid with no counterpart in the
// paper, built into its own library (libniv_peaks.so) that only the benchmark loads, so the
// product library exports the query path alone.
//
//   int niv_peak_ffma(float* out, int32_t blocks, int32_t iters, cudaStream_t stream);
//
// Launches `blocks` CTAs of 256 threads, each thread running 8 independent FMA chains for
// `iters` steps (2 * 8 * iters FLOP per thread, 4096 * blocks * iters in all); out (device
// float32 [blocks]) is written only in a case that does not occur, so that the chains are
// kept.  Asynchronous on `stream`; time it with events.  Returns 0, -1 for invalid arguments,
// or -3 when the launch fails.
#include <cuda_runtime.h>
#include <stdint.h>

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

extern "C" __attribute__((visibility("default"))) int niv_peak_ffma(float* out, int32_t blocks, int32_t iters,
                                                                    cudaStream_t stream) {
    if (!out || blocks < 1 || iters < 1) return -1;
    peak_ffma_kernel<<<(unsigned)blocks, 256, 0, stream>>>(out, iters, 0.999999f, 1e-6f);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}
