// Peak-rate probes for the rooflines beside the tensor one: independent FP32 FMA chains on
// every thread (the plain FP32 path), and a kernel streaming through page-locked host memory
// (the host-buffer query, whose kernel reads records from and writes results to host memory
// over the host link).  Measurement aids with no counterpart in the paper, built into their
// own library (libniv_peaks.so) that only the benchmark loads, so the product library exports
// the query path alone.
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

// Grid-stride stream over host memory: word i < n_in of src is read, word i < n_out of dst is
// written (16-byte words, coalesced).  The XOR of what was read goes to sink[block] only in a
// case that does not occur, so the loads are kept.
__global__ void __launch_bounds__(256) peak_host_kernel(const uint4* __restrict__ src, uint4* __restrict__ dst,
                                                        int64_t n_in, int64_t n_out, uint32_t* __restrict__ sink) {
    const int64_t n = n_in > n_out ? n_in : n_out;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    uint32_t x = 0u;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += step) {
        if (i < n_in) {
            const uint4 v = __ldcs(src + i);
            x ^= v.x ^ v.y ^ v.z ^ v.w;
        }
        if (i < n_out) __stcs(dst + i, make_uint4((uint32_t)i, 0u, 0u, 0u));
    }
    if (x == 0x9E3779B9u) sink[blockIdx.x] = x;
}

// Device address of page-locked host memory, or nullptr.
const void* host_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

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

// Stream bytes_in bytes from the page-locked host buffer src and bytes_out bytes into the
// page-locked host buffer dst (either may be 0 with its pointer NULL) with `blocks` CTAs of 256
// threads; sink is a device uint32 [blocks].  Sizes must be multiples of 16 bytes and the
// buffers 16-byte aligned.  Asynchronous on `stream`.  Returns 0, -1 for invalid arguments
// (including memory the GPU cannot address), or -3 when the launch fails.
extern "C" __attribute__((visibility("default"))) int niv_peak_host_stream(const void* src, int64_t bytes_in, void* dst,
                                                                           int64_t bytes_out, uint32_t* sink,
                                                                           int32_t blocks, cudaStream_t stream) {
    if (!sink || blocks < 1 || bytes_in < 0 || bytes_out < 0 || (bytes_in | bytes_out) % 16 != 0) return -1;
    if ((bytes_in > 0 && !src) || (bytes_out > 0 && !dst)) return -1;
    const void* ds = bytes_in > 0 ? host_device_ptr(src) : nullptr;
    void* dd = bytes_out > 0 ? const_cast<void*>(host_device_ptr(dst)) : nullptr;
    if ((bytes_in > 0 && !ds) || (bytes_out > 0 && !dd)) return -1;
    if (((uintptr_t)ds | (uintptr_t)dd) % 16 != 0) return -1;
    peak_host_kernel<<<(unsigned)blocks, 256, 0, stream>>>(static_cast<const uint4*>(ds), static_cast<uint4*>(dd),
                                                           bytes_in / 16, bytes_out / 16, sink);
    return cudaGetLastError() == cudaSuccess ? 0 : -3;
}
