// Deferred shading of the indirect term (Eq. 2) plus runtime direct light (Sec. 3, Fig. 3):
//   rgba = (albedo * E / pi + direct, 1), FP32 arithmetic, FP16 records in and out.
// Purely HBM-bound: 24 B read and 8 B written per pixel, 8-byte vector accesses,
// consecutive threads on consecutive pixels.
#include "niv_internal.cuh"

namespace {

__device__ __forceinline__ float4 ld_h4(const uint2* p, int64_t i) {
    uint2 r = __ldcs(p + i);  // streamed once: evict-first
    float2 a = __half22float2(*reinterpret_cast<__half2*>(&r.x));
    float2 b = __half22float2(*reinterpret_cast<__half2*>(&r.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

__global__ void __launch_bounds__(256) shade_kernel(const uint2* __restrict__ albedo, const uint2* __restrict__ direct,
                                                    const uint2* __restrict__ E, int64_t n, uint2* __restrict__ out) {
    const float inv_pi = 0.318309886183790671538f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float4 a = ld_h4(albedo, i), d = ld_h4(direct, i), e = ld_h4(E, i);
        const float r = fmaf(a.x * e.x, inv_pi, d.x);
        const float g = fmaf(a.y * e.y, inv_pi, d.y);
        const float b = fmaf(a.z * e.z, inv_pi, d.z);
        __half2 rg = __floats2half2_rn(r, g), ba = __floats2half2_rn(b, 1.0f);
        uint2 o;
        o.x = *reinterpret_cast<uint32_t*>(&rg);
        o.y = *reinterpret_cast<uint32_t*>(&ba);
        __stcs(out + i, o);
    }
}

}  // namespace

int niv_launch_shade(const void* albedo, const void* direct, const void* E, int64_t n, void* out, cudaStream_t s) {
    int dev = 0, sms = 0;
    NIV_CUDA(cudaGetDevice(&dev));
    NIV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int64_t blocks = (n + 255) / 256;
    const int64_t cap = (int64_t)sms * 8;
    if (blocks > cap) blocks = cap;
    shade_kernel<<<(unsigned)blocks, 256, 0, s>>>((const uint2*)albedo, (const uint2*)direct, (const uint2*)E, n,
                                                  (uint2*)out);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}
