// Random numbers and direction sampling shared by the Monte Carlo integrator and the
// ambient-occlusion pass: Philox4x32-10 (Salmon et al., SC'11), u32 -> (0, 1) as
// (x >> 8) 2^-24 + 2^-25, the orthonormal basis of Duff et al. (JCGT 2017) and cosine-
// distributed directions (Malley's method).
#pragma once

#include <stdint.h>

namespace {

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
        const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ float u01(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f) + (1.0f / 33554432.0f); }

// orthonormal basis around unit n (Duff et al., JCGT 2017)
__device__ __forceinline__ void onb(float3 n, float3& t, float3& b) {
    const float sgn = copysignf(1.0f, n.z), a = -1.0f / (sgn + n.z), bb = n.x * n.y * a;
    t = make_float3(1.0f + sgn * n.x * n.x * a, sgn * bb, -sgn * n.x);
    b = make_float3(bb, sgn + n.y * n.y * a, -n.y);
}

__device__ __forceinline__ float3 cosine_dir(float3 n, float u1, float u2) {
    float3 t, b;
    onb(n, t, b);
    const float r = sqrtf(u1), phi = 6.283185307179586f * u2;
    const float x = r * cosf(phi), y = r * sinf(phi), z = sqrtf(fmaxf(1.0f - u1, 0.0f));
    return make_float3(x * t.x + y * b.x + z * n.x, x * t.y + y * b.y + z * n.y, x * t.z + y * b.z + z * n.z);
}

}  // namespace
