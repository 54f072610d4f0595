// Primary-visibility G-buffer of the analytic scene: per pixel the first-hit world position,
// surface normal and albedo, the buffers the per-pixel query of Sec. 4.4 reads (the
// deferred-shading inputs of Fig. 3).  A pinhole camera looks down +z with +y up; each
// pixel's ray passes through the pixel centre.  The intersection rules are the scene's own
// (scene.cuh, FP32), so the G-buffer, the Monte Carlo targets and the probe visibility rays
// all see the same geometry.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "niv.h"
#include "niv_internal.cuh"
#include "scene.cuh"

namespace {

constexpr int kGbW = 16, kGbH = 8;  // one CTA: a 16 x 8 pixel block (warps of 16 x 2 pixels)

// Record i of a [n][4] buffer: FP16 (8 bytes) or FP32 (16 bytes), pad 0.
__device__ __forceinline__ void gb_store(void* base, int64_t i, float3 v, bool f16) {
    if (f16) {
        const __half2 a = __floats2half2_rn(v.x, v.y), b = __floats2half2_rn(v.z, 0.0f);
        uint2 r;
        r.x = *reinterpret_cast<const uint32_t*>(&a);
        r.y = *reinterpret_cast<const uint32_t*>(&b);
        reinterpret_cast<uint2*>(base)[i] = r;
    } else {
        reinterpret_cast<float4*>(base)[i] = make_float4(v.x, v.y, v.z, 0.0f);
    }
}

// sx = tan(vfov / 2) * width / height, sy = tan(vfov / 2): the ray of pixel (i, j) has the
// direction ((2 (i + 0.5) / W - 1) sx, (1 - 2 (j + 0.5) / H) sy, 1), normalised.
__global__ void __launch_bounds__(kGbW * kGbH) gbuffer_raycast_kernel(SceneArg scene, int32_t width, int32_t height,
                                                                      float sx, float sy, float3 eye, float t,
                                                                      void* pos, void* nrm, void* alb, bool f16,
                                                                      uint8_t* hit_out) {
    __shared__ float s_scene[kHdr + kSph * kMaxObjects];
    const int len = kHdr + kSph * ((int)scene.v[0] + (int)scene.v[1]);
    for (int k = threadIdx.x; k < len; k += blockDim.x) s_scene[k] = scene.v[k];
    __syncthreads();
    SceneView S;
    S.init(s_scene, t);

    const int i = blockIdx.x * kGbW + (int)(threadIdx.x % kGbW);
    const int j = blockIdx.y * kGbH + (int)(threadIdx.x / kGbW);
    if (i >= width || j >= height) return;
    const float fx = (2.0f * (((float)i + 0.5f) / (float)width) - 1.0f) * sx;
    const float fy = (1.0f - 2.0f * (((float)j + 0.5f) / (float)height)) * sy;
    const float len_d = sqrtf(fx * fx + fy * fy + 1.0f);
    const float3 d = make_float3(fx / len_d, fy / len_d, 1.0f / len_d);
    Hit h;
    const bool any = S.intersect(eye, d, h);
    if (any && h.kind == 1) {  // (p - c) / r is unit only up to the error of the hit point: renormalise
        const float ln = sqrtf(dot3(h.n, h.n));
        h.n = make_float3(h.n.x / ln, h.n.y / ln, h.n.z / ln);
    }
    const float3 zero = make_float3(0.0f, 0.0f, 0.0f);
    const int64_t r = (int64_t)j * width + i;
    gb_store(pos, r, any ? h.p : zero, f16);
    gb_store(nrm, r, any ? h.n : zero, f16);
    if (alb) gb_store(alb, r, any ? S.albedo(h) : zero, f16);
    if (hit_out) hit_out[r] = (uint8_t)any;
}

bool gb_aligned(const void* p, size_t a) { return ((uintptr_t)p % a) == 0; }

}  // namespace

extern "C" int niv_gbuffer_raycast(const float* scene, int64_t scene_len, int32_t width, int32_t height,
                                   double vfov_deg, const float* eye, float t, void* pos, void* nrm, void* alb,
                                   int32_t dtype_out, uint8_t* hit, niv_stream stream) {
    if (!scene || !eye || !pos || !nrm) return niv_fail(NIV_ERR_ARG, "null scene, eye, pos or nrm");
    if (width <= 0 || height <= 0) return niv_fail(NIV_ERR_ARG, "width and height must be positive");
    if ((int64_t)width * height > ((int64_t)1 << 31)) return niv_fail(NIV_ERR_ARG, "at most 2^31 pixels");
    if (!(vfov_deg > 0.0 && vfov_deg < 180.0)) return niv_fail(NIV_ERR_ARG, "vfov_deg must lie in (0, 180)");
    if (dtype_out != NIV_F16 && dtype_out != NIV_F32) return niv_fail(NIV_ERR_ARG, "dtype_out must be NIV_F16 or NIV_F32");
    const size_t a = dtype_out == NIV_F16 ? 8 : 16;
    if (!gb_aligned(pos, a) || !gb_aligned(nrm, a) || (alb && !gb_aligned(alb, a)))
        return niv_fail(NIV_ERR_ALIGN, "records must be aligned to their size");
    if (scene_len < kHdr) return niv_fail(NIV_ERR_ARG, "scene description too short");
    SceneArg arg;
    const int ns = (int)scene[0], nb = (int)scene[1];
    if (ns < 0 || nb < 0 || ns + nb > kMaxObjects) return niv_fail(NIV_ERR_UNSUPPORTED, "at most 56 scene objects");
    if (!niv_scene_arg(scene, scene_len, arg)) return niv_fail(NIV_ERR_ARG, "scene description length mismatch");
    const double th = tan(vfov_deg * M_PI / 180.0 * 0.5);
    const float sx = (float)(th * ((double)width / height)), sy = (float)th;
    const dim3 grid((unsigned)((width + kGbW - 1) / kGbW), (unsigned)((height + kGbH - 1) / kGbH));
    if (grid.y > 65535u) return niv_fail(NIV_ERR_ARG, "height too large");
    gbuffer_raycast_kernel<<<grid, kGbW * kGbH, 0, (cudaStream_t)stream>>>(
        arg, width, height, sx, sy, make_float3(eye[0], eye[1], eye[2]), t, pos, nrm, alb, dtype_out == NIV_F16, hit);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}
