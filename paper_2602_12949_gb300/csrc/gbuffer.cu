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

// ---- triangle meshes inserted into a G-buffer ----
// Three passes over a 64-bit depth key per pixel, (float bits of the hit distance t) << 32 |
// (triangle + 1), whose minimum is the nearest surface (t >= 0, so the float bits order like
// the values; among triangles at the same t the lowest index wins, and a surface already in
// the G-buffer keeps the pixel against a triangle at exactly its distance).
namespace {

constexpr int kMaxMeshes = 64;

struct MeshAlbedo {
    float v[3 * kMaxMeshes];
    int32_t count;
};

struct Camera {
    float3 eye;
    float sx, sy;  // tan(vfov / 2) * width / height, tan(vfov / 2)
    int32_t width, height;

    __device__ __forceinline__ float3 ray(int i, int j) const {
        const float fx = (2.0f * (((float)i + 0.5f) / (float)width) - 1.0f) * sx;
        const float fy = (1.0f - 2.0f * (((float)j + 0.5f) / (float)height)) * sy;
        const float len_d = sqrtf(fx * fx + fy * fy + 1.0f);
        return make_float3(fx / len_d, fy / len_d, 1.0f / len_d);
    }
};

__device__ __forceinline__ float3 sub3(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Moeller-Trumbore: the distance along the unit ray o + t d to triangle (A, B, C), or a
// negative value when the ray misses it (parallel, outside the edges, or t <= 1e-6).  The
// edge tests accept barycentrics up to kBaryEps outside the triangle, so that a ray through
// the edge two triangles share hits at least one of them despite FP32 rounding (a strict
// test leaves cracks through which the ray reaches a surface behind the mesh).
constexpr float kBaryEps = 1e-5f;
__device__ __forceinline__ float ray_triangle(float3 o, float3 d, float3 A, float3 e1, float3 e2) {
    const float3 p = cross3(d, e2);
    const float det = dot3(e1, p);
    if (fabsf(det) < 1e-12f) return -1.0f;
    const float inv = 1.0f / det;
    const float3 s = sub3(o, A);
    const float u = dot3(s, p) * inv;
    if (u < -kBaryEps || u > 1.0f + kBaryEps) return -1.0f;
    const float3 q = cross3(s, e1);
    const float v = dot3(d, q) * inv;
    if (v < -kBaryEps || u + v > 1.0f + kBaryEps) return -1.0f;
    const float t = dot3(e2, q) * inv;
    return t > 1e-6f ? t : -1.0f;
}

__device__ __forceinline__ float3 gb_load(const void* base, int64_t i, bool f16) {
    if (f16) {
        const uint2 r = reinterpret_cast<const uint2*>(base)[i];
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
        const float b = __low2float(*reinterpret_cast<const __half2*>(&r.y));
        return make_float3(a.x, a.y, b);
    }
    const float4 r = reinterpret_cast<const float4*>(base)[i];
    return make_float3(r.x, r.y, r.z);
}

// Pass 1: every pixel's key from the surface already there (distance |pos - eye|), or +inf.
__global__ void mesh_key_init_kernel(Camera cam, const void* pos, bool f16, const uint8_t* hit,
                                     unsigned long long* key, int64_t n) {
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    float t = INFINITY;
    if (hit[r]) {
        const float3 p = sub3(gb_load(pos, r, f16), cam.eye);
        t = sqrtf(dot3(p, p));
    }
    key[r] = (unsigned long long)__float_as_uint(t) << 32;
}

// Pass 2: one thread per triangle over the pixels of its projected bounding box (one pixel
// of margin), keeping the nearest hit per pixel with a 64-bit atomic minimum.
__global__ void mesh_raster_kernel(Camera cam, const float* __restrict__ tri9, int64_t n_tris,
                                   unsigned long long* key) {
    const int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= n_tris) return;
    const float* T = tri9 + 9 * f;
    const float3 A = make_float3(T[0], T[1], T[2]), B = make_float3(T[3], T[4], T[5]), C = make_float3(T[6], T[7], T[8]);
    const float3 V[3] = {A, B, C};
    float imin = 1e30f, imax = -1e30f, jmin = 1e30f, jmax = -1e30f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float3 dv = sub3(V[k], cam.eye);
        if (dv.z <= 1e-3f) return;  // a vertex behind the camera: the triangle is skipped
        const float px = (dv.x / dv.z / cam.sx + 1.0f) * 0.5f * cam.width - 0.5f;
        const float py = (1.0f - dv.y / dv.z / cam.sy) * 0.5f * cam.height - 0.5f;
        imin = fminf(imin, px);
        imax = fmaxf(imax, px);
        jmin = fminf(jmin, py);
        jmax = fmaxf(jmax, py);
    }
    const int i0 = max(0, (int)floorf(fmaxf(imin, -2.0f)) - 1), i1 = min(cam.width - 1, (int)ceilf(fminf(imax, 1e9f)) + 1);
    const int j0 = max(0, (int)floorf(fmaxf(jmin, -2.0f)) - 1), j1 = min(cam.height - 1, (int)ceilf(fminf(jmax, 1e9f)) + 1);
    const float3 e1 = sub3(B, A), e2 = sub3(C, A);
    const unsigned long long tag = (unsigned long long)(f + 1);
    for (int j = j0; j <= j1; ++j)
        for (int i = i0; i <= i1; ++i) {
            const float t = ray_triangle(cam.eye, cam.ray(i, j), A, e1, e2);
            if (t < 0.0f) continue;
            const int64_t r = (int64_t)j * cam.width + i;
            const unsigned long long k = ((unsigned long long)__float_as_uint(t) << 32) | tag;
            if (k < key[r]) atomicMin(key + r, k);
        }
}

// Pass 3: pixels a triangle won get its hit point, its face normal turned toward the camera,
// its mesh's albedo and the mesh index; every pixel gets its mesh index (-1: none).
__global__ void mesh_resolve_kernel(Camera cam, const float* __restrict__ tri9, const int32_t* __restrict__ tri_mesh,
                                    MeshAlbedo alb_m, const unsigned long long* __restrict__ key, void* pos,
                                    void* nrm, void* alb, bool f16, uint8_t* hit, int32_t* mesh_id) {
    const int i = blockIdx.x * kGbW + (int)(threadIdx.x % kGbW);
    const int j = blockIdx.y * kGbH + (int)(threadIdx.x / kGbW);
    if (i >= cam.width || j >= cam.height) return;
    const int64_t r = (int64_t)j * cam.width + i;
    const uint32_t tag = (uint32_t)(key[r] & 0xFFFFFFFFull);
    if (tag == 0u) {
        if (mesh_id) mesh_id[r] = -1;
        return;
    }
    const int64_t f = (int64_t)tag - 1;
    const float* T = tri9 + 9 * f;
    const float3 A = make_float3(T[0], T[1], T[2]), B = make_float3(T[3], T[4], T[5]), C = make_float3(T[6], T[7], T[8]);
    const float3 e1 = sub3(B, A), e2 = sub3(C, A);
    const float3 d = cam.ray(i, j);
    const float t = __uint_as_float((uint32_t)(key[r] >> 32));
    float3 n = cross3(e1, e2);
    const float nl = sqrtf(dot3(n, n));
    const float sg = dot3(n, d) > 0.0f ? -1.0f : 1.0f;
    n = make_float3(sg * n.x / nl, sg * n.y / nl, sg * n.z / nl);
    const int mesh = tri_mesh[f];
    const bool known = mesh >= 0 && mesh < alb_m.count;  // an unknown mesh index gets albedo 0
    gb_store(pos, r, make_float3(cam.eye.x + t * d.x, cam.eye.y + t * d.y, cam.eye.z + t * d.z), f16);
    gb_store(nrm, r, n, f16);
    if (alb)
        gb_store(alb, r, known ? make_float3(alb_m.v[3 * mesh], alb_m.v[3 * mesh + 1], alb_m.v[3 * mesh + 2])
                               : make_float3(0.0f, 0.0f, 0.0f), f16);
    hit[r] = 1;
    if (mesh_id) mesh_id[r] = mesh;
}

}  // namespace

extern "C" int niv_gbuffer_meshes(const float* tri9, const int32_t* tri_mesh, int64_t n_tris, const float* mesh_albedo,
                                  int32_t n_meshes, int32_t width, int32_t height, double vfov_deg, const float* eye,
                                  void* pos, void* nrm, void* alb, int32_t dtype, uint8_t* hit, int32_t* mesh_id,
                                  uint64_t* scratch, niv_stream stream) {
    if (!eye || !pos || !nrm || !hit || !scratch) return niv_fail(NIV_ERR_ARG, "null eye, pos, nrm, hit or scratch");
    if (n_tris < 0 || n_tris >= ((int64_t)1 << 31)) return niv_fail(NIV_ERR_ARG, "n_tris outside [0, 2^31)");
    if (n_tris > 0 && (!tri9 || !tri_mesh)) return niv_fail(NIV_ERR_ARG, "null triangles");
    if (n_meshes < 1 || n_meshes > kMaxMeshes || !mesh_albedo) return niv_fail(NIV_ERR_ARG, "1 to 64 meshes with albedo");
    if (width <= 0 || height <= 0) return niv_fail(NIV_ERR_ARG, "width and height must be positive");
    if ((int64_t)width * height > ((int64_t)1 << 31)) return niv_fail(NIV_ERR_ARG, "at most 2^31 pixels");
    if (!(vfov_deg > 0.0 && vfov_deg < 180.0)) return niv_fail(NIV_ERR_ARG, "vfov_deg must lie in (0, 180)");
    if (dtype != NIV_F16 && dtype != NIV_F32) return niv_fail(NIV_ERR_ARG, "dtype must be NIV_F16 or NIV_F32");
    const size_t a = dtype == NIV_F16 ? 8 : 16;
    if (!gb_aligned(pos, a) || !gb_aligned(nrm, a) || (alb && !gb_aligned(alb, a)) || !gb_aligned(scratch, 8) ||
        !gb_aligned(tri9, 4) || (mesh_id && !gb_aligned(mesh_id, 4)))
        return niv_fail(NIV_ERR_ALIGN, "records must be aligned to their size");
    Camera cam;
    const double th = tan(vfov_deg * M_PI / 180.0 * 0.5);
    cam.eye = make_float3(eye[0], eye[1], eye[2]);
    cam.sx = (float)(th * ((double)width / height));
    cam.sy = (float)th;
    cam.width = width;
    cam.height = height;
    MeshAlbedo am;
    memset(&am, 0, sizeof am);
    memcpy(am.v, mesh_albedo, sizeof(float) * 3 * n_meshes);
    am.count = n_meshes;
    const dim3 grid((unsigned)((width + kGbW - 1) / kGbW), (unsigned)((height + kGbH - 1) / kGbH));
    if (grid.y > 65535u) return niv_fail(NIV_ERR_ARG, "height too large");
    const int64_t n = (int64_t)width * height;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long* key = reinterpret_cast<unsigned long long*>(scratch);
    const bool f16 = dtype == NIV_F16;
    mesh_key_init_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(cam, pos, f16, hit, key, n);
    NIV_CUDA(cudaGetLastError());
    if (n_tris > 0) {
        mesh_raster_kernel<<<(unsigned)((n_tris + 127) / 128), 128, 0, s>>>(cam, tri9, n_tris, key);
        NIV_CUDA(cudaGetLastError());
    }
    mesh_resolve_kernel<<<grid, kGbW * kGbH, 0, s>>>(cam, tri9, tri_mesh, am, key, pos, nrm, alb, f16, hit, mesh_id);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}
