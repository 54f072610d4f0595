// Monte Carlo irradiance (Eq. 1) of the analytic scenes: the training targets of Sec. 4.5.
//
// One thread per query point.  E(x, n) = (pi / S) sum_j L_i(x, w_j) over S cosine-
// distributed directions w_j about n; L_i follows a path with next-event estimation
// toward every emitting sphere (uniform sampling of the subtended cone), cosine
// continuation and Russian roulette after three bounces (at most 32 segments).
// INDIRECT mode (what the paper caches; direct light is added at runtime, Sec. 3)
// drops emission seen by the first segment and sky light reaching x directly.
// A point is flagged for discard when more than half of its first hits are back
// faces (it lies inside geometry, Sec. 4.5) or when its irradiance is zero in
// every channel (App. I).  Geometry runs in FP32; the per-point sum is FP64.
//
// Random numbers: Philox4x32-10 (Salmon et al., SC'11) on counter
// (point lo, point hi, j + (depth << 16), purpose) with key (seed lo, seed hi);
// purpose 0 = bounce direction + roulette, 1 + e = light sample toward emitter e;
// the first direction of path j uses depth 0xFFFF.  u32 -> (0,1): (x >> 8) 2^-24 + 2^-25.
#include <math.h>
#include <string.h>

#include "niv_internal.cuh"
#include "sampling.cuh"
#include "scene.cuh"

namespace {

constexpr int kMaxDepth = 32;

struct Rng {
    uint64_t point, seed;
    __device__ float4 draw(uint32_t j, uint32_t depth, uint32_t purpose) const {
        const uint4 o = philox4x32_10(make_uint4((uint32_t)point, (uint32_t)(point >> 32), j + (depth << 16), purpose),
                                      (uint32_t)seed, (uint32_t)(seed >> 32));
        return make_float4(u01(o.x), u01(o.y), u01(o.z), u01(o.w));
    }
};

// Incident radiance along one path starting at o in direction d.
__device__ float3 path_radiance(const SceneView& S, const Rng& rng, uint32_t j, float3 o, float3 d, int mode,
                                bool& first_hit, bool& first_back) {
    float3 beta = make_float3(1.0f, 1.0f, 1.0f), L = make_float3(0.0f, 0.0f, 0.0f);
    first_hit = false;
    first_back = false;
    for (int depth = 0; depth < kMaxDepth; ++depth) {
        Hit hh;
        if (!S.intersect(o, d, hh)) {
            if (depth > 0 || mode == 0) {
                L.x += beta.x * S.h[10];
                L.y += beta.y * S.h[11];
                L.z += beta.z * S.h[12];
            }
            return L;
        }
        const float cosi = dot3(d, hh.n);
        if (depth == 0) {
            first_hit = true;
            first_back = cosi > 0.0f;
        }
        const float3 Le = S.emission(hh);
        const bool nee_target = hh.kind == 1 && S.emits(hh.id);
        if (depth == 0 ? mode == 0 : !nee_target) {
            L.x += beta.x * Le.x;
            L.y += beta.y * Le.y;
            L.z += beta.z * Le.z;
        }
        const float3 rho = S.albedo(hh);
        if (rho.x <= 0.0f && rho.y <= 0.0f && rho.z <= 0.0f) return L;
        const float3 nf = cosi < 0.0f ? hh.n : make_float3(-hh.n.x, -hh.n.y, -hh.n.z);
        const float3 p = make_float3(hh.p.x + kTEps * nf.x, hh.p.y + kTEps * nf.y, hh.p.z + kTEps * nf.z);
        for (int e = 0; e < S.ns; ++e) {
            if (!S.emits(e)) continue;
            const float3 c = S.centre(e);
            const float r = S.sph[kSph * e + 3];
            float3 w = make_float3(c.x - p.x, c.y - p.y, c.z - p.z);
            const float dist2 = dot3(w, w), dist = sqrtf(dist2);
            if (dist <= r) continue;
            w = make_float3(w.x / dist, w.y / dist, w.z / dist);
            const float cmax = sqrtf(fmaxf(1.0f - r * r / dist2, 0.0f));
            const float4 u = rng.draw(j, (uint32_t)depth, 1u + (uint32_t)e);
            const float ct = 1.0f - u.x * (1.0f - cmax);
            const float st = sqrtf(fmaxf(1.0f - ct * ct, 0.0f)), phi = 6.283185307179586f * u.y;
            float3 tt, bb;
            onb(w, tt, bb);
            const float cs = st * cosf(phi), sn = st * sinf(phi);
            const float3 wl = make_float3(cs * tt.x + sn * bb.x + ct * w.x, cs * tt.y + sn * bb.y + ct * w.y,
                                          cs * tt.z + sn * bb.z + ct * w.z);
            const float cosl = dot3(nf, wl);
            if (cosl <= 0.0f) continue;
            // the shadow ray counts when its closest hit is the emitter: the emitter's own hit
            // distance (as intersect computes it) with nothing hit before it
            float te;
            {
                const float3 oc = make_float3(p.x - c.x, p.y - c.y, p.z - c.z);
                const float b = dot3(oc, wl), disc = b * b - (dot3(oc, oc) - r * r);
                if (disc < 0.0f) continue;
                const float sq = sqrtf(disc);
                te = -b - sq;
                if (te <= kTEps) te = -b + sq;
                if (!(te > kTEps)) continue;
            }
            if (S.occluded(p, wl, te)) continue;
            const float pdf_inv = 6.283185307179586f * (1.0f - cmax);
            const float* Ee = S.sph + kSph * e + 7;
            const float f = cosl * pdf_inv * 0.3183098861837907f;
            L.x += beta.x * rho.x * Ee[0] * f;
            L.y += beta.y * rho.y * Ee[1] * f;
            L.z += beta.z * rho.z * Ee[2] * f;
        }
        const float4 u = rng.draw(j, (uint32_t)depth, 0u);
        if (depth >= 3) {
            const float q = fminf(fmaxf(fmaxf(beta.x, beta.y), beta.z), 0.95f);
            if (u.z >= q) return L;
            beta = make_float3(beta.x / q, beta.y / q, beta.z / q);
        }
        d = cosine_dir(nf, u.x, u.y);
        beta = make_float3(beta.x * rho.x, beta.y * rho.y, beta.z * rho.z);
        o = p;
    }
    return L;
}

__global__ void __launch_bounds__(128) mc_irradiance_kernel(SceneArg scene, const float4* __restrict__ x4,
                                                            const float4* __restrict__ n4, const float* __restrict__ tq,
                                                            int64_t m, int spp, uint64_t seed, uint64_t index_base,
                                                            int mode, double* __restrict__ outE,
                                                            uint8_t* __restrict__ keep) {
    __shared__ float s_scene[kHdr + kSph * kMaxObjects];
    const int len = kHdr + kSph * ((int)scene.v[0] + (int)scene.v[1]);
    for (int k = threadIdx.x; k < len; k += blockDim.x) s_scene[k] = scene.v[k];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= m) return;
    SceneView S;
    S.init(s_scene, tq ? tq[i] : 0.0f);
    const Rng rng{index_base + (uint64_t)i, seed};
    const float4 xq = x4[i], nq4 = n4[i];
    const float3 x = make_float3(xq.x, xq.y, xq.z);
    float3 n = make_float3(nq4.x, nq4.y, nq4.z);
    const float nl = sqrtf(dot3(n, n));
    n = make_float3(n.x / nl, n.y / nl, n.z / nl);
    double ax = 0.0, ay = 0.0, az = 0.0;
    int back = 0;
    for (int j = 0; j < spp; ++j) {
        const float4 u = rng.draw((uint32_t)j, 0xFFFFu, 0u);
        const float3 w = cosine_dir(n, u.x, u.y);
        bool fh, fb;
        const float3 L = path_radiance(S, rng, (uint32_t)j, x, w, mode, fh, fb);
        back += fb;
        ax += L.x;
        ay += L.y;
        az += L.z;
    }
    const double k = 3.141592653589793 / (double)spp;
    outE[3 * i + 0] = ax * k;
    outE[3 * i + 1] = ay * k;
    outE[3 * i + 2] = az * k;
    if (keep) keep[i] = (uint8_t)(!(2 * back > spp) && !(ax == 0.0 && ay == 0.0 && az == 0.0));
}

}  // namespace

int niv_launch_mc(const float* blob, int64_t blob_len, const float* x4, const float* n4, const float* t, int64_t m,
                  int spp, uint64_t seed, uint64_t index_base, int mode, double* outE, uint8_t* keep, cudaStream_t s) {
    const int ns = (int)blob[0], nb = (int)blob[1];
    if (ns < 0 || nb < 0 || ns + nb > kMaxObjects) return niv_fail(NIV_ERR_UNSUPPORTED, "at most 56 scene objects");
    if (blob_len != kHdr + kSph * ns + kBox * nb) return niv_fail(NIV_ERR_ARG, "scene description length mismatch");
    SceneArg arg;
    memset(&arg, 0, sizeof arg);
    memcpy(arg.v, blob, sizeof(float) * blob_len);
    const unsigned blocks = (unsigned)((m + 127) / 128);
    mc_irradiance_kernel<<<blocks, 128, 0, s>>>(arg, (const float4*)x4, (const float4*)n4, t, m, spp, seed, index_base,
                                                mode, outE, keep);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}

// ---- SH probe bake (Sec. 5.1, App. A) ----
// Per probe: second-order real SH (9 coefficients x RGB) of the indirect incident
// radiance, L_lm = (4 pi / S) sum_j L_i(w_j) Y_lm(w_j), directions uniform on the sphere
// from Philox counter (probe lo, probe hi, j + (0xFFFE << 16), 0); the path of ray j uses
// stream index_base + probe * rays + j.  Probes sit at the lattice vertices
// lo + (hi - lo) * ijk / (P - 1), x fastest.
namespace {

__device__ __forceinline__ void sh9(float3 w, float* Y) {
    const float c0 = 0.28209479177387814f;  // 1 / (2 sqrt(pi))
    const float c1 = 0.4886025119029199f;   // sqrt(3 / (4 pi))
    const float c2 = 1.0925484305920792f;   // sqrt(15 / pi) / 2
    const float c20 = 0.31539156525252005f; // sqrt(5 / pi) / 4
    const float c22 = 0.5462742152960396f;  // sqrt(15 / pi) / 4
    Y[0] = c0;
    Y[1] = c1 * w.y;
    Y[2] = c1 * w.z;
    Y[3] = c1 * w.x;
    Y[4] = c2 * w.x * w.y;
    Y[5] = c2 * w.y * w.z;
    Y[6] = c20 * (3.0f * w.z * w.z - 1.0f);
    Y[7] = c2 * w.x * w.z;
    Y[8] = c22 * (w.x * w.x - w.y * w.y);
}

__global__ void __launch_bounds__(128) probe_bake_kernel(SceneArg scene, int px, int py, int pz, float3 lo, float3 hi,
                                                         int rays, uint64_t seed, uint64_t index_base,
                                                         double* __restrict__ out64, __half* __restrict__ out16) {
    __shared__ float s_scene[kHdr + kSph * kMaxObjects];
    const int len = kHdr + kSph * ((int)scene.v[0] + (int)scene.v[1]);
    for (int k = threadIdx.x; k < len; k += blockDim.x) s_scene[k] = scene.v[k];
    __syncthreads();
    const int64_t np = (int64_t)px * py * pz;
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= np) return;
    SceneView S;
    S.init(s_scene, 0.0f);
    const int64_t i = p % px, j = (p / px) % py, k = p / ((int64_t)px * py);
    const float3 x = make_float3(lo.x + (hi.x - lo.x) * (float)i / (float)(px - 1),
                                 lo.y + (hi.y - lo.y) * (float)j / (float)(py - 1),
                                 lo.z + (hi.z - lo.z) * (float)k / (float)(pz - 1));
    double c[27];
#pragma unroll
    for (int q = 0; q < 27; ++q) c[q] = 0.0;
    for (int r = 0; r < rays; ++r) {
        const uint4 o = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)(p >> 32), (uint32_t)r + (0xFFFEu << 16), 0u),
                                      (uint32_t)seed, (uint32_t)(seed >> 32));
        const float z = 1.0f - 2.0f * u01(o.x), rr = sqrtf(fmaxf(1.0f - z * z, 0.0f));
        const float phi = 6.283185307179586f * u01(o.y);
        const float3 w = make_float3(rr * cosf(phi), rr * sinf(phi), z);
        const Rng rng{index_base + (uint64_t)p * (uint64_t)rays + (uint64_t)r, seed};
        bool fh, fb;
        const float3 L = path_radiance(S, rng, 0u, x, w, 1, fh, fb);
        float Y[9];
        sh9(w, Y);
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            c[3 * q + 0] += (double)(L.x * Y[q]);
            c[3 * q + 1] += (double)(L.y * Y[q]);
            c[3 * q + 2] += (double)(L.z * Y[q]);
        }
    }
    const double sc = 4.0 * 3.141592653589793 / (double)rays;
#pragma unroll
    for (int q = 0; q < 27; ++q) {
        if (out64) out64[p * 27 + q] = c[q] * sc;
        if (out16) out16[p * 28 + q] = __float2half_rn((float)(c[q] * sc));
    }
    if (out16) out16[p * 28 + 27] = __float2half_rn(0.0f);
}

// ---- order-preserving compaction of kept Monte Carlo samples ----
constexpr int kCB = 1024;  // elements per block

__global__ void count_kept_kernel(const uint8_t* __restrict__ keep, int64_t m, int* __restrict__ block_counts) {
    __shared__ int s;
    if (threadIdx.x == 0) s = 0;
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)kCB + threadIdx.x;
    int c = 0;
    for (int64_t k = i; k < min(m, (int64_t)(blockIdx.x + 1) * kCB); k += blockDim.x) c += keep[k] != 0;
    c = __reduce_add_sync(0xFFFFFFFFu, c);
    if ((threadIdx.x & 31) == 0) atomicAdd(&s, c);
    __syncthreads();
    if (threadIdx.x == 0) block_counts[blockIdx.x] = s;
}

__global__ void scan_blocks_kernel(int* __restrict__ counts, int nb, int64_t* __restrict__ total) {
    // single thread: nb is small (m / 1024)
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        int64_t acc = 0;
        for (int b = 0; b < nb; ++b) {
            const int c = counts[b];
            counts[b] = (int)acc;
            acc += c;
        }
        *total = acc;
    }
}

__global__ void __launch_bounds__(kCB) scatter_kept_kernel(const float4* __restrict__ x4, const float4* __restrict__ n4,
                                                           const float* __restrict__ t, const double* __restrict__ E,
                                                           const uint8_t* __restrict__ keep, int64_t m,
                                                           const int* __restrict__ offsets, float4* __restrict__ ox4,
                                                           float4* __restrict__ on4, float* __restrict__ ot,
                                                           float4* __restrict__ otarget) {
    __shared__ int warp_sums[kCB / 32];
    const int64_t i = blockIdx.x * (int64_t)kCB + threadIdx.x;
    const int flag = (i < m && keep[i]) ? 1 : 0;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int incl = flag;
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sums[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        int v = warp_sums[lane];
        int sc = v;
        for (int o = 1; o < 32; o <<= 1) {
            const int u = __shfl_up_sync(0xFFFFFFFFu, sc, o);
            if (lane >= o) sc += u;
        }
        warp_sums[lane] = sc - v;  // exclusive prefix over warps
    }
    __syncthreads();
    if (flag) {
        const int64_t dst = (int64_t)offsets[blockIdx.x] + warp_sums[wid] + incl - 1;
        ox4[dst] = x4[i];
        on4[dst] = n4[i];
        if (ot) ot[dst] = t ? t[i] : 0.0f;
        otarget[dst] = make_float4((float)E[3 * i], (float)E[3 * i + 1], (float)E[3 * i + 2], 0.0f);
    }
}

}  // namespace

int niv_launch_probe_bake(const float* blob, int64_t blob_len, const int* P, const float* lo, const float* hi, int rays,
                          uint64_t seed, uint64_t index_base, double* out64, __half* out16, cudaStream_t s) {
    const int ns = (int)blob[0], nb = (int)blob[1];
    if (ns < 0 || nb < 0 || ns + nb > kMaxObjects) return niv_fail(NIV_ERR_UNSUPPORTED, "at most 56 scene objects");
    if (blob_len != kHdr + kSph * ns + kBox * nb) return niv_fail(NIV_ERR_ARG, "scene description length mismatch");
    SceneArg arg;
    memset(&arg, 0, sizeof arg);
    memcpy(arg.v, blob, sizeof(float) * blob_len);
    const int64_t np = (int64_t)P[0] * P[1] * P[2];
    probe_bake_kernel<<<(unsigned)((np + 127) / 128), 128, 0, s>>>(arg, P[0], P[1], P[2], make_float3(lo[0], lo[1], lo[2]),
                                                                  make_float3(hi[0], hi[1], hi[2]), rays, seed, index_base,
                                                                  out64, out16);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}

int niv_launch_compact(const float* x4, const float* n4, const float* t, const double* E, const uint8_t* keep, int64_t m,
                       float* ox4, float* on4, float* ot, float* otarget, int64_t* count_dev, int* scratch,
                       cudaStream_t s) {
    const int nb = (int)((m + kCB - 1) / kCB);
    count_kept_kernel<<<nb, 256, 0, s>>>(keep, m, scratch);
    scan_blocks_kernel<<<1, 32, 0, s>>>(scratch, nb, count_dev);
    scatter_kept_kernel<<<nb, kCB, 0, s>>>((const float4*)x4, (const float4*)n4, t, E, keep, m, scratch, (float4*)ox4,
                                           (float4*)on4, ot, (float4*)otarget);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}

// ---- the device counter-based generator on given counters and keys ----
namespace {
__global__ void philox_selftest_kernel(const uint32_t* __restrict__ in6, int64_t n, uint32_t* __restrict__ out4) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t* p = in6 + 6 * i;
    const uint4 r = philox4x32_10(make_uint4(p[0], p[1], p[2], p[3]), p[4], p[5]);
    out4[4 * i] = r.x;
    out4[4 * i + 1] = r.y;
    out4[4 * i + 2] = r.z;
    out4[4 * i + 3] = r.w;
}
}  // namespace

extern "C" int niv_selftest_philox(const uint32_t* in6, int64_t n, uint32_t* out4, niv_stream stream) {
    if (n < 0) return niv_fail(NIV_ERR_ARG, "n < 0");
    if (n == 0) return NIV_OK;
    if (!in6 || !out4) return niv_fail(NIV_ERR_ARG, "NULL pointer");
    const int64_t blocks = (n + 127) / 128;
    if (blocks > 0x7FFFFFFF) return niv_fail(NIV_ERR_ARG, "n too large");
    philox_selftest_kernel<<<(unsigned)blocks, 128, 0, (cudaStream_t)stream>>>(in6, n, out4);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}

// ---- training-sample candidates (Sec. 4.5 / App. I) ----
// A fraction surface_frac of the points lies on the scene's surfaces with the surface normal
// as direction, spread over the surfaces in proportion to area; the rest is uniform in the
// room with directions uniform on the sphere.  The surfaces ("patches"), in order: the room
// walls (axis 0..2, the wall at room_min first, normals into the room; the ceiling cut into
// the strips around the open skylight: x <= x0, x >= x1, (x0..x1, z <= z0), (x0..x1, z >= z1),
// empty strips left out), the spheres that do not emit (rest position), then the box faces
// (axis 0..2, the face at the low corner first, outward normals).  Sample j = index_base + i
// draws Philox at counters (j lo, j hi, 0x53414D50, 0 and 1) with key (seed lo, seed hi).
namespace {

constexpr int kMaxPatches = 352;
constexpr uint32_t kSampleTag = 0x53414D50u;

struct SamplePatches {
    int count;
    float lo[3], hi[3];
    float cdf[kMaxPatches];    // cumulative area fractions (FP64 sums rounded to FP32), last = 1
    float4 geo0[kMaxPatches];  // rectangle: (0, axis, normal sign, plane); sphere: (1, 0, 0, 0)
    float4 geo1[kMaxPatches];  // rectangle: (a0, a1, b0, b1) along the two other axes; sphere: (c, r)
};

// u in (0, 1) from 24 bits: float(x >> 8) 2^-24 + 2^-25, the product exact, one rounding.
__device__ __forceinline__ float sample_u(uint32_t x) {
    return __fadd_rn(__fmul_rn((float)(x >> 8), 1.0f / 16777216.0f), 1.0f / 33554432.0f);
}

// lo + (hi - lo) u in FP32, each operation rounded once.
__device__ __forceinline__ float sample_span(float lo, float hi, float u) {
    return __fadd_rn(lo, __fmul_rn(__fsub_rn(hi, lo), u));
}

// Uniform direction on the sphere: z = 1 - 2u, phi = 2 pi v.
__device__ __forceinline__ float3 sample_sphere_dir(float u, float v) {
    const float z = __fsub_rn(1.0f, __fmul_rn(2.0f, u));
    const float s = sqrtf(fmaxf(0.0f, 1.0f - z * z));
    float sp, cp;
    sincospif(2.0f * v, &sp, &cp);
    return make_float3(s * cp, s * sp, z);
}

__global__ void __launch_bounds__(128) training_samples_kernel(SamplePatches P, int64_t n, float surface_frac,
                                                               uint64_t seed, uint64_t index_base, float4* __restrict__ x4,
                                                               float4* __restrict__ n4, float* __restrict__ tout,
                                                               int32_t* __restrict__ patch) {
    __shared__ float s_cdf[kMaxPatches];
    for (int k = threadIdx.x; k < P.count; k += blockDim.x) s_cdf[k] = P.cdf[k];
    __syncthreads();
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint64_t j = index_base + (uint64_t)i;
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    const uint4 ra = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)(j >> 32), kSampleTag, 0u), k0, k1);
    const uint4 rb = philox4x32_10(make_uint4((uint32_t)j, (uint32_t)(j >> 32), kSampleTag, 1u), k0, k1);
    float3 p, q;
    int which = -1;
    if (P.count > 0 && sample_u(ra.x) < surface_frac) {
        // first patch k with u < cdf[k] (the cdf does not decrease; the last entry is 1)
        const float u = sample_u(ra.y);
        int lo = 0, hi = P.count - 1;
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (u < s_cdf[mid]) hi = mid;
            else lo = mid + 1;
        }
        which = lo;
        const float4 g0 = P.geo0[lo], g1 = P.geo1[lo];
        if (g0.x == 0.0f) {
            const int axis = (int)g0.y;
            const float a = sample_span(g1.x, g1.y, sample_u(ra.z)), b = sample_span(g1.z, g1.w, sample_u(ra.w));
            // in-plane axes in increasing order
            p = axis == 0 ? make_float3(g0.w, a, b) : (axis == 1 ? make_float3(a, g0.w, b) : make_float3(a, b, g0.w));
            q = make_float3(axis == 0 ? g0.z : 0.0f, axis == 1 ? g0.z : 0.0f, axis == 2 ? g0.z : 0.0f);
        } else {
            q = sample_sphere_dir(sample_u(rb.x), sample_u(rb.y));
            p = make_float3(g1.x + g1.w * q.x, g1.y + g1.w * q.y, g1.z + g1.w * q.z);
        }
    } else {
        p = make_float3(sample_span(P.lo[0], P.hi[0], sample_u(ra.y)), sample_span(P.lo[1], P.hi[1], sample_u(ra.z)),
                        sample_span(P.lo[2], P.hi[2], sample_u(ra.w)));
        q = sample_sphere_dir(sample_u(rb.x), sample_u(rb.y));
    }
    x4[i] = make_float4(p.x, p.y, p.z, 0.0f);
    n4[i] = make_float4(q.x, q.y, q.z, 0.0f);
    if (tout) tout[i] = sample_u(rb.z);
    if (patch) patch[i] = which;
}

// The patch table of a scene description (host); false if it does not fit.
bool build_patches(const float* blob, SamplePatches& P) {
    memset(&P, 0, sizeof P);
    const int ns = (int)blob[0], nb = (int)blob[1];
    double area[kMaxPatches];
    int k = 0;
    auto add_rect = [&](int axis, float sign, float plane, float a0, float a1, float b0, float b1) {
        if (k >= kMaxPatches) return false;
        P.geo0[k] = make_float4(0.0f, (float)axis, sign, plane);
        P.geo1[k] = make_float4(a0, a1, b0, b1);
        area[k] = ((double)a1 - (double)a0) * ((double)b1 - (double)b0);
        ++k;
        return true;
    };
    for (int d = 0; d < 3; ++d) {
        P.lo[d] = blob[4 + d];
        P.hi[d] = blob[7 + d];
    }
    if (blob[2] != 0.0f) {
        const float sx0 = blob[13], sx1 = blob[14], sz0 = blob[15], sz1 = blob[16];
        for (int axis = 0; axis < 3; ++axis) {
            const int a = axis == 0 ? 1 : 0, b = axis == 2 ? 1 : 2;
            if (!add_rect(axis, 1.0f, P.lo[axis], P.lo[a], P.hi[a], P.lo[b], P.hi[b])) return false;
            if (axis == 1 && sx0 < sx1) {  // the ceiling around the skylight (a = x, b = z)
                if (sx0 > P.lo[0] && !add_rect(1, -1.0f, P.hi[1], P.lo[0], sx0, P.lo[2], P.hi[2])) return false;
                if (P.hi[0] > sx1 && !add_rect(1, -1.0f, P.hi[1], sx1, P.hi[0], P.lo[2], P.hi[2])) return false;
                if (sz0 > P.lo[2] && !add_rect(1, -1.0f, P.hi[1], sx0, sx1, P.lo[2], sz0)) return false;
                if (P.hi[2] > sz1 && !add_rect(1, -1.0f, P.hi[1], sx0, sx1, sz1, P.hi[2])) return false;
            } else if (!add_rect(axis, -1.0f, P.hi[axis], P.lo[a], P.hi[a], P.lo[b], P.hi[b])) {
                return false;
            }
        }
    }
    const float* sph = blob + kHdr;
    for (int i = 0; i < ns; ++i) {
        const float* s = sph + kSph * i;
        if (s[7] > 0.0f || s[8] > 0.0f || s[9] > 0.0f) continue;  // emitters are not shaded
        if (k >= kMaxPatches) return false;
        P.geo0[k] = make_float4(1.0f, 0.0f, 0.0f, 0.0f);
        P.geo1[k] = make_float4(s[0], s[1], s[2], s[3]);
        area[k] = 4.0 * 3.141592653589793 * (double)s[3] * (double)s[3];
        ++k;
    }
    const float* box = sph + kSph * ns;
    for (int i = 0; i < nb; ++i) {
        const float* bl = box + kBox * i;
        for (int axis = 0; axis < 3; ++axis) {
            const int a = axis == 0 ? 1 : 0, b = axis == 2 ? 1 : 2;
            if (!add_rect(axis, -1.0f, bl[axis], bl[a], bl[3 + a], bl[b], bl[3 + b])) return false;
            if (!add_rect(axis, 1.0f, bl[3 + axis], bl[a], bl[3 + a], bl[b], bl[3 + b])) return false;
        }
    }
    double total = 0.0, acc = 0.0;
    for (int i = 0; i < k; ++i) total += area[i];
    for (int i = 0; i < k; ++i) {
        acc += area[i];
        P.cdf[i] = (float)(acc / total);
    }
    if (k > 0) P.cdf[k - 1] = 1.0f;
    P.count = k;
    return true;
}

}  // namespace

extern "C" int niv_training_samples(const float* scene, int64_t scene_len, int64_t n, float surface_frac,
                                    uint64_t seed, uint64_t index_base, float* x4, float* n4, float* t,
                                    int32_t* patch, niv_stream stream) {
    if (!scene) return niv_fail(NIV_ERR_ARG, "scene is NULL");
    if (n < 0) return niv_fail(NIV_ERR_ARG, "n < 0");
    if (!(surface_frac >= 0.0f && surface_frac <= 1.0f)) return niv_fail(NIV_ERR_ARG, "surface_frac outside [0, 1]");
    const int ns = (int)scene[0], nb = (int)scene[1];
    if (ns < 0 || nb < 0 || ns + nb > kMaxObjects) return niv_fail(NIV_ERR_UNSUPPORTED, "at most 56 scene objects");
    if (scene_len != kHdr + kSph * ns + kBox * nb) return niv_fail(NIV_ERR_ARG, "scene description length mismatch");
    if (n == 0) return NIV_OK;
    if (!x4 || !n4) return niv_fail(NIV_ERR_ARG, "NULL output");
    if (((uintptr_t)x4 | (uintptr_t)n4) & 15u) return niv_fail(NIV_ERR_ALIGN, "records must be 16-byte aligned");
    SamplePatches P;
    if (!build_patches(scene, P)) return niv_fail(NIV_ERR_UNSUPPORTED, "more surface patches than the sampler holds");
    const int64_t blocks = (n + 127) / 128;
    if (blocks > 0x7FFFFFFF) return niv_fail(NIV_ERR_ARG, "n too large");
    training_samples_kernel<<<(unsigned)blocks, 128, 0, (cudaStream_t)stream>>>(
        P, n, surface_frac, seed, index_base, reinterpret_cast<float4*>(x4), reinterpret_cast<float4*>(n4), t, patch);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}
