// SH probe-grid query (Sec. 5.1, App. A): the non-neural path beside the NIV query.
//
// Per record: the 8 probes of the lattice cell around x, trilinear weights times the
// cosine fall-off max(0, n . normalize(p_probe - x)) (a probe exactly at x keeps 1),
// each clamped below at 1e-6, then renormalised; every probe contributes its SH
// irradiance E(n) = sum_l A_l sum_m L_lm Y_lm(n) with A = (pi, 2 pi / 3, pi / 4)
// (Ramamoorthi & Hanrahan 2001).  Coefficients are FP16, 27 per probe padded to 28
// (56 bytes, so a probe is seven 8-byte loads); arithmetic is FP32.
//
// "+RT" (Sec. 5.1, App. A): visibility-based probe rejection by ray tracing replaces the
// cosine fall-off.  Reading: a shadow ray from x + 0.01 n (world units) toward each probe;
// the probe is rejected (weight 0, then the 1e-6 clamp) when the ray hits scene geometry
// more than 0.01 short of the probe.  The scene is the analytic one of the training
// targets (scene.cuh), at scene parameter t.
#include "niv_internal.cuh"
#include "scene.cuh"

namespace {

struct ProbeArgs {
    int32_t P[3];
    float lo[3], hi[3];
    float inv_cell[3];  // (P - 1) / (hi - lo)
    float cell[3];      // (hi - lo) / (P - 1)
};

__device__ __forceinline__ float sh_irr(const float* c, float3 n, int ch) {
    // coefficient q of channel ch is c[3 q + ch]
    const float x = n.x, y = n.y, z = n.z;
    const float a0 = 3.141592653589793f * 0.28209479177387814f;
    const float a1 = 2.0943951023931953f * 0.4886025119029199f;
    const float a2 = 0.7853981633974483f;
    const float c2 = 1.0925484305920792f, c20 = 0.31539156525252005f, c22 = 0.5462742152960396f;
    return a0 * c[ch] + a1 * (c[3 + ch] * y + c[6 + ch] * z + c[9 + ch] * x) +
           a2 * (c2 * (c[12 + ch] * x * y + c[15 + ch] * y * z + c[21 + ch] * x * z) +
                 c20 * c[18 + ch] * (3.0f * z * z - 1.0f) + c22 * c[24 + ch] * (x * x - y * y));
}

constexpr float kRayBias = 0.01f;  // shadow-ray origin offset along n
constexpr float kRayEnd = 0.01f;   // hits this close to the probe do not reject it

template <bool VIS>
__global__ void __launch_bounds__(128) probe_query_kernel(const uint2* __restrict__ coef, ProbeArgs pa, IoArgs io,
                                                          int64_t n_tiles, SceneArg scene, float t) {
    __shared__ float s_scene[VIS ? kHdr + kSph * kMaxObjects : 1];
    SceneView S;
    if (VIS) {
        const int len = kHdr + kSph * ((int)scene.v[0] + (int)scene.v[1]);
        for (int k = threadIdx.x; k < len; k += blockDim.x) s_scene[k] = scene.v[k];
        __syncthreads();
        S.init(s_scene, t);
    }
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t r = niv_record_of(tile, threadIdx.x, io.n, io.image_width);
        if (r >= io.n) continue;
        const float4 p = niv_load_rec(io.pos, r, io.in_f16);
        const float4 nv = niv_load_rec(io.nrm, r, io.in_f16);
        const float nl = rsqrtf(nv.x * nv.x + nv.y * nv.y + nv.z * nv.z);
        const float3 n = make_float3(nv.x * nl, nv.y * nl, nv.z * nl);
        const float xs[3] = {p.x, p.y, p.z};
        int base[3];
        float f[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            const float g = fminf(fmaxf((xs[a] - pa.lo[a]) * pa.inv_cell[a], 0.0f), (float)(pa.P[a] - 1));
            const int i = min((int)floorf(g), pa.P[a] - 2);
            base[a] = i;
            f[a] = g - (float)i;
        }
        float acc[3] = {0.0f, 0.0f, 0.0f}, wsum = 0.0f;
#pragma unroll
        for (int c = 0; c < 8; ++c) {
            int ijk[3];
            float w = 1.0f;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const int bit = (c >> a) & 1;
                ijk[a] = base[a] + bit;
                w *= bit ? f[a] : 1.0f - f[a];
            }
            const int64_t pi = ijk[0] + (int64_t)pa.P[0] * (ijk[1] + (int64_t)pa.P[1] * ijk[2]);
            const float dx = pa.lo[0] + pa.cell[0] * ijk[0] - xs[0];
            const float dy = pa.lo[1] + pa.cell[1] * ijk[1] - xs[1];
            const float dz = pa.lo[2] + pa.cell[2] * ijk[2] - xs[2];
            if (VIS) {
                const float3 o = make_float3(xs[0] + kRayBias * n.x, xs[1] + kRayBias * n.y, xs[2] + kRayBias * n.z);
                const float3 dv = make_float3(pa.lo[0] + pa.cell[0] * ijk[0] - o.x, pa.lo[1] + pa.cell[1] * ijk[1] - o.y,
                                              pa.lo[2] + pa.cell[2] * ijk[2] - o.z);
                const float dist = sqrtf(dot3(dv, dv));
                bool visible = true;
                if (dist > 0.0f) {
                    const float3 d = make_float3(dv.x / dist, dv.y / dist, dv.z / dist);
                    visible = !S.occluded(o, d, dist - kRayEnd);
                }
                w = fmaxf(visible ? w : 0.0f, 1e-6f);
            } else {
                const float dl = sqrtf(dx * dx + dy * dy + dz * dz);
                const float fall = dl > 0.0f ? fmaxf((dx * n.x + dy * n.y + dz * n.z) / dl, 0.0f) : 1.0f;
                w = fmaxf(w * fall, 1e-6f);
            }
            float cf[28];
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                const uint2 v = __ldg(coef + pi * 7 + q);
                const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&v.x));
                const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&v.y));
                cf[4 * q] = a.x;
                cf[4 * q + 1] = a.y;
                cf[4 * q + 2] = b.x;
                cf[4 * q + 3] = b.y;
            }
#pragma unroll
            for (int ch = 0; ch < 3; ++ch) acc[ch] = fmaf(w, sh_irr(cf, n, ch), acc[ch]);
            wsum += w;
        }
        const float inv = 1.0f / wsum;
        niv_store_rec(io.out, r, acc[0] * inv, acc[1] * inv, acc[2] * inv, io.out_f16);
    }
}

}  // namespace

int niv_launch_probe_query(const void* coef16, const int* P, const float* lo, const float* hi, const IoArgs& io,
                           const float* scene, int64_t scene_len, float t, cudaStream_t s) {
    SceneArg arg;
    if (scene && !niv_scene_arg(scene, scene_len, arg))
        return niv_fail(NIV_ERR_ARG, "scene description invalid (at most 56 objects, length as its header says)");
    ProbeArgs pa;
    for (int a = 0; a < 3; ++a) {
        pa.P[a] = P[a];
        pa.lo[a] = lo[a];
        pa.hi[a] = hi[a];
        pa.inv_cell[a] = (float)((double)(P[a] - 1) / ((double)hi[a] - (double)lo[a]));
        pa.cell[a] = (float)(((double)hi[a] - (double)lo[a]) / (double)(P[a] - 1));
    }
    int dev = 0, sms = 0;
    NIV_CUDA(cudaGetDevice(&dev));
    NIV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    const int64_t tiles = niv_tile_count_host(io.n, io.image_width);
    const int64_t cap = (int64_t)sms * 16;
    const int64_t blocks = tiles < cap ? tiles : cap;
    if (scene)
        probe_query_kernel<true><<<(unsigned)blocks, 128, 0, s>>>((const uint2*)coef16, pa, io, tiles, arg, t);
    else
        probe_query_kernel<false><<<(unsigned)blocks, 128, 0, s>>>((const uint2*)coef16, pa, io, tiles, arg, t);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}
