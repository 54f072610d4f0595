// Half-resolution rendering (Sec. 4.4, Table 1 "half"): irradiance queried at every
// sub-th pixel of every sub-th row is brought back to full resolution by joint
// bilateral upsampling (Kopf et al. 2007) guided by the full-resolution G-buffer,
// and shaded in the same pass with the full-resolution albedo and direct light:
//   samples q of pixel p: the (up to) four low-resolution neighbours, bilinear weight b_q;
//   g_q = max(0, n_p . n_q)^power * exp(-((n_p . (x_q - x_p)) / sigma)^2);
//   E_p = sum b_q (g_q + eps) E_q / sum b_q (g_q + eps);
//   rgba_p = (albedo_p E_p / pi + direct_p, 1) in FP16.
// One thread per full-resolution pixel, 32 x 8 pixel CTA tiles on a 2-D grid; the
// samples' G-buffer records are pixels of the same tile neighbourhood (cache hits).
// The pass streams 40 B per pixel (four 8-byte FP16 records in, one out) plus the
// low-resolution E: HBM-bound.
#include "niv_internal.cuh"

namespace {

constexpr int kTX = 32, kTY = 8;

struct UpArgs {
    const void* pos;
    const void* nrm;
    const void* alb;
    const void* dir;
    const void* E;
    void* out;
    int32_t W, H, w, h, sub, in_f16, e_f16;
    float inv_sub, power, inv_sigma, eps;
};

__global__ void __launch_bounds__(kTX * kTY) upsample_shade_kernel(UpArgs a) {
    const int X = blockIdx.x * kTX + (threadIdx.x % kTX), Y = blockIdx.y * kTY + threadIdx.x / kTX;
    if (X >= a.W || Y >= a.H) return;
    const int64_t p = (int64_t)Y * a.W + X;
    const float4 xp = niv_load_rec(a.pos, p, a.in_f16);
    const float4 np_ = niv_load_rec(a.nrm, p, a.in_f16);
    const int i0 = X / a.sub, j0 = Y / a.sub;
    const int i1 = min(i0 + 1, a.w - 1), j1 = min(j0 + 1, a.h - 1);
    const float fx = (float)(X - a.sub * i0) * a.inv_sub, fy = (float)(Y - a.sub * j0) * a.inv_sub;
    float sw = 0.0f, e0 = 0.0f, e1 = 0.0f, e2 = 0.0f;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float b = ((c & 1) ? fx : 1.0f - fx) * ((c & 2) ? fy : 1.0f - fy);
        if (b == 0.0f) continue;  // on a sample row / column: the far neighbour has no weight
        const int qi = (c & 1) ? i1 : i0, qj = (c & 2) ? j1 : j0;
        const int64_t src = (int64_t)(a.sub * qj) * a.W + (int64_t)a.sub * qi;
        const float4 xq = niv_load_rec(a.pos, src, a.in_f16);
        const float4 nq = niv_load_rec(a.nrm, src, a.in_f16);
        const float dot = np_.x * nq.x + np_.y * nq.y + np_.z * nq.z;
        const float dpl = np_.x * (xq.x - xp.x) + np_.y * (xq.y - xp.y) + np_.z * (xq.z - xp.z);
        const float r = dpl * a.inv_sigma;
        const float g = powf(fmaxf(dot, 0.0f), a.power) * expf(-r * r);
        const float wq = b * (g + a.eps);
        const float4 E = niv_load_rec(a.E, (int64_t)qj * a.w + qi, a.e_f16);
        sw += wq;
        e0 = fmaf(wq, E.x, e0);
        e1 = fmaf(wq, E.y, e1);
        e2 = fmaf(wq, E.z, e2);
    }
    const float inv = 1.0f / sw;
    const float4 al = niv_load_rec(a.alb, p, true), di = niv_load_rec(a.dir, p, true);
    const float inv_pi = 0.318309886183790671538f;
    __half2 rg = __floats2half2_rn(fmaf(al.x * (e0 * inv), inv_pi, di.x), fmaf(al.y * (e1 * inv), inv_pi, di.y));
    __half2 ba = __floats2half2_rn(fmaf(al.z * (e2 * inv), inv_pi, di.z), 1.0f);
    uint2 o;
    o.x = *reinterpret_cast<uint32_t*>(&rg);
    o.y = *reinterpret_cast<uint32_t*>(&ba);
    reinterpret_cast<uint2*>(a.out)[p] = o;
}

}  // namespace

int niv_launch_upsample_shade(const void* pos, const void* nrm, const void* albedo, const void* direct, int32_t width,
                              int32_t height, int32_t in_f16, const void* E_low, int32_t e_f16, int32_t sub, float power,
                              float sigma, float eps, void* out, cudaStream_t s) {
    UpArgs a;
    a.pos = pos;
    a.nrm = nrm;
    a.alb = albedo;
    a.dir = direct;
    a.E = E_low;
    a.out = out;
    a.W = width;
    a.H = height;
    a.sub = sub;
    a.w = (width + sub - 1) / sub;
    a.h = (height + sub - 1) / sub;
    a.in_f16 = in_f16;
    a.e_f16 = e_f16;
    a.inv_sub = 1.0f / (float)sub;
    a.power = power;
    a.inv_sigma = 1.0f / sigma;
    a.eps = eps;
    const dim3 grid((unsigned)((width + kTX - 1) / kTX), (unsigned)((height + kTY - 1) / kTY));
    if (grid.y > 65535u) return niv_fail(NIV_ERR_UNSUPPORTED, "image too tall");
    upsample_shade_kernel<<<grid, kTX * kTY, 0, s>>>(a);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}
