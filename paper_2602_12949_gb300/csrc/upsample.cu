// Half-resolution rendering (Sec. 4.4, Table 1 "half"): irradiance queried at every
// sub-th pixel of every sub-th row is brought back to full resolution by joint
// bilateral upsampling (Kopf et al. 2007) guided by the full-resolution G-buffer,
// and shaded in the same pass with the full-resolution albedo and direct light:
//   samples q of pixel p: the (up to) four low-resolution neighbours, bilinear weight b_q;
//   g_q = max(0, n_p . n_q)^power * exp(-((n_p . (x_q - x_p)) / sigma)^2);
//   E_p = sum b_q (g_q + eps) E_q / sum b_q (g_q + eps);
//   rgba_p = (albedo_p E_p / pi + direct_p, 1) in FP16.
// sub = 2 (half resolution) with FP16 records and an even width: one thread per 2 x 2
// pixel quad, i.e. per low-resolution sample, on a tile staged in shared memory (below);
// the quad's four pixels share the same four samples.  Its top-left pixel is the sample
// itself (E taken as is); the other three blend 2, 2 and 4 samples.  Otherwise one thread
// per pixel on 32 x 8 pixel tiles.  The pass streams 40 B per pixel (four 8-byte FP16
// records in, one out) plus the low-resolution E: HBM-bound.
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

// Range term of sample q for pixel p: max(0, n_p . n_q)^power * exp(-((n_p . (x_q - x_p)) / sigma)^2),
// with the power as exp2(power * log2(dot)) and the Gaussian through the fast exponential.
__device__ __forceinline__ float range_term(const float4& xp, const float4& np_, const float4& xq, const float4& nq,
                                            float power, float inv_sigma) {
    const float dot = np_.x * nq.x + np_.y * nq.y + np_.z * nq.z;
    const float dpl = np_.x * (xq.x - xp.x) + np_.y * (xq.y - xp.y) + np_.z * (xq.z - xp.z);
    const float r = dpl * inv_sigma;
    const float gn = power == 0.0f ? 1.0f : (dot > 0.0f ? exp2f(power * __log2f(dot)) : 0.0f);
    return gn * __expf(-r * r);
}

__device__ __forceinline__ uint2 shade_rgba(const float4& al, const float4& di, float e0, float e1, float e2) {
    const float inv_pi = 0.318309886183790671538f;
    __half2 rg = __floats2half2_rn(fmaf(al.x * e0, inv_pi, di.x), fmaf(al.y * e1, inv_pi, di.y));
    __half2 ba = __floats2half2_rn(fmaf(al.z * e2, inv_pi, di.z), 1.0f);
    uint2 o;
    o.x = *reinterpret_cast<uint32_t*>(&rg);
    o.y = *reinterpret_cast<uint32_t*>(&ba);
    return o;
}

// Any sub / dtype / width: one thread per full-resolution pixel on 32 x 8 pixel tiles.
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
        const float wq = b * (range_term(xp, np_, xq, nq, a.power, a.inv_sigma) + a.eps);
        const float4 E = niv_load_rec(a.E, (int64_t)qj * a.w + qi, a.e_f16);
        sw += wq;
        e0 = fmaf(wq, E.x, e0);
        e1 = fmaf(wq, E.y, e1);
        e2 = fmaf(wq, E.z, e2);
    }
    const float inv = 1.0f / sw;
    const float4 al = niv_load_rec(a.alb, p, true), di = niv_load_rec(a.dir, p, true);
    reinterpret_cast<uint2*>(a.out)[p] = shade_rgba(al, di, e0 * inv, e1 * inv, e2 * inv);
}

// ---- sub = 2, FP16 records, even width: tile staged in shared memory ----
// One CTA per 64 x 16 pixel tile = 32 x 8 quads = the tile's low-resolution samples; one
// thread per quad.  Phase 1 copies the tile's pos / nrm / albedo / direct rows, the halo
// (pixel row 16 and pixel column 64: the samples of the next tiles) and the 33 x 9
// low-resolution E records into shared memory with cp.async (every copy in flight at
// once, no registers held); phase 2 computes from shared memory.  Out-of-image pixels
// are zero-filled and never used (the sample indices are clamped to the image).
constexpr int kTW = 64, kTH = 16, kQW = kTW / 2, kQH = kTH / 2;
constexpr int kPW = kTW + 2;  // pos / nrm row pitch in records (column 64 = halo, 65 = pad)

struct StagedTile {
    uint2 pos[kTH + 1][kPW];
    uint2 nrm[kTH + 1][kPW];
    uint2 alb[kTH][kTW];
    uint2 dir[kTH][kTW];
    uint2 E[kQH + 1][kQW + 1];
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src, bool ok) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 16 : 0)
                 : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src, bool ok) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
                 "l"(src), "r"(ok ? 8 : 0)
                 : "memory");
}

__device__ __forceinline__ float4 h4(uint2 r) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&r.y));
    return make_float4(a.x, a.y, b.x, b.y);
}

#ifndef NIV_UP_MINB
#define NIV_UP_MINB 4
#endif
__global__ void __launch_bounds__(kQW * kQH, NIV_UP_MINB) upsample2_staged_kernel(UpArgs a) {
    extern __shared__ __align__(16) uint8_t smem_raw[];
    StagedTile& t = *reinterpret_cast<StagedTile*>(smem_raw);
    const int tid = threadIdx.x;
    const int X0 = blockIdx.x * kTW, Y0 = blockIdx.y * kTH, qx0 = X0 / 2, qy0 = Y0 / 2;
    const uint2* gpos = reinterpret_cast<const uint2*>(a.pos);
    const uint2* gnrm = reinterpret_cast<const uint2*>(a.nrm);
    const uint2* galb = reinterpret_cast<const uint2*>(a.alb);
    const uint2* gdir = reinterpret_cast<const uint2*>(a.dir);
    const uint2* gE = reinterpret_cast<const uint2*>(a.E);
    // rows 0..16 of pos / nrm and rows 0..15 of albedo / direct in 16-byte chunks (2 pixels):
    // thread (column pair tid % 32, row tid / 32) copies rows r, r + 8 (and 16 for r = 0)
    {
        const int cc = 2 * (tid % kQW), r0 = tid / kQW, X = X0 + cc;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const int row = r0 + kQH * k;
            if (row > kTH) break;
            const int Y = Y0 + row;
            const bool ok = X < a.W && Y < a.H;  // W is even: both pixels of the chunk are inside
            const int64_t g = ok ? (int64_t)Y * a.W + X : 0;
            cp_async16(&t.pos[row][cc], gpos + g, ok);
            cp_async16(&t.nrm[row][cc], gnrm + g, ok);
            if (row < kTH) {
                cp_async16(&t.alb[row][cc], galb + g, ok);
                cp_async16(&t.dir[row][cc], gdir + g, ok);
            }
        }
    }
    // pixel column 64 of pos / nrm (rows 0..16)
    if (tid < 2 * (kTH + 1)) {
        const int buf = tid / (kTH + 1), row = tid % (kTH + 1);
        const int X = X0 + kTW, Y = Y0 + row;
        const bool ok = X < a.W && Y < a.H;
        const int64_t g = ok ? (int64_t)Y * a.W + X : 0;
        cp_async8(buf == 0 ? &t.pos[row][kTW] : &t.nrm[row][kTW], (buf == 0 ? gpos : gnrm) + g, ok);
    }
    // low-resolution E of samples qx0..qx0+32, qy0..qy0+8
    for (int c = tid; c < (kQH + 1) * (kQW + 1); c += kQW * kQH) {
        const int r = c / (kQW + 1), q = c % (kQW + 1);
        const bool ok = qx0 + q < a.w && qy0 + r < a.h;
        const int64_t g = ok ? (int64_t)(qy0 + r) * a.w + qx0 + q : 0;
        cp_async8(&t.E[r][q], gE + g, ok);
    }
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
    __syncthreads();

    const int lqx = tid % kQW, lqy = tid / kQW, qx = qx0 + lqx, qy = qy0 + lqy;
    if (qx >= a.w || qy >= a.h) return;
    const int px = 2 * lqx, py = 2 * lqy;                   // the quad's top-left pixel in the tile
    const bool has_r = X0 + px + 1 < a.W, has_b = Y0 + py + 1 < a.H;
    const int sx = 2 * (min(qx + 1, a.w - 1) - qx0), sy = 2 * (min(qy + 1, a.h - 1) - qy0);  // far samples
    const int ex = min(qx + 1, a.w - 1) - qx0, ey = min(qy + 1, a.h - 1) - qy0;
    const uint4 pr0 = *reinterpret_cast<const uint4*>(&t.pos[py][px]);
    const uint4 nr0 = *reinterpret_cast<const uint4*>(&t.nrm[py][px]);
    const float4 x0 = h4(make_uint2(pr0.x, pr0.y)), n0 = h4(make_uint2(nr0.x, nr0.y));
    const float4 E0 = h4(t.E[lqy][lqx]), E1 = h4(t.E[lqy][ex]), E2 = h4(t.E[ey][lqx]), E3 = h4(t.E[ey][ex]);
    const float4 xs1 = h4(t.pos[py][sx]), ns1 = h4(t.nrm[py][sx]);
    const float4 xs2 = h4(t.pos[sy][px]), ns2 = h4(t.nrm[sy][px]);
    const float4 xs3 = h4(t.pos[sy][sx]), ns3 = h4(t.nrm[sy][sx]);
    const uint4 al0 = *reinterpret_cast<const uint4*>(&t.alb[py][px]);
    const uint4 di0 = *reinterpret_cast<const uint4*>(&t.dir[py][px]);
    uint2 o0 = shade_rgba(h4(make_uint2(al0.x, al0.y)), h4(make_uint2(di0.x, di0.y)), E0.x, E0.y, E0.z), o1;
    if (has_r) {  // pixel (1, 0): samples 0 and 1, bilinear 1/2 each
        const float4 x1 = h4(make_uint2(pr0.z, pr0.w)), n1 = h4(make_uint2(nr0.z, nr0.w));
        const float w0 = 0.5f * (range_term(x1, n1, x0, n0, a.power, a.inv_sigma) + a.eps);
        const float w1 = 0.5f * (range_term(x1, n1, xs1, ns1, a.power, a.inv_sigma) + a.eps);
        const float inv = 1.0f / (w0 + w1);
        o1 = shade_rgba(h4(make_uint2(al0.z, al0.w)), h4(make_uint2(di0.z, di0.w)),
                        fmaf(w1, E1.x, w0 * E0.x) * inv, fmaf(w1, E1.y, w0 * E0.y) * inv,
                        fmaf(w1, E1.z, w0 * E0.z) * inv);
    }
    uint2* out = reinterpret_cast<uint2*>(a.out);
    const int64_t g0 = (int64_t)(Y0 + py) * a.W + X0 + px;
    if (has_r)
        *reinterpret_cast<uint4*>(out + g0) = make_uint4(o0.x, o0.y, o1.x, o1.y);
    else
        out[g0] = o0;
    if (!has_b) return;
    const uint4 pr1 = *reinterpret_cast<const uint4*>(&t.pos[py + 1][px]);
    const uint4 nr1 = *reinterpret_cast<const uint4*>(&t.nrm[py + 1][px]);
    const uint4 al1 = *reinterpret_cast<const uint4*>(&t.alb[py + 1][px]);
    const uint4 di1 = *reinterpret_cast<const uint4*>(&t.dir[py + 1][px]);
    uint2 o2, o3;
    {  // pixel (0, 1): samples 0 and 2
        const float4 x2 = h4(make_uint2(pr1.x, pr1.y)), n2 = h4(make_uint2(nr1.x, nr1.y));
        const float w0 = 0.5f * (range_term(x2, n2, x0, n0, a.power, a.inv_sigma) + a.eps);
        const float w2 = 0.5f * (range_term(x2, n2, xs2, ns2, a.power, a.inv_sigma) + a.eps);
        const float inv = 1.0f / (w0 + w2);
        o2 = shade_rgba(h4(make_uint2(al1.x, al1.y)), h4(make_uint2(di1.x, di1.y)),
                        fmaf(w2, E2.x, w0 * E0.x) * inv, fmaf(w2, E2.y, w0 * E0.y) * inv,
                        fmaf(w2, E2.z, w0 * E0.z) * inv);
    }
    const int64_t g1 = g0 + a.W;
    if (!has_r) {
        out[g1] = o2;
        return;
    }
    {  // pixel (1, 1): all four samples, 1/4 each
        const float4 x3 = h4(make_uint2(pr1.z, pr1.w)), n3 = h4(make_uint2(nr1.z, nr1.w));
        const float w0 = 0.25f * (range_term(x3, n3, x0, n0, a.power, a.inv_sigma) + a.eps);
        const float w1 = 0.25f * (range_term(x3, n3, xs1, ns1, a.power, a.inv_sigma) + a.eps);
        const float w2 = 0.25f * (range_term(x3, n3, xs2, ns2, a.power, a.inv_sigma) + a.eps);
        const float w3 = 0.25f * (range_term(x3, n3, xs3, ns3, a.power, a.inv_sigma) + a.eps);
        const float inv = 1.0f / ((w0 + w1) + (w2 + w3));
        const float e0 = fmaf(w3, E3.x, fmaf(w2, E2.x, fmaf(w1, E1.x, w0 * E0.x)));
        const float e1 = fmaf(w3, E3.y, fmaf(w2, E2.y, fmaf(w1, E1.y, w0 * E0.y)));
        const float e2 = fmaf(w3, E3.z, fmaf(w2, E2.z, fmaf(w1, E1.z, w0 * E0.z)));
        o3 = shade_rgba(h4(make_uint2(al1.z, al1.w)), h4(make_uint2(di1.z, di1.w)), e0 * inv, e1 * inv, e2 * inv);
    }
    *reinterpret_cast<uint4*>(out + g1) = make_uint4(o2.x, o2.y, o3.x, o3.y);
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
    if (sub == 2 && in_f16 && e_f16 && (width & 1) == 0) {
        const dim3 grid((unsigned)((width + kTW - 1) / kTW), (unsigned)((height + kTH - 1) / kTH));
        if (grid.y > 65535u) return niv_fail(NIV_ERR_UNSUPPORTED, "image too tall");
        upsample2_staged_kernel<<<grid, kQW * kQH, sizeof(StagedTile), s>>>(a);
    } else {
        const dim3 grid((unsigned)((width + kTX - 1) / kTX), (unsigned)((height + kTY - 1) / kTY));
        if (grid.y > 65535u) return niv_fail(NIV_ERR_UNSUPPORTED, "image too tall");
        upsample_shade_kernel<<<grid, kTX * kTY, 0, s>>>(a);
    }
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}
