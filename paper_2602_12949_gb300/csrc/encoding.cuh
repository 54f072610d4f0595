// Kernel-side definitions every query kernel shares: the per-call argument blocks and the
// encoding, record and tile helpers (Sec. 4.1 encoding, Sec. 4.4 G-buffer records).
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>

#define NIV_MAX_LEVELS 32
#define NIV_MAX_IN 132  // levels * feat + in_extra upper bound for the plain path

// Spatial-hash constants of the multi-resolution hash encoding adopted in Sec. 4.1
// (Mueller et al. 2022): pi_1 = 1, pi_2 = 2654435761, pi_3 = 805459861.
#define NIV_PI1 1u
#define NIV_PI2 2654435761u
#define NIV_PI3 805459861u

// Per-call description of the encoding, passed by value to the kernels.
struct GridArgs {
    int32_t dims, levels, feat, n_in;
    uint32_t hash_mask;  // T - 1
    uint32_t prime_t;
    uint32_t dense_mask;  // bit l set: level l is dense
    int32_t pe_bands;     // > 0: frequency encoding of the position (no grid levels)
    int32_t t_bands;      // > 0: the scene parameter enters as sin / cos of 2^b pi t after n
    float aabb_min[3];
    float inv_ext[3];
    float t;
    int32_t res[NIV_MAX_LEVELS];
    uint32_t offset[NIV_MAX_LEVELS];  // first entry of each level
    // per-level constants in the form the encoders use them (read as kernel-argument
    // operands, so no tile recomputes them): N and N - 1 as floats (exact), and for dense
    // levels the entry strides N + 1 and (N + 1)^2
    float res_f[NIV_MAX_LEVELS];
    float resm1_f[NIV_MAX_LEVELS];
    uint32_t stride1[NIV_MAX_LEVELS];
    uint32_t stride2[NIV_MAX_LEVELS];
    // the cell search without conversions (NIV_MAGIC_FLOOR): 2^23 + N - 1 as a float, and the
    // offsets that remove the 2^23 bias (0x4B000000 in the bit pattern) from the index terms:
    // dense levels -B (1 + S + S^2 (+ S^3)), the time prime -B pi_t (mod 2^32)
    float resm1_b[NIV_MAX_LEVELS];
    uint32_t dense_off[NIV_MAX_LEVELS];
    uint32_t prime_t_off;
};

#ifndef NIV_MAGIC_FLOOR
#define NIV_MAGIC_FLOOR 0
#endif
// Bit pattern of the float 2^23: a float 2^23 + i (0 <= i < 2^23) has the bits kNivBias + i.
constexpr uint32_t kNivBias = 0x4B000000u;

// Where a kernel finds its records and how it walks them.
struct IoArgs {
    const void* pos;
    const void* nrm;
    void* out;
    int64_t n;
    int32_t image_width;  // > 0: 2-D tile traversal of a row-major image
    int32_t in_f16;       // records are FP16 (else FP32)
    int32_t out_f16;
    // Fused shading (Eq. 2 + direct light): when albedo is set, out receives FP16
    // rgba = (albedo * E / pi + direct, 1) instead of E.  FP16 [n][4] records.
    const void* albedo = nullptr;
    const void* direct = nullptr;
    // Half-resolution rendering (Sec. 4.4): sub > 1 makes record r of the image_width-wide
    // output the pixel (sub x, sub y) of a src_width-wide full-resolution G-buffer, where
    // (x, y) is r's position in the output image.
    int32_t sub = 1;
    int32_t src_width = 0;
};

// G-buffer record read for output record r (see IoArgs::sub).
__device__ __forceinline__ int64_t niv_source_of(const IoArgs& io, int64_t r) {
    if (io.sub <= 1) return r;
    const int64_t y = r / io.image_width, x = r - y * io.image_width;
    return y * io.sub * io.src_width + x * io.sub;
}

// ---- device helpers shared by the query kernels ----

// u = clamp(fp32(fp32(p - lo) * inv), 0, 1): FP32 operations without contraction.
__device__ __forceinline__ float niv_unit(float p, float lo, float inv) {
    float x = __fmul_rn(__fsub_rn(p, lo), inv);
    return fminf(fmaxf(x, 0.0f), 1.0f);
}

// Frequency encoding (the models of Table 1 without grid levels): for a coordinate u of
// the normalised position and band b, (sin(2^b pi u), cos(2^b pi u)); 2^b u is exact in FP32.
__device__ __forceinline__ void niv_pe_pair(float u, int b, float& s, float& c) {
    sincospif(__fmul_rn(u, (float)(1 << b)), &s, &c);
}

// Multilinear weights of the 2^d corners from the per-axis fractions w1 (Sec. 4.1):
// products of per-axis factors (1 - w1, w1); corner c has offset bit d along dimension d.
template <int DIMS>
__device__ __forceinline__ void niv_level_weights(const float* w1, float* wc) {
    constexpr int NC = 1 << DIMS;
    float w0[DIMS];
#pragma unroll
    for (int d = 0; d < DIMS; ++d) w0[d] = 1.0f - w1[d];
    // Products in pairs on the packed FP32 pipe: each lane is an ordinary FP32 product,
    // so the weights are those of the scalar formulas.
    const float2 wy = make_float2(w0[1], w1[1]), wx = make_float2(w0[0], w1[0]);
    float2 wh[NC / 4];  // wh[q] = (w_y0 * w_rest_q, w_y1 * w_rest_q)
    wh[0] = __fmul2_rn(wy, make_float2(w0[2], w0[2]));
    wh[1] = __fmul2_rn(wy, make_float2(w1[2], w1[2]));
    if (DIMS == 4) {
        const float2 t0 = make_float2(w0[DIMS - 1], w0[DIMS - 1]), t1 = make_float2(w1[DIMS - 1], w1[DIMS - 1]);
        wh[2 % (NC / 4)] = __fmul2_rn(wh[0], t1);
        wh[3 % (NC / 4)] = __fmul2_rn(wh[1], t1);
        wh[0] = __fmul2_rn(wh[0], t0);
        wh[1] = __fmul2_rn(wh[1], t0);
    }
#pragma unroll
    for (int q = 0; q < NC / 4; ++q) {
        const float2 a = __fmul2_rn(wx, make_float2(wh[q].x, wh[q].x));
        const float2 b = __fmul2_rn(wx, make_float2(wh[q].y, wh[q].y));
        wc[4 * q] = a.x;
        wc[4 * q + 1] = a.y;
        wc[4 * q + 2] = b.x;
        wc[4 * q + 3] = b.y;
    }
}

// The cell of level l at normalised coordinate u (Sec. 4.1): per axis s = fp32(u N),
// i = min(floor(s), N - 1) and the fraction w1 = s - i (exact).  NIV_MAGIC_FLOOR: floor(s)
// from s + 2^23 rounded down (0 <= s <= N < 2^23 makes that 2^23 + floor(s) exactly), i kept
// with the bias kNivBias in its bits; the index terms below remove it.
template <int DIMS>
__device__ __forceinline__ void niv_level_cell(const GridArgs& g, int l, const float* u, uint32_t* ci, float* w1) {
    const float fN = g.res_f[l];
#pragma unroll
    for (int d = 0; d < DIMS; ++d) {
        const float s = __fmul_rn(u[d], fN);
        if (NIV_MAGIC_FLOOR) {
            const float tb = fminf(__fadd_rd(s, 8388608.0f), g.resm1_b[l]);
            ci[d] = __float_as_uint(tb);
            w1[d] = __fsub_rn(s, __fsub_rn(tb, 8388608.0f));
        } else {
            const float fl = fminf(floorf(s), g.resm1_f[l]);
            ci[d] = (uint32_t)(int)fl;
            w1[d] = __fsub_rn(s, fl);
        }
    }
}

// Corner entries of level l for the cell ci, with the per-corner work factored: per-axis index
// terms (dense strides or hash products) combined per corner.  Corner c has offset bit d along
// dimension d.  ND >= 0: the dense levels are exactly levels 0 .. ND-1, known at compile time
// (with the level unrolled, the dense / hashed choice then costs no branch).
template <int DIMS, int ND = -1>
__device__ __forceinline__ void niv_level_index(const GridArgs& g, int l, const uint32_t* ci, uint32_t* e) {
    constexpr int NC = 1 << DIMS;
    constexpr uint32_t kB = NIV_MAGIC_FLOOR ? kNivBias : 0u;
    if (ND >= 0 ? l < ND : ((g.dense_mask >> l) & 1u) != 0u) {
        const uint32_t S = g.stride1[l], S2 = g.stride2[l];
        uint32_t base = ci[2] * S2 + ci[1] * S + ci[0];
        if (DIMS == 4) base += ci[DIMS - 1] * S2 * S;
        if (NIV_MAGIC_FLOOR) base += g.dense_off[l];
        uint32_t oh[NC / 2];
        oh[0] = base;
        oh[1] = base + S;
        oh[2] = base + S2;
        oh[3] = base + S2 + S;
        if (DIMS == 4) {
#pragma unroll
            for (int q = 0; q < 4; ++q) oh[(q + 4) % (NC / 2)] = oh[q] + S2 * S;
        }
#pragma unroll
        for (int q = 0; q < NC / 2; ++q) {
            e[2 * q] = oh[q];
            e[2 * q + 1] = oh[q] + 1u;
        }
    } else {
        const uint32_t hy0 = ci[1] * NIV_PI2 + (0u - kB * NIV_PI2), hy1 = hy0 + NIV_PI2;
        const uint32_t hz0 = ci[2] * NIV_PI3 + (0u - kB * NIV_PI3), hz1 = hz0 + NIV_PI3;
        uint32_t hh[NC / 2];
        hh[0] = hy0 ^ hz0;
        hh[1] = hy1 ^ hz0;
        hh[2] = hy0 ^ hz1;
        hh[3] = hy1 ^ hz1;
        if (DIMS == 4) {
            const uint32_t ht0 = ci[DIMS - 1] * g.prime_t + (NIV_MAGIC_FLOOR ? g.prime_t_off : 0u),
                           ht1 = ht0 + g.prime_t;
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                hh[(q + 4) % (NC / 2)] = hh[q] ^ ht1;
                hh[q] = hh[q] ^ ht0;
            }
        }
        const uint32_t x0 = ci[0] - kB, x1 = ci[0] + (1u - kB), m = g.hash_mask;
#pragma unroll
        for (int q = 0; q < NC / 2; ++q) {
            e[2 * q] = (x0 ^ hh[q]) & m;
            e[2 * q + 1] = (x1 ^ hh[q]) & m;
        }
    }
}

// Corner entries of level l at normalised coordinate u and the per-axis fractions w1 (Sec. 4.1).
template <int DIMS, int ND = -1>
__device__ __forceinline__ void niv_level_entries(const GridArgs& g, int l, const float* u, uint32_t* e, float* w1) {
    uint32_t ci[DIMS];
    niv_level_cell<DIMS>(g, l, u, ci, w1);
    niv_level_index<DIMS, ND>(g, l, ci, e);
}

// Corner entries and multilinear weights of level l at normalised coordinate u.
template <int DIMS, int ND = -1>
__device__ __forceinline__ void niv_level_corners(const GridArgs& g, int l, const float* u, uint32_t* e,
                                                  float* wc) {
    float w1[DIMS];
    niv_level_entries<DIMS, ND>(g, l, u, e, w1);
    niv_level_weights<DIMS>(w1, wc);
}

// Raw feature words of the corners: F features of type TabT per entry.
template <int F, typename TabT>
struct NivRaw {
    using T = typename std::conditional<
        sizeof(TabT) == 2, typename std::conditional<F == 4, uint2, typename std::conditional<F == 2, uint32_t, unsigned short>::type>::type,
        typename std::conditional<F == 4, float4, typename std::conditional<F == 2, float2, float>::type>::type>::type;
};

template <int NC, int F, typename TabT>
__device__ __forceinline__ void niv_level_gather(const TabT* __restrict__ tab, const uint32_t* e,
                                                 typename NivRaw<F, TabT>::T* raw) {
    using R = typename NivRaw<F, TabT>::T;
#pragma unroll
    for (int c = 0; c < NC; ++c) raw[c] = __ldg(reinterpret_cast<const R*>(tab) + e[c]);
}

__device__ __forceinline__ void niv_unpack(uint32_t r, float* f) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&r));
    f[0] = a.x;
    f[1] = a.y;
}
__device__ __forceinline__ void niv_unpack(uint2 r, float* f) {
    niv_unpack(r.x, f);
    niv_unpack(r.y, f + 2);
}
__device__ __forceinline__ void niv_unpack(unsigned short r, float* f) { f[0] = __half2float(__ushort_as_half(r)); }
__device__ __forceinline__ void niv_unpack(float r, float* f) { f[0] = r; }
__device__ __forceinline__ void niv_unpack(float2 r, float* f) {
    f[0] = r.x;
    f[1] = r.y;
}
__device__ __forceinline__ void niv_unpack(float4 r, float* f) {
    f[0] = r.x;
    f[1] = r.y;
    f[2] = r.z;
    f[3] = r.w;
}

#ifndef NIV_BLEND_PAIRS
#define NIV_BLEND_PAIRS 1
#endif
// Two FP16 features per entry: both features of a corner in one packed FP32 FMA, each
// lane the scalar FMA of its feature in the same corner order.
#ifndef NIV_BLEND_SPLIT
#define NIV_BLEND_SPLIT 0
#endif
template <int NC>
__device__ __forceinline__ void niv_level_blend2(const uint32_t* raw, const float* wc, float* acc) {
    if (NIV_BLEND_SPLIT) {  // even and odd corners in two chains, added at the end (half the depth)
        float2 a = make_float2(0.0f, 0.0f), b = make_float2(0.0f, 0.0f);
#pragma unroll
        for (int c = 0; c < NC; c += 2) {
            a = __ffma2_rn(make_float2(wc[c], wc[c]), __half22float2(*reinterpret_cast<const __half2*>(&raw[c])), a);
            b = __ffma2_rn(make_float2(wc[c + 1], wc[c + 1]),
                           __half22float2(*reinterpret_cast<const __half2*>(&raw[c + 1])), b);
        }
        a = __fadd2_rn(a, b);
        acc[0] = a.x;
        acc[1] = a.y;
        return;
    }
    float2 a = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int c = 0; c < NC; ++c)
        a = __ffma2_rn(make_float2(wc[c], wc[c]), __half22float2(*reinterpret_cast<const __half2*>(&raw[c])), a);
    acc[0] = a.x;
    acc[1] = a.y;
}

#ifndef NIV_BLEND_LERP
#define NIV_BLEND_LERP 0
#endif
// Two FP16 features per entry, multilinear interpolation as nested lerps a + w (b - a) from the
// per-axis fractions w1 (the same interpolant as the corner-weight form, rounded differently):
// along x per corner pair (b - a from the FP16 value of b and the FP32 value of a in one mixed-
// precision add), then along y, z (and t), both features at once on the packed FP32 pipe.
__device__ __forceinline__ float niv_h2f(uint16_t h) {
    float f;
    asm("cvt.f32.f16 %0, %1;" : "=f"(f) : "h"(h));
    return f;
}
__device__ __forceinline__ float niv_h_minus(uint16_t b, float a) {  // fp32(b) - a, one rounding
    float d;
    asm("add.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(b), "f"(-a));
    return d;
}
template <int DIMS>
__device__ __forceinline__ void niv_level_lerp2(const uint32_t* raw, const float* w1, float* acc) {
    constexpr int NC = 1 << DIMS;
    float2 v[NC / 2];
#pragma unroll
    for (int q = 0; q < NC / 2; ++q) {
        const uint32_t a = raw[2 * q], b = raw[2 * q + 1];
        const float a0 = niv_h2f((uint16_t)(a & 0xFFFFu)), a1 = niv_h2f((uint16_t)(a >> 16));
        const float2 d = make_float2(niv_h_minus((uint16_t)(b & 0xFFFFu), a0), niv_h_minus((uint16_t)(b >> 16), a1));
        v[q] = __ffma2_rn(make_float2(w1[0], w1[0]), d, make_float2(a0, a1));
    }
#pragma unroll
    for (int d = 1; d < DIMS; ++d) {
        const int half = NC >> (d + 1);  // pairs along dimension d: entries q and q + ... (bit d-1 of q)
        const float2 wd = make_float2(w1[d], w1[d]);
#pragma unroll
        for (int q = 0; q < half; ++q) {
            const float2 lo = v[2 * q], hi = v[2 * q + 1];
            v[q] = __ffma2_rn(wd, __fadd2_rn(hi, make_float2(-lo.x, -lo.y)), lo);
        }
    }
    acc[0] = v[0].x;
    acc[1] = v[0].y;
}

template <int NC, int F, typename R>
__device__ __forceinline__ void niv_level_blend(const R* raw, const float* wc, float* acc) {
    if constexpr (NIV_BLEND_PAIRS && F == 2 && std::is_same<R, uint32_t>::value) {
        niv_level_blend2<NC>(raw, wc, acc);
        return;
    }
#pragma unroll
    for (int j = 0; j < F; ++j) acc[j] = 0.0f;
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        float f[F];
        niv_unpack(raw[c], f);
#pragma unroll
        for (int j = 0; j < F; ++j) acc[j] = fmaf(wc[c], f[j], acc[j]);
    }
}

// Interpolated features of level l from an FP16 table, as the fused query kernels take them:
// two features per entry in the nested-lerp form (NIV_BLEND_LERP), else corner weights.
// 0: off; 1: every model with two features per entry; 2: the 4-D models only (measured: 1%
// faster on config 3's 4-D grid, 2-5% slower on the 3-D config-1 grid)
#ifndef NIV_DENSE_PAIRS
#define NIV_DENSE_PAIRS 2
#endif
#ifndef NIV_WARP_COOP
#define NIV_WARP_COOP 0  // levels 0 .. NIV_WARP_COOP-1 try the warp-cooperative gather
#endif
// pair (optional, two FP16 features per entry, dense levels 0 .. ND-1 known at compile time):
// entry e of a dense level holds the words of entries e and e + 1, the two corners of a cell
// edge along x, so one 8-byte load serves both.
template <int DIMS, int F, int ND = -1>
__device__ __forceinline__ void niv_level_features16(const GridArgs& g, const __half* __restrict__ tab, int l,
                                                     const float* u, float* acc, const uint2* __restrict__ pair = nullptr) {
    constexpr int NC = 1 << DIMS;
    using R = typename NivRaw<F, __half>::T;
    uint32_t e[NC];
    R raw[NC];
    if constexpr (NIV_WARP_COOP > 0 && F == 2 && ND >= 0) {
        // Levels coarser than the warp's 8 x 4 pixel block: when all 32 queries of the warp lie
        // in one cell, lane j fetches corner j mod 2^d once and the corners reach every lane by
        // warp shuffles (8 or 16 shuffles in place of the per-lane index work and gathers).
        if (l < NIV_WARP_COOP) {
            float w1[DIMS];
            uint32_t ci[DIMS];
            niv_level_cell<DIMS>(g, l, u, ci, w1);
            constexpr uint32_t kB = NIV_MAGIC_FLOOR ? kNivBias : 0u;
            const uint32_t key = (ci[0] - kB) | ((ci[1] - kB) << 11) | ((ci[2] - kB) << 22);
            if (__all_sync(0xFFFFFFFFu, key == __shfl_sync(0xFFFFFFFFu, key, 0))) {
                const int c = (int)(threadIdx.x & (NC - 1));
                uint32_t v[DIMS];
#pragma unroll
                for (int d = 0; d < DIMS; ++d) v[d] = ci[d] - kB + ((c >> d) & 1);
                uint32_t idx;
                if (l < ND) {
                    const uint32_t S = g.stride1[l], S2 = g.stride2[l];
                    idx = v[2] * S2 + v[1] * S + v[0];
                    if (DIMS == 4) idx += v[DIMS - 1] * S2 * S;
                } else {
                    idx = v[0] ^ (v[1] * NIV_PI2) ^ (v[2] * NIV_PI3);
                    if (DIMS == 4) idx ^= v[DIMS - 1] * g.prime_t;
                    idx &= g.hash_mask;
                }
                const uint32_t mine = __ldg(reinterpret_cast<const uint32_t*>(tab) + idx);
#pragma unroll
                for (int k = 0; k < NC; ++k) raw[k] = __shfl_sync(0xFFFFFFFFu, mine, k);
                float wc[NC];
                niv_level_weights<DIMS>(w1, wc);
                niv_level_blend<NC, F>(raw, wc, acc);
                return;
            }
            niv_level_index<DIMS, ND>(g, l, ci, e);
            niv_level_gather<NC, F, __half>(tab, e, raw);
            float wc[NC];
            niv_level_weights<DIMS>(w1, wc);
            niv_level_blend<NC, F>(raw, wc, acc);
            return;
        }
    }
    if constexpr ((NIV_DENSE_PAIRS == 1 || (NIV_DENSE_PAIRS == 2 && DIMS == 4)) && F == 2 && ND > 0) {
        if (pair != nullptr && l < ND) {
            float w1[DIMS];
            niv_level_entries<DIMS, ND>(g, l, u, e, w1);
            const uint2* pt = pair + g.offset[l];
#pragma unroll
            for (int q = 0; q < NC / 2; ++q) {
                const uint2 v = __ldg(pt + e[2 * q]);
                raw[2 * q] = v.x;
                raw[2 * q + 1] = v.y;
            }
            if constexpr (NIV_BLEND_LERP) {
                niv_level_lerp2<DIMS>(raw, w1, acc);
            } else {
                float wc[NC];
                niv_level_weights<DIMS>(w1, wc);
                niv_level_blend<NC, F>(raw, wc, acc);
            }
            return;
        }
    }
    if constexpr (NIV_BLEND_LERP && F == 2) {
        float w1[DIMS];
        niv_level_entries<DIMS, ND>(g, l, u, e, w1);
        niv_level_gather<NC, F, __half>(tab, e, raw);
        niv_level_lerp2<DIMS>(raw, w1, acc);
    } else {
        float wc[NC];
        niv_level_corners<DIMS, ND>(g, l, u, e, wc);
        niv_level_gather<NC, F, __half>(tab, e, raw);
        niv_level_blend<NC, F>(raw, wc, acc);
    }
}

// Interpolated features of level l (corners, gathers, blend).
template <int DIMS, int F, typename TabT>
__device__ __forceinline__ void niv_encode_level(const GridArgs& g, const TabT* __restrict__ grid, int l,
                                                 const float* u, float* acc) {
    constexpr int NC = 1 << DIMS;
    uint32_t e[NC];
    float wc[NC];
    niv_level_corners<DIMS>(g, l, u, e, wc);
    typename NivRaw<F, TabT>::T raw[NC];
    niv_level_gather<NC, F, TabT>(grid + (size_t)g.offset[l] * F, e, raw);
    niv_level_blend<NC, F>(raw, wc, acc);
}

// Image tiles: NIV_TILE_W x (128 / NIV_TILE_W) pixels, each warp of a tile an NIV_WARP_W x
// (32 / NIV_WARP_W) block, the warps row-major in the tile.
#ifndef NIV_TILE_W
#define NIV_TILE_W 32
#endif
#ifndef NIV_WARP_W
#define NIV_WARP_W 8
#endif
constexpr int kTileW = NIV_TILE_W, kTileH = 128 / NIV_TILE_W;
constexpr int kWarpW = NIV_WARP_W, kWarpH = 32 / NIV_WARP_W;
static_assert(kTileW * kTileH == 128 && kWarpW * kWarpH == 32 && kTileW % kWarpW == 0 && kTileH % kWarpH == 0,
              "tile and warp shapes must tile 128 and 32 records");
// Rows of a whole band of tiles (host-side chunking works in whole bands).
#define NIV_TILE_ROWS (128 / NIV_TILE_W)

// Pixel offset (x, y) of thread slot k inside its tile.
__host__ __device__ __forceinline__ int niv_slot_x(int k) {
    return ((k >> 5) % (kTileW / kWarpW)) * kWarpW + (k & 31) % kWarpW;
}
__host__ __device__ __forceinline__ int niv_slot_y(int k) {
    return ((k >> 5) / (kTileW / kWarpW)) * kWarpH + (k & 31) / kWarpW;
}

// Linear record index of thread slot `k` of tile `tile` (128-record tiles).  For images a tile
// is a kTileW x kTileH pixel block and each warp of it a kWarpW x kWarpH sub-block, so the 32
// queries of a warp are close on screen (and so in the scene).
__device__ __forceinline__ int64_t niv_record_of(int64_t tile, int k, int64_t n, int32_t width) {
    if (width <= 0) return tile * 128 + k;
    int64_t tiles_x = (width + kTileW - 1) / kTileW;
    int64_t ty = tile / tiles_x, tx = tile - ty * tiles_x;
    int64_t px = tx * kTileW + niv_slot_x(k), py = ty * kTileH + niv_slot_y(k);
    if (px >= width) return n;  // outside the image: no record
    return py * width + px;
}

// Persistent walk over 128-record tiles with a fixed stride, in the record order of
// niv_record_of: the image tile coordinates (tx, ty) advance by the stride's column and
// row parts, so no tile costs a 64-bit division.
struct NivTileWalk {
    int64_t tile, stride, ty, sy;
    int32_t tiles_x, tx, sx, ox, oy;

    __device__ __forceinline__ void init(int64_t first, int64_t step, int k, int32_t width) {
        tile = first;
        stride = step;
        ox = niv_slot_x(k);
        oy = niv_slot_y(k);
        tiles_x = width > 0 ? (width + kTileW - 1) / kTileW : 1;
        ty = first / tiles_x;
        tx = (int32_t)(first - ty * tiles_x);
        sy = step / tiles_x;
        sx = (int32_t)(step - sy * tiles_x);
    }
    __device__ __forceinline__ void next() {
        tile += stride;
        tx += sx;
        ty += sy;
        if (tx >= tiles_x) {
            tx -= tiles_x;
            ++ty;
        }
    }
    // Record of thread slot k (n: outside the image).
    __device__ __forceinline__ int64_t record(int k, int64_t n, int32_t width) const {
        if (width <= 0) return tile * 128 + k;
        const int32_t px = tx * kTileW + ox;
        if (px >= width) return n;
        return (ty * kTileH + oy) * (int64_t)width + px;
    }
    // G-buffer record of this thread's output record r (see IoArgs::sub).
    __device__ __forceinline__ int64_t source(int64_t r, const IoArgs& io) const {
        if (io.sub <= 1) return r;
        return (ty * kTileH + oy) * io.sub * (int64_t)io.src_width + (int64_t)(tx * kTileW + ox) * io.sub;
    }
};

__host__ __device__ __forceinline__ int64_t niv_tile_count(int64_t n, int32_t width) {
    if (width <= 0) return (n + 127) / 128;
    int64_t rows = (n + width - 1) / width;
    return ((width + kTileW - 1) / kTileW) * ((rows + kTileH - 1) / kTileH);
}

__host__ __forceinline__ int64_t niv_tile_count_host(int64_t n, int32_t width) { return niv_tile_count(n, width); }

// Load one [4] record (FP16 or FP32) as float4.
__device__ __forceinline__ float4 niv_load_rec(const void* base, int64_t i, bool f16) {
    if (f16) {
        uint2 r = __ldg(reinterpret_cast<const uint2*>(base) + i);
        __half2 a = *reinterpret_cast<__half2*>(&r.x), b = *reinterpret_cast<__half2*>(&r.y);
        float2 fa = __half22float2(a), fb = __half22float2(b);
        return make_float4(fa.x, fa.y, fb.x, fb.y);
    }
    return __ldg(reinterpret_cast<const float4*>(base) + i);
}

__device__ __forceinline__ void niv_store_rec(void* base, int64_t i, float x, float y, float z, bool f16) {
    if (f16) {
        __half2 a = __floats2half2_rn(x, y), b = __floats2half2_rn(z, 0.0f);
        uint2 r;
        r.x = *reinterpret_cast<uint32_t*>(&a);
        r.y = *reinterpret_cast<uint32_t*>(&b);
        reinterpret_cast<uint2*>(base)[i] = r;
    } else {
        reinterpret_cast<float4*>(base)[i] = make_float4(x, y, z, 0.0f);
    }
}

// Final store of a query: E, or the shaded rgba when the call fused shading.
__device__ __forceinline__ void niv_store_result(const IoArgs& io, int64_t i, float e0, float e1, float e2) {
    if (io.albedo) {
        const float inv_pi = 0.318309886183790671538f;
        const float4 a = niv_load_rec(io.albedo, i, true), d = niv_load_rec(io.direct, i, true);
        __half2 rg = __floats2half2_rn(fmaf(a.x * e0, inv_pi, d.x), fmaf(a.y * e1, inv_pi, d.y));
        __half2 ba = __floats2half2_rn(fmaf(a.z * e2, inv_pi, d.z), 1.0f);
        uint2 r;
        r.x = *reinterpret_cast<uint32_t*>(&rg);
        r.y = *reinterpret_cast<uint32_t*>(&ba);
        reinterpret_cast<uint2*>(io.out)[i] = r;
    } else {
        niv_store_rec(io.out, i, e0, e1, e2, io.out_f16);
    }
}

// softplus(z) = max(z, 0) + log1p(exp(-|z|)) in FP32 with CUDA's libm functions.
__device__ __forceinline__ float niv_softplus(float z) { return fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z))); }

// The same for the reduced-precision paths (FP16 / E4M3 networks): CUDA's fast exp and log
// intrinsics, whose error (about 1e-7 absolute here, log(1 + x) near x = 0 included) lies far
// below the 2^-11 relative resolution those paths keep.
#ifndef NIV_FAST_SOFTPLUS
#define NIV_FAST_SOFTPLUS 1
#endif
__device__ __forceinline__ float niv_softplus_lp(float z) {
    if (!NIV_FAST_SOFTPLUS) return niv_softplus(z);
    return fmaxf(z, 0.0f) + __logf(1.0f + __expf(-fabsf(z)));
}
