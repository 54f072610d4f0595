// FP8 (E4M3) fused query on the tensor cores, its calibration and its weight packing.
//
// Same tile pipeline as the FP16 path (query_tc.cu): persistent CTAs of 8 warpgroups that
// share one copy of the weights; a warpgroup encodes 128 records (FP16 grid features, FP32
// interpolation), writes the network input as E4M3 bytes into its K-major shared-memory
// tile, and every layer runs as tcgen05.mma of
// kind::f8f6f4 (E4M3 x E4M3, K = 32 per instruction) into an FP32 TMEM accumulator.
// Per-layer power-of-two scales: v = W / s_w and v = a / s_a.  One E4M3 code keeps only 3
// mantissa bits, so every scaled value is carried as two codes at the same scale,
// h = e4m3(v) and l = e4m3(v - h) (about 8 bits together), stored side by side: a tile of
// K inputs is K columns of h codes followed by K columns of l codes.  A layer is the MMA
// chain  acc = H Wh^T + L Wh^T + H Wl^T  (the L Wl^T term lies below both codes'
// resolution), and the epilogue forms
//   z = acc * (s_w * s_a) + b,  ReLU,  then the two codes of z / s_a' for the next layer;
// the output layer finishes with softplus in FP32.  s_a comes from niv_fp8_calibrate
// (amax of each layer's FP32 input over a calibration batch), s_w from amax|W|.
#include <cuda_fp8.h>
#include <math.h>
#include <string.h>

#include <vector>

#include "niv_internal.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int kT = 128;
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr int kHdr = 128;
constexpr int kNO = 16;

// Byte offset of (row r, column k) in a K-major tile of 8-bit elements with K columns:
// 8-row x 16-byte core matrices, 128 B apart along K, (K/16)*128 B apart along rows.
__host__ __device__ __forceinline__ uint32_t core_off8(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K >> 4) * 128 + (k >> 4) * 128 + (r & 7) * 16 + (k & 15));
}

struct F8Layout {
    // K1: network inputs per code tile (h and l tiles each K1 columns wide); col_extra: column
    // of n.x (the features end before it)
    int32_t K1, W, n_hidden, col_extra;
    uint32_t w1, wh, wo, scal, total;    // byte offsets; scal = FP32 block [c | qmul | biases | cq | bq]
};

// Float offset of b / s_a' inside the FP32 block at `scal`: after c (nh+1), 1/s_a (nh+1),
// the biases (nh W + 3, padded to + 4) and c / s_a' (nh), rounded up to a multiple of 4 so
// that the hidden epilogue loads it in 16-byte pieces.
__host__ __device__ __forceinline__ int f8_bq_offset(int nh, int W) { return (2 * (nh + 1) + nh * W + 4 + nh + 3) & ~3; }

// The two E4M3 codes of a pair of values (a in the low, b in the high byte of each code
// pair): h = e4m3(v) and l = e4m3(v - h), both rounded to nearest with saturation to +-448.
// v is first rounded to FP16 (2^-11 relative, far below l's resolution of about 2^-8), so
// that v - h is one exact FP16 subtraction (h lies within a factor of two of v).  RELU: v is
// max(v, 0).  Returns h in the low and l in the high 16 bits.
template <bool RELU>
__device__ __forceinline__ uint32_t e4m3_pair2(float a, float b) {
    uint32_t v, hf, r;
    uint16_t h, l;
    if (RELU) asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(v) : "f"(b), "f"(a));
    else asm("cvt.rn.f16x2.f32 %0, %1, %2;" : "=r"(v) : "f"(b), "f"(a));
    asm("cvt.rn.satfinite.e4m3x2.f16x2 %0, %1;" : "=h"(h) : "r"(v));
    asm("cvt.rn.f16x2.e4m3x2 %0, %1;" : "=r"(hf) : "h"(h));
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(r) : "r"(v), "r"(hf));
    asm("cvt.rn.satfinite.e4m3x2.f16x2 %0, %1;" : "=h"(l) : "r"(r));
    return (uint32_t)h | ((uint32_t)l << 16);
}

// The codes of 16 values (max(v, 0)), in order: h codes to hi, l codes to lo.
__device__ __forceinline__ void e4m3_pairs16_relu(const float* v, uint4& hi, uint4& lo) {
    uint32_t p[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) p[j] = e4m3_pair2<true>(v[2 * j], v[2 * j + 1]);
    hi = make_uint4((p[0] & 0xFFFFu) | (p[1] << 16), (p[2] & 0xFFFFu) | (p[3] << 16), (p[4] & 0xFFFFu) | (p[5] << 16),
                    (p[6] & 0xFFFFu) | (p[7] << 16));
    lo = make_uint4((p[0] >> 16) | (p[1] & 0xFFFF0000u), (p[2] >> 16) | (p[3] & 0xFFFF0000u),
                    (p[4] >> 16) | (p[5] & 0xFFFF0000u), (p[6] >> 16) | (p[7] & 0xFFFF0000u));
}

__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
    uint32_t r[4];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}

// One layer over K inputs: the tiles at act ([H | L], 2K columns) and w ([Wh | Wl], 2K
// columns) give acc = H Wh^T + L Wh^T + H Wl^T, then `bar` is signalled.
__device__ __forceinline__ void issue_layer8(uint32_t tmem, uint32_t act, uint32_t w, uint32_t K, uint32_t idesc,
                                             uint32_t bar) {
    const uint32_t sbo = (2u * K >> 4) * 128u;  // 8-row groups of a 2K-column tile
    const uint32_t lo = (K >> 4) * 128u;        // first core matrix of the l codes
    for (uint32_t ks = 0; ks < K / 32; ++ks)
        tc::mma_e4m3(tmem, tc::smem_desc(act + ks * 256u, 128u, sbo), tc::smem_desc(w + ks * 256u, 128u, sbo), idesc,
                     ks > 0 ? 1u : 0u);
    for (uint32_t ks = 0; ks < K / 32; ++ks)
        tc::mma_e4m3(tmem, tc::smem_desc(act + lo + ks * 256u, 128u, sbo), tc::smem_desc(w + ks * 256u, 128u, sbo),
                     idesc, 1u);
    for (uint32_t ks = 0; ks < K / 32; ++ks)
        tc::mma_e4m3(tmem, tc::smem_desc(act + ks * 256u, 128u, sbo), tc::smem_desc(w + lo + ks * 256u, 128u, sbo),
                     idesc, 1u);
    tc::mma_commit(bar);
}

// Encode levels [l0, l0 + 16/F) of one record into one 16-byte chunk of h codes (hi) and one
// of l codes (lo) of the E4M3 inputs (value times q0, the inverse input scale), each level
// converted as soon as it is blended.
template <int DIMS, int F, int ND = -1>
__device__ __forceinline__ void encode_chunk8(const GridArgs& g, const __half* __restrict__ grid16, int l0, int L,
                                              const float* u, float q0, uint4& hi, uint4& lo,
                                              const uint2* __restrict__ pair = nullptr) {
    constexpr int NC = 1 << DIMS, G = 16 / F;
    using R = typename NivRaw<F, __half>::T;
    uint32_t wd[4] = {0u, 0u, 0u, 0u}, wl[4] = {0u, 0u, 0u, 0u};
#pragma unroll
    for (int q = 0; q < G; ++q) {
        if (l0 + q >= L) continue;
        float acc[F];
        niv_level_features16<DIMS, F, ND>(g, grid16 + (size_t)g.offset[l0 + q] * F, l0 + q, u, acc, pair);
        if (F == 1) {
            const uint32_t p = e4m3_pair2<false>(acc[0] * q0, 0.0f);
            wd[q >> 2] |= (p & 0xFFu) << (8 * (q & 3));
            wl[q >> 2] |= ((p >> 16) & 0xFFu) << (8 * (q & 3));
        } else if (F == 2) {
            const float2 a = __fmul2_rn(make_float2(acc[0], acc[1 % F]), make_float2(q0, q0));
            const uint32_t p = e4m3_pair2<false>(a.x, a.y);
            wd[(q >> 1) & 3] |= (q & 1) ? (p << 16) : (p & 0xFFFFu);
            wl[(q >> 1) & 3] |= (q & 1) ? (p & 0xFFFF0000u) : (p >> 16);
        } else {
            const uint32_t p0 = e4m3_pair2<false>(acc[0] * q0, acc[1 % F] * q0);
            const uint32_t p1 = e4m3_pair2<false>(acc[2 % F] * q0, acc[3 % F] * q0);
            wd[q & 3] = (p0 & 0xFFFFu) | (p1 << 16);
            wl[q & 3] = (p0 >> 16) | (p1 & 0xFFFF0000u);
        }
    }
    hi = make_uint4(wd[0], wd[1], wd[2], wd[3]);
    lo = make_uint4(wl[0], wl[1], wl[2], wl[3]);
}

#ifndef NIV_TC_ND
#define NIV_TC_ND 1
#endif
#ifndef NIV_F8_WG
#define NIV_F8_WG 8
#endif
constexpr int kWG = NIV_F8_WG;  // warpgroups (independent tile pipelines) per CTA sharing the weights

__device__ __forceinline__ void group_sync8(int wg) { asm volatile("bar.sync %0, 128;" ::"r"(1 + wg) : "memory"); }

// kWG warpgroups per CTA, persistent over 128-record tiles; each warpgroup owns an activation
// tile, an mbarrier, a named barrier and its TMEM columns.  LV > 0: level count fixed at
// compile time (the level loop unrolls).  WT, KT, NHT > 0: network width, first-layer input
// width and hidden-layer count fixed at compile time (layer and column loops unroll).  ND >= 0:
// levels 0 .. ND-1 are the dense ones.
template <int DIMS, int F, int LV, int WT = 0, int KT = 0, int NHT = 0, int ND = -1>
__global__ void __launch_bounds__(kT * kWG, 1) query_f8_kernel(GridArgs g, IoArgs io, const __half* __restrict__ grid16,
                                                                const uint8_t* __restrict__ packed, F8Layout lay,
                                                                int out_act, int64_t n_tiles, uint32_t tmem_cols,
                                                                int* __restrict__ status,
                                                                const uint2* __restrict__ pair) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem);  // one per warpgroup
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + 64);
    uint8_t* s_net = smem + kHdr;
    const int K1 = KT > 0 ? KT : lay.K1, W = WT > 0 ? WT : lay.W, nh = NHT > 0 ? NHT : lay.n_hidden;
    const int col_extra = LV > 0 ? ((LV * F + 15) & ~15) : lay.col_extra;  // column of n.x
    const uint32_t act_bytes = (uint32_t)kT * 2u * (uint32_t)(K1 > W ? K1 : W);  // h and l codes
    const int wg = threadIdx.x / kT, tid = threadIdx.x % kT, warp = tid >> 5;
    uint8_t* s_act = s_net + ((lay.total + 127u) & ~127u) + wg * act_bytes;

    for (uint32_t i = threadIdx.x; i < lay.total / 16; i += kT * kWG)
        reinterpret_cast<uint4*>(s_net)[i] = __ldg(reinterpret_cast<const uint4*>(packed) + i);
    if (threadIdx.x == 0) {
        for (int i = 0; i < kWG; ++i) tc::mbar_init(s_bar + i, 1);
        tc::fence_mbar_init();
    }
    if (threadIdx.x < 32) {
        tc::tmem_alloc(tc::smem_u32(s_tmem), tmem_cols);
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    const uint32_t wg_cols = W <= 32 ? 32u : 64u;
    const uint32_t tmem = *s_tmem + (uint32_t)wg * wg_cols;
    const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t bar = tc::smem_u32(s_bar + wg);
    const uint32_t act_a = tc::smem_u32(s_act), net_a = tc::smem_u32(s_net);
    const uint32_t idesc_h = tc::idesc_e4m3(128, W), idesc_o = tc::idesc_e4m3(128, kNO);
    const float* s_c = reinterpret_cast<const float*>(s_net + lay.scal);  // acc -> z multipliers
    const float* s_q = s_c + (nh + 1);                                   // 1 / s_a per matrix input
    const float* s_b = s_q + (nh + 1);                                   // biases
    const float* s_cq = s_b + nh * W + 4;                                // hidden layers: c / s_a'
    const float* s_bq = s_c + f8_bq_offset(nh, W);                       // hidden layers: b / s_a'
    const int L = LV > 0 ? LV : g.levels, LF = L * F;
    constexpr int G = 16 / F;  // levels per 16-byte chunk of E4M3 inputs
    uint32_t phase = 0;
    bool ok = true;

    NivTileWalk walk;
    walk.init((int64_t)blockIdx.x * kWG + wg, (int64_t)gridDim.x * kWG, tid, io.image_width);
    for (; walk.tile < n_tiles && ok; walk.next()) {
        const int64_t r = walk.record(tid, io.n, io.image_width);
        const bool valid = r < io.n;
        const int64_t rr = valid ? walk.source(r, io) : 0;
        const float4 p = niv_load_rec(io.pos, rr, io.in_f16);
        const float4 nv = niv_load_rec(io.nrm, rr, io.in_f16);
        float u[4];
        u[0] = niv_unit(p.x, g.aabb_min[0], g.inv_ext[0]);
        u[1] = niv_unit(p.y, g.aabb_min[1], g.inv_ext[1]);
        u[2] = niv_unit(p.z, g.aabb_min[2], g.inv_ext[2]);
        u[3] = fminf(fmaxf(g.t, 0.0f), 1.0f);

        // ---- encoding -> E4M3 input row: h codes in columns [0, K1), l codes in [K1, 2 K1) ----
        const float q0 = s_q[0];
        const int K2 = 2 * K1;
        if (LV > 0) {
#pragma unroll
            for (int l0 = 0; l0 < LV; l0 += G) {
                uint4 hi, lo;
                encode_chunk8<DIMS, F, ND>(g, grid16, l0, LV, u, q0, hi, lo, pair);
                *reinterpret_cast<uint4*>(s_act + core_off8(tid, l0 * F, K2)) = hi;
                *reinterpret_cast<uint4*>(s_act + core_off8(tid, K1 + l0 * F, K2)) = lo;
            }
        } else {
            for (int l0 = 0; l0 < L; l0 += G) {
                uint4 hi, lo;
                encode_chunk8<DIMS, F>(g, grid16, l0, L, u, q0, hi, lo);
                *reinterpret_cast<uint4*>(s_act + core_off8(tid, l0 * F, K2)) = hi;
                *reinterpret_cast<uint4*>(s_act + core_off8(tid, K1 + l0 * F, K2)) = lo;
            }
        }
        {
            const float tv = g.n_in > LF + 3 ? u[3] : 0.0f;
            const uint32_t p0 = e4m3_pair2<false>(nv.x * q0, nv.y * q0), p1 = e4m3_pair2<false>(nv.z * q0, tv * q0);
            *reinterpret_cast<uint4*>(s_act + core_off8(tid, col_extra, K2)) =
                make_uint4((p0 & 0xFFFFu) | (p1 << 16), 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(s_act + core_off8(tid, K1 + col_extra, K2)) =
                make_uint4((p0 >> 16) | (p1 & 0xFFFF0000u), 0u, 0u, 0u);
        }
        for (int k = col_extra + 16; k < K1; k += 16) {
            *reinterpret_cast<uint4*>(s_act + core_off8(tid, k, K2)) = make_uint4(0u, 0u, 0u, 0u);
            *reinterpret_cast<uint4*>(s_act + core_off8(tid, K1 + k, K2)) = make_uint4(0u, 0u, 0u, 0u);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        group_sync8(wg);

        // ---- hidden layers ----
        uint32_t K = (uint32_t)K1, w_off = lay.w1;
#pragma unroll
        for (int layer = 0; layer < nh && ok; ++layer) {
            if (tid == 0) {
                tc::fence_after_sync();
                issue_layer8(tmem, act_a, net_a + w_off, K, idesc_h, bar);
            }
            if (!tc::mbar_wait_bounded(bar, phase, kWaitLimitNs)) {
                atomicExch(status, 1);
                ok = false;
                break;
            }
            phase ^= 1u;
            tc::fence_after_sync();
            const float cq = s_cq[layer];
            const float* bq = s_bq + layer * W;
#pragma unroll
            for (int ch = 0; ch < W / 16; ++ch) {
                float v[16];
                tc::tmem_ld16(tmem_row + (uint32_t)(ch * 16), v);
#pragma unroll
                for (int j = 0; j < 8; ++j) {  // packed pairs: each lane is the FMA fma(acc, c / s_a', b / s_a')
                    const float2 r = __ffma2_rn(make_float2(v[2 * j], v[2 * j + 1]), make_float2(cq, cq),
                                                reinterpret_cast<const float2*>(bq + ch * 16)[j]);
                    v[2 * j] = r.x;
                    v[2 * j + 1] = r.y;
                }
                uint4 hi, lo;
                e4m3_pairs16_relu(v, hi, lo);
                *reinterpret_cast<uint4*>(s_act + core_off8(tid, ch * 16, 2 * W)) = hi;
                *reinterpret_cast<uint4*>(s_act + core_off8(tid, W + ch * 16, 2 * W)) = lo;
            }
            tc::fence_async_smem();
            tc::fence_before_sync();
            group_sync8(wg);
            w_off = layer == 0 ? lay.wh : w_off + (uint32_t)(2 * W * W);
            K = (uint32_t)W;
        }
        if (!ok) break;

        // ---- output layer (N = 16, three live columns) ----
        if (tid == 0) {
            tc::fence_after_sync();
            issue_layer8(tmem, act_a, net_a + lay.wo, (uint32_t)W, idesc_o, bar);
        }
        if (!tc::mbar_wait_bounded(bar, phase, kWaitLimitNs)) {
            atomicExch(status, 1);
            ok = false;
            break;
        }
        phase ^= 1u;
        tc::fence_after_sync();
        float zz[4];
        tmem_ld4(tmem_row, zz);
        const float c = s_c[nh];
        const float* bo = s_b + nh * W;
        float z0 = fmaf(zz[0], c, bo[0]), z1 = fmaf(zz[1], c, bo[1]), z2 = fmaf(zz[2], c, bo[2]);
        if (out_act == 1) {
            z0 = niv_softplus_lp(z0);
            z1 = niv_softplus_lp(z1);
            z2 = niv_softplus_lp(z2);
        }
        if (valid) niv_store_result(io, r, z0, z1, z2);
        tc::fence_before_sync();
        group_sync8(wg);  // the next tile's encoder overwrites the activation tile
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(*s_tmem, tmem_cols);
}

template <int DIMS, int F, int LV, int WT = 0, int KT = 0, int NHT = 0, int ND = -1>
int launch8(const niv_model* m, const GridArgs& g, const IoArgs& io, cudaStream_t s) {
    const F8Layout* lay = reinterpret_cast<const F8Layout*>(m->f8_layout);
    if ((WT > 0 && lay->W != WT) || (KT > 0 && lay->K1 != KT) || (NHT > 0 && lay->n_hidden != NHT))
        return niv_fail(NIV_ERR_UNSUPPORTED, "network shape differs from the kernel's");
    if (ND >= 0 && g.dense_mask != (ND >= 32 ? ~0u : ((1u << ND) - 1u)))
        return niv_fail(NIV_ERR_UNSUPPORTED, "dense levels differ from the kernel's");
    auto kern = query_f8_kernel<DIMS, F, LV, WT, KT, NHT, ND>;
    const int kmax = lay->K1 > lay->W ? lay->K1 : lay->W;
    const size_t smem = (size_t)kHdr + ((lay->total + 127u) & ~127u) + (size_t)kWG * kT * 2 * kmax;
    NIV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, smem_per_sm = 0, regs_per_sm = 0;
    NIV_CUDA(cudaGetDevice(&dev));
    NIV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    NIV_CUDA(cudaDeviceGetAttribute(&smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
    NIV_CUDA(cudaDeviceGetAttribute(&regs_per_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
    cudaFuncAttributes fa;
    NIV_CUDA(cudaFuncGetAttributes(&fa, kern));
    // residency from the register and shared-memory budgets (the occupancy API reports a
    // single CTA per SM for kernels that allocate tensor memory)
    const int regs = fa.numRegs > 0 ? ((fa.numRegs + 7) & ~7) : 1;
    int per_sm = smem_per_sm / (int)(smem + 1024);
    if (regs_per_sm / (kT * kWG * regs) < per_sm) per_sm = regs_per_sm / (kT * kWG * regs);
    uint32_t cols = 32u;  // TMEM is allocated in powers of two from 32 to 512 columns
    while (cols < (lay->W <= 32 ? 32u : 64u) * (uint32_t)kWG) cols <<= 1;
    if (cols > 512u) return niv_fail(NIV_ERR_UNSUPPORTED, "too many warpgroups for tensor memory");
    if (per_sm > (int)(512 / cols)) per_sm = (int)(512 / cols);
    if (per_sm < 1) return niv_fail(NIV_ERR_UNSUPPORTED, "FP8 query kernel does not fit on an SM");
    // shared memory for the resident CTAs only; the rest of the SM's storage is L1 for the gathers
    int carve = (int)((100 * (int64_t)per_sm * (int64_t)(smem + 1024) + smem_per_sm - 1) / smem_per_sm);
    if (carve > 100) carve = 100;
    NIV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carve));
    int* status = niv_status_word();
    if (!status) return niv_fail(NIV_ERR_CUDA, "status word unavailable");
    const int64_t tiles = niv_tile_count_host(io.n, io.image_width);
    const int64_t need = (tiles + kWG - 1) / kWG;
    const int64_t blocks = need < (int64_t)sms * per_sm ? need : (int64_t)sms * per_sm;
    kern<<<(unsigned)blocks, kT * kWG, smem, s>>>(g, io, m->grid_f16, m->mlp_f8, *lay, m->d.out_act, tiles, cols,
                                                  status, m->grid_pair16);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}

// ---- calibration: amax of every matrix product's FP32 input over n records ----
__device__ __forceinline__ void amax_update(unsigned* slot, float v) {
    // non-negative floats order like their bit patterns
    const unsigned bits = __reduce_max_sync(0xFFFFFFFFu, __float_as_uint(v));
    if ((threadIdx.x & 31) == 0) atomicMax(slot, bits);
}

template <int DIMS, int F>
__global__ void __launch_bounds__(128) calib_kernel(GridArgs g, IoArgs io, const float* __restrict__ grid,
                                                    const float* __restrict__ mlp, int W, int nh,
                                                    unsigned* __restrict__ amax) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool valid = q < io.n;
    const int64_t qq = valid ? q : 0;
    const float4 p = niv_load_rec(io.pos, qq, io.in_f16);
    const float4 nv = niv_load_rec(io.nrm, qq, io.in_f16);
    float u[4];
    u[0] = niv_unit(p.x, g.aabb_min[0], g.inv_ext[0]);
    u[1] = niv_unit(p.y, g.aabb_min[1], g.inv_ext[1]);
    u[2] = niv_unit(p.z, g.aabb_min[2], g.inv_ext[2]);
    u[3] = fminf(fmaxf(g.t, 0.0f), 1.0f);
    float x[NIV_MAX_IN], h[64], h2[64];
    float mx = 0.0f;
    for (int l = 0; l < g.levels; ++l) {
        float acc[F];
        niv_encode_level<DIMS, F, float>(g, grid, l, u, acc);
        for (int j = 0; j < F; ++j) {
            x[l * F + j] = acc[j];
            mx = fmaxf(mx, fabsf(acc[j]));
        }
    }
    const int LF = g.levels * F;
    x[LF] = nv.x;
    x[LF + 1] = nv.y;
    x[LF + 2] = nv.z;
    if (g.n_in > LF + 3) x[LF + 3] = u[3];
    for (int i = LF; i < g.n_in; ++i) mx = fmaxf(mx, fabsf(x[i]));
    amax_update(amax, valid ? mx : 0.0f);
    const float* w = mlp;
    int k_in = g.n_in;
    const float* in = x;
    for (int layer = 0; layer < nh; ++layer) {
        float* out = (layer & 1) ? h2 : h;
        float m2 = 0.0f;
        for (int o = 0; o < W; ++o) {
            float z = w[W * k_in + o];
            for (int i = 0; i < k_in; ++i) z = fmaf(w[o * k_in + i], in[i], z);
            out[o] = fmaxf(z, 0.0f);
            m2 = fmaxf(m2, out[o]);
        }
        amax_update(amax + layer + 1, valid ? m2 : 0.0f);
        w += W * k_in + W;
        k_in = W;
        in = out;
    }
}

double pow2_scale(double amax) {  // 2^ceil(log2(amax / 448)), 1 for amax = 0
    if (!(amax > 0.0)) return 1.0;
    int e;
    const double mnt = frexp(amax / 448.0, &e);
    return mnt == 0.5 ? ldexp(1.0, e - 1) : ldexp(1.0, e);
}

uint8_t to_e4m3(float v) { return (uint8_t)__nv_cvt_float_to_fp8(v, __NV_SATFINITE, __NV_E4M3); }

float from_e4m3(uint8_t c) {
    const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)c, __NV_E4M3);
    return __half2float(__half(h));
}

}  // namespace

// Pack the E4M3 network from host FP32 parameters and the activation scales m->fp8_sact:
// [W1 (W x 2 K1) | hidden (W x 2 W) ... | W_out (16 x 2 W) bytes | c[nh+1] | qmul[nh+1] | biases],
// each weight tile [Wh | Wl]: the h codes e4m3(W / s_w), then the l codes e4m3(W / s_w - h).
int niv_pack_f8(niv_model* m, const float* mlp_host, cudaStream_t s) {
    const int W = m->d.width, nh = m->d.n_hidden, n_in = m->n_in, LF = m->d.levels * m->d.feat;
    F8Layout lay;
    memset(&lay, 0, sizeof lay);
    lay.col_extra = (LF + 15) & ~15;
    lay.K1 = (lay.col_extra + m->d.in_extra + 31) & ~31;
    lay.W = W;
    lay.n_hidden = nh;
    auto up = [](uint32_t x) { return (x + 127u) & ~127u; };
    lay.w1 = 0;
    lay.wh = up(lay.w1 + (uint32_t)(W * 2 * lay.K1));
    lay.wo = up(lay.wh + (uint32_t)((nh - 1) * W * 2 * W));
    lay.scal = up(lay.wo + (uint32_t)(kNO * 2 * W));
    // [c (nh+1) | 1/s_a (nh+1) | biases (nh W + 3, padded to + 4) | c / s_a' (nh) | pad | b / s_a' (nh W)]
    lay.total = up(lay.scal + (uint32_t)((f8_bq_offset(nh, W) + nh * W) * 4));
    static_assert(sizeof(F8Layout) <= sizeof(((niv_model*)0)->f8_layout), "layout slot too small");
    std::vector<uint8_t> buf(lay.total, 0);
    float* c = reinterpret_cast<float*>(&buf[lay.scal]);
    float* qm = c + (nh + 1);
    float* bias = qm + (nh + 1);
    const float* p = mlp_host;
    int k_in = n_in;
    for (int l = 0; l <= nh; ++l) {
        const bool last = l == nh;
        const int n_out = last ? 3 : W;
        float amax = 0.0f;
        for (int i = 0; i < n_out * k_in; ++i) amax = fmaxf(amax, fabsf(p[i]));
        const double sw = pow2_scale(amax);
        m->fp8_sw[l] = (float)sw;
        const float inv = (float)(1.0 / sw);  // exact: a power of two
        const uint32_t base = l == 0 ? lay.w1 : last ? lay.wo : lay.wh + (uint32_t)((l - 1) * W * 2 * W);
        const int K = l == 0 ? lay.K1 : W;
        for (int r = 0; r < n_out; ++r)
            for (int i = 0; i < k_in; ++i) {
                const int col = (l == 0 && i >= LF) ? lay.col_extra + (i - LF) : i;
                const float v = p[(size_t)r * k_in + i] * inv;  // exact: inv is a power of two
                const uint8_t h = to_e4m3(v);
                buf[base + core_off8(r, col, 2 * K)] = h;
                buf[base + core_off8(r, K + col, 2 * K)] = to_e4m3(v - from_e4m3(h));  // v - h exact
            }
        p += (size_t)n_out * k_in;
        for (int r = 0; r < n_out; ++r) bias[l * W + r] = p[r];
        p += n_out;
        c[l] = (float)(sw * (double)m->fp8_sact[l]);
        qm[l] = (float)(1.0 / (double)m->fp8_sact[l]);
        k_in = n_out;
    }
    // hidden layers' epilogue in one FMA: (acc c + b) / s_a' with the next input scale s_a' a
    // power of two, so c / s_a' and b / s_a' are exact and fma(acc, c / s_a', b / s_a') equals
    // the rounded (acc c + b) scaled
    float* cq = bias + nh * W + 4;
    float* bq = c + f8_bq_offset(nh, W);
    for (int l = 0; l < nh; ++l) {
        cq[l] = c[l] * qm[l + 1];
        for (int r = 0; r < W; ++r) bq[l * W + r] = bias[l * W + r] * qm[l + 1];
    }
    memcpy(m->f8_layout, &lay, sizeof lay);
    if (m->mlp_f8_bytes < lay.total) {
        cudaFree(m->mlp_f8);
        m->mlp_f8 = nullptr;
        m->mlp_f8_bytes = 0;
        NIV_CUDA(cudaMalloc(&m->mlp_f8, lay.total));
        m->mlp_f8_bytes = lay.total;
    }
    NIV_CUDA(cudaMemcpyAsync(m->mlp_f8, buf.data(), lay.total, cudaMemcpyHostToDevice, s));
    NIV_CUDA(cudaStreamSynchronize(s));
    return NIV_OK;
}

// Run the calibration pass over n records and set the activation scales (host side waits).
int niv_calibrate_f8(niv_model* m, const GridArgs& g, const IoArgs& io, cudaStream_t s) {
    if (m->d.pe_bands > 0 || m->d.t_bands > 0)
        return niv_fail(NIV_ERR_UNSUPPORTED, "the FP8 path takes grid models with a raw t only");
    if (m->d.width > 64 || m->n_in > NIV_MAX_IN) return niv_fail(NIV_ERR_UNSUPPORTED, "calibration shape");
    const int nh = m->d.n_hidden;
    if (!m->fp8_amax) NIV_CUDA(cudaMalloc(&m->fp8_amax, sizeof(unsigned) * 8));
    NIV_CUDA(cudaMemsetAsync(m->fp8_amax, 0, sizeof(unsigned) * 8, s));
    const unsigned blocks = (unsigned)((io.n + 127) / 128);
    const float* mlp = m->params + m->n_grid;
    if (m->d.dims == 4) {
        switch (m->d.feat) {
            case 1: calib_kernel<4, 1><<<blocks, 128, 0, s>>>(g, io, m->params, mlp, m->d.width, nh, m->fp8_amax); break;
            case 2: calib_kernel<4, 2><<<blocks, 128, 0, s>>>(g, io, m->params, mlp, m->d.width, nh, m->fp8_amax); break;
            default: calib_kernel<4, 4><<<blocks, 128, 0, s>>>(g, io, m->params, mlp, m->d.width, nh, m->fp8_amax); break;
        }
    } else {
        switch (m->d.feat) {
            case 1: calib_kernel<3, 1><<<blocks, 128, 0, s>>>(g, io, m->params, mlp, m->d.width, nh, m->fp8_amax); break;
            case 2: calib_kernel<3, 2><<<blocks, 128, 0, s>>>(g, io, m->params, mlp, m->d.width, nh, m->fp8_amax); break;
            default: calib_kernel<3, 4><<<blocks, 128, 0, s>>>(g, io, m->params, mlp, m->d.width, nh, m->fp8_amax); break;
        }
    }
    NIV_CUDA(cudaGetLastError());
    unsigned bits[8];
    NIV_CUDA(cudaMemcpyAsync(bits, m->fp8_amax, sizeof bits, cudaMemcpyDeviceToHost, s));
    NIV_CUDA(cudaStreamSynchronize(s));
    for (int l = 0; l <= nh; ++l) {
        float a;
        memcpy(&a, &bits[l], 4);
        m->fp8_amax_host[l] = a;
        m->fp8_sact[l] = (float)pow2_scale(a);
    }
    std::vector<float> mlp_host((size_t)m->n_mlp);
    NIV_CUDA(cudaMemcpyAsync(mlp_host.data(), mlp, sizeof(float) * m->n_mlp, cudaMemcpyDeviceToHost, s));
    NIV_CUDA(cudaStreamSynchronize(s));
    int rc = niv_pack_f8(m, mlp_host.data(), s);
    if (rc) return rc;
    m->fp8_ready = 1;
    return NIV_OK;
}

int niv_launch_query_f8(const niv_model* m, const GridArgs& g, const IoArgs& io, cudaStream_t s) {
    if (m->d.pe_bands > 0 || m->d.t_bands > 0)
        return niv_fail(NIV_ERR_UNSUPPORTED, "the FP8 path takes grid models with a raw t only");
    if (!m->fp8_ready) return niv_fail(NIV_ERR_ARG, "FP8 path needs niv_fp8_calibrate after the last niv_set_params");
    const F8Layout* lay = reinterpret_cast<const F8Layout*>(m->f8_layout);
    if (lay->K1 > 128) return niv_fail(NIV_ERR_UNSUPPORTED, "FP8 path needs a network input of <= 112 values");
    // fully unrolled encoders for 16 levels of 2 features (configs 1, 3, 4), a runtime loop otherwise
    const bool l16 = g.levels == 16 && m->d.feat == 2;
    // fixed shapes: width 64, 64 input columns, 2 (3-D) or 3 (4-D) hidden layers
    const bool fixed2 = lay->W == 64 && lay->K1 == 64 && lay->n_hidden == 2;
    const bool fixed3 = lay->W == 64 && lay->K1 == 64 && lay->n_hidden == 3;
    if (m->d.dims == 4) {
        if (NIV_TC_ND && l16 && fixed3 && g.dense_mask == 0x3u) return launch8<4, 2, 16, 64, 64, 3, 2>(m, g, io, s);
        if (l16 && fixed3) return launch8<4, 2, 16, 64, 64, 3>(m, g, io, s);
        if (l16) return launch8<4, 2, 16>(m, g, io, s);
        switch (m->d.feat) {
            case 1: return launch8<4, 1, 0>(m, g, io, s);
            case 2: return launch8<4, 2, 0>(m, g, io, s);
            default: return launch8<4, 4, 0>(m, g, io, s);
        }
    }
    if (NIV_TC_ND && l16 && fixed2 && g.dense_mask == 0xFu) return launch8<3, 2, 16, 64, 64, 2, 4>(m, g, io, s);
    if (l16 && fixed2) return launch8<3, 2, 16, 64, 64, 2>(m, g, io, s);
    if (l16) return launch8<3, 2, 16>(m, g, io, s);
    switch (m->d.feat) {
        case 1: return launch8<3, 1, 0>(m, g, io, s);
        case 2: return launch8<3, 2, 0>(m, g, io, s);
        default: return launch8<3, 4, 0>(m, g, io, s);
    }
}
