// Fused query path on the 5th-generation tensor cores (sm_103a).
//
// A warpgroup (128 threads) owns a tile of 128 G-buffer records at a time (a 32 x 4
// pixel block for images) and walks tiles persistently.  Per tile:
//   1. every thread encodes its own record (Sec. 4.1: per level the cell, the
//      2^d corner entries -- dense or hashed --, FP16 feature gathers served from
//      L2, multilinear weights in FP32; or, for the models of Table 1 without
//      grid, the sin / cos pairs of the frequency encoding) and writes its row of the network input
//      [features | n, (t), 1 | 0-pad] as FP16, in 16-byte chunks, into a shared-memory
//      tile laid out in the tensor core's canonical K-major format (the constant 1
//      multiplies the first layer's bias, stored as an extra weight column);
//   2. one thread issues tcgen05.mma (M = 128 records, N = width, K = 16 per
//      instruction) against the weights resident in shared memory, then one more
//      K = 16 MMA that adds the layer's bias (a constant tile of ones against a
//      tile holding the biases); the FP32 accumulator lives in tensor memory (TMEM);
//   3. each warp reads its 32 rows back with tcgen05.ld, rounds to FP16, applies
//      ReLU on packed halves and writes the next layer's input tile; repeat per
//      hidden layer;
//   4. the output layer (N = 16, three live columns) also runs on the tensor
//      core; softplus in FP32 and the store of E finish the record.
// Parameters are FP16 (weights, biases, grid features: all parameters in half
// precision, Table 1), accumulation FP32.  Every wait on the MMA-completion
// barrier is bounded (2 s); on expiry the kernel records a failure in the status
// word, releases its TMEM and returns.
//
// Tuning knobs (compile-time): NIV_TC_WG warpgroups per CTA sharing one copy of the
// weights, NIV_TC_ILP levels whose gathers are in flight together, NIV_TC_MINB the
// launch-bounds residency target, NIV_TC_OUT_FMA output layer on the CUDA cores,
// NIV_TC_FIXW kernels compiled for the 16-level models' network shapes (width 64, 48
// input columns, 2 or 3 hidden layers), NIV_TC_ND those kernels also compiled for their
// dense-level counts, NIV_TC_BIAS_MMA biases added by the tensor core, NIV_TC_NRM_EARLY
// normal records loaded at the start of a tile (NIV_BLEND_PAIRS in
// encoding.cuh: a corner's two features blended as one packed FP32 pair).
#include <cuda_fp8.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "niv_internal.cuh"
#include "tc_ptx.cuh"

namespace {

#ifndef NIV_TC_PPT
#define NIV_TC_PPT 1  // records per thread: 2 gives each warpgroup two 128-row tiles at a time
#endif
#ifndef NIV_TC_WG
#define NIV_TC_WG (NIV_TC_PPT == 2 ? 4 : 8)
#endif
#ifndef NIV_TC_ILP
#define NIV_TC_ILP 1
#endif
#ifndef NIV_TC_MINB
#define NIV_TC_MINB 1
#endif
#ifndef NIV_TC_FIXW
#define NIV_TC_FIXW 1
#endif
#ifndef NIV_TC_ND
#define NIV_TC_ND 1
#endif

constexpr int kT = 128;          // rows per tile = threads per warpgroup
constexpr int kWG = NIV_TC_WG;   // warpgroups (independent tile pipelines) per CTA
constexpr int kP = NIV_TC_PPT;   // 128-row tiles a warpgroup carries at a time (records per thread)
constexpr int kILP = NIV_TC_ILP; // levels whose gathers are in flight together (1 or 2)
constexpr uint64_t kWaitLimitNs = 2000000000ull;
#ifndef NIV_TC_OUT_FMA
#define NIV_TC_OUT_FMA 0
#endif
// Biases of the hidden layers after the first and of the output layer added by the tensor core:
// one more K = 16 MMA per layer, of a constant tile whose column 0 is 1 against a tile whose
// column 0 holds the layer's FP16 biases (exact products), in place of the FP32 adds of the
// epilogue (measured 3% faster at 1080p).  Layer 1's bias always rides in a column of W1.
#ifndef NIV_TC_BIAS_MMA
#define NIV_TC_BIAS_MMA 1
#endif
constexpr bool kBiasMma = NIV_TC_BIAS_MMA != 0;
// FP16 records: the normal loaded with the position at the start of a tile and held as its raw
// 8 bytes through the encoding, so that its latency hides behind the encoding (measured 3%
// faster at 1080p, 1% on the 4-D config-3 model at 4K); FP32 records read it after the encoding.
#ifndef NIV_TC_NRM_EARLY
#define NIV_TC_NRM_EARLY 1
#endif
constexpr bool kNrmEarly = NIV_TC_NRM_EARLY != 0 && kP == 1;

__device__ __forceinline__ float4 rec16_to_float4(uint2 r) {
    const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&r.x));
    const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&r.y));
    return make_float4(a.x, a.y, b.x, b.y);
}
constexpr int kHdr = 128;    // barriers + TMEM address slot at the start of dynamic shared memory
constexpr int kNO = 16;      // rows of the output-layer tile (3 live)
constexpr bool kOutFma = NIV_TC_OUT_FMA != 0;  // output layer on the CUDA cores instead of the tensor core

// Byte offset of element (row r, column k) of a K-major tile with K columns, built from
// 8-row x 16-byte core matrices: adjacent along K 128 B apart, along rows (K/8)*128 B apart.
__host__ __device__ __forceinline__ uint32_t core_off(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

struct TcLayout {
    int32_t K1, W, n_hidden, col_extra;  // col_extra: tile column of n.x (features end before it)
    int32_t col_one;                     // tile column holding the constant 1 (first-layer bias)
    uint32_t w1, wh, wo, bias, wout, total;  // byte offsets inside the packed network
    uint32_t ones, bt;  // NIV_TC_BIAS_MMA: the 128 x 16 ones tile, then the W x 16 bias tiles and 16 x 16 b_out tile
};

__device__ __forceinline__ uint32_t pack_half2(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&h);
}

// FP16 pair (lo, hi) of max(x, 0), rounded to nearest: one conversion with ReLU.
__device__ __forceinline__ uint32_t relu_pack_half2(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.f16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
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

// Issue one layer for each of the kP tiles: sum over K/16 steps of act x W^T into TMEM (tile p
// reads act + p act_stride and accumulates at tmem + p tmem_stride), then signal `bar`.
// ones != 0: then add the bias, ones-tile x bias-tile^T (both K = 16, column 0 live).
__device__ __forceinline__ void issue_layer(uint32_t tmem, uint32_t act, uint32_t w, uint32_t K, uint32_t idesc,
                                            uint32_t bar, uint32_t act_stride = 0, uint32_t tmem_stride = 0,
                                            uint32_t ones = 0u, uint32_t bias = 0u) {
    const uint32_t sbo = (K >> 3) * 128u;
#pragma unroll
    for (int p = 0; p < kP; ++p) {
        for (uint32_t ks = 0; ks < K / 16; ++ks)
            tc::mma_f16(tmem + p * tmem_stride, tc::smem_desc(act + p * act_stride + ks * 256u, 128u, sbo),
                        tc::smem_desc(w + ks * 256u, 128u, sbo), idesc, ks > 0 ? 1u : 0u);
        if (kBiasMma && ones != 0u)
            tc::mma_f16(tmem + p * tmem_stride, tc::smem_desc(ones, 128u, 256u), tc::smem_desc(bias, 128u, 256u),
                        idesc, 1u);
    }
    tc::mma_commit(bar);
}

// Frequency encoding of one record (PE bands, PE > 0 fixed at compile time, PE < 0 taken
// from g): the pairs (sin, cos)(2^b pi u_d) in FP16, d-major then b, columns [0, 6B); the
// columns up to the next multiple of 8 are zero.
template <int PE>
__device__ __forceinline__ void encode_pe(const GridArgs& g, const float* u, uint8_t* s_act, int tid, int K1) {
    if (PE > 0 && PE % 4 == 0) {  // whole 16-byte chunks of 4 pairs
#pragma unroll 1
        for (int q = 0; q < 3 * PE / 4; ++q) {
            const int d = q / (PE / 4), b0 = (q % (PE / 4)) * 4;
            const float ud = d == 0 ? u[0] : (d == 1 ? u[1] : u[2]);
            uint32_t wd[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                float sv, cv;
                niv_pe_pair(ud, b0 + j, sv, cv);
                wd[j] = pack_half2(sv, cv);
            }
            *reinterpret_cast<uint4*>(s_act + core_off(tid, 8 * q, K1)) = make_uint4(wd[0], wd[1], wd[2], wd[3]);
        }
    } else {
        const int B = g.pe_bands, pairs = 3 * B;
        for (int p = 0; p < ((pairs + 3) & ~3); ++p) {
            uint32_t v = 0u;
            if (p < pairs) {
                const int d = p / B;
                float sv, cv;
                niv_pe_pair(d == 0 ? u[0] : (d == 1 ? u[1] : u[2]), p - d * B, sv, cv);
                v = pack_half2(sv, cv);
            }
            *reinterpret_cast<uint32_t*>(s_act + core_off(tid, 2 * p, K1)) = v;
        }
    }
}

// Encode levels [l0, l0 + G) of one record into one 16-byte chunk of FP16 features,
// kILP levels' gathers in flight at a time.
template <int DIMS, int F, typename TabT, int ND = -1>
__device__ __forceinline__ uint4 encode_chunk(const GridArgs& g, const TabT* __restrict__ grid, int l0, int L,
                                              const float* u, const uint2* __restrict__ pair = nullptr) {
    constexpr int NC = 1 << DIMS, G = 8 / F;
    using R = typename NivRaw<F, TabT>::T;
    uint32_t wd[4] = {0u, 0u, 0u, 0u};
    if constexpr (kILP == 1 && std::is_same<TabT, __half>::value) {
#pragma unroll
        for (int q = 0; q < G; ++q) {
            if (l0 + q >= L) continue;
            float acc[F];
            niv_level_features16<DIMS, F, ND>(g, grid + (size_t)g.offset[l0 + q] * F, l0 + q, u, acc, pair);
            if (F == 1) {
                const uint32_t v = (uint32_t)__half_as_ushort(__float2half_rn(acc[0]));
                wd[q >> 1] |= (q & 1) ? (v << 16) : v;
            } else if (F == 2) {
                wd[q % 4] = pack_half2(acc[0], acc[1 % F]);
            } else {
                wd[(2 * q) % 4] = pack_half2(acc[0], acc[1 % F]);
                wd[(2 * q + 1) % 4] = pack_half2(acc[2 % F], acc[3 % F]);
            }
        }
        return make_uint4(wd[0], wd[1], wd[2], wd[3]);
    }
#pragma unroll
    for (int q = 0; q < G; q += kILP) {
        const int la = l0 + q, lb = l0 + q + 1;
        const bool has_a = la < L, has_b = kILP == 2 && (q + 1 < G) && lb < L;
        uint32_t ea[NC], eb[NC];
        float wa[NC], wb[NC];
        R ra[NC], rb[NC];
        if (has_a) niv_level_corners<DIMS, ND>(g, la, u, ea, wa);
        if (has_b) niv_level_corners<DIMS, ND>(g, lb, u, eb, wb);
        if (has_a) niv_level_gather<NC, F, TabT>(grid + (size_t)g.offset[la] * F, ea, ra);
        if (has_b) niv_level_gather<NC, F, TabT>(grid + (size_t)g.offset[lb] * F, eb, rb);
        float acc[F];
#pragma unroll
        for (int h = 0; h < kILP; ++h) {
            if (h == 0 ? !has_a : !has_b) continue;
            niv_level_blend<NC, F>(h == 0 ? ra : rb, h == 0 ? wa : wb, acc);
            const int qq = q + h;
            if (F == 1) {
                const uint32_t v = (uint32_t)__half_as_ushort(__float2half_rn(acc[0]));
                wd[qq >> 1] |= (qq & 1) ? (v << 16) : v;
            } else if (F == 2) {
                wd[qq % 4] = pack_half2(acc[0], acc[1 % F]);
            } else {
                wd[(2 * qq) % 4] = pack_half2(acc[0], acc[1 % F]);
                wd[(2 * qq + 1) % 4] = pack_half2(acc[2 % F], acc[3 % F]);
            }
        }
    }
    return make_uint4(wd[0], wd[1], wd[2], wd[3]);
}

__device__ __forceinline__ void group_sync(int wg) { asm volatile("bar.sync %0, 128;" ::"r"(1 + wg) : "memory"); }

#ifndef NIV_TC_WAIT1
#define NIV_TC_WAIT1 0
#endif
// OR of v over the warpgroup's 128 threads at its named barrier (all of them wait there).
__device__ __forceinline__ bool group_any(int wg, bool v) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 q, %1, 0;\n\t"
        "bar.red.or.pred p, %2, 128, q;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)v), "r"(1 + wg)
        : "memory");
    return r != 0;
}

// Wait for the warpgroup's MMA-completion barrier (phase `parity`), bounded.  NIV_TC_WAIT1: the
// first warp polls the barrier while the other three wait at the named barrier, which takes no
// issue slots; the outcome reaches all four warps through the barrier's OR.  Returns false when
// the wait ran out.
__device__ __forceinline__ bool group_wait_mma(uint32_t bar, uint32_t parity, int warp, int wg) {
    if (!NIV_TC_WAIT1) return tc::mbar_wait_bounded(bar, parity, kWaitLimitNs);
    bool fail = false;
    if (warp == 0) {
        fail = !tc::mbar_wait_bounded(bar, parity, kWaitLimitNs);
        tc::fence_before_sync();
    }
    return !group_any(wg, fail);
}


// kWG independent warpgroups per CTA; each owns a 128-row tile pipeline (activation tile,
// mbarrier, named barrier, 64 TMEM columns) and all share the weights in shared memory.
// LV > 0: the level count is a compile-time constant, so the level loop unrolls fully and
// every per-level constant (resolution, table offset, dense flag) is an immediate operand.
// PE != 0: frequency-encoded model without grid (PE > 0: that many bands, fixed at compile time).
// WT, KT, NHT > 0: network width, first-layer input width and hidden-layer count fixed at
// compile time (loops over layers and tile columns unroll with constant offsets).  ND >= 0:
// levels 0 .. ND-1 are the dense ones.
template <int DIMS, int F, int LV, int PE, typename TabT, int WT = 0, int KT = 0, int NHT = 0, int ND = -1>
__global__ void __launch_bounds__(kT * kWG, NIV_TC_MINB) query_tc_f16_kernel(GridArgs g, IoArgs io,
                                                                const TabT* __restrict__ grid,
                                                                const uint8_t* __restrict__ packed, TcLayout lay,
                                                                int out_act, int64_t n_tiles, uint32_t tmem_cols,
                                                                int* __restrict__ status,
                                                                const uint2* __restrict__ pair) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem);  // one per warpgroup
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + 64);
    uint8_t* s_net = smem + kHdr;
    static_assert(kP == 1 || !kOutFma, "two tiles per warpgroup take the output layer on the tensor core");
    const uint32_t tile_bytes = (uint32_t)kT * (uint32_t)(lay.K1 > lay.W ? lay.K1 : lay.W) * 2u;  // one 128-row tile
    const uint32_t act_bytes = tile_bytes * kP;

    const int wg = threadIdx.x / kT, tid = threadIdx.x % kT, warp = tid >> 5;
    uint8_t* s_act = s_net + ((lay.total + 127u) & ~127u) + wg * act_bytes;
    const int K1 = KT > 0 ? KT : lay.K1, W = WT > 0 ? WT : lay.W, NH = NHT > 0 ? NHT : lay.n_hidden;
    // column of n.x: the features end before it (round_up(L F, 8) for grid models)
    const int col_extra = (LV > 0 && PE == 0) ? ((LV * F + 7) & ~7) : lay.col_extra;

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

    const uint32_t wg_cols = lay.W <= 32 ? 32u : 64u;  // accumulator columns of one 128-row tile
    const uint32_t tmem = *s_tmem + (uint32_t)wg * wg_cols * kP;
    const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t bar = tc::smem_u32(s_bar + wg);
    const uint32_t act_a = tc::smem_u32(s_act), net_a = tc::smem_u32(s_net);
    const float* s_bias = reinterpret_cast<const float*>(s_net + lay.bias);  // layers 1.. and b_out
    const float* s_wout = reinterpret_cast<const float*>(s_net + lay.wout);  // FP32 [3][W]
    const uint32_t idesc_h = tc::idesc_f16(128, W), idesc_o = tc::idesc_f16(128, kNO);
    const int L = LV > 0 ? LV : g.levels;
    constexpr int G = 8 / F;
    uint32_t phase = 0;
    bool ok = true;

    // tile p of this warpgroup's pair is tile (first + p) of the walk; both walkers advance together
    NivTileWalk walk[kP];
#pragma unroll
    for (int p = 0; p < kP; ++p)
        walk[p].init(((int64_t)blockIdx.x * kWG + wg) * kP + p, (int64_t)gridDim.x * kWG * kP, tid, io.image_width);
    for (; walk[0].tile < n_tiles && ok;) {
        int64_t r[kP], rr[kP];
        float u[kP][4];
        uint2 nrm_raw = make_uint2(0u, 0u);
#pragma unroll
        for (int p = 0; p < kP; ++p) {
            r[p] = walk[p].record(tid, io.n, io.image_width);
            rr[p] = r[p] < io.n ? walk[p].source(r[p], io) : 0;
            if (kNrmEarly && io.in_f16) nrm_raw = __ldg(reinterpret_cast<const uint2*>(io.nrm) + rr[p]);
            const float4 pv = niv_load_rec(io.pos, rr[p], io.in_f16);
            u[p][0] = niv_unit(pv.x, g.aabb_min[0], g.inv_ext[0]);
            u[p][1] = niv_unit(pv.y, g.aabb_min[1], g.inv_ext[1]);
            u[p][2] = niv_unit(pv.z, g.aabb_min[2], g.inv_ext[2]);
            u[p][3] = fminf(fmaxf(g.t, 0.0f), 1.0f);
        }

        // ---- 1. encoding -> FP16 input row, one 16-byte chunk per G levels (the kP records of
        // this thread chunk by chunk, so that their independent work interleaves) ----
        if (PE != 0) {
#pragma unroll
            for (int p = 0; p < kP; ++p) encode_pe<PE>(g, u[p], s_act + p * tile_bytes, tid, K1);
        } else if constexpr (LV > 0) {
#pragma unroll
            for (int l0 = 0; l0 < LV; l0 += G)
#pragma unroll
                for (int p = 0; p < kP; ++p)
                    *reinterpret_cast<uint4*>(s_act + p * tile_bytes + core_off(tid, l0 * F, K1)) =
                        encode_chunk<DIMS, F, TabT, ND>(g, grid, l0, LV, u[p], pair);
        } else {
            for (int l0 = 0; l0 < L; l0 += G)
#pragma unroll
                for (int p = 0; p < kP; ++p)
                    *reinterpret_cast<uint4*>(s_act + p * tile_bytes + core_off(tid, l0 * F, K1)) =
                        encode_chunk<DIMS, F>(g, grid, l0, L, u[p]);
        }
#pragma unroll
        for (int p = 0; p < kP; ++p) {
        uint8_t* s_row = s_act + p * tile_bytes;
        // FP32 records: read late, not live during the encoding
        const float4 nv = (kNrmEarly && io.in_f16) ? rec16_to_float4(nrm_raw) : niv_load_rec(io.nrm, rr[p], io.in_f16);
        int tail = 8;  // columns written from col_extra on
        if (g.t_bands == 0) {  // [n.x, n.y, n.z, (t), 1, 0, ...]: the 1 multiplies the first layer's bias column
            const bool has_t = g.n_in > (PE != 0 ? 0 : L * F) + 6 * g.pe_bands + 3;
            const uint32_t one = (uint32_t)__half_as_ushort(__float2half_rn(1.0f));
            uint4 c = make_uint4(pack_half2(nv.x, nv.y), has_t ? pack_half2(nv.z, u[p][3]) : (pack_half2(nv.z, 0.0f) & 0xFFFFu) | (one << 16), 0u, 0u);
            if (has_t) c.z = one;
            *reinterpret_cast<uint4*>(s_row + core_off(tid, col_extra, K1)) = c;
        } else {  // Sec. 6: [n.x, n.y, n.z, sin, cos of 2^b pi t (b < t_bands <= 6), 1, 0, ...]
            float v[16];
#pragma unroll
            for (int i = 0; i < 16; ++i) v[i] = 0.0f;
            v[0] = nv.x;
            v[1] = nv.y;
            v[2] = nv.z;
#pragma unroll
            for (int b = 0; b < 6; ++b)
                if (b < g.t_bands) niv_pe_pair(u[p][3], b, v[3 + 2 * b], v[4 + 2 * b]);
#pragma unroll
            for (int i = 3; i < 16; ++i)
                if (i == 3 + 2 * g.t_bands) v[i] = 1.0f;
            *reinterpret_cast<uint4*>(s_row + core_off(tid, col_extra, K1)) =
                make_uint4(pack_half2(v[0], v[1]), pack_half2(v[2], v[3]), pack_half2(v[4], v[5]), pack_half2(v[6], v[7]));
            if (4 + 2 * g.t_bands > 8) {
                *reinterpret_cast<uint4*>(s_row + core_off(tid, col_extra + 8, K1)) =
                    make_uint4(pack_half2(v[8], v[9]), pack_half2(v[10], v[11]), pack_half2(v[12], v[13]),
                               pack_half2(v[14], v[15]));
                tail = 16;
            }
        }
        for (int k = col_extra + tail; k < K1; k += 8)
            *reinterpret_cast<uint4*>(s_row + core_off(tid, k, K1)) = make_uint4(0u, 0u, 0u, 0u);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        group_sync(wg);

        // ---- 2, 3. hidden layers (the last one feeds the output layer) ----
        uint32_t K = (uint32_t)K1, w_off = lay.w1;
        float z0 = 0.0f, z1 = 0.0f, z2 = 0.0f;
#pragma unroll
        for (int layer = 0; layer < NH && ok; ++layer) {
            if (tid == 0) {
                tc::fence_after_sync();
                issue_layer(tmem, act_a, net_a + w_off, K, idesc_h, bar, tile_bytes, wg_cols,
                            kBiasMma && layer > 0 ? net_a + lay.ones : 0u,
                            net_a + lay.bt + (uint32_t)((layer > 0 ? layer - 1 : 0) * W * 32));
            }
            if (!group_wait_mma(bar, phase, warp, wg)) {
                if (tid == 0) atomicExch(status, 1);
                ok = false;
                break;
            }
            phase ^= 1u;
            tc::fence_after_sync();
            const float* bias = s_bias + (layer - 1) * W;  // layer 0's bias came through the MMA
            const bool last = layer == NH - 1;
            if (kOutFma && last) {
                z0 = s_bias[(NH - 1) * W + 0];
                z1 = s_bias[(NH - 1) * W + 1];
                z2 = s_bias[(NH - 1) * W + 2];
            }
#pragma unroll
            for (int pc = 0; pc < kP * (W / 16); ++pc) {
                const int p = pc / (W / 16), c = pc % (W / 16);
                uint8_t* s_row = s_act + p * tile_bytes;
                float v[16];
                tc::tmem_ld16(tmem_row + (uint32_t)(p * wg_cols + c * 16), v);
                if (layer > 0 && !kBiasMma) {
#pragma unroll
                    for (int j = 0; j < 4; ++j) {  // biases 16-byte aligned: one load per four
                        const float4 b = reinterpret_cast<const float4*>(bias + c * 16)[j];
                        const float2 lo = __fadd2_rn(make_float2(v[4 * j], v[4 * j + 1]), make_float2(b.x, b.y));
                        const float2 hi = __fadd2_rn(make_float2(v[4 * j + 2], v[4 * j + 3]), make_float2(b.z, b.w));
                        v[4 * j] = lo.x;
                        v[4 * j + 1] = lo.y;
                        v[4 * j + 2] = hi.x;
                        v[4 * j + 3] = hi.y;
                    }
                }
                if (kOutFma && last) {
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int o = c * 16 + j;
                        const float a = fmaxf(v[j], 0.0f);
                        z0 = fmaf(s_wout[o], a, z0);
                        z1 = fmaf(s_wout[W + o], a, z1);
                        z2 = fmaf(s_wout[2 * W + o], a, z2);
                    }
                } else {
                    uint32_t h[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) h[j] = relu_pack_half2(v[2 * j], v[2 * j + 1]);
                    *reinterpret_cast<uint4*>(s_row + core_off(tid, c * 16, W)) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4*>(s_row + core_off(tid, c * 16 + 8, W)) = make_uint4(h[4], h[5], h[6], h[7]);
                }
            }
            if (!(kOutFma && last)) {
                tc::fence_async_smem();
                tc::fence_before_sync();
                group_sync(wg);
            }
            w_off = layer == 0 ? lay.wh : w_off + (uint32_t)(W * W * 2);
            K = (uint32_t)W;
        }
        if (!ok) break;

        // ---- 4. output layer (tensor core, N = 16, or CUDA cores above) and softplus ----
        if (!kOutFma) {
            if (tid == 0) {
                tc::fence_after_sync();
                issue_layer(tmem, act_a, net_a + lay.wo, (uint32_t)W, idesc_o, bar, tile_bytes, wg_cols,
                            kBiasMma ? net_a + lay.ones : 0u, net_a + lay.bt + (uint32_t)((NH - 1) * W * 32));
            }
            if (!group_wait_mma(bar, phase, warp, wg)) {
                if (tid == 0) atomicExch(status, 1);
                ok = false;
                break;
            }
            phase ^= 1u;
            tc::fence_after_sync();
        }
#pragma unroll
        for (int p = 0; p < kP; ++p) {
            if (!kOutFma) {
                float z[4];
                tmem_ld4(tmem_row + (uint32_t)(p * wg_cols), z);
                if (kBiasMma) {
                    z0 = z[0];
                    z1 = z[1];
                    z2 = z[2];
                } else {
                    const float* bo = s_bias + (NH - 1) * W;
                    z0 = z[0] + bo[0];
                    z1 = z[1] + bo[1];
                    z2 = z[2] + bo[2];
                }
            }
            if (out_act == 1) {
                z0 = niv_softplus_lp(z0);
                z1 = niv_softplus_lp(z1);
                z2 = niv_softplus_lp(z2);
            }
            if (r[p] < io.n) niv_store_result(io, r[p], z0, z1, z2);
        }
        tc::fence_before_sync();
        group_sync(wg);  // the next tile's encoder overwrites the activation tile
#pragma unroll
        for (int p = 0; p < kP; ++p) walk[p].next();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (threadIdx.x < 32) tc::tmem_dealloc(*s_tmem, tmem_cols);
}

size_t tc_smem_bytes(const TcLayout& lay) {
    const int kmax = lay.K1 > lay.W ? lay.K1 : lay.W;
    return (size_t)kHdr + ((lay.total + 127u) & ~127u) + (size_t)kWG * kP * kT * kmax * 2;
}

template <int DIMS, int F, int LV, int PE = 0, int WT = 0, int KT = 0, int NHT = 0, int ND = -1>
int launch(const niv_model* m, const GridArgs& g, const IoArgs& io, cudaStream_t s, int* status) {
    const TcLayout* lay = reinterpret_cast<const TcLayout*>(m->tc_layout);
    if ((WT > 0 && lay->W != WT) || (KT > 0 && lay->K1 != KT) || (NHT > 0 && lay->n_hidden != NHT))
        return niv_fail(NIV_ERR_UNSUPPORTED, "network shape differs from the kernel's");
    if (ND >= 0 && g.dense_mask != (ND >= 32 ? ~0u : ((1u << ND) - 1u)))
        return niv_fail(NIV_ERR_UNSUPPORTED, "dense levels differ from the kernel's");
    auto kern = query_tc_f16_kernel<DIMS, F, LV, PE, __half, WT, KT, NHT, ND>;
    const __half* grid = m->grid_f16;
    const size_t smem = tc_smem_bytes(*lay);
    int dev = 0;
    NIV_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return niv_fail(NIV_ERR_UNSUPPORTED, "device ordinal above 63");
    // The launch configuration of this kernel instance on a device depends only on its
    // shared-memory size: it is worked out with a dozen runtime queries on first use and
    // reused after (the tuning variables NIV_TC_BLOCKS_PER_SM, NIV_TC_CARVEOUT and
    // NIV_VERBOSE are read then).
    static std::mutex mu;
    static struct { size_t smem; int sms, per_sm; uint32_t cols; } conf[64];
    int sms = 0, per_sm = 0;
    uint32_t cols = 0;
    {
        std::lock_guard<std::mutex> lock(mu);
        if (conf[dev].smem != smem) {
            NIV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
            NIV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
            // Residency from the register and shared-memory budgets (the occupancy API reports a
            // single CTA per SM for kernels that allocate tensor memory).
            cudaFuncAttributes fa;
            NIV_CUDA(cudaFuncGetAttributes(&fa, kern));
            int smem_per_sm = 0, regs_per_sm = 0;
            NIV_CUDA(cudaDeviceGetAttribute(&smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
            NIV_CUDA(cudaDeviceGetAttribute(&regs_per_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev));
            const int by_smem = smem_per_sm / (int)(smem + 1024);  // 1 KB per CTA reserved by the driver
            const int regs = fa.numRegs > 0 ? ((fa.numRegs + 7) & ~7) : 1;
            const int by_regs = regs_per_sm / (kT * kWG * regs);
            per_sm = by_smem < by_regs ? by_smem : by_regs;
            // TMEM is allocated in powers of two from 32 to 512 columns: round the CTA's need up.
            cols = 32u;
            while (cols < (lay->W <= 32 ? 32u : 64u) * (uint32_t)(kWG * kP)) cols <<= 1;
            if (cols > 512u) return niv_fail(NIV_ERR_UNSUPPORTED, "too many warpgroups for tensor memory");
            const int forced = niv_env_int("NIV_TC_BLOCKS_PER_SM", 0);
            if (forced > 0) per_sm = forced;
            if (per_sm > (int)(512 / cols)) per_sm = (int)(512 / cols);  // never oversubscribe TMEM
            if (per_sm < 1) return niv_fail(NIV_ERR_UNSUPPORTED, "tensor-core query kernel does not fit on an SM");
            // Ask for just the shared memory the resident CTAs need: the rest of the SM's unified
            // L1 / shared storage then serves as L1 cache for the feature gathers.
            int carve = (int)((100 * (int64_t)per_sm * (int64_t)(smem + 1024) + smem_per_sm - 1) / smem_per_sm);
            carve = niv_env_int("NIV_TC_CARVEOUT", carve);
            if (carve > 100) carve = 100;
            NIV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, carve));
            if (niv_env_int("NIV_VERBOSE", 0))
                fprintf(stderr, "niv: fp16 query: smem %zu B, regs %d, smem %d/SM, regs %d/SM, launching %d/SM, carveout %d%%\n",
                        smem, fa.numRegs, by_smem, by_regs, per_sm, carve);
            conf[dev].sms = sms;
            conf[dev].per_sm = per_sm;
            conf[dev].cols = cols;
            conf[dev].smem = smem;
        }
        sms = conf[dev].sms;
        per_sm = conf[dev].per_sm;
        cols = conf[dev].cols;
    }
    if (!status) status = niv_status_word();
    if (!status) return niv_fail(NIV_ERR_CUDA, "status word unavailable");
    const int64_t tiles = niv_tile_count_host(io.n, io.image_width);
    const int64_t need = (tiles + kWG * kP - 1) / (kWG * kP);
    const int64_t blocks = need < (int64_t)sms * per_sm ? need : (int64_t)sms * per_sm;
    kern<<<(unsigned)blocks, kT * kWG, smem, s>>>(g, io, grid, m->mlp_tc, *lay, m->d.out_act, tiles, cols,
                                                 status, m->grid_pair16);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}

template <int DIMS>
int by_feat(const niv_model* m, const GridArgs& g, const IoArgs& io, cudaStream_t s, int* status) {
    // fully unrolled encoders for the common level counts (16: configs 1, 3, 4; 8: config 0 and the
    // paper's 8-level model), a runtime loop otherwise
    if (m->d.pe_bands > 0) {  // no grid: the frequency encoding (8 bands in Table 1)
        if constexpr (DIMS == 3) {
            if (m->d.pe_bands == 8) return launch<DIMS, 2, 0, 8>(m, g, io, s, status);
            return launch<DIMS, 2, 0, -1>(m, g, io, s, status);
        }
        return niv_fail(NIV_ERR_UNSUPPORTED, "frequency encoding is 3-D");
    }
    switch (m->d.feat) {
        case 1: return launch<DIMS, 1, 0>(m, g, io, s, status);
        case 2:
            if (g.levels == 16) {
                // fixed shapes of the 16-level models: width 64, 48 input columns, 2 or 3 hidden layers
                const TcLayout* lay = reinterpret_cast<const TcLayout*>(m->tc_layout);
                // and, when the dense levels are the first 2, 4 or 5 (configs 3, 1, 4), that count
                const bool f2 = NIV_TC_FIXW && lay->W == 64 && lay->K1 == 48 && lay->n_hidden == 2;
                const bool f3 = NIV_TC_FIXW && lay->W == 64 && lay->K1 == 48 && lay->n_hidden == 3;
                const uint32_t dm = NIV_TC_ND ? g.dense_mask : 0xFFFFFFFFu;
                if constexpr (DIMS == 3) {
                    if (f2 && dm == 0xFu) return launch<DIMS, 2, 16, 0, 64, 48, 2, 4>(m, g, io, s, status);
                    if (f2 && dm == 0x1Fu) return launch<DIMS, 2, 16, 0, 64, 48, 2, 5>(m, g, io, s, status);
                } else {
                    if (f3 && dm == 0x3u) return launch<DIMS, 2, 16, 0, 64, 48, 3, 2>(m, g, io, s, status);
                }
                if (f2) return launch<DIMS, 2, 16, 0, 64, 48, 2>(m, g, io, s, status);
                if (f3) return launch<DIMS, 2, 16, 0, 64, 48, 3>(m, g, io, s, status);
                if (NIV_TC_FIXW && lay->W == 64) return launch<DIMS, 2, 16, 0, 64>(m, g, io, s, status);
                return launch<DIMS, 2, 16>(m, g, io, s, status);
            }
            if (g.levels == 8) return launch<DIMS, 2, 8>(m, g, io, s, status);
            return launch<DIMS, 2, 0>(m, g, io, s, status);
        case 4:
            if (g.levels == 8) return launch<DIMS, 4, 8>(m, g, io, s, status);
            return launch<DIMS, 4, 0>(m, g, io, s, status);
    }
    return niv_fail(NIV_ERR_UNSUPPORTED, "feat must be 1, 2 or 4");
}

}  // namespace

// Pack the network for the tensor-core kernel from host FP32 parameters:
// [W1 (W x K1, FP16 tile) | hidden W (W x W) ... | W_out (16 x W) | biases of layers 1.. and
// b_out (FP32) | W_out (FP32, 3 x W)].  Input i of the network sits in tile column i for
// the encoded features and in column col_extra + (i - L*F) for n and t, col_extra =
// round_up(L*F, 8); the first layer's bias sits in column col_one, which the kernel
// fills with 1 in every input row.
int niv_pack_tc(niv_model* m, const float* mlp_host, cudaStream_t s) {
    const int W = m->d.width, nh = m->d.n_hidden, n_in = m->n_in;
    const int LF = m->d.levels * m->d.feat + 6 * m->d.pe_bands;  // encoding values
    TcLayout lay;
    memset(&lay, 0, sizeof lay);
    lay.col_extra = (LF + 7) & ~7;
    lay.col_one = lay.col_extra + m->d.in_extra + 2 * m->d.t_bands;
    lay.K1 = (lay.col_one + 1 + 15) & ~15;
    lay.W = W;
    lay.n_hidden = nh;
    auto up = [](uint32_t x) { return (x + 127u) & ~127u; };
    lay.w1 = 0;
    lay.wh = up(lay.w1 + (uint32_t)(W * lay.K1 * 2));
    lay.wo = up(lay.wh + (uint32_t)((nh - 1) * W * W * 2));
    lay.bias = up(lay.wo + (uint32_t)(kNO * W * 2));
    lay.wout = up(lay.bias + (uint32_t)(((nh - 1) * W + 4) * 4));
    lay.total = up(lay.wout + (uint32_t)(3 * W * 4));
    if (kBiasMma) {
        lay.ones = lay.total;
        lay.bt = up(lay.ones + (uint32_t)(kT * 16 * 2));
        lay.total = up(lay.bt + (uint32_t)(((nh - 1) * W + kNO) * 16 * 2));
    }
    static_assert(sizeof(TcLayout) <= sizeof(((niv_model*)0)->tc_layout), "layout slot too small");
    memcpy(m->tc_layout, &lay, sizeof lay);
    std::vector<uint8_t> buf(lay.total, 0);
    auto put = [&](uint32_t base, int r, int k, int K, float v) {
        __half h = __float2half_rn(v);
        memcpy(&buf[base + core_off(r, k, K)], &h, 2);
    };
    float* bias = reinterpret_cast<float*>(&buf[lay.bias]);
    float* wout = reinterpret_cast<float*>(&buf[lay.wout]);
    auto h16 = [](float v) { return __half2float(__float2half_rn(v)); };  // FP16-stored parameters
    const float* p = mlp_host;
    for (int r = 0; r < W; ++r)
        for (int i = 0; i < n_in; ++i) put(lay.w1, r, i < LF ? i : lay.col_extra + (i - LF), lay.K1, p[(size_t)r * n_in + i]);
    p += (size_t)W * n_in;
    for (int r = 0; r < W; ++r) put(lay.w1, r, lay.col_one, lay.K1, p[r]);
    p += W;
    for (int h = 1; h < nh; ++h) {
        const uint32_t base = lay.wh + (uint32_t)((h - 1) * W * W * 2);
        for (int r = 0; r < W; ++r)
            for (int k = 0; k < W; ++k) put(base, r, k, W, p[(size_t)r * W + k]);
        p += (size_t)W * W;
        for (int r = 0; r < W; ++r) bias[(h - 1) * W + r] = h16(p[r]);
        p += W;
    }
    for (int r = 0; r < 3; ++r)
        for (int k = 0; k < W; ++k) {
            put(lay.wo, r, k, W, p[(size_t)r * W + k]);
            wout[r * W + k] = h16(p[(size_t)r * W + k]);
        }
    p += 3 * W;
    for (int r = 0; r < 3; ++r) bias[(nh - 1) * W + r] = h16(p[r]);
    if (kBiasMma) {  // column 0 of the ones tile is 1; column 0 of each bias tile the layer's biases
        for (int r = 0; r < kT; ++r) put(lay.ones, r, 0, 16, 1.0f);
        for (int h = 1; h < nh; ++h)
            for (int r = 0; r < W; ++r) put(lay.bt + (uint32_t)((h - 1) * W * 32), r, 0, 16, bias[(h - 1) * W + r]);
        for (int r = 0; r < 3; ++r) put(lay.bt + (uint32_t)((nh - 1) * W * 32), r, 0, 16, bias[(nh - 1) * W + r]);
    }
    if (m->mlp_tc_bytes < lay.total) {
        cudaFree(m->mlp_tc);
        m->mlp_tc = nullptr;
        m->mlp_tc_bytes = 0;
        NIV_CUDA(cudaMalloc(&m->mlp_tc, lay.total));
        m->mlp_tc_bytes = lay.total;
    }
    NIV_CUDA(cudaMemcpyAsync(m->mlp_tc, buf.data(), lay.total, cudaMemcpyHostToDevice, s));
    NIV_CUDA(cudaStreamSynchronize(s));
    return NIV_OK;
}

int niv_launch_query_tc(const niv_model* m, const GridArgs& g, const IoArgs& io, int precision, cudaStream_t s,
                        int* status) {
    if (precision != NIV_FP16) return niv_fail(NIV_ERR_UNSUPPORTED, "tensor-core path: precision not supported");
    // niv_create leaves the packed network unset (a zero layout would pass the shape checks
    // below and launch the kernel on a null weight pointer)
    if (!m->mlp_tc) return niv_fail(NIV_ERR_ARG, "parameters not set: call niv_set_params or niv_load first");
    const TcLayout* lay = reinterpret_cast<const TcLayout*>(m->tc_layout);
    if (lay->K1 > 128) return niv_fail(NIV_ERR_UNSUPPORTED, "tensor-core path needs a network input of <= 120 values");
    return m->d.dims == 4 ? by_feat<4>(m, g, io, s, status) : by_feat<3>(m, g, io, s, status);
}

// ---- tensor-core operand-layout self-test ----
// D[128][64] = A[128][K] * B[64][K]^T with small integers (exact in FP32), A and B written
// in the same canonical layouts the query kernels use.  mode 0: FP16, K = 32; mode 1: the
// same with the two descriptor stride fields exchanged (a diagnostic of the layout
// convention; both variants address only inside the operand buffers); mode 2: E4M3, K = 64.
namespace {
__global__ void __launch_bounds__(128) tc_selftest_kernel(int mode, float* __restrict__ out, int* __restrict__ status) {
    __shared__ __align__(1024) uint8_t s_a[128 * 32 * 2];
    __shared__ __align__(1024) uint8_t s_b[64 * 32 * 2];
    __shared__ uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    const int t = threadIdx.x, warp = t >> 5;
    const bool f8 = mode == 2;
    const int K = f8 ? 64 : 32;
    for (int k = 0; k < K; ++k) {
        const int a = (t * 3 + k * 5) % 7 - 3;
        if (f8) s_a[(t >> 3) * 512 + (k >> 4) * 128 + (t & 7) * 16 + (k & 15)] =
            (uint8_t)__nv_cvt_float_to_fp8((float)a, __NV_SATFINITE, __NV_E4M3);
        else *reinterpret_cast<__half*>(s_a + core_off(t, k, 32)) = __int2half_rn(a);
    }
    if (t < 64)
        for (int k = 0; k < K; ++k) {
            const int b = (t * 5 + k * 3) % 5 - 2;
            if (f8) s_b[(t >> 3) * 512 + (k >> 4) * 128 + (t & 7) * 16 + (k & 15)] =
                (uint8_t)__nv_cvt_float_to_fp8((float)b, __NV_SATFINITE, __NV_E4M3);
            else *reinterpret_cast<__half*>(s_b + core_off(t, k, 32)) = __int2half_rn(b);
        }
    if (t == 0) {
        tc::mbar_init(&s_bar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&s_tmem), 64);
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = s_tmem;
    const uint32_t lbo = mode == 1 ? 512u : 128u, sbo = mode == 1 ? 128u : 512u;
    if (t == 0) {
        for (int ks = 0; ks < 2; ++ks) {
            const uint32_t kstep = (uint32_t)ks * 256u;  // two core matrices along K
            const uint64_t ad = tc::smem_desc(tc::smem_u32(s_a) + kstep, lbo, sbo);
            const uint64_t bd = tc::smem_desc(tc::smem_u32(s_b) + kstep, lbo, sbo);
            if (f8) tc::mma_e4m3(tmem, ad, bd, tc::idesc_e4m3(128, 64), ks > 0);
            else tc::mma_f16(tmem, ad, bd, tc::idesc_f16(128, 64), ks > 0);
        }
        tc::mma_commit(tc::smem_u32(&s_bar));
    }
    const bool ok = tc::mbar_wait_bounded(tc::smem_u32(&s_bar), 0, kWaitLimitNs);
    if (!ok) atomicExch(status, 2);
    tc::fence_after_sync();
    if (ok) {
        for (int c = 0; c < 4; ++c) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(c * 16), v);
#pragma unroll
            for (int j = 0; j < 16; ++j) out[t * 64 + c * 16 + j] = v[j];
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 64);
}
}  // namespace

// ---- expiry of a bounded wait ----
// The same bounded mbarrier wait the query kernels use, on a barrier whose phase nothing
// completes: the kernel holds TMEM like a query kernel, issues no tensor-core operation (so
// nothing is in flight when it gives up), waits limit_ns, latches failure code 3 in the
// status word, frees its TMEM and returns.
namespace {
__global__ void __launch_bounds__(128) wait_expiry_kernel(uint64_t limit_ns, int* __restrict__ status) {
    __shared__ __align__(8) uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) {
        tc::mbar_init(&s_bar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(&s_tmem), 32);
        tc::tmem_relinquish();
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const bool ok = tc::mbar_wait_bounded(tc::smem_u32(&s_bar), 0, limit_ns);  // no arrival will come
    if (!ok && threadIdx.x == 0) atomicExch(status, 3);
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(s_tmem, 32);
}
}  // namespace

extern "C" int niv_selftest_wait_expiry(uint32_t limit_us, niv_stream stream) {
    if (limit_us < 1 || limit_us > 1000000) return niv_fail(NIV_ERR_ARG, "limit_us must be in [1, 1000000]");
    int* status = niv_status_word();
    if (!status) return niv_fail(NIV_ERR_CUDA, "status word unavailable");
    wait_expiry_kernel<<<1, 128, 0, (cudaStream_t)stream>>>((uint64_t)limit_us * 1000ull, status);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}

extern "C" int niv_selftest_mma(int32_t mode, float* out, niv_stream stream) {
    if (!out) return niv_fail(NIV_ERR_ARG, "out is NULL");
    if (mode < 0 || mode > 2) return niv_fail(NIV_ERR_ARG, "mode must be 0, 1 or 2");
    int* status = niv_status_word();
    if (!status) return niv_fail(NIV_ERR_CUDA, "status word unavailable");
    tc_selftest_kernel<<<1, 128, 0, (cudaStream_t)stream>>>(mode, out, status);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}
