// Fused query path on the 5th-generation tensor cores (sm_103a).
//
// One CTA of 128 threads owns a tile of 128 G-buffer records at a time (a 16 x 8
// pixel block for images) and walks tiles persistently.  Per tile:
//   1. every thread encodes its own record (Sec. 4.1: per level the cell, the
//      2^d corner indices -- dense or hashed --, FP16 feature gathers served from
//      L2, multilinear weights in FP32) and writes its row of the network input
//      [features, n, (t), 0-pad] as FP16 into a shared-memory tile laid out in the
//      tensor core's canonical K-major format;
//   2. one thread issues tcgen05.mma (M = 128 records, N = width, K = 16 per
//      instruction) with the weights resident in shared memory; the FP32
//      accumulator lives in tensor memory (TMEM);
//   3. each warp reads its 32 rows back with tcgen05.ld, adds the bias, applies
//      ReLU and writes the next layer's FP16 input tile; repeat per hidden layer;
//   4. the 3-wide output layer (192 multiply-adds per record) and softplus run in
//      FP32 on the CUDA cores straight from the last accumulator, and E is stored.
// Every wait on the MMA-completion barrier is bounded (2 s); on expiry the kernel
// records a failure in the status word, releases its TMEM and returns.
#include <vector>

#include "niv_internal.cuh"
#include "tc_ptx.cuh"

namespace {

constexpr int kT = 128;
constexpr uint64_t kWaitLimitNs = 2000000000ull;
constexpr int kHdr = 128;  // barrier + TMEM address slot at the start of dynamic shared memory

// Byte offset of element (row r, column k) of a K-major tile with K columns, built from
// 8-row x 16-byte core matrices: adjacent along K 128 B apart, along rows (K/8)*128 B apart.
__host__ __device__ __forceinline__ uint32_t core_off(int r, int k, int K) {
    return (uint32_t)((r >> 3) * (K >> 3) * 128 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

struct TcLayout {
    int32_t K1, W, n_hidden, pad;
    uint32_t w1, wh, bias, wout, total;  // byte offsets inside the packed network
};

template <int DIMS, int F>
__device__ __forceinline__ void encode_level(const GridArgs& g, const __half* __restrict__ grid16, int l,
                                             const float* u, float* acc) {
    const int32_t N = g.res[l];
    const bool dense = (g.dense_mask >> l) & 1u;
    uint32_t ci[DIMS];
    float cw[DIMS];
#pragma unroll
    for (int d = 0; d < DIMS; ++d) niv_cell(u[d], N, ci[d], cw[d]);
    uint32_t e[1 << DIMS];
    float wc[1 << DIMS];
#pragma unroll
    for (int c = 0; c < (1 << DIMS); ++c) {
        uint32_t v[DIMS];
        float w = 1.0f;
#pragma unroll
        for (int d = 0; d < DIMS; ++d) {
            const int bit = (c >> d) & 1;
            v[d] = ci[d] + bit;
            w *= bit ? cw[d] : 1.0f - cw[d];
        }
        e[c] = niv_vertex_index<DIMS>(dense, (uint32_t)N + 1u, v, g.hash_mask, g.prime_t);
        wc[c] = w;
    }
#pragma unroll
    for (int j = 0; j < F; ++j) acc[j] = 0.0f;
    if (F == 2) {
        const uint32_t* tab = reinterpret_cast<const uint32_t*>(grid16) + g.offset[l];
        uint32_t raw[1 << DIMS];
#pragma unroll
        for (int c = 0; c < (1 << DIMS); ++c) raw[c] = __ldg(tab + e[c]);
#pragma unroll
        for (int c = 0; c < (1 << DIMS); ++c) {
            const float2 f = __half22float2(*reinterpret_cast<const __half2*>(&raw[c]));
            acc[0] = fmaf(wc[c], f.x, acc[0]);
            acc[1 % F] = fmaf(wc[c], f.y, acc[1 % F]);
        }
    } else if (F == 4) {
        const uint2* tab = reinterpret_cast<const uint2*>(grid16) + g.offset[l];
        uint2 raw[1 << DIMS];
#pragma unroll
        for (int c = 0; c < (1 << DIMS); ++c) raw[c] = __ldg(tab + e[c]);
#pragma unroll
        for (int c = 0; c < (1 << DIMS); ++c) {
            const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw[c].x));
            const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw[c].y));
            acc[0] = fmaf(wc[c], a.x, acc[0]);
            acc[1 % F] = fmaf(wc[c], a.y, acc[1 % F]);
            acc[2 % F] = fmaf(wc[c], b.x, acc[2 % F]);
            acc[3 % F] = fmaf(wc[c], b.y, acc[3 % F]);
        }
    } else {
        const __half* tab = grid16 + g.offset[l];
#pragma unroll
        for (int c = 0; c < (1 << DIMS); ++c) acc[0] = fmaf(wc[c], __half2float(tab[e[c]]), acc[0]);
    }
}

template <int DIMS, int F>
__global__ void __launch_bounds__(kT) query_tc_f16_kernel(GridArgs g, IoArgs io, const __half* __restrict__ grid16,
                                                           const uint8_t* __restrict__ packed, TcLayout lay,
                                                           int out_act, int64_t n_tiles, uint32_t tmem_cols,
                                                           int* __restrict__ status) {
    extern __shared__ __align__(1024) uint8_t smem[];
    uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem);
    uint32_t* s_tmem = reinterpret_cast<uint32_t*>(smem + 8);
    uint8_t* s_net = smem + kHdr;
    uint8_t* s_act = s_net + ((lay.total + 1023u) & ~1023u);

    const int tid = threadIdx.x, warp = tid >> 5;
    const int K1 = lay.K1, W = lay.W;

    for (uint32_t i = tid; i < lay.total / 16; i += kT)
        reinterpret_cast<uint4*>(s_net)[i] = __ldg(reinterpret_cast<const uint4*>(packed) + i);
    if (tid == 0) {
        tc::mbar_init(s_bar, 1);
        tc::fence_mbar_init();
    }
    if (warp == 0) {
        tc::tmem_alloc(tc::smem_u32(s_tmem), tmem_cols);
        tc::tmem_relinquish();
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();

    const uint32_t tmem = *s_tmem;
    const uint32_t tmem_row = tmem + ((uint32_t)(warp * 32) << 16);
    const uint32_t bar = tc::smem_u32(s_bar);
    const uint32_t act_a = tc::smem_u32(s_act), net_a = tc::smem_u32(s_net);
    const uint32_t idesc = tc::idesc_f16(128, W);
    const float* s_bias = reinterpret_cast<const float*>(s_net + lay.bias);
    const float* s_wout = reinterpret_cast<const float*>(s_net + lay.wout);
    const int LF = g.levels * F;
    uint32_t phase = 0;
    bool ok = true;

    for (int64_t tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x) {
        const int64_t r = niv_record_of(tile, tid, io.n, io.image_width);
        const bool valid = r < io.n;
        const int64_t rr = valid ? r : 0;
        const float4 p = niv_load_rec(io.pos, rr, io.in_f16);
        const float4 nv = niv_load_rec(io.nrm, rr, io.in_f16);
        float u[4];
        u[0] = niv_unit(p.x, g.aabb_min[0], g.inv_ext[0]);
        u[1] = niv_unit(p.y, g.aabb_min[1], g.inv_ext[1]);
        u[2] = niv_unit(p.z, g.aabb_min[2], g.inv_ext[2]);
        u[3] = fminf(fmaxf(g.t, 0.0f), 1.0f);

        // ---- 1. encoding -> FP16 input row ----
        for (int l = 0; l < g.levels; ++l) {
            float acc[F];
            encode_level<DIMS, F>(g, grid16, l, u, acc);
            if (F == 2) {
                *reinterpret_cast<__half2*>(s_act + core_off(tid, 2 * l, K1)) = __floats2half2_rn(acc[0], acc[1 % F]);
            } else if (F == 4) {
                __half2 a = __floats2half2_rn(acc[0], acc[1 % F]), b = __floats2half2_rn(acc[2 % F], acc[3 % F]);
                uint2 w2;
                w2.x = *reinterpret_cast<uint32_t*>(&a);
                w2.y = *reinterpret_cast<uint32_t*>(&b);
                *reinterpret_cast<uint2*>(s_act + core_off(tid, 4 * l, K1)) = w2;
            } else {
                *reinterpret_cast<__half*>(s_act + core_off(tid, l, K1)) = __float2half_rn(acc[0]);
            }
        }
        for (int k = LF; k < K1; ++k) {
            float x = 0.0f;
            if (k == LF) x = nv.x;
            else if (k == LF + 1) x = nv.y;
            else if (k == LF + 2) x = nv.z;
            else if (k == LF + 3 && g.n_in > LF + 3) x = u[3];
            *reinterpret_cast<__half*>(s_act + core_off(tid, k, K1)) = __float2half_rn(x);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();

        // ---- 2..4. network ----
        int K = K1;
        uint32_t w_off = lay.w1;
        for (int layer = 0; layer < lay.n_hidden; ++layer) {
            if (tid == 0) {
                tc::fence_after_sync();
                const uint32_t sbo = (uint32_t)(K >> 3) * 128u;
                for (int ks = 0; ks < K / 16; ++ks) {
                    const uint64_t ad = tc::smem_desc(act_a + ks * 256u, 128u, sbo);
                    const uint64_t bd = tc::smem_desc(net_a + w_off + ks * 256u, 128u, sbo);
                    tc::mma_f16(tmem, ad, bd, idesc, ks > 0 ? 1u : 0u);
                }
                tc::mma_commit(bar);
            }
            if (!tc::mbar_wait_bounded(bar, phase, kWaitLimitNs)) {
                atomicExch(status, 1);
                ok = false;
                break;
            }
            phase ^= 1u;
            tc::fence_after_sync();
            const float* bias = s_bias + layer * W;
            if (layer < lay.n_hidden - 1) {
                // hidden epilogue: relu(acc + b) -> FP16 input tile of the next layer (K = W)
                for (int c = 0; c < W / 16; ++c) {
                    float v[16];
                    tc::tmem_ld16(tmem_row + (uint32_t)(c * 16), v);
                    uint32_t h[8];
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        __half2 hh = __floats2half2_rn(fmaxf(v[2 * j] + bias[c * 16 + 2 * j], 0.0f),
                                                       fmaxf(v[2 * j + 1] + bias[c * 16 + 2 * j + 1], 0.0f));
                        h[j] = *reinterpret_cast<uint32_t*>(&hh);
                    }
                    *reinterpret_cast<uint4*>(s_act + core_off(tid, c * 16, W)) = make_uint4(h[0], h[1], h[2], h[3]);
                    *reinterpret_cast<uint4*>(s_act + core_off(tid, c * 16 + 8, W)) = make_uint4(h[4], h[5], h[6], h[7]);
                }
                tc::fence_async_smem();
                tc::fence_before_sync();
                __syncthreads();
                w_off = (layer == 0) ? lay.wh : w_off + (uint32_t)(W * W * 2);
                K = W;
            } else {
                // output layer on the CUDA cores: z = W_out relu(acc + b) + b_out, E = softplus(z)
                float z0 = s_wout[3 * W + 0], z1 = s_wout[3 * W + 1], z2 = s_wout[3 * W + 2];
                for (int c = 0; c < W / 16; ++c) {
                    float v[16];
                    tc::tmem_ld16(tmem_row + (uint32_t)(c * 16), v);
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int o = c * 16 + j;
                        const float a = fmaxf(v[j] + bias[o], 0.0f);
                        z0 = fmaf(s_wout[o], a, z0);
                        z1 = fmaf(s_wout[W + o], a, z1);
                        z2 = fmaf(s_wout[2 * W + o], a, z2);
                    }
                }
                if (out_act == 1) {
                    z0 = niv_softplus(z0);
                    z1 = niv_softplus(z1);
                    z2 = niv_softplus(z2);
                }
                if (valid) niv_store_rec(io.out, r, z0, z1, z2, io.out_f16);
                tc::fence_before_sync();
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, tmem_cols);
}

template <int DIMS, int F>
int launch(const niv_model* m, const GridArgs& g, const IoArgs& io, cudaStream_t s) {
    const TcLayout* lay = reinterpret_cast<const TcLayout*>(m->tc_layout);
    auto kern = query_tc_f16_kernel<DIMS, F>;
    const int kmax = lay->K1 > lay->W ? lay->K1 : lay->W;
    const size_t smem = kHdr + ((lay->total + 1023u) & ~1023u) + (size_t)kT * kmax * 2;
    NIV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int dev = 0, sms = 0, per_sm = 0;
    NIV_CUDA(cudaGetDevice(&dev));
    NIV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    NIV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kT, smem));
    const uint32_t cols = lay->W <= 32 ? 32u : 64u;
    if (per_sm > (int)(512 / cols)) per_sm = (int)(512 / cols);  // never oversubscribe TMEM
    if (per_sm < 1) return niv_fail(NIV_ERR_UNSUPPORTED, "tensor-core query kernel does not fit on an SM");
    int* status = niv_status_word();
    if (!status) return niv_fail(NIV_ERR_CUDA, "status word unavailable");
    const int64_t tiles = niv_tile_count_host(io.n, io.image_width);
    const int64_t blocks = tiles < (int64_t)sms * per_sm ? tiles : (int64_t)sms * per_sm;
    kern<<<(unsigned)blocks, kT, smem, s>>>(g, io, m->grid_f16, m->mlp_tc, *lay, m->d.out_act, tiles, cols, status);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}

template <int DIMS>
int by_feat(const niv_model* m, const GridArgs& g, const IoArgs& io, cudaStream_t s) {
    switch (m->d.feat) {
        case 1: return launch<DIMS, 1>(m, g, io, s);
        case 2: return launch<DIMS, 2>(m, g, io, s);
        case 4: return launch<DIMS, 4>(m, g, io, s);
    }
    return niv_fail(NIV_ERR_UNSUPPORTED, "feat must be 1, 2 or 4");
}

}  // namespace

// Pack the network for the tensor-core kernel from host FP32 parameters:
// [W1 fp16 tile (W x K1) | hidden fp16 tiles (W x W) | biases fp32 | W_out fp32 (3 x W) + b_out].
int niv_pack_tc(niv_model* m, const float* mlp_host, cudaStream_t s) {
    const int W = m->d.width, nh = m->d.n_hidden, n_in = m->n_in;
    const int K1 = (n_in + 15) & ~15;
    TcLayout lay;
    memset(&lay, 0, sizeof lay);
    lay.K1 = K1;
    lay.W = W;
    lay.n_hidden = nh;
    auto up = [](uint32_t x) { return (x + 127u) & ~127u; };
    lay.w1 = 0;
    lay.wh = up(lay.w1 + (uint32_t)(W * K1 * 2));
    lay.bias = up(lay.wh + (uint32_t)((nh - 1) * W * W * 2));
    lay.wout = up(lay.bias + (uint32_t)(nh * W * 4));
    lay.total = up(lay.wout + (uint32_t)((3 * W + 3) * 4));
    static_assert(sizeof(TcLayout) <= sizeof(((niv_model*)0)->tc_layout), "layout slot too small");
    memcpy(m->tc_layout, &lay, sizeof lay);
    std::vector<uint8_t> buf(lay.total, 0);
    auto put_tile = [&](uint32_t base, const float* Wsrc, int rows, int cols, int K) {
        for (int r = 0; r < rows; ++r)
            for (int k = 0; k < cols; ++k) {
                __half h = __float2half_rn(Wsrc[(size_t)r * cols + k]);
                memcpy(&buf[base + core_off(r, k, K)], &h, 2);
            }
    };
    const float* p = mlp_host;
    float* bias = reinterpret_cast<float*>(&buf[lay.bias]);
    put_tile(lay.w1, p, W, n_in, K1);
    p += (size_t)W * n_in;
    memcpy(bias, p, sizeof(float) * W);
    p += W;
    for (int h = 1; h < nh; ++h) {
        put_tile(lay.wh + (uint32_t)((h - 1) * W * W * 2), p, W, W, W);
        p += (size_t)W * W;
        memcpy(bias + h * W, p, sizeof(float) * W);
        p += W;
    }
    memcpy(&buf[lay.wout], p, sizeof(float) * (3 * W + 3));
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

int niv_launch_query_tc(const niv_model* m, const GridArgs& g, const IoArgs& io, int precision, cudaStream_t s) {
    if (precision != NIV_FP16) return niv_fail(NIV_ERR_UNSUPPORTED, "tensor-core path: precision not supported");
    if (m->n_in > 64) return niv_fail(NIV_ERR_UNSUPPORTED, "tensor-core path needs levels*feat + in_extra <= 64");
    return m->d.dims == 4 ? by_feat<4>(m, g, io, s) : by_feat<3>(m, g, io, s);
}

// ---- tensor-core operand-layout self-test ----
// D[128][64] = A[128][32] * B[64][32]^T with small integers (exact in FP32), A and B
// written in the same canonical layout as the query kernels use.  `swap` exchanges
// the two descriptor stride fields (a diagnostic of the layout convention); both
// variants address only inside the 12 KB operand area.
namespace {
__global__ void __launch_bounds__(128) tc_selftest_kernel(int swap, float* __restrict__ out, int* __restrict__ status) {
    __shared__ __align__(1024) uint8_t s_a[128 * 32 * 2];
    __shared__ __align__(1024) uint8_t s_b[64 * 32 * 2];
    __shared__ uint64_t s_bar;
    __shared__ uint32_t s_tmem;
    const int t = threadIdx.x, warp = t >> 5;
    for (int k = 0; k < 32; ++k)
        *reinterpret_cast<__half*>(s_a + core_off(t, k, 32)) = __int2half_rn((t * 3 + k * 5) % 7 - 3);
    if (t < 64)
        for (int k = 0; k < 32; ++k)
            *reinterpret_cast<__half*>(s_b + core_off(t, k, 32)) = __int2half_rn((t * 5 + k * 3) % 5 - 2);
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
    const uint32_t lbo = swap ? 512u : 128u, sbo = swap ? 128u : 512u;
    if (t == 0) {
        for (int ks = 0; ks < 2; ++ks) {
            const uint32_t kstep = (uint32_t)ks * 256u;  // two core matrices along K
            tc::mma_f16(tmem, tc::smem_desc(tc::smem_u32(s_a) + kstep, lbo, sbo),
                        tc::smem_desc(tc::smem_u32(s_b) + kstep, lbo, sbo), tc::idesc_f16(128, 64), ks > 0);
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

extern "C" int niv_selftest_mma(int32_t swap_strides, float* out, niv_stream stream) {
    if (!out) return niv_fail(NIV_ERR_ARG, "out is NULL");
    int* status = niv_status_word();
    if (!status) return niv_fail(NIV_ERR_CUDA, "status word unavailable");
    tc_selftest_kernel<<<1, 128, 0, (cudaStream_t)stream>>>(swap_strides, out, status);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}
