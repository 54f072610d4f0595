// Plain FP32 query path (the baseline beside the fused tensor-core paths).
//
// One thread per query on the CUDA cores; FP32 grid features, weights and
// arithmetic throughout.  Steps per query (Sec. 4.4 with the Sec. 4.1 model):
//   load the G-buffer record -> normalise -> per level: cell, 2^d corner
//   indices (dense or hashed), gathers, multilinear interpolation -> network
//   input [features, n, (t)] -> ReLU hidden layers -> softplus output -> store.
// Network weights live in shared memory and are read as warp-wide broadcasts;
// the per-thread input vector sits in a [k][128] shared-memory column.  The products run
// on the packed FP32 pipe (NIV_FP32_PACKED): two FP32 FMAs per instruction, each lane an
// ordinary FP32 FMA -- over output pairs in the first layer, over even and odd inputs
// (two partial sums, added at the end) in the others.
#include "niv_internal.cuh"

#ifndef NIV_FP32_PACKED
#define NIV_FP32_PACKED 1
#endif

namespace {

constexpr int kThreads = 128;

// a + sum_i w[i] h[i] over W inputs (w: shared-memory row, 16-byte aligned).
template <int W>
__device__ __forceinline__ float dot_row(const float* w, const float* h, float a) {
    const float4* wrow = reinterpret_cast<const float4*>(w);
    if (NIV_FP32_PACKED) {
        float2 acc = make_float2(a, 0.0f);  // even and odd inputs
#pragma unroll
        for (int q = 0; q < W / 4; ++q) {
            const float4 w4 = wrow[q];
            acc = __ffma2_rn(make_float2(w4.x, w4.y), make_float2(h[4 * q + 0], h[4 * q + 1]), acc);
            acc = __ffma2_rn(make_float2(w4.z, w4.w), make_float2(h[4 * q + 2], h[4 * q + 3]), acc);
        }
        return acc.x + acc.y;
    }
#pragma unroll
    for (int q = 0; q < W / 4; ++q) {
        const float4 w4 = wrow[q];
        a = fmaf(w4.x, h[4 * q + 0], a);
        a = fmaf(w4.y, h[4 * q + 1], a);
        a = fmaf(w4.z, h[4 * q + 2], a);
        a = fmaf(w4.w, h[4 * q + 3], a);
    }
    return a;
}

template <int DIMS, int F, int W>
__global__ void __launch_bounds__(kThreads) query_fp32_kernel(GridArgs g, IoArgs io, const float* __restrict__ grid,
                                                               const float* __restrict__ mlp, int mlp_len,
                                                               int mlp_stride, int n_hidden, int out_act,
                                                               int64_t n_tiles) {
    extern __shared__ float smem[];
    float* s_w = smem;
    float* s_x = smem + mlp_stride;  // [max(n_in, W)][kThreads]
    for (int i = threadIdx.x; i < mlp_len; i += kThreads) s_w[i] = mlp[i];
    __syncthreads();

    const int k = threadIdx.x;
    const int LG = g.levels * F, LF = LG + 6 * g.pe_bands;  // grid values, all encoding values
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t r = niv_record_of(tile, k, io.n, io.image_width);
        const bool valid = r < io.n;
        const int64_t rr = valid ? niv_source_of(io, r) : 0;
        const float4 p = niv_load_rec(io.pos, rr, io.in_f16);
        const float4 nv = niv_load_rec(io.nrm, rr, io.in_f16);
        float u[4];
        u[0] = niv_unit(p.x, g.aabb_min[0], g.inv_ext[0]);
        u[1] = niv_unit(p.y, g.aabb_min[1], g.inv_ext[1]);
        u[2] = niv_unit(p.z, g.aabb_min[2], g.inv_ext[2]);
        u[3] = fminf(fmaxf(g.t, 0.0f), 1.0f);

        // ---- encoding ----
        for (int l = 0; l < g.levels; ++l) {
            float acc[F];
            niv_encode_level<DIMS, F, float>(g, grid, l, u, acc);
#pragma unroll
            for (int j = 0; j < F; ++j) s_x[(l * F + j) * kThreads + k] = acc[j];
        }
        for (int d = 0; d < 3 && g.pe_bands > 0; ++d)
            for (int b = 0; b < g.pe_bands; ++b) {
                float sv, cv;
                niv_pe_pair(u[d], b, sv, cv);
                s_x[(LG + 2 * (d * g.pe_bands + b)) * kThreads + k] = sv;
                s_x[(LG + 2 * (d * g.pe_bands + b) + 1) * kThreads + k] = cv;
            }
        s_x[(LF + 0) * kThreads + k] = nv.x;
        s_x[(LF + 1) * kThreads + k] = nv.y;
        s_x[(LF + 2) * kThreads + k] = nv.z;
        if (g.t_bands > 0) {  // Sec. 6: the scene parameter frequency-encoded after n
            for (int b = 0; b < g.t_bands; ++b) {
                float sv, cv;
                niv_pe_pair(u[3], b, sv, cv);
                s_x[(LF + 3 + 2 * b) * kThreads + k] = sv;
                s_x[(LF + 4 + 2 * b) * kThreads + k] = cv;
            }
        } else if (g.n_in > LF + 3) {
            s_x[(LF + 3) * kThreads + k] = u[3];
        }

        // ---- first hidden layer: x (shared column) -> h (registers) ----
        const float* W1t = s_w;  // [n_in][W]
        const float* b1 = W1t + g.n_in * W;
        float h[W];
#pragma unroll
        for (int o = 0; o < W; ++o) h[o] = b1[o];
        for (int i = 0; i < g.n_in; ++i) {
            const float xi = s_x[i * kThreads + k];
            const float4* wrow = reinterpret_cast<const float4*>(W1t + i * W);
#pragma unroll
            for (int o4 = 0; o4 < W / 4; ++o4) {
                const float4 w4 = wrow[o4];
                if (NIV_FP32_PACKED) {
                    const float2 x2 = make_float2(xi, xi);
                    const float2 lo = __ffma2_rn(make_float2(w4.x, w4.y), x2, make_float2(h[4 * o4 + 0], h[4 * o4 + 1]));
                    const float2 hi = __ffma2_rn(make_float2(w4.z, w4.w), x2, make_float2(h[4 * o4 + 2], h[4 * o4 + 3]));
                    h[4 * o4 + 0] = lo.x;
                    h[4 * o4 + 1] = lo.y;
                    h[4 * o4 + 2] = hi.x;
                    h[4 * o4 + 3] = hi.y;
                } else {
                    h[4 * o4 + 0] = fmaf(w4.x, xi, h[4 * o4 + 0]);
                    h[4 * o4 + 1] = fmaf(w4.y, xi, h[4 * o4 + 1]);
                    h[4 * o4 + 2] = fmaf(w4.z, xi, h[4 * o4 + 2]);
                    h[4 * o4 + 3] = fmaf(w4.w, xi, h[4 * o4 + 3]);
                }
            }
        }
#pragma unroll
        for (int o = 0; o < W; ++o) h[o] = fmaxf(h[o], 0.0f);
        const float* wp = b1 + W;

        // ---- middle hidden layers: h -> shared column -> h ----
        for (int layer = 1; layer < n_hidden - 1; ++layer) {
            const float* Wl = wp;  // [W][W] row-major
            const float* bl = wp + W * W;
            for (int o = 0; o < W; ++o) s_x[o * kThreads + k] = fmaxf(dot_row<W>(Wl + o * W, h, bl[o]), 0.0f);
#pragma unroll
            for (int q = 0; q < W; ++q) h[q] = s_x[q * kThreads + k];
            wp += W * W + W;
        }

        // ---- last hidden layer streamed into the 3-wide output layer ----
        float z0, z1, z2;
        if (n_hidden >= 2) {
            const float* Wl = wp;
            const float* bl = wp + W * W;
            const float* Wo = bl + W;  // [3][W]
            const float* bo = Wo + 3 * W;
            z0 = bo[0];
            z1 = bo[1];
            z2 = bo[2];
            for (int o = 0; o < W; ++o) {
                const float a = fmaxf(dot_row<W>(Wl + o * W, h, bl[o]), 0.0f);
                z0 = fmaf(Wo[o], a, z0);
                z1 = fmaf(Wo[W + o], a, z1);
                z2 = fmaf(Wo[2 * W + o], a, z2);
            }
        } else {
            const float* Wo = wp;
            const float* bo = Wo + 3 * W;
            z0 = bo[0];
            z1 = bo[1];
            z2 = bo[2];
#pragma unroll
            for (int q = 0; q < W; ++q) {
                z0 = fmaf(Wo[q], h[q], z0);
                z1 = fmaf(Wo[W + q], h[q], z1);
                z2 = fmaf(Wo[2 * W + q], h[q], z2);
            }
        }
        if (out_act == 1) {
            z0 = niv_softplus(z0);
            z1 = niv_softplus(z1);
            z2 = niv_softplus(z2);
        }
        if (valid) niv_store_result(io, r, z0, z1, z2);
    }
}

template <int DIMS, int F, int W>
int launch(const niv_model* m, const GridArgs& g, const IoArgs& io, cudaStream_t s) {
    auto kern = query_fp32_kernel<DIMS, F, W>;
    const int stride = (int)((m->mlp_plain_len + 3) & ~3LL);
    const int rows = g.n_in > W ? g.n_in : W;
    const size_t smem = (size_t)(stride + rows * kThreads) * sizeof(float);
    NIV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    NIV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared));
    int dev = 0, sms = 0, per_sm = 0;
    NIV_CUDA(cudaGetDevice(&dev));
    NIV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    NIV_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, smem));
    if (per_sm < 1) return niv_fail(NIV_ERR_UNSUPPORTED, "plain query kernel does not fit on an SM");
    const int64_t tiles = niv_tile_count_host(io.n, io.image_width);
    const int64_t grid_blocks = tiles < (int64_t)sms * per_sm ? tiles : (int64_t)sms * per_sm;
    kern<<<(unsigned)grid_blocks, kThreads, smem, s>>>(g, io, m->params, m->mlp_plain, (int)m->mlp_plain_len, stride,
                                                      m->d.n_hidden, m->d.out_act, tiles);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}

template <int DIMS, int F>
int by_width(const niv_model* m, const GridArgs& g, const IoArgs& io, cudaStream_t s) {
    switch (m->d.width) {
        case 16: return launch<DIMS, F, 16>(m, g, io, s);
        case 32: return launch<DIMS, F, 32>(m, g, io, s);
        case 64: return launch<DIMS, F, 64>(m, g, io, s);
    }
    return niv_fail(NIV_ERR_UNSUPPORTED, "width must be 16, 32 or 64");
}

template <int DIMS>
int by_feat(const niv_model* m, const GridArgs& g, const IoArgs& io, cudaStream_t s) {
    switch (m->d.feat) {
        case 1: return by_width<DIMS, 1>(m, g, io, s);
        case 2: return by_width<DIMS, 2>(m, g, io, s);
        case 4: return by_width<DIMS, 4>(m, g, io, s);
    }
    return niv_fail(NIV_ERR_UNSUPPORTED, "feat must be 1, 2 or 4");
}

}  // namespace

int niv_launch_query_fp32(const niv_model* m, const GridArgs& g, const IoArgs& io, cudaStream_t s) {
    return m->d.dims == 4 ? by_feat<4>(m, g, io, s) : by_feat<3>(m, g, io, s);
}
