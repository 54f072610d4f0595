// Encoding only (Sec. 4.1): per query the L*F interpolated features, then the
// 6 * pe_bands frequency-encoding values of a model without grid, and on request
// the 2^d corner entry indices of every level.  Used to check the integer index
// pipeline bit for bit and the FP32 interpolation on its own.
#include "niv_internal.cuh"

namespace {

template <int DIMS, int F>
__global__ void __launch_bounds__(128) encode_kernel(GridArgs g, IoArgs io, const float* __restrict__ grid,
                                                     float* __restrict__ enc, uint32_t* __restrict__ idx) {
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= io.n) return;
    const float4 p = niv_load_rec(io.pos, q, io.in_f16);
    float u[4];
    u[0] = niv_unit(p.x, g.aabb_min[0], g.inv_ext[0]);
    u[1] = niv_unit(p.y, g.aabb_min[1], g.inv_ext[1]);
    u[2] = niv_unit(p.z, g.aabb_min[2], g.inv_ext[2]);
    u[3] = fminf(fmaxf(g.t, 0.0f), 1.0f);
    constexpr int NC = 1 << DIMS;
    const int LG = g.levels * F, ne = LG + 6 * g.pe_bands;
    for (int d = 0; d < 3 && g.pe_bands > 0 && enc; ++d)
        for (int b = 0; b < g.pe_bands; ++b) {
            float sv, cv;
            niv_pe_pair(u[d], b, sv, cv);
            enc[q * ne + LG + 2 * (d * g.pe_bands + b)] = sv;
            enc[q * ne + LG + 2 * (d * g.pe_bands + b) + 1] = cv;
        }
    // the corner entries and weights of every level come from the helper the query and training
    // kernels use, so that the index output checks their integer pipeline itself
    for (int l = 0; l < g.levels; ++l) {
        uint32_t e[NC];
        float wc[NC];
        niv_level_corners<DIMS>(g, l, u, e, wc);
        const float* tab = grid + (size_t)g.offset[l] * F;
        float acc[F];
#pragma unroll
        for (int j = 0; j < F; ++j) acc[j] = 0.0f;
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            if (idx) idx[(q * g.levels + l) * NC + c] = e[c];
#pragma unroll
            for (int j = 0; j < F; ++j) acc[j] = fmaf(wc[c], __ldg(tab + (size_t)e[c] * F + j), acc[j]);
        }
        if (enc)
#pragma unroll
            for (int j = 0; j < F; ++j) enc[q * ne + l * F + j] = acc[j];
    }
}

template <int DIMS>
int launch(const niv_model* m, const GridArgs& g, const IoArgs& io, float* enc, uint32_t* idx, cudaStream_t s) {
    const unsigned blocks = (unsigned)((io.n + 127) / 128);
    switch (m->d.feat) {
        case 1: encode_kernel<DIMS, 1><<<blocks, 128, 0, s>>>(g, io, m->params, enc, idx); break;
        case 2: encode_kernel<DIMS, 2><<<blocks, 128, 0, s>>>(g, io, m->params, enc, idx); break;
        case 4: encode_kernel<DIMS, 4><<<blocks, 128, 0, s>>>(g, io, m->params, enc, idx); break;
        default: return niv_fail(NIV_ERR_UNSUPPORTED, "feat must be 1, 2 or 4");
    }
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}

}  // namespace

int niv_launch_encode(const niv_model* m, const GridArgs& g, const IoArgs& io, float* enc, uint32_t* idx,
                      cudaStream_t s) {
    return m->d.dims == 4 ? launch<4>(m, g, io, enc, idx, s) : launch<3>(m, g, io, enc, idx, s);
}
