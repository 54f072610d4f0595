// Internal declarations of libniv: the model object, kernel argument blocks and
// the encoding helpers every query kernel shares.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "niv.h"

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
    float aabb_min[3];
    float inv_ext[3];
    float t;
    int32_t res[NIV_MAX_LEVELS];
    uint32_t offset[NIV_MAX_LEVELS];  // first entry of each level
};

// Where a kernel finds its records and how it walks them.
struct IoArgs {
    const void* pos;
    const void* nrm;
    void* out;
    int64_t n;
    int32_t image_width;  // > 0: 2-D tile traversal of a row-major image
    int32_t in_f16;       // records are FP16 (else FP32)
    int32_t out_f16;
};

struct niv_model {
    niv_model_desc d;
    int device;
    int32_t res[NIV_MAX_LEVELS];
    int32_t dense[NIV_MAX_LEVELS];
    int64_t offset[NIV_MAX_LEVELS];
    int64_t entries[NIV_MAX_LEVELS];
    int64_t total_entries;
    int n_in;
    int64_t n_grid, n_mlp;  // parameter counts
    // FP32 master parameters [grid | network], owned.
    float* params;
    // Inference copies rebuilt by niv_set_params.
    __half* grid_f16;        // grid values in FP16
    float* mlp_plain;        // network packed for the plain FP32 kernel
    int64_t mlp_plain_len;
    uint8_t* mlp_tc;         // network packed for the tensor-core kernels (FP16 tiles)
    uint32_t mlp_tc_bytes;
    alignas(8) uint8_t tc_layout[64];  // offsets inside mlp_tc (query_tc.cu)
    // Host staging for niv_query_host.
    void* stage;
    size_t stage_bytes;
};

// ---- error reporting (thread-local message) ----
int niv_fail(int code, const std::string& msg);
int niv_cuda_fail(cudaError_t e, const char* what);
#define NIV_CUDA(call)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return niv_cuda_fail(e_, #call); \
    } while (0)

// Device status word of the current device (allocated on first use; kernels whose
// bounded waits expire write a nonzero code into it).  nullptr on failure.
int* niv_status_word();

GridArgs niv_grid_args(const niv_model* m, const niv_query_params* p);

// ---- kernel launchers (one per translation unit) ----
int niv_launch_query_fp32(const niv_model* m, const GridArgs& g, const IoArgs& io, cudaStream_t s);
int niv_launch_encode(const niv_model* m, const GridArgs& g, const IoArgs& io, float* enc, uint32_t* idx,
                      cudaStream_t s);
int niv_launch_shade(const void* albedo, const void* direct, const void* E, int64_t n, void* out, cudaStream_t s);
int niv_pack_plain(niv_model* m, const float* mlp_host, cudaStream_t s);
int niv_pack_tc(niv_model* m, const float* mlp_host, cudaStream_t s);
int niv_launch_query_tc(const niv_model* m, const GridArgs& g, const IoArgs& io, int precision, cudaStream_t s);

// ---- device helpers shared by the query kernels ----

// u = clamp(fp32(fp32(p - lo) * inv), 0, 1): FP32 operations without contraction.
__device__ __forceinline__ float niv_unit(float p, float lo, float inv) {
    float x = __fmul_rn(__fsub_rn(p, lo), inv);
    return fminf(fmaxf(x, 0.0f), 1.0f);
}

// Cell of one coordinate at resolution N: s = fp32(u * N), i = min(floor(s), N - 1), w = s - i (exact).
__device__ __forceinline__ void niv_cell(float u, int32_t N, uint32_t& i, float& w) {
    float s = __fmul_rn(u, (float)N);
    int ii = min((int)floorf(s), N - 1);
    i = (uint32_t)ii;
    w = __fsub_rn(s, (float)ii);
}

// Entry index of vertex v at a level: dense row-major (x fastest) or spatial hash.
template <int DIMS>
__device__ __forceinline__ uint32_t niv_vertex_index(bool dense, uint32_t stride, const uint32_t* v,
                                                     uint32_t mask, uint32_t prime_t) {
    if (dense) {
        uint32_t idx = v[DIMS - 1];
#pragma unroll
        for (int k = DIMS - 2; k >= 0; --k) idx = idx * stride + v[k];
        return idx;
    }
    uint32_t h = v[0] * NIV_PI1 ^ v[1] * NIV_PI2 ^ v[2] * NIV_PI3;
    if (DIMS == 4) h ^= v[3] * prime_t;
    return h & mask;
}

// Linear record index of thread slot `k` of tile `tile` (128-record tiles; 16 x 8 pixels for images).
__device__ __forceinline__ int64_t niv_record_of(int64_t tile, int k, int64_t n, int32_t width) {
    if (width <= 0) return tile * 128 + k;
    int64_t tiles_x = (width + 15) / 16;
    int64_t ty = tile / tiles_x, tx = tile - ty * tiles_x;
    int64_t px = tx * 16 + (k & 15), py = ty * 8 + (k >> 4);
    if (px >= width) return n;  // outside the image: no record
    return py * width + px;
}

__device__ __forceinline__ int64_t niv_tile_count(int64_t n, int32_t width) {
    if (width <= 0) return (n + 127) / 128;
    int64_t rows = (n + width - 1) / width;
    return ((width + 15) / 16) * ((rows + 7) / 8);
}

__host__ __forceinline__ int64_t niv_tile_count_host(int64_t n, int32_t width) {
    if (width <= 0) return (n + 127) / 128;
    int64_t rows = (n + width - 1) / width;
    return ((width + 15) / 16) * ((rows + 7) / 8);
}

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

// softplus(z) = max(z, 0) + log1p(exp(-|z|)) in FP32 with CUDA's libm functions.
__device__ __forceinline__ float niv_softplus(float z) { return fmaxf(z, 0.0f) + log1pf(expf(-fabsf(z))); }
