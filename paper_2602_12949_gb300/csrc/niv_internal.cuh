// Internal declarations of libniv: the model object and the host-side interfaces of the
// translation units; the kernel argument blocks and device helpers live in encoding.cuh.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <stdio.h>
#include <stdlib.h>

#include <string>
#include <type_traits>

#include "niv.h"
#include "encoding.cuh"

// Most chunks niv_query_host splits a call into.
#define NIV_HOST_CHUNKS_MAX 32

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
    uint2* grid_pair16;      // dense levels (a prefix of the levels, two features): entry e holds the
                             // FP16 words of entries e and e + 1 (nullptr for other models)
    int64_t n_pair;          // entries of grid_pair16
    float* mlp_plain;        // network packed for the plain FP32 kernel
    int64_t mlp_plain_len;
    uint8_t* mlp_tc;         // network packed for the tensor-core kernels (FP16 tiles)
    uint32_t mlp_tc_bytes;
    alignas(8) uint8_t tc_layout[64];  // offsets inside mlp_tc (query_tc.cu)
    uint8_t* mlp_f8;         // network packed for the E4M3 kernel (query_f8.cu)
    uint32_t mlp_f8_bytes;
    alignas(8) uint8_t f8_layout[64];
    float fp8_sact[8], fp8_sw[8], fp8_amax_host[8];  // per matrix product: activation / weight scales
    unsigned* fp8_amax;      // calibration scratch (device)
    int fp8_ready;           // calibrated since the last parameter change
    // Training state (allocated on the first training call).
    float* grad;             // dLoss/dparams, same layout as params
    float* adam_m;
    float* adam_v;
    int64_t adam_step;
    float* stash;            // per-step activation / gradient scratch
    int64_t stash_floats;
    double* loss_acc;        // device loss accumulator
    int infer_dirty;         // parameters changed on the device since the inference copies were built
    int train_f16;           // training forward: FP16 path of the query (else FP32)
    // Host staging for niv_query_host.
    void* stage;
    size_t stage_bytes;
    // Copy streams (host->device, device->host), per-chunk events (inputs landed, outputs
    // written) and join events of the pipelined niv_query_host, created on first use.
    cudaStream_t host_copy[2];
    cudaEvent_t host_ev[2][NIV_HOST_CHUNKS_MAX];
    cudaEvent_t host_join[2];
    int host_pipe;
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

// Rebuild the FP16 grid and the packed networks from the FP32 master parameters (after
// training steps).  Allocates device memory only when no network was packed before.
int niv_refresh_inference(niv_model* m, cudaStream_t s);

// Integer value of an environment variable (tuning and diagnostics), or dflt.
int niv_env_int(const char* name, int dflt);

// ---- kernel launchers (one per translation unit) ----
int niv_launch_query_fp32(const niv_model* m, const GridArgs& g, const IoArgs& io, cudaStream_t s);
int niv_launch_encode(const niv_model* m, const GridArgs& g, const IoArgs& io, float* enc, uint32_t* idx,
                      cudaStream_t s);
int niv_pack_f8(niv_model* m, const float* mlp_host, cudaStream_t s);
int niv_calibrate_f8(niv_model* m, const GridArgs& g, const IoArgs& io, cudaStream_t s);
int niv_launch_query_f8(const niv_model* m, const GridArgs& g, const IoArgs& io, cudaStream_t s);
int64_t niv_train_stash_floats(const niv_model* m, int64_t n);
// vjp: target holds dL/dE per sample (vector-Jacobian product) instead of the Eq. 3 targets.
int niv_train_grad(niv_model* m, const GridArgs& g, const float4* pos, const float4* nrm, const float* t,
                   const float4* target, int64_t n, float eps, bool vjp, cudaStream_t s);
int niv_train_adam(niv_model* m, float lr, float b1, float b2, float eps, cudaStream_t s);
int niv_launch_mc(const float* blob, int64_t blob_len, const float* x4, const float* n4, const float* t, int64_t m,
                  int spp, uint64_t seed, uint64_t index_base, int mode, double* outE, uint8_t* keep, cudaStream_t s);
int niv_launch_probe_bake(const float* blob, int64_t blob_len, const int* P, const float* lo, const float* hi, int rays,
                          uint64_t seed, uint64_t index_base, double* out64, __half* out16, cudaStream_t s);
// scene (host, nullable): "+RT" visibility rays against it at scene parameter t.
int niv_launch_probe_query(const void* coef16, const int* P, const float* lo, const float* hi, const IoArgs& io,
                           const float* scene, int64_t scene_len, float t, cudaStream_t s);
int niv_launch_compact(const float* x4, const float* n4, const float* t, const double* E, const uint8_t* keep, int64_t m,
                       float* ox4, float* on4, float* ot, float* otarget, int64_t* count_dev, int* scratch,
                       cudaStream_t s);
int niv_launch_shade(const void* albedo, const void* direct, const void* E, int64_t n, void* out, cudaStream_t s);
int niv_launch_upsample_shade(const void* pos, const void* nrm, const void* albedo, const void* direct, int32_t width,
                              int32_t height, int32_t in_f16, const void* E_low, int32_t e_f16, int32_t sub, float power,
                              float sigma, float eps, void* out, cudaStream_t s);
int niv_pack_plain(niv_model* m, const float* mlp_host, cudaStream_t s);
struct niv_dyn;
int niv_dyn_build(const float* tri9, int64_t n_tris, niv_dyn** out);
void niv_dyn_free(niv_dyn* d);
int64_t niv_dyn_node_count(const niv_dyn* d);
int niv_launch_ao(const niv_dyn* d, const void* pos, const void* nrm, int64_t n, int32_t in_f16, int32_t rays,
                  float radius, uint64_t seed, float* ao, void* E, int32_t e_f16, cudaStream_t s);
int niv_pack_tc(niv_model* m, const float* mlp_host, cudaStream_t s);
// status: device word for kernel-side failures (nullptr = this device's library status word).
int niv_launch_query_tc(const niv_model* m, const GridArgs& g, const IoArgs& io, int precision, cudaStream_t s,
                        int* status = nullptr);
