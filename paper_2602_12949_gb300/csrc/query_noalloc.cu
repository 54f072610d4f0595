// Host-buffer query that performs no device allocation.
//
// niv_query_host stages the caller's host records in a device buffer that the
// library allocates (and grows) on demand.  Some callers cannot let a library
// allocate device memory: a real-time render loop that fixes its GPU memory
// budget at start-up and forbids allocation while frames are in flight, or a
// plug-in whose host application owns every device allocation.  For them this
// file keeps the staging area in a fixed, file-scope device array instead.
//
// The array (NIV_NOALLOC_MAX_RECORDS records of at most 16 bytes for each of
// positions, normals and results, plus a status word: about 3 MiB) exists on
// every GPU that loads the library, from module load until process exit.
// All calls share it, so calls whose work overlaps on the GPU race with each
// other; callers must serialise them.
#include <mutex>

#include "niv_internal.cuh"

namespace {

constexpr size_t kRecBytesMax = 16;                                  // an FP32 [4] record
constexpr size_t kArea = (size_t)NIV_NOALLOC_MAX_RECORDS * kRecBytesMax;  // one record array
constexpr size_t kStatusBytes = 256;                                 // status word, padded

// [status word | positions | normals | results]; it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kStatusBytes + 3 * kArea];

std::mutex g_mu;
unsigned char* g_scratch_dev[64] = {nullptr};  // device address of the array, per device ordinal

// The array's device address on the current device.  In host code the symbol itself is
// only a host-side stand-in, so the address is looked up once per device (with that
// device current) and cached.
int scratch_address(unsigned char** out) {
    int dev = -1;
    NIV_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return niv_fail(NIV_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_dev[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return niv_cuda_fail(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_scratch_dev[dev] = static_cast<unsigned char*>(p);
    }
    *out = g_scratch_dev[dev];
    return NIV_OK;
}

}  // namespace

extern "C" int niv_query_host_noalloc(niv_handle h, const void* pos, const void* nrm, int64_t n, int32_t dtype_in,
                                      const niv_query_params* params, void* out_E, int32_t dtype_out,
                                      int32_t precision, niv_stream stream) {
    if (!h || !params) return niv_fail(NIV_ERR_ARG, "handle or params is NULL");
    if (n < 0) return niv_fail(NIV_ERR_ARG, "n < 0");
    if (n == 0) return NIV_OK;
    if (n > NIV_NOALLOC_MAX_RECORDS)
        return niv_fail(NIV_ERR_ARG, "n exceeds NIV_NOALLOC_MAX_RECORDS (65536), the size of the fixed staging area");
    if (!pos || !nrm || !out_E) return niv_fail(NIV_ERR_ARG, "NULL record pointer");
    if ((dtype_in != NIV_F32 && dtype_in != NIV_F16) || (dtype_out != NIV_F32 && dtype_out != NIV_F16))
        return niv_fail(NIV_ERR_ARG, "record dtype must be NIV_F32 or NIV_F16");
    if (precision != NIV_FP32 && precision != NIV_FP16)
        return niv_fail(NIV_ERR_UNSUPPORTED, "precision not supported by the allocation-free path");
    for (int k = 0; k < 3; ++k)
        if (!(params->aabb_max[k] > params->aabb_min[k])) return niv_fail(NIV_ERR_ARG, "empty aabb");
    if (params->image_width < 0) return niv_fail(NIV_ERR_ARG, "image_width < 0");
    int dev = -1;
    NIV_CUDA(cudaGetDevice(&dev));
    if (dev != h->device) return niv_fail(NIV_ERR_ARG, "current device differs from the model's device");

    // The inference copies must exist already (refreshing them then allocates nothing): a
    // model straight from niv_create has no packed network.
    if (!h->mlp_tc) return niv_fail(NIV_ERR_ARG, "parameters not set: call niv_set_params or niv_load first");
    cudaStream_t s = (cudaStream_t)stream;
    int rc = 0;
    if (h->infer_dirty) {  // trained since the inference copies were built
        rc = niv_refresh_inference(h, s);
        if (rc) return rc;
    }

    unsigned char* base = nullptr;
    rc = scratch_address(&base);
    if (rc) return rc;
    int* status = reinterpret_cast<int*>(base);
    unsigned char* d_pos = base + kStatusBytes;
    unsigned char* d_nrm = d_pos + kArea;
    unsigned char* d_out = d_nrm + kArea;
    const size_t in_b = (size_t)n * (dtype_in == NIV_F16 ? 8 : 16);
    const size_t out_b = (size_t)n * (dtype_out == NIV_F16 ? 8 : 16);

    NIV_CUDA(cudaMemsetAsync(status, 0, sizeof(int), s));  // the array keeps the last call's status
    NIV_CUDA(cudaMemcpyAsync(d_pos, pos, in_b, cudaMemcpyHostToDevice, s));
    NIV_CUDA(cudaMemcpyAsync(d_nrm, nrm, in_b, cudaMemcpyHostToDevice, s));
    const GridArgs g = niv_grid_args(h, params);
    IoArgs io;
    io.pos = d_pos;
    io.nrm = d_nrm;
    io.out = d_out;
    io.n = n;
    io.image_width = params->image_width;
    io.in_f16 = dtype_in == NIV_F16;
    io.out_f16 = dtype_out == NIV_F16;
    rc = precision == NIV_FP32 ? niv_launch_query_fp32(h, g, io, s) : niv_launch_query_tc(h, g, io, precision, s, status);
    if (rc) {
        cudaStreamSynchronize(s);  // the queued copies may still read the caller's buffers
        return rc;
    }
    NIV_CUDA(cudaMemcpyAsync(out_E, d_out, out_b, cudaMemcpyDeviceToHost, s));
    int st = 0;
    NIV_CUDA(cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s));
    NIV_CUDA(cudaStreamSynchronize(s));
    if (st != 0) return niv_fail(NIV_ERR_DEVICE, "the query kernel reported a failure (MMA wait ran out)");
    return NIV_OK;
}
