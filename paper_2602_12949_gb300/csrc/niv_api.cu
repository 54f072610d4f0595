// Host side of the C ABI: model objects, parameter management, argument checks
// and dispatch of the query / shading kernels.
#include <math.h>

#include <cmath>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <string>
#include <vector>

#include "niv_internal.cuh"

namespace {

thread_local std::string t_err;

bool aligned16(const void* p) { return ((uintptr_t)p & 15u) == 0; }

// Device status words, one per device ordinal, allocated on first use.
std::mutex g_status_mu;
int* g_status[64] = {nullptr};

// Scratch of the sample compaction (block offsets + count), per device ordinal, grown on demand.
std::mutex g_compact_mu;
void* g_compact[64] = {nullptr};
size_t g_compact_bytes[64] = {0};

__global__ void f32_to_f16_kernel(const float* __restrict__ src, __half* __restrict__ dst, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = __float2half_rn(src[i]);
}

// Pair table of the dense levels: entry e = (word e, word e + 1) of the FP16 grid (two features
// per word); the last entry's second word is 0.
__global__ void pair_table_kernel(const uint32_t* __restrict__ words, uint2* __restrict__ pair, int64_t n) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        pair[i] = make_uint2(words[i], i + 1 < n ? words[i + 1] : 0u);
}

int validate_desc(const niv_model_desc* d) {
    if (!d) return niv_fail(NIV_ERR_ARG, "desc is NULL");
    if (d->dims != 3 && d->dims != 4) return niv_fail(NIV_ERR_ARG, "dims must be 3 or 4");
    if (d->pe_bands < 0 || d->pe_bands > 16) return niv_fail(NIV_ERR_ARG, "pe_bands must be in 0..16");
    if (d->pe_bands > 0) {
        if (d->levels != 0) return niv_fail(NIV_ERR_UNSUPPORTED, "a frequency-encoded model has no grid levels");
        if (d->dims != 3) return niv_fail(NIV_ERR_UNSUPPORTED, "frequency encoding is 3-D");
    } else if (d->levels < 1 || d->levels > NIV_MAX_LEVELS) {
        return niv_fail(NIV_ERR_ARG, "levels must be in 1..32");
    }
    if (d->feat != 1 && d->feat != 2 && d->feat != 4) return niv_fail(NIV_ERR_UNSUPPORTED, "feat must be 1, 2 or 4");
    if (d->log2_T < 4 || d->log2_T > 24) return niv_fail(NIV_ERR_ARG, "log2_T must be in 4..24");
    if (!(d->base >= 1.0) || !(d->growth >= 1.0)) return niv_fail(NIV_ERR_ARG, "base and growth must be >= 1");
    if (d->n_hidden < 1 || d->n_hidden > 4) return niv_fail(NIV_ERR_UNSUPPORTED, "n_hidden must be in 1..4");
    if (d->width != 16 && d->width != 32 && d->width != 64)
        return niv_fail(NIV_ERR_UNSUPPORTED, "width must be 16, 32 or 64");
    if (d->in_extra != 3 && d->in_extra != 4) return niv_fail(NIV_ERR_ARG, "in_extra must be 3 or 4");
    if (d->t_bands < 0 || d->t_bands > 6) return niv_fail(NIV_ERR_ARG, "t_bands must be in 0..6");
    if (d->t_bands > 0 && (d->dims != 3 || d->in_extra != 3))
        return niv_fail(NIV_ERR_ARG, "a frequency-encoded scene parameter needs dims = 3 and in_extra = 3");
    if (d->out_dim != 3) return niv_fail(NIV_ERR_UNSUPPORTED, "out_dim must be 3");
    if (d->out_act != 0 && d->out_act != 1) return niv_fail(NIV_ERR_ARG, "out_act must be 0 or 1");
    if (d->levels * d->feat + 6 * d->pe_bands + d->in_extra + 2 * d->t_bands > NIV_MAX_IN)
        return niv_fail(NIV_ERR_UNSUPPORTED, "network input too wide");
    if (d->dims == 4 && (d->prime_t & 1u) == 0) return niv_fail(NIV_ERR_ARG, "prime_t must be odd");
    return NIV_OK;
}

int check_device(const niv_model* m) {
    int dev = -1;
    NIV_CUDA(cudaGetDevice(&dev));
    if (dev != m->device) return niv_fail(NIV_ERR_ARG, "current device differs from the model's device");
    return NIV_OK;
}

int convert_grid_f16(niv_model* m, cudaStream_t s) {
    int64_t n = m->n_grid;
    if (n == 0) return NIV_OK;  // frequency-encoded model: no grid
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    f32_to_f16_kernel<<<(unsigned)blocks, 256, 0, s>>>(m->params, m->grid_f16, n);
    NIV_CUDA(cudaGetLastError());
    if (m->grid_pair16) {
        int64_t pb = (m->n_pair + 255) / 256;
        if (pb > 4096) pb = 4096;
        pair_table_kernel<<<(unsigned)pb, 256, 0, s>>>(reinterpret_cast<const uint32_t*>(m->grid_f16), m->grid_pair16,
                                                      m->n_pair);
        NIV_CUDA(cudaGetLastError());
    }
    return NIV_OK;
}

void free_model(niv_model* m) {
    if (!m) return;
    cudaFree(m->params);
    cudaFree(m->grid_f16);
    cudaFree(m->grid_pair16);
    cudaFree(m->mlp_plain);
    cudaFree(m->mlp_tc);
    cudaFree(m->mlp_f8);
    cudaFree(m->fp8_amax);
    cudaFree(m->grad);
    cudaFree(m->adam_m);
    cudaFree(m->adam_v);
    cudaFree(m->stash);
    cudaFree(m->loss_acc);
    cudaFree(m->stage);
    if (m->host_pipe) {
        for (int i = 0; i < 2; ++i) {
            cudaStreamDestroy(m->host_copy[i]);
            cudaEventDestroy(m->host_join[i]);
            for (int c = 0; c < NIV_HOST_CHUNKS_MAX; ++c) cudaEventDestroy(m->host_ev[i][c]);
        }
    }
    delete m;
}

// Rebuild the FP16 grid and the packed networks from the master parameters on the device.
int refresh_inference(niv_model* h, cudaStream_t s) {
    int rc = convert_grid_f16(h, s);
    if (rc) return rc;
    std::vector<float> mlp_host((size_t)h->n_mlp);
    NIV_CUDA(cudaMemcpyAsync(mlp_host.data(), h->params + h->n_grid, sizeof(float) * h->n_mlp, cudaMemcpyDeviceToHost, s));
    NIV_CUDA(cudaStreamSynchronize(s));
    rc = niv_pack_plain(h, mlp_host.data(), s);
    if (rc) return rc;
    rc = niv_pack_tc(h, mlp_host.data(), s);
    if (rc) return rc;
    h->fp8_ready = 0;  // the E4M3 network must be recalibrated for new parameters
    h->infer_dirty = 0;
    return NIV_OK;
}

int ensure_training_state(niv_model* h) {
    const int64_t n = h->n_grid + h->n_mlp;
    if (!h->grad) NIV_CUDA(cudaMalloc(&h->grad, sizeof(float) * n));
    if (!h->adam_m) {
        NIV_CUDA(cudaMalloc(&h->adam_m, sizeof(float) * n));
        NIV_CUDA(cudaMemset(h->adam_m, 0, sizeof(float) * n));
    }
    if (!h->adam_v) {
        NIV_CUDA(cudaMalloc(&h->adam_v, sizeof(float) * n));
        NIV_CUDA(cudaMemset(h->adam_v, 0, sizeof(float) * n));
    }
    if (!h->loss_acc) NIV_CUDA(cudaMalloc(&h->loss_acc, sizeof(double)));
    return NIV_OK;
}

}  // namespace

int niv_refresh_inference(niv_model* m, cudaStream_t s) { return refresh_inference(m, s); }

int niv_env_int(const char* name, int dflt) {
    const char* v = getenv(name);
    return (v && *v) ? atoi(v) : dflt;
}

int niv_fail(int code, const std::string& msg) {
    t_err = msg;
    return code;
}

int niv_cuda_fail(cudaError_t e, const char* what) {
    t_err = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? NIV_ERR_NOMEM : NIV_ERR_CUDA;
}

int* niv_status_word() {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lk(g_status_mu);
    if (!g_status[dev]) {
        int* p = nullptr;
        if (cudaMalloc(&p, sizeof(int)) != cudaSuccess) return nullptr;
        if (cudaMemset(p, 0, sizeof(int)) != cudaSuccess) return nullptr;
        g_status[dev] = p;
    }
    return g_status[dev];
}

GridArgs niv_grid_args(const niv_model* m, const niv_query_params* p) {
    GridArgs g;
    memset(&g, 0, sizeof g);
    g.dims = m->d.dims;
    g.levels = m->d.levels;
    g.pe_bands = m->d.pe_bands;
    g.t_bands = m->d.t_bands;
    g.feat = m->d.feat;
    g.n_in = m->n_in;
    g.hash_mask = (uint32_t)((1ull << m->d.log2_T) - 1ull);
    g.prime_t = m->d.prime_t;
    for (int l = 0; l < m->d.levels; ++l) {
        g.res[l] = m->res[l];
        g.offset[l] = (uint32_t)m->offset[l];
        g.res_f[l] = (float)m->res[l];
        g.resm1_f[l] = (float)(m->res[l] - 1);
        g.stride1[l] = (uint32_t)m->res[l] + 1u;
        g.stride2[l] = g.stride1[l] * g.stride1[l];
        g.resm1_b[l] = (float)(8388608.0 + (double)(m->res[l] - 1));  // exact: N <= 2^20
        uint32_t span = 1u + g.stride1[l] + g.stride2[l];
        if (m->d.dims == 4) span += g.stride2[l] * g.stride1[l];
        g.dense_off[l] = 0u - kNivBias * span;
        if (m->dense[l]) g.dense_mask |= 1u << l;
    }
    g.prime_t_off = 0u - kNivBias * g.prime_t;
    for (int k = 0; k < 3; ++k) {
        g.aabb_min[k] = p->aabb_min[k];
        g.inv_ext[k] = (float)(1.0 / ((double)p->aabb_max[k] - (double)p->aabb_min[k]));
    }
    g.t = p->t;
    return g;
}

// Network packed for the plain kernel: [W1^T (n_in x W) | b1 | (W_l row-major | b_l) ... | W_out | b_out].
int niv_pack_plain(niv_model* m, const float* src, cudaStream_t s) {
    const int W = m->d.width, n_in = m->n_in;
    std::vector<float> dst((size_t)m->mlp_plain_len);
    size_t o = 0, i = 0;
    for (int r = 0; r < n_in; ++r)
        for (int c = 0; c < W; ++c) dst[o + (size_t)r * W + c] = src[i + (size_t)c * n_in + r];
    o += (size_t)n_in * W;
    i += (size_t)n_in * W;
    for (int c = 0; c < W; ++c) dst[o++] = src[i++];
    const size_t rest = (size_t)m->n_mlp - i;
    memcpy(dst.data() + o, src + i, rest * sizeof(float));
    NIV_CUDA(cudaMemcpyAsync(m->mlp_plain, dst.data(), sizeof(float) * dst.size(), cudaMemcpyHostToDevice, s));
    NIV_CUDA(cudaStreamSynchronize(s));
    return NIV_OK;
}

extern "C" {

const char* niv_version(void) { return "niv 0.2 (sm_103a)"; }

const char* niv_last_error(void) { return t_err.c_str(); }

int niv_sync_status(niv_stream stream) {
    NIV_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    int* w = niv_status_word();
    if (!w) return niv_fail(NIV_ERR_CUDA, "status word unavailable");
    int v = 0;
    NIV_CUDA(cudaMemcpy(&v, w, sizeof(int), cudaMemcpyDeviceToHost));
    if (v != 0) {
        NIV_CUDA(cudaMemset(w, 0, sizeof(int)));
        char buf[96];
        snprintf(buf, sizeof buf, "a kernel reported failure code %d", v);
        return niv_fail(NIV_ERR_DEVICE, buf);
    }
    return NIV_OK;
}

int niv_create(const niv_model_desc* desc, niv_handle* out) {
    if (!out) return niv_fail(NIV_ERR_ARG, "out is NULL");
    *out = nullptr;
    int rc = validate_desc(desc);
    if (rc) return rc;
    niv_model* m = new niv_model();
    memset((void*)m, 0, sizeof(niv_model));
    m->d = *desc;
    const int64_t T = 1ll << desc->log2_T;
    int64_t off = 0;
    for (int l = 0; l < desc->levels; ++l) {
        const double Nd = floor(desc->base * pow(desc->growth, (double)l));
        if (Nd > (double)(1 << 20)) {
            free_model(m);
            return niv_fail(NIV_ERR_UNSUPPORTED, "level resolution above 2^20");
        }
        const int32_t N = (int32_t)Nd;
        int64_t verts = 1;
        for (int k = 0; k < desc->dims && verts <= T; ++k) verts *= (int64_t)(N + 1);
        m->res[l] = N;
        m->dense[l] = verts <= T;
        m->offset[l] = off;
        m->entries[l] = m->dense[l] ? verts : T;
        off += m->entries[l];
    }
    m->total_entries = off;
    m->n_in = desc->levels * desc->feat + 6 * desc->pe_bands + desc->in_extra + 2 * desc->t_bands;
    m->n_grid = off * desc->feat;
    int64_t n = 0, k = m->n_in;
    for (int h = 0; h < desc->n_hidden; ++h) {
        n += (int64_t)desc->width * k + desc->width;
        k = desc->width;
    }
    n += (int64_t)desc->out_dim * k + desc->out_dim;
    m->n_mlp = n;
    m->mlp_plain_len = n;
    cudaError_t e = cudaGetDevice(&m->device);
    if (e == cudaSuccess) e = cudaMalloc(&m->params, sizeof(float) * (m->n_grid + m->n_mlp));
    if (e == cudaSuccess) e = cudaMalloc(&m->grid_f16, sizeof(__half) * (m->n_grid > 0 ? m->n_grid : 1));
    if (e == cudaSuccess) e = cudaMalloc(&m->mlp_plain, sizeof(float) * m->mlp_plain_len);
    if (e == cudaSuccess) e = cudaMemset(m->params, 0, sizeof(float) * (m->n_grid + m->n_mlp));
    if (e == cudaSuccess) e = cudaMemset(m->grid_f16, 0, sizeof(__half) * (m->n_grid > 0 ? m->n_grid : 1));
    if (e == cudaSuccess) e = cudaMemset(m->mlp_plain, 0, sizeof(float) * m->mlp_plain_len);
    // pair table when the dense levels are the first ones and an entry is one 32-bit word
    int nd = 0;
    while (nd < desc->levels && m->dense[nd]) ++nd;
    bool prefix = nd > 0 && desc->feat == 2 && (NIV_DENSE_PAIRS == 1 || (NIV_DENSE_PAIRS == 2 && desc->dims == 4));
    for (int l = nd; l < desc->levels; ++l) prefix = prefix && !m->dense[l];
    if (e == cudaSuccess && prefix) {
        m->n_pair = nd < desc->levels ? m->offset[nd] : m->total_entries;
        e = cudaMalloc(&m->grid_pair16, sizeof(uint2) * m->n_pair);
        if (e == cudaSuccess) e = cudaMemset(m->grid_pair16, 0, sizeof(uint2) * m->n_pair);
    }
    if (e != cudaSuccess) {
        free_model(m);
        return niv_cuda_fail(e, "niv_create allocation");
    }
    *out = m;
    return NIV_OK;
}

int niv_destroy(niv_handle h) {
    if (!h) return NIV_OK;
    cudaDeviceSynchronize();
    free_model(h);
    return NIV_OK;
}

int niv_level_info(niv_handle h, int32_t level, int32_t* res, int32_t* dense, int64_t* first_entry,
                   int64_t* entries) {
    if (!h) return niv_fail(NIV_ERR_ARG, "handle is NULL");
    if (level < 0 || level >= h->d.levels) return niv_fail(NIV_ERR_ARG, "level out of range");
    if (res) *res = h->res[level];
    if (dense) *dense = h->dense[level];
    if (first_entry) *first_entry = h->offset[level];
    if (entries) *entries = h->entries[level];
    return NIV_OK;
}

int niv_param_count(niv_handle h, int64_t* n_grid_values, int64_t* n_mlp_values) {
    if (!h) return niv_fail(NIV_ERR_ARG, "handle is NULL");
    if (n_grid_values) *n_grid_values = h->n_grid;
    if (n_mlp_values) *n_mlp_values = h->n_mlp;
    return NIV_OK;
}

int niv_set_params(niv_handle h, const float* params, int64_t n, niv_stream stream) {
    if (!h || !params) return niv_fail(NIV_ERR_ARG, "handle or params is NULL");
    if (n != h->n_grid + h->n_mlp) return niv_fail(NIV_ERR_ARG, "parameter count mismatch");
    int rc = check_device(h);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    NIV_CUDA(cudaMemcpyAsync(h->params, params, sizeof(float) * n, cudaMemcpyDefault, s));
    rc = refresh_inference(h, s);
    if (rc) return rc;
    // new parameters start a new optimisation
    h->adam_step = 0;
    if (h->adam_m) NIV_CUDA(cudaMemsetAsync(h->adam_m, 0, sizeof(float) * n, s));
    if (h->adam_v) NIV_CUDA(cudaMemsetAsync(h->adam_v, 0, sizeof(float) * n, s));
    NIV_CUDA(cudaStreamSynchronize(s));
    return NIV_OK;
}

int niv_get_params(niv_handle h, float* out, int64_t n, niv_stream stream) {
    if (!h || !out) return niv_fail(NIV_ERR_ARG, "handle or out is NULL");
    if (n != h->n_grid + h->n_mlp) return niv_fail(NIV_ERR_ARG, "parameter count mismatch");
    int rc = check_device(h);
    if (rc) return rc;
    NIV_CUDA(cudaMemcpyAsync(out, h->params, sizeof(float) * n, cudaMemcpyDefault, (cudaStream_t)stream));
    NIV_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return NIV_OK;
}

namespace {
// Model files (little-endian hosts): "NIVM", version, the description field by field, the
// parameter count, the FP32 parameters; version 2 adds the optimiser state (training forward
// precision, Adam step count, whether the moments follow, the two FP32 moment vectors).
constexpr char kFileMagic[4] = {'N', 'I', 'V', 'M'};
constexpr uint32_t kFileVersion = 2;

bool put_bytes(FILE* f, const void* v, size_t n) { return fwrite(v, n, 1, f) == 1; }
bool get_bytes(FILE* f, void* v, size_t n) { return fread(v, n, 1, f) == 1; }
#define put(f, v) put_bytes((f), &(v), sizeof(v))
#define get(f, v) get_bytes((f), &(v), sizeof(v))

bool put_desc(FILE* f, const niv_model_desc& d) {
    return put(f, d.dims) && put(f, d.levels) && put(f, d.feat) && put(f, d.log2_T) && put(f, d.base) &&
           put(f, d.growth) && put(f, d.n_hidden) && put(f, d.width) && put(f, d.in_extra) && put(f, d.out_dim) &&
           put(f, d.out_act) && put(f, d.prime_t) && put(f, d.pe_bands) && put(f, d.t_bands);
}
bool get_desc(FILE* f, niv_model_desc& d) {
    return get(f, d.dims) && get(f, d.levels) && get(f, d.feat) && get(f, d.log2_T) && get(f, d.base) &&
           get(f, d.growth) && get(f, d.n_hidden) && get(f, d.width) && get(f, d.in_extra) && get(f, d.out_dim) &&
           get(f, d.out_act) && get(f, d.prime_t) && get(f, d.pe_bands) && get(f, d.t_bands);
}
}  // namespace

int niv_save(niv_handle h, const char* path, niv_stream stream) {
    if (!h || !path) return niv_fail(NIV_ERR_ARG, "handle or path is NULL");
    const int64_t n = h->n_grid + h->n_mlp;
    std::vector<float> params((size_t)n);
    int rc = niv_get_params(h, params.data(), n, stream);
    if (rc) return rc;
    // the optimiser state: Adam moments exist once a training call has run
    const int32_t fwd = h->train_f16 ? NIV_FP16 : NIV_FP32;
    const int64_t step = h->adam_step;
    const int32_t has_moments = (h->adam_m && h->adam_v) ? 1 : 0;
    std::vector<float> mom;
    if (has_moments) {
        mom.resize(2 * (size_t)n);
        cudaStream_t s = (cudaStream_t)stream;
        NIV_CUDA(cudaMemcpyAsync(mom.data(), h->adam_m, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
        NIV_CUDA(cudaMemcpyAsync(mom.data() + n, h->adam_v, sizeof(float) * n, cudaMemcpyDeviceToHost, s));
        NIV_CUDA(cudaStreamSynchronize(s));
    }
    FILE* f = fopen(path, "wb");
    if (!f) return niv_fail(NIV_ERR_ARG, std::string("cannot open for writing: ") + path);
    bool ok = fwrite(kFileMagic, 1, 4, f) == 4 && put(f, kFileVersion) && put_desc(f, h->d) && put(f, n) &&
              fwrite(params.data(), sizeof(float), (size_t)n, f) == (size_t)n && put(f, fwd) && put(f, step) &&
              put(f, has_moments) && (!has_moments || fwrite(mom.data(), sizeof(float), mom.size(), f) == mom.size());
    ok = (fclose(f) == 0) && ok;
    if (!ok) return niv_fail(NIV_ERR_ARG, std::string("write failed: ") + path);
    return NIV_OK;
}

int niv_load(const char* path, niv_handle* out) {
    if (!path || !out) return niv_fail(NIV_ERR_ARG, "path or out is NULL");
    FILE* f = fopen(path, "rb");
    if (!f) return niv_fail(NIV_ERR_ARG, std::string("cannot open: ") + path);
    char magic[4];
    uint32_t version = 0;
    niv_model_desc d;
    memset(&d, 0, sizeof d);
    int64_t n = 0;
    if (fread(magic, 1, 4, f) != 4 || memcmp(magic, kFileMagic, 4) != 0 || !get(f, version)) {
        fclose(f);
        return niv_fail(NIV_ERR_ARG, "not a model file (magic)");
    }
    if (version < 1 || version > kFileVersion || !get_desc(f, d) || !get(f, n)) {
        fclose(f);
        return niv_fail(NIV_ERR_ARG, "unsupported model file version or truncated header");
    }
    int rc = validate_desc(&d);
    if (rc) {
        fclose(f);
        return rc;
    }
    niv_handle h = nullptr;
    rc = niv_create(&d, &h);
    if (rc) {
        fclose(f);
        return rc;
    }
    if (n != h->n_grid + h->n_mlp) {
        fclose(f);
        niv_destroy(h);
        return niv_fail(NIV_ERR_ARG, "parameter count differs from the description's");
    }
    std::vector<float> params((size_t)n), mom;
    bool full = fread(params.data(), sizeof(float), (size_t)n, f) == (size_t)n;
    int32_t fwd = NIV_FP32, has_moments = 0;
    int64_t step = 0;
    if (full && version >= 2) {  // the optimiser state
        full = get(f, fwd) && get(f, step) && get(f, has_moments) && (fwd == NIV_FP32 || fwd == NIV_FP16) &&
               step >= 0 && (has_moments == 0 || has_moments == 1);
        if (full && has_moments) {
            mom.resize(2 * (size_t)n);
            full = fread(mom.data(), sizeof(float), mom.size(), f) == mom.size();
        }
    }
    fclose(f);
    if (!full) {
        niv_destroy(h);
        return niv_fail(NIV_ERR_ARG, "model file truncated or its optimiser state malformed");
    }
    rc = niv_set_params(h, params.data(), n, nullptr);
    if (!rc && has_moments) rc = ensure_training_state(h);
    if (!rc && has_moments) {
        cudaError_t e = cudaMemcpy(h->adam_m, mom.data(), sizeof(float) * n, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = cudaMemcpy(h->adam_v, mom.data() + n, sizeof(float) * n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) rc = niv_cuda_fail(e, "niv_load: Adam moments");
    }
    if (rc) {
        niv_destroy(h);
        return rc;
    }
    h->train_f16 = fwd == NIV_FP16;
    h->adam_step = step;
    *out = h;
    return NIV_OK;
}

#undef put
#undef get

int niv_query(niv_handle h, const void* pos, const void* nrm, int64_t n, int32_t dtype_in,
              const niv_query_params* params, void* out_E, int32_t dtype_out, int32_t precision,
              niv_stream stream) {
    if (!h || !params) return niv_fail(NIV_ERR_ARG, "handle or params is NULL");
    if (n < 0) return niv_fail(NIV_ERR_ARG, "n < 0");
    if (n == 0) return NIV_OK;
    if (!pos || !nrm || !out_E) return niv_fail(NIV_ERR_ARG, "NULL record pointer");
    if (!aligned16(pos) || !aligned16(nrm) || !aligned16(out_E))
        return niv_fail(NIV_ERR_ALIGN, "record pointers must be 16-byte aligned");
    if ((dtype_in != NIV_F32 && dtype_in != NIV_F16) || (dtype_out != NIV_F32 && dtype_out != NIV_F16))
        return niv_fail(NIV_ERR_ARG, "record dtype must be NIV_F32 or NIV_F16");
    for (int k = 0; k < 3; ++k)
        if (!(params->aabb_max[k] > params->aabb_min[k])) return niv_fail(NIV_ERR_ARG, "empty aabb");
    if (params->image_width < 0) return niv_fail(NIV_ERR_ARG, "image_width < 0");
    int rc = check_device(h);
    if (rc) return rc;
    if (h->infer_dirty) {  // trained since the inference copies were built
        rc = refresh_inference(h, (cudaStream_t)stream);
        if (rc) return rc;
    }
    GridArgs g = niv_grid_args(h, params);
    IoArgs io;
    io.pos = pos;
    io.nrm = nrm;
    io.out = out_E;
    io.n = n;
    io.image_width = params->image_width;
    io.in_f16 = dtype_in == NIV_F16;
    io.out_f16 = dtype_out == NIV_F16;
    switch (precision) {
        case NIV_FP32: return niv_launch_query_fp32(h, g, io, (cudaStream_t)stream);
        case NIV_FP16: return niv_launch_query_tc(h, g, io, precision, (cudaStream_t)stream);
        case NIV_FP8: return niv_launch_query_f8(h, g, io, (cudaStream_t)stream);
        default: return niv_fail(NIV_ERR_UNSUPPORTED, "precision not supported");
    }
}

namespace {
// Streams and events of the pipelined host query, created once per handle.
int host_pipe_init(niv_model* h) {
    if (h->host_pipe) return NIV_OK;
    for (int i = 0; i < 2; ++i) {
        NIV_CUDA(cudaStreamCreateWithFlags(&h->host_copy[i], cudaStreamNonBlocking));
        NIV_CUDA(cudaEventCreateWithFlags(&h->host_join[i], cudaEventDisableTiming));
        for (int c = 0; c < NIV_HOST_CHUNKS_MAX; ++c)
            NIV_CUDA(cudaEventCreateWithFlags(&h->host_ev[i][c], cudaEventDisableTiming));
    }
    h->host_pipe = 1;
    return NIV_OK;
}

// Chunking of one host query: `count` chunks of `per` records (the last one shorter).
struct HostChunks {
    int64_t per;
    int count;
};

// Chunks of whole tiles (whole bands of NIV_TILE_ROWS rows of tiles for images) of about two
// waves of the tensor-core kernel (8 warpgroups on every SM), at least 65,536 records
// each and at most NIV_HOST_CHUNKS_MAX of them; NIV_HOST_CHUNKS sets the count instead.
HostChunks host_chunks(int64_t n, int64_t W) {
    const int64_t granule = W > 0 ? NIV_TILE_ROWS * W : 128;  // records of one band / one tile
    const int64_t granule_tiles = W > 0 ? (W + kTileW - 1) / kTileW : 1;
    const int64_t granules = (n + granule - 1) / granule;
    int dev = 0, sms = 148;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    int64_t per_g = (2 * 8 * (int64_t)sms + granule_tiles / 2) / granule_tiles;  // granules per chunk
    const int forced = niv_env_int("NIV_HOST_CHUNKS", 0);
    if (forced > 0) per_g = (granules + forced - 1) / forced;
    const int64_t min_g = (65536 + granule - 1) / granule;
    if (per_g < min_g) per_g = min_g;
    if (per_g < 1) per_g = 1;
    if ((granules + per_g - 1) / per_g > NIV_HOST_CHUNKS_MAX) per_g = (granules + NIV_HOST_CHUNKS_MAX - 1) / NIV_HOST_CHUNKS_MAX;
    HostChunks c;
    c.per = per_g * granule;
    c.count = (int)((n + c.per - 1) / c.per);
    return c;
}

// Queue the chunked pipeline: host->device copies on host_copy[0], queries on `s`,
// device->host copies on host_copy[1], ordered after the work already queued on `s` and
// joined back into it.  All copies in and queries are queued before the first copy out,
// so that a copy out (which can hold the calling thread with pageable memory) never holds
// up the queueing of later chunks.
int host_pipeline(niv_model* h, const void* pos, const void* nrm, int64_t n, int32_t dtype_in,
                  const niv_query_params* params, void* out_E, int32_t dtype_out, int32_t precision,
                  cudaStream_t s, const HostChunks& ch) {
    const size_t rin = dtype_in == NIV_F16 ? 8 : 16, rout = dtype_out == NIV_F16 ? 8 : 16;
    const size_t a_in = ((size_t)n * rin + 255) & ~(size_t)255;
    char* base = (char*)h->stage;
    cudaStream_t up = h->host_copy[0], down = h->host_copy[1];
    NIV_CUDA(cudaEventRecord(h->host_join[0], s));
    NIV_CUDA(cudaStreamWaitEvent(up, h->host_join[0], 0));
    for (int c = 0; c < ch.count; ++c) {
        const int64_t r0 = c * ch.per, m = n - r0 < ch.per ? n - r0 : ch.per;
        char* dpos = base + r0 * rin;
        char* dnrm = base + a_in + r0 * rin;
        NIV_CUDA(cudaMemcpyAsync(dpos, (const char*)pos + r0 * rin, m * rin, cudaMemcpyHostToDevice, up));
        NIV_CUDA(cudaMemcpyAsync(dnrm, (const char*)nrm + r0 * rin, m * rin, cudaMemcpyHostToDevice, up));
        NIV_CUDA(cudaEventRecord(h->host_ev[0][c], up));
        NIV_CUDA(cudaStreamWaitEvent(s, h->host_ev[0][c], 0));
        int rc = niv_query(h, dpos, dnrm, m, dtype_in, params, base + 2 * a_in + r0 * rout, dtype_out, precision,
                           (niv_stream)s);
        if (rc) return rc;
        NIV_CUDA(cudaEventRecord(h->host_ev[1][c], s));
    }
    for (int c = 0; c < ch.count; ++c) {
        const int64_t r0 = c * ch.per, m = n - r0 < ch.per ? n - r0 : ch.per;
        NIV_CUDA(cudaStreamWaitEvent(down, h->host_ev[1][c], 0));
        NIV_CUDA(cudaMemcpyAsync((char*)out_E + r0 * rout, base + 2 * a_in + r0 * rout, m * rout,
                                 cudaMemcpyDeviceToHost, down));
    }
    NIV_CUDA(cudaEventRecord(h->host_join[1], down));
    NIV_CUDA(cudaStreamWaitEvent(s, h->host_join[1], 0));
    return NIV_OK;
}

// Device address of page-locked host memory that kernels may load and store directly
// (over NVLink-C2C on Grace systems, PCIe elsewhere); nullptr for other memory.
void* mapped_host(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

}  // namespace

// Page-locked host buffers that the GPU can address are read and written by the query
// kernel itself (over NVLink-C2C on Grace systems): one launch, no staging copies.  Other
// host memory is split into chunks of whole tiles (whole bands of tile rows of the image when
// image_width > 0) that flow through three engines at once: the host->device copy of
// chunk c+1, the query of chunk c and the device->host copy of chunk c-1 overlap, so a
// call costs about the slowest of the three plus one chunk of each of the others.
int niv_query_host(niv_handle h, const void* pos, const void* nrm, int64_t n, int32_t dtype_in,
                   const niv_query_params* params, void* out_E, int32_t dtype_out, int32_t precision,
                   niv_stream stream) {
    if (!h || !params) return niv_fail(NIV_ERR_ARG, "handle or params is NULL");
    if (n < 0) return niv_fail(NIV_ERR_ARG, "n < 0");
    if (n == 0) return NIV_OK;
    if (!pos || !nrm || !out_E) return niv_fail(NIV_ERR_ARG, "NULL record pointer");
    if ((dtype_in != NIV_F32 && dtype_in != NIV_F16) || (dtype_out != NIV_F32 && dtype_out != NIV_F16))
        return niv_fail(NIV_ERR_ARG, "record dtype must be NIV_F32 or NIV_F16");
    if (params->image_width < 0) return niv_fail(NIV_ERR_ARG, "image_width < 0");
    int rc = check_device(h);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    // NIV_HOST_MODE: 0 (default) direct where possible, 1 always the chunked pipeline
    if (niv_env_int("NIV_HOST_MODE", 0) == 0) {
        const void* dpos = mapped_host(pos);
        const void* dnrm = mapped_host(nrm);
        void* dout = mapped_host(out_E);
        if (dpos && dnrm && dout && aligned16(dpos) && aligned16(dnrm) && aligned16(dout)) {
            rc = niv_query(h, dpos, dnrm, n, dtype_in, params, dout, dtype_out, precision, stream);
            if (rc) {
                cudaStreamSynchronize(s);
                return rc;
            }
            NIV_CUDA(cudaStreamSynchronize(s));
            return NIV_OK;
        }
    }
    const size_t rin = dtype_in == NIV_F16 ? 8 : 16, rout = dtype_out == NIV_F16 ? 8 : 16;
    const size_t a_in = ((size_t)n * rin + 255) & ~(size_t)255, need = 2 * a_in + (size_t)n * rout;
    if (h->stage_bytes < need) {
        NIV_CUDA(cudaStreamSynchronize(s));
        cudaFree(h->stage);
        h->stage = nullptr;
        h->stage_bytes = 0;
        NIV_CUDA(cudaMalloc(&h->stage, need));
        h->stage_bytes = need;
    }
    rc = host_pipe_init(h);
    if (rc) return rc;
    rc = host_pipeline(h, pos, nrm, n, dtype_in, params, out_E, dtype_out, precision, s,
                       host_chunks(n, params->image_width));
    if (rc) {
        for (int i = 0; i < 2; ++i) cudaStreamSynchronize(h->host_copy[i]);
        cudaStreamSynchronize(s);
        return rc;
    }
    NIV_CUDA(cudaStreamSynchronize(s));
    return NIV_OK;
}

int niv_encode(niv_handle h, const void* pos, int64_t n, int32_t dtype_in, const niv_query_params* params,
               float* out_enc, uint32_t* out_idx, niv_stream stream) {
    if (!h || !params) return niv_fail(NIV_ERR_ARG, "handle or params is NULL");
    if (n < 0) return niv_fail(NIV_ERR_ARG, "n < 0");
    if (n == 0) return NIV_OK;
    if (!pos) return niv_fail(NIV_ERR_ARG, "pos is NULL");
    if (!aligned16(pos)) return niv_fail(NIV_ERR_ALIGN, "pos must be 16-byte aligned");
    if (dtype_in != NIV_F32 && dtype_in != NIV_F16) return niv_fail(NIV_ERR_ARG, "bad dtype");
    for (int k = 0; k < 3; ++k)
        if (!(params->aabb_max[k] > params->aabb_min[k])) return niv_fail(NIV_ERR_ARG, "empty aabb");
    int rc = check_device(h);
    if (rc) return rc;
    GridArgs g = niv_grid_args(h, params);
    IoArgs io;
    memset(&io, 0, sizeof io);
    io.pos = pos;
    io.n = n;
    io.in_f16 = dtype_in == NIV_F16;
    return niv_launch_encode(h, g, io, out_enc, out_idx, (cudaStream_t)stream);
}

int niv_fp8_calibrate(niv_handle h, const void* pos, const void* nrm, int64_t n, int32_t dtype_in,
                      const niv_query_params* params, niv_stream stream) {
    if (!h || !params) return niv_fail(NIV_ERR_ARG, "handle or params is NULL");
    if (n <= 0) return niv_fail(NIV_ERR_ARG, "calibration needs at least one record");
    if (!pos || !nrm) return niv_fail(NIV_ERR_ARG, "NULL record pointer");
    if (!aligned16(pos) || !aligned16(nrm)) return niv_fail(NIV_ERR_ALIGN, "record pointers must be 16-byte aligned");
    if (dtype_in != NIV_F32 && dtype_in != NIV_F16) return niv_fail(NIV_ERR_ARG, "bad dtype");
    if (h->d.width < 32) return niv_fail(NIV_ERR_UNSUPPORTED, "the FP8 path needs width 32 or 64");
    for (int k = 0; k < 3; ++k)
        if (!(params->aabb_max[k] > params->aabb_min[k])) return niv_fail(NIV_ERR_ARG, "empty aabb");
    int rc = check_device(h);
    if (rc) return rc;
    GridArgs g = niv_grid_args(h, params);
    IoArgs io;
    memset(&io, 0, sizeof io);
    io.pos = pos;
    io.nrm = nrm;
    io.n = n;
    io.in_f16 = dtype_in == NIV_F16;
    return niv_calibrate_f8(h, g, io, (cudaStream_t)stream);
}

int niv_fp8_get_scales(niv_handle h, float* s_act, float* s_w, float* amax, int32_t count) {
    if (!h) return niv_fail(NIV_ERR_ARG, "handle is NULL");
    if (!h->fp8_ready) return niv_fail(NIV_ERR_ARG, "not calibrated");
    if (count != h->d.n_hidden + 1) return niv_fail(NIV_ERR_ARG, "count must be n_hidden + 1");
    for (int l = 0; l < count; ++l) {
        if (s_act) s_act[l] = h->fp8_sact[l];
        if (s_w) s_w[l] = h->fp8_sw[l];
        if (amax) amax[l] = h->fp8_amax_host[l];
    }
    return NIV_OK;
}

namespace {
int grad_common(niv_handle h, const float* pos, const float* nrm, const float* t, const float* target, int64_t n,
                const niv_query_params* params, float eps, bool vjp, double* loss_out, niv_stream stream) {
    if (!h || !params) return niv_fail(NIV_ERR_ARG, "handle or params is NULL");
    if (n <= 0) return niv_fail(NIV_ERR_ARG, "n must be positive");
    if (!pos || !nrm || !target) return niv_fail(NIV_ERR_ARG, "NULL record pointer");
    if (!aligned16(pos) || !aligned16(nrm) || !aligned16(target))
        return niv_fail(NIV_ERR_ALIGN, "record pointers must be 16-byte aligned");
    if (t && ((uintptr_t)t & 3u)) return niv_fail(NIV_ERR_ALIGN, "t must be 4-byte aligned");
    if (!(eps > 0.0f)) return niv_fail(NIV_ERR_ARG, "eps must be positive");
    for (int k = 0; k < 3; ++k)
        if (!(params->aabb_max[k] > params->aabb_min[k])) return niv_fail(NIV_ERR_ARG, "empty aabb");
    int rc = check_device(h);
    if (rc) return rc;
    rc = ensure_training_state(h);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    GridArgs g = niv_grid_args(h, params);
    rc = niv_train_grad(h, g, (const float4*)pos, (const float4*)nrm, t, (const float4*)target, n, eps, vjp, s);
    if (rc) return rc;
    if (loss_out) {
        double acc = 0.0;
        NIV_CUDA(cudaMemcpyAsync(&acc, h->loss_acc, sizeof(double), cudaMemcpyDeviceToHost, s));
        NIV_CUDA(cudaStreamSynchronize(s));
        *loss_out = acc / (3.0 * (double)n);
    }
    return NIV_OK;
}
}  // namespace

int niv_set_train_forward(niv_handle h, int32_t precision) {
    if (!h) return niv_fail(NIV_ERR_ARG, "handle is NULL");
    if (precision != NIV_FP32 && precision != NIV_FP16)
        return niv_fail(NIV_ERR_UNSUPPORTED, "training forward precision must be NIV_FP32 or NIV_FP16");
    h->train_f16 = precision == NIV_FP16;
    return NIV_OK;
}

int niv_grad(niv_handle h, const float* pos, const float* nrm, const float* t, const float* target, int64_t n,
             const niv_query_params* params, float eps, double* loss_out, niv_stream stream) {
    return grad_common(h, pos, nrm, t, target, n, params, eps, false, loss_out, stream);
}

int niv_backward(niv_handle h, const float* pos, const float* nrm, const float* t, const float* grad_E, int64_t n,
                 const niv_query_params* params, niv_stream stream) {
    return grad_common(h, pos, nrm, t, grad_E, n, params, 1.0f, true, nullptr, stream);
}

int niv_get_grads(niv_handle h, float* out, int64_t n, niv_stream stream) {
    if (!h || !out) return niv_fail(NIV_ERR_ARG, "handle or out is NULL");
    if (n != h->n_grid + h->n_mlp) return niv_fail(NIV_ERR_ARG, "gradient count mismatch");
    if (!h->grad) return niv_fail(NIV_ERR_ARG, "no gradients computed yet");
    NIV_CUDA(cudaMemcpyAsync(out, h->grad, sizeof(float) * n, cudaMemcpyDefault, (cudaStream_t)stream));
    NIV_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return NIV_OK;
}

int niv_set_grads(niv_handle h, const float* grads, int64_t n, niv_stream stream) {
    if (!h || !grads) return niv_fail(NIV_ERR_ARG, "handle or grads is NULL");
    if (n != h->n_grid + h->n_mlp) return niv_fail(NIV_ERR_ARG, "gradient count mismatch");
    int rc = check_device(h);
    if (rc) return rc;
    rc = ensure_training_state(h);
    if (rc) return rc;
    NIV_CUDA(cudaMemcpyAsync(h->grad, grads, sizeof(float) * n, cudaMemcpyDefault, (cudaStream_t)stream));
    NIV_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return NIV_OK;
}

int niv_adam_step(niv_handle h, float lr, float beta1, float beta2, float eps, niv_stream stream) {
    if (!h) return niv_fail(NIV_ERR_ARG, "handle is NULL");
    if (!h->grad) return niv_fail(NIV_ERR_ARG, "no gradients computed yet");
    if (!(beta1 >= 0.0f && beta1 < 1.0f && beta2 >= 0.0f && beta2 < 1.0f) || !(eps >= 0.0f))
        return niv_fail(NIV_ERR_ARG, "betas must lie in [0, 1) and eps >= 0");
    int rc = check_device(h);
    if (rc) return rc;
    return niv_train_adam(h, lr, beta1, beta2, eps, (cudaStream_t)stream);
}

int niv_fit(niv_handle h, const float* pos, const float* nrm, const float* t, const float* target, int64_t n,
            const niv_query_params* params, const niv_fit_params* fp, double* loss_out, niv_stream stream) {
    if (!fp) return niv_fail(NIV_ERR_ARG, "fit params is NULL");
    int rc = niv_grad(h, pos, nrm, t, target, n, params, fp->loss_eps, loss_out, stream);
    if (rc) return rc;
    return niv_adam_step(h, fp->lr, fp->beta1, fp->beta2, fp->adam_eps, stream);
}

int niv_mc_irradiance(const float* scene, int64_t scene_len, const float* x4, const float* n4, const float* t,
                      int64_t m, int32_t spp, uint64_t seed, uint64_t index_base, int32_t mode, double* out_E,
                      uint8_t* out_keep, niv_stream stream) {
    if (!scene || scene_len < 48) return niv_fail(NIV_ERR_ARG, "scene description missing or too short");
    if (m < 0) return niv_fail(NIV_ERR_ARG, "m < 0");
    if (m == 0) return NIV_OK;
    if (!x4 || !n4 || !out_E) return niv_fail(NIV_ERR_ARG, "NULL pointer");
    if (!aligned16(x4) || !aligned16(n4)) return niv_fail(NIV_ERR_ALIGN, "record pointers must be 16-byte aligned");
    if (spp < 1 || spp > 65535) return niv_fail(NIV_ERR_ARG, "spp must be in 1..65535");
    if (mode != NIV_MC_TOTAL && mode != NIV_MC_INDIRECT) return niv_fail(NIV_ERR_ARG, "mode must be total or indirect");
    return niv_launch_mc(scene, scene_len, x4, n4, t, m, spp, seed, index_base, mode, out_E, out_keep,
                         (cudaStream_t)stream);
}

int niv_probe_bake(const float* scene, int64_t scene_len, const int32_t* P, const float* lo, const float* hi,
                   int32_t rays, uint64_t seed, uint64_t index_base, double* out_coef64, void* out_coef16,
                   niv_stream stream) {
    if (!scene || scene_len < 48 || !P || !lo || !hi) return niv_fail(NIV_ERR_ARG, "NULL argument");
    for (int a = 0; a < 3; ++a) {
        if (P[a] < 2) return niv_fail(NIV_ERR_ARG, "every lattice axis needs at least 2 probes");
        if (!(hi[a] > lo[a])) return niv_fail(NIV_ERR_ARG, "empty probe box");
    }
    if (rays < 1) return niv_fail(NIV_ERR_ARG, "rays must be positive");
    if (!out_coef64 && !out_coef16) return niv_fail(NIV_ERR_ARG, "no output");
    if (out_coef16 && !aligned16(out_coef16)) return niv_fail(NIV_ERR_ALIGN, "out_coef16 must be 16-byte aligned");
    return niv_launch_probe_bake(scene, scene_len, P, lo, hi, rays, seed, index_base, out_coef64, (__half*)out_coef16,
                                 (cudaStream_t)stream);
}

namespace {
int probe_query_common(const void* coef16, const int32_t* P, const float* lo, const float* hi, const float* scene,
                       int64_t scene_len, float t, const void* pos, const void* nrm, int64_t n, int32_t dtype_in,
                       void* out_E, int32_t dtype_out, int32_t image_width, niv_stream stream) {
    if (!coef16 || !P || !lo || !hi) return niv_fail(NIV_ERR_ARG, "NULL argument");
    if (n < 0) return niv_fail(NIV_ERR_ARG, "n < 0");
    if (n == 0) return NIV_OK;
    if (!pos || !nrm || !out_E) return niv_fail(NIV_ERR_ARG, "NULL record pointer");
    if (!aligned16(pos) || !aligned16(nrm) || !aligned16(out_E) || !aligned16(coef16))
        return niv_fail(NIV_ERR_ALIGN, "pointers must be 16-byte aligned");
    if ((dtype_in != NIV_F32 && dtype_in != NIV_F16) || (dtype_out != NIV_F32 && dtype_out != NIV_F16))
        return niv_fail(NIV_ERR_ARG, "record dtype must be NIV_F32 or NIV_F16");
    for (int a = 0; a < 3; ++a) {
        if (P[a] < 2) return niv_fail(NIV_ERR_ARG, "every lattice axis needs at least 2 probes");
        if (!(hi[a] > lo[a])) return niv_fail(NIV_ERR_ARG, "empty probe box");
    }
    if (image_width < 0) return niv_fail(NIV_ERR_ARG, "image_width < 0");
    IoArgs io;
    io.pos = pos;
    io.nrm = nrm;
    io.out = out_E;
    io.n = n;
    io.image_width = image_width;
    io.in_f16 = dtype_in == NIV_F16;
    io.out_f16 = dtype_out == NIV_F16;
    return niv_launch_probe_query(coef16, P, lo, hi, io, scene, scene_len, t, (cudaStream_t)stream);
}
}  // namespace

int niv_probe_query(const void* coef16, const int32_t* P, const float* lo, const float* hi, const void* pos,
                    const void* nrm, int64_t n, int32_t dtype_in, void* out_E, int32_t dtype_out, int32_t image_width,
                    niv_stream stream) {
    return probe_query_common(coef16, P, lo, hi, nullptr, 0, 0.0f, pos, nrm, n, dtype_in, out_E, dtype_out,
                              image_width, stream);
}

int niv_probe_query_rt(const void* coef16, const int32_t* P, const float* lo, const float* hi, const float* scene,
                       int64_t scene_len, float t, const void* pos, const void* nrm, int64_t n, int32_t dtype_in,
                       void* out_E, int32_t dtype_out, int32_t image_width, niv_stream stream) {
    if (!scene) return niv_fail(NIV_ERR_ARG, "scene is NULL");
    return probe_query_common(coef16, P, lo, hi, scene, scene_len, t, pos, nrm, n, dtype_in, out_E, dtype_out,
                              image_width, stream);
}

int niv_compact_targets(const float* x4, const float* n4, const float* t, const double* E, const uint8_t* keep,
                        int64_t m, float* out_x4, float* out_n4, float* out_t, float* out_target4, int64_t* out_count,
                        niv_stream stream) {
    if (!x4 || !n4 || !E || !keep || !out_x4 || !out_n4 || !out_target4 || !out_count)
        return niv_fail(NIV_ERR_ARG, "NULL argument");
    if (m < 0) return niv_fail(NIV_ERR_ARG, "m < 0");
    *out_count = 0;
    if (m == 0) return NIV_OK;
    if (!aligned16(x4) || !aligned16(n4) || !aligned16(out_x4) || !aligned16(out_n4) || !aligned16(out_target4))
        return niv_fail(NIV_ERR_ALIGN, "record pointers must be 16-byte aligned");
    int dev = 0;
    NIV_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return niv_fail(NIV_ERR_UNSUPPORTED, "device ordinal above 63");
    const size_t nb = (size_t)((m + 1023) / 1024);
    const size_t need = 64 + nb * sizeof(int);
    cudaStream_t s = (cudaStream_t)stream;
    std::lock_guard<std::mutex> lk(g_compact_mu);
    if (g_compact_bytes[dev] < need) {
        NIV_CUDA(cudaStreamSynchronize(s));
        cudaFree(g_compact[dev]);
        g_compact[dev] = nullptr;
        g_compact_bytes[dev] = 0;
        NIV_CUDA(cudaMalloc(&g_compact[dev], need));
        g_compact_bytes[dev] = need;
    }
    int64_t* count_dev = (int64_t*)g_compact[dev];
    int* offsets = (int*)((char*)g_compact[dev] + 64);
    int rc = niv_launch_compact(x4, n4, t, E, keep, m, out_x4, out_n4, out_t, out_target4, count_dev, offsets, s);
    if (rc) return rc;
    NIV_CUDA(cudaMemcpyAsync(out_count, count_dev, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    NIV_CUDA(cudaStreamSynchronize(s));
    return NIV_OK;
}

int niv_query_shade(niv_handle h, const void* pos, const void* nrm, const void* albedo, const void* direct, int64_t n,
                    int32_t dtype_in, const niv_query_params* params, void* out_rgba, int32_t precision,
                    niv_stream stream) {
    if (!h || !params) return niv_fail(NIV_ERR_ARG, "handle or params is NULL");
    if (n < 0) return niv_fail(NIV_ERR_ARG, "n < 0");
    if (n == 0) return NIV_OK;
    if (!pos || !nrm || !albedo || !direct || !out_rgba) return niv_fail(NIV_ERR_ARG, "NULL record pointer");
    if (!aligned16(pos) || !aligned16(nrm) || !aligned16(albedo) || !aligned16(direct) || !aligned16(out_rgba))
        return niv_fail(NIV_ERR_ALIGN, "record pointers must be 16-byte aligned");
    if (dtype_in != NIV_F32 && dtype_in != NIV_F16) return niv_fail(NIV_ERR_ARG, "record dtype must be NIV_F32 or NIV_F16");
    for (int k = 0; k < 3; ++k)
        if (!(params->aabb_max[k] > params->aabb_min[k])) return niv_fail(NIV_ERR_ARG, "empty aabb");
    if (params->image_width < 0) return niv_fail(NIV_ERR_ARG, "image_width < 0");
    int rc = check_device(h);
    if (rc) return rc;
    if (h->infer_dirty) {
        rc = refresh_inference(h, (cudaStream_t)stream);
        if (rc) return rc;
    }
    GridArgs g = niv_grid_args(h, params);
    IoArgs io;
    io.pos = pos;
    io.nrm = nrm;
    io.out = out_rgba;
    io.n = n;
    io.image_width = params->image_width;
    io.in_f16 = dtype_in == NIV_F16;
    io.out_f16 = 1;
    io.albedo = albedo;
    io.direct = direct;
    switch (precision) {
        case NIV_FP32: return niv_launch_query_fp32(h, g, io, (cudaStream_t)stream);
        case NIV_FP16: return niv_launch_query_tc(h, g, io, precision, (cudaStream_t)stream);
        case NIV_FP8: return niv_launch_query_f8(h, g, io, (cudaStream_t)stream);
        default: return niv_fail(NIV_ERR_UNSUPPORTED, "precision not supported");
    }
}

int niv_dyn_create(const float* tris, int64_t n_tris, niv_dyn_handle* out) {
    if (!tris || !out) return niv_fail(NIV_ERR_ARG, "NULL argument");
    *out = nullptr;
    return niv_dyn_build(tris, n_tris, out);
}

int niv_dyn_destroy(niv_dyn_handle d) {
    if (!d) return NIV_OK;
    cudaDeviceSynchronize();
    niv_dyn_free(d);
    return NIV_OK;
}

int64_t niv_dyn_node_count(niv_dyn_handle d) { return d ? niv_dyn_node_count(static_cast<const niv_dyn*>(d)) : 0; }

int niv_dyn_ao(niv_dyn_handle d, const void* pos, const void* nrm, int64_t n, int32_t dtype_in, int32_t rays,
               float radius, uint64_t seed, float* out_ao, void* E_inout, int32_t dtype_E, niv_stream stream) {
    if (!d) return niv_fail(NIV_ERR_ARG, "dynamic geometry handle is NULL");
    if (n < 0) return niv_fail(NIV_ERR_ARG, "n < 0");
    if (n == 0) return NIV_OK;
    if (rays < 1 || rays > 1024) return niv_fail(NIV_ERR_ARG, "rays must be in 1..1024");
    if (!(radius > 0.0f) || !std::isfinite(radius)) return niv_fail(NIV_ERR_ARG, "radius must be > 0");
    if (!pos || !nrm) return niv_fail(NIV_ERR_ARG, "NULL record pointer");
    if (!aligned16(pos) || !aligned16(nrm) || (E_inout && !aligned16(E_inout)))
        return niv_fail(NIV_ERR_ALIGN, "record pointers must be 16-byte aligned");
    if ((dtype_in != NIV_F32 && dtype_in != NIV_F16) || (E_inout && dtype_E != NIV_F32 && dtype_E != NIV_F16))
        return niv_fail(NIV_ERR_ARG, "record dtype must be NIV_F32 or NIV_F16");
    int dev = -1;
    NIV_CUDA(cudaGetDevice(&dev));
    return niv_launch_ao(d, pos, nrm, n, dtype_in == NIV_F16, rays, radius, seed, out_ao, E_inout,
                         dtype_E == NIV_F16, (cudaStream_t)stream);
}

int niv_query_sub(niv_handle h, const void* pos, const void* nrm, int32_t full_width, int32_t full_height,
                  int32_t sub, int32_t dtype_in, const niv_query_params* params, void* out_E, int32_t dtype_out,
                  int32_t precision, niv_stream stream) {
    if (!h || !params) return niv_fail(NIV_ERR_ARG, "handle or params is NULL");
    if (full_width < 0 || full_height < 0) return niv_fail(NIV_ERR_ARG, "negative image size");
    if (sub < 1) return niv_fail(NIV_ERR_ARG, "sub must be >= 1");
    if (full_width == 0 || full_height == 0) return NIV_OK;
    if ((int64_t)full_width * sub > INT32_MAX) return niv_fail(NIV_ERR_UNSUPPORTED, "image too wide");
    if (!pos || !nrm || !out_E) return niv_fail(NIV_ERR_ARG, "NULL record pointer");
    if (!aligned16(pos) || !aligned16(nrm) || !aligned16(out_E))
        return niv_fail(NIV_ERR_ALIGN, "record pointers must be 16-byte aligned");
    if ((dtype_in != NIV_F32 && dtype_in != NIV_F16) || (dtype_out != NIV_F32 && dtype_out != NIV_F16))
        return niv_fail(NIV_ERR_ARG, "record dtype must be NIV_F32 or NIV_F16");
    for (int k = 0; k < 3; ++k)
        if (!(params->aabb_max[k] > params->aabb_min[k])) return niv_fail(NIV_ERR_ARG, "empty aabb");
    int rc = check_device(h);
    if (rc) return rc;
    if (h->infer_dirty) {
        rc = refresh_inference(h, (cudaStream_t)stream);
        if (rc) return rc;
    }
    const int32_t w = (full_width + sub - 1) / sub, hh = (full_height + sub - 1) / sub;
    GridArgs g = niv_grid_args(h, params);
    IoArgs io;
    io.pos = pos;
    io.nrm = nrm;
    io.out = out_E;
    io.n = (int64_t)w * hh;
    io.image_width = w;
    io.in_f16 = dtype_in == NIV_F16;
    io.out_f16 = dtype_out == NIV_F16;
    io.sub = sub;
    io.src_width = full_width;
    switch (precision) {
        case NIV_FP32: return niv_launch_query_fp32(h, g, io, (cudaStream_t)stream);
        case NIV_FP16: return niv_launch_query_tc(h, g, io, precision, (cudaStream_t)stream);
        case NIV_FP8: return niv_launch_query_f8(h, g, io, (cudaStream_t)stream);
        default: return niv_fail(NIV_ERR_UNSUPPORTED, "precision not supported");
    }
}

int niv_upsample_shade(const void* pos, const void* nrm, const void* albedo, const void* direct, int32_t full_width,
                       int32_t full_height, int32_t dtype_in, const void* E_low, int32_t dtype_E, int32_t sub,
                       const niv_upsample_params* up, void* out_rgba, niv_stream stream) {
    if (!up) return niv_fail(NIV_ERR_ARG, "upsample params are NULL");
    if (full_width < 0 || full_height < 0) return niv_fail(NIV_ERR_ARG, "negative image size");
    if (sub < 1) return niv_fail(NIV_ERR_ARG, "sub must be >= 1");
    if (full_width == 0 || full_height == 0) return NIV_OK;
    if (!(up->sigma > 0.0f) || !(up->eps > 0.0f) || !(up->power >= 0.0f))
        return niv_fail(NIV_ERR_ARG, "sigma and eps must be > 0, power >= 0");
    if (!pos || !nrm || !albedo || !direct || !E_low || !out_rgba) return niv_fail(NIV_ERR_ARG, "NULL record pointer");
    if (!aligned16(pos) || !aligned16(nrm) || !aligned16(albedo) || !aligned16(direct) || !aligned16(E_low) ||
        !aligned16(out_rgba))
        return niv_fail(NIV_ERR_ALIGN, "record pointers must be 16-byte aligned");
    if ((dtype_in != NIV_F32 && dtype_in != NIV_F16) || (dtype_E != NIV_F32 && dtype_E != NIV_F16))
        return niv_fail(NIV_ERR_ARG, "record dtype must be NIV_F32 or NIV_F16");
    return niv_launch_upsample_shade(pos, nrm, albedo, direct, full_width, full_height, dtype_in == NIV_F16, E_low,
                                     dtype_E == NIV_F16, sub, up->power, up->sigma, up->eps, out_rgba,
                                     (cudaStream_t)stream);
}

int niv_shade(const void* albedo, const void* direct, const void* E, int64_t n, void* out_rgba,
              niv_stream stream) {
    if (n < 0) return niv_fail(NIV_ERR_ARG, "n < 0");
    if (n == 0) return NIV_OK;
    if (!albedo || !direct || !E || !out_rgba) return niv_fail(NIV_ERR_ARG, "NULL record pointer");
    if (!aligned16(albedo) || !aligned16(direct) || !aligned16(E) || !aligned16(out_rgba))
        return niv_fail(NIV_ERR_ALIGN, "record pointers must be 16-byte aligned");
    return niv_launch_shade(albedo, direct, E, n, out_rgba, (cudaStream_t)stream);
}

}  // extern "C"

