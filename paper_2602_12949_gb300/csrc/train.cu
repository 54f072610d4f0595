// Training step of Sec. 4.5: relative-L2 loss (Eq. 3), hand-written backward pass and Adam.
//
// Three kernels per step, FP32 against the FP32 master parameters (optionally with the FP16
// forward of the query, see kModeF16Fwd):
//   1. fwd_bwd_kernel (one thread per sample): encoding and network forward, the loss
//      (E - y)^2 / (sg(E^2) + eps) averaged over samples and channels, and the backward
//      pass through softplus, the output layer and every ReLU layer down to the network
//      input; the encoding part of the input gradient is scattered into the grid-feature
//      gradients with atomicAdd (hash collisions add, as in the sum over corners).  Each
//      layer's input a_l and output gradient dz_l are stashed in scratch for step 2.
//   2. weight_grad_kernel: dW_l = sum_s dz_l[s] a_l[s]^T and db_l = sum_s dz_l[s], a
//      reduction over the batch in shared-memory tiles, one atomicAdd per entry per CTA.
//   3. adam_kernel: m, v and the parameters for every value (Kingma & Ba).
#include <math.h>

#include "niv_internal.cuh"

namespace {

constexpr int kT = 128;
constexpr int kMaxIn = 64;  // widest network input the training kernels take

__device__ __forceinline__ float sigmoidf(float z) { return 1.0f / (1.0f + expf(-z)); }

// fwd_bwd_kernel mode bits: the target records hold dL/dE (vector-Jacobian product, no
// loss); the output layer is the identity instead of softplus; the forward runs the FP16
// path of the query (grid values, weights and biases, the network input and the hidden
// activations rounded to binary16; FP32 sums), and the backward is the gradient of that
// function taken straight through the roundings, applied to the FP32 master parameters.
constexpr int kModeVjp = 1, kModeIdentityOut = 2, kModeF16Fwd = 4;

__device__ __forceinline__ float r16(float x) { return __half2float(__float2half_rn(x)); }

// Row stride (floats) of stashed layer inputs: n_in rounded up to 4, or W.
__host__ __device__ __forceinline__ int stash_stride(int k) { return (k + 3) & ~3; }

template <int DIMS, int F, int W>
__global__ void __launch_bounds__(kT) fwd_bwd_kernel(GridArgs g, const float4* __restrict__ pos,
                                                     const float4* __restrict__ nrm, const float* __restrict__ tsamp,
                                                     const float4* __restrict__ target, int64_t n,
                                                     const float* __restrict__ params, int64_t n_grid, int nh,
                                                     float eps, float inv_count, int mode, float* __restrict__ grad,
                                                     float* __restrict__ stash, double* __restrict__ loss_sum) {
    extern __shared__ float smem[];
    const int n_in = g.n_in, LG = g.levels * F, LF = LG + 6 * g.pe_bands;  // grid values, all encoding values
    // weights of every layer, row-major as stored: [W1 | b1 | W2 | b2 | ... | Wo | bo]
    const int n_mlp = W * n_in + W + (nh - 1) * (W * W + W) + 3 * W + 3;
    float* s_w = smem;
    float* s_a = smem + ((n_mlp + 3) & ~3);   // [kMaxIn][kT] current layer input, then scratch
    float* s_b = s_a + kMaxIn * kT;           // [W][kT] current layer output
    const bool f16 = mode & kModeF16Fwd;
    for (int i = threadIdx.x; i < n_mlp; i += kT) s_w[i] = f16 ? r16(params[n_grid + i]) : params[n_grid + i];
    __syncthreads();

    const int tid = threadIdx.x;
    const int64_t q = blockIdx.x * (int64_t)kT + tid;
    const bool valid = q < n;
    const int64_t qq = valid ? q : 0;
    const float4 p = pos[qq], nv = nrm[qq], y = target[qq];
    const float tq = tsamp ? tsamp[qq] : g.t;
    float u[4];
    u[0] = niv_unit(p.x, g.aabb_min[0], g.inv_ext[0]);
    u[1] = niv_unit(p.y, g.aabb_min[1], g.inv_ext[1]);
    u[2] = niv_unit(p.z, g.aabb_min[2], g.inv_ext[2]);
    u[3] = fminf(fmaxf(tq, 0.0f), 1.0f);

    // ---- forward: encoding ----
    for (int l = 0; l < g.levels; ++l) {
        float acc[F];
        if (f16) {  // grid values rounded as they are gathered
            constexpr int NC = 1 << DIMS;
            uint32_t e[NC];
            float wc[NC];
            niv_level_corners<DIMS>(g, l, u, e, wc);
            const float* tab = params + (size_t)g.offset[l] * F;
#pragma unroll
            for (int j = 0; j < F; ++j) acc[j] = 0.0f;
#pragma unroll
            for (int c = 0; c < NC; ++c)
#pragma unroll
                for (int j = 0; j < F; ++j) acc[j] = fmaf(wc[c], r16(tab[(size_t)e[c] * F + j]), acc[j]);
        } else {
            niv_encode_level<DIMS, F, float>(g, params, l, u, acc);
        }
#pragma unroll
        for (int j = 0; j < F; ++j) s_a[(l * F + j) * kT + tid] = f16 ? r16(acc[j]) : acc[j];
    }
    for (int d = 0; d < 3 && g.pe_bands > 0; ++d)
        for (int b = 0; b < g.pe_bands; ++b) {
            float sv, cv;
            niv_pe_pair(u[d], b, sv, cv);
            s_a[(LG + 2 * (d * g.pe_bands + b)) * kT + tid] = f16 ? r16(sv) : sv;
            s_a[(LG + 2 * (d * g.pe_bands + b) + 1) * kT + tid] = f16 ? r16(cv) : cv;
        }
    s_a[(LF + 0) * kT + tid] = f16 ? r16(nv.x) : nv.x;
    s_a[(LF + 1) * kT + tid] = f16 ? r16(nv.y) : nv.y;
    s_a[(LF + 2) * kT + tid] = f16 ? r16(nv.z) : nv.z;
    if (g.t_bands > 0) {  // Sec. 6: the scene parameter frequency-encoded after n
        for (int b = 0; b < g.t_bands; ++b) {
            float sv, cv;
            niv_pe_pair(u[3], b, sv, cv);
            s_a[(LF + 3 + 2 * b) * kT + tid] = f16 ? r16(sv) : sv;
            s_a[(LF + 4 + 2 * b) * kT + tid] = f16 ? r16(cv) : cv;
        }
    } else if (n_in > LF + 3) {
        s_a[(LF + 3) * kT + tid] = f16 ? r16(u[3]) : u[3];
    }

    // stash layout per layer l (input of matrix l): [n][stride_l]; then dz_l: [n][W or 4]
    float* st = stash;
    const int64_t nn = n;
    // ---- forward: hidden layers; stash every matrix input ----
    const float* w = s_w;
    int k_in = n_in;
    for (int layer = 0; layer < nh; ++layer) {
        const int sk = stash_stride(k_in);
        if (valid)
            for (int i = 0; i < k_in; ++i) st[qq * sk + i] = s_a[i * kT + tid];
        st += nn * sk;
        const float* bl = w + W * k_in;
        for (int o = 0; o < W; ++o) {
            float z = bl[o];
            for (int i = 0; i < k_in; ++i) z = fmaf(w[o * k_in + i], s_a[i * kT + tid], z);
            s_b[o * kT + tid] = f16 ? r16(fmaxf(z, 0.0f)) : fmaxf(z, 0.0f);
        }
        for (int o = 0; o < W; ++o) s_a[o * kT + tid] = s_b[o * kT + tid];
        w = bl + W;
        k_in = W;
    }
    {   // input of the output layer
        if (valid)
            for (int i = 0; i < W; ++i) st[qq * W + i] = s_a[i * kT + tid];
        st += nn * W;
    }
    // ---- output layer, softplus, loss, dLoss/dz ----
    const float* wo = w;
    const float* bo = wo + 3 * W;
    float z[3] = {bo[0], bo[1], bo[2]};
    for (int i = 0; i < W; ++i) {
        const float a = s_a[i * kT + tid];
        z[0] = fmaf(wo[i], a, z[0]);
        z[1] = fmaf(wo[W + i], a, z[1]);
        z[2] = fmaf(wo[2 * W + i], a, z[2]);
    }
    const float yy[3] = {y.x, y.y, y.z};
    const bool vjp = mode & kModeVjp, soft = !(mode & kModeIdentityOut);
    float dz[3];
    double lsum = 0.0;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float act = soft ? sigmoidf(z[c]) : 1.0f;  // d E / d z
        if (vjp) {  // the record holds dL/dE from the caller
            dz[c] = valid ? yy[c] * act : 0.0f;
        } else {
            const float E = soft ? niv_softplus(z[c]) : z[c];
            const float den = E * E + eps;  // held constant (stop-gradient)
            const float diff = E - yy[c];
            lsum += (double)(diff * diff / den);
            dz[c] = valid ? 2.0f * diff / den * inv_count * act : 0.0f;
        }
    }
    if (!valid) lsum = 0.0;
    // block reduction of the loss
    for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xFFFFFFFFu, lsum, o);
    if ((tid & 31) == 0) atomicAdd(loss_sum, lsum);

    // stash dz of the output layer: [n][4]
    float* dz_out = st;
    if (valid) reinterpret_cast<float4*>(dz_out)[qq] = make_float4(dz[0], dz[1], dz[2], 0.0f);
    st += nn * 4;

    // ---- backward: gradient w.r.t. the last hidden output ----
    for (int i = 0; i < W; ++i) {
        const float a = s_a[i * kT + tid];
        const float gsum = wo[i] * dz[0] + wo[W + i] * dz[1] + wo[2 * W + i] * dz[2];
        s_b[i * kT + tid] = a > 0.0f ? gsum : 0.0f;  // dz of the last hidden layer (ReLU'(0) = 0)
    }
    // dz stash of hidden layers is laid out from the last layer down: [n][W] each
    const float* wl_end = wo;  // walk the weight blocks backwards
    for (int layer = nh - 1; layer >= 0; --layer) {
        const int kl = layer == 0 ? n_in : W;
        const float* wl = wl_end - (W * kl + W);  // W_layer, followed by its bias
        if (valid)
            for (int o = 0; o < W; ++o) st[qq * W + o] = s_b[o * kT + tid];
        st += nn * W;
        // input of this layer, re-read from the stash written in the forward pass
        const float* a_in = stash;
        for (int ll = 0; ll < layer; ++ll) a_in += nn * stash_stride(ll == 0 ? n_in : W);
        const int sk = stash_stride(kl);
        for (int i = 0; i < kl; ++i) {
            float gsum = 0.0f;
            for (int o = 0; o < W; ++o) gsum = fmaf(wl[o * kl + i], s_b[o * kT + tid], gsum);
            const float a = valid ? a_in[qq * sk + i] : 0.0f;
            s_a[i * kT + tid] = (layer == 0 || a > 0.0f) ? gsum : 0.0f;
        }
        for (int i = 0; i < kl && layer > 0; ++i) s_b[i * kT + tid] = s_a[i * kT + tid];
        wl_end = wl;
    }
    // s_a now holds dLoss/dx for the network input; scatter the encoding part
    if (valid) {
        for (int l = 0; l < g.levels; ++l) {
            uint32_t e[1 << DIMS];
            float wc[1 << DIMS];
            niv_level_corners<DIMS>(g, l, u, e, wc);
            float* gl = grad + (size_t)g.offset[l] * F;
#pragma unroll
            for (int c = 0; c < (1 << DIMS); ++c)
#pragma unroll
                for (int j = 0; j < F; ++j) atomicAdd(gl + (size_t)e[c] * F + j, wc[c] * s_a[(l * F + j) * kT + tid]);
        }
    }
}

// dW[o][i] (+)= sum_s D[s][o] A[s][i] for i < k_in, and db[o] (+)= sum_s D[s][o] at column k_in.
// D: [n][ds] (row stride ds), A: [n][as].  Each CTA reduces a slice of samples.
constexpr int kWG_S = 32;  // samples per shared-memory tile
__global__ void __launch_bounds__(256) weight_grad_kernel(const float* __restrict__ D, int ds, const float* __restrict__ A,
                                                          int as, int64_t n, int n_out, int k_in, int64_t per_cta,
                                                          float* __restrict__ dW, float* __restrict__ db) {
    __shared__ float sD[kWG_S][64];
    __shared__ float sA[kWG_S][kMaxIn + 1];
    const int tid = threadIdx.x;
    const int entries = n_out * (k_in + 1);
    float acc[17];
#pragma unroll
    for (int r = 0; r < 17; ++r) acc[r] = 0.0f;
    const int64_t s0 = blockIdx.x * per_cta, s1 = min(n, s0 + per_cta);
    for (int64_t base = s0; base < s1; base += kWG_S) {
        for (int idx = tid; idx < kWG_S * 64; idx += 256) {
            const int s = idx / 64, c = idx % 64;
            const int64_t row = base + s;
            sD[s][c] = (row < s1 && c < n_out) ? D[row * ds + c] : 0.0f;
        }
        for (int idx = tid; idx < kWG_S * (kMaxIn + 1); idx += 256) {
            const int s = idx / (kMaxIn + 1), c = idx % (kMaxIn + 1);
            const int64_t row = base + s;
            sA[s][c] = (row < s1 && c < k_in) ? A[row * as + c] : (c == k_in && row < s1 ? 1.0f : 0.0f);
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < 17; ++r) {
            const int e = tid + r * 256;
            if (e < entries) {
                const int o = e / (k_in + 1), i = e % (k_in + 1);
                float a = acc[r];
                for (int s = 0; s < kWG_S; ++s) a = fmaf(sD[s][o], sA[s][i], a);
                acc[r] = a;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int r = 0; r < 17; ++r) {
        const int e = tid + r * 256;
        if (e < entries) {
            const int o = e / (k_in + 1), i = e % (k_in + 1);
            if (i < k_in) atomicAdd(dW + (size_t)o * k_in + i, acc[r]);
            else atomicAdd(db + o, acc[r]);
        }
    }
}

__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                            const float* __restrict__ g, int64_t n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = g[i];
        const float mi = b1 * m[i] + (1.0f - b1) * gi;
        const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        theta[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

template <int DIMS, int F, int W>
int launch_fwd_bwd(niv_model* m, const GridArgs& g, const float4* pos, const float4* nrm, const float* t,
                   const float4* target, int64_t n, float eps, int mode, cudaStream_t s) {
    auto kern = fwd_bwd_kernel<DIMS, F, W>;
    const int nh = m->d.n_hidden;
    const size_t smem = (size_t)(((m->n_mlp + 3) & ~3) + kMaxIn * kT + W * kT) * sizeof(float);
    NIV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    NIV_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared));
    const unsigned blocks = (unsigned)((n + kT - 1) / kT);
    kern<<<blocks, kT, smem, s>>>(g, pos, nrm, t, target, n, m->params, m->n_grid, nh, eps, 1.0f / (3.0f * (float)n),
                                  mode | (m->d.out_act == 1 ? 0 : kModeIdentityOut), m->grad, m->stash, m->loss_acc);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}

template <int DIMS, int F>
int by_width(niv_model* m, const GridArgs& g, const float4* pos, const float4* nrm, const float* t,
             const float4* target, int64_t n, float eps, int mode, cudaStream_t s) {
    switch (m->d.width) {
        case 16: return launch_fwd_bwd<DIMS, F, 16>(m, g, pos, nrm, t, target, n, eps, mode, s);
        case 32: return launch_fwd_bwd<DIMS, F, 32>(m, g, pos, nrm, t, target, n, eps, mode, s);
        case 64: return launch_fwd_bwd<DIMS, F, 64>(m, g, pos, nrm, t, target, n, eps, mode, s);
    }
    return niv_fail(NIV_ERR_UNSUPPORTED, "width must be 16, 32 or 64");
}

}  // namespace

// Size in floats of the per-step scratch for n samples.
int64_t niv_train_stash_floats(const niv_model* m, int64_t n) {
    const int W = m->d.width, nh = m->d.n_hidden;
    int64_t per = stash_stride(m->n_in) + (int64_t)(nh - 1) * W + W  // inputs of every matrix
                  + 4 + (int64_t)nh * W;                             // dz of the output and hidden layers
    return per * n;
}

int niv_train_grad(niv_model* m, const GridArgs& g, const float4* pos, const float4* nrm, const float* t,
                   const float4* target, int64_t n, float eps, bool vjp, cudaStream_t s) {
    const int mode = (vjp ? kModeVjp : 0) | (m->train_f16 ? kModeF16Fwd : 0);
    const int W = m->d.width, nh = m->d.n_hidden, n_in = m->n_in;
    if (n_in > kMaxIn) return niv_fail(NIV_ERR_UNSUPPORTED, "training needs a network input of <= 64 values");
    const int64_t need = niv_train_stash_floats(m, n);
    if (m->stash_floats < need) {
        NIV_CUDA(cudaStreamSynchronize(s));
        cudaFree(m->stash);
        m->stash = nullptr;
        m->stash_floats = 0;
        NIV_CUDA(cudaMalloc(&m->stash, sizeof(float) * need));
        m->stash_floats = need;
    }
    NIV_CUDA(cudaMemsetAsync(m->grad, 0, sizeof(float) * (m->n_grid + m->n_mlp), s));
    NIV_CUDA(cudaMemsetAsync(m->loss_acc, 0, sizeof(double), s));
    int rc;
    if (m->d.dims == 4) {
        switch (m->d.feat) {
            case 1: rc = by_width<4, 1>(m, g, pos, nrm, t, target, n, eps, mode, s); break;
            case 2: rc = by_width<4, 2>(m, g, pos, nrm, t, target, n, eps, mode, s); break;
            default: rc = by_width<4, 4>(m, g, pos, nrm, t, target, n, eps, mode, s); break;
        }
    } else {
        switch (m->d.feat) {
            case 1: rc = by_width<3, 1>(m, g, pos, nrm, t, target, n, eps, mode, s); break;
            case 2: rc = by_width<3, 2>(m, g, pos, nrm, t, target, n, eps, mode, s); break;
            default: rc = by_width<3, 4>(m, g, pos, nrm, t, target, n, eps, mode, s); break;
        }
    }
    if (rc) return rc;
    // weight gradients, layer by layer; the stash holds the matrix inputs (first layer to the
    // output layer), then dz of the output layer [n][4], then dz of the hidden layers from the
    // last one down to the first.
    int sms = 0, dev = 0;
    NIV_CUDA(cudaGetDevice(&dev));
    NIV_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int64_t ctas = (int64_t)sms * 4;
    int64_t per_cta = (n + ctas - 1) / ctas;
    per_cta = (per_cta + kWG_S - 1) / kWG_S * kWG_S;
    ctas = (n + per_cta - 1) / per_cta;
    const float* a_ptr[8];
    int a_stride[8];
    const float* p = m->stash;
    for (int l = 0; l <= nh; ++l) {
        const int k = l == 0 ? n_in : W;
        a_ptr[l] = p;
        a_stride[l] = stash_stride(k);
        p += n * stash_stride(k);
    }
    const float* dz_out = p;
    p += n * 4;
    const float* dz_h[8];
    for (int l = nh - 1; l >= 0; --l) {
        dz_h[l] = p;
        p += n * W;
    }
    float* gW = m->grad + m->n_grid;
    for (int l = 0; l <= nh; ++l) {
        const int k = l == 0 ? n_in : W;
        const int n_out = l == nh ? 3 : W;
        const float* D = l == nh ? dz_out : dz_h[l];
        const int ds = l == nh ? 4 : W;
        weight_grad_kernel<<<(unsigned)ctas, 256, 0, s>>>(D, ds, a_ptr[l], a_stride[l], n, n_out, k, per_cta, gW,
                                                          gW + (size_t)n_out * k);
        NIV_CUDA(cudaGetLastError());
        gW += (size_t)n_out * k + n_out;
    }
    return NIV_OK;
}

int niv_train_adam(niv_model* m, float lr, float b1, float b2, float eps, cudaStream_t s) {
    m->adam_step += 1;
    const double c1 = 1.0 - pow((double)b1, (double)m->adam_step);
    const double c2 = 1.0 - pow((double)b2, (double)m->adam_step);
    const int64_t n = m->n_grid + m->n_mlp;
    int64_t blocks = (n + 255) / 256;
    if (blocks > 8192) blocks = 8192;
    adam_kernel<<<(unsigned)blocks, 256, 0, s>>>(m->params, m->adam_m, m->adam_v, m->grad, n, lr, b1, b2, eps,
                                                  (float)c1, (float)c2);
    NIV_CUDA(cudaGetLastError());
    m->infer_dirty = 1;
    return NIV_OK;
}
