/*
 * CPU FP64 oracle of the Neural Irradiance Volume query, its loss and its gradient.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the benchmark's
 * CPU-baseline / reference leg may load this code.  It shares no source with
 * the CUDA library; the two meet only through the seeded inputs of niv_inputs.
 *
 * Every function follows the paper's description step by step, in plain loops:
 *  - Sec. 4.1 (multi-level hash-grid encoding of Mueller et al. 2022, which the
 *    paper adopts): per level a resolution N_l = floor(base * growth^l); dense
 *    storage of the (N_l+1)^d vertices when that fits in T entries, otherwise the
 *    spatial hash  (XOR_k v_k * pi_k) mod T  with pi = (1, 2654435761, 805459861);
 *    multilinear interpolation of the F features stored at the 2^d cell corners.
 *  - Sec. 4.1 / Table 1: the smaller models replace the grid by an eight-band
 *    frequency (positional) encoding of the position (Mildenhall et al. 2020):
 *    sin(2^k pi u_d) and cos(2^k pi u_d), k = 0..B-1, for each coordinate d;
 *  - Sec. 4.1: a fully connected network with ReLU on all but the final layer,
 *    mapping (encoded position, direction) to irradiance; the final activation is
 *    softplus (keeps E >= 0).
 *  - Eq. 3 (Sec. 4.5): relative L2 loss (E_theta - E)^2 / (sg(E_theta^2) + eps).
 *  - Sec. 4.5: Adam.
 *
 * Readings where the paper is silent (also listed in the design notes):
 *  - position normalisation u = (p - aabb_min) * inv_extent, clamped to [0,1],
 *    each step an FP32 operation (so that grid indices are well defined); here
 *    emulated exactly by rounding FP64 results of FP32 operands to float;
 *  - s = u * N_l (FP32 product), i = min(floor(s), N_l - 1), w = s - i, vertices
 *    at integer coordinates 0..N_l (no half-cell offset);
 *  - 4th (time) grid dimension hashed with a caller-chosen odd constant;
 *  - network input = [level 0 features, ..., level L-1 features, n.xyz, (t)];
 *  - frequency encoding of the normalised coordinate u in [0, 1], no identity term,
 *    ordered per coordinate, then per band, sin before cos; it follows the grid
 *    features in the network input (a model has one or the other).
 *
 * Parity status: every function here is pinned by tests (closed forms, brute
 * force, library special cases, finite differences).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_LEVELS 32
#define ORC_MAX_DIMS 4
#define ORC_MAX_LAYERS 8
#define ORC_MAX_WIDTH 256
#define ORC_MAX_BANDS 16
#define ORC_MAX_ENC (ORC_MAX_LEVELS * 8 + 6 * ORC_MAX_BANDS) /* encoding values of one query */

typedef struct {
    int32_t dims;      /* 3 (x,y,z) or 4 (x,y,z,t) */
    int32_t levels;    /* L */
    int32_t feat;      /* F features per table entry */
    int32_t log2_T;    /* hashed table size T = 2^log2_T */
    double base;       /* N_0 */
    double growth;     /* per-level scale */
    int32_t n_hidden;  /* hidden layers */
    int32_t width;     /* hidden width */
    int32_t in_extra;  /* raw inputs after the encoding: 3 (normal) or 4 (normal, t) */
    int32_t out_dim;   /* 3 */
    int32_t out_act;   /* 0 identity, 1 softplus */
    uint32_t prime_t;  /* hash constant of the 4th dimension */
    int32_t pe_bands;  /* > 0: frequency encoding of the position with that many bands (levels may be 0) */
    int32_t t_bands;   /* > 0: the scene parameter enters as sin / cos of 2^b pi t after n (Sec. 6) */
} orc_desc;

typedef struct {
    int32_t res[ORC_MAX_LEVELS];
    int32_t dense[ORC_MAX_LEVELS];
    int64_t offset[ORC_MAX_LEVELS]; /* first entry of the level */
    int64_t entries[ORC_MAX_LEVELS];
    int64_t total;                  /* entries over all levels */
} orc_layout_t;

/* threads the oracle's parallel loops use (1 without OpenMP) */
int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the following parallel loops (timing on a given number of host cores). */
void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

static const uint32_t ORC_PI[3] = {1u, 2654435761u, 805459861u};

/* ---- FP32 operations emulated in FP64 (exact: operands are floats) ---- */
static float f32_sub(float a, float b) { return (float)((double)a - (double)b); }
static float f32_mul(float a, float b) { return (float)((double)a * (double)b); }

/* ---- level layout (Sec. 4.1) ---- */
int64_t orc_layout(const orc_desc* d, int32_t* res, int32_t* dense, int64_t* offset, int64_t* entries)
{
    if (d->levels < 0 || d->levels > ORC_MAX_LEVELS || d->dims < 3 || d->dims > ORC_MAX_DIMS) return -1;
    if (d->pe_bands < 0 || d->pe_bands > ORC_MAX_BANDS || (d->levels == 0 && d->pe_bands == 0)) return -1;
    const int64_t T = (int64_t)1 << d->log2_T;
    int64_t off = 0;
    for (int l = 0; l < d->levels; ++l) {
        int32_t N = (int32_t)floor(d->base * pow(d->growth, (double)l));
        int64_t verts = 1;
        for (int k = 0; k < d->dims; ++k) verts *= (int64_t)(N + 1);
        int is_dense = verts <= T;
        if (res) res[l] = N;
        if (dense) dense[l] = is_dense;
        if (offset) offset[l] = off;
        if (entries) entries[l] = is_dense ? verts : T;
        off += is_dense ? verts : T;
    }
    return off;
}

static int fill_layout(const orc_desc* d, orc_layout_t* L)
{
    L->total = orc_layout(d, L->res, L->dense, L->offset, L->entries);
    return L->total < 0 ? -1 : 0;
}

/* index of vertex v in level l (dense row-major with x fastest, or spatial hash) */
static int64_t vertex_index(const orc_desc* d, const orc_layout_t* L, int l, const int64_t* v)
{
    if (L->dense[l]) {
        int64_t stride = 1, idx = 0;
        for (int k = 0; k < d->dims; ++k) { idx += v[k] * stride; stride *= (int64_t)(L->res[l] + 1); }
        return idx;
    }
    uint32_t h = 0;
    for (int k = 0; k < d->dims; ++k) {
        uint32_t p = k < 3 ? ORC_PI[k] : d->prime_t;
        h ^= (uint32_t)v[k] * p; /* product mod 2^32 */
    }
    return (int64_t)(h & (uint32_t)(((uint64_t)1 << d->log2_T) - 1));
}

/* normalised grid coordinate of one query (FP32 operations, emulated exactly) */
static void normalise(const orc_desc* d, const float* p, const float* aabb_min, const float* aabb_max,
                      float t, float* u)
{
    for (int k = 0; k < 3; ++k) {
        float inv = (float)(1.0 / ((double)aabb_max[k] - (double)aabb_min[k]));
        float x = f32_mul(f32_sub(p[k], aabb_min[k]), inv);
        u[k] = x < 0.0f ? 0.0f : (x > 1.0f ? 1.0f : x);
    }
    if (d->dims == 4) u[3] = t < 0.0f ? 0.0f : (t > 1.0f ? 1.0f : t);
}

/* per-level cell and weights: s = u*N (FP32), i = min(floor(s), N-1), w = s - i */
static void cell_of(const orc_desc* d, int32_t N, const float* u, int64_t* i, double* w)
{
    for (int k = 0; k < d->dims; ++k) {
        float s = f32_mul(u[k], (float)N);
        int64_t ik = (int64_t)floor((double)s);
        if (ik > N - 1) ik = N - 1;
        i[k] = ik;
        w[k] = (double)s - (double)ik;
    }
}

/*
 * Encoding of one query.  enc[l*F + j] = sum over the 2^d corners c of
 * prod_k (c_k ? w_k : 1 - w_k) * table_l[index(i + c)][j].
 * Optionally records the corner indices (level-major, corner-minor) and weights.
 */
static void encode_point(const orc_desc* d, const orc_layout_t* L, const double* grid, const float* u,
                         double* enc, int64_t* idx_out, double* w_out)
{
    const int F = d->feat, nc = 1 << d->dims;
    for (int l = 0; l < d->levels; ++l) {
        int64_t i[ORC_MAX_DIMS];
        double w[ORC_MAX_DIMS];
        cell_of(d, L->res[l], u, i, w);
        for (int j = 0; j < F; ++j) enc[l * F + j] = 0.0;
        for (int c = 0; c < nc; ++c) {
            int64_t v[ORC_MAX_DIMS];
            double wc = 1.0;
            for (int k = 0; k < d->dims; ++k) {
                int bit = (c >> k) & 1;
                v[k] = i[k] + bit;
                wc *= bit ? w[k] : 1.0 - w[k];
            }
            int64_t e = vertex_index(d, L, l, v);
            for (int j = 0; j < F; ++j) enc[l * F + j] += wc * grid[(L->offset[l] + e) * F + j];
            if (idx_out) idx_out[l * nc + c] = e;
            if (w_out) w_out[l * nc + c] = wc;
        }
    }
    /* frequency encoding: sin / cos of 2^b * pi * u_k (the FP32 u taken exactly) */
    double* pe = enc + d->levels * F;
    for (int k = 0; k < 3; ++k)
        for (int b = 0; b < d->pe_bands; ++b) {
            double a = M_PI * ldexp((double)u[k], b);
            pe[(k * d->pe_bands + b) * 2 + 0] = sin(a);
            pe[(k * d->pe_bands + b) * 2 + 1] = cos(a);
        }
}

/* encoding values of one query: grid features, then frequency-encoding values */
int orc_enc_dim(const orc_desc* d) { return d->levels * d->feat + 6 * d->pe_bands; }

int orc_net_inputs(const orc_desc* d) { return orc_enc_dim(d) + d->in_extra + 2 * d->t_bands; }

/* number of network parameters (all layers, weights and biases) */
int64_t orc_mlp_param_count(const orc_desc* d)
{
    int64_t n = 0, k = orc_net_inputs(d);
    for (int h = 0; h < d->n_hidden; ++h) { n += (int64_t)d->width * k + d->width; k = d->width; }
    n += (int64_t)d->out_dim * k + d->out_dim;
    return n;
}

static double softplus(double z) { return (z > 0.0 ? z : 0.0) + log1p(exp(-fabs(z))); }
static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

double orc_f16(double x);

/*
 * Network forward for one input vector x (length n_in).  Stores every layer's
 * pre-activation z_k (layer-major) and post-activation a_k when requested.
 * Returns E (out_dim values).  f16: every hidden activation is rounded to binary16.
 */
static void mlp_forward(const orc_desc* d, const double* mlp, const double* x, double* z_all, double* a_all,
                        double* E, int f16)
{
    double buf_a[ORC_MAX_WIDTH], buf_b[ORC_MAX_WIDTH];
    const double* in = x;
    int k_in = orc_net_inputs(d);
    const double* p = mlp;
    int layers = d->n_hidden + 1;
    for (int layer = 0; layer < layers; ++layer) {
        int last = layer == layers - 1;
        int n_out = last ? d->out_dim : d->width;
        const double* W = p;
        const double* b = p + (int64_t)n_out * k_in;
        double* out = (layer & 1) ? buf_b : buf_a;
        for (int o = 0; o < n_out; ++o) {
            double z = b[o];
            for (int i = 0; i < k_in; ++i) z += W[(int64_t)o * k_in + i] * in[i];
            if (z_all) z_all[layer * ORC_MAX_WIDTH + o] = z;
            double a;
            if (!last) a = f16 ? orc_f16(z > 0.0 ? z : 0.0) : (z > 0.0 ? z : 0.0); /* ReLU */
            else a = d->out_act == 1 ? softplus(z) : z;         /* final layer */
            out[o] = a;
            if (a_all) a_all[layer * ORC_MAX_WIDTH + o] = a;
            if (last) E[o] = a;
        }
        p = b + n_out;
        in = out;
        k_in = n_out;
    }
}

/* assemble the network input of one query: [encoding, n.xyz, (t or its frequency encoding)] */
static void net_input(const orc_desc* d, const double* enc, const float* nrm, float t, double* x)
{
    int ne = orc_enc_dim(d);
    for (int i = 0; i < ne; ++i) x[i] = enc[i];
    x[ne + 0] = nrm[0];
    x[ne + 1] = nrm[1];
    x[ne + 2] = nrm[2];
    /* the scene parameter enters clamped to [0, 1], as it does the grid's 4th axis; with
     * t_bands > 0 (Sec. 6) as the pairs sin, cos of 2^b pi t instead */
    const double tc = t < 0.0f ? 0.0 : (t > 1.0f ? 1.0 : (double)t);
    if (d->in_extra == 4) x[ne + 3] = tc;
    for (int b = 0; b < d->t_bands; ++b) {
        x[ne + 3 + 2 * b] = sin(M_PI * ldexp(tc, b));
        x[ne + 4 + 2 * b] = cos(M_PI * ldexp(tc, b));
    }
}

/*
 * Encoding only: enc[n][L*F + 6*B] (grid features, then frequency encoding).  Optionally the corner indices idx[n][L][2^d]
 * (uint32) and corner weights w[n][L][2^d].
 */
int orc_encode(const orc_desc* d, const double* grid, const float* pos4, int64_t n, const float* aabb_min,
               const float* aabb_max, float t, double* enc, uint32_t* idx, double* wts)
{
    orc_layout_t L;
    if (fill_layout(d, &L)) return -1;
    const int nc = 1 << d->dims, ne = orc_enc_dim(d);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) {
        float u[ORC_MAX_DIMS];
        int64_t ix[ORC_MAX_LEVELS * 16];
        double wc[ORC_MAX_LEVELS * 16];
        normalise(d, pos4 + 4 * q, aabb_min, aabb_max, t, u);
        encode_point(d, &L, grid, u, enc + q * ne, ix, wc);
        for (int e = 0; e < d->levels * nc; ++e) {
            if (idx) idx[q * d->levels * nc + e] = (uint32_t)ix[e];
            if (wts) wts[q * d->levels * nc + e] = wc[e];
        }
    }
    return 0;
}

/* network only: x[n][n_in] -> E[n][out_dim] */
int orc_mlp(const orc_desc* d, const double* mlp, const double* x, int64_t n, double* E)
{
    const int n_in = orc_net_inputs(d);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) mlp_forward(d, mlp, x + q * n_in, NULL, NULL, E + q * d->out_dim, 0);
    return 0;
}

/*
 * Full query (Sec. 4.4): G-buffer position and normal -> E(x, n).
 * params = [grid values | network parameters] in FP64; pos4/nrm4 are [n][4] FP32
 * records (FP16 G-buffers are widened exactly by the caller); t is the scene
 * parameter of a 4-D model (ignored otherwise); out E[n][out_dim].
 */
int orc_query(const orc_desc* d, const double* params, const float* pos4, const float* nrm4, int64_t n,
              const float* aabb_min, const float* aabb_max, float t, double* E)
{
    orc_layout_t L;
    if (fill_layout(d, &L)) return -1;
    const double* mlp = params + L.total * d->feat;
    const int n_in = orc_net_inputs(d);
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) {
        float u[ORC_MAX_DIMS];
        double enc[ORC_MAX_ENC], x[ORC_MAX_ENC + 8];
        normalise(d, pos4 + 4 * q, aabb_min, aabb_max, t, u);
        encode_point(d, &L, params, u, enc, NULL, NULL);
        net_input(d, enc, nrm4 + 4 * q, t, x);
        (void)n_in;
        mlp_forward(d, mlp, x, NULL, NULL, E + q * d->out_dim, 0);
    }
    return 0;
}

/*
 * Loss (Eq. 3, mean over samples and channels, eps = 0.01 unless given) and its
 * gradient with respect to every parameter, by reverse-mode differentiation of
 * the steps above.  The denominator is a constant (stop-gradient).  ReLU'(0) = 0.
 * Grid gradients sum over corners and samples (hash collisions add).
 * t4 (nullable) gives a per-sample time input for 4-D models.
 * f16: the forward is the FP16 path (the caller passes parameters already rounded to
 * binary16; the network input and the hidden activations are rounded here) and the
 * gradient is taken straight through the roundings.  The ReLU derivative is 1 where the
 * stored activation is positive.
 * grad must hold as many values as params and is overwritten.
 */
int orc_loss_grad(const orc_desc* d, const double* params, const float* pos4, const float* nrm4,
                  const float* t_per_sample, const double* target, int64_t n, const float* aabb_min,
                  const float* aabb_max, double eps, double* loss_out, double* grad, int f16)
{
    orc_layout_t L;
    if (fill_layout(d, &L)) return -1;
    const int F = d->feat, nc = 1 << d->dims, C = d->out_dim, layers = d->n_hidden + 1;
    const int n_in = orc_net_inputs(d);
    const int64_t n_grid = L.total * F;
    const int64_t n_mlp = orc_mlp_param_count(d);
    const double* mlp = params + n_grid;
    memset(grad, 0, sizeof(double) * (size_t)(n_grid + n_mlp));
    double loss = 0.0;
    double* z_all = (double*)malloc(sizeof(double) * ORC_MAX_LAYERS * ORC_MAX_WIDTH);
    double* a_all = (double*)malloc(sizeof(double) * ORC_MAX_LAYERS * ORC_MAX_WIDTH);
    for (int64_t q = 0; q < n; ++q) {
        float u[ORC_MAX_DIMS];
        double enc[ORC_MAX_ENC], x[ORC_MAX_ENC + 8], E[8];
        int64_t ix[ORC_MAX_LEVELS * 16];
        double wc[ORC_MAX_LEVELS * 16];
        float tq = t_per_sample ? t_per_sample[q] : 0.0f;
        normalise(d, pos4 + 4 * q, aabb_min, aabb_max, tq, u);
        encode_point(d, &L, params, u, enc, ix, wc);
        net_input(d, enc, nrm4 + 4 * q, tq, x);
        if (f16)
            for (int i = 0; i < n_in; ++i) x[i] = orc_f16(x[i]);
        mlp_forward(d, mlp, x, z_all, a_all, E, f16);
        /* dLoss/dE with the denominator held constant */
        double g_out[ORC_MAX_WIDTH], g_in[ORC_MAX_WIDTH + ORC_MAX_ENC];
        for (int c = 0; c < C; ++c) {
            double y = target[q * C + c];
            double den = E[c] * E[c] + eps;
            loss += (E[c] - y) * (E[c] - y) / den;
            double dE = 2.0 * (E[c] - y) / den / ((double)n * C);
            double z = z_all[(layers - 1) * ORC_MAX_WIDTH + c];
            g_out[c] = d->out_act == 1 ? dE * sigmoid(z) : dE;
        }
        /* walk the layers backwards; parameter offsets recomputed per layer */
        for (int layer = layers - 1; layer >= 0; --layer) {
            int k_in = layer == 0 ? n_in : d->width;
            int n_out = layer == layers - 1 ? C : d->width;
            int64_t off = 0;
            for (int ll = 0, kk = n_in; ll < layer; ++ll) { off += (int64_t)d->width * kk + d->width; kk = d->width; }
            const double* W = mlp + off;
            double* gW = grad + n_grid + off;
            double* gb = gW + (int64_t)n_out * k_in;
            const double* in = layer == 0 ? x : a_all + (layer - 1) * ORC_MAX_WIDTH;
            for (int o = 0; o < n_out; ++o) {
                gb[o] += g_out[o];
                for (int i = 0; i < k_in; ++i) gW[(int64_t)o * k_in + i] += g_out[o] * in[i];
            }
            for (int i = 0; i < k_in; ++i) {
                double s = 0.0;
                for (int o = 0; o < n_out; ++o) s += W[(int64_t)o * k_in + i] * g_out[o];
                g_in[i] = s;
            }
            if (layer > 0) { /* through the ReLU of the layer below */
                for (int i = 0; i < k_in; ++i)
                    g_out[i] = a_all[(layer - 1) * ORC_MAX_WIDTH + i] > 0.0 ? g_in[i] : 0.0;
            }
        }
        /* g_in now holds dLoss/dx; scatter the encoding part into the tables */
        for (int l = 0; l < d->levels; ++l)
            for (int c = 0; c < nc; ++c)
                for (int j = 0; j < F; ++j)
                    grad[(L.offset[l] + ix[l * nc + c]) * F + j] += wc[l * nc + c] * g_in[l * F + j];
    }
    free(z_all);
    free(a_all);
    *loss_out = loss / ((double)n * C);
    return 0;
}

/*
 * One Adam step (Kingma & Ba 2014; Sec. 4.5 uses Adam) on every parameter:
 * m = b1 m + (1-b1) g;  v = b2 v + (1-b2) g^2;
 * theta -= lr * (m / (1-b1^step)) / (sqrt(v / (1-b2^step)) + eps).
 * step counts from 1.
 */
void orc_adam(double* theta, double* m, double* v, const double* g, int64_t n, double lr, double b1,
              double b2, double eps, int64_t step)
{
    double c1 = 1.0 - pow(b1, (double)step), c2 = 1.0 - pow(b2, (double)step);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * g[i];
        v[i] = b2 * v[i] + (1.0 - b2) * g[i] * g[i];
        theta[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}

/* Diffuse shading (Eq. 2 plus direct light): rgb = albedo * E / pi + direct. */
void orc_shade(const double* albedo3, const double* E3, const double* direct3, int64_t n, double* out3)
{
    for (int64_t i = 0; i < 3 * n; ++i) out3[i] = albedo3[i] * E3[i] / M_PI + direct3[i];
}

/*
 * Half-resolution rendering (Sec. 4.4): irradiance queried at every s-th pixel of
 * every s-th row, brought back to full resolution by joint bilateral upsampling
 * (Kopf et al. 2007, the practice the paper points to) guided by the full-
 * resolution G-buffer, then shaded with the full-resolution albedo.  Reading:
 *   low-resolution sample q = (i, j), i < w = ceil(W / s), j < h = ceil(H / s),
 *   holds E queried at full-resolution pixel (s i, s j);
 *   pixel p = (X, Y): i0 = floor(X / s), fx = X / s - i0, i1 = min(i0 + 1, w - 1),
 *   likewise j0, fy, j1; the four samples carry bilinear weights b_q;
 *   range term g_q = max(0, n_p . n_q)^P * exp(-((n_p . (x_q - x_p)) / sigma)^2)
 *   (normal agreement, distance of the sample from p's tangent plane);
 *   w_q = b_q (g_q + eps): eps keeps the sum positive and makes the result a
 *   continuous function of the inputs (plain bilinear where every g_q vanishes);
 *   E_p = sum w_q E_q / sum w_q; out_p = albedo_p E_p / pi + direct_p.
 * pos4 / nrm4 / alb4 / dir4: full-resolution [W*H][4] records (row-major);
 * E_low3: [h*w][3]; out3: [W*H][3].
 */
void orc_upsample_shade(const float* pos4, const float* nrm4, const float* alb4, const float* dir4, int W, int H,
                        const double* E_low3, int s, double P, double sigma, double eps, double* out3)
{
    const int w = (W + s - 1) / s, h = (H + s - 1) / s;
#pragma omp parallel for schedule(static)
    for (int Y = 0; Y < H; ++Y)
        for (int X = 0; X < W; ++X) {
            const int64_t p = (int64_t)Y * W + X;
            const int i0 = X / s, j0 = Y / s;
            const int i1 = i0 + 1 < w ? i0 + 1 : w - 1, j1 = j0 + 1 < h ? j0 + 1 : h - 1;
            const double fx = (double)(X - s * i0) / s, fy = (double)(Y - s * j0) / s;
            const int qi[4] = {i0, i1, i0, i1}, qj[4] = {j0, j0, j1, j1};
            const double b[4] = {(1 - fx) * (1 - fy), fx * (1 - fy), (1 - fx) * fy, fx * fy};
            const float* xp = pos4 + 4 * p;
            const float* np_ = nrm4 + 4 * p;
            double sw = 0.0, se[3] = {0.0, 0.0, 0.0};
            for (int c = 0; c < 4; ++c) {
                const int64_t src = (int64_t)(s * qj[c]) * W + s * qi[c];
                const float* xq = pos4 + 4 * src;
                const float* nq = nrm4 + 4 * src;
                double dot = 0.0, dpl = 0.0;
                for (int k = 0; k < 3; ++k) {
                    dot += (double)np_[k] * nq[k];
                    dpl += (double)np_[k] * ((double)xq[k] - xp[k]);
                }
                const double g = pow(dot > 0.0 ? dot : 0.0, P) * exp(-(dpl / sigma) * (dpl / sigma));
                const double wq = b[c] * (g + eps);
                const int64_t q = (int64_t)qj[c] * w + qi[c];
                sw += wq;
                for (int k = 0; k < 3; ++k) se[k] += wq * E_low3[3 * q + k];
            }
            for (int k = 0; k < 3; ++k)
                out3[3 * p + k] = (double)alb4[4 * p + k] * (se[k] / sw) / M_PI + dir4[4 * p + k];
        }
}

/*
 * Round to the nearest FP8 E4M3 value (1 sign, 4 exponent bits with bias 7,
 * 3 mantissa bits, subnormal step 2^-9, largest finite 448, no infinities),
 * ties to even, saturating to +-448.  Written from the format's definition.
 */
double orc_e4m3(double x)
{
    if (isnan(x)) return x;
    double a = fabs(x);
    if (a >= 448.0) return copysign(448.0, x);
    double step;
    if (a < ldexp(1.0, -6)) {
        step = ldexp(1.0, -9);
    } else {
        int e2;
        frexp(a, &e2);           /* a = m * 2^e2, m in [0.5, 1) */
        step = ldexp(1.0, e2 - 1 - 3);
    }
    double q = nearbyint(a / step) * step; /* default rounding mode: ties to even */
    if (q > 448.0) q = 448.0;
    return copysign(q, x);
}

void orc_e4m3_array(const double* x, int64_t n, double* out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_e4m3(x[i]);
}

/*
 * Nearest IEEE binary16 value of x (round to nearest, ties to even), written from
 * the format's definition: 11 significant bits for normal values (>= 2^-14),
 * spacing 2^-24 below; |x| >= 65520 (the midpoint between 65504 and 2^16) rounds
 * to infinity.
 */
double orc_f16(double x)
{
    if (isnan(x) || isinf(x)) return x;
    double a = fabs(x);
    if (a >= 65520.0) return copysign(INFINITY, x);
    int e2;
    frexp(a, &e2); /* a = m * 2^e2, m in [0.5, 1) */
    int ulp = e2 - 11;
    if (ulp < -24) ulp = -24;
    double q = ldexp(nearbyint(ldexp(a, -ulp)), ulp); /* default rounding mode: ties to even */
    return copysign(q, x);
}

void orc_f16_array(const double* x, int64_t n, double* out)
{
    for (int64_t i = 0; i < n; ++i) out[i] = orc_f16(x[i]);
}

/*
 * The FP16 network path as defined by Table 1's "all parameters in half
 * precision" with FP16 activations: the caller passes parameters already
 * rounded to binary16; every network input value and every hidden activation
 * (after ReLU) is rounded to binary16; sums are exact-ish in FP64; the output
 * layer's sum and softplus stay in FP64.
 */
static void mlp_forward_f16(const orc_desc* d, const double* mlp, const double* x_in, double* E)
{
    double buf_a[ORC_MAX_ENC + 8], buf_b[ORC_MAX_WIDTH];
    int k_in = orc_net_inputs(d);
    for (int i = 0; i < k_in; ++i) buf_a[i] = orc_f16(x_in[i]);
    const double* in = buf_a;
    const double* p = mlp;
    int layers = d->n_hidden + 1;
    double tmp[ORC_MAX_WIDTH];
    for (int layer = 0; layer < layers; ++layer) {
        int last = layer == layers - 1;
        int n_out = last ? d->out_dim : d->width;
        const double* W = p;
        const double* b = p + (int64_t)n_out * k_in;
        for (int o = 0; o < n_out; ++o) {
            double z = b[o];
            for (int i = 0; i < k_in; ++i) z += W[(int64_t)o * k_in + i] * in[i];
            if (last) E[o] = d->out_act == 1 ? softplus(z) : z;
            else tmp[o] = orc_f16(z > 0.0 ? z : 0.0);
        }
        if (!last) {
            for (int o = 0; o < n_out; ++o) buf_b[o] = tmp[o];
            in = buf_b;
        }
        p = b + n_out;
        k_in = n_out;
    }
}

/* Full query on the FP16 network path (see mlp_forward_f16); grid values as given. */
int orc_query_f16(const orc_desc* d, const double* params, const float* pos4, const float* nrm4, int64_t n,
                  const float* aabb_min, const float* aabb_max, float t, double* E)
{
    orc_layout_t L;
    if (fill_layout(d, &L)) return -1;
    const double* mlp = params + L.total * d->feat;
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) {
        float u[ORC_MAX_DIMS];
        double enc[ORC_MAX_ENC], x[ORC_MAX_ENC + 8];
        normalise(d, pos4 + 4 * q, aabb_min, aabb_max, t, u);
        encode_point(d, &L, params, u, enc, NULL, NULL);
        net_input(d, enc, nrm4 + 4 * q, t, x);
        mlp_forward_f16(d, mlp, x, E + q * d->out_dim);
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * FP8 (E4M3) network path.  Reading of "FP8 E4M3 with per-layer scales" (the
 * paper runs FP16; the FP8 form is an extension): every matrix product takes
 * E4M3 operands with one power-of-two scale per operand and layer,
 *   s = 2^ceil(log2(amax / 448)),
 * so that scaling is exact.  Weights: s_w from amax|W| of the layer.
 * Activations: s_a from the amax of the layer's FP32 input over a calibration
 * batch (the unquantised network).  One E4M3 code keeps 3 mantissa bits, which
 * moves E of He-initialised networks by 3-5% of its range; so each scaled value
 * v is carried as two E4M3 codes at the same scale, h = e4m3(v) and
 * l = e4m3(v - h), whose sum keeps about 8 bits.  Layer l computes
 *   z = (sum_i hW*ha + hW*la + lW*ha) * s_w * s_a + b
 * with (hW, lW) the pair of W[o][i]/s_w and (ha, la) that of a[i]/s_a (the
 * product lW*la lies below both codes' resolution and is left out), ReLU on
 * hidden layers, softplus on the output.  Biases stay in FP32.
 * ------------------------------------------------------------------------ */

/* 2^ceil(log2(amax / 448)) (1 when amax is 0) */
double orc_fp8_scale(double amax)
{
    if (!(amax > 0.0)) return 1.0;
    int e;
    double m = frexp(amax / 448.0, &e); /* amax/448 = m * 2^e, m in [0.5, 1) */
    return m == 0.5 ? ldexp(1.0, e - 1) : ldexp(1.0, e);
}

/*
 * Per-layer input amax of the unquantised network over n records:
 * amax[0] for the network input, amax[l] for the input of matrix l (l = 1..n_hidden).
 */
int orc_fp8_act_amax(const orc_desc* d, const double* params, const float* pos4, const float* nrm4, int64_t n,
                     const float* aabb_min, const float* aabb_max, float t, double* amax)
{
    orc_layout_t L;
    if (fill_layout(d, &L)) return -1;
    const double* mlp = params + L.total * d->feat;
    const int n_in = orc_net_inputs(d), layers = d->n_hidden + 1;
    for (int l = 0; l < layers; ++l) amax[l] = 0.0;
    double* z_all = (double*)malloc(sizeof(double) * ORC_MAX_LAYERS * ORC_MAX_WIDTH);
    double* a_all = (double*)malloc(sizeof(double) * ORC_MAX_LAYERS * ORC_MAX_WIDTH);
    for (int64_t q = 0; q < n; ++q) {
        float u[ORC_MAX_DIMS];
        double enc[ORC_MAX_ENC], x[ORC_MAX_ENC + 8], E[8];
        normalise(d, pos4 + 4 * q, aabb_min, aabb_max, t, u);
        encode_point(d, &L, params, u, enc, NULL, NULL);
        net_input(d, enc, nrm4 + 4 * q, t, x);
        mlp_forward(d, mlp, x, z_all, a_all, E, 0);
        for (int i = 0; i < n_in; ++i) amax[0] = fabs(x[i]) > amax[0] ? fabs(x[i]) : amax[0];
        for (int l = 1; l < layers; ++l)
            for (int o = 0; o < d->width; ++o) {
                double a = a_all[(l - 1) * ORC_MAX_WIDTH + o];
                amax[l] = a > amax[l] ? a : amax[l];
            }
    }
    free(z_all);
    free(a_all);
    return 0;
}

/*
 * FP8 query with the activation scales s_act[0..n_hidden] given (as computed from
 * orc_fp8_act_amax); weight scales are derived here from the parameters.
 */
int orc_query_fp8(const orc_desc* d, const double* params, const double* s_act, const float* pos4,
                  const float* nrm4, int64_t n, const float* aabb_min, const float* aabb_max, float t, double* Eout)
{
    orc_layout_t L;
    if (fill_layout(d, &L)) return -1;
    const double* mlp = params + L.total * d->feat;
    const int n_in = orc_net_inputs(d), layers = d->n_hidden + 1;
    double s_w[ORC_MAX_LAYERS];
    {
        const double* p = mlp;
        int k_in = n_in;
        for (int l = 0; l < layers; ++l) {
            int n_out = l == layers - 1 ? d->out_dim : d->width;
            double amax = 0.0;
            for (int64_t i = 0; i < (int64_t)n_out * k_in; ++i) amax = fabs(p[i]) > amax ? fabs(p[i]) : amax;
            s_w[l] = orc_fp8_scale(amax);
            p += (int64_t)n_out * k_in + n_out;
            k_in = n_out;
        }
    }
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < n; ++q) {
        float u[ORC_MAX_DIMS];
        double enc[ORC_MAX_ENC], a[ORC_MAX_WIDTH + ORC_MAX_ENC], z[ORC_MAX_WIDTH];
        double ah[ORC_MAX_WIDTH + ORC_MAX_ENC], al[ORC_MAX_WIDTH + ORC_MAX_ENC];
        normalise(d, pos4 + 4 * q, aabb_min, aabb_max, t, u);
        encode_point(d, &L, params, u, enc, NULL, NULL);
        net_input(d, enc, nrm4 + 4 * q, t, a);
        const double* p = mlp;
        int k_in = n_in;
        for (int l = 0; l < layers; ++l) {
            int last = l == layers - 1, n_out = last ? d->out_dim : d->width;
            const double* W = p;
            const double* b = p + (int64_t)n_out * k_in;
            for (int i = 0; i < k_in; ++i) {  /* the two codes of each scaled input */
                double v = a[i] / s_act[l];
                ah[i] = orc_e4m3(v);
                al[i] = orc_e4m3(v - ah[i]);
            }
            for (int o = 0; o < n_out; ++o) {
                double acc = 0.0;
                for (int i = 0; i < k_in; ++i) {
                    double v = W[(int64_t)o * k_in + i] / s_w[l];
                    double wh = orc_e4m3(v), wl = orc_e4m3(v - wh);
                    acc += wh * ah[i] + wh * al[i] + wl * ah[i];
                }
                z[o] = acc * s_w[l] * s_act[l] + b[o];
            }
            for (int o = 0; o < n_out; ++o) {
                if (!last) a[o] = z[o] > 0.0 ? z[o] : 0.0;
                else Eout[q * d->out_dim + o] = d->out_act == 1 ? softplus(z[o]) : z[o];
            }
            p = b + n_out;
            k_in = n_out;
        }
    }
    return 0;
}
