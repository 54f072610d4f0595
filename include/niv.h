/*
 * niv.h -- C ABI of the Neural Irradiance Volume query library (libniv.so).
 *
 * The library evaluates, per G-buffer pixel, the learned indirect irradiance
 * E(x, n) of "Real-time Rendering with a Neural Irradiance Volume" (Sec. 4.4:
 * the position and normal buffers are the model's input and the model infers
 * E for every pixel in one batch), shades it (Eq. 2), and trains the model
 * (Sec. 4.5) from Monte Carlo targets (Eq. 1).  All compute runs in CUDA
 * kernels for sm_103a on one GPU.
 *
 * Conventions shared by every entry point:
 *  - Every function returns an int status: NIV_OK (0) or a negative NIV_ERR_*.
 *    niv_last_error() returns a message for the calling thread's last failure.
 *  - "Device pointer" arguments are caller-owned CUDA device memory; the library
 *    never frees them.  Records are contiguous [n][4] arrays of float32 or
 *    float16 (xyz + one pad component), so each record is 16 or 8 bytes;
 *    pointers must be 16-byte aligned (NIV_ERR_ALIGN otherwise).
 *  - Work is enqueued asynchronously on the given stream (NULL = the legacy
 *    default stream) unless a function says it synchronises.  Kernel-side
 *    failures (a bounded wait that ran out) are latched in a device status word
 *    and reported by niv_sync_status().
 *  - A handle may be used from one host thread / stream at a time.
 */
#ifndef NIV_H
#define NIV_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define NIV_API __attribute__((visibility("default")))
#else
#define NIV_API
#endif

typedef struct CUstream_st* niv_stream; /* a cudaStream_t */
typedef struct niv_model* niv_handle;

#define NIV_OK 0
#define NIV_ERR_ARG (-1)         /* invalid argument or shape */
#define NIV_ERR_ALIGN (-2)       /* pointer not 16-byte aligned */
#define NIV_ERR_CUDA (-3)        /* a CUDA runtime call failed */
#define NIV_ERR_UNSUPPORTED (-4) /* valid description that this build does not support */
#define NIV_ERR_DEVICE (-5)      /* a kernel reported a failure (see niv_sync_status) */
#define NIV_ERR_NOMEM (-6)       /* device allocation failed */

/* network precision of a query */
#define NIV_FP32 0 /* plain path: FP32 features, weights and arithmetic on CUDA cores */
#define NIV_FP16 1 /* fused path: FP16 features and weights, tensor-core MLP, FP32 accumulate */
#define NIV_FP8 2  /* fused path: E4M3 weights and activations (two codes each) with per-layer
                      scales, FP32 accumulate */

/* element type of [n][4] record buffers */
#define NIV_F32 0
#define NIV_F16 1

/*
 * Model description (Sec. 4.1).  The encoding is the multi-level hash grid the
 * paper adopts: level l has resolution N_l = floor(base * growth^l) (FP64 on
 * the host); it stores its (N_l+1)^dims vertices densely (x fastest) when that
 * count is <= T = 2^log2_T, else T entries addressed by the spatial hash
 * (XOR_k v_k * pi_k) mod T with pi = (1, 2654435761, 805459861, prime_t).
 * Each entry holds `feat` features.  The network is fully connected: n_hidden
 * ReLU layers of `width`, then `out_dim` outputs with softplus (out_act = 1) or
 * identity (0).  Its input is [level features (level-major), n.xyz, (t)], so
 * in_extra is 3, or 4 when a scene parameter t is appended (Sec. 6).
 *
 * pe_bands > 0 selects the smaller models of Sec. 4.1 / Table 1, which have no
 * grid (levels = 0, dims = 3) and frequency-encode the position instead: for
 * each coordinate u_k of the normalised position (k = 0, 1, 2) and each band
 * b < pe_bands the pair (sin(2^b pi u_k), cos(2^b pi u_k)), in that order,
 * coordinate-major; the network input is then [those 6 * pe_bands values,
 * n.xyz].  Such models run in FP32 and FP16 (NIV_FP8 returns
 * NIV_ERR_UNSUPPORTED).  pe_bands = 0 for grid models.
 *
 * t_bands > 0 is Sec. 6's form of a higher-dimensional field: the grid stays 3-D and the
 * scene parameter t (clamped to [0, 1]) enters the network frequency-encoded, as the
 * pairs (sin(2^b pi t), cos(2^b pi t)) for b < t_bands after n.xyz; in_extra must be 3
 * and dims 3.  FP32 and FP16 (NIV_FP8 returns NIV_ERR_UNSUPPORTED).
 */
typedef struct niv_model_desc {
    int32_t dims;     /* 3, or 4 for a time-varying field (x, y, z, t) */
    int32_t levels;   /* 1..32 */
    int32_t feat;     /* 1, 2 or 4 */
    int32_t log2_T;   /* 4..24 */
    double base;      /* coarsest resolution */
    double growth;    /* resolution scale between levels */
    int32_t n_hidden; /* 1..4 */
    int32_t width;    /* 16, 32 or 64 */
    int32_t in_extra; /* 3 or 4 */
    int32_t out_dim;  /* 3 */
    int32_t out_act;  /* 0 identity, 1 softplus */
    uint32_t prime_t; /* odd hash constant of the 4th dimension */
    int32_t pe_bands; /* 0: hash grid; 1..16: frequency encoding, no grid */
    int32_t t_bands;  /* 0: t raw (in_extra 4) or absent; 1..6: t frequency-encoded (Sec. 6) */
} niv_model_desc;

/*
 * Per-call query parameters.  Positions map to grid coordinates by
 * u = clamp((p - aabb_min) * inv_extent, 0, 1), inv_extent = fp32(1 / (max - min)),
 * each step an FP32 operation; t (clamped to [0, 1]) is the 4th coordinate and
 * the appended network input of 4-D models.  image_width > 0 declares the
 * records to be a row-major image of that width, which the kernels traverse in
 * 2-D tiles for cache locality (results are identical either way).
 */
typedef struct niv_query_params {
    float aabb_min[3];
    float aabb_max[3];
    float t;
    int32_t image_width;
} niv_query_params;

/* Library version string. */
NIV_API const char* niv_version(void);

/* Message describing the calling thread's most recent failed call ("" if none). */
NIV_API const char* niv_last_error(void);

/*
 * Wait for all work queued on `stream`, then read and clear the device status
 * word of the current device.  Returns NIV_OK, NIV_ERR_DEVICE if a kernel
 * latched a failure (message in niv_last_error), or NIV_ERR_CUDA.
 */
NIV_API int niv_sync_status(niv_stream stream);

/*
 * Create a model on the current CUDA device (Sec. 4.1).  Allocates the FP32
 * master parameters (all zero) and derived inference copies; the library owns
 * them until niv_destroy.  NIV_ERR_ARG for an invalid description,
 * NIV_ERR_UNSUPPORTED for a valid one outside the kernels' limits, NIV_ERR_NOMEM.
 */
NIV_API int niv_create(const niv_model_desc* desc, niv_handle* out);

/* Free everything the handle owns (synchronises the device first).  NULL is accepted. */
NIV_API int niv_destroy(niv_handle h);

/*
 * Level layout of the encoding (Sec. 4.1): for level l, its resolution N_l,
 * whether it is dense (1) or hashed (0), its first entry and its entry count.
 * Any output pointer may be NULL.  Host pointers.
 */
NIV_API int niv_level_info(niv_handle h, int32_t level, int32_t* res, int32_t* dense, int64_t* first_entry,
                   int64_t* entries);

/*
 * Parameter counts: grid values (entries x feat) and network values (every
 * layer's W[out][in] row-major followed by b[out]).  The flat parameter vector
 * is [grid | network].  Host pointers, either may be NULL.
 */
NIV_API int niv_param_count(niv_handle h, int64_t* n_grid_values, int64_t* n_mlp_values);

/*
 * Replace all parameters with the n float32 values at `params` (host or device
 * memory, detected), rebuild the FP16 / FP8 inference copies, reset the Adam
 * state.  n must equal grid + network counts.  Synchronises `stream`.
 */
NIV_API int niv_set_params(niv_handle h, const float* params, int64_t n, niv_stream stream);

/* Copy the n FP32 master parameters to `out` (host or device memory).  Synchronises `stream`. */
NIV_API int niv_get_params(niv_handle h, float* out, int64_t n, niv_stream stream);

/*
 * Save a model to a file, and load one into a new handle on the current device.  The
 * file holds, little-endian: the 4 bytes "NIVM", uint32 format version 2; the model
 * description field by field in the order of niv_model_desc (int32 dims, levels, feat,
 * log2_T; float64 base, growth; int32 n_hidden, width, in_extra, out_dim, out_act;
 * uint32 prime_t; int32 pe_bands, t_bands); int64 n; the n FP32 master parameters in
 * the order of niv_set_params; then the optimiser state, so that training resumes where
 * it stopped: int32 training forward precision (NIV_FP32 or NIV_FP16), int64 Adam step
 * count, int32 1 if the Adam moments follow (a training call has run) else 0, and then
 * the n FP32 first moments and the n FP32 second moments.  Version 1 files (no
 * optimiser state) still load, starting a new optimisation.
 *  - niv_save synchronises `stream` (parameters and moments are read from the device).
 *  - niv_load reads and checks the header before it touches the device: a missing file,
 *    another magic or version, or a description that niv_create refuses is NIV_ERR_ARG
 *    with a message.  A parameter count that differs from the description's, or a short
 *    file, is NIV_ERR_ARG too (the model created for it is released again).  On any
 *    error *out is unchanged.
 */
NIV_API int niv_save(niv_handle h, const char* path, niv_stream stream);
NIV_API int niv_load(const char* path, niv_handle* out);

/*
 * The per-pixel query (Sec. 4.4): E = net(encode(u(p)), n, t) for n records.
 * pos, nrm: device [n][4] records of type dtype_in (NIV_F32 / NIV_F16);
 * out_E: device [n][4] records of type dtype_out holding E.rgb and 0.
 * precision: NIV_FP32, NIV_FP16 or NIV_FP8 (NIV_FP8 requires niv_fp8_calibrate
 * first).  n == 0 is a no-op.  Asynchronous on `stream`.
 */
NIV_API int niv_query(niv_handle h, const void* pos, const void* nrm, int64_t n, int32_t dtype_in,
              const niv_query_params* params, void* out_E, int32_t dtype_out, int32_t precision,
              niv_stream stream);

/*
 * niv_query for HOST buffers (pageable or pinned); results are those of niv_query,
 * bit for bit, and `stream` is synchronised before returning.
 *  - Page-locked buffers that the GPU can address (cudaHostAlloc, torch pin_memory;
 *    16-byte aligned): one query reads the records from host memory and writes E to
 *    out_E directly (over NVLink-C2C on Grace systems), with no staging copies.
 *  - Other memory: pos/nrm are copied to a handle-owned device staging area and E
 *    back.  Calls of more than 131072 records are split into up to 32 chunks of whole
 *    128-record tiles (whole bands of 4-row tiles of the image when image_width > 0), about
 *    two waves of the FP16 kernel each, whose host-to-device copy, query and
 *    device-to-host copy run on three streams at once (two copy streams owned by the
 *    handle, ordered after the work already queued on `stream`).
 * Environment: NIV_HOST_MODE=1 forces the staged path; NIV_HOST_CHUNKS=k sets the
 * chunk count of the staged path.
 */
NIV_API int niv_query_host(niv_handle h, const void* pos, const void* nrm, int64_t n, int32_t dtype_in,
                   const niv_query_params* params, void* out_E, int32_t dtype_out, int32_t precision,
                   niv_stream stream);

/* Optimiser settings of niv_fit (Sec. 4.5: Adam, learning rate 1e-2). */
typedef struct niv_fit_params {
    float lr;        /* learning rate */
    float beta1;     /* Adam first-moment decay, e.g. 0.9 */
    float beta2;     /* Adam second-moment decay, e.g. 0.99 */
    float adam_eps;  /* Adam denominator epsilon, e.g. 1e-15 */
    float loss_eps;  /* epsilon of the relative L2 loss (Eq. 3): 0.01 */
} niv_fit_params;

/*
 * Loss and gradient of one batch (Sec. 4.5, Eq. 3): the relative L2 loss
 * (E_theta - E)^2 / (sg(E_theta^2) + loss_eps), averaged over the n samples and the
 * 3 channels, and its gradient w.r.t. every parameter, written to the handle's
 * gradient buffer (read it with niv_get_grads).  The forward pass runs in FP32
 * against the FP32 master parameters.  pos, nrm, target: device float32 [n][4]
 * records (x, normal, target E); t: device float32 [n] per-sample scene parameter
 * of a 4-D model, or NULL to use params->t.  loss_out (host, nullable): the loss,
 * which makes the call synchronise `stream`.  The first call allocates the training
 * state (gradients, Adam moments, activation scratch).
 */
NIV_API int niv_grad(niv_handle h, const float* pos, const float* nrm, const float* t, const float* target, int64_t n,
                     const niv_query_params* params, float loss_eps, double* loss_out, niv_stream stream);

/*
 * Vector-Jacobian product of the query (the hand-written backward of Sec. 4.5 with the
 * loss left to the caller): for device float32 [n][4] records pos, nrm and grad_E (dL/dE
 * per sample in xyz), the gradient buffer receives dL/dtheta = sum over samples of
 * grad_E . dE/dtheta for every parameter (grid values with their hash collisions summed,
 * weights, biases), E being the FP32 forward against the FP32 master parameters.  t as
 * in niv_grad.  Read the result with niv_get_grads.  Asynchronous.
 */
NIV_API int niv_backward(niv_handle h, const float* pos, const float* nrm, const float* t, const float* grad_E,
                         int64_t n, const niv_query_params* params, niv_stream stream);

/*
 * Forward precision of niv_grad, niv_fit and niv_backward (config 2: "FP16 forward / FP32
 * master weights").  NIV_FP32 (the default): FP32 throughout against the master
 * parameters.  NIV_FP16: the forward is the FP16 path of niv_query -- grid values, weights
 * and biases rounded to binary16 as they are read, the network input and every hidden
 * activation rounded to binary16, FP32 sums -- and the gradient is that of this function
 * taken straight through the roundings, applied to the FP32 master parameters.
 */
NIV_API int niv_set_train_forward(niv_handle h, int32_t precision);

/* Copy the n gradient values of the last niv_grad to `out` (host or device).  Synchronises. */
NIV_API int niv_get_grads(niv_handle h, float* out, int64_t n, niv_stream stream);

/* Overwrite the gradient buffer with n values (host or device), e.g. to drive niv_adam_step. */
NIV_API int niv_set_grads(niv_handle h, const float* grads, int64_t n, niv_stream stream);

/*
 * One Adam step (Kingma & Ba; Sec. 4.5) on every parameter from the gradient
 * buffer: m = b1 m + (1-b1) g, v = b2 v + (1-b2) g^2, theta -= lr m_hat / (sqrt(v_hat) + eps)
 * with bias corrections 1 - b^step (step counts calls since the last niv_set_params).
 * The inference copies are rebuilt on the next niv_query.  Asynchronous.
 */
NIV_API int niv_adam_step(niv_handle h, float lr, float beta1, float beta2, float eps, niv_stream stream);

/* niv_grad followed by niv_adam_step with the settings in fp. */
NIV_API int niv_fit(niv_handle h, const float* pos, const float* nrm, const float* t, const float* target, int64_t n,
                    const niv_query_params* params, const niv_fit_params* fp, double* loss_out, niv_stream stream);

/*
 * Calibrate the E4M3 network path (NIV_FP8).  Runs the FP32 network over the n
 * device records pos/nrm ([n][4], dtype_in) and takes, for every matrix product,
 * the amax of its FP32 input; the activation scale is s_a = 2^ceil(log2(amax/448))
 * (1 if amax = 0).  Weight scales s_w = 2^ceil(log2(amax|W|/448)) per layer.  Every
 * scaled weight v = W / s_w is packed for the tensor cores as two E4M3 codes,
 * h = e4m3(v) and l = e4m3(v - h); the query forms the layer inputs the same way from
 * a / s_a and sums the products h_W h_a + h_W l_a + l_W h_a in FP32 (one code keeps 3
 * mantissa bits, two about 8).  Must be called again after niv_set_params.
 * Synchronises `stream`.  NIV_ERR_UNSUPPORTED for width 16.
 */
NIV_API int niv_fp8_calibrate(niv_handle h, const void* pos, const void* nrm, int64_t n, int32_t dtype_in,
                              const niv_query_params* params, niv_stream stream);

/*
 * The scales of the last calibration, count = n_hidden + 1 entries each (one per
 * matrix product; entry 0 is the network input): activation scale, weight scale
 * and the measured activation amax.  Host pointers, any may be NULL.
 */
NIV_API int niv_fp8_get_scales(niv_handle h, float* s_act, float* s_w, float* amax, int32_t count);

/* Monte Carlo modes: every radiance reaching x, or only light that bounced at least once. */
#define NIV_MC_TOTAL 0
#define NIV_MC_INDIRECT 1

/*
 * Training-sample candidates (Sec. 4.5 / App. I): a fraction surface_frac (0.2 in
 * the paper) of the n points lie on the scene's surfaces, spread over them in
 * proportion to area, with the surface normal as direction; the rest are uniform
 * in the room with directions uniform on the sphere.  The surfaces, in order: the
 * room walls (axis 0..2, the wall at room_min first, normals into the room; the
 * ceiling cut into the strips around the open skylight), every sphere that does
 * not emit (at rest), every box face (outward normals).  Sample j = index_base + i
 * draws Philox4x32-10 at counters (j lo, j hi, 0x53414D50, 0 | 1), key (seed lo,
 * seed hi); u = float(r >> 8) 2^-24 + 2^-25.  Surface iff u(r0) < surface_frac;
 * surface k = first k with u(r1) < cdf[k] (cumulative area fractions, FP64 sums
 * rounded to FP32); rectangle coordinates lo + (hi - lo) u in FP32; sphere points
 * c + r d; t = u(r6).
 * scene: host description as in niv_mc_irradiance; x4, n4: device float32 [n][4]
 * (16-byte aligned); t: device float32 [n] or NULL; patch: device int32 [n] or NULL
 * (-1 for volume samples, else the surface index).  Candidates inside geometry are
 * left in (niv_mc_irradiance flags them).  Asynchronous.
 */
NIV_API int niv_training_samples(const float* scene, int64_t scene_len, int64_t n, float surface_frac, uint64_t seed,
                                 uint64_t index_base, float* x4, float* n4, float* t, int32_t* patch,
                                 niv_stream stream);

/*
 * Monte Carlo irradiance of the analytic scene (Eq. 1): the training targets of
 * Sec. 4.5.  For each of m points x (device float32 [m][4]) with normal n
 * ([m][4]): E = (pi / spp) sum_j L_i(x, w_j), w_j cosine-distributed about n; paths
 * use next-event estimation toward emitting spheres and Russian roulette after three
 * bounces.  NIV_MC_INDIRECT (the paper's E, Sec. 3) omits emission seen directly
 * from x and direct sky light.  out_E: device float64 [m][3].  out_keep (device
 * uint8 [m], nullable): 0 for points whose first hits are mostly back faces (inside
 * geometry, Sec. 4.5) or whose E is zero (App. I), else 1.  t (device float32 [m],
 * nullable): time of the rotating sphere per point.  Random numbers:
 * Philox4x32-10, counter (point index_base + i, path j, bounce, purpose), key seed.
 * scene: the host float32 scene description (niv_inputs.scenes layout, at most 56
 * objects) of scene_len values.  Asynchronous.
 */
NIV_API int niv_mc_irradiance(const float* scene, int64_t scene_len, const float* x4, const float* n4, const float* t,
                              int64_t m, int32_t spp, uint64_t seed, uint64_t index_base, int32_t mode, double* out_E,
                              uint8_t* out_keep, niv_stream stream);

/*
 * Primary-visibility G-buffer of the analytic scene: the world position, normal and
 * albedo per pixel that the per-pixel query reads (Sec. 4.4; the deferred-shading inputs
 * of Fig. 3).  A pinhole camera at eye (host float[3]) looks down +z with +y up; the
 * ray of pixel (i, j), row 0 at the top, has direction
 * ((2 (i + 0.5) / width - 1) s width / height, (1 - 2 (j + 0.5) / height) s, 1),
 * normalised, with s = tan(vfov_deg / 2).  The first hit beyond 1e-4 follows
 * niv_mc_irradiance's geometry in FP32 with the rotating sphere at scene parameter t:
 * unit normals, outward for spheres and boxes, into the room for the walls; a ray leaving
 * through the open skylight hits nothing.  pos, nrm, alb: device [width * height][4]
 * records of dtype_out (NIV_F16 or NIV_F32; xyz and a pad of 0; all zero where nothing
 * is hit), aligned to the record size; alb and hit (device uint8 [width * height]: 1
 * where the ray hit) may be NULL.  scene: host description as in niv_mc_irradiance.
 * NIV_ERR_ARG for sizes <= 0, more than 2^31 pixels or vfov_deg outside (0, 180).
 * Asynchronous.
 */
NIV_API int niv_gbuffer_raycast(const float* scene, int64_t scene_len, int32_t width, int32_t height, double vfov_deg,
                                const float* eye, float t, void* pos, void* nrm, void* alb, int32_t dtype_out,
                                uint8_t* hit, niv_stream stream);

/*
 * Triangle meshes inserted into a G-buffer made by niv_gbuffer_raycast (the dynamic
 * objects of Sec. 4.4 in the deferred-shading inputs), with the same camera arguments.
 * A pixel's ray hits triangle (A, B, C) at distance t > 1e-6 (Moeller-Trumbore in FP32,
 * barycentrics accepted to 1e-5 outside the edges so that shared edges leave no cracks); the
 * nearest hit closer than the surface already in the pixel (|pos - eye| where hit = 1)
 * replaces it: position eye + t d, the face normal (B - A) x (C - A) normalised and turned
 * toward the camera, the mesh's albedo, hit = 1.  Among triangles at the same t the lowest
 * index wins.  Triangles with a vertex less than 1e-3 in front of the camera plane
 * (z - eye_z <= 1e-3) are skipped.  tri9: device float32 [n_tris][9] (the three vertices),
 * tri_mesh: device int32 [n_tris] (mesh index; an index outside [0, n_meshes) gives albedo
 * 0), mesh_albedo: host float32 [n_meshes][3], 1 <= n_meshes <= 64.  pos, nrm, alb (may be
 * NULL): device [width * height][4] records of dtype (NIV_F16 / NIV_F32), updated in place;
 * hit: device uint8 [width * height], read and updated; mesh_id (may be NULL): device int32
 * [width * height], set to the winning mesh or -1; scratch: device uint64 [width * height].
 * A triangle's work is its projected bounding box, so a triangle that covers much of the
 * screen is slow.  Asynchronous.
 */
NIV_API int niv_gbuffer_meshes(const float* tri9, const int32_t* tri_mesh, int64_t n_tris, const float* mesh_albedo,
                               int32_t n_meshes, int32_t width, int32_t height, double vfov_deg, const float* eye,
                               void* pos, void* nrm, void* alb, int32_t dtype, uint8_t* hit, int32_t* mesh_id,
                               uint64_t* scratch, niv_stream stream);

/*
 * Keep the samples niv_mc_irradiance flagged out_keep = 1 (Sec. 4.5 culling, App. I
 * null discard), in their original order: out_x4, out_n4 (device float32 [m][4]),
 * out_t (device float32 [m], nullable; copies t, or 0 when t is NULL) and
 * out_target4 (device float32 [m][4]: E rounded to FP32, w = 0) receive the first
 * *out_count (host) entries.  Synchronises `stream`.
 */
NIV_API int niv_compact_targets(const float* x4, const float* n4, const float* t, const double* E, const uint8_t* keep,
                                int64_t m, float* out_x4, float* out_n4, float* out_t, float* out_target4,
                                int64_t* out_count, niv_stream stream);

/*
 * Bake the SH probe grid of Sec. 5.1 / App. A: second-order real SH (9 coefficients
 * per RGB channel) of the indirect incident radiance at every probe, projected from
 * `rays` directions uniform on the sphere (one indirect path each).  Probes sit at the
 * lattice vertices lo + (hi - lo) * ijk / (P - 1), x fastest; P, lo, hi are host
 * arrays of 3.  out_coef64 (device float64 [Np][27], coefficient q of channel c at
 * 3q + c; nullable) and/or out_coef16 (device float16 [Np][28], the same rounded to
 * half precision plus one zero pad: 54 bytes of coefficients per probe; nullable).
 * Random numbers: Philox4x32-10 as in niv_mc_irradiance (directions: counter
 * (probe, ray + (0xFFFE << 16), 0); paths: stream index_base + probe * rays + ray).
 * Asynchronous.
 */
NIV_API int niv_probe_bake(const float* scene, int64_t scene_len, const int32_t* P, const float* lo, const float* hi,
                           int32_t rays, uint64_t seed, uint64_t index_base, double* out_coef64, void* out_coef16,
                           niv_stream stream);

/*
 * Probe-grid irradiance at G-buffer records (App. A): trilinear weights over the 8
 * probes of the cell around x, times the cosine fall-off max(0, n . normalize(p - x)),
 * clamped below at 1e-6 and renormalised; each probe contributes its SH irradiance
 * (Ramamoorthi & Hanrahan).  coef16: device float16 [Np][28] from niv_probe_bake.
 * Records as in niv_query (image_width > 0: image traversal).  Asynchronous.
 */
NIV_API int niv_probe_query(const void* coef16, const int32_t* P, const float* lo, const float* hi, const void* pos,
                            const void* nrm, int64_t n, int32_t dtype_in, void* out_E, int32_t dtype_out,
                            int32_t image_width, niv_stream stream);

/*
 * The probe query with ray-traced visibility ("+ RT", Sec. 5.1 and App. A: visibility-
 * based probe rejection replaces the cosine fall-off).  Reading: a shadow ray leaves
 * x + 0.01 n (world units, n normalised) toward each of the 8 probes; a probe whose ray
 * hits scene geometry more than 0.01 before reaching it gets weight 0 before the 1e-6
 * clamp and the renormalisation.  scene, scene_len: the host scene description of
 * niv_mc_irradiance, at scene parameter t.  Other arguments as niv_probe_query.
 * Asynchronous.
 */
NIV_API int niv_probe_query_rt(const void* coef16, const int32_t* P, const float* lo, const float* hi,
                               const float* scene, int64_t scene_len, float t, const void* pos, const void* nrm,
                               int64_t n, int32_t dtype_in, void* out_E, int32_t dtype_out, int32_t image_width,
                               niv_stream stream);

/*
 * Largest n accepted by niv_query_host_noalloc: the number of records its fixed
 * staging area holds.
 */
#define NIV_NOALLOC_MAX_RECORDS 65536

/*
 * niv_query_host for callers that must not have the library allocate device
 * memory, e.g. a real-time render loop that fixes its GPU memory budget at
 * start-up and forbids allocation while frames are in flight, or a plug-in whose
 * host application owns every device allocation.  The paper has no counterpart:
 * this is an integration variant of the query.
 *
 * Same arguments and results as niv_query_host (host buffers in and out,
 * precision NIV_FP32 or NIV_FP16, synchronises `stream`), but the records are
 * staged in a fixed file-scope device array of NIV_NOALLOC_MAX_RECORDS records
 * (about 3 MiB, held by every GPU that loads the library until the process exits)
 * instead of a library allocation.  No cudaMalloc or cudaFree is called.
 *  - n > NIV_NOALLOC_MAX_RECORDS: NIV_ERR_ARG with a message, nothing runs.
 *  - The first call on a device looks up the array's device address (once per
 *    device, with that device current); make that first call before any stream
 *    capture begins.
 *  - Every call shares the one array, which keeps the last call's contents; calls
 *    whose work overlaps on the GPU race with each other, so serialise them.
 *  - The model's parameters must have been set (niv_set_params or niv_load):
 *    otherwise NIV_ERR_ARG.  After training steps the call first rebuilds the
 *    model's inference copies in place, as niv_query does (no allocation).
 *  - The array's address is cached per device ordinal for the life of the
 *    process: do not reset a device (cudaDeviceReset) while this library is
 *    loaded.  The library's device status word is cached the same way.
 */
NIV_API int niv_query_host_noalloc(niv_handle h, const void* pos, const void* nrm, int64_t n, int32_t dtype_in,
                                   const niv_query_params* params, void* out_E, int32_t dtype_out,
                                   int32_t precision, niv_stream stream);

/*
 * The query with shading fused into its epilogue (Sec. 4.4 then Eq. 2 and the
 * runtime direct light of Sec. 3 / Fig. 3): for each record the kernel evaluates E
 * and writes rgba = (albedo * E / pi + direct, 1) straight to out_rgba, so E never
 * reaches memory.  albedo, direct, out_rgba: device FP16 [n][4] records; pos, nrm as
 * in niv_query.  Asynchronous.
 */
NIV_API int niv_query_shade(niv_handle h, const void* pos, const void* nrm, const void* albedo, const void* direct,
                            int64_t n, int32_t dtype_in, const niv_query_params* params, void* out_rgba,
                            int32_t precision, niv_stream stream);

/*
 * Encoding only (Sec. 4.1), for inspection and parity checks: for each of the n
 * position records, out_enc (device float32 [n][levels*feat + 6*pe_bands],
 * nullable) receives the interpolated level features in FP32 from the FP32
 * master grid, then the frequency-encoding values of a model without grid,
 * and out_idx (device uint32 [n][levels][2^dims], nullable) the table entry of
 * every cell corner, corner c having offset bit k set along dimension k.
 * Same normalisation and index arithmetic as niv_query.  Asynchronous.
 */
NIV_API int niv_encode(niv_handle h, const void* pos, int64_t n, int32_t dtype_in, const niv_query_params* params,
                       float* out_enc, uint32_t* out_idx, niv_stream stream);

/*
 * Shading (Eq. 2 plus the runtime direct light of Sec. 3 / Fig. 3):
 * rgba = (albedo * E / pi + direct, 1), FP32 arithmetic, FP16 output.
 * albedo, direct, E: device [n][4] FP16 records; out_rgba: device [n][4] FP16.
 */
NIV_API int niv_shade(const void* albedo, const void* direct, const void* E, int64_t n, void* out_rgba,
              niv_stream stream);

/*
 * Dynamic ambient occlusion (Sec. 4.4 "Dynamic Ambient Occlusion": the hemisphere
 * obstruction at the shading point by the dynamic geometry only, which the cached
 * irradiance does not know; it darkens the dynamic objects themselves and the static
 * surfaces near them).  The paper gives no formula; this library's reading:
 *   from o = x + 0.01 n (world units, n normalised), `rays` cosine-distributed
 *   directions about n, direction j drawn from Philox4x32-10 (as niv_mc_irradiance) on
 *   counter (record lo, record hi, j, 0xA0) with key (seed lo, seed hi); a ray is
 *   blocked when it meets a dynamic triangle at 0 < t <= radius;
 *   AO = 1 - blocked / rays, and the irradiance is scaled E <- AO E before shading.
 *
 * niv_dyn_create takes the frame's dynamic triangles (host float32 [n_tris][9]: three
 * world-space vertices each), builds a bounding-volume hierarchy over them on the host
 * and uploads it to the current device; niv_dyn_destroy frees it.  niv_dyn_ao runs the
 * pass for n records (pos, nrm: device [n][4] of dtype_in): out_ao (device float32 [n],
 * nullable) receives AO, and E_inout (device [n][4] of dtype_E, nullable, e.g. the
 * output of niv_query) is scaled in place.  rays in 1..1024, radius > 0.  Asynchronous.
 */
typedef struct niv_dyn* niv_dyn_handle;
NIV_API int niv_dyn_create(const float* tris, int64_t n_tris, niv_dyn_handle* out);
NIV_API int niv_dyn_destroy(niv_dyn_handle d);
/* Number of hierarchy nodes (diagnostics). */
NIV_API int64_t niv_dyn_node_count(niv_dyn_handle d);
NIV_API int niv_dyn_ao(niv_dyn_handle d, const void* pos, const void* nrm, int64_t n, int32_t dtype_in, int32_t rays,
                       float radius, uint64_t seed, float* out_ao, void* E_inout, int32_t dtype_E, niv_stream stream);

/*
 * Half-resolution rendering (Sec. 4.4 "Half-resolution Rendering"; Table 1, column
 * "half": a quarter of the pixels queried, the full-size albedo buffer kept).
 *
 * niv_query_sub queries the pixels (sub x, sub y) of a full_width x full_height
 * row-major G-buffer (pos, nrm as in niv_query) and writes E for them to out_E, a
 * row-major [h][w][4] buffer, w = ceil(full_width / sub), h = ceil(full_height / sub).
 * sub >= 1 (2 for half resolution).  Precisions and dtypes as in niv_query;
 * params->image_width is ignored.  Asynchronous.
 */
NIV_API int niv_query_sub(niv_handle h, const void* pos, const void* nrm, int32_t full_width, int32_t full_height,
                          int32_t sub, int32_t dtype_in, const niv_query_params* params, void* out_E,
                          int32_t dtype_out, int32_t precision, niv_stream stream);

/*
 * Joint bilateral upsampling of the irradiance (the practice Sec. 4.4 points to:
 * Kopf et al. 2007), fused with the shading of niv_shade.  The paper leaves the
 * weights open; this library's reading: pixel p = (X, Y) blends the low-resolution
 * samples q = (i, j), i in {i0, i1}, j in {j0, j1}, i0 = floor(X / sub),
 * i1 = min(i0 + 1, w - 1) (likewise j), with the bilinear weights b_q of
 * (X / sub - i0, Y / sub - j0) times a range term on the full-resolution G-buffer
 * record of q's pixel (sub i, sub j):
 *   g_q = max(0, n_p . n_q)^power * exp(-((n_p . (x_q - x_p)) / sigma)^2),
 *   E_p = sum b_q (g_q + eps) E_q / sum b_q (g_q + eps),
 *   rgba_p = (albedo_p E_p / pi + direct_p, 1),
 * FP32 arithmetic, FP16 output.  pos, nrm: full-resolution [H][W][4] records of
 * dtype_in; albedo, direct, out_rgba: FP16 [H][W][4]; E_low: [h][w][4] records of
 * dtype_E as niv_query_sub writes them.  sigma (world units) and eps must be > 0.
 * No counterpart of these exact weights in the paper.  Asynchronous.
 */
typedef struct niv_upsample_params {
    float power; /* exponent of the normal agreement, e.g. 8 */
    float sigma; /* plane-distance scale in world units, e.g. 0.05 */
    float eps;   /* weight floor, e.g. 1e-4 */
} niv_upsample_params;

NIV_API int niv_upsample_shade(const void* pos, const void* nrm, const void* albedo, const void* direct,
                               int32_t full_width, int32_t full_height, int32_t dtype_in, const void* E_low,
                               int32_t dtype_E, int32_t sub, const niv_upsample_params* up, void* out_rgba,
                               niv_stream stream);

/*
 * Diagnostic (no counterpart in the paper): one 128 x 64 x K tensor-core product
 * of fixed small-integer operands, A[m][k] = (3m + 5k) mod 7 - 3 and
 * B[n][k] = (5n + 3k) mod 5 - 2, written to out (device float32 [128][64],
 * D = A B^T, exact).  mode 0: FP16 operands, K = 32; mode 1: the same with the
 * two stride fields of the operand descriptors exchanged (a layout-convention
 * probe that stays inside the operands); mode 2: E4M3 operands, K = 64.
 * Asynchronous; a timeout of the completion wait is reported by niv_sync_status.
 */
NIV_API int niv_selftest_mma(int32_t mode, float* out, niv_stream stream);

/*
 * Diagnostic (no counterpart in the paper): makes the bounded wait that every
 * tensor-core query kernel uses run out, without a fault.  One block allocates
 * tensor memory as a query kernel does, issues no tensor-core operation, waits
 * limit_us microseconds (1 .. 1000000, else NIV_ERR_ARG) on an mbarrier phase
 * that nothing completes, latches failure code 3 in the device status word,
 * frees its tensor memory and returns.  niv_sync_status() then reports
 * NIV_ERR_DEVICE (and clears the word); the context stays usable.  Asynchronous.
 */
NIV_API int niv_selftest_wait_expiry(uint32_t limit_us, niv_stream stream);

/*
 * Diagnostic (no counterpart in the paper): the device counter-based generator
 * that the Monte Carlo integrator, the probe bake and the ambient-occlusion pass
 * draw from, Philox4x32-10 (Salmon et al., "Parallel Random Numbers: As Easy as
 * 1, 2, 3", SC'11), applied to given inputs, so that it can be checked against
 * the published known-answer vectors.  in6: device uint32 [n][6] = counter c0..c3,
 * key k0, k1; out4: device uint32 [n][4].  Asynchronous.
 */
NIV_API int niv_selftest_philox(const uint32_t* in6, int64_t n, uint32_t* out4, niv_stream stream);

#ifdef __cplusplus
}
#endif

#endif /* NIV_H */
