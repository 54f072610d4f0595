/*
 * CPU FP64 Monte Carlo irradiance integrator for the analytic scenes.
 *
 * TEST INFRASTRUCTURE ONLY (tests/, the smoke check and the benchmark's CPU
 * baseline).  Shares no source with the CUDA library.
 *
 * Computes Eq. 1 of the paper, E(x, n) = int L_i(x, w) <w, n>^+ dw, with the
 * estimator E ~ (pi / S) sum_j L_i(x, w_j) over cosine-distributed w_j around n.
 * Mode TOTAL counts every radiance arriving at x; mode INDIRECT (the quantity
 * the paper caches, Sec. 3: direct light D is added at runtime) omits radiance
 * emitted by the first surface hit from x and sky light reaching x directly.
 * Paths continue by cosine sampling with next-event estimation toward emitting
 * spheres (uniform cone sampling) and Russian roulette after three bounces.
 * Per Sec. 4.5 / App. I a sample is flagged for discard when the majority of its
 * first hits are back faces (the point is inside geometry) or when its
 * irradiance is zero in every channel.
 *
 * Random numbers: Philox4x32-10 (Salmon et al., SC'11), implemented here from
 * its published definition; counter = (sample lo, sample hi, j + (depth << 16),
 * purpose), key = (seed lo, seed hi).  purpose 0 = bounce direction and
 * roulette, 1 + e = light sample toward emitter e.  u32 -> (0,1) via
 * (x >> 8) * 2^-24 + 2^-25.
 *
 * Scene description: the flat float layout written by niv_inputs.scenes.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define HDR 48
#define SPH 12
#define BOX 12
#define T_EPS 1e-4
#define MAX_DEPTH 32

enum { MC_TOTAL = 0, MC_INDIRECT = 1 };

/* ---------------- Philox4x32-10 ---------------- */
static void mulhilo32(uint32_t a, uint32_t b, uint32_t* hi, uint32_t* lo)
{
    uint64_t p = (uint64_t)a * (uint64_t)b;
    *hi = (uint32_t)(p >> 32);
    *lo = (uint32_t)p;
}

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0, lo0, hi1, lo1;
        mulhilo32(0xD2511F53u, c[0], &hi0, &lo0);
        mulhilo32(0xCD9E8D57u, c[2], &hi1, &lo1);
        uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    memcpy(out, c, sizeof c);
}

static double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0) + (1.0 / 33554432.0); }

typedef struct { uint64_t sample; uint64_t seed; } rng_ctx;

static void draw(const rng_ctx* r, uint32_t j, uint32_t depth, uint32_t purpose, double u[4])
{
    uint32_t ctr[4] = {(uint32_t)r->sample, (uint32_t)(r->sample >> 32), j + (depth << 16), purpose};
    uint32_t key[2] = {(uint32_t)r->seed, (uint32_t)(r->seed >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    for (int i = 0; i < 4; ++i) u[i] = u01(o[i]);
}

/* ---------------- scene ---------------- */
typedef struct {
    const float* h;
    const float* sph;
    const float* box;
    int ns, nb, room;
    double sph_c[64][3]; /* sphere centres after the time rotation */
    double grow;         /* every solid thickened by this much (0 except for visibility margins) */
} scene_t;

static void scene_init(scene_t* s, const float* blob, double t)
{
    s->h = blob;
    s->ns = (int)blob[0];
    s->nb = (int)blob[1];
    s->room = blob[2] != 0.0f;
    s->sph = blob + HDR;
    s->box = blob + HDR + SPH * s->ns;
    s->grow = 0.0;
    int rot = (int)blob[3];
    for (int i = 0; i < s->ns && i < 64; ++i) {
        const float* c = s->sph + SPH * i;
        s->sph_c[i][0] = c[0];
        s->sph_c[i][1] = c[1];
        s->sph_c[i][2] = c[2];
        if (i == rot) { /* rotate by 2 pi t about +y through the axis point */
            double a = 2.0 * M_PI * t, ca = cos(a), sa = sin(a);
            double px = blob[36], pz = blob[38];
            double dx = c[0] - px, dz = c[2] - pz;
            s->sph_c[i][0] = px + ca * dx + sa * dz;
            s->sph_c[i][2] = pz - sa * dx + ca * dz;
        }
    }
}

enum { HIT_NONE = 0, HIT_SPHERE, HIT_BOX, HIT_WALL };

typedef struct {
    int kind, id;     /* id: sphere/box index or wall 0..5 (-x,+x,-y,+y,-z,+z) */
    double t, p[3], n[3]; /* n: geometric normal (outward for objects, into the room for walls) */
} hit_t;

static double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

static int intersect(const scene_t* s, const double* o, const double* d, hit_t* h)
{
    h->kind = HIT_NONE;
    h->t = INFINITY;
    for (int i = 0; i < s->ns; ++i) {
        const double* c = s->sph_c[i];
        double r = s->sph[SPH * i + 3] + s->grow;
        double oc[3] = {o[0] - c[0], o[1] - c[1], o[2] - c[2]};
        double b = dot3(oc, d), cc = dot3(oc, oc) - r * r, disc = b * b - cc;
        if (disc < 0.0) continue;
        double sq = sqrt(disc), t = -b - sq;
        if (t <= T_EPS) t = -b + sq;
        if (t > T_EPS && t < h->t) { h->t = t; h->kind = HIT_SPHERE; h->id = i; }
    }
    for (int i = 0; i < s->nb; ++i) {
        const float* bx = s->box + BOX * i;
        double tn = -INFINITY, tf = INFINITY;
        int an = 0, af = 0;
        for (int k = 0; k < 3; ++k) {
            double t1 = ((double)bx[k] - s->grow - o[k]) / d[k], t2 = ((double)bx[3 + k] + s->grow - o[k]) / d[k];
            double lo = t1 < t2 ? t1 : t2, hi = t1 < t2 ? t2 : t1;
            if (lo > tn) { tn = lo; an = k; }
            if (hi < tf) { tf = hi; af = k; }
        }
        if (tf < tn) continue;
        double t;
        int ax;
        if (tn > T_EPS) { t = tn; ax = an; } else if (tf > T_EPS) { t = tf; ax = af; } else continue;
        if (t < h->t) { h->t = t; h->kind = HIT_BOX; h->id = i * 3 + ax; }
    }
    if (s->room) {
        const float* lo = s->h + 4;
        const float* hi = s->h + 7;
        double tw = INFINITY;
        int wall = -1;
        for (int k = 0; k < 3; ++k) {
            double t;
            if (d[k] > 0) t = ((double)hi[k] - s->grow - o[k]) / d[k];
            else if (d[k] < 0) t = ((double)lo[k] + s->grow - o[k]) / d[k];
            else continue;
            if (t < tw) { tw = t; wall = 2 * k + (d[k] > 0); }
        }
        if (wall >= 0 && tw < h->t) {
            double px = o[0] + tw * d[0], pz = o[2] + tw * d[2];
            const float* sk = s->h + 13;
            const double g = s->grow;
            int open = wall == 3 && sk[0] < sk[1] && px >= sk[0] + g && px <= sk[1] - g && pz >= sk[2] + g &&
                       pz <= sk[3] - g;
            if (!open) { h->t = tw; h->kind = HIT_WALL; h->id = wall; }
        }
    }
    if (h->kind == HIT_NONE) return 0;
    for (int k = 0; k < 3; ++k) h->p[k] = o[k] + h->t * d[k];
    if (h->kind == HIT_SPHERE) {
        const double* c = s->sph_c[h->id];
        double r = s->sph[SPH * h->id + 3];
        for (int k = 0; k < 3; ++k) h->n[k] = (h->p[k] - c[k]) / r;
    } else if (h->kind == HIT_BOX) {
        int ax = h->id % 3;
        h->n[0] = h->n[1] = h->n[2] = 0.0;
        const float* bx = s->box + BOX * (h->id / 3);
        double mid = 0.5 * ((double)bx[ax] + (double)bx[3 + ax]);
        h->n[ax] = h->p[ax] > mid ? 1.0 : -1.0;
        h->id /= 3;
    } else {
        int ax = h->id / 2;
        h->n[0] = h->n[1] = h->n[2] = 0.0;
        h->n[ax] = (h->id & 1) ? -1.0 : 1.0;
    }
    return 1;
}

static void albedo_of(const scene_t* s, const hit_t* h, double* a)
{
    const float* src = h->kind == HIT_SPHERE ? s->sph + SPH * h->id + 4
                     : h->kind == HIT_BOX    ? s->box + BOX * h->id + 6
                                             : s->h + 18 + 3 * h->id;
    for (int k = 0; k < 3; ++k) a[k] = src[k];
}

static void emission_of(const scene_t* s, const hit_t* h, double* e)
{
    for (int k = 0; k < 3; ++k)
        e[k] = h->kind == HIT_SPHERE ? s->sph[SPH * h->id + 7 + k] : h->kind == HIT_WALL ? s->h[17] : 0.0;
}

static int sphere_emits(const scene_t* s, int i)
{
    const float* e = s->sph + SPH * i + 7;
    return e[0] > 0.0f || e[1] > 0.0f || e[2] > 0.0f;
}

/* orthonormal basis around unit n (Duff et al., JCGT 2017) */
static void onb(const double* n, double* t, double* b)
{
    double sgn = copysign(1.0, n[2]);
    double a = -1.0 / (sgn + n[2]);
    double bb = n[0] * n[1] * a;
    t[0] = 1.0 + sgn * n[0] * n[0] * a; t[1] = sgn * bb; t[2] = -sgn * n[0];
    b[0] = bb; b[1] = sgn + n[1] * n[1] * a; b[2] = -n[1];
}

/* cosine-distributed direction around n */
static void cosine_dir(const double* n, double u1, double u2, double* w)
{
    double t[3], b[3];
    onb(n, t, b);
    double r = sqrt(u1), phi = 2.0 * M_PI * u2;
    double x = r * cos(phi), y = r * sin(phi), z = sqrt(1.0 - u1 > 0.0 ? 1.0 - u1 : 0.0);
    for (int k = 0; k < 3; ++k) w[k] = x * t[k] + y * b[k] + z * n[k];
}

/*
 * Radiance arriving at o from direction d (the integrand L_i of Eq. 1).
 * first_backface (nullable) reports whether the first hit is a back face.
 */
static void radiance(const scene_t* s, const rng_ctx* rng, uint32_t j, const double* o_in, const double* d_in,
                     int mode, double* L, int* first_hit, int* first_backface)
{
    double o[3] = {o_in[0], o_in[1], o_in[2]}, d[3] = {d_in[0], d_in[1], d_in[2]};
    double beta[3] = {1.0, 1.0, 1.0};
    L[0] = L[1] = L[2] = 0.0;
    *first_hit = 0;
    *first_backface = 0;
    for (int depth = 0; depth < MAX_DEPTH; ++depth) {
        hit_t h;
        if (!intersect(s, o, d, &h)) {
            if (depth > 0 || mode == MC_TOTAL)
                for (int k = 0; k < 3; ++k) L[k] += beta[k] * s->h[10 + k];
            return;
        }
        double cosi = dot3(d, h.n);
        if (depth == 0) { *first_hit = 1; *first_backface = cosi > 0.0; }
        double Le[3];
        emission_of(s, &h, Le);
        int nee_target = h.kind == HIT_SPHERE && sphere_emits(s, h.id);
        int count = depth == 0 ? mode == MC_TOTAL : !nee_target;
        if (count)
            for (int k = 0; k < 3; ++k) L[k] += beta[k] * Le[k];
        double rho[3];
        albedo_of(s, &h, rho);
        if (rho[0] <= 0.0 && rho[1] <= 0.0 && rho[2] <= 0.0) return;
        /* shading normal on the side the ray arrives from */
        double nf[3];
        for (int k = 0; k < 3; ++k) nf[k] = cosi < 0.0 ? h.n[k] : -h.n[k];
        double p[3];
        for (int k = 0; k < 3; ++k) p[k] = h.p[k] + T_EPS * nf[k];
        /* next-event estimation toward each emitting sphere */
        for (int e = 0; e < s->ns; ++e) {
            if (!sphere_emits(s, e)) continue;
            const double* c = s->sph_c[e];
            double r = s->sph[SPH * e + 3];
            double w[3] = {c[0] - p[0], c[1] - p[1], c[2] - p[2]};
            double dist2 = dot3(w, w), dist = sqrt(dist2);
            if (dist <= r) continue;
            for (int k = 0; k < 3; ++k) w[k] /= dist;
            double sin2 = r * r / dist2;
            double cmax = sqrt(1.0 - sin2 > 0.0 ? 1.0 - sin2 : 0.0);
            double u[4];
            draw(rng, j, (uint32_t)depth, 1u + (uint32_t)e, u);
            double ct = 1.0 - u[0] * (1.0 - cmax);
            double st = sqrt(1.0 - ct * ct > 0.0 ? 1.0 - ct * ct : 0.0), phi = 2.0 * M_PI * u[1];
            double tt[3], bb[3], wl[3];
            onb(w, tt, bb);
            for (int k = 0; k < 3; ++k) wl[k] = st * cos(phi) * tt[k] + st * sin(phi) * bb[k] + ct * w[k];
            double cosl = dot3(nf, wl);
            if (cosl <= 0.0) continue;
            hit_t hs;
            if (!intersect(s, p, wl, &hs) || hs.kind != HIT_SPHERE || hs.id != e) continue;
            double pdf_inv = 2.0 * M_PI * (1.0 - cmax);
            const float* Ee = s->sph + SPH * e + 7;
            for (int k = 0; k < 3; ++k) L[k] += beta[k] * (rho[k] / M_PI) * Ee[k] * cosl * pdf_inv;
        }
        double u[4];
        draw(rng, j, (uint32_t)depth, 0u, u);
        /* Russian roulette after three bounces */
        if (depth >= 3) {
            double q = beta[0] > beta[1] ? beta[0] : beta[1];
            q = q > beta[2] ? q : beta[2];
            q = q < 0.95 ? q : 0.95;
            if (u[2] >= q) return;
            for (int k = 0; k < 3; ++k) beta[k] /= q;
        }
        cosine_dir(nf, u[0], u[1], d);
        for (int k = 0; k < 3; ++k) { beta[k] *= rho[k]; o[k] = p[k]; }
    }
}

/*
 * Irradiance at m query points.  x4, n4: [m][4] float records; t (nullable):
 * per-sample time of the rotating sphere.  Sample i uses rng stream i + index_base.
 * out_E: [m][3] doubles; out_keep (nullable): 1 keep / 0 discard.
 */
/*
 * out_se (nullable): per point and channel the standard error of the estimate,
 * pi sqrt(s^2 / spp) with s^2 the sample variance of the spp path radiances.
 */
int orc_mc_irradiance(const float* blob, const float* x4, const float* n4, const float* t, int64_t m, int spp,
                      uint64_t seed, uint64_t index_base, int mode, double* out_E, uint8_t* out_keep, double* out_se)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < m; ++i) {
        scene_t s;
        scene_init(&s, blob, t ? (double)t[i] : 0.0);
        rng_ctx rng = {index_base + (uint64_t)i, seed};
        double x[3] = {x4[4 * i], x4[4 * i + 1], x4[4 * i + 2]};
        double n[3] = {n4[4 * i], n4[4 * i + 1], n4[4 * i + 2]};
        double nl = sqrt(dot3(n, n));
        for (int k = 0; k < 3; ++k) n[k] /= nl;
        double acc[3] = {0.0, 0.0, 0.0}, acc2[3] = {0.0, 0.0, 0.0};
        int hits = 0, back = 0;
        for (int j = 0; j < spp; ++j) {
            double u[4], w[3], L[3];
            draw(&rng, (uint32_t)j, 0xFFFFu, 0u, u);
            cosine_dir(n, u[0], u[1], w);
            int fh, fb;
            radiance(&s, &rng, (uint32_t)j, x, w, mode, L, &fh, &fb);
            hits += fh;
            back += fb;
            for (int k = 0; k < 3; ++k) {
                acc[k] += L[k];
                acc2[k] += L[k] * L[k];
            }
        }
        for (int k = 0; k < 3; ++k) out_E[3 * i + k] = M_PI * acc[k] / (double)spp;
        if (out_se)
            for (int k = 0; k < 3; ++k) {
                double var = spp > 1 ? (acc2[k] - acc[k] * acc[k] / spp) / (spp - 1) : 0.0;
                out_se[3 * i + k] = M_PI * sqrt((var > 0.0 ? var : 0.0) / spp);
            }
        if (out_keep) {
            int zero = out_E[3 * i] == 0.0 && out_E[3 * i + 1] == 0.0 && out_E[3 * i + 2] == 0.0;
            out_keep[i] = (uint8_t)(!(2 * back > spp) && !zero);
        }
    }
    return 0;
}

/*
 * Incoming radiance L_i(x, w) for m (point, direction) pairs, averaged over spp
 * independent paths (used by the probe bake).  Same path rules as above; mode
 * INDIRECT omits emission at the first hit and direct sky.
 */
int orc_mc_radiance(const float* blob, const float* x4, const float* d4, int64_t m, int spp, uint64_t seed,
                    uint64_t index_base, int mode, double* out_L)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < m; ++i) {
        scene_t s;
        scene_init(&s, blob, 0.0);
        rng_ctx rng = {index_base + (uint64_t)i, seed};
        double x[3] = {x4[4 * i], x4[4 * i + 1], x4[4 * i + 2]};
        double w[3] = {d4[4 * i], d4[4 * i + 1], d4[4 * i + 2]};
        double acc[3] = {0.0, 0.0, 0.0};
        for (int j = 0; j < spp; ++j) {
            double L[3];
            int fh, fb;
            radiance(&s, &rng, (uint32_t)j, x, w, mode, L, &fh, &fb);
            for (int k = 0; k < 3; ++k) acc[k] += L[k];
        }
        for (int k = 0; k < 3; ++k) out_L[3 * i + k] = acc[k] / (double)spp;
    }
    return 0;
}

/*
 * Visibility of point p from point o through the scene at parameter t, with every solid
 * thickened by `grow` (the room's walls and the skylight's rim moved inward): 0 when the
 * ray o -> p hits geometry at a distance below |p - o| - end_tol, else 1.
 */
int orc_visible(const float* blob, double t, double grow, const double* o, const double* p, double end_tol)
{
    scene_t s;
    scene_init(&s, blob, t);
    s.grow = grow;
    double d[3] = {p[0] - o[0], p[1] - o[1], p[2] - o[2]};
    double dist = sqrt(dot3(d, d));
    if (!(dist > 0.0)) return 1;
    for (int k = 0; k < 3; ++k) d[k] /= dist;
    hit_t h;
    return !(intersect(&s, o, d, &h) && h.t < dist - end_tol);
}

/* Cosine-distributed direction about unit n from two uniform numbers (for the other oracle files). */
void orc_cosine_dir(const double* n, double u1, double u2, double* w) { cosine_dir(n, u1, u2, w); }
