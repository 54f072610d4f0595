/*
 * Training-sample candidates of Sec. 4.5 / App. I: a fraction of the points lie on
 * the scene's surfaces, taking the surface normal as their direction; the rest are
 * uniform in the room with directions uniform on the sphere.  Surface points are
 * spread over the surfaces in proportion to area.
 *
 * TEST INFRASTRUCTURE ONLY (tests/, the smoke check and the benchmark's CPU
 * baseline).  Shares no source with the CUDA library.
 *
 * Definition (written from the description above, the steps in order):
 *  - surfaces ("patches"), in this order: the six room walls (axis 0..2, the wall
 *    at room_min first, normal into the room), the ceiling (axis 1 at room_max)
 *    cut around the open skylight [x0,x1] x [z0,z1] into the strips
 *    x <= x0, x >= x1, (x0..x1, z <= z0), (x0..x1, z >= z1), empty strips left out;
 *    then every sphere that does not emit (at its rest position), area 4 pi r^2;
 *    then every box face (axis 0..2, the face at the box's low corner first,
 *    outward normal).  cdf[k] = float(sum_{j<=k} area_j / total) with the sums in
 *    double, cdf[last] = 1.
 *  - sample i draws Philox4x32-10 at counter (j lo, j hi, 0x53414D50, 0) and
 *    (j lo, j hi, 0x53414D50, 1), j = index_base + i, key (seed lo, seed hi):
 *    r0..r7; u(r) = float(r >> 8) 2^-24 + 2^-25 in FP32.
 *  - surface iff u(r0) < surface_frac.  Volume: p_k = lo_k + (hi_k - lo_k) u(r_{1+k})
 *    (FP32, product then sum), direction uniform on the sphere from u(r4), u(r5):
 *    z = 1 - 2u, phi = 2 pi u', d = (sqrt(1 - z^2) cos phi, sqrt(1 - z^2) sin phi, z).
 *    Surface: patch k = first k with u(r1) < cdf[k]; on a wall or box face the two
 *    in-plane coordinates (increasing axis order) are a0 + (a1 - a0) u(r2) and
 *    b0 + (b1 - b0) u(r3) (FP32), the third the plane's; on a sphere p = c + r d
 *    with d from u(r4), u(r5) as above and n = d.
 *  - t = u(r6) when a per-sample scene parameter is asked for.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define S_HDR 48
#define S_SPH 12
#define S_BOX 12

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]);

typedef struct {
    int kind;      /* 0 rectangle, 1 sphere */
    int axis;      /* rectangle: the plane's axis */
    float sign;    /* rectangle: normal = sign * e_axis */
    float plane;   /* rectangle: coordinate along axis */
    float a0, a1, b0, b1;  /* rectangle: bounds along the two other axes, increasing axis order */
    float c[3], r; /* sphere */
    double area;
} patch_t;

static float uf(uint32_t x) { return (float)(x >> 8) * (1.0f / 16777216.0f) + (1.0f / 33554432.0f); }

static void rect(patch_t* p, int axis, float sign, float plane, float a0, float a1, float b0, float b1)
{
    memset(p, 0, sizeof *p);
    p->kind = 0;
    p->axis = axis;
    p->sign = sign;
    p->plane = plane;
    p->a0 = a0;
    p->a1 = a1;
    p->b0 = b0;
    p->b1 = b1;
    p->area = ((double)a1 - (double)a0) * ((double)b1 - (double)b0);
}

/* The patch list of a scene description; returns the count (<= cap) or -1. */
int orc_sample_patches(const float* blob, int64_t blob_len, patch_t* out, int cap)
{
    const int ns = (int)blob[0], nb = (int)blob[1];
    if (ns < 0 || nb < 0 || blob_len != S_HDR + S_SPH * ns + S_BOX * nb) return -1;
    const float* lo = blob + 4;
    const float* hi = blob + 7;
    const float* sky = blob + 13; /* x0 x1 z0 z1 */
    int k = 0;
    if (blob[2] != 0.0f) {
        for (int axis = 0; axis < 3; ++axis) {
            const int a = axis == 0 ? 1 : 0, b = axis == 2 ? 1 : 2;
            for (int side = 0; side < 2; ++side) {
                const int ceiling = axis == 1 && side == 1;
                if (ceiling && sky[0] < sky[1]) {
                    /* a = x (0), b = z (2) */
                    if (k + 4 > cap) return -1;
                    if (sky[0] > lo[0]) rect(&out[k++], 1, -1.0f, hi[1], lo[0], sky[0], lo[2], hi[2]);
                    if (hi[0] > sky[1]) rect(&out[k++], 1, -1.0f, hi[1], sky[1], hi[0], lo[2], hi[2]);
                    if (sky[2] > lo[2]) rect(&out[k++], 1, -1.0f, hi[1], sky[0], sky[1], lo[2], sky[2]);
                    if (hi[2] > sky[3]) rect(&out[k++], 1, -1.0f, hi[1], sky[0], sky[1], sky[3], hi[2]);
                    continue;
                }
                if (k + 1 > cap) return -1;
                rect(&out[k++], axis, side ? -1.0f : 1.0f, side ? hi[axis] : lo[axis], lo[a], hi[a], lo[b], hi[b]);
            }
        }
    }
    const float* sph = blob + S_HDR;
    for (int i = 0; i < ns; ++i) {
        const float* s = sph + S_SPH * i;
        if (s[7] > 0.0f || s[8] > 0.0f || s[9] > 0.0f) continue; /* emitters are not shaded */
        if (k + 1 > cap) return -1;
        memset(&out[k], 0, sizeof out[k]);
        out[k].kind = 1;
        out[k].c[0] = s[0];
        out[k].c[1] = s[1];
        out[k].c[2] = s[2];
        out[k].r = s[3];
        out[k].area = 4.0 * M_PI * (double)s[3] * (double)s[3];
        ++k;
    }
    const float* box = sph + S_SPH * ns;
    for (int i = 0; i < nb; ++i) {
        const float* bl = box + S_BOX * i;
        const float* bh = bl + 3;
        for (int axis = 0; axis < 3; ++axis) {
            const int a = axis == 0 ? 1 : 0, b = axis == 2 ? 1 : 2;
            for (int side = 0; side < 2; ++side) {
                if (k + 1 > cap) return -1;
                rect(&out[k++], axis, side ? 1.0f : -1.0f, side ? bh[axis] : bl[axis], bl[a], bh[a], bl[b], bh[b]);
            }
        }
    }
    return k;
}

static void sphere_dir(float u4, float u5, double d[3])
{
    const double z = 1.0 - 2.0 * (double)u4, phi = 2.0 * M_PI * (double)u5;
    const double s = sqrt(fmax(0.0, 1.0 - z * z));
    d[0] = s * cos(phi);
    d[1] = s * sin(phi);
    d[2] = z;
}

/*
 * n candidates: x4, n4 float [n][4] (pad 0), t float [n] (NULL: none), patch int [n]
 * (NULL: none; -1 for volume samples, else the patch index).  Returns the number of
 * patches, or -1 for a bad scene description.
 */
int orc_training_samples(const float* blob, int64_t blob_len, int64_t n, float surface_frac, uint64_t seed,
                         uint64_t index_base, float* x4, float* n4, float* t, int32_t* patch)
{
    patch_t* P = (patch_t*)malloc(sizeof(patch_t) * 512);
    const int K = orc_sample_patches(blob, blob_len, P, 512);
    if (K < 0) {
        free(P);
        return -1;
    }
    float* cdf = (float*)malloc(sizeof(float) * (K > 0 ? K : 1));
    double total = 0.0;
    for (int k = 0; k < K; ++k) total += P[k].area;
    double acc = 0.0;
    for (int k = 0; k < K; ++k) {
        acc += P[k].area;
        cdf[k] = (float)(acc / total);
    }
    if (K > 0) cdf[K - 1] = 1.0f;
    const float* lo = blob + 4;
    const float* hi = blob + 7;
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        const uint64_t j = index_base + (uint64_t)i;
        uint32_t c0[4] = {(uint32_t)j, (uint32_t)(j >> 32), 0x53414D50u, 0u}, c1[4] = {(uint32_t)j, (uint32_t)(j >> 32),
                                                                                      0x53414D50u, 1u};
        uint32_t r[8];
        orc_philox4x32_10(c0, key, r);
        orc_philox4x32_10(c1, key, r + 4);
        float p[3], q[3];
        int which = -1;
        if (K > 0 && uf(r[0]) < surface_frac) {
            const float u1 = uf(r[1]);
            int k = 0;
            while (k < K - 1 && !(u1 < cdf[k])) ++k;
            which = k;
            const patch_t* pp = &P[k];
            if (pp->kind == 0) {
                const int a = pp->axis == 0 ? 1 : 0, b = pp->axis == 2 ? 1 : 2;
                const float ea = pp->a1 - pp->a0, eb = pp->b1 - pp->b0;
                const float pa = ea * uf(r[2]), pb = eb * uf(r[3]);
                p[a] = pp->a0 + pa;
                p[b] = pp->b0 + pb;
                p[pp->axis] = pp->plane;
                q[0] = q[1] = q[2] = 0.0f;
                q[pp->axis] = pp->sign;
            } else {
                double d[3];
                sphere_dir(uf(r[4]), uf(r[5]), d);
                for (int m = 0; m < 3; ++m) {
                    p[m] = (float)((double)pp->c[m] + (double)pp->r * d[m]);
                    q[m] = (float)d[m];
                }
            }
        } else {
            for (int m = 0; m < 3; ++m) {
                const float e = hi[m] - lo[m], s = e * uf(r[1 + m]);
                p[m] = lo[m] + s;
            }
            double d[3];
            sphere_dir(uf(r[4]), uf(r[5]), d);
            for (int m = 0; m < 3; ++m) q[m] = (float)d[m];
        }
        for (int m = 0; m < 3; ++m) {
            x4[4 * i + m] = p[m];
            n4[4 * i + m] = q[m];
        }
        x4[4 * i + 3] = 0.0f;
        n4[4 * i + 3] = 0.0f;
        if (t) t[i] = uf(r[6]);
        if (patch) patch[i] = which;
    }
    free(cdf);
    free(P);
    return K;
}

/* Patch table for tests: per patch kind, axis, sign, plane, a0, a1, b0, b1, cx, cy, cz, r, area. */
int orc_sample_patch_table(const float* blob, int64_t blob_len, double* out13, int cap)
{
    patch_t* P = (patch_t*)malloc(sizeof(patch_t) * 512);
    const int K = orc_sample_patches(blob, blob_len, P, 512);
    for (int k = 0; k < K && k < cap; ++k) {
        double* o = out13 + 13 * k;
        o[0] = P[k].kind;
        o[1] = P[k].axis;
        o[2] = P[k].sign;
        o[3] = P[k].plane;
        o[4] = P[k].a0;
        o[5] = P[k].a1;
        o[6] = P[k].b0;
        o[7] = P[k].b1;
        o[8] = P[k].c[0];
        o[9] = P[k].c[1];
        o[10] = P[k].c[2];
        o[11] = P[k].r;
        o[12] = P[k].area;
    }
    free(P);
    return K;
}
