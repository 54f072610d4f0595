/*
 * CPU FP64 oracle of the dynamic ambient-occlusion pass (Sec. 4.4: the hemisphere
 * obstruction at the shading point by the dynamic geometry only).
 *
 * TEST INFRASTRUCTURE ONLY (tests/, the smoke check and the benchmark's CPU
 * baseline).  Shares no source with the CUDA library.
 *
 * Reading (the paper gives no formula): from o = x + 0.01 n (n normalised), `rays`
 * cosine-distributed directions about n, direction j from Philox4x32-10 on counter
 * (record lo, record hi, j, 0xA0) with key (seed lo, seed hi), u32 -> (0,1) as in the
 * Monte Carlo oracle; a ray is blocked when it meets a triangle at 0 < t <= R, with the
 * triangle taken as the points v0 + u e1 + v e2, u, v >= 0, u + v <= 1 (Moeller &
 * Trumbore's parametrisation).  AO = 1 - blocked / rays.
 *
 * Plain brute force over the triangles, with two shortcuts that cannot change the
 * answer: a record whose origin lies farther than R from the triangles' bounding box
 * has no ray to test, and a triangle whose bounding sphere lies farther than R from o
 * cannot be met.  Each ray's decision is also taken with every triangle grown and
 * shrunk in u, v and 1 - u - v by an estimate of the FP32 rounding of those parameters,
 * 16 * 2^-24 * (|o| + |v0|) * max(|e1|, |e2|) / |det| (the ray origin and the vertex carry
 * absolute errors of order 2^-24 of their size, magnified by the triangle's shape), and
 * with R moved by 1e-5 R; a record where some decision differs between the two is
 * flagged ambiguous (FP32 arithmetic may decide it either way, e.g. on a shared edge).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]);
void orc_cosine_dir(const double* n, double u1, double u2, double* w);

static double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0) + (1.0 / 33554432.0); }

static double norm3(const double* a) { return sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]); }

/* ray-triangle parameters and the rounding margin of u, v in FP32 (see above); returns 0 when
 * the ray is parallel to the triangle's plane */
static int mt_params(const double* v0, const double* e1, const double* e2, const double* o, const double* d,
                     double* u, double* v, double* t, double* margin)
{
    double p[3] = {d[1] * e2[2] - d[2] * e2[1], d[2] * e2[0] - d[0] * e2[2], d[0] * e2[1] - d[1] * e2[0]};
    double det = e1[0] * p[0] + e1[1] * p[1] + e1[2] * p[2];
    if (det == 0.0) return 0;
    double le = norm3(e1) > norm3(e2) ? norm3(e1) : norm3(e2);
    *margin = 16.0 * ldexp(1.0, -24) * (norm3(o) + norm3(v0)) * le / fabs(det);
    double s[3] = {o[0] - v0[0], o[1] - v0[1], o[2] - v0[2]};
    double q[3] = {s[1] * e1[2] - s[2] * e1[1], s[2] * e1[0] - s[0] * e1[2], s[0] * e1[1] - s[1] * e1[0]};
    *u = (s[0] * p[0] + s[1] * p[1] + s[2] * p[2]) / det;
    *v = (d[0] * q[0] + d[1] * q[1] + d[2] * q[2]) / det;
    *t = (e2[0] * q[0] + e2[1] * q[1] + e2[2] * q[2]) / det;
    return 1;
}

static int inside(double u, double v, double t, double m, double tmax)
{
    return u >= -m && v >= -m && u + v <= 1.0 + m && t > 0.0 && t <= tmax;
}

/*
 * tri9: [T][9] vertices; x4, n4: [m][4] records; out: ao[m] (nullable), blocked[m]
 * (nullable), ambiguous[m] (nullable).
 */
int orc_dyn_ao(const float* tri9, int64_t T, const float* x4, const float* n4, int64_t m, int rays, double R,
               uint64_t seed, double* ao, int32_t* blocked_out, uint8_t* ambiguous)
{
    double lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    double* sph = (double*)malloc(sizeof(double) * 4 * (size_t)(T > 0 ? T : 1));
    for (int64_t i = 0; i < T; ++i) {
        const float* t = tri9 + 9 * i;
        double c[3];
        for (int k = 0; k < 3; ++k) {
            c[k] = ((double)t[k] + t[3 + k] + t[6 + k]) / 3.0;
            for (int v = 0; v < 3; ++v) {
                if (t[3 * v + k] < lo[k]) lo[k] = t[3 * v + k];
                if (t[3 * v + k] > hi[k]) hi[k] = t[3 * v + k];
            }
        }
        double r2 = 0.0;
        for (int v = 0; v < 3; ++v) {
            double d2 = 0.0;
            for (int k = 0; k < 3; ++k) d2 += (t[3 * v + k] - c[k]) * (t[3 * v + k] - c[k]);
            if (d2 > r2) r2 = d2;
        }
        sph[4 * i] = c[0];
        sph[4 * i + 1] = c[1];
        sph[4 * i + 2] = c[2];
        sph[4 * i + 3] = sqrt(r2);
    }
    const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
#pragma omp parallel
    {
        int64_t* cand = (int64_t*)malloc(sizeof(int64_t) * (size_t)(T > 0 ? T : 1));
#pragma omp for schedule(dynamic, 16)
        for (int64_t q = 0; q < m; ++q) {
            double n[3] = {n4[4 * q], n4[4 * q + 1], n4[4 * q + 2]};
            double nl = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            for (int k = 0; k < 3; ++k) n[k] /= nl;
            double o[3];
            for (int k = 0; k < 3; ++k) o[k] = (double)x4[4 * q + k] + 0.01 * n[k];
            double g2 = 0.0;
            for (int k = 0; k < 3; ++k) {
                double g = lo[k] - o[k] > o[k] - hi[k] ? lo[k] - o[k] : o[k] - hi[k];
                if (g > 0.0) g2 += g * g;
            }
            int blocked = 0, amb = 0;
            if (T > 0 && g2 <= R * R) {
                int64_t nc = 0;
                for (int64_t i = 0; i < T; ++i) {
                    double d2 = 0.0;
                    for (int k = 0; k < 3; ++k) d2 += (sph[4 * i + k] - o[k]) * (sph[4 * i + k] - o[k]);
                    double reach = R * (1.0 + 1e-5) + sph[4 * i + 3];
                    if (d2 <= reach * reach) cand[nc++] = i;
                }
                for (int j = 0; j < rays && nc > 0; ++j) {
                    uint32_t ctr[4] = {(uint32_t)q, (uint32_t)((uint64_t)q >> 32), (uint32_t)j, 0xA0u}, r4[4];
                    orc_philox4x32_10(ctr, key, r4);
                    double d[3];
                    orc_cosine_dir(n, u01(r4[0]), u01(r4[1]), d);
                    int hit = 0, grown = 0, shrunk = 0;
                    for (int64_t c = 0; c < nc; ++c) {
                        const float* t = tri9 + 9 * cand[c];
                        double v0[3] = {t[0], t[1], t[2]};
                        double e1[3] = {(double)t[3] - t[0], (double)t[4] - t[1], (double)t[5] - t[2]};
                        double e2[3] = {(double)t[6] - t[0], (double)t[7] - t[1], (double)t[8] - t[2]};
                        double u, v, tt, mg;
                        if (!mt_params(v0, e1, e2, o, d, &u, &v, &tt, &mg)) continue;
                        hit |= inside(u, v, tt, 0.0, R);
                        grown |= inside(u, v, tt, mg, R * (1.0 + 1e-5));
                        shrunk |= inside(u, v, tt, -mg, R * (1.0 - 1e-5));
                    }
                    blocked += hit;
                    if (grown != shrunk) amb = 1;
                }
            }
            if (ao) ao[q] = 1.0 - (double)blocked / (double)rays;
            if (blocked_out) blocked_out[q] = blocked;
            if (ambiguous) ambiguous[q] = (uint8_t)amb;
        }
        free(cand);
    }
    free(sph);
    return 0;
}
