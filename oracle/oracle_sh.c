/*
 * CPU FP64 oracle of the spherical-harmonic probe grid, the non-neural
 * comparison of Sec. 5.1 / App. A.
 *
 * TEST INFRASTRUCTURE ONLY (tests/, the smoke check and the benchmark's CPU
 * baseline).  Shares no source with the CUDA library.
 *
 *  - Per probe, second-order real SH (9 coefficients per colour channel) of the
 *    indirect incident radiance, projected by Monte Carlo with directions uniform
 *    on the sphere: L_lm = (4 pi / S) sum_j L_i(w_j) Y_lm(w_j).  The caller rounds
 *    the coefficients to half precision (54 bytes per probe).
 *  - Irradiance from SH (Ramamoorthi & Hanrahan 2001): E(n) = sum_l A_l sum_m
 *    L_lm Y_lm(n) with A_0 = pi, A_1 = 2 pi / 3, A_2 = pi / 4.
 *  - Query: trilinear weights over the 8 surrounding probes, each multiplied by
 *    the cosine fall-off max(0, n . normalize(p_probe - x)) (a probe exactly at x
 *    keeps factor 1), clamped below at 1e-6, then renormalised (App. A).
 *  - Probes sit at the vertices of a regular P_x x P_y x P_z lattice spanning
 *    the box [lo, hi] (P_k >= 2).
 *  - "+ RT" (Sec. 5.1, App. A): visibility-based rejection replaces the fall-off.
 *    Reading: a ray from x + 0.01 n toward each probe; a probe whose ray hits the
 *    scene more than 0.01 before reaching it gets weight 0, then the 1e-6 clamp and
 *    the renormalisation.  The same test with every solid thickened and thinned by
 *    1e-5 (ten times the FP32 error of these intersections in a 10 m room) flags the
 *    records whose decision depends on rounding (rays grazing an object).
 */
#include <math.h>
#include <stdint.h>

void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]);
int orc_mc_radiance(const float* blob, const float* x4, const float* d4, int64_t m, int spp, uint64_t seed,
                    uint64_t index_base, int mode, double* out_L);
int orc_visible(const float* blob, double t, double grow, const double* o, const double* p, double end_tol);

/* real SH basis, bands 0..2, from the normalised associated Legendre definitions */
void orc_sh9(const double* w, double* Y)
{
    const double x = w[0], y = w[1], z = w[2];
    const double c0 = 0.5 * sqrt(1.0 / M_PI);
    const double c1 = sqrt(3.0 / (4.0 * M_PI));
    const double c2 = 0.5 * sqrt(15.0 / M_PI);
    const double c20 = 0.25 * sqrt(5.0 / M_PI);
    const double c22 = 0.25 * sqrt(15.0 / M_PI);
    Y[0] = c0;
    Y[1] = c1 * y;
    Y[2] = c1 * z;
    Y[3] = c1 * x;
    Y[4] = c2 * x * y;
    Y[5] = c2 * y * z;
    Y[6] = c20 * (3.0 * z * z - 1.0);
    Y[7] = c2 * x * z;
    Y[8] = c22 * (x * x - y * y);
}

/* irradiance E(n) (3 channels) from coefficients c[9][3] */
void orc_sh_irradiance(const double* c, const double* n, double* E)
{
    static const double A[9] = {M_PI, 2.0 * M_PI / 3.0, 2.0 * M_PI / 3.0, 2.0 * M_PI / 3.0,
                                M_PI / 4.0, M_PI / 4.0, M_PI / 4.0, M_PI / 4.0, M_PI / 4.0};
    double Y[9];
    orc_sh9(n, Y);
    for (int k = 0; k < 3; ++k) {
        double s = 0.0;
        for (int i = 0; i < 9; ++i) s += A[i] * c[i * 3 + k] * Y[i];
        E[k] = s;
    }
}

/* SH projection of given radiance samples L[S][3] along directions dirs[S][3] (uniform on S^2) */
void orc_sh_project(const double* dirs, const double* L, int64_t S, double* c)
{
    for (int i = 0; i < 27; ++i) c[i] = 0.0;
    for (int64_t j = 0; j < S; ++j) {
        double Y[9];
        orc_sh9(dirs + 3 * j, Y);
        for (int i = 0; i < 9; ++i)
            for (int k = 0; k < 3; ++k) c[i * 3 + k] += L[3 * j + k] * Y[i];
    }
    for (int i = 0; i < 27; ++i) c[i] *= 4.0 * M_PI / (double)S;
}

static double u01(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0) + (1.0 / 33554432.0); }

/* uniform direction on the sphere for bake ray j of probe p */
static void bake_dir(uint64_t p, uint32_t j, uint64_t seed, double* w)
{
    uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), j + (0xFFFEu << 16), 0u};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t o[4];
    orc_philox4x32_10(ctr, key, o);
    double z = 1.0 - 2.0 * u01(o[0]);
    double r = sqrt(1.0 - z * z > 0.0 ? 1.0 - z * z : 0.0), phi = 2.0 * M_PI * u01(o[1]);
    w[0] = r * cos(phi);
    w[1] = r * sin(phi);
    w[2] = z;
}

static void probe_pos(const int* P, const float* lo, const float* hi, int64_t p, double* x)
{
    int64_t i = p % P[0], j = (p / P[0]) % P[1], k = p / ((int64_t)P[0] * P[1]);
    int64_t ijk[3] = {i, j, k};
    for (int a = 0; a < 3; ++a) x[a] = lo[a] + ((double)hi[a] - lo[a]) * (double)ijk[a] / (double)(P[a] - 1);
}

/*
 * Bake: coefficients out[P][9][3] for every probe (x fastest), `rays` uniform
 * directions per probe, one indirect path each.  Probe p's paths use rng stream
 * index_base + p*rays + j.
 */
/*
 * out_se (nullable): per coefficient the standard error of the estimate,
 * 4 pi sqrt(s^2 / rays) with s^2 the sample variance of L(w_j) Y(w_j) over the rays.
 */
int orc_probe_bake(const float* blob, const int* P, const float* lo, const float* hi, int rays, uint64_t seed,
                   uint64_t index_base, double* out, double* out_se)
{
    int64_t np = (int64_t)P[0] * P[1] * P[2];
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < np; ++p) {
        double x[3];
        probe_pos(P, lo, hi, p, x);
        double c[27], c2[27];
        for (int i = 0; i < 27; ++i) c[i] = c2[i] = 0.0;
        for (int j = 0; j < rays; ++j) {
            double w[3], L[3], Y[9];
            bake_dir(p, (uint32_t)j, seed, w);
            float x4[4] = {(float)x[0], (float)x[1], (float)x[2], 0.0f};
            float d4[4] = {(float)w[0], (float)w[1], (float)w[2], 0.0f};
            orc_mc_radiance(blob, x4, d4, 1, 1, seed, index_base + (uint64_t)p * rays + j, 1, L);
            orc_sh9(w, Y);
            for (int i = 0; i < 9; ++i)
                for (int k = 0; k < 3; ++k) {
                    c[i * 3 + k] += L[k] * Y[i];
                    c2[i * 3 + k] += L[k] * Y[i] * L[k] * Y[i];
                }
        }
        for (int i = 0; i < 27; ++i) out[p * 27 + i] = c[i] * 4.0 * M_PI / (double)rays;
        if (out_se)
            for (int i = 0; i < 27; ++i) {
                double var = rays > 1 ? (c2[i] - c[i] * c[i] / rays) / (rays - 1) : 0.0;
                out_se[p * 27 + i] = 4.0 * M_PI * sqrt((var > 0.0 ? var : 0.0) / rays);
            }
    }
    return 0;
}

/* Query: E[m][3] at (x, n) from coefficients coef[P][9][3] (already rounded by the caller). */
int orc_probe_query(const double* coef, const int* P, const float* lo, const float* hi, const float* x4,
                    const float* n4, int64_t m, double* E)
{
#pragma omp parallel for schedule(static)
    for (int64_t q = 0; q < m; ++q) {
        const float* xq = x4 + 4 * q;
        double nq[3] = {n4[4 * q], n4[4 * q + 1], n4[4 * q + 2]};
        double nl = sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2]);
        for (int a = 0; a < 3; ++a) nq[a] /= nl;
        int64_t base[3];
        double f[3];
        for (int a = 0; a < 3; ++a) {
            double g = ((double)xq[a] - lo[a]) / ((double)hi[a] - lo[a]) * (double)(P[a] - 1);
            if (g < 0.0) g = 0.0;
            if (g > P[a] - 1) g = P[a] - 1;
            int64_t i = (int64_t)floor(g);
            if (i > P[a] - 2) i = P[a] - 2;
            base[a] = i;
            f[a] = g - (double)i;
        }
        double acc[3] = {0.0, 0.0, 0.0}, wsum = 0.0;
        for (int c = 0; c < 8; ++c) {
            int64_t ijk[3];
            double w = 1.0;
            for (int a = 0; a < 3; ++a) {
                int bit = (c >> a) & 1;
                ijk[a] = base[a] + bit;
                w *= bit ? f[a] : 1.0 - f[a];
            }
            int64_t p = ijk[0] + (int64_t)P[0] * (ijk[1] + (int64_t)P[1] * ijk[2]);
            double pp[3];
            probe_pos(P, lo, hi, p, pp);
            double dir[3] = {pp[0] - xq[0], pp[1] - xq[1], pp[2] - xq[2]};
            double dl = sqrt(dir[0] * dir[0] + dir[1] * dir[1] + dir[2] * dir[2]);
            double fall = 1.0;
            if (dl > 0.0) {
                fall = (dir[0] * nq[0] + dir[1] * nq[1] + dir[2] * nq[2]) / dl;
                if (fall < 0.0) fall = 0.0;
            }
            w *= fall;
            if (w < 1e-6) w = 1e-6;
            double Ep[3];
            orc_sh_irradiance(coef + p * 27, nq, Ep);
            for (int k = 0; k < 3; ++k) acc[k] += w * Ep[k];
            wsum += w;
        }
        for (int k = 0; k < 3; ++k) E[3 * q + k] = acc[k] / wsum;
    }
    return 0;
}

/*
 * Query with ray-traced visibility ("+ RT"): as orc_probe_query with the fall-off
 * replaced by the visibility of each probe from x + 0.01 n in scene `blob` at
 * parameter t.  ambiguous[q] (nullable) = 1 when some probe's visibility differs
 * between the scene thickened and thinned by 1e-5.
 */
int orc_probe_query_rt(const double* coef, const int* P, const float* lo, const float* hi, const float* blob,
                       double t, const float* x4, const float* n4, int64_t m, double* E, uint8_t* ambiguous)
{
    const double bias = 0.01, end_tol = 0.01, margin = 1e-5;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t q = 0; q < m; ++q) {
        const float* xq = x4 + 4 * q;
        double nq[3] = {n4[4 * q], n4[4 * q + 1], n4[4 * q + 2]};
        double nl = sqrt(nq[0] * nq[0] + nq[1] * nq[1] + nq[2] * nq[2]);
        for (int a = 0; a < 3; ++a) nq[a] /= nl;
        const double o[3] = {xq[0] + bias * nq[0], xq[1] + bias * nq[1], xq[2] + bias * nq[2]};
        int64_t base[3];
        double f[3];
        for (int a = 0; a < 3; ++a) {
            double g = ((double)xq[a] - lo[a]) / ((double)hi[a] - lo[a]) * (double)(P[a] - 1);
            if (g < 0.0) g = 0.0;
            if (g > P[a] - 1) g = P[a] - 1;
            int64_t i = (int64_t)floor(g);
            if (i > P[a] - 2) i = P[a] - 2;
            base[a] = i;
            f[a] = g - (double)i;
        }
        double acc[3] = {0.0, 0.0, 0.0}, wsum = 0.0;
        int amb = 0;
        for (int c = 0; c < 8; ++c) {
            int64_t ijk[3];
            double w = 1.0;
            for (int a = 0; a < 3; ++a) {
                int bit = (c >> a) & 1;
                ijk[a] = base[a] + bit;
                w *= bit ? f[a] : 1.0 - f[a];
            }
            int64_t p = ijk[0] + (int64_t)P[0] * (ijk[1] + (int64_t)P[1] * ijk[2]);
            double pp[3];
            probe_pos(P, lo, hi, p, pp);
            int vis = orc_visible(blob, t, 0.0, o, pp, end_tol);
            if (ambiguous && orc_visible(blob, t, margin, o, pp, end_tol) != orc_visible(blob, t, -margin, o, pp, end_tol))
                amb = 1;
            if (!vis) w = 0.0;
            if (w < 1e-6) w = 1e-6;
            double Ep[3];
            orc_sh_irradiance(coef + p * 27, nq, Ep);
            for (int k = 0; k < 3; ++k) acc[k] += w * Ep[k];
            wsum += w;
        }
        for (int k = 0; k < 3; ++k) E[3 * q + k] = acc[k] / wsum;
        if (ambiguous) ambiguous[q] = (uint8_t)amb;
    }
    return 0;
}
