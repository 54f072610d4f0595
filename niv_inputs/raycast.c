/*
 * Primary-visibility ray cast of the analytic scene (input generation only): the
 * same rules as niv_inputs/gbuffer.py's numpy version, in double precision, one
 * pixel at a time.  Output per pixel: first-hit position, unit normal (facing
 * the camera for walls and box faces, outward for spheres), albedo and a hit flag.
 */
#include <math.h>
#include <stdint.h>

#define HDR 48
#define SPH 12
#define BOX 12

void niv_raycast(const float* blob, int width, int height, double vfov_deg, const double* origin, double* pos,
                 double* nrm, double* alb, uint8_t* hit)
{
    const int ns = (int)blob[0], nb = (int)blob[1], room = blob[2] != 0.0f;
    const float* sph = blob + HDR;
    const float* box = sph + SPH * ns;
    const double th = tan(vfov_deg * M_PI / 180.0 * 0.5), aspect = (double)width / height;
    const double eps = 1e-7;
#pragma omp parallel for schedule(static)
    for (int64_t pix = 0; pix < (int64_t)width * height; ++pix) {
        const int i = (int)(pix % width), j = (int)(pix / width);
        double d[3] = {(2.0 * ((i + 0.5) / width) - 1.0) * th * aspect, (1.0 - 2.0 * ((j + 0.5) / height)) * th, 1.0};
        const double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int k = 0; k < 3; ++k) d[k] /= dl;
        const double* o = origin;
        double tb = INFINITY, n[3] = {0, 0, 0}, a[3] = {0, 0, 0};
        if (room) {
            const float* lo = blob + 4;
            const float* hi = blob + 7;
            int axis = -1, side = 0;
            double tw = INFINITY;
            for (int k = 0; k < 3; ++k) {
                double t = d[k] > 0 ? (hi[k] - o[k]) / d[k] : d[k] < 0 ? (lo[k] - o[k]) / d[k] : INFINITY;
                if (t < tw) { tw = t; axis = k; side = d[k] > 0; }
            }
            const int wall = 2 * axis + side;
            const double px = o[0] + tw * d[0], pz = o[2] + tw * d[2];
            const float* sk = blob + 13;
            const int open = wall == 3 && sk[0] < sk[1] && px >= sk[0] && px <= sk[1] && pz >= sk[2] && pz <= sk[3];
            if (!open) {
                tb = tw;
                n[axis] = side ? -1.0 : 1.0;
                for (int k = 0; k < 3; ++k) a[k] = blob[18 + 3 * wall + k];
            }
        }
        for (int s = 0; s < ns; ++s) {
            const float* S = sph + SPH * s;
            const double oc[3] = {o[0] - S[0], o[1] - S[1], o[2] - S[2]};
            const double b = oc[0] * d[0] + oc[1] * d[1] + oc[2] * d[2];
            const double cc = oc[0] * oc[0] + oc[1] * oc[1] + oc[2] * oc[2] - (double)S[3] * S[3];
            const double disc = b * b - cc;
            const double sq = sqrt(disc > 0.0 ? disc : 0.0);
            double t = -b - sq;
            if (!(t > eps)) t = -b + sq;
            if (disc >= 0 && t > eps && t < tb) {
                tb = t;
                for (int k = 0; k < 3; ++k) {
                    n[k] = (o[k] + t * d[k] - S[k]) / S[3];
                    a[k] = S[4 + k];
                }
            }
        }
        for (int q = 0; q < nb; ++q) {
            const float* B = box + BOX * q;
            double tn[3], tmin = -INFINITY, tmax = INFINITY;
            int ax = 0;
            for (int k = 0; k < 3; ++k) {
                const double t1 = (B[k] - o[k]) / d[k], t2 = (B[3 + k] - o[k]) / d[k];
                tn[k] = t1 < t2 ? t1 : t2;
                const double tf = t1 < t2 ? t2 : t1;
                if (tn[k] > tmin) { tmin = tn[k]; ax = k; }
                if (tf < tmax) tmax = tf;
            }
            if (tmax >= (tmin > eps ? tmin : eps) && tmin > eps && tmin < tb) {
                tb = tmin;
                n[0] = n[1] = n[2] = 0.0;
                n[ax] = d[ax] > 0 ? -1.0 : (d[ax] < 0 ? 1.0 : 0.0);
                for (int k = 0; k < 3; ++k) a[k] = B[6 + k];
            }
        }
        const int h = isfinite(tb);
        hit[pix] = (uint8_t)h;
        for (int k = 0; k < 3; ++k) {
            pos[3 * pix + k] = h ? o[k] + tb * d[k] : 0.0;
            nrm[3 * pix + k] = h ? n[k] : 0.0;
            alb[3 * pix + k] = h ? a[k] : 0.0;
        }
    }
}
