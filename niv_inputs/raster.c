/*
 * Insert triangle meshes into an existing G-buffer (input generation only).
 *
 * For every triangle: project its vertices with the pinhole camera, visit the
 * pixels of its screen bounding box, and intersect each pixel's camera ray with the
 * triangle (Moeller-Trumbore, double precision).  A hit closer than the pixel's
 * current surface replaces position, normal (the face normal turned toward the
 * camera) and albedo.  Triangles with a vertex behind the camera are skipped.
 */
#include <math.h>
#include <stdint.h>

void niv_raster_meshes(const double* verts, const int32_t* tris, const int32_t* tri_mesh, int64_t n_tris,
                       const double* mesh_albedo, int width, int height, double vfov_deg, const double* cam,
                       double* pos, double* nrm, double* alb, uint8_t* hit, int32_t* mesh_id)
{
    const double th = tan(vfov_deg * M_PI / 180.0 * 0.5), aspect = (double)width / height;
    for (int64_t f = 0; f < n_tris; ++f) {
        const double* A = verts + 3 * tris[3 * f];
        const double* B = verts + 3 * tris[3 * f + 1];
        const double* C = verts + 3 * tris[3 * f + 2];
        const double* V[3] = {A, B, C};
        double imin = 1e30, imax = -1e30, jmin = 1e30, jmax = -1e30;
        int behind = 0;
        for (int k = 0; k < 3; ++k) {
            const double dx = V[k][0] - cam[0], dy = V[k][1] - cam[1], dz = V[k][2] - cam[2];
            if (dz <= 1e-3) { behind = 1; break; }
            const double sx = dx / dz / (th * aspect), sy = dy / dz / th;
            const double pi = (sx + 1.0) * 0.5 * width - 0.5, pj = (1.0 - sy) * 0.5 * height - 0.5;
            if (pi < imin) imin = pi;
            if (pi > imax) imax = pi;
            if (pj < jmin) jmin = pj;
            if (pj > jmax) jmax = pj;
        }
        if (behind) continue;
        int i0 = (int)floor(imin), i1 = (int)ceil(imax), j0 = (int)floor(jmin), j1 = (int)ceil(jmax);
        if (i0 < 0) i0 = 0;
        if (j0 < 0) j0 = 0;
        if (i1 > width - 1) i1 = width - 1;
        if (j1 > height - 1) j1 = height - 1;
        const double e1[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        const double e2[3] = {C[0] - A[0], C[1] - A[1], C[2] - A[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        const double nl = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(nl > 0.0)) continue;
        for (int k = 0; k < 3; ++k) n[k] /= nl;
        for (int j = j0; j <= j1; ++j)
            for (int i = i0; i <= i1; ++i) {
                double d[3] = {(2.0 * ((i + 0.5) / width) - 1.0) * th * aspect, (1.0 - 2.0 * ((j + 0.5) / height)) * th, 1.0};
                const double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
                for (int k = 0; k < 3; ++k) d[k] /= dl;
                const double p[3] = {d[1] * e2[2] - d[2] * e2[1], d[2] * e2[0] - d[0] * e2[2], d[0] * e2[1] - d[1] * e2[0]};
                const double det = e1[0] * p[0] + e1[1] * p[1] + e1[2] * p[2];
                if (fabs(det) < 1e-14) continue;
                const double inv = 1.0 / det;
                const double s[3] = {cam[0] - A[0], cam[1] - A[1], cam[2] - A[2]};
                const double u = (s[0] * p[0] + s[1] * p[1] + s[2] * p[2]) * inv;
                if (u < 0.0 || u > 1.0) continue;
                const double q[3] = {s[1] * e1[2] - s[2] * e1[1], s[2] * e1[0] - s[0] * e1[2], s[0] * e1[1] - s[1] * e1[0]};
                const double v = (d[0] * q[0] + d[1] * q[1] + d[2] * q[2]) * inv;
                if (v < 0.0 || u + v > 1.0) continue;
                const double t = (e2[0] * q[0] + e2[1] * q[1] + e2[2] * q[2]) * inv;
                if (t <= 1e-6) continue;
                const int64_t pix = (int64_t)j * width + i;
                double tcur = INFINITY;
                if (hit[pix]) {
                    const double* P = pos + 3 * pix;
                    tcur = sqrt((P[0] - cam[0]) * (P[0] - cam[0]) + (P[1] - cam[1]) * (P[1] - cam[1]) +
                                (P[2] - cam[2]) * (P[2] - cam[2]));
                }
                if (t >= tcur) continue;
                const double sg = (n[0] * d[0] + n[1] * d[1] + n[2] * d[2]) > 0.0 ? -1.0 : 1.0;
                const int mesh = tri_mesh[f];
                for (int k = 0; k < 3; ++k) {
                    pos[3 * pix + k] = cam[k] + t * d[k];
                    nrm[3 * pix + k] = sg * n[k];
                    alb[3 * pix + k] = mesh_albedo[3 * mesh + k];
                }
                hit[pix] = 1;
                mesh_id[pix] = mesh;
            }
    }
}
