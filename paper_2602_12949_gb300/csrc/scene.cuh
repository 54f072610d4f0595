// The analytic scenes of the training targets and of the probe visibility rays: a room
// (axis-aligned, seen from inside, with an optional open skylight in the ceiling),
// spheres (one of them optionally rotating about +y with the scene parameter t) and
// axis-aligned boxes, in the flat float layout of niv_mc_irradiance's scene argument.
// Geometry runs in FP32.
#pragma once

#include <math.h>
#include <stdint.h>
#include <string.h>

namespace {

constexpr int kHdr = 48, kSph = 12, kBox = 12;
constexpr int kMaxObjects = 56;
constexpr float kTEps = 1e-4f;

struct SceneArg {
    float v[kHdr + kSph * kMaxObjects];
};

struct Hit {
    int kind;  // 0 none, 1 sphere, 2 box, 3 wall
    int id;
    float t;
    float3 p, n;  // n: outward for objects, into the room for walls
};

__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float comp(float3 a, int k) { return k == 0 ? a.x : (k == 1 ? a.y : a.z); }

struct SceneView {
    const float* h;    // the scene description, in shared memory
    const float* sph;
    const float* box;
    int ns, nb, room, rot;
    float3 rotc;       // centre of the rotating sphere at this point's time

    __device__ void init(const float* blob, float t) {
        h = blob;
        ns = (int)blob[0];
        nb = (int)blob[1];
        room = blob[2] != 0.0f;
        sph = blob + kHdr;
        box = sph + kSph * ns;
        rot = (int)blob[3];
        rotc = make_float3(0.0f, 0.0f, 0.0f);
        if (rot >= 0 && rot < ns) {  // rotate by 2 pi t about +y through the axis point
            const float* c = sph + kSph * rot;
            const float a = 6.283185307179586f * t, ca = cosf(a), sa = sinf(a);
            const float dx = c[0] - blob[36], dz = c[2] - blob[38];
            rotc = make_float3(blob[36] + ca * dx + sa * dz, c[1], blob[38] - sa * dx + ca * dz);
        }
    }

    __device__ __forceinline__ float3 centre(int i) const {
        const float* c = sph + kSph * i;
        return i == rot ? rotc : make_float3(c[0], c[1], c[2]);
    }

    __device__ bool emits(int i) const {
        const float* e = sph + kSph * i + 7;
        return e[0] > 0.0f || e[1] > 0.0f || e[2] > 0.0f;
    }

    // Whether the ray o + t d hits anything before tmax, for shadow rays: each object's hit
    // distance is the one intersect takes (the sphere's first root beyond kTEps, the box's
    // entry or exit beyond kTEps, the room's first wall unless it is the open skylight), so
    // the answer is intersect's closest hit t < tmax; the search stops at the first such hit.
    // The slab distances use the ray's reciprocal directions instead of divisions.
    __device__ bool occluded(float3 o, float3 d, float tmax) const {
        for (int i = 0; i < ns; ++i) {
            const float r = sph[kSph * i + 3];
            const float3 ci = centre(i);
            const float3 oc = make_float3(o.x - ci.x, o.y - ci.y, o.z - ci.z);
            const float b = dot3(oc, d), disc = b * b - (dot3(oc, oc) - r * r);
            if (disc < 0.0f) continue;
            const float sq = sqrtf(disc);
            float t = -b - sq;
            if (t <= kTEps) t = -b + sq;
            if (t > kTEps && t < tmax) return true;
        }
        const float3 inv = make_float3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);
        for (int i = 0; i < nb; ++i) {
            const float* B = box + kBox * i;
            const float tx1 = (B[0] - o.x) * inv.x, tx2 = (B[3] - o.x) * inv.x;
            const float ty1 = (B[1] - o.y) * inv.y, ty2 = (B[4] - o.y) * inv.y;
            const float tz1 = (B[2] - o.z) * inv.z, tz2 = (B[5] - o.z) * inv.z;
            const float tn = fmaxf(fmaxf(fminf(tx1, tx2), fminf(ty1, ty2)), fminf(tz1, tz2));
            const float tf = fminf(fminf(fmaxf(tx1, tx2), fmaxf(ty1, ty2)), fmaxf(tz1, tz2));
            if (tf < tn) continue;
            const float t = tn > kTEps ? tn : tf;
            if (t > kTEps && t < tmax) return true;
        }
        if (room) {
            float tw = INFINITY;
            int wall = -1;
            for (int k = 0; k < 3; ++k) {
                const float dk = comp(d, k), ok = comp(o, k);
                float t;
                if (dk > 0.0f) t = (h[7 + k] - ok) * comp(inv, k);
                else if (dk < 0.0f) t = (h[4 + k] - ok) * comp(inv, k);
                else continue;
                if (t < tw) { tw = t; wall = 2 * k + (dk > 0.0f); }
            }
            if (wall >= 0 && tw < tmax) {
                const float px = o.x + tw * d.x, pz = o.z + tw * d.z;
                const float* sk = h + 13;
                const bool open = wall == 3 && sk[0] < sk[1] && px >= sk[0] && px <= sk[1] && pz >= sk[2] && pz <= sk[3];
                if (!open) return true;
            }
        }
        return false;
    }

    __device__ bool intersect(float3 o, float3 d, Hit& hit) const {
        hit.kind = 0;
        hit.t = INFINITY;
        for (int i = 0; i < ns; ++i) {
            const float r = sph[kSph * i + 3];
            const float3 ci = centre(i);
            const float3 oc = make_float3(o.x - ci.x, o.y - ci.y, o.z - ci.z);
            const float b = dot3(oc, d), disc = b * b - (dot3(oc, oc) - r * r);
            if (disc < 0.0f) continue;
            const float sq = sqrtf(disc);
            float t = -b - sq;
            if (t <= kTEps) t = -b + sq;
            if (t > kTEps && t < hit.t) {
                hit.t = t;
                hit.kind = 1;
                hit.id = i;
            }
        }
        const float3 inv = make_float3(1.0f / d.x, 1.0f / d.y, 1.0f / d.z);  // slab distances by multiplication
        for (int i = 0; i < nb; ++i) {
            const float* B = box + kBox * i;
            float tn = -INFINITY, tf = INFINITY;
            int an = 0, af = 0;
            for (int k = 0; k < 3; ++k) {
                const float t1 = (B[k] - comp(o, k)) * comp(inv, k), t2 = (B[3 + k] - comp(o, k)) * comp(inv, k);
                const float lo = fminf(t1, t2), hi = fmaxf(t1, t2);
                if (lo > tn) { tn = lo; an = k; }
                if (hi < tf) { tf = hi; af = k; }
            }
            if (tf < tn) continue;
            float t;
            int ax;
            if (tn > kTEps) { t = tn; ax = an; }
            else if (tf > kTEps) { t = tf; ax = af; }
            else continue;
            if (t < hit.t) {
                hit.t = t;
                hit.kind = 2;
                hit.id = i * 3 + ax;
            }
        }
        if (room) {
            float tw = INFINITY;
            int wall = -1;
            for (int k = 0; k < 3; ++k) {
                const float dk = comp(d, k), ok = comp(o, k);
                float t;
                if (dk > 0.0f) t = (h[7 + k] - ok) * comp(inv, k);
                else if (dk < 0.0f) t = (h[4 + k] - ok) * comp(inv, k);
                else continue;
                if (t < tw) { tw = t; wall = 2 * k + (dk > 0.0f); }
            }
            if (wall >= 0 && tw < hit.t) {
                const float px = o.x + tw * d.x, pz = o.z + tw * d.z;
                const float* sk = h + 13;
                const bool open = wall == 3 && sk[0] < sk[1] && px >= sk[0] && px <= sk[1] && pz >= sk[2] && pz <= sk[3];
                if (!open) {
                    hit.t = tw;
                    hit.kind = 3;
                    hit.id = wall;
                }
            }
        }
        if (hit.kind == 0) return false;
        hit.p = make_float3(o.x + hit.t * d.x, o.y + hit.t * d.y, o.z + hit.t * d.z);
        if (hit.kind == 1) {
            const float r = sph[kSph * hit.id + 3];
            const float3 c = centre(hit.id);
            hit.n = make_float3((hit.p.x - c.x) / r, (hit.p.y - c.y) / r, (hit.p.z - c.z) / r);
        } else if (hit.kind == 2) {
            const int ax = hit.id % 3;
            const float* B = box + kBox * (hit.id / 3);
            const float mid = 0.5f * (B[ax] + B[3 + ax]);
            const float s = comp(hit.p, ax) > mid ? 1.0f : -1.0f;
            hit.n = make_float3(ax == 0 ? s : 0.0f, ax == 1 ? s : 0.0f, ax == 2 ? s : 0.0f);
            hit.id /= 3;
        } else {
            const int ax = hit.id / 2;
            const float s = (hit.id & 1) ? -1.0f : 1.0f;
            hit.n = make_float3(ax == 0 ? s : 0.0f, ax == 1 ? s : 0.0f, ax == 2 ? s : 0.0f);
        }
        return true;
    }

    __device__ float3 albedo(const Hit& hh) const {
        const float* a = hh.kind == 1 ? sph + kSph * hh.id + 4 : hh.kind == 2 ? box + kBox * hh.id + 6 : h + 18 + 3 * hh.id;
        return make_float3(a[0], a[1], a[2]);
    }

    __device__ float3 emission(const Hit& hh) const {
        if (hh.kind == 1) {
            const float* e = sph + kSph * hh.id + 7;
            return make_float3(e[0], e[1], e[2]);
        }
        return hh.kind == 3 ? make_float3(h[17], h[17], h[17]) : make_float3(0.0f, 0.0f, 0.0f);
    }
};

// Scene description copied into a kernel argument (validated by the caller).
inline bool niv_scene_arg(const float* blob, int64_t blob_len, SceneArg& arg) {
    const int ns = (int)blob[0], nb = (int)blob[1];
    if (ns < 0 || nb < 0 || ns + nb > kMaxObjects) return false;
    if (blob_len != kHdr + kSph * ns + kBox * nb) return false;
    memset(&arg, 0, sizeof arg);
    memcpy(arg.v, blob, sizeof(float) * blob_len);
    return true;
}

}  // namespace
