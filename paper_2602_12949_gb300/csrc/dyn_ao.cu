// Dynamic ambient occlusion (Sec. 4.4): the hemisphere obstruction at the shading point by
// the dynamic (inserted) geometry only, which NIV does not know about; it darkens the
// dynamic objects themselves (self-occlusion) and the static surfaces next to them.
//
// Reading (the paper gives no formula): from o = x + 0.01 n (world units, n normalised)
// K cosine-distributed directions about n, drawn from Philox4x32-10 on counter
// (record lo, record hi, ray j, 0xA0) with key (seed lo, seed hi); a ray is blocked when
// it hits a dynamic triangle at 0 < t <= R (Moeller-Trumbore).  AO = 1 - blocked / K, and
// the irradiance is scaled, E <- AO E, before shading.
//
// The triangles (world space, as posed for the frame) are put into a bounding-volume
// hierarchy on the host: binned surface-area-heuristic splits of the centroids (16 bins per
// axis), leaves of at most 4 triangles or where no split pays (up to 16), nodes in
// depth-first order (left child next to its parent), bounds
// padded by 1e-5 of the scene's extent.  On the device every inner node holds the boxes of
// both its children, so one step tests two boxes; one thread per record traverses it with a
// stack, leaves of hit children first, then the hit inner child that the ray enters first
// (any hit ends the ray); records whose ray origin lies farther than R from every depth-3
// node box skip the rays (AO = 1).
#include <algorithm>
#include <cmath>
#include <vector>

#include "niv_internal.cuh"
#include "sampling.cuh"

constexpr int kCullBoxes = 8;  // node boxes at depth 3: a record traces rays only within R of one

struct niv_dyn {
    int device;
    int64_t n_tris, n_nodes;  // n_nodes: nodes of the binary hierarchy
    // per inner node, for each of its two children: (lo.xyz, ref), (hi.xyz, count);
    // count > 0: a leaf of `count` triangles from `ref`; 0: the inner node `ref`;
    // < 0: no child (a leaf root's second slot)
    float4* nodes;
    float4* tris;  // per triangle: v0, e1 = v1 - v0, e2 = v2 - v0
    int n_cull;
    float cull_lo[kCullBoxes][3], cull_hi[kCullBoxes][3];
};

namespace {

struct HostNode {
    float lo[3], hi[3];
    int32_t a, b;
};

inline float box_area(const float* lo, const float* hi) {
    const float dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    return dx * dy + dy * dz + dz * dx;
}

struct Builder {
    const float* tri;  // [T][9]
    std::vector<float> cen;
    std::vector<int32_t> order;
    std::vector<HostNode> nodes;
    float pad;

    int32_t build(int32_t b, int32_t e, int depth) {
        const int32_t me = (int32_t)nodes.size();
        nodes.push_back(HostNode());
        HostNode nd;
        float clo[3], chi[3];
        for (int k = 0; k < 3; ++k) {
            nd.lo[k] = clo[k] = INFINITY;
            nd.hi[k] = chi[k] = -INFINITY;
        }
        for (int32_t i = b; i < e; ++i) {
            const float* t = tri + 9 * (int64_t)order[i];
            for (int v = 0; v < 3; ++v)
                for (int k = 0; k < 3; ++k) {
                    nd.lo[k] = std::min(nd.lo[k], t[3 * v + k]);
                    nd.hi[k] = std::max(nd.hi[k], t[3 * v + k]);
                }
            for (int k = 0; k < 3; ++k) {
                clo[k] = std::min(clo[k], cen[3 * (int64_t)order[i] + k]);
                chi[k] = std::max(chi[k], cen[3 * (int64_t)order[i] + k]);
            }
        }
        for (int k = 0; k < 3; ++k) {
            nd.lo[k] -= pad;
            nd.hi[k] += pad;
        }
        int axis = 0;
        for (int k = 1; k < 3; ++k)
            if (chi[k] - clo[k] > chi[axis] - clo[axis]) axis = k;
        if (e - b <= 4 || !(chi[axis] > clo[axis]) || depth >= 60) {
            nd.a = b;
            nd.b = e - b;
            nodes[me] = nd;
            return me;
        }
        // binned surface-area heuristic: for 16 centroid bins per axis, the split whose two
        // sides minimise area x count; a leaf when no split beats testing every triangle
        constexpr int kBins = 16;
        float best = INFINITY;
        int best_axis = axis, best_bin = kBins / 2;
        for (int k = 0; k < 3; ++k) {
            if (!(chi[k] > clo[k])) continue;
            const float scale = kBins / (chi[k] - clo[k]);
            int cnt[kBins] = {0};
            float blo[kBins][3], bhi[kBins][3];
            for (int i = 0; i < kBins; ++i)
                for (int c = 0; c < 3; ++c) {
                    blo[i][c] = INFINITY;
                    bhi[i][c] = -INFINITY;
                }
            for (int32_t i = b; i < e; ++i) {
                const int64_t t = order[i];
                const int bin = std::min(kBins - 1, (int)((cen[3 * t + k] - clo[k]) * scale));
                ++cnt[bin];
                for (int v = 0; v < 3; ++v)
                    for (int c = 0; c < 3; ++c) {
                        blo[bin][c] = std::min(blo[bin][c], tri[9 * t + 3 * v + c]);
                        bhi[bin][c] = std::max(bhi[bin][c], tri[9 * t + 3 * v + c]);
                    }
            }
            float right_area[kBins];
            int right_cnt[kBins];
            float rl[3] = {INFINITY, INFINITY, INFINITY}, rh[3] = {-INFINITY, -INFINITY, -INFINITY};
            int rc = 0;
            for (int i = kBins - 1; i > 0; --i) {
                rc += cnt[i];
                for (int c = 0; c < 3; ++c) {
                    rl[c] = std::min(rl[c], blo[i][c]);
                    rh[c] = std::max(rh[c], bhi[i][c]);
                }
                right_cnt[i] = rc;
                right_area[i] = rc ? box_area(rl, rh) : 0.0f;
            }
            float ll[3] = {INFINITY, INFINITY, INFINITY}, lh[3] = {-INFINITY, -INFINITY, -INFINITY};
            int lc = 0;
            for (int i = 0; i < kBins - 1; ++i) {
                lc += cnt[i];
                for (int c = 0; c < 3; ++c) {
                    ll[c] = std::min(ll[c], blo[i][c]);
                    lh[c] = std::max(lh[c], bhi[i][c]);
                }
                if (lc == 0 || right_cnt[i + 1] == 0) continue;
                const float cost = lc * box_area(ll, lh) + right_cnt[i + 1] * right_area[i + 1];
                if (cost < best) {
                    best = cost;
                    best_axis = k;
                    best_bin = i;
                }
            }
        }
        const float leaf_cost = (float)(e - b) * box_area(nd.lo, nd.hi);
        if (!(best < INFINITY) || (e - b <= 16 && best >= leaf_cost)) {
            nd.a = b;
            nd.b = e - b;
            nodes[me] = nd;
            return me;
        }
        axis = best_axis;
        const float scale = kBins / (chi[axis] - clo[axis]);
        int32_t mid = (int32_t)(std::partition(order.begin() + b, order.begin() + e, [&](int32_t t) {
                                    return std::min(kBins - 1, (int)((cen[3 * (int64_t)t + axis] - clo[axis]) * scale)) <=
                                           best_bin;
                                }) - order.begin());
        if (mid == b || mid == e) {  // cannot happen for a split with both sides counted; median as a guard
            mid = b + (e - b) / 2;
            std::nth_element(order.begin() + b, order.begin() + mid, order.begin() + e, [&](int32_t x, int32_t y) {
                return cen[3 * (int64_t)x + axis] < cen[3 * (int64_t)y + axis];
            });
        }
        build(b, mid, depth + 1);
        nd.a = build(mid, e, depth + 1);
        nd.b = -(axis + 1);
        nodes[me] = nd;
        return me;
    }
};

// Boxes of the nodes at depth 3 (or of shallower leaves): together they hold every triangle.
void collect_cull(const std::vector<HostNode>& nodes, int32_t i, int depth, std::vector<int32_t>& out) {
    const HostNode& n = nodes[(size_t)i];
    if (depth == 3 || n.b > 0) {
        out.push_back(i);
        return;
    }
    collect_cull(nodes, i + 1, depth + 1, out);
    collect_cull(nodes, n.a, depth + 1, out);
}

constexpr int kStack = 64;
constexpr float kRayBias = 0.01f;

// Moeller-Trumbore: hit at 0 < t <= tmax inside the triangle (v0, e1, e2).
__device__ __forceinline__ bool tri_hit(const float4& v0, const float4& e1, const float4& e2, float3 o, float3 d,
                                        float tmax) {
    const float px = d.y * e2.z - d.z * e2.y, py = d.z * e2.x - d.x * e2.z, pz = d.x * e2.y - d.y * e2.x;
    const float det = e1.x * px + e1.y * py + e1.z * pz;
    if (det == 0.0f) return false;
    const float inv = 1.0f / det;
    const float sx = o.x - v0.x, sy = o.y - v0.y, sz = o.z - v0.z;
    const float u = (sx * px + sy * py + sz * pz) * inv;
    if (u < 0.0f || u > 1.0f) return false;
    const float qx = sy * e1.z - sz * e1.y, qy = sz * e1.x - sx * e1.z, qz = sx * e1.y - sy * e1.x;
    const float v = (d.x * qx + d.y * qy + d.z * qz) * inv;
    if (v < 0.0f || u + v > 1.0f) return false;
    const float t = (e2.x * qx + e2.y * qy + e2.z * qz) * inv;
    return t > 0.0f && t <= tmax;
}

// Entry distance of the ray o + t d, t in [0, tmax], into a node box (inv: finite
// reciprocals of d, oi = o * inv); false when it misses.  The box bounds are padded, so
// the FMA's rounding cannot lose a hit.
__device__ __forceinline__ bool box_enter(const float4& lo, const float4& hi, float3 oi, float3 inv, float tmax,
                                          float& tn) {
    const float tx0 = fmaf(lo.x, inv.x, -oi.x), tx1 = fmaf(hi.x, inv.x, -oi.x);
    const float ty0 = fmaf(lo.y, inv.y, -oi.y), ty1 = fmaf(hi.y, inv.y, -oi.y);
    const float tz0 = fmaf(lo.z, inv.z, -oi.z), tz1 = fmaf(hi.z, inv.z, -oi.z);
    tn = fmaxf(fmaxf(fminf(tx0, tx1), fminf(ty0, ty1)), fmaxf(fminf(tz0, tz1), 0.0f));
    const float tf = fminf(fminf(fmaxf(tx0, tx1), fmaxf(ty0, ty1)), fminf(fmaxf(tz0, tz1), tmax));
    return tn <= tf;
}

__device__ __forceinline__ bool leaf_hit(const float4* __restrict__ tris, int first, int count, float3 o, float3 d,
                                         float tmax) {
    for (int i = first; i < first + count; ++i)
        if (tri_hit(__ldg(tris + 3 * i), __ldg(tris + 3 * i + 1), __ldg(tris + 3 * i + 2), o, d, tmax)) return true;
    return false;
}

__device__ bool any_hit(const float4* __restrict__ nodes, const float4* __restrict__ tris, float3 o, float3 d,
                        float tmax) {
    const float3 inv = make_float3(1.0f / (fabsf(d.x) > 1e-20f ? d.x : copysignf(1e-20f, d.x)),
                                   1.0f / (fabsf(d.y) > 1e-20f ? d.y : copysignf(1e-20f, d.y)),
                                   1.0f / (fabsf(d.z) > 1e-20f ? d.z : copysignf(1e-20f, d.z)));
    const float3 oi = make_float3(o.x * inv.x, o.y * inv.y, o.z * inv.z);
    int stack[kStack];
    int sp = 0, node = 0;
    while (true) {
        const float4 l0 = __ldg(nodes + 4 * node), h0 = __ldg(nodes + 4 * node + 1);
        const float4 l1 = __ldg(nodes + 4 * node + 2), h1 = __ldg(nodes + 4 * node + 3);
        const int r0 = __float_as_int(l0.w), c0 = __float_as_int(h0.w);
        const int r1 = __float_as_int(l1.w), c1 = __float_as_int(h1.w);
        float t0, t1;
        const bool in0 = c0 >= 0 && box_enter(l0, h0, oi, inv, tmax, t0);
        const bool in1 = c1 >= 0 && box_enter(l1, h1, oi, inv, tmax, t1);
        if (in0 && c0 > 0 && leaf_hit(tris, r0, c0, o, d, tmax)) return true;
        if (in1 && c1 > 0 && leaf_hit(tris, r1, c1, o, d, tmax)) return true;
        const bool go0 = in0 && c0 == 0, go1 = in1 && c1 == 0;
        if (go0 && go1) {
            const bool first0 = t0 <= t1;
            if (sp < kStack) stack[sp++] = first0 ? r1 : r0;  // the builder caps the depth at 60
            node = first0 ? r0 : r1;
        } else if (go0) {
            node = r0;
        } else if (go1) {
            node = r1;
        } else {
            if (sp == 0) return false;
            node = stack[--sp];
        }
    }
}

struct AoArgs {
    const float4* nodes;
    const float4* tris;
    const void* pos;
    const void* nrm;
    int64_t n;
    int32_t in_f16, rays, e_f16, n_cull;
    float radius;
    uint32_t k0, k1;
    float cull_lo[kCullBoxes][3], cull_hi[kCullBoxes][3];
    float* ao;
    void* E;
};

__global__ void __launch_bounds__(128) ao_kernel(AoArgs a) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= a.n) return;
    const float4 p = niv_load_rec(a.pos, r, a.in_f16), nv = niv_load_rec(a.nrm, r, a.in_f16);
    const float nl = sqrtf(nv.x * nv.x + nv.y * nv.y + nv.z * nv.z);
    const float3 n = make_float3(nv.x / nl, nv.y / nl, nv.z / nl);
    const float3 o = make_float3(p.x + kRayBias * n.x, p.y + kRayBias * n.y, p.z + kRayBias * n.z);
    bool near = false;  // within R of a depth-3 node box (every triangle lies in one)
    for (int c = 0; c < a.n_cull; ++c) {
        const float gx = fmaxf(fmaxf(a.cull_lo[c][0] - o.x, o.x - a.cull_hi[c][0]), 0.0f);
        const float gy = fmaxf(fmaxf(a.cull_lo[c][1] - o.y, o.y - a.cull_hi[c][1]), 0.0f);
        const float gz = fmaxf(fmaxf(a.cull_lo[c][2] - o.z, o.z - a.cull_hi[c][2]), 0.0f);
        near |= gx * gx + gy * gy + gz * gz <= a.radius * a.radius;
    }
    int blocked = 0;
    if (near) {
        for (int j = 0; j < a.rays; ++j) {
            const uint4 u = philox4x32_10(make_uint4((uint32_t)r, (uint32_t)(r >> 32), (uint32_t)j, 0xA0u), a.k0, a.k1);
            const float3 d = cosine_dir(n, u01(u.x), u01(u.y));
            blocked += any_hit(a.nodes, a.tris, o, d, a.radius);
        }
    }
    const float ao = 1.0f - (float)blocked / (float)a.rays;
    if (a.ao) a.ao[r] = ao;
    if (a.E) {
        const float4 e = niv_load_rec(a.E, r, a.e_f16);
        niv_store_rec(a.E, r, e.x * ao, e.y * ao, e.z * ao, a.e_f16);
    }
}

}  // namespace

int niv_dyn_build(const float* tri9, int64_t n_tris, niv_dyn** out) {
    if (n_tris < 1 || n_tris > (int64_t)1 << 30) return niv_fail(NIV_ERR_ARG, "triangle count must be in 1..2^30");
    Builder B;
    B.tri = tri9;
    B.cen.resize(3 * (size_t)n_tris);
    B.order.resize((size_t)n_tris);
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t i = 0; i < n_tris; ++i) {
        B.order[(size_t)i] = (int32_t)i;
        for (int k = 0; k < 3; ++k) {
            const float a = tri9[9 * i + k], b = tri9[9 * i + 3 + k], c = tri9[9 * i + 6 + k];
            if (!std::isfinite(a) || !std::isfinite(b) || !std::isfinite(c))
                return niv_fail(NIV_ERR_ARG, "non-finite triangle vertex");
            B.cen[3 * (size_t)i + k] = (a + b + c) * (1.0f / 3.0f);
            lo[k] = std::min(lo[k], std::min(a, std::min(b, c)));
            hi[k] = std::max(hi[k], std::max(a, std::max(b, c)));
        }
    }
    float ext = 0.0f;
    for (int k = 0; k < 3; ++k) ext = std::max(ext, hi[k] - lo[k]);
    B.pad = 1e-5f * std::max(ext, 1e-3f);
    B.build(0, (int32_t)n_tris, 0);
    // device nodes: one per inner node of the binary hierarchy (a leaf root gets one with a
    // single child), each holding both children's boxes
    std::vector<int32_t> wide_of(B.nodes.size(), -1);
    int32_t n_wide = 0;
    for (size_t i = 0; i < B.nodes.size(); ++i)
        if (B.nodes[i].b <= 0) wide_of[i] = n_wide++;
    auto as_float = [](int32_t v) {
        float f;
        memcpy(&f, &v, 4);
        return f;
    };
    auto put_child = [&](float4* slot, int32_t c) {
        const HostNode& h = B.nodes[(size_t)c];
        const bool leaf = h.b > 0;
        slot[0] = make_float4(h.lo[0], h.lo[1], h.lo[2], as_float(leaf ? h.a : wide_of[(size_t)c]));
        slot[1] = make_float4(h.hi[0], h.hi[1], h.hi[2], as_float(leaf ? h.b : 0));
    };
    std::vector<float4> nodes(4 * (size_t)std::max(n_wide, 1)), tris(3 * (size_t)n_tris);
    if (n_wide == 0) {
        put_child(&nodes[0], 0);
        nodes[2] = make_float4(0.0f, 0.0f, 0.0f, as_float(0));
        nodes[3] = make_float4(0.0f, 0.0f, 0.0f, as_float(-1));
    } else {
        for (size_t i = 0; i < B.nodes.size(); ++i) {
            if (wide_of[i] < 0) continue;
            put_child(&nodes[4 * (size_t)wide_of[i]], (int32_t)i + 1);
            put_child(&nodes[4 * (size_t)wide_of[i] + 2], B.nodes[i].a);
        }
    }
    for (int64_t i = 0; i < n_tris; ++i) {
        const float* t = tri9 + 9 * (int64_t)B.order[(size_t)i];
        tris[3 * i] = make_float4(t[0], t[1], t[2], 0.0f);
        tris[3 * i + 1] = make_float4(t[3] - t[0], t[4] - t[1], t[5] - t[2], 0.0f);
        tris[3 * i + 2] = make_float4(t[6] - t[0], t[7] - t[1], t[8] - t[2], 0.0f);
    }
    niv_dyn* d = new niv_dyn();
    d->n_tris = n_tris;
    d->n_nodes = (int64_t)B.nodes.size();
    std::vector<int32_t> cull;
    collect_cull(B.nodes, 0, 0, cull);
    d->n_cull = (int)cull.size();  // at most 2^3 = kCullBoxes
    for (int c = 0; c < d->n_cull; ++c)
        for (int k = 0; k < 3; ++k) {
            d->cull_lo[c][k] = B.nodes[(size_t)cull[c]].lo[k];
            d->cull_hi[c][k] = B.nodes[(size_t)cull[c]].hi[k];
        }
    cudaError_t e = cudaGetDevice(&d->device);
    d->nodes = nullptr;
    d->tris = nullptr;
    if (e == cudaSuccess) e = cudaMalloc(&d->nodes, sizeof(float4) * nodes.size());
    if (e == cudaSuccess) e = cudaMalloc(&d->tris, sizeof(float4) * tris.size());
    if (e == cudaSuccess) e = cudaMemcpy(d->nodes, nodes.data(), sizeof(float4) * nodes.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(d->tris, tris.data(), sizeof(float4) * tris.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        cudaFree(d->nodes);
        cudaFree(d->tris);
        delete d;
        return niv_cuda_fail(e, "dynamic geometry upload");
    }
    *out = d;
    return NIV_OK;
}

void niv_dyn_free(niv_dyn* d) {
    if (!d) return;
    cudaFree(d->nodes);
    cudaFree(d->tris);
    delete d;
}

int64_t niv_dyn_node_count(const niv_dyn* d) { return d->n_nodes; }

int niv_launch_ao(const niv_dyn* d, const void* pos, const void* nrm, int64_t n, int32_t in_f16, int32_t rays,
                  float radius, uint64_t seed, float* ao, void* E, int32_t e_f16, cudaStream_t s) {
    AoArgs a;
    a.nodes = d->nodes;
    a.tris = d->tris;
    a.pos = pos;
    a.nrm = nrm;
    a.n = n;
    a.in_f16 = in_f16;
    a.rays = rays;
    a.e_f16 = e_f16;
    a.radius = radius;
    a.k0 = (uint32_t)seed;
    a.k1 = (uint32_t)(seed >> 32);
    a.n_cull = d->n_cull;
    for (int c = 0; c < d->n_cull; ++c)
        for (int k = 0; k < 3; ++k) {
            a.cull_lo[c][k] = d->cull_lo[c][k];
            a.cull_hi[c][k] = d->cull_hi[c][k];
        }
    a.ao = ao;
    a.E = E;
    ao_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(a);
    NIV_CUDA(cudaGetLastError());
    return NIV_OK;
}
