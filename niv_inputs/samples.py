"""Seeded training-sample candidates (the data distribution of Sec. 4.5 / App. I).

A fraction `surface_frac` (0.2 in the paper) of the points lie on the scene's surfaces
with the direction set to the surface normal; the rest are uniform in the room box with
directions uniform on the sphere.  Surfaces are chosen in proportion to their area:
the six room walls (the skylight opening excluded), every non-emitting sphere and
every box face.  Candidates inside geometry are left in: the Monte Carlo pass flags
them (backface majority) and the compaction drops them.
"""
import math

import numpy as np

from .queries import sphere_directions


def _surface_patches(scene):
    """List of (area, sampler(rng, k) -> (points[k][3], normals[k][3]))."""
    patches = []
    lo = np.asarray(scene.room_min, np.float64)
    hi = np.asarray(scene.room_max, np.float64)
    if scene.has_room:
        x0, x1, z0, z1 = scene.skylight
        for axis in range(3):
            for side in (0, 1):
                a, b = [k for k in range(3) if k != axis]
                area = (hi[a] - lo[a]) * (hi[b] - lo[b])
                is_ceiling = axis == 1 and side == 1
                if is_ceiling and x0 < x1:
                    area -= (x1 - x0) * (z1 - z0)

                def sample(rng, k, axis=axis, side=side, a=a, b=b, is_ceiling=is_ceiling):
                    p = np.empty((k, 3))
                    p[:, a] = rng.uniform(lo[a], hi[a], k)
                    p[:, b] = rng.uniform(lo[b], hi[b], k)
                    p[:, axis] = hi[axis] if side else lo[axis]
                    if is_ceiling and x0 < x1:  # redraw points that fall into the opening
                        bad = (p[:, 0] >= x0) & (p[:, 0] <= x1) & (p[:, 2] >= z0) & (p[:, 2] <= z1)
                        while bad.any():
                            p[bad, a] = rng.uniform(lo[a], hi[a], bad.sum())
                            p[bad, b] = rng.uniform(lo[b], hi[b], bad.sum())
                            bad = (p[:, 0] >= x0) & (p[:, 0] <= x1) & (p[:, 2] >= z0) & (p[:, 2] <= z1)
                    n = np.zeros((k, 3))
                    n[:, axis] = -1.0 if side else 1.0
                    return p, n
                patches.append((area, sample))
    for s in np.asarray(scene.spheres, np.float64):
        if np.any(s[7:10] > 0):
            continue  # emitters are not shaded
        c, r = s[:3], s[3]

        def sample(rng, k, c=c, r=r):
            d = sphere_directions(rng, k)
            return c + r * d, d
        patches.append((4 * math.pi * r * r, sample))
    for bx in np.asarray(scene.boxes, np.float64):
        blo, bhi = bx[:3], bx[3:6]
        for axis in range(3):
            for side in (0, 1):
                a, b = [k for k in range(3) if k != axis]

                def sample(rng, k, axis=axis, side=side, a=a, b=b, blo=blo, bhi=bhi):
                    p = np.empty((k, 3))
                    p[:, a] = rng.uniform(blo[a], bhi[a], k)
                    p[:, b] = rng.uniform(blo[b], bhi[b], k)
                    p[:, axis] = bhi[axis] if side else blo[axis]
                    n = np.zeros((k, 3))
                    n[:, axis] = 1.0 if side else -1.0
                    return p, n
                patches.append(((bhi[a] - blo[a]) * (bhi[b] - blo[b]), sample))
    return patches


def training_pool(scene, n, seed=0, surface_frac=0.2, with_t=False):
    """(x4, n4, t) candidates: float32 [n][4] records (and a float32 [n] time, or None)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ns = int(round(surface_frac * n))
    nv = n - ns
    lo = np.asarray(scene.room_min, np.float64)
    hi = np.asarray(scene.room_max, np.float64)
    pts = [lo + (hi - lo) * rng.random((nv, 3))]
    nrm = [sphere_directions(rng, nv)]
    patches = _surface_patches(scene)
    if ns > 0 and patches:
        areas = np.array([a for a, _ in patches])
        counts = rng.multinomial(ns, areas / areas.sum())
        for (_, sample), k in zip(patches, counts):
            if k:
                p, q = sample(rng, int(k))
                pts.append(p)
                nrm.append(q)
    P = np.concatenate(pts)
    N = np.concatenate(nrm)
    order = rng.permutation(len(P))
    x4 = np.zeros((len(P), 4), np.float32)
    n4 = np.zeros((len(P), 4), np.float32)
    x4[:, :3] = P[order]
    n4[:, :3] = N[order]
    t = rng.random(len(P)).astype(np.float32) if with_t else None
    return x4, n4, t
