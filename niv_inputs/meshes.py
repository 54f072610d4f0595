"""Procedural dynamic objects and the full shading frame (input generation only).

Three meshes are inserted into the room G-buffer, like the unseen dynamic objects
that NIV shades at runtime:
  * a torus of 250 x 100 quads (50,000 triangles),
  * an icosphere subdivided 6 times (81,920 triangles),
  * a box with 64 x 64 quads per face (49,152 triangles), twisted about its vertical axis.
Each gets a seeded pose inside the view and a seeded albedo U(0.1, 0.9) per channel.
The direct-light buffer is seeded U(0, 0.5) per channel.
"""
import ctypes
import math
import os
import subprocess

import numpy as np

from .scenes import CAMERA_POS

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None


def _raster_lib():
    global _LIB
    if _LIB is None:
        src = os.path.join(_HERE, "raster.c")
        so = os.path.join(_HERE, "libraster.so")
        if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
            tmp = so + ".tmp%d" % os.getpid()
            subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", src, "-o", tmp, "-lm"], check=True,
                           capture_output=True)
            os.replace(tmp, so)
        lib = ctypes.CDLL(so)
        vp = ctypes.c_void_p
        lib.niv_raster_meshes.argtypes = [vp, vp, vp, ctypes.c_int64, vp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                          vp, vp, vp, vp, vp, vp]
        lib.niv_raster_meshes.restype = None
        _LIB = lib
    return _LIB


def torus(R=0.7, r=0.25, nu=250, nv=100):
    u = np.arange(nu) * 2 * math.pi / nu
    v = np.arange(nv) * 2 * math.pi / nv
    U, V = np.meshgrid(u, v, indexing="ij")
    verts = np.stack([(R + r * np.cos(V)) * np.cos(U), r * np.sin(V), (R + r * np.cos(V)) * np.sin(U)], -1).reshape(-1, 3)
    i = np.arange(nu)[:, None]
    j = np.arange(nv)[None, :]
    a = i * nv + j
    b = ((i + 1) % nu) * nv + j
    c = ((i + 1) % nu) * nv + (j + 1) % nv
    d = i * nv + (j + 1) % nv
    tris = np.concatenate([np.stack([a, b, c], -1).reshape(-1, 3), np.stack([a, c, d], -1).reshape(-1, 3)])
    return verts, tris.astype(np.int32)


def icosphere(subdiv=6, radius=0.6):
    t = (1.0 + math.sqrt(5.0)) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0], [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], np.float64)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11], [1, 5, 9], [5, 11, 4], [11, 10, 2],
                  [10, 7, 6], [7, 1, 8], [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9], [4, 9, 5], [2, 4, 11],
                  [6, 2, 10], [8, 6, 7], [9, 8, 1]], np.int64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    for _ in range(subdiv):
        edges = np.concatenate([f[:, [0, 1]], f[:, [1, 2]], f[:, [2, 0]]])
        key = np.sort(edges, axis=1)
        uniq, inv = np.unique(key, axis=0, return_inverse=True)
        mid = v[uniq[:, 0]] + v[uniq[:, 1]]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        m = len(v) + inv.reshape(3, -1)  # midpoint index of edges 01, 12, 20 per face
        v = np.concatenate([v, mid])
        a, b, c = f[:, 0], f[:, 1], f[:, 2]
        f = np.concatenate([np.stack([a, m[0], m[2]], -1), np.stack([b, m[1], m[0]], -1),
                            np.stack([c, m[2], m[1]], -1), np.stack([m[0], m[1], m[2]], -1)])
    return v * radius, f.astype(np.int32)


def twisted_box(size=1.0, n=64, twist=math.pi / 2):
    g = np.linspace(-0.5, 0.5, n + 1)
    A, B = np.meshgrid(g, g, indexing="ij")
    verts, tris = [], []
    off = 0
    for axis in range(3):
        for side in (-0.5, 0.5):
            a, b = [k for k in range(3) if k != axis]
            p = np.zeros((n + 1, n + 1, 3))
            p[..., axis] = side
            p[..., a] = A
            p[..., b] = B
            verts.append(p.reshape(-1, 3))
            i = np.arange(n)[:, None]
            j = np.arange(n)[None, :]
            q00, q10, q11, q01 = i * (n + 1) + j, (i + 1) * (n + 1) + j, (i + 1) * (n + 1) + j + 1, i * (n + 1) + j + 1
            tris.append(off + np.concatenate([np.stack([q00, q10, q11], -1).reshape(-1, 3),
                                              np.stack([q00, q11, q01], -1).reshape(-1, 3)]))
            off += (n + 1) ** 2
    v = np.concatenate(verts) * size
    ang = twist * (v[:, 1] / size)
    c, s = np.cos(ang), np.sin(ang)
    v = np.stack([c * v[:, 0] + s * v[:, 2], v[:, 1], -s * v[:, 0] + c * v[:, 2]], -1)
    return v, np.concatenate(tris).astype(np.int32)


def _rotation(rng):
    q = rng.standard_normal(4)
    q /= np.linalg.norm(q)
    w, x, y, z = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def dynamic_objects(seed=0):
    """Three posed meshes: (vertices [V][3], triangles [T][3], mesh id per triangle [T], albedo [3][3])."""
    rng = np.random.Generator(np.random.PCG64(seed + 4242))
    parts, tris, ids = [], [], []
    off = 0
    for k, (v, f) in enumerate([torus(), icosphere(), twisted_box()]):
        R = _rotation(rng)
        centre = np.array([rng.uniform(-2.0, 2.0), rng.uniform(-2.0, 0.5), rng.uniform(-1.0, 1.5)])
        parts.append(v @ R.T + centre)
        tris.append(f + off)
        ids.append(np.full(len(f), k, np.int32))
        off += len(v)
    albedo = rng.uniform(0.1, 0.9, (3, 3))
    return np.concatenate(parts), np.concatenate(tris).astype(np.int32), np.concatenate(ids), albedo


def shading_frame(width, height, seed=0, cache_dir=None):
    """The config-4 frame: FP16 [n][4] records (pos, nrm, albedo, direct) and the object coverage."""
    from .scenes import room_scene
    from .gbuffer import raycast_gbuffer, pack_records
    cache_dir = cache_dir or os.environ.get("NIV_CACHE", "/tmp/niv_cache")
    path = os.path.join(cache_dir, "frame4_s%d_%dx%d.npz" % (seed, width, height))
    if os.path.exists(path):
        try:
            z = np.load(path)
            return z["pos"], z["nrm"], z["alb"], z["direct"], float(z["coverage"])
        except Exception:
            pass
    pos, nrm, alb, hit = raycast_gbuffer(room_scene(seed), width, height)
    verts, tris, ids, albedo = dynamic_objects(seed)
    hit8 = hit.astype(np.uint8)
    mesh_id = np.full(width * height, -1, np.int32)
    pos, nrm, alb = (np.ascontiguousarray(a) for a in (pos, nrm, alb))
    verts = np.ascontiguousarray(verts)
    albedo = np.ascontiguousarray(albedo)
    cam = np.asarray(CAMERA_POS, np.float64)
    _raster_lib().niv_raster_meshes(verts.ctypes.data, tris.ctypes.data, ids.ctypes.data, len(tris),
                                    albedo.ctypes.data, width, height, 60.0, cam.ctypes.data, pos.ctypes.data,
                                    nrm.ctypes.data, alb.ctypes.data, hit8.ctypes.data, mesh_id.ctypes.data)
    rng = np.random.Generator(np.random.PCG64(seed + 99))
    direct = rng.uniform(0.0, 0.5, (width * height, 3))
    out = (pack_records(pos, np.float16), pack_records(nrm, np.float16), pack_records(alb, np.float16),
           pack_records(direct, np.float16), float((mesh_id >= 0).mean()))
    try:
        os.makedirs(cache_dir, exist_ok=True)
        tmp = path + ".tmp%d.npz" % os.getpid()
        np.savez(tmp, pos=out[0], nrm=out[1], alb=out[2], direct=out[3], coverage=out[4])
        os.replace(tmp, path)
    except OSError:
        pass
    return out
