"""Primary-visibility G-buffers by ray casting the analytic scene (numpy, float64).

This stands in for the rasterisation pass that produces the G-buffer in an
engine: per pixel it returns the first-hit world position, the unit surface
normal and the surface albedo.  Pixels are in row-major order, row 0 at the top.
"""
import ctypes
import math
import os
import subprocess

import numpy as np

from .scenes import CAMERA_POS, SPHERE_LEN, BOX_LEN

_HERE = os.path.dirname(os.path.abspath(__file__))
_C_LIB = None


def _c_raycaster():
    """The C version of the ray cast (raycast.c, same rules), compiled on first use; None if gcc fails."""
    global _C_LIB
    if _C_LIB is None:
        src = os.path.join(_HERE, "raycast.c")
        so = os.path.join(_HERE, "libraycast.so")
        try:
            if not os.path.exists(so) or os.path.getmtime(so) < os.path.getmtime(src):
                tmp = so + ".tmp%d" % os.getpid()
                base = ["gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", src, "-o", tmp, "-lm"]
                try:
                    subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
                except subprocess.CalledProcessError:
                    subprocess.run(base, check=True, capture_output=True)
                os.replace(tmp, so)
            lib = ctypes.CDLL(so)
            lib.niv_raycast.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double] + [ctypes.c_void_p] * 5
            lib.niv_raycast.restype = None
            _C_LIB = lib
        except (OSError, subprocess.CalledProcessError):
            _C_LIB = False
    return _C_LIB or None


def camera_rays(width, height, vfov_deg=60.0, origin=CAMERA_POS):
    """Pinhole camera looking down +z with +y up; one ray through each pixel centre."""
    th = math.tan(math.radians(vfov_deg) * 0.5)
    aspect = width / height
    i = (np.arange(width) + 0.5) / width
    j = (np.arange(height) + 0.5) / height
    x = (2.0 * i - 1.0) * th * aspect
    y = (1.0 - 2.0 * j) * th
    dx, dy = np.meshgrid(x, y)
    d = np.stack([dx.ravel(), dy.ravel(), np.ones(width * height)], axis=1)
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    o = np.broadcast_to(np.asarray(origin, np.float64), d.shape)
    return o, d


def _cast_chunk(scene, o, d):
    n = len(d)
    t_best = np.full(n, np.inf)
    nrm = np.zeros((n, 3))
    alb = np.zeros((n, 3))
    eps = 1e-7
    if scene.has_room:
        lo = np.asarray(scene.room_min, np.float64)
        hi = np.asarray(scene.room_max, np.float64)
        with np.errstate(divide="ignore", invalid="ignore"):
            tb = np.where(d > 0, (hi - o) / d, np.where(d < 0, (lo - o) / d, np.inf))
        axis = np.argmin(tb, axis=1)
        t_room = tb[np.arange(n), axis]
        side = np.where(d[np.arange(n), axis] > 0, 1, 0)  # 1: the +axis wall
        wall = 2 * axis + side
        p = o + t_room[:, None] * d
        x0, x1, z0, z1 = scene.skylight
        open_ = (wall == 3) & (x0 < x1) & (p[:, 0] >= x0) & (p[:, 0] <= x1) & (p[:, 2] >= z0) & (p[:, 2] <= z1)
        ok = ~open_
        t_best = np.where(ok, t_room, np.inf)
        wn = np.zeros((n, 3))
        wn[np.arange(n), axis] = np.where(side == 1, -1.0, 1.0)
        nrm = np.where(ok[:, None], wn, 0.0)
        alb = np.where(ok[:, None], np.asarray(scene.wall_albedo, np.float64)[wall], 0.0)
    for s in np.asarray(scene.spheres, np.float64).reshape(-1, SPHERE_LEN):
        c, r = s[0:3], s[3]
        oc = o - c
        b = np.einsum("ij,ij->i", oc, d)
        cc = np.einsum("ij,ij->i", oc, oc) - r * r
        disc = b * b - cc
        sq = np.sqrt(np.maximum(disc, 0.0))
        t = -b - sq
        t = np.where(t > eps, t, -b + sq)
        hit = (disc >= 0) & (t > eps) & (t < t_best)
        t_best = np.where(hit, t, t_best)
        p = o + t[:, None] * d
        nrm = np.where(hit[:, None], (p - c) / r, nrm)
        alb = np.where(hit[:, None], s[4:7], alb)
    for bx in np.asarray(scene.boxes, np.float64).reshape(-1, BOX_LEN):
        lo, hi = bx[0:3], bx[3:6]
        with np.errstate(divide="ignore", invalid="ignore"):
            t1 = (lo - o) / d
            t2 = (hi - o) / d
        tn = np.minimum(t1, t2)
        tf = np.maximum(t1, t2)
        tmin = np.max(tn, axis=1)
        tmax = np.min(tf, axis=1)
        hit = (tmax >= np.maximum(tmin, eps)) & (tmin > eps) & (tmin < t_best)
        axis = np.argmax(tn, axis=1)
        bn = np.zeros((n, 3))
        bn[np.arange(n), axis] = -np.sign(d[np.arange(n), axis])
        t_best = np.where(hit, tmin, t_best)
        nrm = np.where(hit[:, None], bn, nrm)
        alb = np.where(hit[:, None], bx[6:9], alb)
    hit_any = np.isfinite(t_best)
    pos = np.where(hit_any[:, None], o + np.where(hit_any, t_best, 0.0)[:, None] * d, 0.0)
    return pos, nrm, alb, hit_any


def raycast_gbuffer(scene, width, height, vfov_deg=60.0, chunk=1 << 20, impl="auto"):
    """Return float64 ``(pos[n][3], nrm[n][3], albedo[n][3], hit[n])`` for a ``width x height`` frame.

    impl: "c" (raycast.c), "numpy", or "auto" (C when it compiles, else numpy).
    """
    lib = _c_raycaster() if impl in ("auto", "c") else None
    if impl == "c" and lib is None:
        raise RuntimeError("C ray caster unavailable")
    if lib is not None:
        n = width * height
        pos, nrm, alb = (np.zeros((n, 3)) for _ in range(3))
        hit = np.zeros(n, np.uint8)
        blob = np.ascontiguousarray(scene.blob(), np.float32)
        origin = np.asarray(CAMERA_POS, np.float64)
        lib.niv_raycast(blob.ctypes.data, width, height, float(vfov_deg), origin.ctypes.data, pos.ctypes.data,
                        nrm.ctypes.data, alb.ctypes.data, hit.ctypes.data)
        return pos, nrm, alb, hit.astype(bool)
    o, d = camera_rays(width, height, vfov_deg)
    n = len(d)
    pos = np.empty((n, 3))
    nrm = np.empty((n, 3))
    alb = np.empty((n, 3))
    hit = np.empty(n, bool)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        pos[s:e], nrm[s:e], alb[s:e], hit[s:e] = _cast_chunk(scene, o[s:e], d[s:e])
    return pos, nrm, alb, hit


def pack_records(xyz, dtype=np.float16, w=0.0):
    """Contiguous ``[n][4]`` records of ``dtype`` with the fourth component set to ``w``."""
    xyz = np.asarray(xyz)
    out = np.empty((len(xyz), 4), dtype=dtype)
    out[:, :3] = xyz
    out[:, 3] = w
    return out
