"""CPU FP64 oracle of the Neural Irradiance Volume path (ctypes wrapper).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and bench.py's
CPU-baseline / reference leg may import this package; the product path
(``paper_2602_12949_gb300``) never does.  The C sources here share nothing with
the CUDA library.

``build()`` compiles ``liboracle.so`` next to this file with gcc (OpenMP when
available, ``-ffp-contract=off`` so that the FP32 operations it emulates are
never fused).
"""
import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SOURCES = ["niv_oracle.c", "oracle_mc.c", "oracle_sh.c", "oracle_ao.c", "oracle_samples.c"]
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None

MC_TOTAL = 0
MC_INDIRECT = 1


def build(force=False):
    """Compile liboracle.so (gcc, -O2, OpenMP if the compiler supports it)."""
    srcs = [os.path.join(_HERE, s) for s in _SOURCES]
    if not force and os.path.exists(_LIB_PATH):
        newest = max(os.path.getmtime(s) for s in srcs)
        if os.path.getmtime(_LIB_PATH) >= newest:
            return _LIB_PATH
    base = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math"]
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    try:
        subprocess.run(base + ["-fopenmp"] + srcs + ["-o", tmp, "-lm"], check=True,
                       capture_output=True, text=True)
    except subprocess.CalledProcessError:
        subprocess.run(base + srcs + ["-o", tmp, "-lm"], check=True, capture_output=True, text=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Desc(ctypes.Structure):
    """Model description as the oracle reads it (its own struct; see niv_oracle.c)."""
    _fields_ = [
        ("dims", ctypes.c_int32), ("levels", ctypes.c_int32), ("feat", ctypes.c_int32),
        ("log2_T", ctypes.c_int32), ("base", ctypes.c_double), ("growth", ctypes.c_double),
        ("n_hidden", ctypes.c_int32), ("width", ctypes.c_int32), ("in_extra", ctypes.c_int32),
        ("out_dim", ctypes.c_int32), ("out_act", ctypes.c_int32), ("prime_t", ctypes.c_uint32),
        ("pe_bands", ctypes.c_int32), ("t_bands", ctypes.c_int32),
    ]


@dataclass
class Model:
    """Hyper-parameters of one model (the oracle's view)."""
    dims: int = 3
    levels: int = 8
    feat: int = 2
    log2_T: int = 14
    base: float = 4.0
    growth: float = 1.5
    n_hidden: int = 2
    width: int = 64
    in_extra: int = 3
    out_dim: int = 3
    out_act: int = 1
    prime_t: int = 0x9E3779B1
    pe_bands: int = 0  # > 0: frequency-encoded position (Table 1's models without grid levels)
    t_bands: int = 0   # > 0: the scene parameter t frequency-encoded after n (Sec. 6)

    def cdesc(self):
        return Desc(self.dims, self.levels, self.feat, self.log2_T, self.base, self.growth,
                    self.n_hidden, self.width, self.in_extra, self.out_dim, self.out_act, self.prime_t,
                    self.pe_bands, self.t_bands)

    @property
    def enc_dim(self):
        return self.levels * self.feat + 6 * self.pe_bands

    @property
    def n_in(self):
        return self.enc_dim + self.in_extra + 2 * self.t_bands


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P = ctypes.POINTER
        d, i64, f, u64 = ctypes.c_double, ctypes.c_int64, ctypes.c_float, ctypes.c_uint64
        vp = ctypes.c_void_p
        L.orc_num_threads.restype = ctypes.c_int
        L.orc_num_threads.argtypes = []
        L.orc_set_num_threads.restype = None
        L.orc_set_num_threads.argtypes = [ctypes.c_int]
        L.orc_layout.restype = i64
        L.orc_layout.argtypes = [P(Desc), vp, vp, vp, vp]
        L.orc_mlp_param_count.restype = i64
        L.orc_mlp_param_count.argtypes = [P(Desc)]
        L.orc_encode.argtypes = [P(Desc), vp, vp, i64, vp, vp, f, vp, vp, vp]
        L.orc_mlp.argtypes = [P(Desc), vp, vp, i64, vp]
        L.orc_query.argtypes = [P(Desc), vp, vp, vp, i64, vp, vp, f, vp]
        L.orc_loss_grad.argtypes = [P(Desc), vp, vp, vp, vp, vp, i64, vp, vp, d, vp, vp, ctypes.c_int]
        L.orc_adam.argtypes = [vp, vp, vp, vp, i64, d, d, d, d, i64]
        L.orc_adam.restype = None
        L.orc_shade.argtypes = [vp, vp, vp, i64, vp]
        L.orc_shade.restype = None
        L.orc_e4m3.argtypes = [d]
        L.orc_e4m3.restype = d
        L.orc_f16.argtypes = [d]
        L.orc_f16.restype = d
        L.orc_f16_array.argtypes = [vp, i64, vp]
        L.orc_f16_array.restype = None
        L.orc_query_f16.argtypes = [P(Desc), vp, vp, vp, i64, vp, vp, f, vp]
        L.orc_upsample_shade.argtypes = [vp, vp, vp, vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int, d, d, d, vp]
        L.orc_upsample_shade.restype = None
        L.orc_e4m3_array.argtypes = [vp, i64, vp]
        L.orc_e4m3_array.restype = None
        L.orc_fp8_scale.argtypes = [d]
        L.orc_fp8_scale.restype = d
        L.orc_fp8_act_amax.argtypes = [P(Desc), vp, vp, vp, i64, vp, vp, f, vp]
        L.orc_query_fp8.argtypes = [P(Desc), vp, vp, vp, vp, i64, vp, vp, f, vp]
        L.orc_training_samples.argtypes = [vp, i64, i64, f, ctypes.c_uint64, ctypes.c_uint64, vp, vp, vp, vp]
        L.orc_training_samples.restype = ctypes.c_int
        L.orc_sample_patch_table.argtypes = [vp, i64, vp, ctypes.c_int]
        L.orc_sample_patch_table.restype = ctypes.c_int
        L.orc_philox4x32_10.argtypes = [vp, vp, vp]
        L.orc_philox4x32_10.restype = None
        L.orc_mc_irradiance.argtypes = [vp, vp, vp, vp, i64, ctypes.c_int, u64, u64, ctypes.c_int, vp, vp, vp]
        L.orc_mc_radiance.argtypes = [vp, vp, vp, i64, ctypes.c_int, u64, u64, ctypes.c_int, vp]
        L.orc_sh9.argtypes = [vp, vp]
        L.orc_sh9.restype = None
        L.orc_sh_irradiance.argtypes = [vp, vp, vp]
        L.orc_sh_irradiance.restype = None
        L.orc_sh_project.argtypes = [vp, vp, i64, vp]
        L.orc_sh_project.restype = None
        L.orc_probe_bake.argtypes = [vp, vp, vp, vp, ctypes.c_int, u64, u64, vp, vp]
        L.orc_probe_query.argtypes = [vp, vp, vp, vp, vp, vp, i64, vp]
        L.orc_probe_query_rt.argtypes = [vp, vp, vp, vp, vp, d, vp, vp, i64, vp, vp]
        L.orc_visible.argtypes = [vp, d, d, vp, vp, d]
        L.orc_visible.restype = ctypes.c_int
        L.orc_dyn_ao.argtypes = [vp, i64, vp, vp, i64, ctypes.c_int, d, u64, vp, vp, vp]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def layout(model):
    """Per-level resolution, dense flag, first entry and entry count; plus the total."""
    L = model.levels
    res = np.zeros(L, np.int32)
    dense = np.zeros(L, np.int32)
    off = np.zeros(L, np.int64)
    ent = np.zeros(L, np.int64)
    total = lib().orc_layout(ctypes.byref(model.cdesc()), _p(res), _p(dense), _p(off), _p(ent))
    if total < 0:
        raise ValueError("invalid model description")
    return {"res": res, "dense": dense, "offset": off, "entries": ent, "total": int(total)}


def grid_value_count(model):
    return layout(model)["total"] * model.feat


def mlp_param_count(model):
    return int(lib().orc_mlp_param_count(ctypes.byref(model.cdesc())))


def layer_shapes(model):
    shapes, k = [], model.n_in
    for _ in range(model.n_hidden):
        shapes.append((model.width, k))
        k = model.width
    shapes.append((model.out_dim, k))
    return shapes


def encode(model, params, pos4, aabb_min=(0, 0, 0), aabb_max=(1, 1, 1), t=0.0, want_corners=False):
    """Encoding of every query: enc[n][L*F + 6*B] (grid features, then frequency encoding),
    and the grid corners' indices / weights if asked."""
    pos4 = _f32(pos4)
    n = len(pos4)
    nc = 1 << model.dims
    enc = np.zeros((n, model.enc_dim))
    idx = np.zeros((n, model.levels, nc), np.uint32) if want_corners else None
    w = np.zeros((n, model.levels, nc)) if want_corners else None
    lib().orc_encode(ctypes.byref(model.cdesc()), _p(_f64(params)), _p(pos4), n, _p(_f32(aabb_min)),
                     _p(_f32(aabb_max)), float(t), _p(enc), _p(idx), _p(w))
    return (enc, idx, w) if want_corners else enc


def mlp(model, mlp_params, x):
    x = _f64(x)
    E = np.zeros((len(x), model.out_dim))
    lib().orc_mlp(ctypes.byref(model.cdesc()), _p(_f64(mlp_params)), _p(x), len(x), _p(E))
    return E


def query(model, params, pos4, nrm4, aabb_min=(0, 0, 0), aabb_max=(1, 1, 1), t=0.0):
    """E(x, n) for every G-buffer record: float64 [n][out_dim]."""
    pos4, nrm4 = _f32(pos4), _f32(nrm4)
    E = np.zeros((len(pos4), model.out_dim))
    rc = lib().orc_query(ctypes.byref(model.cdesc()), _p(_f64(params)), _p(pos4), _p(nrm4), len(pos4),
                         _p(_f32(aabb_min)), _p(_f32(aabb_max)), float(t), _p(E))
    if rc:
        raise ValueError("orc_query failed")
    return E


def f16(x):
    """Nearest binary16 values (ties to even) of an array, as float64."""
    x = _f64(x)
    out = np.empty_like(x)
    lib().orc_f16_array(_p(x), x.size, _p(out))
    return out


def query_f16(model, params16, pos4, nrm4, aabb_min=(0, 0, 0), aabb_max=(1, 1, 1), t=0.0):
    """E(x, n) on the FP16 network path: params16 already rounded to binary16, network
    input and hidden activations rounded to binary16, FP64 sums and softplus."""
    pos4, nrm4 = _f32(pos4), _f32(nrm4)
    E = np.zeros((len(pos4), model.out_dim))
    rc = lib().orc_query_f16(ctypes.byref(model.cdesc()), _p(_f64(params16)), _p(pos4), _p(nrm4), len(pos4),
                             _p(_f32(aabb_min)), _p(_f32(aabb_max)), float(t), _p(E))
    if rc:
        raise ValueError("orc_query_f16 failed")
    return E


def upsample_shade(pos4, nrm4, alb4, dir4, width, height, E_low, sub=2, power=8.0, sigma=0.05, eps=1e-4):
    """Full-resolution shaded rgb [W*H][3] from the irradiance E_low [h*w][3] queried at every
    sub-th pixel (joint bilateral upsampling guided by the full-resolution G-buffer)."""
    n = width * height
    out = np.zeros((n, 3))
    E = _f64(np.asarray(E_low)[:, :3])
    lib().orc_upsample_shade(_p(_f32(pos4)), _p(_f32(nrm4)), _p(_f32(alb4)), _p(_f32(dir4)), int(width),
                             int(height), _p(E), int(sub), float(power), float(sigma), float(eps), _p(out))
    return out


def loss_grad(model, params, pos4, nrm4, target, aabb_min=(0, 0, 0), aabb_max=(1, 1, 1), t=None, eps=0.01,
              f16=False):
    """(loss, grad) of Eq. 3 averaged over samples and channels; grad has params' shape.
    f16: the FP16 forward path (pass binary16-rounded params), straight-through gradient."""
    params = _f64(params)
    g = np.zeros_like(params)
    loss = ctypes.c_double()
    tt = None if t is None else _f32(t)
    rc = lib().orc_loss_grad(ctypes.byref(model.cdesc()), _p(params), _p(_f32(pos4)), _p(_f32(nrm4)), _p(tt),
                             _p(_f64(target)), len(pos4), _p(_f32(aabb_min)), _p(_f32(aabb_max)), eps,
                             ctypes.byref(loss), _p(g), int(bool(f16)))
    if rc:
        raise ValueError("orc_loss_grad failed")
    return loss.value, g


def adam(theta, m, v, g, lr, b1, b2, eps, step):
    """In-place Adam step on float64 arrays."""
    lib().orc_adam(_p(theta), _p(m), _p(v), _p(_f64(g)), len(theta), lr, b1, b2, eps, step)


def shade(albedo3, E3, direct3):
    albedo3, E3, direct3 = _f64(albedo3), _f64(E3), _f64(direct3)
    out = np.zeros_like(E3)
    lib().orc_shade(_p(albedo3), _p(E3), _p(direct3), len(E3), _p(out))
    return out


def e4m3(x):
    x = _f64(x)
    out = np.zeros_like(x)
    lib().orc_e4m3_array(_p(x), x.size, _p(out))
    return out


def fp8_scale(amax):
    """Power-of-two E4M3 scale 2^ceil(log2(amax / 448))."""
    return lib().orc_fp8_scale(float(amax))


def fp8_act_amax(model, params, pos4, nrm4, aabb_min=(0, 0, 0), aabb_max=(1, 1, 1), t=0.0):
    """amax of each matrix product's input (network input, then each hidden layer's output)."""
    out = np.zeros(model.n_hidden + 1)
    rc = lib().orc_fp8_act_amax(ctypes.byref(model.cdesc()), _p(_f64(params)), _p(_f32(pos4)), _p(_f32(nrm4)),
                                len(pos4), _p(_f32(aabb_min)), _p(_f32(aabb_max)), float(t), _p(out))
    if rc:
        raise ValueError("orc_fp8_act_amax failed")
    return out


def query_fp8(model, params, s_act, pos4, nrm4, aabb_min=(0, 0, 0), aabb_max=(1, 1, 1), t=0.0):
    """E(x, n) of the E4M3 network path with activation scales s_act (one per matrix product):
    every scaled weight and input carried as two E4M3 codes h = e4m3(v), l = e4m3(v - h)."""
    pos4, nrm4 = _f32(pos4), _f32(nrm4)
    E = np.zeros((len(pos4), model.out_dim))
    rc = lib().orc_query_fp8(ctypes.byref(model.cdesc()), _p(_f64(params)), _p(_f64(s_act)), _p(pos4), _p(nrm4),
                             len(pos4), _p(_f32(aabb_min)), _p(_f32(aabb_max)), float(t), _p(E))
    if rc:
        raise ValueError("orc_query_fp8 failed")
    return E


def training_samples(blob, n, surface_frac=0.2, seed=0, index_base=0, with_t=False):
    """Training-sample candidates of Sec. 4.5 / App. I (see oracle_samples.c):
    (x4 float32 [n][4], n4 float32 [n][4], t float32 [n] or None, patch int32 [n], -1 = volume)."""
    b = np.ascontiguousarray(blob, np.float32)
    x4 = np.zeros((n, 4), np.float32)
    n4 = np.zeros((n, 4), np.float32)
    t = np.zeros(n, np.float32) if with_t else None
    patch = np.zeros(n, np.int32)
    k = lib().orc_training_samples(_p(b), b.size, n, float(surface_frac), int(seed), int(index_base), _p(x4), _p(n4),
                                   _p(t) if t is not None else None, _p(patch))
    if k < 0:
        raise ValueError("bad scene description")
    return x4, n4, t, patch


def sample_patches(blob):
    """The surfaces the samples are spread over, in order: float64 [K][13] rows of kind (0 rectangle,
    1 sphere), axis, normal sign, plane, a0, a1, b0, b1, cx, cy, cz, r, area."""
    b = np.ascontiguousarray(blob, np.float32)
    out = np.zeros((512, 13))
    k = lib().orc_sample_patch_table(_p(b), b.size, _p(out), 512)
    if k < 0:
        raise ValueError("bad scene description")
    return out[:k]


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, np.uint32)
    k = np.ascontiguousarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def mc_irradiance(blob, x4, n4, spp, seed=0, mode=MC_INDIRECT, t=None, index_base=0, want_se=False):
    """(E[m][3], keep[m]) by Monte Carlo on the scene blob; with want_se also the standard
    error of each estimate ([m][3], from the sample variance of the path radiances)."""
    x4, n4 = _f32(x4), _f32(n4)
    m = len(x4)
    E = np.zeros((m, 3))
    keep = np.zeros(m, np.uint8)
    se = np.zeros((m, 3)) if want_se else None
    tt = None if t is None else _f32(t)
    lib().orc_mc_irradiance(_p(_f32(blob)), _p(x4), _p(n4), _p(tt), m, int(spp), int(seed), int(index_base),
                            int(mode), _p(E), _p(keep), _p(se))
    return (E, keep, se) if want_se else (E, keep)


def mc_radiance(blob, x4, d4, spp, seed=0, mode=MC_INDIRECT, index_base=0):
    x4, d4 = _f32(x4), _f32(d4)
    L = np.zeros((len(x4), 3))
    lib().orc_mc_radiance(_p(_f32(blob)), _p(x4), _p(d4), len(x4), int(spp), int(seed), int(index_base),
                          int(mode), _p(L))
    return L


def sh9(w):
    w = _f64(w)
    Y = np.zeros(9)
    lib().orc_sh9(_p(w), _p(Y))
    return Y


def sh_irradiance(coef, n):
    E = np.zeros(3)
    lib().orc_sh_irradiance(_p(_f64(coef)), _p(_f64(n)), _p(E))
    return E


def sh_project(dirs, L):
    dirs, L = _f64(dirs), _f64(L)
    c = np.zeros(27)
    lib().orc_sh_project(_p(dirs), _p(L), len(dirs), _p(c))
    return c.reshape(9, 3)


def probe_bake(blob, P, lo, hi, rays, seed=0, index_base=0, want_se=False):
    """SH9 x RGB coefficients [probes][9][3]; with want_se also their standard errors (same shape,
    from the sample variance of L Y over the rays)."""
    P = np.ascontiguousarray(P, np.int32)
    out = np.zeros((int(np.prod(P)), 9, 3))
    se = np.zeros_like(out) if want_se else None
    lib().orc_probe_bake(_p(_f32(blob)), _p(P), _p(_f32(lo)), _p(_f32(hi)), int(rays), int(seed),
                         int(index_base), _p(out), _p(se))
    return (out, se) if want_se else out


def probe_query(coef, P, lo, hi, x4, n4):
    P = np.ascontiguousarray(P, np.int32)
    x4, n4 = _f32(x4), _f32(n4)
    E = np.zeros((len(x4), 3))
    lib().orc_probe_query(_p(_f64(coef)), _p(P), _p(_f32(lo)), _p(_f32(hi)), _p(x4), _p(n4), len(x4), _p(E))
    return E


def probe_query_rt(coef, P, lo, hi, scene_blob, x4, n4, t=0.0):
    """Probe irradiance with ray-traced visibility ("+ RT"): (E [m][3], ambiguous [m] bool), the
    second flagging records whose visibility decisions flip under +-1e-5 of geometry."""
    P = np.ascontiguousarray(P, np.int32)
    x4, n4 = _f32(x4), _f32(n4)
    E = np.zeros((len(x4), 3))
    amb = np.zeros(len(x4), np.uint8)
    lib().orc_probe_query_rt(_p(_f64(coef)), _p(P), _p(_f32(lo)), _p(_f32(hi)), _p(_f32(scene_blob)), float(t),
                             _p(x4), _p(n4), len(x4), _p(E), _p(amb))
    return E, amb.astype(bool)


def visible(scene_blob, o, p, t=0.0, grow=0.0, end_tol=0.01):
    """1 when the segment o -> p is free of scene geometry (up to end_tol before p)."""
    return int(lib().orc_visible(_p(_f32(scene_blob)), float(t), float(grow), _p(_f64(o)), _p(_f64(p)),
                                 float(end_tol)))


def dyn_ao(tri9, x4, n4, rays, radius, seed=0):
    """Dynamic ambient occlusion: (AO [m], blocked ray counts [m], ambiguous [m] bool) for
    records x4, n4 against triangles tri9 ([T][9] world-space vertices)."""
    tri9 = _f32(np.asarray(tri9).reshape(-1, 9))
    x4, n4 = _f32(x4), _f32(n4)
    m = len(x4)
    ao = np.zeros(m)
    blocked = np.zeros(m, np.int32)
    amb = np.zeros(m, np.uint8)
    lib().orc_dyn_ao(_p(tri9), len(tri9), _p(x4), _p(n4), m, int(rays), float(radius), int(seed), _p(ao),
                     _p(blocked), _p(amb))
    return ao, blocked, amb.astype(bool)
