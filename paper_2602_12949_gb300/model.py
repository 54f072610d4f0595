"""Python face of the library: a model handle plus torch-tensor marshalling.

Tensors are plain containers here (device memory and streams); every step of
the query, shading, training and Monte Carlo paths runs in libniv's kernels.
"""
import ctypes
import os
import struct

import numpy as np
import torch

from . import _lib
from ._lib import check, lib, ModelDesc, QueryParams, FitParams, UpsampleParams

PRECISIONS = {"fp32": _lib.NIV_FP32, "fp16": _lib.NIV_FP16, "fp8": _lib.NIV_FP8}


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _rec_dtype(t):
    if t.dtype == torch.float16:
        return _lib.NIV_F16
    if t.dtype == torch.float32:
        return _lib.NIV_F32
    raise TypeError("records must be float16 or float32, got %s" % t.dtype)


def _check_records(t, name, n=None, dtype=None):
    """A contiguous [n][4] device tensor of FP16 or FP32 records (the kernels read and write
    whole records, so a wrong shape or type would take them outside the buffer)."""
    if not isinstance(t, torch.Tensor) or t.dim() != 2 or t.shape[1] != 4 or not t.is_contiguous():
        raise ValueError("%s must be a contiguous [n][4] tensor" % name)
    if not t.is_cuda:
        raise ValueError("%s must live on the GPU (use query_host for host buffers)" % name)
    if t.dtype not in (torch.float16, torch.float32) or (dtype is not None and t.dtype != dtype):
        raise TypeError("%s must hold %s records, got %s" % (name, dtype or "float16 or float32", t.dtype))
    if n is not None and t.shape[0] != n:
        raise ValueError("%s must hold %d records, got %d" % (name, n, t.shape[0]))


def _check_dev(t, name, dtype, shape):
    """A contiguous device tensor of the given dtype and shape."""
    if not isinstance(t, torch.Tensor) or not t.is_cuda or not t.is_contiguous():
        raise ValueError("%s must be a contiguous CUDA tensor" % name)
    if t.dtype != dtype:
        raise TypeError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s, got %s" % (name, tuple(shape), tuple(t.shape)))


def _cuda_device(device):
    d = torch.device(device)
    if d.type != "cuda":
        raise ValueError("device must be a CUDA device, got %s" % d)
    return d


class NIVModel:
    """One Neural Irradiance Volume on the current CUDA device."""

    def __init__(self, dims=3, levels=16, feat=2, log2_T=17, base=16.0, growth=1.38, n_hidden=2, width=64,
                 in_extra=None, out_dim=3, out_act=1, prime_t=0x9E3779B1, pe_bands=0, t_bands=0):
        if in_extra is None:
            in_extra = 4 if dims == 4 else 3
        self.desc = ModelDesc(dims, levels, feat, log2_T, float(base), float(growth), n_hidden, width, in_extra,
                              out_dim, out_act, prime_t, pe_bands, t_bands)
        h = ctypes.c_void_p()
        check(lib().niv_create(ctypes.byref(self.desc), ctypes.byref(h)))
        self._h = h

    # model files: "NIVM", version, the description field by field, the count, the FP32 parameters
    # (then, from version 2, the optimiser state; see niv.h)
    _FILE_HEAD = struct.Struct("<4sI4i2d5iI2iq")

    def save(self, path, stream=None):
        """Write the description, the FP32 master parameters and the optimiser state (Adam
        moments, step count, training forward) to `path` (niv_save)."""
        check(lib().niv_save(self._h, os.fsencode(path), _stream(stream)))

    @classmethod
    def load(cls, path):
        """A model read from a file written by save (niv_load), on the current device."""
        with open(path, "rb") as f:
            head = f.read(cls._FILE_HEAD.size)
        h = ctypes.c_void_p()
        check(lib().niv_load(os.fsencode(path), ctypes.byref(h)))  # checks the header itself
        fields = cls._FILE_HEAD.unpack(head)[2:16]
        self = cls.__new__(cls)
        self.desc = ModelDesc(*fields)
        self._h = h
        return self

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().niv_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    @property
    def n_in(self):
        return (self.desc.levels * self.desc.feat + 6 * self.desc.pe_bands + self.desc.in_extra
                + 2 * self.desc.t_bands)

    def param_count(self):
        g, m = ctypes.c_int64(), ctypes.c_int64()
        check(lib().niv_param_count(self._h, ctypes.byref(g), ctypes.byref(m)))
        return g.value, m.value

    def level_info(self, level):
        r, d, f, e = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int64(), ctypes.c_int64()
        check(lib().niv_level_info(self._h, level, ctypes.byref(r), ctypes.byref(d), ctypes.byref(f),
                                   ctypes.byref(e)))
        return {"res": r.value, "dense": d.value, "first_entry": f.value, "entries": e.value}

    def layer_shapes(self):
        shapes, k = [], self.n_in
        for _ in range(self.desc.n_hidden):
            shapes.append((self.desc.width, k))
            k = self.desc.width
        shapes.append((self.desc.out_dim, k))
        return shapes

    def set_params(self, params):
        """Load the flat FP32 vector [grid | network] (numpy array or torch tensor, host or device)."""
        if isinstance(params, np.ndarray):
            params = np.ascontiguousarray(params, np.float32)
            ptr, n = params.ctypes.data, params.size
        else:
            params = params.contiguous().float()
            ptr, n = params.data_ptr(), params.numel()
        check(lib().niv_set_params(self._h, ctypes.c_void_p(ptr), n, _stream()))

    def get_params(self):
        g, m = self.param_count()
        out = np.empty(g + m, np.float32)
        check(lib().niv_get_params(self._h, ctypes.c_void_p(out.ctypes.data), out.size, _stream()))
        return out

    @staticmethod
    def query_params(aabb_min=(0.0, 0.0, 0.0), aabb_max=(1.0, 1.0, 1.0), t=0.0, image_width=0):
        return QueryParams((ctypes.c_float * 3)(*aabb_min), (ctypes.c_float * 3)(*aabb_max), float(t),
                           int(image_width))

    def query(self, pos, nrm, out=None, precision="fp16", aabb_min=(0.0, 0.0, 0.0), aabb_max=(1.0, 1.0, 1.0),
              t=0.0, image_width=0, out_dtype=None, stream=None):
        """E(x, n) for every record of device tensors pos, nrm ([n][4]); returns out ([n][4])."""
        _check_records(pos, "pos")
        _check_records(nrm, "nrm")
        if pos.shape != nrm.shape or pos.dtype != nrm.dtype:
            raise ValueError("pos and nrm must have the same shape and dtype")
        if out is None:
            out = torch.empty(pos.shape, dtype=out_dtype or pos.dtype, device=pos.device)
        _check_records(out, "out")
        if out.shape[0] != pos.shape[0]:
            raise ValueError("out must have one record per query")
        qp = self.query_params(aabb_min, aabb_max, t, image_width)
        check(lib().niv_query(self._h, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(nrm.data_ptr()),
                              pos.shape[0], _rec_dtype(pos), ctypes.byref(qp), ctypes.c_void_p(out.data_ptr()),
                              _rec_dtype(out), PRECISIONS[precision], _stream(stream)))
        return out

    def query_sub(self, pos, nrm, width, height, sub=2, out=None, precision="fp16", aabb_min=(0.0, 0.0, 0.0),
                  aabb_max=(1.0, 1.0, 1.0), t=0.0, out_dtype=None, stream=None):
        """E at the pixels (sub x, sub y) of a width x height G-buffer (device [H*W][4] records);
        returns out ([h*w][4], h = ceil(height / sub), w = ceil(width / sub))."""
        _check_records(pos, "pos")
        _check_records(nrm, "nrm")
        if pos.shape != nrm.shape or pos.dtype != nrm.dtype or pos.shape[0] != width * height:
            raise ValueError("pos and nrm must both hold width * height records of one dtype")
        n_low = ((width + sub - 1) // sub) * ((height + sub - 1) // sub)
        if out is None:
            out = torch.empty((n_low, 4), dtype=out_dtype or pos.dtype, device=pos.device)
        _check_records(out, "out")
        if out.shape[0] != n_low:
            raise ValueError("out must hold ceil(width / sub) * ceil(height / sub) records")
        qp = self.query_params(aabb_min, aabb_max, t, 0)
        check(lib().niv_query_sub(self._h, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(nrm.data_ptr()),
                                  int(width), int(height), int(sub), _rec_dtype(pos), ctypes.byref(qp),
                                  ctypes.c_void_p(out.data_ptr()), _rec_dtype(out), PRECISIONS[precision],
                                  _stream(stream)))
        return out

    def query_shade(self, pos, nrm, albedo, direct, out=None, precision="fp16", aabb_min=(0.0, 0.0, 0.0),
                    aabb_max=(1.0, 1.0, 1.0), t=0.0, image_width=0, stream=None):
        """Fused query + shading: FP16 rgba = (albedo * E / pi + direct, 1) for every record."""
        _check_records(pos, "pos")
        n = pos.shape[0]
        _check_records(nrm, "nrm", n, pos.dtype)
        _check_records(albedo, "albedo", n, torch.float16)
        _check_records(direct, "direct", n, torch.float16)
        if out is None:
            out = torch.empty((n, 4), dtype=torch.float16, device=pos.device)
        _check_records(out, "out", n, torch.float16)
        qp = self.query_params(aabb_min, aabb_max, t, image_width)
        check(lib().niv_query_shade(self._h, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(nrm.data_ptr()),
                                    ctypes.c_void_p(albedo.data_ptr()), ctypes.c_void_p(direct.data_ptr()),
                                    pos.shape[0], _rec_dtype(pos), ctypes.byref(qp), ctypes.c_void_p(out.data_ptr()),
                                    PRECISIONS[precision], _stream(stream)))
        return out

    def query_host(self, pos, nrm, out=None, precision="fp16", aabb_min=(0.0, 0.0, 0.0),
                   aabb_max=(1.0, 1.0, 1.0), t=0.0, image_width=0, stream=None):
        """Same as query for host arrays (numpy or CPU tensors), copied or read in place inside
        the call (page-locked buffers are read and written by the kernel directly)."""
        to_np = (lambda a: a.numpy()) if isinstance(pos, torch.Tensor) else (lambda a: a)
        p, n = np.ascontiguousarray(to_np(pos)), np.ascontiguousarray(to_np(nrm))
        if p.ndim != 2 or p.shape[1] != 4 or p.shape != n.shape or p.dtype != n.dtype:
            raise ValueError("pos and nrm must be matching [n][4] arrays")
        if p.dtype not in (np.float16, np.float32):
            raise TypeError("pos and nrm must hold float16 or float32 records, got %s" % p.dtype)
        dt = _lib.NIV_F16 if p.dtype == np.float16 else _lib.NIV_F32
        if out is None:
            out = np.empty(p.shape, p.dtype)
        o = to_np(out) if isinstance(out, torch.Tensor) else out
        if not (isinstance(o, np.ndarray) and o.flags["C_CONTIGUOUS"] and o.shape == p.shape):
            raise ValueError("out must be a contiguous [n][4] array")
        if o.dtype not in (np.float16, np.float32):
            raise TypeError("out must hold float16 or float32 records, got %s" % o.dtype)
        odt = _lib.NIV_F16 if o.dtype == np.float16 else _lib.NIV_F32
        # a per-frame call: the parameter block is cached and the pointers are passed as ints
        key = (tuple(aabb_min), tuple(aabb_max), float(t), int(image_width))
        cache = self.__dict__.setdefault("_qp_cache", {})
        qp = cache.get(key)
        if qp is None:
            if len(cache) >= 64:
                cache.clear()
            qp = cache[key] = self.query_params(*key)
        check(lib().niv_query_host(self._h, p.__array_interface__["data"][0], n.__array_interface__["data"][0],
                                   p.shape[0], dt, ctypes.byref(qp), o.__array_interface__["data"][0], odt,
                                   PRECISIONS[precision], _stream(stream)))
        return out

    def _train_args(self, pos, nrm, target, t):
        _check_records(pos, "pos", None, torch.float32)
        for a, name in ((nrm, "nrm"), (target, "target")):
            _check_records(a, name, pos.shape[0], torch.float32)
        tp = 0
        if t is not None:
            if t.dtype != torch.float32 or not t.is_cuda or t.numel() != pos.shape[0]:
                raise ValueError("t must be a float32 device vector with one value per sample")
            tp = t.contiguous().data_ptr()
        return tp

    def grad(self, pos, nrm, target, t=None, aabb_min=(0.0, 0.0, 0.0), aabb_max=(1.0, 1.0, 1.0), loss_eps=0.01,
             stream=None):
        """Loss (Eq. 3) of the batch; gradients land in the model's gradient buffer."""
        tp = self._train_args(pos, nrm, target, t)
        qp = self.query_params(aabb_min, aabb_max, 0.0, 0)
        loss = ctypes.c_double()
        check(lib().niv_grad(self._h, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(nrm.data_ptr()),
                             ctypes.c_void_p(tp), ctypes.c_void_p(target.data_ptr()), pos.shape[0], ctypes.byref(qp),
                             float(loss_eps), ctypes.byref(loss), _stream(stream)))
        return loss.value

    def set_train_forward(self, precision):
        """Forward precision of grad / fit / backward: "fp32" (default) or "fp16" (the FP16 path of
        the query, straight-through gradients onto the FP32 master parameters)."""
        check(lib().niv_set_train_forward(self._h, PRECISIONS[precision]))

    def backward(self, pos, nrm, grad_E, t=None, aabb_min=(0.0, 0.0, 0.0), aabb_max=(1.0, 1.0, 1.0), t_scalar=0.0,
                 stream=None):
        """Vector-Jacobian product: dL/dtheta for the upstream dL/dE (device float32 [n][4]
        records, xyz used) lands in the model's gradient buffer."""
        tp = self._train_args(pos, nrm, grad_E, t)
        qp = self.query_params(aabb_min, aabb_max, t_scalar, 0)
        check(lib().niv_backward(self._h, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(nrm.data_ptr()),
                                 ctypes.c_void_p(tp), ctypes.c_void_p(grad_E.data_ptr()), pos.shape[0],
                                 ctypes.byref(qp), _stream(stream)))

    def grads_into(self, out):
        """Copy the gradient buffer into a float32 tensor of param_count() values (host or device)."""
        if not isinstance(out, torch.Tensor) or out.dtype != torch.float32 or not out.is_contiguous():
            raise TypeError("out must be a contiguous float32 tensor")
        check(lib().niv_get_grads(self._h, ctypes.c_void_p(out.data_ptr()), out.numel(), _stream()))
        return out

    def get_grads(self):
        g, m = self.param_count()
        out = np.empty(g + m, np.float32)
        check(lib().niv_get_grads(self._h, ctypes.c_void_p(out.ctypes.data), out.size, _stream()))
        return out

    def set_grads(self, grads):
        grads = np.ascontiguousarray(grads, np.float32)
        check(lib().niv_set_grads(self._h, ctypes.c_void_p(grads.ctypes.data), grads.size, _stream()))

    def adam_step(self, lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-15, stream=None):
        check(lib().niv_adam_step(self._h, float(lr), float(beta1), float(beta2), float(eps), _stream(stream)))

    def fit(self, pos, nrm, target, t=None, aabb_min=(0.0, 0.0, 0.0), aabb_max=(1.0, 1.0, 1.0), lr=1e-2,
            beta1=0.9, beta2=0.99, adam_eps=1e-15, loss_eps=0.01, want_loss=True, stream=None):
        """One optimisation step (Sec. 4.5) on the batch; returns the batch loss (or None)."""
        tp = self._train_args(pos, nrm, target, t)
        qp = self.query_params(aabb_min, aabb_max, 0.0, 0)
        fp = FitParams(lr, beta1, beta2, adam_eps, loss_eps)
        loss = ctypes.c_double()
        check(lib().niv_fit(self._h, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(nrm.data_ptr()),
                            ctypes.c_void_p(tp), ctypes.c_void_p(target.data_ptr()), pos.shape[0], ctypes.byref(qp),
                            ctypes.byref(fp), ctypes.byref(loss) if want_loss else None, _stream(stream)))
        return loss.value if want_loss else None

    def fp8_calibrate(self, pos, nrm, aabb_min=(0.0, 0.0, 0.0), aabb_max=(1.0, 1.0, 1.0), t=0.0, stream=None):
        """Set the E4M3 path's activation scales from device records pos, nrm ([n][4])."""
        _check_records(pos, "pos")
        _check_records(nrm, "nrm", pos.shape[0], pos.dtype)
        qp = self.query_params(aabb_min, aabb_max, t, 0)
        check(lib().niv_fp8_calibrate(self._h, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(nrm.data_ptr()),
                                      pos.shape[0], _rec_dtype(pos), ctypes.byref(qp), _stream(stream)))

    def fp8_scales(self):
        """(activation scales, weight scales, activation amax), one entry per matrix product."""
        n = self.desc.n_hidden + 1
        sa, sw, am = (np.zeros(n, np.float32) for _ in range(3))
        check(lib().niv_fp8_get_scales(self._h, ctypes.c_void_p(sa.ctypes.data), ctypes.c_void_p(sw.ctypes.data),
                                       ctypes.c_void_p(am.ctypes.data), n))
        return sa, sw, am

    def encode(self, pos, aabb_min=(0.0, 0.0, 0.0), aabb_max=(1.0, 1.0, 1.0), t=0.0, want_idx=True, stream=None):
        """(encoding [n][L*F + 6*pe_bands] float32, corner indices [n][L][2^dims] int32 or None)
        for device records."""
        _check_records(pos, "pos")
        n = pos.shape[0]
        L, F, nc = self.desc.levels, self.desc.feat, 1 << self.desc.dims
        enc = torch.empty((n, L * F + 6 * self.desc.pe_bands), dtype=torch.float32, device=pos.device)
        idx = torch.empty((n, L, nc), dtype=torch.int32, device=pos.device) if want_idx else None
        qp = self.query_params(aabb_min, aabb_max, t, 0)
        check(lib().niv_encode(self._h, ctypes.c_void_p(pos.data_ptr()), n, _rec_dtype(pos), ctypes.byref(qp),
                               ctypes.c_void_p(enc.data_ptr()),
                               ctypes.c_void_p(idx.data_ptr() if idx is not None else 0), _stream(stream)))
        return enc, idx


class _QueryFunction(torch.autograd.Function):
    """E(x, n; theta) in FP32 with the hand-written backward (Sec. 4.5) as its gradient."""

    @staticmethod
    def forward(ctx, params, pos, nrm, model, aabb_min, aabb_max, t):
        model.set_params(params.detach())
        E = model.query(pos, nrm, precision="fp32", out_dtype=torch.float32, aabb_min=aabb_min, aabb_max=aabb_max,
                        t=t)
        ctx.save_for_backward(pos, nrm)
        ctx.model, ctx.box, ctx.t = model, (aabb_min, aabb_max), t
        return E

    @staticmethod
    def backward(ctx, grad_E):
        pos, nrm = ctx.saved_tensors
        model = ctx.model
        model.backward(pos, nrm, grad_E.detach().contiguous().float(), aabb_min=ctx.box[0], aabb_max=ctx.box[1],
                       t_scalar=ctx.t)
        g, m = model.param_count()
        grad = model.grads_into(torch.empty(g + m, dtype=torch.float32, device=grad_E.device))
        return grad, None, None, None, None, None, None


class NIVModule(torch.nn.Module):
    """A model as a torch module: the flat FP32 parameter vector [grid | network] is an
    nn.Parameter, forward returns E ([n][4] float32 records) from the FP32 query, and autograd
    runs the library's hand-written backward (niv_backward)."""

    def __init__(self, model, params, aabb_min=(0.0, 0.0, 0.0), aabb_max=(1.0, 1.0, 1.0), device="cuda"):
        super().__init__()
        self.model = model
        self.aabb_min, self.aabb_max = tuple(aabb_min), tuple(aabb_max)
        self.params = torch.nn.Parameter(torch.as_tensor(np.asarray(params, np.float32), device=device).clone())

    def forward(self, pos, nrm, t=0.0):
        return _QueryFunction.apply(self.params, pos, nrm, self.model, self.aabb_min, self.aabb_max, float(t))


class DynamicGeometry:
    """The frame's dynamic triangles (host float32 [T][9], world space) in a bounding-volume
    hierarchy on the current device, for the dynamic ambient-occlusion pass (Sec. 4.4)."""

    def __init__(self, tri9):
        tri9 = np.ascontiguousarray(np.asarray(tri9, np.float32).reshape(-1, 9))
        h = ctypes.c_void_p()
        check(lib().niv_dyn_create(ctypes.c_void_p(tri9.ctypes.data), len(tri9), ctypes.byref(h)))
        self._h = h
        self.n_tris = len(tri9)

    @property
    def node_count(self):
        return int(lib().niv_dyn_node_count(self._h))

    def ao(self, pos, nrm, rays=8, radius=0.5, seed=0, out=None, E=None, stream=None):
        """AO in [0, 1] per device record (float32 [n]); E ([n][4] device records, optional) is
        scaled by it in place."""
        _check_records(pos, "pos")
        n = pos.shape[0]
        _check_records(nrm, "nrm", n, pos.dtype)
        if out is None:
            out = torch.empty(n, dtype=torch.float32, device=pos.device)
        _check_dev(out, "out", torch.float32, (n,))
        if E is not None:
            _check_records(E, "E", n)
        check(lib().niv_dyn_ao(self._h, ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(nrm.data_ptr()),
                               pos.shape[0], _rec_dtype(pos), int(rays), float(radius), int(seed),
                               ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(E.data_ptr() if E is not None else 0),
                               _rec_dtype(E) if E is not None else 0, _stream(stream)))
        return out

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            lib().niv_dyn_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def upsample_shade(pos, nrm, albedo, direct, width, height, E_low, sub=2, power=8.0, sigma=0.05, eps=1e-4,
                   out=None, stream=None):
    """Full-resolution FP16 rgba from irradiance E_low queried at every sub-th pixel (joint
    bilateral upsampling guided by the G-buffer, then albedo * E / pi + direct)."""
    n = int(width) * int(height)
    _check_records(pos, "pos", n)
    _check_records(nrm, "nrm", n, pos.dtype)
    _check_records(albedo, "albedo", n, torch.float16)
    _check_records(direct, "direct", n, torch.float16)
    if int(sub) >= 1:  # the library refuses sub < 1 itself
        n_low = ((int(width) + int(sub) - 1) // int(sub)) * ((int(height) + int(sub) - 1) // int(sub))
        _check_records(E_low, "E_low", n_low)
    else:
        _check_records(E_low, "E_low")
    if out is None:
        out = torch.empty((n, 4), dtype=torch.float16, device=pos.device)
    _check_records(out, "out", n, torch.float16)
    up = UpsampleParams(float(power), float(sigma), float(eps))
    check(lib().niv_upsample_shade(ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(nrm.data_ptr()),
                                   ctypes.c_void_p(albedo.data_ptr()), ctypes.c_void_p(direct.data_ptr()),
                                   int(width), int(height), _rec_dtype(pos), ctypes.c_void_p(E_low.data_ptr()),
                                   _rec_dtype(E_low), int(sub), ctypes.byref(up), ctypes.c_void_p(out.data_ptr()),
                                   _stream(stream)))
    return out


def shade(albedo, direct, E, out=None, stream=None):
    """rgba = (albedo * E / pi + direct, 1) on FP16 [n][4] device tensors."""
    _check_records(E, "E", None, torch.float16)
    for t, name in ((albedo, "albedo"), (direct, "direct")):
        _check_records(t, name, E.shape[0], torch.float16)
    if out is None:
        out = torch.empty_like(E)
    _check_records(out, "out", E.shape[0], torch.float16)
    check(lib().niv_shade(ctypes.c_void_p(albedo.data_ptr()), ctypes.c_void_p(direct.data_ptr()),
                          ctypes.c_void_p(E.data_ptr()), E.shape[0], ctypes.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def mc_irradiance(scene_blob, x4, n4, spp, seed=0, mode="indirect", t=None, index_base=0, stream=None):
    """Monte Carlo irradiance (Eq. 1) at device points x4 / normals n4 ([m][4] float32).

    Returns (E [m][3] float64 device tensor, keep [m] uint8 device tensor)."""
    blob = np.ascontiguousarray(scene_blob, np.float32)
    _check_records(x4, "x4", None, torch.float32)
    m = x4.shape[0]
    _check_records(n4, "n4", m, torch.float32)
    E = torch.empty((m, 3), dtype=torch.float64, device=x4.device)
    keep = torch.empty(m, dtype=torch.uint8, device=x4.device)
    tp = 0
    if t is not None:
        _check_dev(t, "t", torch.float32, (m,))
        tp = t.data_ptr()
    md = {"total": _lib.NIV_MC_TOTAL, "indirect": _lib.NIV_MC_INDIRECT}[mode]
    check(lib().niv_mc_irradiance(ctypes.c_void_p(blob.ctypes.data), blob.size, ctypes.c_void_p(x4.data_ptr()),
                                  ctypes.c_void_p(n4.data_ptr()), ctypes.c_void_p(tp), m, int(spp), int(seed),
                                  int(index_base), md, ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(keep.data_ptr()),
                                  _stream(stream)))
    return E, keep


def training_samples(scene_blob, n, surface_frac=0.2, seed=0, index_base=0, with_t=False, want_patch=False,
                     device="cuda", stream=None):
    """Training-sample candidates of Sec. 4.5 / App. I on the device (niv_training_samples):
    (x4 [n][4], n4 [n][4], t [n] or None, patch [n] int32 or None), float32 device tensors."""
    blob = np.ascontiguousarray(scene_blob, np.float32)
    device = _cuda_device(device)
    x4 = torch.empty((n, 4), dtype=torch.float32, device=device)
    n4 = torch.empty((n, 4), dtype=torch.float32, device=device)
    t = torch.empty(n, dtype=torch.float32, device=device) if with_t else None
    patch = torch.empty(n, dtype=torch.int32, device=device) if want_patch else None
    check(lib().niv_training_samples(ctypes.c_void_p(blob.ctypes.data), blob.size, int(n), float(surface_frac),
                                     int(seed), int(index_base), ctypes.c_void_p(x4.data_ptr()),
                                     ctypes.c_void_p(n4.data_ptr()), ctypes.c_void_p(t.data_ptr() if t is not None else 0),
                                     ctypes.c_void_p(patch.data_ptr() if patch is not None else 0), _stream(stream)))
    return x4, n4, t, patch


def gbuffer_raycast(scene_blob, width, height, eye, vfov_deg=60.0, t=0.0, dtype=torch.float16, want_albedo=True,
                    want_hit=False, device="cuda", stream=None):
    """Primary-visibility G-buffer of the analytic scene on the device (niv_gbuffer_raycast):
    (pos [W*H][4], nrm [W*H][4], albedo [W*H][4] or None, hit [W*H] uint8 or None), records of
    ``dtype`` (float16 or float32), row 0 at the top."""
    blob = np.ascontiguousarray(scene_blob, np.float32)
    eye3 = np.ascontiguousarray(eye, np.float32).reshape(3)
    device = _cuda_device(device)
    if dtype not in (torch.float16, torch.float32):
        raise TypeError("dtype must be torch.float16 or torch.float32")
    n = int(width) * int(height)
    pos, nrm = (torch.empty((n, 4), dtype=dtype, device=device) for _ in range(2))
    alb = torch.empty((n, 4), dtype=dtype, device=device) if want_albedo else None
    hit = torch.empty(n, dtype=torch.uint8, device=device) if want_hit else None
    check(lib().niv_gbuffer_raycast(ctypes.c_void_p(blob.ctypes.data), blob.size, int(width), int(height),
                                    float(vfov_deg), ctypes.c_void_p(eye3.ctypes.data), float(t),
                                    ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(nrm.data_ptr()),
                                    ctypes.c_void_p(alb.data_ptr() if alb is not None else 0), _rec_dtype(pos),
                                    ctypes.c_void_p(hit.data_ptr() if hit is not None else 0), _stream(stream)))
    return pos, nrm, alb, hit


def gbuffer_meshes(tri9, tri_mesh, mesh_albedo, pos, nrm, alb, hit, width, height, eye, vfov_deg=60.0,
                   want_mesh_id=False, stream=None):
    """Insert triangle meshes into a G-buffer in place (niv_gbuffer_meshes): tri9 device float32
    [T][9], tri_mesh device int32 [T], mesh_albedo host [M][3]; pos/nrm/alb records and hit
    (uint8) as made by gbuffer_raycast.  Returns the mesh index per pixel (int32, -1: none) or None."""
    alb3 = np.ascontiguousarray(mesh_albedo, np.float32).reshape(-1, 3)
    eye3 = np.ascontiguousarray(eye, np.float32).reshape(3)
    n = int(width) * int(height)
    if not isinstance(tri9, torch.Tensor) or tri9.dim() != 2:
        raise ValueError("tri9 must be a [T][9] tensor")
    T = tri9.shape[0]
    _check_dev(tri9, "tri9", torch.float32, (T, 9))
    _check_dev(tri_mesh, "tri_mesh", torch.int32, (T,))
    _check_records(pos, "pos", n)
    _check_records(nrm, "nrm", n, pos.dtype)
    if alb is not None:
        _check_records(alb, "alb", n, pos.dtype)
    _check_dev(hit, "hit", torch.uint8, (n,))
    scratch = torch.empty(n, dtype=torch.int64, device=pos.device)
    mesh_id = torch.empty(n, dtype=torch.int32, device=pos.device) if want_mesh_id else None
    ptr = lambda t: ctypes.c_void_p(t.data_ptr() if t is not None else 0)
    check(lib().niv_gbuffer_meshes(ptr(tri9), ptr(tri_mesh), int(tri9.shape[0]), ctypes.c_void_p(alb3.ctypes.data),
                                   len(alb3), int(width), int(height), float(vfov_deg), ctypes.c_void_p(eye3.ctypes.data),
                                   ptr(pos), ptr(nrm), ptr(alb), _rec_dtype(pos), ptr(hit), ptr(mesh_id), ptr(scratch),
                                   _stream(stream)))
    return mesh_id


def compact_targets(x4, n4, E, keep, t=None, stream=None):
    """Kept samples in order: (x4, n4, target4, t or None), each cut to the kept count."""
    _check_records(x4, "x4", None, torch.float32)
    m = x4.shape[0]
    _check_records(n4, "n4", m, torch.float32)
    _check_dev(E, "E", torch.float64, (m, 3))
    _check_dev(keep, "keep", torch.uint8, (m,))
    if t is not None:
        _check_dev(t, "t", torch.float32, (m,))
    ox, on, ot4 = (torch.empty((m, 4), dtype=torch.float32, device=x4.device) for _ in range(3))
    ot = torch.empty(m, dtype=torch.float32, device=x4.device) if t is not None else None
    cnt = ctypes.c_int64()
    check(lib().niv_compact_targets(ctypes.c_void_p(x4.data_ptr()), ctypes.c_void_p(n4.data_ptr()),
                                    ctypes.c_void_p(t.data_ptr() if t is not None else 0),
                                    ctypes.c_void_p(E.data_ptr()), ctypes.c_void_p(keep.data_ptr()), m,
                                    ctypes.c_void_p(ox.data_ptr()), ctypes.c_void_p(on.data_ptr()),
                                    ctypes.c_void_p(ot.data_ptr() if ot is not None else 0),
                                    ctypes.c_void_p(ot4.data_ptr()), ctypes.byref(cnt), _stream(stream)))
    k = cnt.value
    return ox[:k], on[:k], ot4[:k], (ot[:k] if ot is not None else None)


class ProbeGrid:
    """SH probe lattice over [lo, hi] with P[0] x P[1] x P[2] probes (App. A); FP16 coefficients."""

    def __init__(self, P, lo, hi, device="cuda"):
        self.P = np.ascontiguousarray(P, np.int32)
        self.lo = np.ascontiguousarray(lo, np.float32)
        self.hi = np.ascontiguousarray(hi, np.float32)
        self.count = int(np.prod(self.P))
        self.coef16 = torch.zeros((self.count, 28), dtype=torch.float16, device=_cuda_device(device))

    @property
    def nbytes(self):
        return 54 * self.count  # coefficient bytes (the stored records add a 2-byte pad)

    def bake(self, scene_blob, rays, seed=0, index_base=0, want_f64=False, stream=None):
        blob = np.ascontiguousarray(scene_blob, np.float32)
        c64 = torch.empty((self.count, 27), dtype=torch.float64, device=self.coef16.device) if want_f64 else None
        check(lib().niv_probe_bake(ctypes.c_void_p(blob.ctypes.data), blob.size, ctypes.c_void_p(self.P.ctypes.data),
                                   ctypes.c_void_p(self.lo.ctypes.data), ctypes.c_void_p(self.hi.ctypes.data),
                                   int(rays), int(seed), int(index_base),
                                   ctypes.c_void_p(c64.data_ptr() if c64 is not None else 0),
                                   ctypes.c_void_p(self.coef16.data_ptr()), _stream(stream)))
        return c64

    def query(self, pos, nrm, out=None, image_width=0, out_dtype=None, scene_blob=None, t=0.0, stream=None):
        """Probe irradiance at device records; with scene_blob, probes are rejected by
        ray-traced visibility ("+ RT") instead of the cosine fall-off."""
        _check_records(pos, "pos")
        _check_records(nrm, "nrm", pos.shape[0], pos.dtype)
        if out is None:
            out = torch.empty(pos.shape, dtype=out_dtype or pos.dtype, device=pos.device)
        _check_records(out, "out", pos.shape[0])
        grid = (ctypes.c_void_p(self.coef16.data_ptr()), ctypes.c_void_p(self.P.ctypes.data),
                ctypes.c_void_p(self.lo.ctypes.data), ctypes.c_void_p(self.hi.ctypes.data))
        recs = (ctypes.c_void_p(pos.data_ptr()), ctypes.c_void_p(nrm.data_ptr()), pos.shape[0], _rec_dtype(pos),
                ctypes.c_void_p(out.data_ptr()), _rec_dtype(out), int(image_width), _stream(stream))
        if scene_blob is None:
            check(lib().niv_probe_query(*grid, *recs))
        else:
            blob = np.ascontiguousarray(scene_blob, dtype=np.float32)
            check(lib().niv_probe_query_rt(*grid, ctypes.c_void_p(blob.ctypes.data), blob.size, float(t), *recs))
        return out


def sync_status(stream=None):
    check(lib().niv_sync_status(_stream(stream)))
