"""The C-ABI library loads and exports every declared entry point; host-side argument checks."""
import ctypes
import glob
import os
import re

import pytest

from conftest import ROOT


@pytest.fixture(scope="module")
def libniv():
    from paper_2602_12949_gb300.build import build
    build()
    from paper_2602_12949_gb300 import lib
    return lib()


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        names |= set(re.findall(r"NIV_API\s+[\w\s\*]*?\b(niv_\w+)\s*\(", text))
    return names


def test_header_declares_entry_points():
    names = _declared()
    for required in ("niv_create", "niv_destroy", "niv_query", "niv_shade", "niv_set_params", "niv_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(libniv):
    missing = [n for n in sorted(_declared()) if not hasattr(libniv, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2602_12949_gb300 import _lib
    bound = {name for name, _, _ in _lib._SIGNATURES}
    assert _declared() <= bound, sorted(_declared() - bound)


def test_version_and_invalid_descriptions_fail_on_the_host(libniv):
    from paper_2602_12949_gb300._lib import ModelDesc, NIV_ERR_ARG, NIV_ERR_UNSUPPORTED
    assert b"sm_103a" in libniv.niv_version()
    h = ctypes.c_void_p()
    bad = [
        ModelDesc(5, 8, 2, 14, 4.0, 1.5, 2, 64, 3, 3, 1, 1),      # dims
        ModelDesc(3, 0, 2, 14, 4.0, 1.5, 2, 64, 3, 3, 1, 1),      # levels
        ModelDesc(3, 8, 2, 30, 4.0, 1.5, 2, 64, 3, 3, 1, 1),      # log2_T
        ModelDesc(3, 8, 2, 14, 0.5, 1.5, 2, 64, 3, 3, 1, 1),      # base
        ModelDesc(4, 8, 2, 14, 4.0, 1.5, 2, 64, 4, 3, 1, 2),      # even prime_t
    ]
    for d in bad:
        assert libniv.niv_create(ctypes.byref(d), ctypes.byref(h)) == NIV_ERR_ARG
        assert h.value is None
        assert libniv.niv_last_error()
    d = ModelDesc(3, 8, 3, 14, 4.0, 1.5, 2, 64, 3, 3, 1, 1)       # feat 3
    assert libniv.niv_create(ctypes.byref(d), ctypes.byref(h)) == NIV_ERR_UNSUPPORTED
    d = ModelDesc(3, 8, 2, 14, 4.0, 1.5, 2, 48, 3, 3, 1, 1)       # width 48
    assert libniv.niv_create(ctypes.byref(d), ctypes.byref(h)) == NIV_ERR_UNSUPPORTED


def test_null_handles_are_rejected(libniv):
    from paper_2602_12949_gb300._lib import NIV_ERR_ARG, QueryParams
    qp = QueryParams()
    assert libniv.niv_query(None, None, None, 10, 0, ctypes.byref(qp), None, 0, 0, None) == NIV_ERR_ARG
    assert libniv.niv_param_count(None, None, None) == NIV_ERR_ARG
    assert libniv.niv_shade(None, None, None, 4, None, None) == NIV_ERR_ARG
    assert libniv.niv_destroy(None) == 0


def test_model_files_are_checked_before_the_device(libniv, tmp_path):
    # niv_load refuses a missing file, a foreign file, another format version and a bad
    # description on the host, leaving *out unchanged
    import struct
    from paper_2602_12949_gb300._lib import NIV_ERR_ARG
    h = ctypes.c_void_p(1234)
    assert libniv.niv_load(str(tmp_path / "missing.niv").encode(), ctypes.byref(h)) == NIV_ERR_ARG
    foreign = tmp_path / "foreign.niv"
    foreign.write_bytes(b"PK\x03\x04" + bytes(100))
    assert libniv.niv_load(str(foreign).encode(), ctypes.byref(h)) == NIV_ERR_ARG
    assert b"magic" in libniv.niv_last_error()
    head = struct.Struct("<4sI4i2d5iI2iq")
    newer = tmp_path / "newer.niv"
    newer.write_bytes(head.pack(b"NIVM", 3, 3, 8, 2, 14, 4.0, 1.5, 2, 64, 3, 3, 1, 1, 0, 0, 10))
    assert libniv.niv_load(str(newer).encode(), ctypes.byref(h)) == NIV_ERR_ARG
    bad_desc = tmp_path / "bad.niv"
    bad_desc.write_bytes(head.pack(b"NIVM", 1, 5, 8, 2, 14, 4.0, 1.5, 2, 64, 3, 3, 1, 1, 0, 0, 10))  # dims 5
    assert libniv.niv_load(str(bad_desc).encode(), ctypes.byref(h)) == NIV_ERR_ARG
    short = tmp_path / "short.niv"
    short.write_bytes(b"NIVM\x01\x00\x00\x00" + bytes(6))
    assert libniv.niv_load(str(short).encode(), ctypes.byref(h)) == NIV_ERR_ARG
    assert h.value == 1234
    assert libniv.niv_save(None, b"x", None) == NIV_ERR_ARG


def test_gbuffer_raycast_arguments_fail_on_the_host(libniv):
    import numpy as np
    from paper_2602_12949_gb300._lib import NIV_ERR_ARG, NIV_ERR_ALIGN, NIV_F16, NIV_F32
    from niv_inputs import room_scene
    blob = np.ascontiguousarray(room_scene(0).blob(), np.float32)
    eye = np.zeros(3, np.float32)
    bp, ep = ctypes.c_void_p(blob.ctypes.data), ctypes.c_void_p(eye.ctypes.data)
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: every case fails before a launch

    def call(w=8, h=8, fov=60.0, pos=fake, nrm=fake, dt=NIV_F16, n=blob.size, scene=bp):
        return libniv.niv_gbuffer_raycast(scene, n, w, h, fov, ep, 0.0, pos, nrm, None, dt, None, None)

    assert call(scene=None) == NIV_ERR_ARG
    assert call(pos=None) == NIV_ERR_ARG
    assert call(w=0) == NIV_ERR_ARG
    assert call(h=-1) == NIV_ERR_ARG
    assert call(w=1 << 16, h=1 << 16) == NIV_ERR_ARG  # 2^32 pixels
    assert call(fov=0.0) == NIV_ERR_ARG
    assert call(fov=180.0) == NIV_ERR_ARG
    assert call(dt=7) == NIV_ERR_ARG
    assert call(n=blob.size - 1) == NIV_ERR_ARG
    assert call(pos=ctypes.c_void_p((1 << 20) + 8), dt=NIV_F32) == NIV_ERR_ALIGN
    assert call(nrm=ctypes.c_void_p((1 << 20) + 4)) == NIV_ERR_ALIGN
    assert libniv.niv_last_error()


def test_gbuffer_meshes_arguments_fail_on_the_host(libniv):
    import numpy as np
    from paper_2602_12949_gb300._lib import NIV_ERR_ARG, NIV_ERR_ALIGN, NIV_F16
    eye = np.zeros(3, np.float32)
    alb = np.ones((2, 3), np.float32)
    ep, ap = ctypes.c_void_p(eye.ctypes.data), ctypes.c_void_p(alb.ctypes.data)
    fake = ctypes.c_void_p(1 << 20)  # never dereferenced: every case fails before a launch

    def call(nt=4, nm=2, w=8, h=8, fov=60.0, pos=fake, scratch=fake, hit=fake, tri=fake, dt=NIV_F16):
        return libniv.niv_gbuffer_meshes(tri, fake, nt, ap, nm, w, h, fov, ep, pos, fake, None, dt, hit, None,
                                         scratch, None)

    assert call(hit=None) == NIV_ERR_ARG
    assert call(scratch=None) == NIV_ERR_ARG
    assert call(nt=-1) == NIV_ERR_ARG
    assert call(tri=None) == NIV_ERR_ARG
    assert call(nm=0) == NIV_ERR_ARG
    assert call(nm=65) == NIV_ERR_ARG
    assert call(w=0) == NIV_ERR_ARG
    assert call(fov=200.0) == NIV_ERR_ARG
    assert call(dt=3) == NIV_ERR_ARG
    assert call(pos=ctypes.c_void_p((1 << 20) + 4)) == NIV_ERR_ALIGN
    assert call(scratch=ctypes.c_void_p((1 << 20) + 4)) == NIV_ERR_ALIGN
