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
