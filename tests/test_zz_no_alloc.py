"""The allocation-free host query against the ordinary host query, through the C ABI.

niv_query_host_noalloc serves callers that cannot let the library allocate device
memory (a render loop with a fixed GPU budget, a plug-in whose host owns all device
allocation): it stages records in a fixed device array instead of a library
allocation.  Its results must equal niv_query_host's on the same inputs, call after
call, with the array reused.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

from niv_inputs import init_params, uniform_queries
from niv_inputs.configs import MODEL_C1, ROOM_MIN, ROOM_MAX

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MAX_RECORDS = 65536  # NIV_NOALLOC_MAX_RECORDS in include/niv.h
FP16_BOUND = 2e-3    # the FP16 path's parity bound used by the other GPU tests


@pytest.fixture(scope="module")
def niv():
    from paper_2602_12949_gb300.build import build
    build()
    import paper_2602_12949_gb300 as P
    return P


def _noalloc(P, m, pos, nrm, precision, qp):
    from paper_2602_12949_gb300 import _lib
    out = np.zeros(pos.shape, pos.dtype)
    dt = _lib.NIV_F16 if pos.dtype == np.float16 else _lib.NIV_F32
    rc = P.lib().niv_query_host_noalloc(m.handle, ctypes.c_void_p(pos.ctypes.data), ctypes.c_void_p(nrm.ctypes.data),
                                        len(pos), dt, ctypes.byref(qp), ctypes.c_void_p(out.ctypes.data), dt,
                                        P.PRECISIONS[precision],
                                        ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, out


def _rel(got, ref):
    got, ref = got.astype(np.float64), ref.astype(np.float64)
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    return float(np.max(np.abs(got - ref) / den))


@pytest.mark.parametrize("precision,dtype", [("fp16", np.float16), ("fp32", np.float32)])
def test_noalloc_query_matches_host_query_on_consecutive_calls(niv, precision, dtype):
    m = niv.NIVModel(**MODEL_C1)
    g, _ = m.param_count()
    m.set_params(init_params(g, m.layer_shapes(), seed=11, bias_std=0.1))
    kw = dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)
    qp = m.query_params(ROOM_MIN, ROOM_MAX, 0.0, 0)
    for call, n in enumerate((MAX_RECORDS, 40000 + 7)):  # two calls in a row, the second smaller
        pos, nrm = uniform_queries(n, seed=100 + call, lo=ROOM_MIN, hi=ROOM_MAX, dtype=dtype)
        ref = m.query_host(pos, nrm, precision=precision, **kw)
        rc, out = _noalloc(niv, m, pos, nrm, precision, qp)
        assert rc == 0, niv.lib().niv_last_error()
        assert _rel(out[:, :3], ref[:, :3]) <= FP16_BOUND
        np.testing.assert_array_equal(out, ref)  # same kernel, same inputs: identical results
    m.close()


def test_noalloc_rejects_more_than_its_capacity(niv):
    m = niv.NIVModel(**MODEL_C1)
    pos, nrm = uniform_queries(MAX_RECORDS + 1, seed=1, dtype=np.float16)
    rc, _ = _noalloc(niv, m, pos, nrm, "fp16", m.query_params(ROOM_MIN, ROOM_MAX, 0.0, 0))
    assert rc == -1
    assert b"NIV_NOALLOC_MAX_RECORDS" in niv.lib().niv_last_error()
    m.close()


@pytest.mark.parametrize("precision", ["fp16", "fp32"])
def test_noalloc_query_after_a_training_step_uses_the_trained_parameters(niv, precision):
    """An Adam step changes the FP32 master parameters on the device; the allocation-free
    call must rebuild the inference copies first, as niv_query does, so both agree."""
    m = niv.NIVModel(**MODEL_C1)
    g, _ = m.param_count()
    m.set_params(init_params(g, m.layer_shapes(), seed=12, bias_std=0.1))
    tpos, tnrm = uniform_queries(8192, seed=7, lo=ROOM_MIN, hi=ROOM_MAX, dtype=np.float32)
    target = np.zeros_like(tpos)
    target[:, :3] = np.random.default_rng(8).uniform(0.1, 2.0, (len(tpos), 3))
    m.fit(torch.from_numpy(tpos).cuda(), torch.from_numpy(tnrm).cuda(), torch.from_numpy(target).cuda(),
          aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, lr=1e-2)
    pos, nrm = uniform_queries(30000 + 5, seed=9, lo=ROOM_MIN, hi=ROOM_MAX, dtype=np.float16)
    qp = m.query_params(ROOM_MIN, ROOM_MAX, 0.0, 0)
    rc, out = _noalloc(niv, m, pos, nrm, precision, qp)  # first: the call that must refresh
    assert rc == 0, niv.lib().niv_last_error()
    ref = m.query_host(pos, nrm, precision=precision, aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)
    np.testing.assert_array_equal(out, ref)
    m.close()


def test_noalloc_refuses_a_model_without_parameters(niv):
    m = niv.NIVModel(**MODEL_C1)
    pos, nrm = uniform_queries(100, seed=2, dtype=np.float16)
    rc, _ = _noalloc(niv, m, pos, nrm, "fp16", m.query_params(ROOM_MIN, ROOM_MAX, 0.0, 0))
    assert rc == -1
    assert b"parameters not set" in niv.lib().niv_last_error()
    m.close()
