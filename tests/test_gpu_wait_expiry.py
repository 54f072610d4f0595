"""A bounded device wait that runs out is reported on the host, and the device stays usable.

Every tensor-core query kernel bounds its waits on the MMA-completion barrier; on expiry it
latches a failure code in the library's device status word, frees its tensor memory and
returns.  niv_selftest_wait_expiry runs that same bounded wait on a barrier phase that nothing
completes, with a short limit, so the expiry path runs without any fault.
"""
import ctypes
import time

import numpy as np
import pytest

import oracle
from niv_inputs import init_params, uniform_queries
from niv_inputs.configs import MODEL_C0

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def niv():
    from paper_2602_12949_gb300.build import build
    build()
    import paper_2602_12949_gb300 as P
    return P


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def test_wait_expiry_is_reported_and_the_device_stays_usable(niv):
    L = niv.lib()
    assert L.niv_sync_status(_stream()) == 0  # nothing latched before
    t0 = time.perf_counter()
    assert L.niv_selftest_wait_expiry(2000, _stream()) == 0  # a 2 ms limit
    rc = L.niv_sync_status(_stream())
    dt = time.perf_counter() - t0
    assert rc == niv._lib.NIV_ERR_DEVICE
    assert b"failure code 3" in L.niv_last_error()
    assert dt >= 2e-3  # the kernel did wait for its limit
    assert L.niv_sync_status(_stream()) == 0  # reading the status cleared it
    # a normal query on the same device afterwards runs and matches the oracle
    m = niv.NIVModel(**MODEL_C0)
    g, _ = m.param_count()
    params = init_params(g, m.layer_shapes(), seed=4)
    m.set_params(params)
    pos, nrm = uniform_queries(5000, seed=9)
    E = m.query(torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda(), precision="fp16",
                out_dtype=torch.float32)
    niv.sync_status()
    om = oracle.Model(**MODEL_C0)
    ref = oracle.query(om, params.astype(np.float16).astype(np.float64), pos, nrm)
    got = E[:, :3].double().cpu().numpy()
    err = np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max()))
    assert err <= 2e-3
    m.close()


def test_wait_expiry_limit_is_checked_on_the_host(niv):
    L = niv.lib()
    assert L.niv_selftest_wait_expiry(0, _stream()) == niv._lib.NIV_ERR_ARG
    assert L.niv_selftest_wait_expiry(1000001, _stream()) == niv._lib.NIV_ERR_ARG
    assert L.niv_sync_status(_stream()) == 0
