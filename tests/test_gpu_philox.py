"""The device Philox4x32-10 (the Monte Carlo, probe-bake and AO streams) against the published
known-answer vectors and against the oracle's generator on random counters and keys."""
import ctypes

import numpy as np
import pytest

import oracle
from test_oracle_philox import kat_vectors

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_device_philox_matches_known_answers_and_oracle():
    from paper_2602_12949_gb300.build import build
    build()
    import paper_2602_12949_gb300 as P
    kat = kat_vectors()
    rnd = np.random.default_rng(5).integers(0, 2 ** 32, (1000, 6), dtype=np.uint64).astype(np.uint32)
    inp = np.concatenate([kat[:, :6], rnd])
    d_in = torch.from_numpy(inp.view(np.int32).copy()).cuda()
    d_out = torch.zeros((len(inp), 4), dtype=torch.int32, device="cuda")
    assert P.lib().niv_selftest_philox(ctypes.c_void_p(d_in.data_ptr()), len(inp), ctypes.c_void_p(d_out.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    P.sync_status()
    out = d_out.cpu().numpy().view(np.uint32)
    np.testing.assert_array_equal(out[:len(kat)], kat[:, 6:10])
    ref = np.stack([oracle.philox(r[:4], r[4:6]) for r in rnd])
    np.testing.assert_array_equal(out[len(kat):], ref)
