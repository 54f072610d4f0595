"""The learned part (Sec. 4.5, Sec. 5.1): NIV trained on the GPU from GPU Monte Carlo targets
beats the SH probe grid of the same memory on held-out samples.

The paper reports at least 10x lower MSE than probes at the same budget on its scenes
(its training runs 10-50k steps on path-traced targets); this test runs a short
schedule on the seeded room and requires NIV to win, printing the ratio.  The
comparison is parity-unpinned: no paper number exists for this synthetic scene.
"""
import numpy as np
import pytest

from niv_inputs import room_scene, init_params
from niv_inputs.configs import MODEL_C1, ROOM_MIN, ROOM_MAX

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def niv():
    from paper_2602_12949_gb300.build import build
    build()
    import paper_2602_12949_gb300 as P
    return P


def test_trained_niv_beats_same_memory_probes(niv):
    from paper_2602_12949_gb300 import fitting
    scene = room_scene(0)
    hx, hn, hE, _ = fitting.held_out(scene, 1 << 14, 4096, seed=99)
    m = niv.NIVModel(**MODEL_C1)
    g, nm = m.param_count()
    niv_bytes = 2 * (g + nm)  # FP16 parameters
    P = int((niv_bytes / 54) ** (1 / 3))
    grid = niv.ProbeGrid((P,) * 3, ROOM_MIN, ROOM_MAX)
    assert grid.nbytes <= niv_bytes
    grid.bake(scene.blob(), rays=1024, seed=3)
    probe_mse, probe_rel = fitting.errors(grid.query(hx, hn, out_dtype=torch.float32), hE)
    m.set_params(init_params(g, m.layer_shapes(), seed=0))
    info = fitting.train(m, scene, steps=2000, batch=1 << 16, pool=1 << 18, spp=128, reuse=2, seed=1, log_every=500)
    niv_mse, niv_rel = fitting.errors(m.query(hx, hn, precision="fp16", out_dtype=torch.float32,
                                              aabb_min=ROOM_MIN, aabb_max=ROOM_MAX), hE)
    print("probes %d^3 (%.2f MB): MSE %.3g rel %.3g | NIV (%.2f MB, FP16 query): MSE %.3g rel %.3g | ratio %.1fx"
          % (P, grid.nbytes / 1e6, probe_mse, probe_rel, niv_bytes / 1e6, niv_mse, niv_rel, probe_mse / niv_mse))
    print("loss", info["loss"])
    assert info["loss"][-1][1] < 0.2 * info["loss"][0][1]
    assert niv_mse < probe_mse
    m.close()
