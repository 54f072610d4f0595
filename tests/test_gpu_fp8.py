"""GPU parity of the E4M3 tensor-core query against the oracle's E4M3 network path.

The FP8 path quantises weights and every layer input to E4M3 with per-layer
power-of-two scales and accumulates in FP32.  Parity is taken against the oracle's
FP8 forward with the oracle's own calibration, so it measures the kernel; the
departure of the FP8 format from the FP64 network is reported beside it.

Each E4M3 code is an integer decided by floating point: the kernel decides it from
FP32 pre-activations, the oracle from FP64 ones, and where the two straddle a
rounding point they pick neighbouring codes (one E4M3 step, 2^-3 relative, of one
activation).  So the bar is: at least 98% of samples agree to 1e-5 of the frame's
max irradiance (every decision identical), and every sample stays within
FP8_FLIP_BOUND = 2e-2 + one flip's worth (4e-2 in all).
"""
import ctypes

import numpy as np
import pytest

import oracle
from niv_inputs import init_params, uniform_queries
from niv_inputs.configs import MODEL_C0, MODEL_C3, ROOM_MIN, ROOM_MAX, room_gbuffer

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FP8_AGREE = 1e-5        # normalised error of samples whose quantisation decisions all agree
FP8_AGREE_FRAC = 0.98    # fraction of samples that must agree
FP8_FLIP_BOUND = 4e-2    # any sample, isolated rounding-point flips included


def fp8_parity(E, ref8):
    """(max normalised error, fraction of samples within FP8_AGREE)."""
    e = np.abs(E - ref8).max(axis=1) / np.abs(ref8).max()
    return float(e.max()), float((e <= FP8_AGREE).mean())


@pytest.fixture(scope="module")
def niv():
    from paper_2602_12949_gb300.build import build
    build()
    import paper_2602_12949_gb300 as P
    return P


def test_fp8_tensor_core_layout_selftest(niv):
    m_ = np.arange(128)[:, None]
    n_ = np.arange(64)[:, None]
    k_ = np.arange(64)[None, :]
    ref = (((m_ * 3 + k_ * 5) % 7 - 3) @ ((n_ * 5 + k_ * 3) % 5 - 2).T).astype(np.float32)
    out = torch.zeros((128, 64), dtype=torch.float32, device="cuda")
    assert niv.lib().niv_selftest_mma(2, ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
    niv.sync_status()
    np.testing.assert_array_equal(out.cpu().numpy(), ref)


def _run(niv, spec, pos, nrm, kw, seed=0, bias_std=0.0, cal=None):
    m = niv.NIVModel(**spec)
    g, _ = m.param_count()
    params = init_params(g, m.layer_shapes(), seed=seed, bias_std=bias_std)
    m.set_params(params)
    om = oracle.Model(**spec)
    cpos, cnrm = cal if cal is not None else (pos, nrm)
    m.fp8_calibrate(torch.from_numpy(cpos).cuda(), torch.from_numpy(cnrm).cuda(), **kw)
    sa, sw, am = m.fp8_scales()
    o_amax = oracle.fp8_act_amax(om, params, cpos.astype(np.float32), cnrm.astype(np.float32), **kw)
    o_sact = np.array([oracle.fp8_scale(a) for a in o_amax])
    np.testing.assert_allclose(am, o_amax, rtol=1e-5)
    np.testing.assert_array_equal(sa, o_sact)  # power-of-two scales: the same decision on both sides
    E = m.query(torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda(), precision="fp8",
                out_dtype=torch.float32, **kw)[:, :3].cpu().numpy()
    ref8 = oracle.query_fp8(om, params, o_sact, pos.astype(np.float32), nrm.astype(np.float32), **kw)
    ref = oracle.query(om, params, pos.astype(np.float32), nrm.astype(np.float32), **kw)
    e8, agree = fp8_parity(E, ref8)
    e = np.max(np.abs(E - ref)) / np.abs(ref).max()
    print("fp8: max abs err (normalised) %.3g vs FP8 oracle (%.4f of samples within %g), %.3g vs FP64 network"
          % (e8, agree, FP8_AGREE, e))
    m.close()
    return e8, agree, e


@pytest.mark.parametrize("spec,kw", [
    (MODEL_C0, {}),
    (dict(MODEL_C0, width=32, n_hidden=1), {}),
    (MODEL_C3, dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, t=0.4)),
    # 16-level models: the config-1 grid (4 dense levels, a compiled shape), 5 and 3 dense
    # levels, and a 4-D grid without dense levels (the shape-only kernels)
    (dict(MODEL_C3, dims=3, in_extra=3, n_hidden=2, log2_T=17), dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)),
    (dict(MODEL_C3, dims=3, in_extra=3, n_hidden=2), dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)),
    (dict(MODEL_C3, dims=3, in_extra=3, n_hidden=2, log2_T=15), dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)),
    (dict(MODEL_C3, log2_T=15), dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, t=0.6)),
])
def test_fp8_matches_fp8_oracle(niv, spec, kw):
    lo, hi = kw.get("aabb_min", (0, 0, 0)), kw.get("aabb_max", (1, 1, 1))
    pos, nrm = uniform_queries(8192 + 3, seed=21, lo=lo, hi=hi)
    e8, agree, e = _run(niv, spec, pos, nrm, kw, seed=2, bias_std=0.1)
    assert agree >= FP8_AGREE_FRAC
    assert e8 <= FP8_FLIP_BOUND
    assert e <= 0.1


def test_fp8_config3_model_on_room_frame(niv):
    """The 4-D config-3 model on the full 1080p room G-buffer (image traversal), sampled pixels checked."""
    pos, nrm, _ = room_gbuffer(1920, 1080)
    kw = dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, t=0.25)
    pick = np.random.default_rng(3).choice(len(pos), 8192, replace=False)
    cal = (pos[:: 31].copy(), nrm[:: 31].copy())  # calibration batch: every 31st pixel
    m = niv.NIVModel(**MODEL_C3)
    g, _ = m.param_count()
    params = init_params(g, m.layer_shapes(), seed=0)
    m.set_params(params)
    m.fp8_calibrate(torch.from_numpy(cal[0]).cuda(), torch.from_numpy(cal[1]).cuda(), **kw)
    E = m.query(torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda(), precision="fp8", image_width=1920,
                out_dtype=torch.float32, **kw)[:, :3].cpu().numpy()
    om = oracle.Model(**MODEL_C3)
    o_sact = [oracle.fp8_scale(a) for a in oracle.fp8_act_amax(om, params, cal[0].astype(np.float32),
                                                                cal[1].astype(np.float32), **kw)]
    ref8 = oracle.query_fp8(om, params, o_sact, pos[pick].astype(np.float32), nrm[pick].astype(np.float32), **kw)
    e8, agree = fp8_parity(E[pick], ref8)
    print("fp8 config-3 frame: max %.3g, %.4f of samples within %g" % (e8, agree, FP8_AGREE))
    assert agree >= FP8_AGREE_FRAC
    assert e8 <= FP8_FLIP_BOUND
    m.close()


def test_fp8_requires_calibration(niv):
    m = niv.NIVModel(**MODEL_C0)
    pos, nrm = uniform_queries(100, seed=1)
    with pytest.raises(niv.NivError):
        m.query(torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda(), precision="fp8")
    m.close()
