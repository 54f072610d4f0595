"""GPU parity of the E4M3 tensor-core query.

The FP8 path carries every weight and every layer input, divided by its per-layer
power-of-two scale, as two E4M3 codes (h = e4m3(v), l = e4m3(v - h)) and accumulates
the products hW ha + hW la + lW ha in FP32.  The bar is the FP8 tolerance against the
unquantised FP64 oracle: max |E - E_fp64| / max E_fp64 <= FP8_BOUND = 2e-2, per result.

Secondary check of the kernel: the oracle's own two-code E4M3 forward (grid values
rounded to FP16 as the kernel stores them).  Each code is an integer decided by
floating point (FP16 residuals on the GPU, FP64 in the oracle), so the two sides may
pick neighbouring codes; either pair lies within 2^-8 |v| of v, so the two forwards
differ by at most about twice the two-code form's own departure from the FP64 network
(<= 1.7e-3 on these networks): FP8_ORACLE_BOUND = 5e-3.
"""
import ctypes

import numpy as np
import pytest

import oracle
from niv_inputs import init_params, uniform_queries
from niv_inputs.configs import MODEL_C0, MODEL_C3, ROOM_MIN, ROOM_MAX, room_gbuffer

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FP8_BOUND = 2e-2         # against the FP64 network, normalised by the frame's max E
FP8_ORACLE_BOUND = 5e-3  # against the oracle's two-code E4M3 forward


def norm_err(E, ref):
    """max |E - ref| / max |ref| (abs error on irradiance normalised to [0, 1])."""
    return float(np.max(np.abs(E - ref)) / np.abs(ref).max())


def grid16(model, params):
    """params with the grid values rounded to FP16, as the kernels store them."""
    g = oracle.grid_value_count(model)
    p = np.asarray(params, np.float64).copy()
    p[:g] = p[:g].astype(np.float16).astype(np.float64)
    return p


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


def _run(niv, spec, pos, nrm, kw, seed=0, bias_std=0.0, cal=None, image_width=0):
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
                out_dtype=torch.float32, image_width=image_width, **kw)[:, :3].cpu().numpy()
    m.close()
    return E, params, om, o_sact


def _check(E, params, om, o_sact, pos, nrm, kw, label):
    p32, n32 = pos.astype(np.float32), nrm.astype(np.float32)
    ref = oracle.query(om, params, p32, n32, **kw)
    ref8 = oracle.query_fp8(om, grid16(om, params), o_sact, p32, n32, **kw)
    e, e8 = norm_err(E, ref), norm_err(E, ref8)
    print("fp8 %s: max abs err (normalised) %.3g vs the FP64 network (bar %g), %.3g vs the oracle's E4M3 "
          "forward (bound %g)" % (label, e, FP8_BOUND, e8, FP8_ORACLE_BOUND))
    assert e <= FP8_BOUND
    assert e8 <= FP8_ORACLE_BOUND


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
def test_fp8_within_bar_of_fp64_oracle(niv, spec, kw):
    lo, hi = kw.get("aabb_min", (0, 0, 0)), kw.get("aabb_max", (1, 1, 1))
    pos, nrm = uniform_queries(8192 + 3, seed=21, lo=lo, hi=hi)
    E, params, om, o_sact = _run(niv, spec, pos, nrm, kw, seed=2, bias_std=0.1)
    _check(E, params, om, o_sact, pos, nrm, kw, "random queries")


@pytest.mark.parametrize("t,W,H", [(0.0, 1920, 1080), (0.25, 1920, 1080), (0.6369616873214543, 1920, 1080),
                                   (1.0, 1920, 1080), (0.6369616873214543, 3840, 2160)])
def test_fp8_config3_model_on_room_frame(niv, t, W, H):
    """The 4-D config-3 model on the full room G-buffer (1080p, and 4K as in the benchmark; image
    traversal) at several values of the scene parameter; sampled pixels checked against both
    oracles."""
    pos, nrm, _ = room_gbuffer(W, H)
    kw = dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, t=t)
    cal = (pos[:: 31].copy(), nrm[:: 31].copy())  # calibration batch: every 31st pixel
    E, params, om, o_sact = _run(niv, MODEL_C3, pos, nrm, kw, seed=0, cal=cal, image_width=W)
    pick = np.random.default_rng(3).choice(len(pos), 8192, replace=False)
    _check(E[pick], params, om, o_sact, pos[pick], nrm[pick], kw, "config-3 %dx%d frame, t=%g" % (W, H, t))


def test_fp8_requires_calibration(niv):
    m = niv.NIVModel(**MODEL_C0)
    pos, nrm = uniform_queries(100, seed=1)
    with pytest.raises(niv.NivError):
        m.query(torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda(), precision="fp8")
    m.close()
