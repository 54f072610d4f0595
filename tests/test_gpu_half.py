"""GPU parity of half-resolution rendering (Sec. 4.4, Table 1 "half") through the C ABI.

niv_query_sub queries every sub-th pixel of every sub-th row of a full-resolution
G-buffer in place; it must equal niv_query on an explicitly strided copy bit for bit
(same kernels, same arithmetic).  niv_upsample_shade (joint bilateral upsampling and
shading, FP32 arithmetic, FP16 output) must match the FP64 oracle of the same
definition (pinned in tests/test_oracle_upsample.py) within the FP16 output rounding
(2^-11 relative) plus 1e-5.
"""
import math

import numpy as np
import pytest

import oracle
from niv_inputs import init_params
from niv_inputs.configs import MODEL_C1, MODEL_PE64, ROOM_MIN, ROOM_MAX, room_gbuffer
from niv_inputs.meshes import shading_frame

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

UP_BOUND = 2.0 ** -11 + 1e-5
KW = dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)


@pytest.fixture(scope="module")
def niv():
    from paper_2602_12949_gb300.build import build
    build()
    import paper_2602_12949_gb300 as P
    return P


def make(P, spec):
    m = P.NIVModel(**spec)
    g, _ = m.param_count()
    m.set_params(init_params(g, m.layer_shapes(), seed=1, bias_std=0.05))
    return m


def strided(a, W, H, s):
    return np.ascontiguousarray(a.reshape(H, W, 4)[::s, ::s].reshape(-1, 4))


def rel_err(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    return float(np.max(np.abs(got - ref) / den))


@pytest.mark.parametrize("W,H,s", [(1920, 1080, 2), (161, 91, 2), (100, 37, 3), (33, 17, 1)])
@pytest.mark.parametrize("precision", ["fp16", "fp32"])
def test_query_sub_equals_query_on_strided_copy(niv, W, H, s, precision):
    pos, nrm, _ = room_gbuffer(W, H)
    m = make(niv, MODEL_C1)
    dp, dn = torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda()
    low = m.query_sub(dp, dn, W, H, sub=s, precision=precision, out_dtype=torch.float32, **KW)
    w = (W + s - 1) // s
    sp, sn = torch.from_numpy(strided(pos, W, H, s)).cuda(), torch.from_numpy(strided(nrm, W, H, s)).cuda()
    ref = m.query(sp, sn, precision=precision, image_width=w, out_dtype=torch.float32, **KW)
    assert low.shape == ref.shape
    assert torch.equal(low, ref)
    m.close()


def test_query_sub_frequency_model_and_fp8(niv):
    W, H, s = 160, 90, 2
    pos, nrm, _ = room_gbuffer(W, H)
    dp, dn = torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda()
    sp, sn = torch.from_numpy(strided(pos, W, H, s)).cuda(), torch.from_numpy(strided(nrm, W, H, s)).cuda()
    m = make(niv, MODEL_PE64)
    assert torch.equal(m.query_sub(dp, dn, W, H, sub=s, **KW), m.query(sp, sn, image_width=W // s, **KW))
    m.close()
    m = make(niv, MODEL_C1)
    m.fp8_calibrate(dp, dn, **KW)
    assert torch.equal(m.query_sub(dp, dn, W, H, sub=s, precision="fp8", **KW),
                       m.query(sp, sn, precision="fp8", image_width=W // s, **KW))
    m.close()


@pytest.mark.parametrize("W,H,s,in_f16", [(1920, 1080, 2, True), (161, 91, 2, True), (100, 37, 3, False),
                                          (64, 48, 1, True)])
def test_upsample_shade_matches_oracle(niv, W, H, s, in_f16):
    pos, nrm, alb, direct, _ = shading_frame(W, H, seed=0)
    m = make(niv, MODEL_C1)
    cast = (lambda a: a) if in_f16 else (lambda a: a.astype(np.float32))
    dp, dn = torch.from_numpy(cast(pos)).cuda(), torch.from_numpy(cast(nrm)).cuda()
    low = m.query_sub(dp, dn, W, H, sub=s, out_dtype=torch.float32, **KW)
    da, dd = torch.from_numpy(alb).cuda(), torch.from_numpy(direct).cuda()
    out = niv.upsample_shade(dp, dn, da, dd, W, H, low, sub=s, power=8.0, sigma=0.05, eps=1e-4)
    ref = oracle.upsample_shade(pos.astype(np.float32), nrm.astype(np.float32), alb.astype(np.float32),
                                direct.astype(np.float32), W, H, low[:, :3].cpu().numpy(), sub=s, power=8.0,
                                sigma=0.05, eps=1e-4)
    got = out.float().cpu().numpy()
    assert np.all(got[:, 3] == 1.0)
    err = rel_err(got[:, :3], ref)
    print("upsample %dx%d sub %d: max rel err %.2e" % (W, H, s, err))
    assert err <= UP_BOUND
    m.close()


def test_upsample_with_sub_one_is_shading(niv):
    W, H = 96, 40
    pos, nrm, alb, direct, _ = shading_frame(W, H, seed=0)
    E = np.zeros((W * H, 4), np.float16)
    E[:, :3] = np.random.default_rng(2).uniform(0.0, 4.0, (W * H, 3))
    t = lambda a: torch.from_numpy(a).cuda()
    up = niv.upsample_shade(t(pos), t(nrm), t(alb), t(direct), W, H, t(E), sub=1)
    sh = niv.shade(t(alb), t(direct), t(E))
    diff = (up.float() - sh.float()).abs() / sh.float().abs().clamp_min(1e-3)
    assert float(diff.max()) <= 2.0 ** -10  # one FP16 step: E * w / w may differ from E by an FP32 ulp


def test_upsample_rejects_bad_parameters(niv):
    W, H = 8, 8
    z = torch.zeros((W * H, 4), dtype=torch.float16, device="cuda")
    low = torch.zeros((16, 4), dtype=torch.float16, device="cuda")
    for kw in (dict(sigma=0.0), dict(eps=0.0), dict(power=-1.0), dict(sub=0)):
        with pytest.raises(niv.NivError):
            niv.upsample_shade(z, z, z, z, W, H, low, **{**dict(sub=2), **kw})
