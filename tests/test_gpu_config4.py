"""Config 4: the full shading frame with dynamic objects; the fused query + shading epilogue
against the oracle's E followed by the oracle's shading (Eq. 2 plus direct light)."""
import numpy as np
import pytest

import oracle
from niv_inputs import init_params
from niv_inputs.configs import MODEL_C4, ROOM_MIN, ROOM_MAX
from niv_inputs.meshes import shading_frame

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def niv():
    from paper_2602_12949_gb300.build import build
    build()
    import paper_2602_12949_gb300 as P
    return P


def _rel(got, ref):
    return float(np.max(np.abs(got - ref) / np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())))


@pytest.mark.parametrize("w,h", [(960, 540), (3840, 2160)])
def test_fused_shade_matches_oracle(niv, w, h):
    pos, nrm, alb, direct, cov = shading_frame(w, h)
    m = niv.NIVModel(**MODEL_C4)
    g, _ = m.param_count()
    params = init_params(g, m.layer_shapes(), seed=4)
    m.set_params(params)
    om = oracle.Model(**MODEL_C4)
    d = lambda a: torch.from_numpy(a).cuda()
    dp, dn, da, dd = d(pos), d(nrm), d(alb), d(direct)
    kw = dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)
    pick = np.random.default_rng(0).choice(len(pos), 6000, replace=False)
    E_ref = oracle.query(om, params, pos[pick].astype(np.float32), nrm[pick].astype(np.float32), **kw)
    E_ref16 = oracle.query(om, params.astype(np.float16).astype(np.float64), pos[pick].astype(np.float32),
                           nrm[pick].astype(np.float32), **kw)
    a64, d64 = alb[pick, :3].astype(np.float64), direct[pick, :3].astype(np.float64)
    for prec, ref_E, bound in (("fp32", E_ref, 1e-5), ("fp16", E_ref16, 2e-3)):
        rgba = m.query_shade(dp, dn, da, dd, precision=prec, image_width=w, **kw).float().cpu().numpy()
        ref = oracle.shade(a64, ref_E, d64)
        err = _rel(rgba[pick, :3], ref)
        print("%dx%d %s fused shade: max rel %.3g (coverage %.3f)" % (w, h, prec, err, cov))
        assert err <= bound + 2.0 ** -11  # plus the final FP16 rounding of rgba
        assert np.all(rgba[:, 3] == 1.0)
    m.close()


def test_fused_equals_query_then_shade(niv):
    pos, nrm, alb, direct, _ = shading_frame(960, 540)
    m = niv.NIVModel(**MODEL_C4)
    g, _ = m.param_count()
    m.set_params(init_params(g, m.layer_shapes(), seed=5))
    d = lambda a: torch.from_numpy(a).cuda()
    dp, dn, da, dd = d(pos), d(nrm), d(alb), d(direct)
    kw = dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, image_width=960)
    fused = m.query_shade(dp, dn, da, dd, precision="fp16", **kw).float()
    E32 = m.query(dp, dn, precision="fp16", out_dtype=torch.float32, **kw)
    two = (da.float()[:, :3] * E32[:, :3] / np.pi + dd.float()[:, :3])
    # same E in FP32; only the final FP16 rounding of rgba remains
    assert torch.max(torch.abs(fused[:, :3] - two) / torch.clamp(two.abs(), min=1e-3)).item() <= 2.0 ** -10
    m.close()
