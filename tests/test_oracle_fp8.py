"""Pins of the oracle's E4M3 network path against numpy + torch's float8_e4m3fn rounding.

The path carries every scaled weight and input v as two E4M3 codes h = e4m3(v),
l = e4m3(v - h) and forms each product as hW*ha + hW*la + lW*ha.
"""
import numpy as np
import pytest

import oracle
from niv_inputs import init_params, uniform_queries

torch = pytest.importorskip("torch")


def _e4m3(x):
    return torch.from_numpy(np.asarray(x, np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()


def _layers(model, mlp):
    out, off = [], 0
    for (o, i) in oracle.layer_shapes(model):
        W = mlp[off:off + o * i].reshape(o, i)
        b = mlp[off + o * i:off + o * i + o]
        out.append((W, b))
        off += o * i + o
    return out


def test_fp8_scale_is_power_of_two_covering_the_range():
    for amax in [1e-6, 0.3, 1.0, 447.9, 448.0, 448.1, 3e4]:
        s = oracle.fp8_scale(amax)
        assert np.log2(s) == np.round(np.log2(s))
        assert 224.0 < amax / s <= 448.0


def test_calibration_amax_matches_numpy_forward():
    m = oracle.Model()
    L = oracle.layout(m)
    params = init_params(L["total"] * m.feat, oracle.layer_shapes(m), seed=3, bias_std=0.1).astype(np.float64)
    pos, nrm = uniform_queries(2000, seed=4)
    amax = oracle.fp8_act_amax(m, params, pos, nrm)
    x = np.concatenate([oracle.encode(m, params, pos), nrm[:, :3].astype(np.float64)], axis=1)
    ref = [np.abs(x).max()]
    h = x
    for (W, b) in _layers(m, params[L["total"] * m.feat:])[:-1]:
        h = np.maximum(h @ W.T + b, 0.0)
        ref.append(h.max())
    np.testing.assert_allclose(amax, ref, rtol=1e-12)


def _pair(v):
    h = _e4m3(v)
    return h, _e4m3(v - h)


def test_two_code_pair_keeps_eight_bits():
    """|h + l - v| <= 2^-4 |v - h| <= 2^-8 |v| for v in E4M3's normal range (each code rounds
    to 3 mantissa bits); below it the subnormal step 2^-9 bounds l's rounding."""
    v = np.random.default_rng(0).uniform(-448.0, 448.0, 200000)
    v = np.concatenate([v, v * 2.0 ** -8, [0.0, 2.0 ** -6, 448.0, -448.0]])
    h = oracle.e4m3(v)
    l = oracle.e4m3(v - h)
    err = np.abs(h + l - v)
    assert np.all(err <= np.maximum(2.0 ** -8 * np.abs(v), 2.0 ** -10) * (1 + 1e-12))
    assert np.all(np.abs(h - v) <= np.maximum(2.0 ** -4 * np.abs(v), 2.0 ** -10) * (1 + 1e-12))
    # and the single code alone does not (the second code matters)
    assert np.max(np.abs(h - v) / np.maximum(np.abs(v), 1.0)) > 2.0 ** -6


@pytest.mark.parametrize("n_hidden", [2, 3])
def test_fp8_forward_matches_numpy_with_torch_quantiser(n_hidden):
    """Split W/s_w and a/s_a into two codes with torch's E4M3 cast, form hW ha + hW la + lW ha in
    FP64, rescale: same E as the oracle."""
    m = oracle.Model(n_hidden=n_hidden)
    L = oracle.layout(m)
    params = init_params(L["total"] * m.feat, oracle.layer_shapes(m), seed=5, bias_std=0.1).astype(np.float64)
    pos, nrm = uniform_queries(1500, seed=6)
    amax = oracle.fp8_act_amax(m, params, pos, nrm)
    s_act = np.array([oracle.fp8_scale(a) for a in amax])
    got = oracle.query_fp8(m, params, s_act, pos, nrm)
    x = np.concatenate([oracle.encode(m, params, pos), nrm[:, :3].astype(np.float64)], axis=1)
    a = x
    layers = _layers(m, params[L["total"] * m.feat:])
    for li, (W, b) in enumerate(layers):
        s_w = 2.0 ** np.ceil(np.log2(np.abs(W).max() / 448.0))
        ah, al = _pair(a / s_act[li])
        wh, wl = _pair(W / s_w)
        z = (ah @ wh.T + al @ wh.T + ah @ wl.T) * (s_w * s_act[li]) + b
        a = np.maximum(z, 0.0) if li < len(layers) - 1 else np.logaddexp(0.0, z)
    np.testing.assert_allclose(got, a, rtol=1e-12, atol=1e-14)


def test_fp8_is_close_to_full_precision():
    """Two E4M3 codes keep about 8 bits: outputs stay within the FP8 bar (2e-2 of the range) of
    the FP64 network, yet are visibly quantised."""
    m = oracle.Model()
    L = oracle.layout(m)
    params = init_params(L["total"] * m.feat, oracle.layer_shapes(m), seed=7).astype(np.float64)
    pos, nrm = uniform_queries(3000, seed=8)
    s_act = [oracle.fp8_scale(a) for a in oracle.fp8_act_amax(m, params, pos, nrm)]
    E8 = oracle.query_fp8(m, params, s_act, pos, nrm)
    E = oracle.query(m, params, pos, nrm)
    err = np.abs(E8 - E).max() / np.abs(E).max()
    assert 1e-5 < err < 2e-2
