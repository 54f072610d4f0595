"""Pins of the oracle's network, full query, loss gradient and Adam (Sec. 4.1, Eq. 3, Sec. 4.5)."""
import numpy as np
import pytest

import oracle
from niv_inputs import init_params, uniform_queries
from conftest import read_golden


def _numpy_forward(model, mlp_params, x):
    """Textbook forward with numpy.matmul: ReLU hidden layers, softplus output."""
    p = np.asarray(mlp_params, np.float64)
    h = np.asarray(x, np.float64)
    off = 0
    for (o, i) in oracle.layer_shapes(model):
        W = p[off:off + o * i].reshape(o, i)
        b = p[off + o * i:off + o * i + o]
        off += o * i + o
        z = h @ W.T + b
        h = np.maximum(z, 0.0) if o != model.out_dim or off != len(p) else z
    return np.logaddexp(0.0, h) if model.out_act == 1 else h


def test_worked_example_by_hand():
    m = oracle.Model(levels=1, feat=1, base=1.0, growth=1.0, log2_T=10, n_hidden=1, width=2, out_dim=1)
    grid = np.arange(8, dtype=np.float64)
    mlp = np.array([1, 0, 0, 0, -1, 0, 0, 1, 0, 0.5, 0.5, 1, -2], np.float64)
    params = np.concatenate([grid, mlp])
    assert len(mlp) == oracle.mlp_param_count(m)
    rows = np.array(read_golden("tiny_network.txt"))
    pos = np.zeros((len(rows), 4), np.float32)
    pos[:, :3] = rows[:, :3]
    nrm = np.zeros_like(pos)
    nrm[:, 2] = 1.0
    enc = oracle.encode(m, params, pos)
    np.testing.assert_allclose(enc[:, 0], rows[:, 3], rtol=0, atol=1e-15)
    E = oracle.query(m, params, pos, nrm)
    np.testing.assert_allclose(E[:, 0], rows[:, 4], rtol=1e-15)


@pytest.mark.parametrize("n_hidden", [2, 3])
def test_network_matches_numpy_matmul(n_hidden):
    m = oracle.Model(n_hidden=n_hidden)
    x = np.random.default_rng(0).standard_normal((512, m.n_in))
    params = init_params(0, oracle.layer_shapes(m), seed=2, bias_std=0.3)
    np.testing.assert_allclose(oracle.mlp(m, params, x), _numpy_forward(m, params, x), rtol=1e-13, atol=1e-14)


def test_zero_weights_reduce_to_softplus_of_bias():
    m = oracle.Model()
    params = np.zeros(oracle.mlp_param_count(m))
    params[-3:] = [-30.0, 0.0, 30.0]
    E = oracle.mlp(m, params, np.random.default_rng(1).standard_normal((4, m.n_in)))
    np.testing.assert_allclose(E, np.tile(np.logaddexp(0, [-30.0, 0.0, 30.0]), (4, 1)), rtol=1e-15)


def test_query_is_encoding_then_network():
    m = oracle.Model()
    L = oracle.layout(m)
    shapes = oracle.layer_shapes(m)
    params = init_params(L["total"] * m.feat, shapes, seed=4, bias_std=0.1)
    pos, nrm = uniform_queries(1024, seed=3)
    enc = oracle.encode(m, params, pos)
    x = np.concatenate([enc, nrm[:, :3].astype(np.float64)], axis=1)
    ref = _numpy_forward(m, params[L["total"] * m.feat:], x)
    np.testing.assert_allclose(oracle.query(m, params, pos, nrm), ref, rtol=1e-12)


def _loss_frozen_denominator(m, params, pos, nrm, target, den, t=None):
    if t is None:
        E = oracle.query(m, params, pos, nrm)
    else:
        E = np.concatenate([oracle.query(m, params, pos[i:i + 1], nrm[i:i + 1], t=float(t[i]))
                            for i in range(len(pos))])
    return np.mean((E - target) ** 2 / den)


@pytest.mark.parametrize("dims", [3, 4])
def test_gradient_matches_central_differences(dims):
    """Eq. 3 with sg() on the denominator: the gradient equals FD of the loss with the denominator frozen."""
    if dims == 3:
        m = oracle.Model(levels=4, log2_T=8, base=4, growth=1.5, width=16)  # collisions at hashed levels
    else:
        m = oracle.Model(dims=4, levels=3, log2_T=8, base=3, growth=1.5, width=16, in_extra=4, n_hidden=3)
    L = oracle.layout(m)
    assert not all(L["dense"])
    shapes = oracle.layer_shapes(m)
    params = init_params(L["total"] * m.feat, shapes, seed=5, feat_range=0.5, bias_std=0.2).astype(np.float64)
    pos, nrm = uniform_queries(24, seed=6)
    t = np.random.default_rng(2).random(24).astype(np.float32) if dims == 4 else None
    target = np.random.default_rng(3).uniform(0.1, 2.0, (24, 3))
    loss, g = oracle.loss_grad(m, params, pos, nrm, target, t=t)
    if t is None:
        E0 = oracle.query(m, params, pos, nrm)
    else:
        E0 = np.concatenate([oracle.query(m, params, pos[i:i + 1], nrm[i:i + 1], t=float(t[i])) for i in range(24)])
    den = E0 ** 2 + 0.01
    assert loss == pytest.approx(np.mean((E0 - target) ** 2 / den), rel=1e-12)
    rng = np.random.default_rng(7)
    n_grid = L["total"] * m.feat
    touched = np.nonzero(g[:n_grid])[0]
    picks = np.concatenate([rng.choice(touched, 12, replace=False), n_grid + rng.choice(len(params) - n_grid, 24, replace=False)])
    h = 1e-5  # truncation O(h^2) and rounding O(1e-16/h) both stay below 1e-10
    for i in picks:
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        fd = (_loss_frozen_denominator(m, pp, pos, nrm, target, den, t)
              - _loss_frozen_denominator(m, pm, pos, nrm, target, den, t)) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-6, abs=1e-10), i


def test_adam_matches_textbook_update():
    """Kingma & Ba Algorithm 1 written out with numpy for a few steps."""
    rng = np.random.default_rng(0)
    theta = rng.standard_normal(100)
    m = np.zeros(100)
    v = np.zeros(100)
    t_ref, m_ref, v_ref = theta.copy(), m.copy(), v.copy()
    for step in range(1, 6):
        g = rng.standard_normal(100)
        oracle.adam(theta, m, v, g, 1e-2, 0.9, 0.99, 1e-15, step)
        m_ref = 0.9 * m_ref + 0.1 * g
        v_ref = 0.99 * v_ref + 0.01 * g * g
        mh = m_ref / (1 - 0.9 ** step)
        vh = v_ref / (1 - 0.99 ** step)
        t_ref = t_ref - 1e-2 * mh / (np.sqrt(vh) + 1e-15)
    np.testing.assert_allclose(theta, t_ref, rtol=1e-14)
    # first step of Adam moves every coordinate by lr * sign(g)
    th = np.zeros(5); mm = np.zeros(5); vv = np.zeros(5)
    g = np.array([3.0, -2.0, 0.5, -1e-3, 7.0])
    oracle.adam(th, mm, vv, g, 0.01, 0.9, 0.99, 1e-15, 1)
    np.testing.assert_allclose(th, -0.01 * np.sign(g), rtol=1e-9)


def test_shade_is_albedo_times_irradiance_over_pi_plus_direct():
    """Eq. 2: L_r = rho / pi * E; a white surface under E = pi reflects radiance 1."""
    E = np.full((4, 3), np.pi)
    out = oracle.shade(np.ones((4, 3)), E, np.zeros((4, 3)))
    np.testing.assert_allclose(out, 1.0, rtol=1e-15)
    out = oracle.shade(np.full((4, 3), 0.5), E, np.full((4, 3), 0.25))
    np.testing.assert_allclose(out, 0.75, rtol=1e-15)


def test_e4m3_matches_torch_float8():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 50, rng.standard_normal(20000) * 1e-2,
                        rng.uniform(-448, 448, 20000), [0.0, 2.0 ** -9, 3 * 2.0 ** -10, 448.0, -448.0, 1.0625,
                                                        1.1875, 2.0 ** -7 * 1.0625]])
    x = x[np.abs(x) <= 448]
    ref = torch.from_numpy(x.astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    np.testing.assert_array_equal(oracle.e4m3(x.astype(np.float32).astype(np.float64)), ref)
    assert oracle.e4m3(np.array([1000.0, -500.0])).tolist() == [448.0, -448.0]


# ---- the FP16 forward of training (config 2: FP16 forward, FP32 master weights) ----

def _batch(n, seed):
    from niv_inputs import uniform_queries
    pos, nrm = uniform_queries(n, seed=seed)
    y = np.random.default_rng(seed + 1).uniform(0.1, 2.0, (n, 3))
    return pos, nrm, y


def test_f16_loss_is_eq3_of_the_f16_path_forward():
    """The loss of the FP16 mode is Eq. 3 evaluated on the FP16 path's forward (query_f16,
    itself pinned to numpy's binary16 conversion)."""
    from niv_inputs import init_params
    m = oracle.Model(levels=4, log2_T=10, base=3.0, growth=1.6, width=16)
    params = init_params(oracle.grid_value_count(m), oracle.layer_shapes(m), seed=1, feat_range=0.3, bias_std=0.2)
    p16 = oracle.f16(params)
    pos, nrm, y = _batch(300, 2)
    loss, _ = oracle.loss_grad(m, p16, pos, nrm, y, f16=True)
    E = oracle.query_f16(m, p16, pos, nrm)
    assert loss == pytest.approx(np.mean((E - y) ** 2 / (E * E + 0.01)), rel=1e-13)


def test_f16_gradient_equals_fp32_gradient_when_nothing_rounds():
    """With grid values, inputs and weights that are dyadic (exact in binary16) and queries on
    lattice vertices, every activation is exact in binary16, so the FP16 mode's gradient is
    the FP32 gradient exactly."""
    m = oracle.Model(levels=1, feat=2, log2_T=10, base=4.0, growth=1.0, n_hidden=2, width=16)
    rng = np.random.default_rng(3)
    g = oracle.grid_value_count(m)
    grid = rng.integers(-4, 5, g) / 8.0
    mlp = []
    for (o, i) in oracle.layer_shapes(m):
        mlp += [rng.integers(-2, 3, o * i) / 4.0, rng.integers(-2, 3, o) / 4.0]
    params = np.concatenate([grid] + mlp)
    assert np.array_equal(oracle.f16(params), params)
    n = 64
    pos = np.zeros((n, 4), np.float32)
    pos[:, :3] = rng.integers(0, 5, (n, 3)) / 4.0  # u N is an integer: each query sits on a vertex
    nrm = np.zeros((n, 4), np.float32)
    nrm[:, :3] = rng.integers(-2, 3, (n, 3)) / 2.0
    y = rng.integers(1, 8, (n, 3)) / 4.0
    l16, g16 = oracle.loss_grad(m, params, pos, nrm, y, f16=True)
    l32, g32 = oracle.loss_grad(m, params, pos, nrm, y)
    assert l16 == l32
    assert np.array_equal(g16, g32)


def test_f16_gradient_is_close_to_fp32_gradient():
    from niv_inputs import init_params
    m = oracle.Model(levels=6, log2_T=12, base=3.0, growth=1.6, width=32, n_hidden=2)
    params = init_params(oracle.grid_value_count(m), oracle.layer_shapes(m), seed=4, feat_range=0.3, bias_std=0.2)
    pos, nrm, y = _batch(2000, 5)
    _, g16 = oracle.loss_grad(m, oracle.f16(params), pos, nrm, y, f16=True)
    _, g32 = oracle.loss_grad(m, params, pos, nrm, y)
    rel = np.abs(g16 - g32).max() / np.abs(g32).max()
    assert 0.0 < rel < 2e-2
