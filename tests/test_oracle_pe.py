"""Pins of the oracle's frequency encoding (the models of Table 1 without grid levels).

Sec. 4.1: the smaller models replace the hash grid by an eight-band positional
encoding of the position (Mildenhall et al. 2020).  Reading: for the normalised
coordinate u_k (k = 0, 1, 2) and band b the pair (sin(2^b pi u_k), cos(2^b pi u_k)),
coordinate-major, then band, sin before cos; the network input is
[6 B encoding values, n.xyz].  Each pin below fails for a plausible mistake:
a wrong band exponent (double-angle relation), a swapped sin / cos or coordinate
order (closed forms at dyadic points, coordinate separation), or a misplaced
normal (hand-built network).
"""
import math

import numpy as np
import pytest

import oracle

B = 8


def pe_model(width=16, n_hidden=3, bands=B, out_act=1):
    return oracle.Model(dims=3, levels=0, feat=2, log2_T=14, pe_bands=bands, n_hidden=n_hidden, width=width,
                        out_act=out_act)


def enc_of(u3, bands=B):
    m = pe_model(bands=bands)
    pos = np.zeros((len(u3), 4), np.float32)
    pos[:, :3] = u3
    return oracle.encode(m, np.zeros(0), pos).reshape(len(u3), 3, bands, 2)


def test_sizes_match_table1_memory():
    # Table 1: widths 16 / 32 / 64 without grid take 0.003 / 0.01 / 0.03 MB in half precision.
    # 48 encoding values + 3 normal inputs, three hidden layers, 3 outputs, with biases.
    for width, mb in ((16, 0.003), (32, 0.01), (64, 0.03)):
        m = pe_model(width=width)
        assert m.n_in == 51
        assert oracle.grid_value_count(m) == 0
        nbytes = 2 * oracle.mlp_param_count(m)
        assert abs(nbytes / 1e6 - mb) <= 0.0075, (width, nbytes)


def test_closed_forms_at_dyadic_points():
    # u = 0: every band is (0, 1).  u = 2^-m: band m-1 is (1, 0), band m is (0, -1),
    # later bands (0, 1); band m-2 is (sqrt(1/2), sqrt(1/2)).
    u = np.array([[0.0, 0.5, 0.25], [0.125, 1.0, 0.0]], np.float32)
    e = enc_of(u)
    np.testing.assert_allclose(e[0, 0], np.tile([0.0, 1.0], (B, 1)), atol=1e-15)
    # y = 1/2 (m = 1)
    np.testing.assert_allclose(e[0, 1, 0], [1.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(e[0, 1, 1], [0.0, -1.0], atol=1e-15)
    np.testing.assert_allclose(e[0, 1, 2:], np.tile([0.0, 1.0], (B - 2, 1)), atol=1e-13)
    # z = 1/4 (m = 2)
    r = math.sqrt(0.5)
    np.testing.assert_allclose(e[0, 2, 0], [r, r], atol=1e-15)
    np.testing.assert_allclose(e[0, 2, 1], [1.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(e[0, 2, 2], [0.0, -1.0], atol=1e-15)
    # x = 1/8 (m = 3); y = 1: band 0 is (0, -1), later bands (0, 1)
    np.testing.assert_allclose(e[1, 0, 2], [1.0, 0.0], atol=1e-15)
    np.testing.assert_allclose(e[1, 0, 3], [0.0, -1.0], atol=1e-15)
    np.testing.assert_allclose(e[1, 1, 0], [0.0, -1.0], atol=1e-15)
    np.testing.assert_allclose(e[1, 1, 1:], np.tile([0.0, 1.0], (B - 1, 1)), atol=1e-13)


def test_unit_circle_and_double_angle_between_bands():
    rng = np.random.default_rng(3)
    u = rng.random((256, 3)).astype(np.float32)
    e = enc_of(u)
    s, c = e[..., 0], e[..., 1]
    np.testing.assert_allclose(s * s + c * c, 1.0, atol=1e-14)
    # band b+1 is the double angle of band b
    np.testing.assert_allclose(s[..., 1:], 2.0 * s[..., :-1] * c[..., :-1], atol=1e-12)
    np.testing.assert_allclose(c[..., 1:], c[..., :-1] ** 2 - s[..., :-1] ** 2, atol=1e-12)
    # band 0 is sin / cos of pi u (the lowest frequency): u in (0, 1) gives sin > 0
    assert np.all(s[..., 0] > 0.0) and np.all(np.abs(np.arccos(c[..., 0]) / math.pi - u) < 1e-6)


def test_coordinates_are_separate():
    rng = np.random.default_rng(4)
    u = rng.random((16, 3)).astype(np.float32)
    base = enc_of(u)
    for k in range(3):
        v = u.copy()
        v[:, k] = rng.random(16).astype(np.float32)
        e = enc_of(v)
        for j in range(3):
            same = np.array_equal(e[:, j], base[:, j])
            assert same == (j != k), (k, j)


def test_odd_band_count():
    u = np.array([[0.3, 0.6, 0.9]], np.float32)
    e3 = enc_of(u, bands=3)
    e8 = enc_of(u, bands=8)
    np.testing.assert_allclose(e3[0], e8[0, :, :3], atol=0)


def test_hand_built_network_picks_one_value_and_the_normal():
    # One hidden layer of 16: unit 0 = +sin(4 pi u_y), unit 1 = -sin(4 pi u_y), unit 2 = n_x;
    # output 0 = unit0 - unit1 = sin(4 pi u_y); output 1 = unit 2 = relu(n_x); output 2 = 0.
    m = pe_model(width=16, n_hidden=1)
    n_in = m.n_in
    W1 = np.zeros((16, n_in))
    col = (1 * B + 2) * 2 + 0  # coordinate y, band 2, sine
    W1[0, col] = 1.0
    W1[1, col] = -1.0
    W1[2, 6 * B + 0] = 1.0    # n.x follows the 48 encoding values
    b1 = np.zeros(16)
    W2 = np.zeros((3, 16))
    W2[0, 0], W2[0, 1] = 1.0, -1.0
    W2[1, 2] = 1.0
    b2 = np.zeros(3)
    params = np.concatenate([W1.ravel(), b1, W2.ravel(), b2])
    rng = np.random.default_rng(5)
    pos = np.zeros((64, 4), np.float32)
    pos[:, :3] = rng.random((64, 3))
    nrm = np.zeros((64, 4), np.float32)
    nrm[:, :3] = rng.standard_normal((64, 3))
    E = oracle.query(m, params, pos, nrm)
    sp = lambda z: np.maximum(z, 0) + np.log1p(np.exp(-np.abs(z)))
    uy = pos[:, 1].astype(np.float64)
    np.testing.assert_allclose(E[:, 0], sp(np.sin(4 * math.pi * uy)), rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(E[:, 1], sp(np.maximum(nrm[:, 0].astype(np.float64), 0)), rtol=1e-13)
    np.testing.assert_allclose(E[:, 2], math.log(2.0), rtol=1e-15)


def test_loss_gradient_matches_finite_differences():
    """Eq. 3 with sg() on the denominator: the gradient equals central differences of the
    loss with the denominator frozen at the current prediction."""
    m = pe_model(width=16, n_hidden=2)
    from niv_inputs import init_params
    params = init_params(0, oracle.layer_shapes(m), seed=7, bias_std=0.1).astype(np.float64)
    rng = np.random.default_rng(8)
    pos = np.zeros((32, 4), np.float32)
    pos[:, :3] = rng.random((32, 3))
    nrm = np.zeros((32, 4), np.float32)
    nrm[:, :3] = rng.standard_normal((32, 3))
    target = rng.random((32, 3)) + 0.1
    _, g = oracle.loss_grad(m, params, pos, nrm, target)
    den = oracle.query(m, params, pos, nrm) ** 2 + 0.01

    def frozen(p):
        return np.mean((oracle.query(m, p, pos, nrm) - target) ** 2 / den)

    h = 1e-6
    for i in rng.choice(len(params), 40, replace=False):
        p1, p0 = params.copy(), params.copy()
        p1[i] += h
        p0[i] -= h
        fd = (frozen(p1) - frozen(p0)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def test_grid_and_frequency_need_one_of_them():
    bad = oracle.Model(levels=0, pe_bands=0)
    with pytest.raises(ValueError):
        oracle.layout(bad)


# ---- the FP16 network path (binary16 inputs and activations) ----

def test_f16_rounding_matches_numpy_on_every_value_and_midpoint():
    """binary16 rounding written from the format's definition agrees with numpy's float16
    conversion on every finite value, every midpoint between neighbours (ties to even),
    values beyond the largest finite one, and random values across the exponent range."""
    bits = np.arange(0, 0x7C00, dtype=np.uint16)           # all finite non-negative values
    v = bits.view(np.float16).astype(np.float64)
    mids = (v[:-1] + v[1:]) / 2.0
    above = np.array([65504.0, 65519.99, 65520.0, 70000.0, 1e300])
    rng = np.random.default_rng(11)
    rnd = rng.standard_normal(20000) * np.exp2(rng.uniform(-30, 17, 20000))
    x = np.concatenate([v, mids, above, rnd, -v, -mids, -above])
    got = oracle.f16(x)
    with np.errstate(over="ignore"):
        ref = x.astype(np.float16).astype(np.float64)
    assert np.array_equal(got, ref)


def _one_layer_net(m, w_up, w_out):
    n_in = m.n_in
    col = (1 * B + 2) * 2 + 0  # coordinate y, band 2, sine
    W1 = np.zeros((16, n_in))
    W1[0, col], W1[1, col] = w_up, -w_up
    W2 = np.zeros((3, 16))
    W2[0, 0], W2[0, 1] = w_out, -w_out
    return np.concatenate([W1.ravel(), np.zeros(16), W2.ravel(), np.zeros(3)])


def test_f16_path_rounds_inputs_and_hidden_activations():
    m = pe_model(width=16, n_hidden=1)
    rng = np.random.default_rng(12)
    pos = np.zeros((200, 4), np.float32)
    pos[:, :3] = rng.random((200, 3))
    pos[:3, 1] = [0.0, 0.125, 0.375]                   # sin(4 pi u) = 0, 1, -1 exactly
    nrm = np.zeros((200, 4), np.float32)
    sp = lambda z: np.maximum(z, 0) + np.log1p(np.exp(-np.abs(z)))
    f16 = lambda a: np.asarray(a, np.float64).astype(np.float16).astype(np.float64)
    s = np.sin(4 * np.pi * pos[:, 1].astype(np.float64))
    # weights 1 / 1: only the input value is rounded
    E = oracle.query_f16(m, _one_layer_net(m, 1.0, 1.0), pos, nrm)
    np.testing.assert_allclose(E[:, 0], sp(f16(s)), rtol=1e-15, atol=0)
    E64 = oracle.query(m, _one_layer_net(m, 1.0, 1.0), pos, nrm)
    assert np.array_equal(E[:3, 0], E64[:3, 0])
    assert np.max(np.abs(E[:, 0] - E64[:, 0])) > 0.0
    # up-weight w = f16(1/3): the hidden activation relu(w * f16(s)) is rounded again
    w = float(f16(1.0 / 3.0))
    E = oracle.query_f16(m, _one_layer_net(m, w, 3.0), pos, nrm)
    hid = f16(np.maximum(w * f16(s), 0.0)) - f16(np.maximum(-w * f16(s), 0.0))
    np.testing.assert_allclose(E[:, 0], sp(3.0 * hid), rtol=1e-15, atol=0)


# ---- Sec. 6: the scene parameter t frequency-encoded after n (3-D grid) ----

def t_model(t_bands=4, n_hidden=1):
    return oracle.Model(dims=3, levels=2, feat=2, log2_T=10, base=2.0, growth=2.0, n_hidden=n_hidden, width=16,
                        t_bands=t_bands)


def test_t_encoding_closed_forms_through_a_hand_network():
    # unit 0 = +sin(2^b pi t), unit 1 = -sin(2^b pi t), unit 2 = +cos(2^b pi t), unit 3 = -cos(...)
    # for band b = 2; outputs: sin, cos, 0 through softplus
    m = t_model()
    n_in = m.n_in
    assert n_in == 2 * 2 + 3 + 8
    b = 2
    col_s = 2 * 2 + 3 + 2 * b  # after the 4 grid features and n.xyz
    W1 = np.zeros((16, n_in))
    W1[0, col_s], W1[1, col_s], W1[2, col_s + 1], W1[3, col_s + 1] = 1.0, -1.0, 1.0, -1.0
    W2 = np.zeros((3, 16))
    W2[0, 0], W2[0, 1], W2[1, 2], W2[1, 3] = 1.0, -1.0, 1.0, -1.0
    grid = np.zeros(oracle.grid_value_count(m))
    params = np.concatenate([grid, W1.ravel(), np.zeros(16), W2.ravel(), np.zeros(3)])
    pos = np.full((1, 4), 0.3, np.float32)
    nrm = np.zeros((1, 4), np.float32)
    sp = lambda z: np.maximum(z, 0) + np.log1p(np.exp(-np.abs(z)))
    for t, s4, c4 in ((0.0, 0.0, 1.0), (0.125, 1.0, 0.0), (0.25, 0.0, -1.0), (0.375, -1.0, 0.0),
                      (1.7, 0.0, 1.0), (-0.3, 0.0, 1.0)):  # t is clamped to [0, 1]
        E = oracle.query(m, params, pos, nrm, t=t)[0]
        np.testing.assert_allclose(E[:2], sp(np.array([s4, c4])), atol=1e-15)
        assert E[2] == np.log(2.0)


def test_t_encoding_gradient_matches_finite_differences():
    from niv_inputs import init_params
    m = t_model(t_bands=3, n_hidden=2)
    params = init_params(oracle.grid_value_count(m), oracle.layer_shapes(m), seed=21, feat_range=0.3,
                         bias_std=0.2).astype(np.float64)
    rng = np.random.default_rng(22)
    pos = np.zeros((40, 4), np.float32)
    pos[:, :3] = rng.random((40, 3))
    nrm = np.zeros((40, 4), np.float32)
    nrm[:, :3] = rng.standard_normal((40, 3))
    t = rng.random(40).astype(np.float32)
    y = rng.random((40, 3)) + 0.1
    _, g = oracle.loss_grad(m, params, pos, nrm, y, t=t)

    def frozen(p, den):
        E = np.stack([oracle.query(m, p, pos[i:i + 1], nrm[i:i + 1], t=float(t[i]))[0] for i in range(40)])
        return np.mean((E - y) ** 2 / den)

    E0 = np.stack([oracle.query(m, params, pos[i:i + 1], nrm[i:i + 1], t=float(t[i]))[0] for i in range(40)])
    den = E0 ** 2 + 0.01
    h = 1e-6
    for i in rng.choice(len(params), 25, replace=False):
        p1, p0 = params.copy(), params.copy()
        p1[i] += h
        p0[i] -= h
        fd = (frozen(p1, den) - frozen(p0, den)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])
