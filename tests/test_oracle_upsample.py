"""Pins of the oracle's half-resolution rendering step (Sec. 4.4, Table 1 "half").

Reading: E is queried at every s-th pixel of every s-th row; each full-resolution
pixel blends its (up to) four low-resolution samples with bilinear weights times a
range term max(0, n_p.n_q)^P exp(-(n_p.(x_q - x_p) / sigma)^2) plus eps (joint
bilateral upsampling, Kopf et al. 2007), then shades with its own albedo and direct
light.  Each pin below fails for a plausible mistake: a wrong sample position or
bilinear weight (linear field on a plane), a missing normalisation (constant field),
no depth or normal rejection (step edge, opposite normals), a wrong shading term (s = 1).
"""
import math

import numpy as np

import oracle


def plane_gbuffer(W, H, z=None, normal=(0.0, 0.0, -1.0)):
    """Records of a plane facing the camera: x = X / W, y = Y / H, z per pixel."""
    X, Y = np.meshgrid(np.arange(W), np.arange(H))
    pos = np.zeros((H * W, 4), np.float32)
    pos[:, 0] = (X / W).ravel()
    pos[:, 1] = (Y / H).ravel()
    pos[:, 2] = 1.0 if z is None else np.asarray(z, np.float32).ravel()
    nrm = np.zeros((H * W, 4), np.float32)
    nrm[:, :3] = normal
    return pos, nrm


def materials(n, seed=0):
    rng = np.random.default_rng(seed)
    alb = np.zeros((n, 4), np.float32)
    dr = np.zeros((n, 4), np.float32)
    alb[:, :3] = rng.uniform(0.1, 0.9, (n, 3))
    dr[:, :3] = rng.uniform(0.0, 0.5, (n, 3))
    return alb, dr


def low_res_shape(W, H, s):
    return (W + s - 1) // s, (H + s - 1) // s


def test_sub_one_is_plain_shading():
    W, H = 13, 7
    pos, nrm = plane_gbuffer(W, H)
    alb, dr = materials(W * H)
    E = np.random.default_rng(1).uniform(0.0, 3.0, (W * H, 3))
    out = oracle.upsample_shade(pos, nrm, alb, dr, W, H, E, sub=1)
    ref = alb[:, :3] * E / math.pi + dr[:, :3]
    np.testing.assert_allclose(out, ref, rtol=1e-15, atol=1e-15)


def test_constant_field_passes_through():
    W, H, s = 17, 11, 2
    rng = np.random.default_rng(2)
    pos = np.zeros((W * H, 4), np.float32)
    pos[:, :3] = rng.uniform(-1, 1, (W * H, 3))
    nrm = np.zeros((W * H, 4), np.float32)
    v = rng.standard_normal((W * H, 3))
    nrm[:, :3] = v / np.linalg.norm(v, axis=1, keepdims=True)
    alb, dr = materials(W * H, 3)
    w, h = low_res_shape(W, H, s)
    c = np.array([0.7, 1.3, 2.1])
    out = oracle.upsample_shade(pos, nrm, alb, dr, W, H, np.tile(c, (w * h, 1)), sub=s)
    np.testing.assert_allclose(out, alb[:, :3] * c / math.pi + dr[:, :3], rtol=1e-14)


def test_linear_field_on_a_plane_is_bilinear_interpolation():
    # On one plane every range term is 1, so the weights are the bilinear ones.  A field
    # linear in the full-resolution pixel coordinates of the samples, E(sample at (s i, s j))
    # = a + b (s i) + c (s j), is reproduced exactly at every pixel away from the clamped
    # right / bottom border.
    for s in (2, 3):
        W, H = 20, 12
        pos, nrm = plane_gbuffer(W, H)
        alb = np.ones((W * H, 4), np.float32)  # out = E / pi
        dr = np.zeros((W * H, 4), np.float32)
        w, h = low_res_shape(W, H, s)
        I, J = np.meshgrid(np.arange(w), np.arange(h))
        lin = lambda x, y: np.stack([1.0 + 0.5 * x + 0.25 * y, 2.0 - 0.1 * x, 0.3 * y], -1)
        E = lin(s * I, s * J).reshape(-1, 3)
        out = math.pi * oracle.upsample_shade(pos, nrm, alb, dr, W, H, E, sub=s, eps=0.0).reshape(H, W, 3)
        X, Y = np.meshgrid(np.arange(W), np.arange(H))
        inside = (X // s + 1 < w) & (Y // s + 1 < h)
        np.testing.assert_allclose(out[inside], lin(X, Y)[inside], rtol=0, atol=1e-12)
        # on the clamped border the missing neighbour is the sample itself
        border = ~inside
        Xc = np.minimum(X, s * (w - 1))
        Yc = np.minimum(Y, s * (h - 1))
        ref_b = lin(np.where(X // s + 1 < w, X, Xc), np.where(Y // s + 1 < h, Y, Yc))
        np.testing.assert_allclose(out[border], ref_b[border], rtol=0, atol=1e-12)


def test_depth_step_rejects_the_far_samples():
    # Left part of the image at depth 1 (E = 1), right part at depth 2 (E = 5): pixels of the
    # near part next to the step keep E ~ 1 instead of the bilinear blend.
    W, H, s = 16, 8, 2
    X, Y = np.meshgrid(np.arange(W), np.arange(H))
    z = np.where(X < 9, 1.0, 2.0)
    pos, nrm = plane_gbuffer(W, H, z=z)
    alb = np.ones((W * H, 4), np.float32)
    dr = np.zeros((W * H, 4), np.float32)
    w, h = low_res_shape(W, H, s)
    I, J = np.meshgrid(np.arange(w), np.arange(h))
    E = np.repeat(np.where(s * I < 9, 1.0, 5.0).reshape(-1, 1), 3, 1)
    eps = 1e-4
    out = math.pi * oracle.upsample_shade(pos, nrm, alb, dr, W, H, E, sub=s, sigma=0.05, eps=eps).reshape(H, W, 3)
    # pixel X = 7 (near) blends samples at X = 6 (near) and X = 8 (near): exactly 1
    np.testing.assert_allclose(out[:, 7], 1.0, rtol=1e-15)
    # pixel X = 9 is far; its samples sit at X = 8 (near, rejected) and X = 10 (far)
    g_far = math.exp(-(1.0 / 0.05) ** 2)
    expect = (0.5 * (g_far + eps) * 1.0 + 0.5 * (1.0 + eps) * 5.0) / (0.5 * (g_far + eps) + 0.5 * (1.0 + eps))
    np.testing.assert_allclose(out[:, 9], expect, rtol=1e-13)
    assert abs(expect - 5.0) < 1e-3


def test_opposite_normals_fall_back_to_bilinear():
    W, H, s = 10, 6, 2
    pos, nrm = plane_gbuffer(W, H)
    nrm[1::2, :3] = (0.0, 0.0, 1.0)  # every other pixel flipped: no sample agrees with them
    alb = np.ones((W * H, 4), np.float32)
    dr = np.zeros((W * H, 4), np.float32)
    w, h = low_res_shape(W, H, s)
    E = np.random.default_rng(4).uniform(0.5, 2.0, (w * h, 3))
    out = oracle.upsample_shade(pos, nrm, alb, dr, W, H, E, sub=s)
    bil = oracle.upsample_shade(pos, np.tile(nrm[:1], (W * H, 1)), alb, dr, W, H, E, sub=s, eps=0.0)
    # a pixel whose normal opposes all its samples' normals gets eps-only weights: bilinear
    X, Y = np.meshgrid(np.arange(W), np.arange(H))
    flipped = ((Y * W + X) % 2 == 1).ravel()
    samples_even = ((s * Y) * W + s * X) % 2 == 0  # sample pixels sit at even linear indices here
    assert samples_even.all()
    np.testing.assert_allclose(out[flipped], bil[flipped], rtol=1e-12)
