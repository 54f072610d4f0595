"""Pins of the oracle's SH probe grid (Sec. 5.1, App. A; Ramamoorthi & Hanrahan 2001)."""
import math

import numpy as np

import oracle


def _latlong(n_theta=400, n_phi=800):
    """Midpoint quadrature over the sphere: directions and solid-angle weights."""
    th = (np.arange(n_theta) + 0.5) * math.pi / n_theta
    ph = (np.arange(n_phi) + 0.5) * 2 * math.pi / n_phi
    T, P = np.meshgrid(th, ph, indexing="ij")
    d = np.stack([np.sin(T) * np.cos(P), np.sin(T) * np.sin(P), np.cos(T)], -1).reshape(-1, 3)
    w = (np.sin(T) * (math.pi / n_theta) * (2 * math.pi / n_phi)).ravel()
    return d, w


def test_sh_basis_orthonormal():
    d, w = _latlong(200, 400)
    Y = np.array([oracle.sh9(x) for x in d[::7]])
    G = (Y * w[::7, None] * 7).T @ Y
    np.testing.assert_allclose(G, np.eye(9), atol=2e-3)


def test_constant_and_linear_radiance_give_exact_irradiance():
    """L(w) = a + b (w . d)  =>  E(n) = pi a + (2 pi / 3) b (n . d); SH bands 0-1 hold it exactly."""
    d, w = _latlong(300, 600)
    axis = np.array([0.3, -0.5, 0.8])
    axis /= np.linalg.norm(axis)
    a, b = 0.7, 0.4
    L = np.repeat((a + b * d @ axis)[:, None], 3, axis=1)
    # quadrature projection of L onto the basis (uniform weights would need equal-area samples)
    Y = np.array([oracle.sh9(x) for x in d])
    coef = (Y * w[:, None]).T @ L
    for n in [axis, -axis, np.array([1.0, 0.0, 0.0]), np.array([0.0, 0.6, 0.8])]:
        E = oracle.sh_irradiance(coef, n)
        np.testing.assert_allclose(E, math.pi * a + 2 * math.pi / 3 * b * float(n @ axis), atol=1e-4)


def test_monte_carlo_projection_of_constant_radiance():
    """orc_sh_project with uniform directions: constant L gives E = pi L up to MC error."""
    rng = np.random.default_rng(0)
    v = rng.standard_normal((200000, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    coef = oracle.sh_project(v, np.ones((len(v), 3)))
    E = oracle.sh_irradiance(coef, np.array([0.0, 0.0, 1.0]))
    np.testing.assert_allclose(E, math.pi, rtol=1e-2)
    assert abs(coef[0, 0] - math.sqrt(4 * math.pi)) < 1e-12 * 1e3


def test_probe_query_at_a_probe_returns_that_probe():
    """Trilinear weight 1 at a probe; the other seven fall to the 1e-6 clamp (App. A)."""
    P = np.array([3, 3, 3], np.int32)
    lo, hi = np.array([-1.0, -1.0, -1.0], np.float32), np.array([1.0, 1.0, 1.0], np.float32)
    rng = np.random.default_rng(1)
    coef = rng.uniform(0.0, 1.0, (27, 9, 3))
    coef[:, 0, :] += 3.0
    x = np.array([[0.0, 0.0, 0.0, 0.0]], np.float32)  # the centre probe
    n = np.array([[0.0, 0.0, 1.0, 0.0]], np.float32)
    E = oracle.probe_query(coef, P, lo, hi, x, n)
    ref = oracle.sh_irradiance(coef[13], np.array([0.0, 0.0, 1.0]))
    np.testing.assert_allclose(E[0], ref, rtol=1e-4)


def test_probe_cosine_falloff_excludes_probes_behind_the_normal():
    """Probes behind the shading normal get the clamp weight, so they barely contribute."""
    P = np.array([2, 2, 2], np.int32)
    lo, hi = np.array([0.0, 0.0, 0.0], np.float32), np.array([1.0, 1.0, 1.0], np.float32)
    coef = np.zeros((8, 9, 3))
    # probes with z = 1 (indices 4..7) carry constant irradiance pi*1, probes with z = 0 carry pi*5
    coef[4:, 0, :] = math.sqrt(4 * math.pi) * 1.0
    coef[:4, 0, :] = math.sqrt(4 * math.pi) * 5.0
    x = np.array([[0.5, 0.5, 0.5, 0.0]], np.float32)
    up = oracle.probe_query(coef, P, lo, hi, x, np.array([[0.0, 0.0, 1.0, 0.0]], np.float32))
    down = oracle.probe_query(coef, P, lo, hi, x, np.array([[0.0, 0.0, -1.0, 0.0]], np.float32))
    np.testing.assert_allclose(up[0], math.pi * 1.0, rtol=1e-4)
    np.testing.assert_allclose(down[0], math.pi * 5.0, rtol=1e-4)
    side = oracle.probe_query(coef, P, lo, hi, x, np.array([[1.0, 0.0, 0.0, 0.0]], np.float32))
    np.testing.assert_allclose(side[0], math.pi * 3.0, rtol=1e-4)  # equal weight to both planes


def test_probe_bake_of_furnace_room():
    """Furnace (walls emit 1, albedo 0.5): indirect radiance is 1 in every direction -> E = pi."""
    from niv_inputs import furnace_scene
    blob = furnace_scene(0.5, 1.0).blob()
    P = np.array([2, 2, 2], np.int32)
    lo, hi = np.array([-2.0, -2.0, -2.0], np.float32), np.array([2.0, 2.0, 2.0], np.float32)
    coef = oracle.probe_bake(blob, P, lo, hi, rays=4096, seed=1)
    x = np.array([[0.3, -0.2, 0.1, 0.0]], np.float32)
    n = np.array([[0.0, 1.0, 0.0, 0.0]], np.float32)
    E = oracle.probe_query(coef, P, lo, hi, x, n)
    np.testing.assert_allclose(E[0], math.pi, rtol=0.08)
