"""Pins of the oracle's dynamic ambient-occlusion pass (Sec. 4.4).

Reading: AO = 1 - blocked / K over K cosine-distributed rays from x + 0.01 n, blocked
when a dynamic triangle is met at 0 < t <= R.  Closed forms: a large plane at height h
above the ray origin blocks exactly the directions with cos(theta) >= h / R, which a
cosine-distributed direction has with probability 1 - (h / R)^2 (pins the direction
distribution and the intersection together); a plane behind the point, a plane beyond R
and no triangles at all leave AO = 1 exactly; the blocked counts are integers that add up.
"""
import numpy as np

import oracle


def square(z, half, cx=0.0, cy=0.0):
    """Two triangles covering [cx - half, cx + half] x [cy - half, cy + half] at height z."""
    a, b, c, d = (cx - half, cy - half, z), (cx + half, cy - half, z), (cx + half, cy + half, z), (cx - half, cy + half, z)
    return np.array([a + b + c, a + c + d], np.float32)


def floor_records(m, seed=0, spread=0.05):
    rng = np.random.default_rng(seed)
    x4 = np.zeros((m, 4), np.float32)
    x4[:, :2] = rng.uniform(-spread, spread, (m, 2))
    n4 = np.zeros((m, 4), np.float32)
    n4[:, 2] = 1.0
    return x4, n4


def test_plane_above_blocks_one_minus_c_squared():
    h, R = 0.3, 0.6
    tris = square(0.01 + h, 2.0)  # the ray origins sit at z = 0.01
    x4, n4 = floor_records(256, seed=1)
    K = 256
    ao, blocked, amb = oracle.dyn_ao(tris, x4, n4, K, R, seed=7)
    p = blocked.sum() / (K * len(x4))
    expect = 1.0 - (h / R) ** 2
    sigma = np.sqrt(expect * (1 - expect) / (K * len(x4)))
    assert abs(p - expect) < 4 * sigma, (p, expect, sigma)
    np.testing.assert_array_equal(ao, 1.0 - blocked / K)
    assert amb.mean() < 0.01


def test_no_occlusion_cases_are_exact():
    x4, n4 = floor_records(64, seed=2)
    for tris, R in ((square(-0.5, 2.0), 1.0),            # behind the surface
                    (square(0.01 + 1.5, 2.0), 1.0),      # beyond the radius
                    (np.zeros((0, 9), np.float32), 1.0)):  # nothing dynamic
        ao, blocked, amb = oracle.dyn_ao(tris, x4, n4, 32, R, seed=3)
        assert np.all(ao == 1.0) and np.all(blocked == 0) and not amb.any()


def test_same_seed_same_counts_other_seed_other_directions():
    h, R = 0.3, 0.6
    tris = square(0.01 + h, 2.0)
    x4, n4 = floor_records(128, seed=4)
    _, b1, _ = oracle.dyn_ao(tris, x4, n4, 64, R, seed=11)
    _, b2, _ = oracle.dyn_ao(tris, x4, n4, 64, R, seed=11)
    _, b3, _ = oracle.dyn_ao(tris, x4, n4, 64, R, seed=12)
    np.testing.assert_array_equal(b1, b2)
    assert not np.array_equal(b1, b3)


def test_small_occluder_matches_solid_angle_estimate():
    # a square of side s at height h straight above: for small s, the cosine-weighted
    # probability of meeting it is ~ cos(theta) dOmega / pi = s^2 / (pi h^2)
    h, s, R = 0.5, 0.05, 1.0
    tris = square(0.01 + h, s / 2)
    x4 = np.zeros((1, 4), np.float32)
    n4 = np.zeros((1, 4), np.float32)
    n4[0, 2] = 1.0
    K = 1024
    total = 0
    for seed in range(64):
        _, b, _ = oracle.dyn_ao(tris, x4, n4, K, R, seed=seed)
        total += int(b[0])
    p = total / (64 * K)
    expect = s * s / (np.pi * h * h)
    sigma = np.sqrt(expect * (1 - expect) / (64 * K))
    assert abs(p - expect) < 4 * sigma + 0.02 * expect, (p, expect)
