"""Pins of the oracle's Monte Carlo irradiance (Eq. 1) against closed forms of radiative transfer."""
import math

import numpy as np
import pytest

import oracle
from niv_inputs import empty_scene, furnace_scene, single_emitter_scene, Scene, sphere_directions
from niv_inputs.scenes import SPHERE_LEN


def _records(xyz):
    a = np.zeros((len(xyz), 4), np.float32)
    a[:, :3] = xyz
    return a


def test_uniform_sky_gives_pi_L_for_every_normal():
    """Unoccluded normal under a uniform sky of radiance L: E = pi L (every estimator sample is exact)."""
    blob = empty_scene(sky=1.0).blob()
    rng = np.random.default_rng(0)
    n = sphere_directions(rng, 64)
    x = rng.uniform(-3, 3, (64, 3))
    E, keep = oracle.mc_irradiance(blob, _records(x), _records(n), spp=64, mode=oracle.MC_TOTAL)
    np.testing.assert_allclose(E, math.pi, rtol=1e-15)
    assert keep.all()
    E2, _ = oracle.mc_irradiance(empty_scene(sky=2.5).blob(), _records(x), _records(n), spp=8, mode=oracle.MC_TOTAL)
    np.testing.assert_allclose(E2, 2.5 * math.pi, rtol=1e-15)


def test_indirect_mode_without_bounces_is_zero_and_discarded():
    """With nothing to bounce off, indirect irradiance is null and App. I discards the sample."""
    blob = empty_scene(sky=1.0).blob()
    x = _records(np.zeros((4, 3)))
    n = _records(np.tile([0.0, 1.0, 0.0], (4, 1)))
    E, keep = oracle.mc_irradiance(blob, x, n, spp=32, mode=oracle.MC_INDIRECT)
    assert np.all(E == 0.0)
    assert not keep.any()


@pytest.mark.parametrize("theta_deg,dist", [(0.0, 3.0), (30.0, 2.0), (60.0, 4.0)])
def test_sphere_emitter_closed_form(theta_deg, dist):
    """E = pi L sin^2(alpha) cos(theta), sin(alpha) = r/d, for a sphere fully above the horizon."""
    r, L = 0.5, 4.0
    th = math.radians(theta_deg)
    c = (dist * math.sin(th), dist * math.cos(th), 0.0)  # normal is +y
    blob = single_emitter_scene(c, r, L).blob()
    S = 200000
    E, _ = oracle.mc_irradiance(blob, _records([[0.0, 0.0, 0.0]]), _records([[0.0, 1.0, 0.0]]), spp=S,
                                mode=oracle.MC_TOTAL, seed=11)
    sin_a = r / dist
    expect = math.pi * L * sin_a ** 2 * math.cos(th)
    p = expect / (math.pi * L)
    sigma = math.pi * L * math.sqrt(p * (1 - p) / S)
    assert abs(E[0, 0] - expect) < 4 * sigma
    assert E[0, 0] == E[0, 1] == E[0, 2]


def test_skylight_form_factor():
    """Black room, sky seen through a 4 m x 4 m ceiling opening: E = pi L * 4 F(2/h, 2/h),
    F the point-to-parallel-rectangle form factor for a point below a rectangle corner."""
    s = Scene(has_room=True, sky=(1.0, 1.0, 1.0), skylight=(-2.0, 2.0, -2.0, 2.0),
              wall_albedo=((0.0, 0.0, 0.0),) * 6)
    h = 5.0  # point at the room centre, ceiling at y = 5

    def F(a, b):
        A, B = a / h, b / h
        return (A / math.sqrt(1 + A * A) * math.atan(B / math.sqrt(1 + A * A))
                + B / math.sqrt(1 + B * B) * math.atan(A / math.sqrt(1 + B * B))) / (2 * math.pi)

    expect = math.pi * 4 * F(2.0, 2.0)
    S = 200000
    E, keep = oracle.mc_irradiance(s.blob(), _records([[0.0, 0.0, 0.0]]), _records([[0.0, 1.0, 0.0]]), spp=S,
                                   mode=oracle.MC_TOTAL, seed=3)
    p = expect / math.pi
    sigma = math.pi * math.sqrt(p * (1 - p) / S)
    assert abs(E[0, 0] - expect) < 4 * sigma
    # with the normal turned away from the opening nothing arrives
    E, keep = oracle.mc_irradiance(s.blob(), _records([[0.0, 0.0, 0.0]]), _records([[0.0, -1.0, 0.0]]), spp=64,
                                   mode=oracle.MC_TOTAL)
    assert E[0, 0] == 0.0 and not keep[0]


@pytest.mark.parametrize("mode,expect", [(0, 2.0 * math.pi), (1, math.pi)])
def test_furnace_enclosure(mode, expect):
    """Closed room, every wall emitting L_e = 1 with albedo 0.5: L_o = L_e/(1-rho) everywhere, so
    E_total = pi L_e/(1-rho) = 2 pi and E_indirect = pi L_e rho/(1-rho) = pi."""
    blob = furnace_scene(0.5, 1.0).blob()
    rng = np.random.default_rng(1)
    m = 32
    x = rng.uniform(-4, 4, (m, 3))
    n = sphere_directions(rng, m)
    E, keep = oracle.mc_irradiance(blob, _records(x), _records(n), spp=1024, mode=mode, seed=5)
    est = E[:, 0]
    se = est.std(ddof=1) / math.sqrt(m)
    assert abs(est.mean() - expect) < 4 * se + 1e-12
    assert keep.all()


def test_points_inside_geometry_are_culled():
    """Sec. 4.5: a sample whose first hits are mostly back faces lies inside geometry and is discarded."""
    sph = np.zeros((1, SPHERE_LEN), np.float32)
    sph[0, :4] = [0.0, 0.0, 0.0, 1.0]
    sph[0, 4:7] = 0.5
    s = Scene(spheres=sph, sky=(1.0, 1.0, 1.0))
    x = _records([[0.0, 0.0, 0.0], [0.0, 3.0, 0.0]])
    n = _records([[0.0, 1.0, 0.0], [0.0, 1.0, 0.0]])
    E, keep = oracle.mc_irradiance(s.blob(), x, n, spp=256, mode=oracle.MC_TOTAL)
    assert keep.tolist() == [0, 1]


def test_philox_uniform_and_decorrelated():
    """The counter-based generator's words map to uniform (0,1) values with uncorrelated lanes."""
    u = np.array([oracle.philox([i, 0, 7, 0], [123, 456]) for i in range(20000)], np.float64)
    f = ((u.astype(np.uint32) >> 8) + 0.5) / 2 ** 24
    for lane in range(4):
        counts = np.bincount((f[:, lane] * 64).astype(int), minlength=64)
        chi2 = np.sum((counts - len(f) / 64) ** 2 / (len(f) / 64))
        assert chi2 < 63 + 6 * math.sqrt(2 * 63)
        assert abs(f[:, lane].mean() - 0.5) < 4 * math.sqrt(1 / 12 / len(f))
    c = np.corrcoef(f.T)
    assert np.max(np.abs(c - np.eye(4))) < 0.04
    # different keys give different streams; same counter and key give the same words
    assert not np.array_equal(oracle.philox([1, 2, 3, 4], [0, 0]), oracle.philox([1, 2, 3, 4], [0, 1]))
    assert np.array_equal(oracle.philox([1, 2, 3, 4], [5, 6]), oracle.philox([1, 2, 3, 4], [5, 6]))


def test_standard_error_matches_the_spread_of_independent_estimates():
    """The per-point standard error the oracle reports (sample variance of the path radiances)
    agrees with the spread of independent estimates on other streams."""
    from niv_inputs import room_scene
    blob = room_scene(0).blob()
    x = np.tile(np.array([[1.0, -2.0, 0.5, 0.0]], np.float32), (200, 1))
    n = np.tile(np.array([[0.0, 1.0, 0.0, 0.0]], np.float32), (200, 1))
    # 200 estimates of the same point, each on its own stream (index_base = point index)
    E, keep, se = oracle.mc_irradiance(blob, x, n, 64, seed=3, mode=oracle.MC_INDIRECT, want_se=True)
    spread = E.std(axis=0, ddof=1)
    rms_se = np.sqrt((se ** 2).mean(axis=0))
    np.testing.assert_allclose(rms_se, spread, rtol=0.25)
    # the bake's standard error against 100 bakes of the same probe on other streams
    P = np.array([2, 2, 2], np.int32)
    lo, hi = np.array([-1, -1, -1], np.float32), np.array([1, 1, 1], np.float32)
    bakes = np.stack([oracle.probe_bake(blob, P, lo, hi, 32, seed=10 + k) for k in range(100)])
    _, cse = oracle.probe_bake(blob, P, lo, hi, 32, seed=10, want_se=True)
    spread = bakes.std(axis=0, ddof=1)
    big = spread > 0.05 * spread.max()
    ratio = np.sqrt((cse[big] ** 2).mean()) / np.sqrt((spread[big] ** 2).mean())
    assert 0.8 < ratio < 1.25
