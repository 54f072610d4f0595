"""Pins of the oracle's training-sample candidates (Sec. 4.5 / App. I): a fraction of the
points on the surfaces with the surface normal, the rest uniform in the volume with uniform
directions, surfaces chosen in proportion to area."""
import math

import numpy as np
import pytest

import oracle
from niv_inputs import room_scene

scipy_stats = pytest.importorskip("scipy.stats")

N = 200000


@pytest.fixture(scope="module")
def room():
    sc = room_scene()
    blob = sc.blob()
    x4, n4, t, patch = oracle.training_samples(blob, N, surface_frac=0.2, seed=3, with_t=True)
    return sc, blob, x4.astype(np.float64), n4.astype(np.float64), t, patch


def test_surface_fraction_is_binomial(room):
    _, _, _, _, _, patch = room
    k = int((patch >= 0).sum())
    sigma = math.sqrt(N * 0.2 * 0.8)
    assert abs(k - 0.2 * N) <= 4 * sigma
    for frac in (0.0, 1.0):
        _, _, _, p = oracle.training_samples(room[1], 5000, surface_frac=frac, seed=1)
        assert (p >= 0).mean() == frac


def test_surfaces_are_chosen_in_proportion_to_area(room):
    _, blob, _, _, _, patch = room
    P = oracle.sample_patches(blob)
    area = P[:, 12]
    # the surfaces of the room: 9 wall pieces (ceiling cut around the skylight), 24 spheres, 48 box faces
    assert len(P) == 9 + 24 + 48
    sc = room[0]
    room_area = 2 * 3 * 100.0 - (sc.skylight[1] - sc.skylight[0]) * (sc.skylight[3] - sc.skylight[2])
    assert abs(area[:9].sum() - room_area) < 1e-9
    counts = np.bincount(patch[patch >= 0], minlength=len(P))
    expect = counts.sum() * area / area.sum()
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    assert scipy_stats.chi2.sf(chi2, len(P) - 1) > 1e-4
    # a uniform choice of surface (area ignored) is rejected by the same test
    flat = counts.sum() / len(P)
    chi2_flat = float(((counts - flat) ** 2 / flat).sum())
    assert scipy_stats.chi2.sf(chi2_flat, len(P) - 1) < 1e-12


def test_surface_points_lie_on_their_surface_with_its_normal(room):
    _, blob, x, n, _, patch = room
    P = oracle.sample_patches(blob)
    s = patch >= 0
    rows = P[patch[s]]
    xs, ns = x[s, :3], n[s, :3]
    rect = rows[:, 0] == 0
    ax = rows[rect, 1].astype(int)
    idx = np.nonzero(rect)[0]
    # on the plane, exactly; inside the bounds; normal = sign * e_axis exactly
    assert np.all(xs[idx, ax] == rows[rect, 3].astype(np.float32))
    other = np.array([[1, 2], [0, 2], [0, 1]])[ax]
    a = xs[idx, other[:, 0]]
    b = xs[idx, other[:, 1]]
    assert np.all((a >= rows[rect, 4] - 1e-6) & (a <= rows[rect, 5] + 1e-6))
    assert np.all((b >= rows[rect, 6] - 1e-6) & (b <= rows[rect, 7] + 1e-6))
    nexp = np.zeros((len(idx), 3))
    nexp[np.arange(len(idx)), ax] = rows[rect, 2]
    np.testing.assert_array_equal(ns[idx], nexp)
    # walls face into the room, box faces away from their box
    sph = ~rect
    c, r = rows[sph, 8:11], rows[sph, 11]
    d = xs[sph] - c
    np.testing.assert_allclose(np.linalg.norm(d, axis=1), r, rtol=1e-6)
    np.testing.assert_allclose(ns[sph], d / r[:, None], atol=2e-6)


def test_no_ceiling_sample_in_the_skylight(room):
    sc, _, x, _, _, patch = room
    x0, x1, z0, z1 = sc.skylight
    ceiling = (patch >= 0) & (x[:, 1] == sc.room_max[1])
    inside = (x[:, 0] > x0) & (x[:, 0] < x1) & (x[:, 2] > z0) & (x[:, 2] < z1)
    assert ceiling.sum() > 100
    assert not np.any(ceiling & inside)


def test_volume_points_uniform_in_the_room_with_uniform_directions(room):
    sc, _, x, n, t, patch = room
    v = patch < 0
    lo, hi = np.asarray(sc.room_min), np.asarray(sc.room_max)
    xv, nv = x[v, :3], n[v, :3]
    assert np.all((xv >= lo) & (xv <= hi))
    m = len(xv)
    # uniform in the box: each coordinate's mean and variance
    u = (xv - lo) / (hi - lo)
    assert np.all(np.abs(u.mean(0) - 0.5) <= 4 * math.sqrt(1 / 12 / m))
    np.testing.assert_allclose(np.linalg.norm(nv, axis=1), 1.0, atol=1e-6)
    # uniform on the sphere: mean 0, E[d d^T] = I / 3
    assert np.all(np.abs(nv.mean(0)) <= 4 * math.sqrt(1 / 3 / m))
    cov = nv.T @ nv / m
    assert np.all(np.abs(cov - np.eye(3) / 3) <= 4 * math.sqrt(4 / 45 / m) + 1e-12)
    assert abs(float(t.mean()) - 0.5) <= 4 * math.sqrt(1 / 12 / N)
    assert t.min() > 0 and t.max() < 1


def test_counter_based_streams():
    blob = room_scene().blob()
    a = oracle.training_samples(blob, 100, seed=7, index_base=0, with_t=True)
    b = oracle.training_samples(blob, 90, seed=7, index_base=10, with_t=True)
    for u, v in zip(a, b):
        np.testing.assert_array_equal(u[10:], v)
    c = oracle.training_samples(blob, 100, seed=8, index_base=0)
    assert not np.array_equal(a[0], c[0])
