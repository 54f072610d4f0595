"""Pins of the oracle's probe query with ray-traced visibility ("+ RT", Sec. 5.1, App. A).

Reading: visibility-based probe rejection replaces the cosine fall-off: a ray from
x + 0.01 n toward each of the 8 probes; an occluded probe gets weight 0 before the
1e-6 clamp and the renormalisation.  The pins: with nothing in the way the weights are
the trilinear ones (a linear field of probe values is reproduced exactly); a slab
between x and half of the probes leaves them only the clamp weight (closed form); a
ray grazing a sphere flips under a small thickening of the geometry, a clear one does
not; the floor hides the probes below a floor point.
"""
import math

import numpy as np

import oracle
from niv_inputs.scenes import Scene, BOX_LEN, SPHERE_LEN

A0Y00 = math.pi * 0.28209479177387814  # E of a probe whose only coefficient is c_00 = 1


def lattice_coef(P, value_of_ijk):
    """Coefficients [Np][27] with only the band-0 term: probe irradiance A0 Y00 c00 in every direction."""
    coef = np.zeros((P[0] * P[1] * P[2], 27))
    for k in range(P[2]):
        for j in range(P[1]):
            for i in range(P[0]):
                coef[i + P[0] * (j + P[1] * k), 0:3] = value_of_ijk(i, j, k)
    return coef


def records(pts, nrm):
    x4 = np.zeros((len(pts), 4), np.float32)
    n4 = np.zeros((len(pts), 4), np.float32)
    x4[:, :3] = pts
    n4[:, :3] = nrm
    return x4, n4


def test_unoccluded_weights_are_trilinear():
    P, lo, hi = (4, 3, 5), (0.0, 0.0, 0.0), (3.0, 2.0, 4.0)  # unit cells
    coef = lattice_coef(P, lambda i, j, k: [1.0 + 0.5 * i + 0.25 * j - 0.125 * k] * 3)
    rng = np.random.default_rng(1)
    pts = rng.uniform(0.0, 1.0, (200, 3)) * np.array(hi)
    nrm = rng.standard_normal((200, 3))
    x4, n4 = records(pts, nrm)
    E, amb = oracle.probe_query_rt(coef, P, lo, hi, Scene().blob(), x4, n4)
    x = x4[:, :3].astype(np.float64)
    expect = A0Y00 * (1.0 + 0.5 * x[:, 0] + 0.25 * x[:, 1] - 0.125 * x[:, 2])
    np.testing.assert_allclose(E[:, 0], expect, rtol=1e-12)
    assert not amb.any()


def test_slab_hides_the_far_probes():
    # one cell [0,1]^3; a thin slab at z in [0.6, 0.7] across the whole cell hides the
    # z = 1 probes from points below it
    P, lo, hi = (2, 2, 2), (0.0, 0.0, 0.0), (1.0, 1.0, 1.0)
    coef = lattice_coef(P, lambda i, j, k: [1.0 + i + 2.0 * j + 4.0 * k] * 3)
    box = np.zeros((1, BOX_LEN), np.float32)
    box[0, :6] = (-1.0, -1.0, 0.6, 2.0, 2.0, 0.7)
    scene = Scene(boxes=box).blob()
    pts = np.array([[0.3, 0.6, 0.2], [0.5, 0.5, 0.4], [0.9, 0.1, 0.1]])
    x4, n4 = records(pts, np.tile([0.0, 1.0, 0.0], (3, 1)))  # n along +y: the ray origin stays below the slab
    E, amb = oracle.probe_query_rt(coef, P, lo, hi, scene, x4, n4)
    assert not amb.any()
    for q, (x, y, z) in enumerate(x4[:, :3].astype(np.float64)):
        num = den = 0.0
        for c in range(8):
            i, j, k = c & 1, (c >> 1) & 1, (c >> 2) & 1
            w = (x if i else 1 - x) * (y if j else 1 - y) * (z if k else 1 - z)
            w = max(w if k == 0 else 0.0, 1e-6)
            num += w * A0Y00 * (1.0 + i + 2.0 * j + 4.0 * k)
            den += w
        assert E[q, 0] == np.float64(num / den) or abs(E[q, 0] - num / den) <= 1e-13 * abs(num / den)


def test_grazing_ray_is_ambiguous_and_clear_rays_are_not():
    sph = np.zeros((1, SPHERE_LEN), np.float32)
    sph[0, :4] = (0.5, 0.25, 0.5, 0.25)  # touches the segment y = 0.5 at x = 0.5 from below
    scene = Scene(spheres=sph).blob()
    o = (0.0, 0.5, 0.5)
    p_graze = (1.0, 0.5, 0.5)
    assert oracle.visible(scene, o, p_graze, grow=1e-4) != oracle.visible(scene, o, p_graze, grow=-1e-4)
    p_clear = (1.0, 0.9, 0.5)
    assert oracle.visible(scene, o, p_clear, grow=1e-4) == oracle.visible(scene, o, p_clear, grow=-1e-4) == 1
    p_hidden = (1.0, 0.2, 0.5)  # through the sphere
    assert oracle.visible(scene, o, p_hidden) == 0


def test_floor_hides_probes_below_a_floor_point():
    scene = Scene(has_room=True).blob()  # the room [-5, 5]^3
    # probes on a lattice that straddles the floor y = -5; a floor point sees only those above
    P, lo, hi = (2, 2, 2), (-1.0, -5.5, -1.0), (1.0, -4.5, 1.0)
    coef = lattice_coef(P, lambda i, j, k: [1.0 if j == 1 else 100.0] * 3)
    x4, n4 = records(np.array([[0.1, -5.0, -0.2]]), np.array([[0.0, 1.0, 0.0]]))
    E, amb = oracle.probe_query_rt(coef, P, lo, hi, scene, x4, n4)
    assert not amb.any()
    # the four probes at y = -5.5 are below the floor: clamp weight 1e-6 each against ~1/8 each above
    assert abs(E[0, 0] - A0Y00) < 1e-3 * A0Y00
    assert E[0, 0] > A0Y00
