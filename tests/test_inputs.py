"""The seeded input generators: C and numpy ray casts agree; scenes are as specified."""
import numpy as np

from niv_inputs import room_scene, raycast_gbuffer
from niv_inputs.scenes import ROOM_MIN, ROOM_MAX, CAMERA_POS


def test_c_and_numpy_raycasts_agree():
    s = room_scene(0)
    a = raycast_gbuffer(s, 200, 120, impl="numpy")
    b = raycast_gbuffer(s, 200, 120, impl="c")
    for x, y in zip(a[:3], b[:3]):
        np.testing.assert_allclose(x, y, rtol=0, atol=1e-7)
    np.testing.assert_array_equal(a[3], b[3])


def test_room_scene_recipe():
    s = room_scene(3)
    assert len(s.spheres) == 25 and len(s.boxes) == 8  # 24 random spheres + the emitter
    lo, hi = np.array(ROOM_MIN), np.array(ROOM_MAX)
    for sp in s.spheres[:-1]:
        c, r = sp[:3], sp[3]
        assert 0.2 <= r <= 1.5 and np.all(c - r >= lo - 1e-6) and np.all(c + r <= hi + 1e-6)
        assert np.linalg.norm(c - np.array(CAMERA_POS)) > r
        assert np.all((sp[4:7] >= 0.1) & (sp[4:7] <= 0.9))
    for bx in s.boxes:
        he = (bx[3:6] - bx[:3]) / 2
        assert np.all(he >= 0.2 - 1e-6) and np.all(he <= 1.0 + 1e-6)
    assert s.spheres[-1, 7] == 20.0 and s.rot_sphere == 24


def test_gbuffer_hits_everything_inside_the_closed_room():
    pos, nrm, alb, hit = raycast_gbuffer(room_scene(0), 320, 180)
    assert hit.all()
    np.testing.assert_allclose(np.linalg.norm(nrm, axis=1), 1.0, atol=1e-9)
    assert np.all(np.abs(pos) <= 5.0 + 1e-9)
    # normals face the camera
    d = pos - np.array(CAMERA_POS)
    assert np.all(np.einsum("ij,ij->i", d, nrm) < 0)
