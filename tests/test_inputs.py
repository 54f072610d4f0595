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


def test_dynamic_objects_recipe():
    from niv_inputs.meshes import torus, icosphere, twisted_box, dynamic_objects
    assert len(torus()[1]) == 50000 and len(icosphere()[1]) == 81920 and len(twisted_box()[1]) == 49152
    v, f = torus()
    assert len(v) - (3 * len(f) // 2) + len(f) == 0      # Euler characteristic of a torus
    v, f = icosphere()
    assert len(v) - (3 * len(f) // 2) + len(f) == 2      # ... of a sphere
    np.testing.assert_allclose(np.linalg.norm(v, axis=1), 0.6, rtol=1e-12)
    verts, tris, ids, albedo = dynamic_objects(0)
    assert tris.max() < len(verts) and set(np.unique(ids)) == {0, 1, 2}
    assert np.all((albedo >= 0.1) & (albedo <= 0.9))


def test_shading_frame_coverage(tmp_path):
    from niv_inputs.meshes import shading_frame
    pos, nrm, alb, direct, cov = shading_frame(960, 540, cache_dir=str(tmp_path))
    assert 0.04 <= cov <= 0.12  # dynamic objects cover 5-10% of the frame (Sec. 5.2)
    assert np.all(np.isfinite(pos.astype(np.float32)))
    assert np.all((direct[:, :3] >= 0) & (direct[:, :3] <= 0.5))
