"""GPU parity of the dynamic ambient-occlusion pass (Sec. 4.4) against the FP64 brute-force
oracle, through the C ABI.

The oracle (pinned in tests/test_oracle_ao.py) tests every ray against every triangle;
the GPU traverses a bounding-volume hierarchy in FP32.  Blocked-ray counts are integers:
they must be equal on every record whose decisions are not rounding-sensitive (the oracle
flags those by growing and shrinking each triangle by the FP32 rounding of its
parameters), and flagged records must be rare.  The in-place scaling of E by AO must be
exact in FP32.
"""
import numpy as np
import pytest

import oracle
from niv_inputs.meshes import dynamic_objects, shading_frame

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def niv():
    from paper_2602_12949_gb300.build import build
    build()
    import paper_2602_12949_gb300 as P
    return P


def frame_triangles(seed=0):
    verts, tris, _, _ = dynamic_objects(seed)
    return verts[tris].reshape(-1, 9).astype(np.float32)


@pytest.mark.parametrize("rays,radius,seed", [(8, 0.5, 0), (16, 1.0, 3)])
def test_ao_counts_match_oracle(niv, rays, radius, seed):
    W, H = 160, 90
    pos, nrm, alb, direct, cov = shading_frame(W, H, seed=0)
    tri9 = frame_triangles(0)
    dyn = niv.DynamicGeometry(tri9)
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    ao = dyn.ao(d(pos), d(nrm), rays=rays, radius=radius, seed=seed).cpu().numpy()
    ref, blocked, amb = oracle.dyn_ao(tri9, pos.astype(np.float32), nrm.astype(np.float32), rays, radius, seed=seed)
    got_blocked = np.rint((1.0 - ao) * rays).astype(np.int32)
    np.testing.assert_array_equal(ao, (1.0 - got_blocked / rays).astype(np.float32))
    clear = ~amb
    mism = np.count_nonzero(got_blocked[clear] != blocked[clear])
    print("AO %d rays R=%.1f: %d triangles, %d nodes; %d of %d records occluded somewhat, %d flagged, %d "
          "mismatches on clear records" % (rays, radius, len(tri9), dyn.node_count, np.count_nonzero(blocked),
                                           len(ao), amb.sum(), mism))
    assert mism == 0
    assert amb.mean() < 0.01
    assert np.count_nonzero(blocked) > 0.02 * len(ao)  # the pass does see the meshes
    dyn.close()


def test_ao_scales_irradiance_in_place(niv):
    W, H = 96, 54
    pos, nrm, _, _, _ = shading_frame(W, H, seed=0)
    dyn = niv.DynamicGeometry(frame_triangles(0))
    d = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    E = torch.rand((W * H, 4), device="cuda", dtype=torch.float32) + 0.5
    E0 = E.clone()
    ao = dyn.ao(d(pos), d(nrm), rays=8, radius=0.5, E=E)
    assert torch.equal(E[:, :3], E0[:, :3] * ao[:, None])
    dyn.close()


def test_far_records_are_unoccluded(niv):
    tri9 = frame_triangles(0)
    dyn = niv.DynamicGeometry(tri9)
    x4 = np.zeros((1000, 4), np.float32)
    x4[:, 0] = 100.0 + np.arange(1000, dtype=np.float32) * 0.01
    n4 = np.zeros((1000, 4), np.float32)
    n4[:, 1] = 1.0
    ao = dyn.ao(torch.from_numpy(x4).cuda(), torch.from_numpy(n4).cuda(), rays=8, radius=1.0)
    assert torch.all(ao == 1.0)
    dyn.close()


@pytest.mark.parametrize("n_tris", [1, 2, 7])
def test_small_hierarchies_match_oracle(niv, n_tris):
    # a hierarchy that is a single leaf (1 or 2 triangles) or one split: squares above a
    # floor of records, counts equal to the oracle's on every clear record
    rng = np.random.default_rng(n_tris)
    tris = []
    for i in range(n_tris):
        z, half = 0.2 + 0.1 * i, 0.3
        cx, cy = rng.uniform(-0.3, 0.3, 2)
        a, b, c = (cx - half, cy - half, z), (cx + half, cy - half, z), (cx + half, cy + half, z)
        tris.append(a + b + c)
    tri9 = np.array(tris, np.float32)
    x4 = np.zeros((4096, 4), np.float32)
    x4[:, :2] = rng.uniform(-0.6, 0.6, (4096, 2))
    n4 = np.zeros((4096, 4), np.float32)
    n4[:, 2] = 1.0
    dyn = niv.DynamicGeometry(tri9)
    ao = dyn.ao(torch.from_numpy(x4).cuda(), torch.from_numpy(n4).cuda(), rays=16, radius=1.0, seed=5).cpu().numpy()
    _, blocked, amb = oracle.dyn_ao(tri9, x4, n4, 16, 1.0, seed=5)
    got = np.rint((1.0 - ao) * 16).astype(np.int32)
    clear = ~amb
    assert np.array_equal(got[clear], blocked[clear])
    assert amb.mean() < 0.01 and np.count_nonzero(blocked) > 100
    dyn.close()


def test_bad_arguments_rejected(niv):
    with pytest.raises(niv.NivError):
        niv.DynamicGeometry(np.zeros((0, 9), np.float32))
    dyn = niv.DynamicGeometry(frame_triangles(0)[:100])
    z = torch.zeros((16, 4), device="cuda")
    for kw in (dict(rays=0), dict(rays=2000), dict(radius=0.0)):
        with pytest.raises(niv.NivError):
            dyn.ao(z, z, **kw)
    dyn.close()
