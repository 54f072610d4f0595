"""GPU training-sample candidates (niv_training_samples) against the oracle's sampler.

Integer decisions (surface or volume, which surface) are taken from the same FP32 uniforms
and the same FP32 cumulative area fractions on both sides: bit-exact.  Points on walls and
box faces and in the volume are FP32 products and sums in a fixed order: bit-exact.  Sphere
points and all directions go through sin / cos (CUDA's in FP32, C's in FP64): within 2e-6."""
import numpy as np
import pytest

import oracle
from niv_inputs import room_scene

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def niv():
    from paper_2602_12949_gb300.build import build
    build()
    import paper_2602_12949_gb300 as P
    return P


@pytest.mark.parametrize("n,frac,seed,base", [(200003, 0.2, 5, 0), (4099, 0.2, 6, 1 << 33), (1000, 1.0, 1, 7),
                                              (1000, 0.0, 2, 0)])
def test_samples_match_oracle(niv, n, frac, seed, base):
    blob = room_scene().blob()
    x4, n4, t, patch = niv.training_samples(blob, n, surface_frac=frac, seed=seed, index_base=base, with_t=True,
                                            want_patch=True)
    niv.sync_status()
    ox, on, ot, op = oracle.training_samples(blob, n, surface_frac=frac, seed=seed, index_base=base, with_t=True)
    gp = patch.cpu().numpy()
    np.testing.assert_array_equal(gp, op)
    np.testing.assert_array_equal(t.cpu().numpy(), ot)
    gx, gn = x4.cpu().numpy(), n4.cpu().numpy()
    P = oracle.sample_patches(blob)
    on_sphere = np.zeros(n, bool)
    s = op >= 0
    on_sphere[s] = P[op[s], 0] == 1
    exact = ~on_sphere
    np.testing.assert_array_equal(gx[exact], ox[exact])
    np.testing.assert_array_equal(gn[exact & s], on[exact & s])
    np.testing.assert_allclose(gx[on_sphere], ox[on_sphere], atol=2e-6 * 5)
    np.testing.assert_allclose(gn, on, atol=2e-6)
    assert np.all(gx[:, 3] == 0) and np.all(gn[:, 3] == 0)


def test_samples_without_room_walls(niv):
    """Only objects: every surface sample lands on a sphere or a box face."""
    blob = room_scene().blob().copy()
    blob[2] = 0.0  # no room
    x4, n4, t, patch = niv.training_samples(blob, 5000, surface_frac=1.0, seed=4, want_patch=True)
    ox, on, _, op = oracle.training_samples(blob, 5000, surface_frac=1.0, seed=4)
    np.testing.assert_array_equal(patch.cpu().numpy(), op)
    assert len(oracle.sample_patches(blob)) == 24 + 48
