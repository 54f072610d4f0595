"""Seeded query points: positions uniform in the unit cube, normals uniform on S^2."""
import numpy as np


def sphere_directions(rng, n):
    """Directions uniform on the unit sphere (normalised Gaussian triples), float64 [n][3]."""
    v = rng.standard_normal((n, 3))
    norm = np.linalg.norm(v, axis=1, keepdims=True)
    # A zero-length Gaussian triple has probability 0; guard anyway.
    norm[norm == 0.0] = 1.0
    return v / norm


def uniform_queries(n, seed=0, lo=(0.0, 0.0, 0.0), hi=(1.0, 1.0, 1.0), dtype=np.float32):
    """Return ``(pos, nrm)`` as contiguous ``[n][4]`` arrays of ``dtype``.

    Positions are uniform in the box ``[lo, hi]``; normals are uniform on the
    unit sphere.  The fourth component of every record is zero padding.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    p = lo + (hi - lo) * rng.random((n, 3))
    d = sphere_directions(rng, n)
    pos = np.zeros((n, 4), dtype=dtype)
    nrm = np.zeros((n, 4), dtype=dtype)
    pos[:, :3] = p
    nrm[:, :3] = d
    return pos, nrm
