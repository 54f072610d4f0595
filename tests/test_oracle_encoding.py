"""Pins of the oracle's encoding (Sec. 4.1) against things other than itself."""
import numpy as np
import pytest
from scipy.interpolate import RegularGridInterpolator

import oracle
from niv_inputs import init_params, uniform_queries
from conftest import read_golden


def _mlp_bytes_fp16(levels, feat, width=64, matrices=4, n_out=3, n_extra=3):
    n_in = levels * feat + n_extra
    n, k = 0, n_in
    for _ in range(matrices - 1):
        n += width * k + width
        k = width
    n += n_out * k + n_out
    return 2 * n


def test_table1_memory_column():
    """Table 1: grid of F=4 FP16 features, base 16, scale sqrt(2), T=2^17 -> 1.20/3.30/5.40 MB."""
    for levels, mb in read_golden("table1_memory.txt"):
        levels = int(levels)
        m = oracle.Model(levels=levels, feat=4, base=16.0, growth=2.0 ** 0.5, log2_T=17)
        grid_bytes = oracle.layout(m)["total"] * 4 * 2
        total = grid_bytes + (_mlp_bytes_fp16(levels, 4) if levels == 2 else 0)
        assert round(total / 1e6, 2) == pytest.approx(mb), (levels, total)


def test_table1_rejects_cell_count_reading():
    """The same column under an N^3-cells rule would give 5.30 MB, not 5.40: the vertex rule is pinned."""
    m = oracle.Model(levels=8, feat=4, base=16.0, growth=2.0 ** 0.5, log2_T=17)
    L = oracle.layout(m)
    cells = sum(int(N) ** 3 if int(N) ** 3 <= 2 ** 17 else 2 ** 17 for N in L["res"])
    assert round(cells * 8 / 1e6, 2) != 5.40
    assert round(L["total"] * 8 / 1e6, 2) == 5.40


def _dense_model(levels=3, feat=2):
    # resolutions 2, 4, 8: powers of two so that vertex coordinates are exact in FP32
    return oracle.Model(levels=levels, feat=feat, base=2.0, growth=2.0, log2_T=20)


def test_dense_levels_equal_trilinear_interpolation_on_regular_grid():
    """A dense level is trilinear interpolation of (N+1)^3 vertex values (scipy's RegularGridInterpolator)."""
    m = _dense_model()
    L = oracle.layout(m)
    assert all(L["dense"] == 1)
    params = init_params(L["total"] * m.feat, [], seed=3, feat_range=1.0)
    pos, _ = uniform_queries(4096, seed=5)
    enc = oracle.encode(m, params, pos)
    grid = params.astype(np.float64).reshape(-1, m.feat)
    for l in range(m.levels):
        N = int(L["res"][l])
        tab = grid[L["offset"][l]:L["offset"][l] + L["entries"][l]]
        axes = [np.arange(N + 1) / N] * 3
        for j in range(m.feat):
            vol = tab[:, j].reshape((N + 1,) * 3, order="F")  # x varies fastest
            ref = RegularGridInterpolator(axes, vol, method="linear")(pos[:, :3].astype(np.float64))
            np.testing.assert_allclose(enc[:, l * m.feat + j], ref, rtol=0, atol=1e-12)


def test_vertex_exactness_and_upper_clamp():
    """At u*N integer the encoding is the stored vertex value; u = 1 lands on vertex N (cell N-1, w = 1)."""
    m = _dense_model(levels=1, feat=1)
    L = oracle.layout(m)
    N = int(L["res"][0])
    params = init_params(L["total"], [], seed=7, feat_range=1.0)
    vol = params.astype(np.float64).reshape((N + 1,) * 3, order="F")
    v = np.stack(np.meshgrid(*[np.arange(N + 1)] * 3, indexing="ij"), -1).reshape(-1, 3)
    pos = np.zeros((len(v), 4), np.float32)
    pos[:, :3] = v / N
    enc = oracle.encode(m, params, pos)
    np.testing.assert_array_equal(enc[:, 0], vol[v[:, 0], v[:, 1], v[:, 2]])


def test_multilinear_along_each_axis_inside_a_cell_including_hashed_levels():
    """Inside one cell the encoding is affine along each axis (second differences vanish)."""
    m = oracle.Model()  # 8 levels, 3 hashed
    L = oracle.layout(m)
    params = init_params(L["total"] * m.feat, [], seed=11, feat_range=1.0)
    rng = np.random.default_rng(0)
    for l in range(m.levels):
        N = int(L["res"][l])
        F = m.feat
        for _ in range(20):
            # three points along one axis, all inside the same cell of level l
            c = (rng.integers(0, N, 3) + 0.3) / N
            h = 0.1 / N
            for ax in range(3):
                pts = np.zeros((3, 4), np.float32)
                for s in range(3):
                    pts[s, :3] = c
                    pts[s, ax] += s * h
                e = oracle.encode(m, params, pts)[:, l * F:(l + 1) * F]
                # affine in the cell coordinate s = fp32(u * N) actually used
                u = (pts[:, ax] * np.float32(N)).astype(np.float32).astype(np.float64)
                slope = (e[2] - e[0]) / (u[2] - u[0])
                mid = e[0] + slope * (u[1] - u[0])
                assert np.max(np.abs(mid - e[1])) < 1e-9


def test_weights_partition_of_unity_and_hash_range():
    m = oracle.Model()
    L = oracle.layout(m)
    params = init_params(L["total"] * m.feat, [], seed=1)
    pos, _ = uniform_queries(2048, seed=2)
    _, idx, w = oracle.encode(m, params, pos, want_corners=True)
    np.testing.assert_allclose(w.sum(axis=2), 1.0, atol=1e-12)
    assert np.all(w >= 0)
    T = 1 << m.log2_T
    for l in range(m.levels):
        assert idx[:, l].max() < L["entries"][l]
        if not L["dense"][l]:
            assert idx[:, l].max() < T


def test_hashed_corner_indices_follow_published_constants():
    """Hashed levels index with XOR of v_k * pi_k mod T, pi from Mueller et al. 2022 Eq. 4."""
    primes = [int(p) for _, p in read_golden("hash_primes.txt")]
    m = oracle.Model()
    L = oracle.layout(m)
    params = init_params(L["total"] * m.feat, [], seed=1)
    pos, _ = uniform_queries(512, seed=9)
    _, idx, _ = oracle.encode(m, params, pos, want_corners=True)
    T = 1 << m.log2_T
    for l in np.nonzero(L["dense"] == 0)[0]:
        N = np.float32(L["res"][l])
        s = (pos[:, :3] * N).astype(np.float32)  # one FP32 product
        i = np.minimum(np.floor(s).astype(np.int64), int(N) - 1)
        for c in range(8):
            v = i + np.array([(c >> k) & 1 for k in range(3)])
            h = np.zeros(len(v), np.uint64)
            for k in range(3):
                h ^= (v[:, k].astype(np.uint64) * np.uint64(primes[k])) & np.uint64(0xFFFFFFFF)
            np.testing.assert_array_equal(idx[:, l, c], (h % np.uint64(T)).astype(np.uint32))


def test_hash_occupancy_matches_random_placement():
    """All N^3 cell-origin vertices of a hashed level occupy the table like random placement.

    With V vertices thrown into T slots at random the used fraction is 1 - exp(-V/T).
    The XOR hash of small coordinates is somewhat more clustered than random
    (0.69 vs 0.81 at N = 30), but a hash that drops a dimension or collapses
    bits falls far below it (at most N^2 distinct slots).
    """
    m = oracle.Model(levels=8)
    L = oracle.layout(m)
    params = init_params(L["total"] * m.feat, [], seed=1)
    T = 1 << m.log2_T
    for l in np.nonzero(L["dense"] == 0)[0]:
        N = int(L["res"][l])
        g = (np.arange(N) + 0.5) / N
        cz, cy, cx = np.meshgrid(g, g, g, indexing="ij")
        pos = np.zeros((N ** 3, 4), np.float32)
        pos[:, 0], pos[:, 1], pos[:, 2] = cx.ravel(), cy.ravel(), cz.ravel()
        _, idx, _ = oracle.encode(m, params, pos, want_corners=True)
        used = len(np.unique(idx[:, l, 0])) / T
        expected = 1.0 - np.exp(-(N ** 3) / T)
        assert 0.8 * expected < used <= expected + 0.02, (l, used, expected)


def test_normalisation_is_fp32_sub_then_mul():
    """u = fp32(fp32(p - min) * fp32(1/(max-min))): same encoding as pre-normalised FP32 inputs."""
    m = oracle.Model()
    L = oracle.layout(m)
    params = init_params(L["total"] * m.feat, [], seed=1)
    lo = np.array([-5.0, -5.0, -5.0], np.float32)
    hi = np.array([5.0, 5.0, 5.0], np.float32)
    pos, _ = uniform_queries(4096, seed=6, lo=lo, hi=hi)
    inv = np.float32(1.0 / (np.float64(hi[0]) - np.float64(lo[0])))
    u = np.zeros_like(pos)
    u[:, :3] = np.clip((pos[:, :3] - lo) * inv, 0, 1)  # numpy float32 ops: one rounding each
    np.testing.assert_array_equal(oracle.encode(m, params, pos, lo, hi), oracle.encode(m, params, u))


def test_four_dimensional_grid_is_quadrilinear_in_dense_levels():
    """A dense 4-D level equals 4-linear interpolation of the (N+1)^4 vertex values."""
    m = oracle.Model(dims=4, levels=2, feat=1, base=2.0, growth=2.0, log2_T=20, in_extra=4)
    L = oracle.layout(m)
    assert all(L["dense"] == 1)
    params = init_params(L["total"], [], seed=13, feat_range=1.0)
    pos, _ = uniform_queries(256, seed=8)
    ts = np.random.default_rng(1).random(256).astype(np.float32)
    grid = params.astype(np.float64)
    for q in range(0, 256, 17):
        enc = oracle.encode(m, params, pos[q:q + 1], t=float(ts[q]))
        for l in range(m.levels):
            N = int(L["res"][l])
            vol = grid[L["offset"][l]:L["offset"][l] + L["entries"][l]].reshape((N + 1,) * 4, order="F")
            axes = [np.arange(N + 1) / N] * 4
            pt = np.array([[*pos[q, :3].astype(np.float64), float(ts[q])]])
            ref = RegularGridInterpolator(axes, vol, method="linear")(pt)[0]
            assert enc[0, l] == pytest.approx(ref, abs=1e-12)
