"""GPU parity of the query path (through the C ABI) against the FP64 oracle."""
import numpy as np
import pytest

import oracle
from niv_inputs import init_params, uniform_queries
from niv_inputs.configs import MODEL_C0, MODEL_C1, MODEL_C3, MODEL_PE16, ROOM_MIN, ROOM_MAX, room_gbuffer

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def rel_err(got, ref):
    """max |got - ref| / max(|ref|, 1e-3 max|ref|) -- relative error guarded near zero."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    return float(np.max(np.abs(got - ref) / den))


@pytest.fixture(scope="module")
def niv():
    from paper_2602_12949_gb300.build import build
    build()
    import paper_2602_12949_gb300 as P
    assert torch.cuda.is_available()
    return P


def make(P, spec, seed=0, bias_std=0.0):
    m = P.NIVModel(**spec)
    g, _ = m.param_count()
    params = init_params(g, m.layer_shapes(), seed=seed, bias_std=bias_std)
    m.set_params(params)
    return m, params, oracle.Model(**spec)


def test_param_layout_matches_oracle(niv):
    for spec in (MODEL_C0, MODEL_C1, MODEL_C3):
        m = niv.NIVModel(**spec)
        om = oracle.Model(**spec)
        L = oracle.layout(om)
        g, n_mlp = m.param_count()
        assert g == L["total"] * om.feat and n_mlp == oracle.mlp_param_count(om)
        for l in range(om.levels):
            info = m.level_info(l)
            assert (info["res"], info["dense"], info["first_entry"], info["entries"]) == (
                L["res"][l], L["dense"][l], L["offset"][l], L["entries"][l])
        m.close()


def test_set_get_params_roundtrip(niv):
    m, params, _ = make(niv, MODEL_C0, seed=3)
    np.testing.assert_array_equal(m.get_params(), params)
    m.set_params(torch.from_numpy(params * 2).cuda())
    np.testing.assert_array_equal(m.get_params(), params * 2)
    m.close()


@pytest.mark.parametrize("spec,n,kw", [
    (MODEL_C0, 65536, {}),
    (MODEL_C1, 4096 + 61, dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)),
    (MODEL_C3, 4096 + 5, dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, t=0.37)),
])
def test_corner_indices_bit_exact(niv, spec, n, kw):
    m, params, om = make(niv, spec, seed=1)
    lo, hi = kw.get("aabb_min", (0, 0, 0)), kw.get("aabb_max", (1, 1, 1))
    pos, _ = uniform_queries(n, seed=2, lo=lo, hi=hi)
    enc, idx = m.encode(torch.from_numpy(pos).cuda(), **kw)
    ref_enc, ref_idx, _ = oracle.encode(om, params, pos, lo, hi, kw.get("t", 0.0), want_corners=True)
    np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), ref_idx)
    np.testing.assert_allclose(enc.cpu().numpy(), ref_enc, rtol=0, atol=2e-8)
    m.close()


def test_fp32_query_config0_full(niv):
    """Config 0: 65,536 FP32 queries, the plain path within 1e-5 max relative error of the FP64 oracle."""
    m, params, om = make(niv, MODEL_C0, seed=0)
    pos, nrm = uniform_queries(65536, seed=0)
    ref = oracle.query(om, params, pos, nrm)
    E = m.query(torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda(), precision="fp32")
    assert rel_err(E[:, :3].cpu().numpy(), ref) <= 1e-5
    assert torch.all(E[:, 3] == 0)
    m.close()


@pytest.mark.parametrize("n", [1, 127, 128, 129, 1000, 65536 + 77])
def test_fp32_ragged_sizes_and_biases(niv, n):
    m, params, om = make(niv, MODEL_C0, seed=5, bias_std=0.3)
    pos, nrm = uniform_queries(n, seed=n)
    ref = oracle.query(om, params, pos, nrm)
    E = m.query(torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda(), precision="fp32")
    assert rel_err(E[:, :3].cpu().numpy(), ref) <= 1e-5
    m.close()


@pytest.mark.parametrize("spec", [dict(MODEL_C0, width=16), dict(MODEL_C0, width=32, n_hidden=1),
                                  dict(MODEL_C0, feat=4, levels=4, n_hidden=4), dict(MODEL_C3, levels=6),
                                  dict(MODEL_C0, feat=1, out_act=0)])
def test_fp32_other_shapes(niv, spec):
    m, params, om = make(niv, spec, seed=7, bias_std=0.1)
    pos, nrm = uniform_queries(3000, seed=1)
    ref = oracle.query(om, params, pos, nrm, t=0.6)
    E = m.query(torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda(), precision="fp32", t=0.6)
    got = E[:, :3].cpu().numpy()
    if spec.get("out_act", 1) == 1:
        assert rel_err(got, ref) <= 1e-5
    else:  # signed outputs cross zero: error relative to the output scale
        assert np.max(np.abs(got - ref)) / np.abs(ref).max() <= 1e-5
    m.close()


def test_empty_query_is_noop(niv):
    m, _, _ = make(niv, MODEL_C0)
    z = torch.zeros((0, 4), device="cuda")
    m.query(z, z, precision="fp32")
    m.close()


def test_misaligned_pointer_rejected(niv):
    m, _, _ = make(niv, MODEL_C0)
    buf = torch.zeros(4 * 129, device="cuda")
    bad = buf[1:1 + 4 * 128].view(128, 4)
    with pytest.raises(niv.NivError) as e:
        m.query(bad, bad, precision="fp32")
    assert e.value.code == -2
    m.close()


@pytest.fixture(scope="module")
def gbuf1080():
    return room_gbuffer(1920, 1080)


def test_fp32_full_frame_1080p_sampled(niv, gbuf1080):
    """Config-1 model on the full 1080p FP16 G-buffer, image traversal; 8192 sampled pixels vs the oracle."""
    pos, nrm, _ = gbuf1080
    m, params, om = make(niv, MODEL_C1, seed=0)
    dpos, dnrm = torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda()
    E = m.query(dpos, dnrm, precision="fp32", aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, image_width=1920,
                out_dtype=torch.float32)
    E_lin = m.query(dpos, dnrm, precision="fp32", aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, out_dtype=torch.float32)
    assert torch.equal(E, E_lin)  # tile traversal changes nothing
    pick = np.random.default_rng(0).choice(len(pos), 8192, replace=False)
    ref = oracle.query(om, params, pos[pick].astype(np.float32), nrm[pick].astype(np.float32), ROOM_MIN, ROOM_MAX)
    assert rel_err(E[pick, :3].cpu().numpy(), ref) <= 1e-5
    m.close()


def test_query_host_matches_device_query(niv):
    m, params, om = make(niv, MODEL_C0, seed=2)
    pos, nrm = uniform_queries(10000, seed=3)
    dev = m.query(torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda(), precision="fp32").cpu().numpy()
    host = m.query_host(pos, nrm, precision="fp32")
    np.testing.assert_array_equal(host, dev)
    m.close()


@pytest.mark.parametrize("width,rows,n_extra,precision,rec", [(1000, 537, 0, "fp16", np.float16),
                                                              (0, 0, 300001, "fp32", np.float32),
                                                              (1920, 1080, 0, "fp16", np.float32)])
def test_chunked_host_query_matches_device_query(niv, width, rows, n_extra, precision, rec):
    # large calls are split into chunks of whole bands of tile rows (or 128-record tiles) whose
    # copies overlap the queries of their neighbours: the result must not change by a bit
    m, params, om = make(niv, MODEL_C1, seed=4)
    n = width * rows + n_extra
    pos, nrm = uniform_queries(n, seed=5)
    pos, nrm = pos.astype(rec), nrm.astype(rec)
    kw = dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, image_width=width)
    out_dt = torch.float16 if rec == np.float16 else torch.float32
    dev = m.query(torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda(), precision=precision, out_dtype=out_dt,
                  **kw).cpu().numpy()
    host = m.query_host(pos, nrm, precision=precision, **kw)
    np.testing.assert_array_equal(host, dev)
    m.close()


@pytest.mark.parametrize("mode,rec", [("0", np.float16), ("1", np.float16), ("0", np.float32)])
def test_pinned_host_query_follows_buffer_contents_and_arguments(niv, mode, rec, monkeypatch):
    # page-locked buffers: mode 0 lets one query read and write host memory directly; mode 1
    # stages them through device memory in overlapped chunks.  Each call must read the
    # buffers' current contents, and new arguments (another output buffer, new parameters,
    # another precision) must take effect.
    monkeypatch.setenv("NIV_HOST_MODE", mode)
    m, params, om = make(niv, MODEL_C1, seed=6)
    W, H = 640, 360
    n = W * H
    pos, nrm = uniform_queries(n, seed=7)
    tdt = torch.float16 if rec == np.float16 else torch.float32
    hp = torch.from_numpy(pos.astype(rec)).pin_memory()
    hn = torch.from_numpy(nrm.astype(rec)).pin_memory()
    ho = torch.empty((n, 4), dtype=tdt).pin_memory()
    kw = dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, image_width=W)

    def device(**extra):
        return m.query(hp.cuda(), hn.cuda(), precision="fp16", out_dtype=tdt, **dict(kw, **extra)).cpu()

    for call in range(5):
        if call == 3:  # new contents in the same buffers
            hp.copy_(torch.from_numpy(uniform_queries(n, seed=8)[0].astype(rec)))
        m.query_host(hp.numpy(), hn.numpy(), out=ho.numpy(), precision="fp16", **kw)
        assert torch.equal(ho, device()), call
    ho2 = torch.empty_like(ho).pin_memory()
    m.query_host(hp.numpy(), hn.numpy(), out=ho2.numpy(), precision="fp16", **kw)
    assert torch.equal(ho2, device())
    g, _ = m.param_count()
    m.set_params(init_params(g, m.layer_shapes(), seed=9))
    for call in range(3):
        m.query_host(hp.numpy(), hn.numpy(), out=ho.numpy(), precision="fp16", **kw)
        assert torch.equal(ho, device()), call
    m.query_host(hp.numpy(), hn.numpy(), out=ho.numpy(), precision="fp32", **kw)
    assert torch.equal(ho, m.query(hp.cuda(), hn.cuda(), precision="fp32", out_dtype=tdt, **kw).cpu())
    m.close()


def test_save_and_load_round_trip(niv, tmp_path):
    # the file keeps the description and the FP32 master parameters bit for bit; a model
    # loaded from it answers queries exactly as the saved one
    for spec in (MODEL_C1, MODEL_C3, MODEL_PE16):
        m, params, om = make(niv, spec, seed=11, bias_std=0.1)
        path = tmp_path / "model.niv"
        m.save(path)
        m2 = niv.NIVModel.load(path)
        assert m2.param_count() == m.param_count()
        np.testing.assert_array_equal(m2.get_params(), m.get_params())
        pos, nrm = uniform_queries(4096 + 5, seed=12)
        dp, dn = torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda()
        for prec in ("fp32", "fp16"):
            assert torch.equal(m2.query(dp, dn, precision=prec, t=0.3), m.query(dp, dn, precision=prec, t=0.3))
        m.close()
        m2.close()


def test_shade_matches_oracle(niv):
    rng = np.random.default_rng(0)
    n = 100000 + 3
    alb = rng.uniform(0.1, 0.9, (n, 4)).astype(np.float16)
    E = rng.uniform(0.0, 4.0, (n, 4)).astype(np.float16)
    D = rng.uniform(0.0, 2.0, (n, 4)).astype(np.float16)
    out = niv.shade(*(torch.from_numpy(a).cuda() for a in (alb, D, E))).cpu().numpy()
    ref = oracle.shade(alb[:, :3].astype(np.float64), E[:, :3].astype(np.float64), D[:, :3].astype(np.float64))
    # one FP16 rounding of the result: half an ulp, 2^-11 relative
    np.testing.assert_allclose(out[:, :3].astype(np.float64), ref, rtol=2.0 ** -11, atol=1e-7)
    assert np.all(out[:, 3] == 1.0)


def test_fp16_query_before_parameters_are_set_is_refused(niv):
    """A model straight from niv_create has no packed network: the tensor-core query returns
    NIV_ERR_ARG on the host and launches nothing; the FP32 path runs on the zero network."""
    m = niv.NIVModel(**MODEL_C0)
    pos, nrm = uniform_queries(1000, seed=5)
    dpos, dnrm = torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda()
    with pytest.raises(niv.NivError) as ei:
        m.query(dpos, dnrm, precision="fp16", out_dtype=torch.float32)
    assert ei.value.code == -1 and "parameters not set" in str(ei.value)
    E = m.query(dpos, dnrm, precision="fp32", out_dtype=torch.float32)
    niv.sync_status()
    np.testing.assert_allclose(E[:, :3].cpu().numpy(), np.log(2.0), rtol=1e-6)  # softplus(0)
    m.close()


def _boundary_points(lo, hi, n_levels_res, seed=0):
    """Positions on the box's faces and corners, outside it (clamped to the box), and exactly on
    grid vertices of every level (s = u N integral), plus random points."""
    rng = np.random.default_rng(seed)
    lo, hi = np.asarray(lo, np.float64), np.asarray(hi, np.float64)
    pts = []
    for cx in (0.0, 1.0):
        for cy in (0.0, 1.0):
            for cz in (0.0, 1.0):
                pts.append([cx, cy, cz])
    for axis in range(3):
        for side in (0.0, 1.0):
            p = rng.random((64, 3))
            p[:, axis] = side
            pts.extend(p.tolist())
    p = rng.uniform(-0.5, 1.5, (256, 3))  # outside the box on some axes
    pts.extend(p.tolist())
    for N in n_levels_res:  # on vertices of level N: u = i / N (exact only where i / N is)
        i = rng.integers(0, N + 1, (32, 3))
        pts.extend((i / N).tolist())
    u = np.asarray(pts)
    pos = np.zeros((len(u), 4), np.float32)
    pos[:, :3] = lo + (hi - lo) * u
    return pos


@pytest.mark.parametrize("spec,kw", [
    (MODEL_C0, {}),
    (MODEL_C1, dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)),
    (MODEL_C3, dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, t=1.0)),
])
def test_degenerate_positions(niv, spec, kw):
    """The cases where the cell search clamps or lands on a vertex: points on the box's faces and
    corners (u = 0 or 1, so s = N at the far face and the cell index is clamped to N - 1),
    outside the box (u clamped), on grid vertices, t at its end: corner indices bit-exact, the
    FP32 query within 1e-5 and the FP16 query within 2e-3 of the oracle."""
    m, params, om = make(niv, spec, seed=4, bias_std=0.1)
    lo, hi = kw.get("aabb_min", (0, 0, 0)), kw.get("aabb_max", (1, 1, 1))
    res = [m.level_info(l)["res"] for l in range(om.levels)]
    pos = _boundary_points(lo, hi, res[:6])
    nrm = np.zeros_like(pos)
    nrm[:, :3] = np.random.default_rng(1).normal(size=(len(pos), 3))
    nrm[:, :3] /= np.linalg.norm(nrm[:, :3], axis=1, keepdims=True)
    dp, dn = torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda()
    enc, idx = m.encode(dp, **kw)
    _, ref_idx, _ = oracle.encode(om, params, pos, lo, hi, kw.get("t", 0.0), want_corners=True)
    np.testing.assert_array_equal(idx.cpu().numpy().view(np.uint32), ref_idx)
    ref = oracle.query(om, params, pos, nrm, **kw)
    e32 = m.query(dp, dn, precision="fp32", out_dtype=torch.float32, **kw)[:, :3].cpu().numpy()
    assert rel_err(e32, ref) <= 1e-5
    ref16 = oracle.query(om, oracle_fp16_params(params, om), pos, nrm, **kw)
    e16 = m.query(dp, dn, precision="fp16", out_dtype=torch.float32, **kw)[:, :3].cpu().numpy()
    assert rel_err(e16, ref16) <= 2e-3
    m.close()


def oracle_fp16_params(params, om):
    """The parameters as the FP16 path stores them (grid values, weights and biases in binary16)."""
    return np.asarray(params, np.float32).astype(np.float16).astype(np.float64)
