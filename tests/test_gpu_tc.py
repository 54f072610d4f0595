"""GPU parity of the fused tensor-core query (FP16) against the FP64 oracle, through the C ABI.

The FP16 path stores grid features, weights and biases in FP16 (Table 1: all
parameters in half precision), accumulates in FP32 and rounds hidden activations
to FP16 between layers.  The
parity bound (2e-3 max relative error) is taken against the oracle evaluated on
the same FP16-rounded parameters, so it measures the kernel's arithmetic; the
error against the unrounded FP32 parameters is reported beside it.
"""
import ctypes

import numpy as np
import pytest

import oracle
from niv_inputs import init_params, uniform_queries
from niv_inputs.configs import MODEL_C0, MODEL_C1, MODEL_C3, MODEL_P, ROOM_MIN, ROOM_MAX, room_gbuffer

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

FP16_BOUND = 2e-3


def rel_err(got, ref):
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
    return float(np.max(np.abs(got - ref) / den))


def fp16_stored_params(params, om):
    """The parameters as the FP16 path stores them: every value rounded to FP16."""
    return params.astype(np.float16).astype(np.float64)


@pytest.fixture(scope="module")
def niv():
    from paper_2602_12949_gb300.build import build
    build()
    import paper_2602_12949_gb300 as P
    return P


def make(P, spec, seed=0, bias_std=0.0):
    m = P.NIVModel(**spec)
    g, _ = m.param_count()
    params = init_params(g, m.layer_shapes(), seed=seed, bias_std=bias_std)
    m.set_params(params)
    return m, params, oracle.Model(**spec)


def test_tensor_core_layout_selftest(niv):
    """One tcgen05 product of small integers is exact with the canonical descriptor strides."""
    from paper_2602_12949_gb300 import lib, sync_status
    m_ = np.arange(128)[:, None]
    n_ = np.arange(64)[:, None]
    k_ = np.arange(32)[None, :]
    A = (m_ * 3 + k_ * 5) % 7 - 3
    B = (n_ * 5 + k_ * 3) % 5 - 2
    ref = (A @ B.T).astype(np.float32)
    out = torch.zeros((128, 64), dtype=torch.float32, device="cuda")
    res = {}
    for swap in (0, 1):
        out.zero_()
        assert lib().niv_selftest_mma(swap, ctypes.c_void_p(out.data_ptr()),
                                      ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)) == 0
        sync_status()
        res[swap] = float(np.max(np.abs(out.cpu().numpy() - ref)))
    print("selftest max error: canonical %g, swapped %g" % (res[0], res[1]))
    assert res[0] == 0.0


def _check(m, params, om, pos, nrm, kw, bound=FP16_BOUND, **qkw):
    ref_q = oracle.query(om, fp16_stored_params(params, om), pos.astype(np.float32), nrm.astype(np.float32), **kw)
    ref = oracle.query(om, params, pos.astype(np.float32), nrm.astype(np.float32), **kw)
    dp, dn = torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda()
    E = m.query(dp, dn, precision="fp16", out_dtype=torch.float32, **{**kw, **qkw})
    got = E[:, :3].cpu().numpy()
    e_q, e = rel_err(got, ref_q), rel_err(got, ref)
    print("fp16: max rel err %.3g vs FP16-stored params, %.3g vs FP32 params" % (e_q, e))
    assert e_q <= bound
    assert e <= 10 * bound
    return E


def test_fp16_config0_full(niv):
    m, params, om = make(niv, MODEL_C0, seed=0)
    pos, nrm = uniform_queries(65536, seed=0)
    _check(m, params, om, pos, nrm, {})
    m.close()


@pytest.mark.parametrize("n", [1, 100, 128, 129, 4096 + 77])
def test_fp16_ragged_sizes_and_biases(niv, n):
    m, params, om = make(niv, MODEL_C0, seed=4, bias_std=0.2)
    pos, nrm = uniform_queries(n, seed=n + 1)
    _check(m, params, om, pos, nrm, {})
    m.close()


@pytest.mark.parametrize("spec,kw", [
    (dict(MODEL_C0, width=16), {}),
    (dict(MODEL_C0, width=32, n_hidden=1), {}),
    (dict(MODEL_C0, n_hidden=4), {}),
    (MODEL_P, dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)),
    (MODEL_C3, dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, t=0.71)),
    (dict(MODEL_C0, feat=1, levels=16), {}),
    # 16-level models beside the compiled shapes: 3 dense levels, 4 hidden layers, width 32
    (dict(MODEL_C1, log2_T=15), dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)),
    (dict(MODEL_C1, n_hidden=4), dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)),
    (dict(MODEL_C1, width=32), dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)),
    (dict(MODEL_C3, log2_T=17), dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, t=0.3)),
])
def test_fp16_other_shapes(niv, spec, kw):
    m, params, om = make(niv, spec, seed=9, bias_std=0.1)
    lo, hi = kw.get("aabb_min", (0, 0, 0)), kw.get("aabb_max", (1, 1, 1))
    pos, nrm = uniform_queries(5000, seed=3, lo=lo, hi=hi)
    _check(m, params, om, pos, nrm, kw)
    m.close()


@pytest.mark.parametrize("W,H", [(1920, 1080), (3840, 2160)])
def test_fp16_full_frame_sampled(niv, W, H):
    """Config 1 at full size (1080p and 4K) in the benchmark's launch configuration, 8192 sampled
    pixels checked."""
    pos, nrm, _ = room_gbuffer(W, H)
    m, params, om = make(niv, MODEL_C1, seed=0)
    dp, dn = torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda()
    kw = dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)
    E = m.query(dp, dn, precision="fp16", image_width=W, **kw)
    E_lin = m.query(dp, dn, precision="fp16", **kw)
    assert torch.equal(E, E_lin)
    pick = np.random.default_rng(0).choice(len(pos), 8192, replace=False)
    ref_q = oracle.query(om, fp16_stored_params(params, om), pos[pick].astype(np.float32),
                         nrm[pick].astype(np.float32), **kw)
    got = E[pick, :3].float().cpu().numpy()
    # FP16 output records add one final rounding (2^-11 relative)
    assert rel_err(got, ref_q) <= FP16_BOUND + 2.0 ** -11
    assert torch.all(torch.isfinite(E))
    m.close()


def test_fp16_config3_4k_frame_sampled(niv):
    """The 4-D config-3 model in FP16 on the full 4K room frame, as the benchmark runs it beside
    the E4M3 form; 8192 sampled pixels checked."""
    pos, nrm, _ = room_gbuffer(3840, 2160)
    m, params, om = make(niv, MODEL_C3, seed=0)
    dp, dn = torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda()
    kw = dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, t=0.6369616873214543)
    E = m.query(dp, dn, precision="fp16", image_width=3840, out_dtype=torch.float32, **kw)
    pick = np.random.default_rng(1).choice(len(pos), 8192, replace=False)
    ref_q = oracle.query(om, fp16_stored_params(params, om), pos[pick].astype(np.float32),
                         nrm[pick].astype(np.float32), **kw)
    assert rel_err(E[pick, :3].cpu().numpy(), ref_q) <= FP16_BOUND
    m.close()
