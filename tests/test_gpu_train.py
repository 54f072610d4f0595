"""GPU parity of the training kernels (Sec. 4.5) against the FP64 oracle.

The oracle's gradient is itself pinned to central differences of Eq. 3 (with the
stop-gradient denominator frozen) in tests/test_oracle_network.py; here the
hand-written backward kernels (FP32, through the C ABI) must reproduce it.
"""
import numpy as np
import pytest

import oracle
from niv_inputs import init_params, uniform_queries
from niv_inputs.configs import MODEL_C0, ROOM_MIN, ROOM_MAX

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GRAD_BOUND = 1e-4  # max |g - g_ref| / max |g_ref| per parameter group (FP32 sums over the batch)


@pytest.fixture(scope="module")
def niv():
    from paper_2602_12949_gb300.build import build
    build()
    import paper_2602_12949_gb300 as P
    return P


def _groups(om):
    n_grid = oracle.grid_value_count(om)
    out, off = [("grid", 0, n_grid)], n_grid
    for li, (o, i) in enumerate(oracle.layer_shapes(om)):
        out.append(("W%d" % li, off, off + o * i))
        out.append(("b%d" % li, off + o * i, off + o * i + o))
        off += o * i + o
    return out


@pytest.mark.parametrize("spec,n,use_t", [
    (dict(MODEL_C0, log2_T=10), 4096 + 33, False),                           # hash collisions in the grid
    (dict(MODEL_C0, levels=4, feat=4, n_hidden=3, width=32), 2048, False),
    (dict(dims=4, levels=6, feat=2, log2_T=12, base=3.0, growth=1.6, n_hidden=3, width=64, in_extra=4), 3000, True),
    (dict(MODEL_C0, width=16, n_hidden=1), 1000, False),
])
def test_gradient_matches_oracle(niv, spec, n, use_t):
    m = niv.NIVModel(**spec)
    g, _ = m.param_count()
    params = init_params(g, m.layer_shapes(), seed=3, feat_range=0.3, bias_std=0.2)
    m.set_params(params)
    om = oracle.Model(**spec)
    pos, nrm = uniform_queries(n, seed=4)
    target = np.zeros((n, 4), np.float32)
    target[:, :3] = np.random.default_rng(5).uniform(0.1, 2.0, (n, 3))
    t = np.random.default_rng(6).random(n).astype(np.float32) if use_t else None
    dev = lambda a: torch.from_numpy(a).cuda()
    loss = m.grad(dev(pos), dev(nrm), dev(target), t=dev(t) if use_t else None)
    got = m.get_grads().astype(np.float64)
    ref_loss, ref = oracle.loss_grad(om, params, pos, nrm, target[:, :3], t=t)
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    for name, a, b in _groups(om):
        scale = np.abs(ref[a:b]).max()
        err = np.abs(got[a:b] - ref[a:b]).max() / scale
        print("%s: %.3g" % (name, err))
        assert err <= GRAD_BOUND, name
    m.close()


def test_adam_matches_oracle(niv):
    m = niv.NIVModel(**MODEL_C0)
    g, nm = m.param_count()
    params = init_params(g, m.layer_shapes(), seed=1)
    m.set_params(params)
    theta = params.astype(np.float64)
    mm, vv = np.zeros_like(theta), np.zeros_like(theta)
    rng = np.random.default_rng(2)
    for step in range(1, 4):
        grads = (rng.standard_normal(g + nm) * 10.0 ** rng.uniform(-4, 0, g + nm)).astype(np.float32)
        m.set_grads(grads)
        m.adam_step(lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-15)
        oracle.adam(theta, mm, vv, grads.astype(np.float64), 1e-2, 0.9, 0.99, 1e-15, step)
    got = m.get_params().astype(np.float64)
    np.testing.assert_allclose(got, theta, rtol=0, atol=2e-6)
    m.close()


def test_fit_reduces_loss_and_trained_model_queries_match_oracle(niv):
    """Fitting a smooth synthetic target lowers the loss; the refreshed inference copies follow."""
    spec = dict(MODEL_C0)
    m = niv.NIVModel(**spec)
    g, _ = m.param_count()
    m.set_params(init_params(g, m.layer_shapes(), seed=0))
    n = 1 << 15
    pos, nrm = uniform_queries(n, seed=9)
    tgt = np.zeros((n, 4), np.float32)
    p3, n3 = pos[:, :3].astype(np.float64), nrm[:, :3].astype(np.float64)
    tgt[:, 0] = 1.0 + 0.5 * np.sin(3 * p3[:, 0]) * n3[:, 1]
    tgt[:, 1] = 0.5 + 0.4 * p3[:, 1] * p3[:, 2]
    tgt[:, 2] = 0.8 + 0.3 * np.cos(2 * p3[:, 2] + n3[:, 0])
    dev = lambda a: torch.from_numpy(a).cuda()
    dp, dn, dt = dev(pos), dev(nrm), dev(tgt)
    first = m.fit(dp, dn, dt)
    for _ in range(300):
        last = m.fit(dp, dn, dt, want_loss=False)
    last = m.grad(dp, dn, dt)
    print("loss %.4g -> %.4g" % (first, last))
    assert last < 0.05 * first
    om = oracle.Model(**spec)
    trained = m.get_params()
    E = m.query(dp, dn, precision="fp32")[:, :3].cpu().numpy()
    ref = oracle.query(om, trained, pos, nrm)
    assert np.max(np.abs(E - ref) / np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())) <= 1e-5
    E16 = m.query(dp, dn, precision="fp16", out_dtype=torch.float32)[:, :3].cpu().numpy()
    ref16 = oracle.query(om, trained.astype(np.float16).astype(np.float64), pos, nrm)
    assert np.max(np.abs(E16 - ref16) / np.maximum(np.abs(ref16), 1e-3 * np.abs(ref16).max())) <= 2e-3
    m.close()


def _groups_max_err(om, got, ref):
    worst = 0.0
    for name, a, b in _groups(om):
        if b > a:
            scale = np.abs(ref[a:b]).max()
            if scale > 0:
                worst = max(worst, float(np.max(np.abs(got[a:b] - ref[a:b])) / scale))
    return worst


def test_autograd_with_eq3_in_torch_matches_oracle(niv):
    """NIVModule's backward (niv_backward) under Eq. 3 written in torch, with the stop-gradient
    denominator, gives the oracle's loss gradient."""
    spec = dict(MODEL_C0, log2_T=10)
    m = niv.NIVModel(**spec)
    g, _ = m.param_count()
    params = init_params(g, m.layer_shapes(), seed=3, feat_range=0.3, bias_std=0.2)
    om = oracle.Model(**spec)
    n = 3000
    pos, nrm = uniform_queries(n, seed=4)
    y = np.random.default_rng(5).uniform(0.1, 2.0, (n, 3))
    mod = niv.NIVModule(m, params)
    dp, dn = torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda()
    E = mod(dp, dn)[:, :3]
    yt = torch.from_numpy(y).float().cuda()
    loss = ((E - yt) ** 2 / (E.detach() ** 2 + 0.01)).mean()
    loss.backward()
    got = mod.params.grad.cpu().numpy().astype(np.float64)
    ref_loss, ref = oracle.loss_grad(om, params, pos, nrm, y)
    assert loss.item() == pytest.approx(ref_loss, rel=1e-5)
    err = _groups_max_err(om, got, ref)
    print("autograd Eq. 3: max group error %.2e" % err)
    assert err <= GRAD_BOUND
    m.close()


def test_autograd_linear_functional_matches_finite_differences(niv):
    """dL/dtheta for L = sum w . E with random w: autograd through niv_backward against central
    differences of the FP64 oracle's forward."""
    spec = dict(MODEL_C0, levels=3, log2_T=8, base=3.0, growth=1.6, n_hidden=2, width=16)
    m = niv.NIVModel(**spec)
    g, _ = m.param_count()
    params = init_params(g, m.layer_shapes(), seed=6, feat_range=0.5, bias_std=0.3).astype(np.float64)
    om = oracle.Model(**spec)
    n = 500
    pos, nrm = uniform_queries(n, seed=7)
    w = np.random.default_rng(8).standard_normal((n, 3))
    mod = niv.NIVModule(m, params)
    E = mod(torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda())[:, :3]
    (E * torch.from_numpy(w).float().cuda()).sum().backward()
    got = mod.params.grad.cpu().numpy().astype(np.float64)
    L = lambda p: float(np.sum(w * oracle.query(om, p, pos, nrm)))
    rng = np.random.default_rng(9)
    idx = np.concatenate([rng.choice(g, 30, replace=False), g + rng.choice(len(params) - g, 30, replace=False)])
    h = 1e-6
    fd = np.array([(L(params + h * np.eye(1, len(params), i)[0]) - L(params - h * np.eye(1, len(params), i)[0])) / (2 * h)
                   for i in idx])
    scale = np.abs(fd).max()
    err = np.max(np.abs(got[idx] - fd)) / scale
    print("autograd linear functional vs FD: %.2e of max |g| %.3g" % (err, scale))
    assert err <= 1e-4
    m.close()


def test_identity_output_gradient_matches_oracle(niv):
    spec = dict(MODEL_C0, log2_T=10, out_act=0)
    m = niv.NIVModel(**spec)
    g, _ = m.param_count()
    params = init_params(g, m.layer_shapes(), seed=10, feat_range=0.3, bias_std=0.2)
    m.set_params(params)
    om = oracle.Model(**spec)
    n = 2000
    pos, nrm = uniform_queries(n, seed=11)
    target = np.zeros((n, 4), np.float32)
    target[:, :3] = np.random.default_rng(12).uniform(-1.0, 1.0, (n, 3))
    dev = lambda a: torch.from_numpy(a).cuda()
    loss = m.grad(dev(pos), dev(nrm), dev(target))
    ref_loss, ref = oracle.loss_grad(om, params, pos, nrm, target[:, :3])
    assert loss == pytest.approx(ref_loss, rel=1e-5)
    assert _groups_max_err(om, m.get_grads().astype(np.float64), ref) <= GRAD_BOUND
    m.close()


FP16_FWD_GRAD_BOUND = 1e-3  # binary16 roundings decided from FP32 (GPU) and FP64 (oracle) sums may differ


@pytest.mark.parametrize("spec", [dict(MODEL_C0, log2_T=10), dict(MODEL_C0, levels=6, feat=4, n_hidden=3, width=32)])
def test_fp16_forward_gradient_matches_oracle(niv, spec):
    """Config 2's FP16 forward: the gradient (straight through the roundings, onto the FP32
    master parameters) matches the oracle's FP16 mode."""
    m = niv.NIVModel(**spec)
    g, _ = m.param_count()
    params = init_params(g, m.layer_shapes(), seed=13, feat_range=0.3, bias_std=0.2)
    m.set_params(params)
    m.set_train_forward("fp16")
    om = oracle.Model(**spec)
    n = 3000
    pos, nrm = uniform_queries(n, seed=14)
    target = np.zeros((n, 4), np.float32)
    target[:, :3] = np.random.default_rng(15).uniform(0.1, 2.0, (n, 3))
    dev = lambda a: torch.from_numpy(a).cuda()
    loss = m.grad(dev(pos), dev(nrm), dev(target))
    ref_loss, ref = oracle.loss_grad(om, oracle.f16(params), pos, nrm, target[:, :3], f16=True)
    _, ref32 = oracle.loss_grad(om, params, pos, nrm, target[:, :3])
    got = m.get_grads().astype(np.float64)
    err, err32 = _groups_max_err(om, got, ref), _groups_max_err(om, got, ref32)
    print("fp16 forward: loss %.6g vs %.6g; max group error %.2e (vs the FP32 gradient %.2e)"
          % (loss, ref_loss, err, err32))
    assert loss == pytest.approx(ref_loss, rel=1e-4)
    assert err <= FP16_FWD_GRAD_BOUND
    assert err < err32  # it is the FP16 function's gradient, not the FP32 one
    m.close()


def test_fp16_forward_fit_reduces_loss(niv):
    spec = dict(MODEL_C0, log2_T=12)
    m = niv.NIVModel(**spec)
    g, _ = m.param_count()
    m.set_params(init_params(g, m.layer_shapes(), seed=16))
    m.set_train_forward("fp16")
    n = 1 << 14
    pos, nrm = uniform_queries(n, seed=17)
    target = np.zeros((n, 4), np.float32)
    x = pos[:, :3].astype(np.float64)
    target[:, :3] = (0.5 + 0.4 * np.sin(4.0 * x) * (nrm[:, :3] * 0.5 + 0.5)).astype(np.float32)
    dev = lambda a: torch.from_numpy(a).cuda()
    dp, dn, dy = dev(pos), dev(nrm), dev(target)
    first = m.fit(dp, dn, dy)
    for _ in range(300):
        last = m.fit(dp, dn, dy, want_loss=False)
    last = m.fit(dp, dn, dy)
    assert last < 0.1 * first
    m.close()



def _trained(niv, steps, forward="fp32"):
    """A config-0 model after `steps` fit steps on a fixed batch (Eq. 3, Adam lr 1e-2)."""
    m = niv.NIVModel(**MODEL_C0)
    g, _ = m.param_count()
    m.set_params(init_params(g, m.layer_shapes(), seed=21, bias_std=0.1))
    m.set_train_forward(forward)
    pos, nrm = uniform_queries(4096, seed=22)
    tgt = np.zeros_like(pos)
    tgt[:, :3] = np.random.default_rng(23).uniform(0.1, 2.0, (len(pos), 3))
    batch = tuple(torch.from_numpy(a).cuda() for a in (pos, nrm, tgt))
    for _ in range(steps):
        m.fit(*batch, lr=1e-2, want_loss=False)
    return m, batch


def _same_update(models, n):
    """One Adam step from the same given gradient on every model (no atomic sums involved)."""
    grad = np.random.default_rng(24).normal(0.0, 1e-2, n).astype(np.float32)
    for model in models:
        model.set_grads(grad)
        model.adam_step(lr=1e-2)


def test_checkpoint_resumes_the_optimisation(niv, tmp_path):
    """A model file carries the Adam moments, the step count and the training forward, so that
    training resumes where it stopped.  After 5 fit steps, save and load: the parameters match
    bit for bit, and one Adam update from the same given gradient gives bit-identical parameters
    on the saved and on the loaded model (the step count enters the bias correction, the moments
    the update itself).  Further fit steps from the same batch stay as close to the uninterrupted
    run as a repeat of the uninterrupted run (grid gradients are summed with atomics, whose order
    varies from run to run)."""
    m, batch = _trained(niv, 5, forward="fp16")
    path = tmp_path / "ckpt.niv"
    m.save(path)
    m2 = niv.NIVModel.load(path)
    np.testing.assert_array_equal(m2.get_params(), m.get_params())
    _same_update([m, m2], m.get_params().size)
    np.testing.assert_array_equal(m2.get_params(), m.get_params())
    # a fresh optimisation from the same parameters (what a parameters-only file gives) differs
    fresh = niv.NIVModel(**MODEL_C0)
    m.save(path)
    m3 = niv.NIVModel.load(path)
    fresh.set_params(m3.get_params())
    fresh.set_train_forward("fp16")
    _same_update([m3, fresh], m.get_params().size)
    assert not np.array_equal(fresh.get_params(), m3.get_params())
    # k more fit steps: resumed against uninterrupted, within the run-to-run spread
    for model in (m, m2):
        for _ in range(5):
            model.fit(*batch, lr=1e-2, want_loss=False)
    rerun, rbatch = _trained(niv, 5, forward="fp16")
    rerun2, _ = _trained(niv, 5, forward="fp16")
    spread = np.abs(rerun.get_params() - rerun2.get_params()).max()
    diff = np.abs(m2.get_params() - m.get_params()).max()
    print("resume: max |resumed - uninterrupted| %.3g, run-to-run spread after 5 steps %.3g" % (diff, spread))
    assert diff <= max(10 * spread, 1e-6)
    for model in (m, m2, m3, fresh, rerun, rerun2):
        model.close()
