"""Training driver (Sec. 4.5): Monte Carlo targets -> culling -> Adam steps.

Orchestration only: every numeric step runs in libniv's kernels (Monte Carlo
irradiance, compaction of kept samples, forward/backward, Adam).  The candidate
points come from niv_inputs.samples (the paper's sampling: uniform in the volume
with uniform directions, 20% on surfaces with the surface normal).
"""
import time

import numpy as np
import torch

from .model import mc_irradiance, compact_targets


def train(model, scene, steps, batch, pool=1 << 18, spp=256, reuse=4, seed=0, lr=1e-2, beta1=0.9, beta2=0.99,
          adam_eps=1e-15, loss_eps=0.01, with_t=False, aabb_min=(-5.0, -5.0, -5.0), aabb_max=(5.0, 5.0, 5.0),
          log_every=0, device="cuda"):
    """Train `model` on indirect irradiance of `scene` for `steps` Adam steps.

    A fresh pool of `pool` candidates gets Monte Carlo targets (`spp` paths each);
    the kept samples are cut into batches of `batch`, and each pool serves `reuse`
    passes.  Returns a dict with the loss history and the time spent per phase.
    """
    from niv_inputs.samples import training_pool
    blob = scene.blob()
    hist, t_mc, t_fit = [], 0.0, 0.0
    step, pool_id, index_base = 0, 0, 0
    while step < steps:
        x4, n4, t = training_pool(scene, pool, seed=seed * 1000003 + pool_id, with_t=with_t)
        dx, dn = torch.from_numpy(x4).to(device), torch.from_numpy(n4).to(device)
        dt = torch.from_numpy(t).to(device) if t is not None else None
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        E, keep = mc_irradiance(blob, dx, dn, spp, seed=seed, mode="indirect", t=dt, index_base=index_base)
        kx, kn, ky, kt = compact_targets(dx, dn, E, keep, t=dt)
        torch.cuda.synchronize()
        t_mc += time.perf_counter() - t0
        index_base += pool
        pool_id += 1
        k = kx.shape[0]
        if k < batch:
            continue
        t0 = time.perf_counter()
        for _ in range(reuse):
            for b0 in range(0, k - batch + 1, batch):
                if step >= steps:
                    break
                want = log_every and (step % log_every == 0 or step == steps - 1)
                sl = slice(b0, b0 + batch)
                loss = model.fit(kx[sl], kn[sl], ky[sl], t=kt[sl] if kt is not None else None, aabb_min=aabb_min,
                                 aabb_max=aabb_max, lr=lr, beta1=beta1, beta2=beta2, adam_eps=adam_eps,
                                 loss_eps=loss_eps, want_loss=bool(want))
                if want:
                    hist.append((step, loss))
                step += 1
        torch.cuda.synchronize()
        t_fit += time.perf_counter() - t0
    return {"loss": hist, "seconds_mc": t_mc, "seconds_fit": t_fit, "pools": pool_id}


def held_out(scene, n, spp, seed, with_t=False, device="cuda"):
    """Evaluation samples (kept after culling) and their Monte Carlo reference E (float64, [k][3])."""
    from niv_inputs.samples import training_pool
    x4, n4, t = training_pool(scene, n, seed=seed, with_t=with_t)
    dx, dn = torch.from_numpy(x4).to(device), torch.from_numpy(n4).to(device)
    dt = torch.from_numpy(t).to(device) if t is not None else None
    E, keep = mc_irradiance(scene.blob(), dx, dn, spp, seed=seed + 77, mode="indirect", t=dt, index_base=1 << 40)
    keep_b = keep.bool()
    return dx[keep_b].contiguous(), dn[keep_b].contiguous(), E[keep_b], (dt[keep_b] if dt is not None else None)


def errors(pred, ref):
    """(MSE, relative MSE of Eq. 3's form with eps 0.01) over samples and channels."""
    p = pred[:, :3].double()
    r = ref.double()
    mse = torch.mean((p - r) ** 2).item()
    rel = torch.mean((p - r) ** 2 / (r * r + 0.01)).item()
    return mse, rel
