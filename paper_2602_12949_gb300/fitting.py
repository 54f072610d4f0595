"""Training driver (Sec. 4.5): Monte Carlo targets -> culling -> Adam steps.

Orchestration only: every numeric step runs in libniv's kernels (candidate points,
Monte Carlo irradiance, compaction of kept samples, forward/backward, Adam).  The
candidates follow the paper's sampling (niv_training_samples: uniform in the volume
with uniform directions, 20% on surfaces with the surface normal, by area).
"""
import time

import numpy as np
import torch

from .model import mc_irradiance, compact_targets, training_samples

# Counter ranges of the sample streams: training pools take [0, 2^40), held-out sets start at 2^40.
HELD_OUT_BASE = 1 << 40


def train(model, scene, steps, batch, pool=1 << 18, spp=256, reuse=4, seed=0, lr=1e-2, beta1=0.9, beta2=0.99,
          adam_eps=1e-15, loss_eps=0.01, with_t=False, aabb_min=(-5.0, -5.0, -5.0), aabb_max=(5.0, 5.0, 5.0),
          log_every=0, forward="fp32", device="cuda"):
    """Train `model` on indirect irradiance of `scene` for `steps` Adam steps.

    A fresh pool of `pool` candidates gets Monte Carlo targets (`spp` paths each);
    the kept samples are cut into batches of `batch`, and each pool serves `reuse`
    passes.  forward: "fp16" runs the FP16 path of the query in the forward (config 2), "fp32"
    the FP32 one.  Returns a dict with the loss history and the time spent per phase.
    """
    model.set_train_forward(forward)
    blob = scene.blob()
    hist, t_mc, t_fit = [], 0.0, 0.0
    step, pool_id, index_base = 0, 0, 0
    while step < steps:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        dx, dn, dt, _ = training_samples(blob, pool, seed=seed, index_base=pool_id * pool, with_t=with_t,
                                         device=device)
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


def held_out(scene, n, spp, seed, with_t=False, t_levels=0, device="cuda"):
    """Evaluation samples (kept after culling) and their Monte Carlo reference E (float64, [k][3]).
    t_levels > 0: sample i takes t = ((i mod t_levels) + 1/2) / t_levels instead of a uniform t."""
    dx, dn, dt, _ = training_samples(scene.blob(), n, seed=seed, index_base=HELD_OUT_BASE, with_t=with_t,
                                     device=device)
    if with_t and t_levels > 0:
        t = ((np.arange(n) % t_levels + 0.5) / t_levels).astype(np.float32)
        dt = torch.from_numpy(t).to(device)
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


def memory_error_sweep(scene, log2_Ts, shape, init_params, steps=2000, batch=1 << 16, pool=1 << 18, spp=128,
                       reuse=2, held=(1 << 14, 4096), probe_rays=1024, seed=1, aabb_min=(-5.0, -5.0, -5.0),
                       aabb_max=(5.0, 5.0, 5.0), device="cuda"):
    """Memory-error trade-off (Sec. 4.1's hash-table-size study and Sec. 5.1's comparison with
    probes): for every hash table size 2^log2_T, NIV of the given shape is trained on `scene`,
    and the SH probe grid with the largest cubic lattice that fits the same memory is baked;
    the probes are queried with the cosine fall-off and with ray-traced visibility ("+ RT").
    Returns one row per size with the FP16 memory and the (MSE, relative MSE) of each on the
    same held-out samples (Monte Carlo references at held[1] spp).  init_params(n_grid, layer_shapes,
    seed) gives each model's initial flat parameter vector."""
    import torch
    from .model import NIVModel, ProbeGrid
    hx, hn, hE, _ = held_out(scene, held[0], held[1], seed=99, device=device)
    rows = []
    for lt in log2_Ts:
        m = NIVModel(**dict(shape, log2_T=int(lt)))
        g, nm = m.param_count()
        nbytes = 2 * (g + nm)  # FP16 parameters
        m.set_params(init_params(g, m.layer_shapes(), seed=0))
        train(m, scene, steps=steps, batch=batch, pool=pool, spp=spp, reuse=reuse, seed=seed, aabb_min=aabb_min,
              aabb_max=aabb_max, device=device)
        niv = errors(m.query(hx, hn, precision="fp16", out_dtype=torch.float32, aabb_min=aabb_min,
                             aabb_max=aabb_max), hE)
        m.close()
        P = int((nbytes / 54.0) ** (1.0 / 3.0))
        while (P + 1) ** 3 * 54 <= nbytes:
            P += 1
        while P ** 3 * 54 > nbytes:
            P -= 1
        grid = ProbeGrid((P,) * 3, aabb_min, aabb_max, device=device)
        grid.bake(scene.blob(), rays=probe_rays, seed=3)
        probe = errors(grid.query(hx, hn, out_dtype=torch.float32), hE)
        probe_rt = errors(grid.query(hx, hn, out_dtype=torch.float32, scene_blob=scene.blob()), hE)
        rows.append({"log2_T": int(lt), "mb": nbytes / 1e6, "niv_mse": niv[0], "niv_rel": niv[1],
                     "probes_per_axis": P, "probe_mb": grid.nbytes / 1e6, "probe_mse": probe[0],
                     "probe_rel": probe[1], "probe_rt_mse": probe_rt[0], "probe_rt_rel": probe_rt[1]})
    return rows


def time_field_comparison(scene, shapes, init_params, steps=2000, batch=1 << 16, pool=1 << 18, spp=128, reuse=2,
                          held=(1 << 14, 4096), seed=1, aabb_min=(-5.0, -5.0, -5.0), aabb_max=(5.0, 5.0, 5.0),
                          frame=None, device="cuda"):
    """Fields that change with a scene parameter t (Sec. 6; config 3): every model in `shapes`
    (name -> NIVModel keyword arguments) is trained on samples with a uniform per-sample t of
    `scene` (its rotating emitter moves with t) and scored on the same held-out (x, n, t)
    samples.  frame (optional (pos, nrm, width) device records): the FP16 query time of each
    model on it at t = 0.5.  init_params(n_grid, layer_shapes, seed) gives each model's initial flat
    parameter vector.  Returns one row per model: FP16 memory, MSE, relative MSE, ms."""
    import torch
    from .model import NIVModel
    hx, hn, hE, ht = held_out(scene, held[0], held[1], seed=199, with_t=True, t_levels=16, device=device)
    rows = []
    for name, shape in shapes.items():
        m = NIVModel(**shape)
        g, nm = m.param_count()
        m.set_params(init_params(g, m.layer_shapes(), seed=0))
        train(m, scene, steps=steps, batch=batch, pool=pool, spp=spp, reuse=reuse, seed=seed, with_t=True,
              aabb_min=aabb_min, aabb_max=aabb_max, device=device)
        E = torch.empty((hx.shape[0], 4), dtype=torch.float32, device=hx.device)
        # the query takes one t per call: evaluate the held-out samples grouped by their 16 t values
        order = torch.argsort(ht)
        hts = ht[order].cpu().numpy()
        for t in np.unique(hts):
            sel = order[torch.from_numpy(np.nonzero(hts == t)[0]).to(hx.device)]
            E[sel] = m.query(hx[sel].contiguous(), hn[sel].contiguous(), precision="fp16", out_dtype=torch.float32,
                             aabb_min=aabb_min, aabb_max=aabb_max, t=float(t))
        mse, rel = errors(E, hE)
        row = {"model": name, "mb": 2 * (g + nm) / 1e6, "mse": mse, "rel_mse": rel}
        if frame is not None:
            fp, fn, fw = frame
            out = torch.empty((fp.shape[0], 4), dtype=torch.float16, device=fp.device)
            for _ in range(3):
                m.query(fp, fn, out=out, aabb_min=aabb_min, aabb_max=aabb_max, t=0.5, image_width=fw)
            torch.cuda.synchronize()
            s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            for _ in range(10):
                m.query(fp, fn, out=out, aabb_min=aabb_min, aabb_max=aabb_max, t=0.5, image_width=fw)
            e0.record()
            torch.cuda.synchronize()
            row["fp16_ms_per_frame"] = s0.elapsed_time(e0) / 10
        rows.append(row)
        m.close()
    return rows
