"""Benchmark of the Neural Irradiance Volume query on one GB300 (or N independent replicas).

Workload (default): the 1920x1080 FP16 G-buffer of the seeded 10 m room (24 spheres,
8 boxes, pinhole camera), model with 16 levels x 2 features, base 16, growth 1.38,
2^17-entry hashed tables, network 35-64-64-3 with softplus output.  One step = one
niv_query over the whole frame (load G-buffer, normalise, per-level index, gather,
interpolate, network, store E).  The fused FP16 tensor-core path is the headline;
the plain FP32 path runs on the same frame beside it, and both are compared with
the FP64 CPU oracle on sampled pixels.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl niv|reference]

Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA events on
the launching stream, with a 256 MB write between steps to flush L2 (the frame
and the model are smaller than L2).  Under torchrun every rank renders its own
frame (weak scaling, no data-path collective) and the max time over ranks counts.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FLOP_PER_QUERY = {"c1": 2 * (35 * 64 + 64 * 64 + 64 * 3)}  # 13,056: network multiply-adds x 2
METRIC = "ms/frame @1080p + Gqueries/s: FP16 fused vs FP32 plain at stated err vs FP64"
GBUF_BYTES_PER_QUERY = 18  # 12 B of FP16 position/normal in, 6 B of FP16 E out (algorithmic)
WORKLOAD = ("config1-1080p: seeded 10 m room (24 spheres, 8 boxes, sphere emitter) ray-cast to a "
            "1920x1080 FP16 G-buffer; model 16 levels x 2 features, base 16, growth 1.38, T=2^17, "
            "network 35-64-64-3 softplus, He-init weights")


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="niv", choices=["niv", "reference"])
    ap.add_argument("--precision", default="fp16", choices=["fp32", "fp16", "fp8"])
    ap.add_argument("--res", default="1080p", choices=["1080p", "4k"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true", help="skip the FP32 comparison and error checks")
    ap.add_argument("--workload", default="config1",
                    choices=["config1", "config3", "half", "sweep", "train", "time", "config2", "peaks"],
                    help="config1: the headline (config-1 model on the room frame); config3: the 4-D model at "
                         "--res with t from the seed; half: quarter-pixel query + upsampling and shading; "
                         "sweep: memory-error trade-off (hash table sizes against probes of equal memory); "
                         "train: niv_fit steps at batch 2^18 and the Monte Carlo target rate (config 2); "
                         "time: time-varying fields, config 3's 4-D grid against Sec. 6's frequency-encoded t; "
                         "config2: the training schedule of config 2 (see --train-steps, --spp)")
    ap.add_argument("--train-steps", type=int, default=5000, help="config2: Adam steps")
    ap.add_argument("--spp", type=int, default=1024, help="config2: Monte Carlo paths per training target")
    ap.add_argument("--reuse", type=int, default=1, help="config2: passes over each pool of targets")
    ap.add_argument("--model", default="c4", choices=["c1", "c4"],
                    help="config2: the model trained; c4 (default) is the 2^19-entry model that config 4 names "
                         "as config 2's, c1 the config-1 shape (2^17 entries)")
    return ap.parse_args()


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return {"hbm": p["hbm_gbs"], "tensor": p["bf16_tflops"], "src": "measured"}
    except Exception:
        return {"hbm": 6800.0, "tensor": 1900.0, "src": "fallback"}


def _extra_peaks():
    """FP32 FMA, FP8 tensor, L2 read and host-link rates measured by `bench.py --workload peaks`
    on this GPU model and recorded in profiles/measured_peaks_gb300.md; {} when absent."""
    out = {}
    try:
        with open(os.path.join(ROOT, "profiles", "measured_peaks_gb300.md")) as f:
            for line in f:
                k, _, v = line.partition(":")
                if k.strip() in ("fp32_ffma_tflops", "fp8_tflops", "l2_read_gbs", "host_frame_rw_gbs"):
                    out[k.strip()] = float(v.strip())
    except (OSError, ValueError):
        pass
    return out


def host_link_roofline(bytes_moved, seconds, link_gbs):
    """Roofline of a host-buffer call: the records and results cross the host link inside the
    call, so the link's measured rate for that traffic bounds it; None without a measurement."""
    if not link_gbs or seconds <= 0:
        return None
    achieved = bytes_moved / seconds / 1e9
    return {"bound": "host link", "achieved": achieved, "peak": link_gbs, "unit": "GB/s", "frac": achieved / link_gbs,
            "peak_source": "measured: a kernel streaming the same bytes through page-locked host memory "
                           "(profiles/measured_peaks_gb300.md)"}


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.3)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]

    def summary(self):
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in getattr(self, "lines", []):
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(sm)}


def kernel_code_hash(paths):
    """First 16 hex digits of the SHA-256 of C/C++/CUDA sources with their comments removed
    and every run of whitespace collapsed to one space: the code, not its comments or layout."""
    import hashlib
    import re
    tok = re.compile(r'"(?:\\.|[^"\\\n])*"|\'(?:\\.|[^\'\\\n])*\'|//[^\n]*|/\*.*?\*/', re.S)
    h = hashlib.sha256()
    for p in paths:
        with open(p) as fh:
            text = fh.read()
        code = tok.sub(lambda m: m.group(0) if m.group(0)[0] in "\"'" else " ", text)
        h.update(" ".join(code.split()).encode())
        h.update(b"\0")
    return h.hexdigest()[:16]


def _profiled_record():
    """DRAM bytes and warp instructions per launch of the fused kernel from the committed ncu
    summary, if the kernel's code is unchanged since that capture; else None."""
    path = os.path.join(ROOT, "profiles", "niv_query_fp16_1080p.md")
    srcs = ["query_tc.cu", "encoding.cuh", "tc_ptx.cuh"]  # the kernel and every device helper it includes
    try:
        text = open(path).read()
        rec = dict(l.split(":", 1) for l in text.splitlines()
                   if l.startswith(("traffic_bytes_per_launch:", "code_sha256_16:",
                                    "warp_instructions_per_launch:")))
        digest = kernel_code_hash([os.path.join(ROOT, "paper_2602_12949_gb300", "csrc", f) for f in srcs])
        if digest != rec["code_sha256_16"].strip():
            return None
        return {"traffic": int(rec["traffic_bytes_per_launch"].strip()),
                "instructions": int(rec["warp_instructions_per_launch"].strip())}
    except Exception:
        return None


def reduce_max(values, ws, device=None):
    """Max over ranks of each entry of `values` (floats); the values themselves when ws == 1.
    Every rank must call it with the same number of entries."""
    if ws <= 1:
        return [float(v) for v in values]
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def weak_throughput(units_per_rank, ws, seconds):
    """Whole-job rate (G units/s) of `ws` replicas that each processed `units_per_rank`
    units, the slowest of them in `seconds`."""
    return units_per_rank * ws / seconds / 1e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def _oracle_threads():
    try:
        import oracle
        return int(oracle.lib().orc_num_threads())
    except Exception:
        return os.cpu_count() or 1


def run_reference(a):
    """The oracle as it stands, on the host cores, K timed steps over a bounded sample of the frame."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    from niv_inputs import init_params
    from niv_inputs.configs import MODEL_C1, ROOM_MIN, ROOM_MAX, RESOLUTIONS, room_gbuffer
    w, h = RESOLUTIONS[a.res]
    pos, nrm, _ = room_gbuffer(w, h)
    om = oracle.Model(**MODEL_C1)
    params = init_params(oracle.grid_value_count(om), oracle.layer_shapes(om), seed=0)
    sample = 1 << 16
    rng = np.random.default_rng(1)
    times = []
    for step in range(a.warmup + a.steps):
        pick = rng.choice(len(pos), sample, replace=False)
        p, n = pos[pick].astype(np.float32), nrm[pick].astype(np.float32)
        t0 = time.perf_counter()
        oracle.query(om, params, p, n, ROOM_MIN, ROOM_MAX)
        dt = time.perf_counter() - t0
        if step >= a.warmup:
            times.append(dt)
    tot = sum(times)
    value = sample * a.steps / tot / 1e9
    cores = _oracle_threads()
    line = {
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "Gqueries/s", "n_gpus": a.gpus, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": 1e3 * tot / a.steps, "ms_per_frame": 1e3 * (w * h) / (value * 1e9),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "pixels": w * h, "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": value, "unit": "Gqueries/s", "cores": cores, "kind": "oracle",
                         "sample": "%d random pixels of the frame per step, FP64 C oracle with OpenMP" % sample},
        "e2e": {"value": value, "unit": "Gqueries/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def _time_launches(fn, steps, warmup, flush, stream):
    """Mean device time (ms) of fn() over `steps` launches, L2 flushed before each one."""
    import torch
    from paper_2602_12949_gb300 import sync_status
    for _ in range(warmup):
        fn()
    sync_status()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    torch.cuda.synchronize()
    for s, e in evs:
        flush.zero_()
        s.record(stream)
        fn()
        e.record(stream)
    torch.cuda.synchronize()
    sync_status()
    return statistics.mean(s.elapsed_time(e) for s, e in evs)


def _more_workloads(a, dev, flush, stream, steps=10, warmup=3):
    """Beside the headline: the config-1 model at 4K, the 4-D config-3 model at 4K in FP8 /
    FP16 / FP32 (t drawn from the seed per frame), and shading at 1080p and 4K."""
    import torch
    from paper_2602_12949_gb300 import NIVModel, shade
    from niv_inputs import init_params
    from niv_inputs.configs import MODEL_C1, MODEL_C3, ROOM_MIN, ROOM_MAX, room_gbuffer
    res = {}
    w, h = 3840, 2160
    pos, nrm, alb = room_gbuffer(w, h)
    npx = w * h
    dpos, dnrm = torch.from_numpy(pos).to(dev), torch.from_numpy(nrm).to(dev)
    out16 = torch.empty((npx, 4), dtype=torch.float16, device=dev)
    out32 = torch.empty((npx, 4), dtype=torch.float32, device=dev)
    kw = dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, image_width=w)
    m1 = NIVModel(**MODEL_C1)
    g, _ = m1.param_count()
    m1.set_params(init_params(g, m1.layer_shapes(), seed=0))
    r = {}
    for prec, o in (("fp16", out16), ("fp32", out32)):
        ms = _time_launches(lambda: m1.query(dpos, dnrm, out=o, precision=prec, **kw), steps, warmup, flush, stream)
        r[prec] = {"ms_per_frame": ms, "gqueries_per_s": npx / (ms * 1e-3) / 1e9}
    res["config1_4k"] = r
    m1.close()
    t = float(np.random.default_rng(0).random())  # per-frame scene parameter from the seed
    m3 = NIVModel(**MODEL_C3)
    g, _ = m3.param_count()
    m3.set_params(init_params(g, m3.layer_shapes(), seed=0))
    m3.fp8_calibrate(dpos[::31].contiguous(), dnrm[::31].contiguous(), aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, t=t)
    r = {"t": t}
    for prec, o in (("fp8", out16), ("fp16", out16), ("fp32", out32)):
        ms = _time_launches(lambda: m3.query(dpos, dnrm, out=o, precision=prec, t=t, **kw), steps, warmup, flush,
                            stream)
        r[prec] = {"ms_per_frame": ms, "gqueries_per_s": npx / (ms * 1e-3) / 1e9}
    res["config3_4k"] = r
    m3.close()
    # config 4: room + three inserted meshes, fused query + shading into FP16 rgba
    from niv_inputs.configs import MODEL_C4
    from niv_inputs.meshes import shading_frame
    p4, n4, a4, d4, cov = shading_frame(w, h)
    dp4, dn4, da4, dd4 = (torch.from_numpy(x).to(dev) for x in (p4, n4, a4, d4))
    rgba = torch.empty_like(out16)
    m4 = NIVModel(**MODEL_C4)
    g, _ = m4.param_count()
    m4.set_params(init_params(g, m4.layer_shapes(), seed=0))
    r = {"coverage": cov}
    for prec in ("fp16", "fp32"):
        ms = _time_launches(lambda: m4.query_shade(dp4, dn4, da4, dd4, out=rgba, precision=prec, **kw), steps, warmup,
                            flush, stream)
        r[prec + "_fused"] = {"ms_per_frame": ms, "gqueries_per_s": npx / (ms * 1e-3) / 1e9}
    ms_q = _time_launches(lambda: m4.query(dp4, dn4, out=out16, precision="fp16", **kw), steps, warmup, flush, stream)
    ms_s = _time_launches(lambda: shade(da4, dd4, out16, out=rgba), steps, warmup, flush, stream)
    r["fp16_query_then_shade"] = {"ms_per_frame": ms_q + ms_s, "shade_ms": ms_s,
                                  "shade_gb_per_s": 32 * npx / (ms_s * 1e-3) / 1e9}
    # dynamic ambient occlusion against the three meshes (Sec. 4.4), scaling E in place
    from paper_2602_12949_gb300 import DynamicGeometry
    from niv_inputs.meshes import dynamic_objects
    verts, tris, _, _ = dynamic_objects(0)
    tri9 = verts[tris].reshape(-1, 9).astype(np.float32)
    t0 = time.perf_counter()
    dyn = DynamicGeometry(tri9)
    build_ms = 1e3 * (time.perf_counter() - t0)
    ao = torch.empty(npx, dtype=torch.float32, device=dev)
    ms_ao = _time_launches(lambda: dyn.ao(dp4, dn4, rays=8, radius=0.5, out=ao, E=out16), steps, warmup, flush,
                           stream)
    r["dynamic_ao"] = {"triangles": int(len(tri9)), "nodes": dyn.node_count, "rays": 8, "radius": 0.5,
                       "ms_per_frame": ms_ao, "host_build_and_upload_ms": build_ms}
    dyn.close()
    res["config4_4k"] = r
    m4.close()
    # the non-neural path beside it: SH probe grid with the config-1 model's memory, 1080p frame
    from paper_2602_12949_gb300 import ProbeGrid
    from niv_inputs import room_scene
    pos1, nrm1, _ = room_gbuffer(1920, 1080)
    dp1, dn1 = torch.from_numpy(pos1).to(dev), torch.from_numpy(nrm1).to(dev)
    o1 = torch.empty((1920 * 1080, 4), dtype=torch.float16, device=dev)
    grid = ProbeGrid((50, 50, 50), ROOM_MIN, ROOM_MAX)
    grid.bake(room_scene(0).blob(), rays=256, seed=0)
    ms = _time_launches(lambda: grid.query(dp1, dn1, out=o1, image_width=1920), steps, warmup, flush, stream)
    blob = room_scene(0).blob()
    ms_rt = _time_launches(lambda: grid.query(dp1, dn1, out=o1, image_width=1920, scene_blob=blob), steps, warmup,
                           flush, stream)
    res["probes_1080p"] = {"probes": 125000, "mb": grid.nbytes / 1e6, "ms_per_frame": ms,
                           "gqueries_per_s": 1920 * 1080 / (ms * 1e-3) / 1e9,
                           "rt_visibility_ms_per_frame": ms_rt}
    res.update(_table1_and_half(dev, flush, stream, dp1, dn1, steps, warmup))
    return res


def _table1_and_half(dev, flush, stream, dpos, dnrm, steps, warmup):
    """Every model of Table 1 (frequency-encoded widths 16 / 32 / 64; grids of 2 to 8 levels x F=4)
    on the 1080p room frame in FP16: full resolution, and "half" (the pixels (2x, 2y) queried in
    place), beside the paper's RTX 4090 numbers.  Then the whole half-resolution pipeline with
    the config-1 model: quarter-pixel query + joint bilateral upsampling fused with shading."""
    import torch
    from paper_2602_12949_gb300 import NIVModel, upsample_shade
    from niv_inputs import init_params
    from niv_inputs.configs import TABLE1, MODEL_C1, ROOM_MIN, ROOM_MAX
    from niv_inputs.meshes import shading_frame
    W, H = 1920, 1080
    kw = dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)
    out = torch.empty((W * H, 4), dtype=torch.float16, device=dev)
    low = torch.empty(((W // 2) * (H // 2), 4), dtype=torch.float16, device=dev)
    rows = []
    for spec, paper_full, paper_half, paper_mb in TABLE1:
        m = NIVModel(**spec)
        g, n_mlp = m.param_count()
        m.set_params(init_params(g, m.layer_shapes(), seed=0))
        full = _time_launches(lambda: m.query(dpos, dnrm, out=out, image_width=W, **kw), steps, warmup, flush, stream)
        half = _time_launches(lambda: m.query_sub(dpos, dnrm, W, H, sub=2, out=low, **kw), steps, warmup, flush,
                              stream)
        rows.append({"width": spec["width"], "grid_levels": spec["levels"], "pe_bands": spec.get("pe_bands", 0),
                     "mb_fp16": 2 * (g + n_mlp) / 1e6, "full_ms": full, "half_ms": half,
                     "paper_rtx4090_full_ms": paper_full, "paper_rtx4090_half_ms": paper_half,
                     "paper_mb": paper_mb})
        m.close()
    p4, n4, a4, d4, _ = shading_frame(W, H)
    dp4, dn4, da4, dd4 = (torch.from_numpy(x).to(dev) for x in (p4, n4, a4, d4))
    rgba = torch.empty((W * H, 4), dtype=torch.float16, device=dev)
    m = NIVModel(**MODEL_C1)
    g, _ = m.param_count()
    m.set_params(init_params(g, m.layer_shapes(), seed=0))
    ms_q = _time_launches(lambda: m.query_sub(dp4, dn4, W, H, sub=2, out=low, **kw), steps, warmup, flush, stream)
    ms_u = _time_launches(lambda: upsample_shade(dp4, dn4, da4, dd4, W, H, low, sub=2, out=rgba), steps, warmup,
                          flush, stream)
    ms_f = _time_launches(lambda: m.query_shade(dp4, dn4, da4, dd4, out=rgba, image_width=W, **kw), steps, warmup,
                          flush, stream)
    m.close()
    up_bytes = 40 * W * H + 8 * (W // 2) * (H // 2)  # 4 records in, rgba out, E at quarter resolution
    half = {"query_ms": ms_q, "upsample_shade_ms": ms_u, "ms_per_frame": ms_q + ms_u,
            "full_res_fused_ms": ms_f, "upsample_gb_per_s": up_bytes / (ms_u * 1e-3) / 1e9,
            "upsample_bytes_per_frame": up_bytes}
    return {"table1_1080p_fp16": rows, "half_1080p_config1": half}


def run_peaks(a):
    """Rates the roofline of the other paths needs, measured on this GPU: FP32 FMA (the
    probe kernel of libniv_peaks.so, independent FMA chains on every thread), FP8 dense tensor
    (torch._scaled_mm, E4M3 8192^3), L2 read bandwidth (torch sum over a 64 MiB tensor,
    L2-resident after the first pass) and the host link (libniv_peaks.so's kernel streaming
    through page-locked host memory; copy engines).  Best of the timed repetitions, CUDA events."""
    import ctypes
    import torch
    from paper_2602_12949_gb300.build import BENCH_LIB
    peaks = ctypes.CDLL(BENCH_LIB)
    peaks.niv_peak_ffma.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p]
    peaks.niv_peak_ffma.restype = ctypes.c_int
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream()

    def best(fn, reps):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            fn()
            e0.record(stream)
            torch.cuda.synchronize()
            ts.append(s0.elapsed_time(e0))
        return min(ts)  # ms

    res = {}
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, iters = sms * 8 * 4, 8192
    buf = torch.zeros(blocks, device=dev)
    def ffma():
        if peaks.niv_peak_ffma(ctypes.c_void_p(buf.data_ptr()), blocks, iters, ctypes.c_void_p(stream.cuda_stream)):
            raise RuntimeError("niv_peak_ffma failed")
    ms = best(ffma, 10)
    res["fp32_ffma_tflops"] = 2.0 * 8 * iters * 256 * blocks / (ms * 1e-3) / 1e12
    try:
        n = 8192
        a8 = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn)
        b8 = torch.randn(n, n, device=dev).to(torch.float8_e4m3fn).t()
        one = torch.ones((), device=dev)
        ms = best(lambda: torch._scaled_mm(a8, b8, scale_a=one, scale_b=one, out_dtype=torch.bfloat16), 10)
        res["fp8_tflops"] = 2.0 * n ** 3 / (ms * 1e-3) / 1e12
    except Exception as e:  # FP8 GEMM not offered by this torch build
        res["fp8_tflops"] = None
        res["fp8_error"] = str(e)[:200]
    x = torch.ones(16 << 20, device=dev)  # 64 MiB of FP32
    ms = best(lambda: x.sum(), 50)
    res["l2_read_gbs"] = x.numel() * 4 / (ms * 1e-3) / 1e9
    del x
    # the host link: a kernel streaming through page-locked host memory with coalesced 16-byte
    # words (reads, writes, and both at the 2:1 ratio and sizes of a 1080p frame of FP16
    # records: pos + nrm in, E out, as the host-buffer query moves them), and the copy engines
    peaks.niv_peak_host_stream.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p]
    peaks.niv_peak_host_stream.restype = ctypes.c_int
    hblocks = sms * 8
    sink = torch.zeros(hblocks, dtype=torch.int32, device=dev)
    big = 256 << 20
    hin = torch.empty(big, dtype=torch.uint8).pin_memory()
    hout = torch.empty(big, dtype=torch.uint8).pin_memory()
    hin.fill_(1)

    def host(b_in, b_out):
        rc = peaks.niv_peak_host_stream(ctypes.c_void_p(hin.data_ptr()) if b_in else None, b_in,
                                        ctypes.c_void_p(hout.data_ptr()) if b_out else None, b_out,
                                        ctypes.c_void_p(sink.data_ptr()), hblocks, ctypes.c_void_p(stream.cuda_stream))
        if rc:
            raise RuntimeError("niv_peak_host_stream failed (%d)" % rc)
    res["host_read_gbs"] = big / (best(lambda: host(big, 0), 10) * 1e-3) / 1e9
    res["host_write_gbs"] = big / (best(lambda: host(0, big), 10) * 1e-3) / 1e9
    f_in, f_out = 2 * 1920 * 1080 * 8, 1920 * 1080 * 8
    ms = best(lambda: host(f_in, f_out), 20)
    res["host_frame_rw_gbs"] = (f_in + f_out) / (ms * 1e-3) / 1e9
    res["host_frame_rw_ms"] = ms
    dbuf = torch.empty(big, dtype=torch.uint8, device=dev)
    res["h2d_copy_gbs"] = big / (best(lambda: dbuf.copy_(hin, non_blocking=True), 10) * 1e-3) / 1e9
    res["d2h_copy_gbs"] = big / (best(lambda: hout.copy_(dbuf, non_blocking=True), 10) * 1e-3) / 1e9
    line = {"metric": "measured peaks for the rooflines beside the tensor one", "value": res["fp32_ffma_tflops"],
            "unit": "TFLOP/s (FP32 FMA)", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "peaks": res, "gpu": torch.cuda.get_device_name(dev), "sms": sms}
    print(json.dumps(line), flush=True)


def run_sweep(a):
    """Memory-error trade-off on the seeded room: NIV (config-1 shape) trained at hash table
    sizes 2^13 .. 2^19 against the SH probe grid of the same memory, with and without
    ray-traced visibility; MSE on 2^14 held-out samples with 4096-spp references."""
    import torch
    from paper_2602_12949_gb300 import fitting
    from niv_inputs import init_params, room_scene
    from niv_inputs.configs import MODEL_C1
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    rows = fitting.memory_error_sweep(room_scene(0), [13, 15, 17, 19], MODEL_C1, init_params, steps=2000)
    ref = next(r for r in rows if r["log2_T"] == 17)
    line = {"metric": "held-out MSE, NIV vs SH probes of equal memory (hash table size sweep)",
            "value": ref["probe_mse"] / ref["niv_mse"], "unit": "x (probe MSE / NIV MSE at T=2^17)",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic", "dtype": "f16",
            "config": {"workload": "room scene seed 0; NIV 16 levels x 2 features, base 16, growth 1.38, "
                                   "35-64-64-3; 2000 Adam steps, batch 2^16, 128-spp targets; probes baked "
                                   "with 1024 rays"},
            "rows": rows, "seconds": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


def run_config2(a):
    """Config 2: niv_fit on the room (sky + rotating-free emitter at t = 0) with the FP16 forward and
    FP32 master weights, batch 2^18, --train-steps Adam steps at lr 1e-2, targets from the GPU
    Monte Carlo integrator (INDIRECT, --spp paths) on pools of 2^20 candidates (80% volume, 20%
    surface, culled), each pool serving --reuse passes; then the held-out MSE against 4096-spp
    references beside the SH probe grid of the same memory, with and without ray-traced
    visibility."""
    import torch
    from paper_2602_12949_gb300 import NIVModel, ProbeGrid, fitting
    from niv_inputs import init_params, room_scene
    from niv_inputs.configs import MODEL_C1, MODEL_C4, ROOM_MIN, ROOM_MAX
    torch.cuda.set_device(0)
    scene = room_scene(0)
    spec = MODEL_C4 if a.model == "c4" else MODEL_C1
    m = NIVModel(**spec)
    g, nm = m.param_count()
    m.set_params(init_params(g, m.layer_shapes(), seed=0))
    t0 = time.perf_counter()
    info = fitting.train(m, scene, steps=a.train_steps, batch=1 << 18, pool=1 << 20, spp=a.spp, reuse=a.reuse,
                         seed=1, log_every=500, forward="fp16")
    train_s = time.perf_counter() - t0
    hx, hn, hE, _ = fitting.held_out(scene, 1 << 16, 4096, seed=99)
    q = dict(out_dtype=torch.float32, aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)
    niv = {p: fitting.errors(m.query(hx, hn, precision=p, **q), hE) for p in ("fp16", "fp32")}
    nbytes = 2 * (g + nm)
    P = int((nbytes / 54.0) ** (1.0 / 3.0))
    grid = ProbeGrid((P,) * 3, ROOM_MIN, ROOM_MAX)
    grid.bake(scene.blob(), rays=4096, seed=3)
    probe = fitting.errors(grid.query(hx, hn, out_dtype=torch.float32), hE)
    probe_rt = fitting.errors(grid.query(hx, hn, out_dtype=torch.float32, scene_blob=scene.blob()), hE)
    line = {"metric": "config 2: held-out MSE of the trained NIV vs the same-memory SH probe grid",
            "value": probe[0] / niv["fp16"][0], "unit": "x (probe MSE / NIV FP16 MSE)", "n_gpus": 1,
            "higher_is_better": True, "data": "synthetic", "dtype": "f16 forward, f32 master weights",
            "config": {"workload": "config2: room scene seed 0 (uniform sky through the skylight + sphere emitter), "
                                   "%s (%.2f MB FP16), batch 2^18, lr 1e-2, Adam (0.9, 0.99, 1e-15), "
                                   "pools of 2^20 candidates"
                                   % ("2^19-entry model of config 4" if a.model == "c4" else "config-1 model",
                                      2 * (g + nm) / 1e6), "steps": a.train_steps, "spp": a.spp,
                       "reuse": a.reuse, "held_out": "2^16 samples, 4096-spp references"},
            "niv_mse_fp16": niv["fp16"][0], "niv_rel_mse_fp16": niv["fp16"][1], "niv_mse_fp32": niv["fp32"][0],
            "probe_grid": "%d^3 (%.2f MB)" % (P, grid.nbytes / 1e6), "probe_mse": probe[0], "probe_rel_mse": probe[1],
            "probe_rt_mse": probe_rt[0], "probe_rt_rel_mse": probe_rt[1], "loss": info["loss"],
            "seconds_monte_carlo": info["seconds_mc"], "seconds_fit": info["seconds_fit"], "pools": info["pools"],
            "seconds_total": train_s}
    print(json.dumps(line), flush=True)
    m.close()


def run_time(a):
    """Fields that change with t (Sec. 6; config 3): config 3's 4-D grid, Sec. 6's 3-D grid
    (T = 2^18) with t frequency-encoded after n, and a static model without t, trained alike
    (2000 steps) on the room whose emitter rotates with t; held-out MSE and the FP16 query
    time on the 4K room frame."""
    import torch
    from paper_2602_12949_gb300 import fitting
    from niv_inputs import init_params, room_scene
    from niv_inputs.configs import MODEL_C3, room_gbuffer
    torch.cuda.set_device(0)
    pos, nrm, _ = room_gbuffer(3840, 2160)
    frame = (torch.from_numpy(pos).cuda(), torch.from_numpy(nrm).cuda(), 3840)
    sec6 = dict(dims=3, levels=16, feat=2, log2_T=18, base=16.0, growth=1.38, n_hidden=3, width=64)
    shapes = {"4d_grid_config3": MODEL_C3, "3d_grid_t_bands4_sec6": dict(sec6, t_bands=4), "static_3d_no_t": sec6}
    t0 = time.perf_counter()
    rows = fitting.time_field_comparison(room_scene(0), shapes, init_params, steps=2000, frame=frame)
    by = {r["model"]: r for r in rows}
    line = {"metric": "held-out MSE of time-varying fields (config 3's 4-D grid vs Sec. 6's encoded t)",
            "value": by["4d_grid_config3"]["mse"] / by["3d_grid_t_bands4_sec6"]["mse"],
            "unit": "x (4-D grid MSE / Sec. 6 MSE)", "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "dtype": "f16", "config": {"workload": "room scene seed 0, emitter rotating with t; 2000 Adam steps, "
                                                   "batch 2^16, 128-spp targets with uniform per-sample t; held-out "
                                                   "2^14 samples at 16 values of t, 4096 spp"},
            "rows": rows, "seconds": time.perf_counter() - t0}
    print(json.dumps(line), flush=True)


def run_train(a):
    """Config 2's training step: niv_fit (FP32 forward, hand-written backward, Adam) on batches
    of 2^18 samples of the room, timed with CUDA events over K steps after W warm-up steps;
    beside it the GPU Monte Carlo target rate at 1024 spp (INDIRECT) on 2^16 training
    samples, and the time the whole schedule (5,000 steps, 2^20-sample pools at 1024 spp,
    one pool per 4 steps) takes at these rates."""
    import torch
    from paper_2602_12949_gb300 import NIVModel, mc_irradiance, sync_status, training_samples
    from niv_inputs import init_params, room_scene
    from niv_inputs.configs import MODEL_C1, ROOM_MIN, ROOM_MAX
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    scene = room_scene(0)
    batch = 1 << 18
    dx, dn, _, _ = training_samples(scene.blob(), batch, seed=5, device=dev)
    y = torch.rand((batch, 4), device=dev) * 2.0 + 0.1
    m = NIVModel(**MODEL_C1)
    g, nm = m.param_count()
    m.set_params(init_params(g, m.layer_shapes(), seed=0))
    kw = dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)
    stream = torch.cuda.current_stream()
    s0, e0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step = {}
    for fwd in ("fp32", "fp16"):
        m.set_train_forward(fwd)
        for _ in range(a.warmup):
            m.fit(dx, dn, y, want_loss=False, **kw)
        sync_status()
        s0.record(stream)
        for _ in range(a.steps):
            m.fit(dx, dn, y, want_loss=False, **kw)
        e0.record(stream)
        torch.cuda.synchronize()
        sync_status()
        step[fwd] = s0.elapsed_time(e0) / a.steps
    step_ms = step["fp16"]  # config 2: FP16 forward, FP32 master weights
    mc_n, spp = 1 << 16, 1024
    mxd, mnd, _, _ = training_samples(scene.blob(), mc_n, seed=6, device=dev)
    mc_irradiance(scene.blob(), mxd, mnd, 16, seed=1, mode="indirect")
    torch.cuda.synchronize()
    s0.record(stream)
    mc_irradiance(scene.blob(), mxd, mnd, spp, seed=2, mode="indirect")
    e0.record(stream)
    torch.cuda.synchronize()
    mc_ms = s0.elapsed_time(e0)
    paths_per_s = mc_n * spp / (mc_ms * 1e-3)
    schedule_s = 5000 * step_ms * 1e-3 + (5000 / 4) * (1 << 20) * 1024 / paths_per_s
    line = {"metric": "niv_fit step time at batch 2^18 (config 2) and Monte Carlo target rate",
            "value": 1e3 / step_ms, "unit": "steps/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
            "ms_per_step": step_ms, "ms_per_step_fp32_forward": step["fp32"], "higher_is_better": True,
            "dtype": "f16 forward, f32 master weights", "data": "synthetic",
            "samples_per_s": batch / (step_ms * 1e-3), "mc_paths_per_s": paths_per_s,
            "mc_ms_per_2e16_samples_1024spp": mc_ms, "projected_config2_schedule_s": schedule_s,
            "config": {"workload": "config2-train: config-1 model on 2^18 room training samples (80% volume, "
                                   "20% surface), Eq. 3 loss, Adam lr 1e-2; targets from the GPU Monte Carlo "
                                   "integrator (INDIRECT, 1024 spp)", "batch": batch, "parallelism": "single"}}
    print(json.dumps(line), flush=True)
    m.close()


def run_workload(a):
    """One side workload on one GPU, timed like the headline: K steps after W warm-up steps,
    L2 flushed (256 MB write) before each step, CUDA events on the launching stream."""
    import torch
    if a.workload == "sweep":
        run_sweep(a)
        return
    if a.workload == "peaks":
        run_peaks(a)
        return
    if a.workload == "train":
        run_train(a)
        return
    if a.workload == "time":
        run_time(a)
        return
    if a.workload == "config2":
        run_config2(a)
        return
    from paper_2602_12949_gb300 import NIVModel, upsample_shade
    from niv_inputs import init_params
    from niv_inputs.configs import MODEL_C1, MODEL_C3, ROOM_MIN, ROOM_MAX, RESOLUTIONS, room_gbuffer
    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    W, H = RESOLUTIONS[a.res]
    npx = W * H
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    peaks = _peaks()
    kw = dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX)
    fp8_measured = None
    if a.workload == "config3":
        pos, nrm, _ = room_gbuffer(W, H)
        dp, dn = torch.from_numpy(pos).to(dev), torch.from_numpy(nrm).to(dev)
        t = float(np.random.default_rng(0).random())  # per-frame scene parameter from the seed
        m = NIVModel(**MODEL_C3)
        g, _ = m.param_count()
        m.set_params(init_params(g, m.layer_shapes(), seed=0))
        if a.precision == "fp8":
            m.fp8_calibrate(dp[::31].contiguous(), dn[::31].contiguous(), t=t, **kw)
        out = torch.empty((npx, 4), dtype=torch.float32 if a.precision == "fp32" else torch.float16, device=dev)
        step = lambda: m.query(dp, dn, out=out, precision=a.precision, t=t, image_width=W, **kw)
        flop = 2 * (36 * 64 + 2 * 64 * 64 + 64 * 3)  # 21,376 per query
        fp8_measured = _extra_peaks().get("fp8_tflops") if a.precision == "fp8" else None
        # FP8: the measured E4M3 rate, else the nominal 2x of the measured BF16 one
        tensor_peak = fp8_measured or peaks["tensor"] * (2.0 if a.precision == "fp8" else 1.0)
        config = {"workload": "config3-%s: 4-D model (16 levels x 2 features, T=2^19, 36-64-64-64-3) on the "
                              "%dx%d room frame, t=%.4f" % (a.res, W, H, t), "pixels": npx, "precision": a.precision}
        unit_per_step = npx
    else:
        from niv_inputs.meshes import shading_frame
        p4, n4, a4, d4, _ = shading_frame(W, H)
        dp, dn, da, dd = (torch.from_numpy(x).to(dev) for x in (p4, n4, a4, d4))
        m = NIVModel(**MODEL_C1)
        g, _ = m.param_count()
        m.set_params(init_params(g, m.layer_shapes(), seed=0))
        w, h = (W + 1) // 2, (H + 1) // 2
        low = torch.empty((w * h, 4), dtype=torch.float16, device=dev)
        rgba = torch.empty((npx, 4), dtype=torch.float16, device=dev)

        def step():
            m.query_sub(dp, dn, W, H, sub=2, out=low, precision=a.precision, **kw)
            upsample_shade(dp, dn, da, dd, W, H, low, sub=2, out=rgba)
        flop = 2 * (35 * 64 + 64 * 64 + 64 * 3) / 4.0  # per full-resolution pixel: a quarter of the queries
        tensor_peak = peaks["tensor"]
        config = {"workload": "half-%s: config-1 model queried at the pixels (2x, 2y) of the %dx%d frame with "
                              "three inserted meshes, joint bilateral upsampling + shading to FP16 rgba"
                              % (a.res, W, H), "pixels": npx, "precision": a.precision}
        unit_per_step = npx
    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    with ClockSampler(0) as clk:
        for s0, e0 in evs:
            flush.zero_()
            s0.record(stream)
            step()
            e0.record(stream)
        torch.cuda.synchronize()
    ms = statistics.mean(s0.elapsed_time(e0) for s0, e0 in evs)
    achieved = flop * unit_per_step / (ms * 1e-3) / 1e12
    line = {"metric": "ms/frame and Gpixels/s, %s" % a.workload, "value": unit_per_step / (ms * 1e-3) / 1e9,
            "unit": "Gpixels/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup, "ms_per_step": ms,
            "ms_per_frame": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "fp16": "f16", "fp8": "e4m3"}[a.precision], "data": "synthetic",
            "config": dict(config, l2="flushed between steps (256 MB write)", parallelism="single"),
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": tensor_peak, "unit": "TFLOP/s",
                         "frac": achieved / tensor_peak, "traffic": None,
                         "peak_source": ("measured E4M3 dense rate (profiles/measured_peaks_gb300.md)"
                                         if fp8_measured else
                                         "%s bf16 burst%s" % (peaks["src"], " x 2 (FP8 dense rate)"
                                                              if a.precision == "fp8" else ""))},
            "clocks": clk.summary()}
    print(json.dumps(line), flush=True)
    m.close()


def main():
    a = _args()
    if a.impl == "reference":
        run_reference(a)
        return
    if a.workload != "config1":
        run_workload(a)
        return
    import torch
    import torch.distributed as dist
    ws, rank, local = _dist()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", init_method="env://")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2602_12949_gb300 import NIVModel, sync_status
    from niv_inputs import init_params
    from niv_inputs.configs import MODEL_C1, ROOM_MIN, ROOM_MAX, RESOLUTIONS, room_gbuffer

    w, h = RESOLUTIONS[a.res]
    npx = w * h
    pos, nrm, _ = room_gbuffer(w, h)
    model = NIVModel(**MODEL_C1)
    g, _ = model.param_count()
    params = init_params(g, model.layer_shapes(), seed=0)
    model.set_params(params)
    dpos = torch.from_numpy(pos).to(dev)
    dnrm = torch.from_numpy(nrm).to(dev)
    out = torch.empty((npx, 4), dtype=torch.float16, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()
    qkw = dict(aabb_min=ROOM_MIN, aabb_max=ROOM_MAX, image_width=w)

    def timed(precision, out_t, steps, warmup):
        for _ in range(warmup):
            model.query(dpos, dnrm, out=out_t, precision=precision, **qkw)
        sync_status()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        if ws > 1:
            dist.barrier()
        torch.cuda.synchronize()
        for s, e in evs:
            flush.zero_()
            s.record(stream)
            model.query(dpos, dnrm, out=out_t, precision=precision, **qkw)
            e.record(stream)
        torch.cuda.synchronize()
        if ws > 1:
            dist.barrier()
        sync_status()
        return [s.elapsed_time(e) for s, e in evs]  # ms

    with ClockSampler(torch.cuda.current_device() if ws == 1 else local) as clk:
        ms = timed(a.precision, out, a.steps, a.warmup)

    extra = {}
    if not a.no_compare:
        out32 = torch.empty((npx, 4), dtype=torch.float32, device=dev)
        ms32 = timed("fp32", out32, max(5, a.steps // 2), 3)
        extra["fp32_plain"] = {"ms_per_frame": statistics.median(ms32),
                               "gqueries_per_s": npx / (statistics.median(ms32) * 1e-3) / 1e9}
        ffma = _extra_peaks().get("fp32_ffma_tflops")
        if ffma:  # the plain path runs its network on the FP32 FMA pipes: its bound is the FFMA rate
            ach = FLOP_PER_QUERY["c1"] * npx / (statistics.median(ms32) * 1e-3) / 1e12
            extra["fp32_plain"]["roofline"] = {"bound": "ffma", "achieved": ach, "peak": ffma, "unit": "TFLOP/s",
                                               "frac": ach / ffma,
                                               "peak_source": "measured (profiles/measured_peaks_gb300.md)"}
        extra["more"] = _more_workloads(a, dev, flush, stream)

    # e2e: page-locked host buffers through niv_query_host, which lets the query kernel read
    # the records from host memory and write E back to it (NVLink-C2C); the L2 is flushed
    # before each call, so no record is served from a copy cached by an earlier call
    hp = torch.from_numpy(pos).pin_memory().numpy()
    hn = torch.from_numpy(nrm).pin_memory().numpy()
    ho = torch.empty((npx, 4), dtype=torch.float16).pin_memory().numpy()
    for _ in range(2):  # through the Python binding first (its argument checks), then
        model.query_host(hp, hn, out=ho, precision=a.precision, **qkw)
    # the C-ABI call itself, its arguments marshalled once as a C caller holds them
    import ctypes
    from paper_2602_12949_gb300 import lib as _niv_lib, PRECISIONS
    from paper_2602_12949_gb300._lib import check as _check, NIV_F16
    c_qp = model.query_params(ROOM_MIN, ROOM_MAX, 0.0, w)
    c_args = (model.handle, ctypes.c_void_p(hp.ctypes.data), ctypes.c_void_p(hn.ctypes.data), ctypes.c_int64(npx),
              NIV_F16, ctypes.byref(c_qp), ctypes.c_void_p(ho.ctypes.data), NIV_F16, PRECISIONS[a.precision],
              ctypes.c_void_p(stream.cuda_stream))
    query_host_c = _niv_lib().niv_query_host
    e2e_t = []
    for _ in range(max(3, a.steps)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc = query_host_c(*c_args)
        e2e_t.append(time.perf_counter() - t0)
        _check(rc)
    # per-step figures: the median over the timed steps (mean beside it), max over ranks
    ms_med, e2e_med, ms_total = reduce_max([statistics.median(ms), statistics.median(e2e_t), sum(ms)], ws, dev)
    ms_step = ms_med
    value = weak_throughput(npx, ws, ms_step * 1e-3)
    e2e_val = weak_throughput(npx, ws, e2e_med)

    if rank != 0:
        if ws > 1:
            dist.destroy_process_group()
        return

    peaks = _peaks()
    mean_ms = ms_med  # the roofline and the records below use the median step
    flop = FLOP_PER_QUERY["c1"] * npx
    achieved = flop / (mean_ms * 1e-3) / 1e12
    prof = _profiled_record() if (a.precision == "fp16" and a.res == "1080p") else None
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peaks["tensor"], "unit": "TFLOP/s",
                "frac": achieved / peaks["tensor"], "traffic": prof["traffic"] if prof else None,
                "peak_source": "%s bf16 burst (fp16 dense rate equal)" % peaks["src"],
                "hbm_achieved_gbs": GBUF_BYTES_PER_QUERY * npx / (mean_ms * 1e-3) / 1e9}
    if prof:
        # encoding-aware bound: the kernel's warp instructions (ncu) issued at one per cycle on
        # each of the 4 schedulers of every SM, at the SM clock sampled during the timed steps
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        clk_mhz = clk.summary().get("sm_mhz") or clk.summary().get("sm_max_mhz") or 2070.0
        issue_ms = prof["instructions"] / (sms * 4 * clk_mhz * 1e6) * 1e3
        roofline["issue_bound"] = {"ms": issue_ms, "frac": issue_ms / mean_ms, "warp_instructions": prof["instructions"],
                                   "sm_mhz": clk_mhz}

    cpu = None
    errs = {}
    if not a.no_cpu_baseline and ws == 1:
        import oracle
        om = oracle.Model(**MODEL_C1)
        sample = 1 << 17
        pick = np.random.default_rng(1).choice(npx, sample, replace=False)
        p32, n32 = pos[pick].astype(np.float32), nrm[pick].astype(np.float32)
        oracle.query(om, params, p32[:1024], n32[:1024], ROOM_MIN, ROOM_MAX)
        t0 = time.perf_counter()
        ref = oracle.query(om, params, p32, n32, ROOM_MIN, ROOM_MAX)
        dt = time.perf_counter() - t0
        cpu = {"value": sample / dt / 1e9, "unit": "Gqueries/s", "cores": _oracle_threads(), "kind": "oracle",
               "sample": "%d random pixels of the frame, FP64 C oracle (OpenMP)" % sample,
               "ms_per_frame_extrapolated": 1e3 * dt * npx / sample,
               "ms_per_4k_frame_extrapolated": 4e3 * dt * npx / sample}
        # the same oracle on one host core, over a sixteenth of the sample
        all_cores = _oracle_threads()
        oracle.lib().orc_set_num_threads(1)
        try:
            s1 = sample // 16
            t0 = time.perf_counter()
            oracle.query(om, params, p32[:s1], n32[:s1], ROOM_MIN, ROOM_MAX)
            dt1 = time.perf_counter() - t0
        finally:
            oracle.lib().orc_set_num_threads(all_cores)
        cpu["one_core"] = {"value": s1 / dt1 / 1e9, "unit": "Gqueries/s", "cores": 1,
                           "sample": "%d of those pixels" % s1, "ms_per_frame_extrapolated": 1e3 * dt1 * npx / s1}
        got = out[pick, :3].double().cpu().numpy()
        den = np.maximum(np.abs(ref), 1e-3 * np.abs(ref).max())
        errs[a.precision] = {"max_rel": float(np.max(np.abs(got - ref) / den)),
                             "max_abs_normalised": float(np.max(np.abs(got - ref)) / np.abs(ref).max())}
        if "fp32_plain" in extra:
            got32 = out32[pick, :3].double().cpu().numpy()
            errs["fp32"] = {"max_rel": float(np.max(np.abs(got32 - ref) / den)),
                            "max_abs_normalised": float(np.max(np.abs(got32 - ref)) / np.abs(ref).max())}

    e2e = {"value": e2e_val, "unit": "Gqueries/s", "h2d_bytes_per_step": int(2 * hp.nbytes),
           "d2h_bytes_per_step": int(ho.nbytes), "ms_per_frame": 1e3 * e2e_med,
           "calls": len(e2e_t), "statistic": "median wall-clock time of the calls",
           "path": "the niv_query_host C-ABI call (ctypes, arguments marshalled once) on page-locked "
                   "buffers: the query kernel reads pos/nrm from host memory and writes E to it over "
                   "NVLink-C2C; L2 flushed before each call"}
    link_roofline = host_link_roofline(2 * hp.nbytes + ho.nbytes, e2e_med, _extra_peaks().get("host_frame_rw_gbs"))
    if link_roofline:
        e2e["roofline"] = link_roofline

    line = {
        "metric": METRIC, "value": value, "unit": "Gqueries/s", "n_gpus": ws, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": ms_step, "ms_per_frame": mean_ms, "ms_per_step_mean": ms_total / a.steps,
        "timing": "CUDA events per step on the launching stream; median of the timed steps",
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {"fp32": "f32", "fp16": "f16", "fp8": "e4m3"}[a.precision],
        "data": "synthetic",
        "config": {"workload": WORKLOAD.replace("1920x1080", "%dx%d" % (w, h)), "pixels": npx,
                   "precision": a.precision, "l2": "flushed between steps (256 MB write)",
                   "parallelism": "replicas" if ws > 1 else "single"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "clocks": clk.summary(),
        "gpu_launches": a.steps,
        "err_vs_fp64": errs,
        "paper_context": {"ms_per_frame_rtx4090_table1_8lv_f4": 1.35, "note": "different model and GPU"},
    }
    line.update(extra)
    print(json.dumps(line), flush=True)
    model.close()
    if ws > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
