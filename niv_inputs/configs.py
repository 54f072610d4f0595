"""Model shapes and workloads of the evaluated configurations (hyper-parameters only).

C0: plain FP32 forward, 65,536 queries uniform in the unit cube.
C1: 1920x1080 FP16 G-buffer of the seeded room; 16 x 2 levels, base 16, growth 1.38, T = 2^17.
C3: 3840x2160 time-varying field; 4-D grid, T = 2^19, three hidden layers, t appended.
C4: 3840x2160 shading frame; 3-D grid with T = 2^19.
P:  the paper's largest Table 1 model (8 levels x F = 4, base 16, scale sqrt(2), T = 2^17,
    four weight matrices), for a like-for-like comparison with its 1.35 ms on an RTX 4090.
PE16 / PE32 / PE64: Table 1's models without grid levels (eight-band frequency encoding of the
    position, widths 16 / 32 / 64, four weight matrices).
TABLE1: every row of Table 1 (width, grid levels) with the paper's RTX 4090 full / half ms.
"""
import os

import numpy as np

MODEL_C0 = dict(dims=3, levels=8, feat=2, log2_T=14, base=4.0, growth=1.5, n_hidden=2, width=64)
MODEL_C1 = dict(dims=3, levels=16, feat=2, log2_T=17, base=16.0, growth=1.38, n_hidden=2, width=64)
MODEL_C3 = dict(dims=4, levels=16, feat=2, log2_T=19, base=16.0, growth=1.38, n_hidden=3, width=64, in_extra=4)
MODEL_C4 = dict(dims=3, levels=16, feat=2, log2_T=19, base=16.0, growth=1.38, n_hidden=2, width=64)
MODEL_P = dict(dims=3, levels=8, feat=4, log2_T=17, base=16.0, growth=2.0 ** 0.5, n_hidden=3, width=64)
MODEL_PE16 = dict(dims=3, levels=0, feat=2, log2_T=17, pe_bands=8, n_hidden=3, width=16)
MODEL_PE32 = dict(MODEL_PE16, width=32)
MODEL_PE64 = dict(MODEL_PE16, width=64)
TABLE1 = [  # (model, paper full-HD ms, paper quarter-resolution ms, paper MB)
    (MODEL_PE16, 0.19, 0.029, 0.003),
    (MODEL_PE32, 0.20, 0.031, 0.01),
    (MODEL_PE64, 0.25, 0.069, 0.03),
    (dict(MODEL_P, levels=2), 0.31, 0.088, 0.16),
    (dict(MODEL_P, levels=4), 0.67, 0.18, 1.20),
    (dict(MODEL_P, levels=6), 1.06, 0.26, 3.30),
    (MODEL_P, 1.35, 0.37, 5.40),
]

ROOM_MIN = (-5.0, -5.0, -5.0)
ROOM_MAX = (5.0, 5.0, 5.0)

RESOLUTIONS = {"1080p": (1920, 1080), "4k": (3840, 2160)}


def room_gbuffer(width, height, seed=0, cache_dir=None):
    """FP16 [n][4] position / normal / albedo records of the seeded room at width x height.

    Cached as .npz under ``cache_dir`` (default: $NIV_CACHE or /tmp/niv_cache) because
    the numpy ray cast takes seconds per megapixel.
    """
    from .scenes import room_scene
    from .gbuffer import raycast_gbuffer, pack_records
    cache_dir = cache_dir or os.environ.get("NIV_CACHE", "/tmp/niv_cache")
    path = os.path.join(cache_dir, "room_s%d_%dx%d.npz" % (seed, width, height))
    if os.path.exists(path):
        try:
            z = np.load(path)
            return z["pos"], z["nrm"], z["alb"]
        except Exception:
            pass
    pos, nrm, alb, _ = raycast_gbuffer(room_scene(seed), width, height)
    out = (pack_records(pos, np.float16), pack_records(nrm, np.float16), pack_records(alb, np.float16))
    try:
        os.makedirs(cache_dir, exist_ok=True)
        tmp = path + ".tmp%d.npz" % os.getpid()
        np.savez(tmp, pos=out[0], nrm=out[1], alb=out[2])
        os.replace(tmp, path)
    except OSError:
        pass
    return out
