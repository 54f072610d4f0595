"""Fields that change with a scene parameter t (Sec. 6; config 3) on the seeded room, whose
emitter rotates about the vertical axis with t.

Three designs, trained alike on Monte Carlo targets with a per-sample t and scored on the
same held-out (x, n, t) samples: config 3's 4-D grid (t as the 4th grid axis and a raw
input), Sec. 6's form (a 3-D grid with the hash table doubled to 2^18 and t frequency-
encoded after n), and a static model without t.  Parity unpinned (no paper numbers for
this scene); what is checked: both time-aware designs beat the static one, i.e. the t input
is learned.  The table is printed.
"""
import pytest

from niv_inputs import init_params, room_scene
from niv_inputs.configs import MODEL_C3

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

SHAPES = {
    "4-D grid (config 3)": MODEL_C3,
    "3-D grid T=2^18 + t frequency-encoded (Sec. 6)": dict(dims=3, levels=16, feat=2, log2_T=18, base=16.0,
                                                           growth=1.38, n_hidden=3, width=64, t_bands=4),
    "static 3-D grid T=2^18, no t": dict(dims=3, levels=16, feat=2, log2_T=18, base=16.0, growth=1.38, n_hidden=3,
                                         width=64),
}


@pytest.fixture(scope="module")
def niv():
    from paper_2602_12949_gb300.build import build
    build()
    import paper_2602_12949_gb300 as P
    return P


def test_time_aware_designs_learn_t(niv):
    from paper_2602_12949_gb300 import fitting
    rows = fitting.time_field_comparison(room_scene(0), SHAPES, init_params, steps=1500)
    for r in rows:
        print("%-48s %6.2f MB  MSE %.3g  rel %.3g" % (r["model"], r["mb"], r["mse"], r["rel_mse"]))
    mse = {r["model"]: r["mse"] for r in rows}
    static = mse["static 3-D grid T=2^18, no t"]
    assert mse["4-D grid (config 3)"] < static
    assert mse["3-D grid T=2^18 + t frequency-encoded (Sec. 6)"] < static
