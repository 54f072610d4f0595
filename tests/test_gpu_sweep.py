"""Memory-error trade-off on the seeded room (Sec. 4.1's hash-table-size study, Sec. 5.1's
comparison with probes at equal memory, with and without ray-traced visibility).

The paper's figures come from its own scenes (parity unpinned here).  What this checks
on the synthetic room: (1) hash collisions cost little, i.e. the smallest table's MSE
stays within a few times the largest's while its memory is an order of magnitude lower;
(2) at every budget the trained NIV beats the probe grid of the same memory; (3) ray-traced
visibility changes the probe answer.  The table is printed.
"""
import pytest

from niv_inputs import init_params, room_scene
from niv_inputs.configs import MODEL_C1

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def niv():
    from paper_2602_12949_gb300.build import build
    build()
    import paper_2602_12949_gb300 as P
    return P


def test_memory_error_tradeoff(niv):
    from paper_2602_12949_gb300 import fitting
    rows = fitting.memory_error_sweep(room_scene(0), [13, 15, 17], MODEL_C1, init_params, steps=1500)
    for r in rows:
        print("T=2^%d %6.2f MB: NIV MSE %.3g | probes %d^3 (%.2f MB) MSE %.3g, +RT %.3g | ratio %.1fx"
              % (r["log2_T"], r["mb"], r["niv_mse"], r["probes_per_axis"], r["probe_mb"], r["probe_mse"],
                 r["probe_rt_mse"], r["probe_mse"] / r["niv_mse"]))
    assert rows[0]["mb"] * 8 < rows[-1]["mb"]
    assert rows[0]["niv_mse"] < 4.0 * rows[-1]["niv_mse"]
    for r in rows:
        assert r["niv_mse"] < r["probe_mse"]
        assert r["probe_rt_mse"] != r["probe_mse"]
