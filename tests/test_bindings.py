"""The Python binding refuses arguments that would send a kernel outside its buffers: host
tensors where device memory is required, records of the wrong type, and tensors whose
lengths disagree.  Every refusal happens before the library is called."""
import numpy as np
import pytest
import torch

from niv_inputs import room_scene
from niv_inputs.scenes import CAMERA_POS


def test_device_arguments_must_be_cuda():
    import paper_2602_12949_gb300 as P
    blob = room_scene(0).blob()
    with pytest.raises(ValueError):
        P.gbuffer_raycast(blob, 8, 8, CAMERA_POS, device="cpu")
    with pytest.raises(ValueError):
        P.training_samples(blob, 16, device="cpu")
    with pytest.raises(ValueError):
        P.ProbeGrid((2, 2, 2), (0, 0, 0), (1, 1, 1), device="cpu")
    cpu = torch.zeros((4, 4))
    with pytest.raises(ValueError):
        P.shade(cpu.half(), cpu.half(), cpu.half())
    with pytest.raises(ValueError):
        P.mc_irradiance(blob, cpu, cpu, 4)
    with pytest.raises(ValueError):
        P.compact_targets(cpu, cpu, torch.zeros((4, 3), dtype=torch.float64), torch.zeros(4, dtype=torch.uint8))


@pytest.mark.gpu
def test_mismatched_device_arguments_are_refused():
    import paper_2602_12949_gb300 as P
    from paper_2602_12949_gb300.build import build
    from niv_inputs.configs import MODEL_C0
    build()
    dev = torch.device("cuda", 0)
    blob = room_scene(0).blob()
    r32 = lambda n: torch.zeros((n, 4), dtype=torch.float32, device=dev)
    r16 = lambda n: torch.zeros((n, 4), dtype=torch.float16, device=dev)
    with pytest.raises(TypeError):
        P.mc_irradiance(blob, r16(8), r16(8), 4)
    with pytest.raises(ValueError):
        P.mc_irradiance(blob, r32(8), r32(7), 4)
    with pytest.raises(ValueError):
        P.mc_irradiance(blob, r32(8), r32(8), 4, t=torch.zeros(7, device=dev))
    with pytest.raises(ValueError):
        P.compact_targets(r32(8), r32(8), torch.zeros((7, 3), dtype=torch.float64, device=dev),
                          torch.zeros(8, dtype=torch.uint8, device=dev))
    with pytest.raises(ValueError):
        P.shade(r16(8), r16(7), r16(8))
    with pytest.raises(ValueError):
        P.upsample_shade(r16(16), r16(16), r16(16), r16(16), 4, 4, r16(3), sub=2)
    pos, nrm, alb, hit = P.gbuffer_raycast(blob, 8, 4, CAMERA_POS, want_hit=True)
    tri9 = torch.zeros((2, 9), device=dev)
    with pytest.raises(ValueError):
        P.gbuffer_meshes(tri9, torch.zeros(1, dtype=torch.int32, device=dev), np.ones((1, 3)), pos, nrm, alb, hit,
                         8, 4, CAMERA_POS)
    with pytest.raises(TypeError):
        P.gbuffer_meshes(tri9, torch.zeros(2, dtype=torch.int32, device=dev), np.ones((1, 3)), pos, nrm, alb,
                         hit.to(torch.int32), 8, 4, CAMERA_POS)
    with pytest.raises(ValueError):
        P.gbuffer_meshes(tri9, torch.zeros(2, dtype=torch.int32, device=dev), np.ones((1, 3)), pos, nrm, alb, hit,
                         8, 5, CAMERA_POS)
    m = P.NIVModel(**MODEL_C0)
    try:
        with pytest.raises(ValueError):
            m.query_shade(r16(8), r16(7), r16(8), r16(8))
        with pytest.raises(ValueError):
            m.fit(r32(8), r32(8), r32(7))
        with pytest.raises(TypeError):
            m.query_host(np.zeros((8, 4)), np.zeros((8, 4)))
        with pytest.raises(TypeError):
            m.grads_into(torch.zeros(m.param_count()[0] + m.param_count()[1], dtype=torch.float16))
        P.sync_status()
    finally:
        m.close()
