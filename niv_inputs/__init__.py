"""Seeded synthetic inputs shared by the CUDA path's tests/bench and by the oracle.

This module is deliberately free of the method's arithmetic: it draws random
numbers, builds scene descriptions and casts primary rays to produce G-buffers.
It never evaluates an encoding, a network, irradiance or shading.  Both sides
(the C-ABI library and the CPU oracle) consume exactly the arrays produced here.

Record layout shared by both sides (an interface, not arithmetic):
  * points / normals / colours: contiguous ``[n][4]`` records, xyz(w) + pad.
  * parameters: one flat float32 vector = grid values (level-major, entry-major,
    ``F`` features per entry) followed, for every layer in order, by the weight
    matrix ``W[out][in]`` (row-major) and the bias ``b[out]``.
"""
from .queries import uniform_queries, sphere_directions
from .params import init_params, mlp_layer_shapes
from .scenes import Scene, room_scene, empty_scene, furnace_scene, single_emitter_scene
from .gbuffer import raycast_gbuffer, pack_records, camera_rays

__all__ = [
    "uniform_queries", "sphere_directions", "init_params", "mlp_layer_shapes",
    "Scene", "room_scene", "empty_scene", "furnace_scene", "single_emitter_scene",
    "raycast_gbuffer", "pack_records", "camera_rays",
]
