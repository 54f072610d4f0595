"""Neural Irradiance Volume query path for one GB300 (sm_103a).

``libniv.so`` (hand-written CUDA kernels behind a C ABI, see include/niv.h) does
all the work; this package marshals torch tensors into it.
"""
from ._lib import lib, NivError, LIB_PATH
from .model import (NIVModel, NIVModule, ProbeGrid, DynamicGeometry, shade, upsample_shade, sync_status, mc_irradiance,
                    compact_targets, training_samples, gbuffer_raycast, gbuffer_meshes, PRECISIONS)

__all__ = ["lib", "NivError", "LIB_PATH", "NIVModel", "NIVModule", "ProbeGrid", "DynamicGeometry", "shade", "upsample_shade",
           "sync_status",
           "mc_irradiance", "compact_targets", "training_samples", "gbuffer_raycast", "gbuffer_meshes", "PRECISIONS"]
