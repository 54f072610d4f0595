"""Seeded initial parameters: U(-r, r) grid features, He-normal weights, zero biases.

The number of grid values is passed in by the caller (it depends on the level
layout, which belongs to the method, not to this module).
"""
import numpy as np


def mlp_layer_shapes(n_in, width, n_hidden, n_out):
    """``[(out, in), ...]`` for ``n_hidden`` hidden layers of ``width`` and one output layer."""
    shapes = []
    k = n_in
    for _ in range(n_hidden):
        shapes.append((width, k))
        k = width
    shapes.append((n_out, k))
    return shapes


def init_params(n_grid_values, layer_shapes, seed=0, feat_range=1e-2, bias_std=0.0):
    """Flat float32 parameter vector ``[grid | W0 b0 | W1 b1 | ...]``.

    Grid values ~ U(-feat_range, feat_range); weights ~ N(0, 2/fan_in) (He);
    biases zero unless ``bias_std`` > 0, in which case ~ N(0, bias_std^2)
    (used by tests so that bias handling is exercised).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    parts = [rng.uniform(-feat_range, feat_range, size=int(n_grid_values))]
    for (out, fan_in) in layer_shapes:
        parts.append(rng.standard_normal(out * fan_in) * np.sqrt(2.0 / fan_in))
        if bias_std > 0.0:
            parts.append(rng.standard_normal(out) * bias_std)
        else:
            parts.append(np.zeros(out))
    return np.concatenate(parts).astype(np.float32)
