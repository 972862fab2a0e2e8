"""Seeded random inputs: displacement fields and integration-point states.

Used by both the oracle tests and the GPU parity tests so that the two sides
see identical inputs.  Nothing here evaluates the constitutive model; the
draws only set magnitudes so that a mix of elastic and plastic points arises.
"""
from __future__ import annotations

import numpy as np


def rng(seed: int) -> np.random.Generator:
    return np.random.default_rng(seed)


def random_displacement(coords: np.ndarray, dirichlet: np.ndarray, scale: float, seed: int,
                        affine: float = 1.0) -> np.ndarray:
    """A smooth-plus-noise displacement field [n_n*dim] with zeros on prescribed DOFs.

    The field is an affine map of the coordinates (amplitude `affine*scale`) plus
    independent Gaussian noise per DOF (amplitude `scale`), then multiplied by
    the free mask.
    """
    g = rng(seed)
    n, d = coords.shape
    A = g.standard_normal((d, d)) * affine * scale
    u = coords @ A.T + g.standard_normal((n, d)) * scale
    return (u.ravel() * (1 - dirichlet.astype(np.float64)))


def random_strains(n: int, n_comp: int, scale: float, seed: int) -> np.ndarray:
    """Strain-type Voigt vectors [n_comp][n] with Gaussian entries of std `scale`."""
    g = rng(seed)
    return g.standard_normal((n_comp, n)) * scale


def random_state(n_int: int, n_comp: int, scale: float, seed: int, hard_scale: float = 0.0):
    """Plastic strain [n_comp][n_int] (strain-type) and hardening variable [n_int] >= 0."""
    g = rng(seed)
    ep = g.standard_normal((n_comp, n_int)) * scale
    alpha = np.abs(g.standard_normal(n_int)) * hard_scale
    return ep, alpha


def mlp_init(seed: int = 0, out_scale: float = 0.1, bias_scale: float = 0.0) -> np.ndarray:
    """Initial parameters of the 16 -> 128 -> 128 -> 4 warm-start network as one float32 vector in
    the order W1 [128][16], b1, W2 [128][128], b2, W3 [4][128], b3: weights uniform in
    +-sqrt(6 / fan_in) (the last layer scaled by `out_scale`), biases uniform in +-bias_scale."""
    g = rng(seed)
    parts = []
    for fan_out, fan_in, sc in ((128, 16, 1.0), (128, 128, 1.0), (4, 128, out_scale)):
        a = np.sqrt(6.0 / fan_in) * sc
        parts.append(g.uniform(-a, a, fan_out * fan_in))
        parts.append(g.uniform(-bias_scale, bias_scale, fan_out) if bias_scale > 0 else np.zeros(fan_out))
    return np.concatenate(parts).astype(np.float32)


def mlp_rows(n: int, seed: int, n_in: int = 16, n_out: int = 4):
    """Random (X [n][n_in], T [n][n_out]) float32 rows: standard normal inputs, targets with three
    normal components and a fourth in [0, 1]."""
    g = rng(seed)
    X = g.standard_normal((n, n_in)).astype(np.float32)
    T = np.concatenate([g.standard_normal((n, n_out - 1)), g.uniform(0, 1, (n, 1))], axis=1).astype(np.float32)
    return X, T
