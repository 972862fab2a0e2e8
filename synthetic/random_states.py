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
