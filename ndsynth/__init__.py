"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle.

This module holds no arithmetic of the method: it only draws random numbers
(numpy's PCG64 with a fixed seed) in the shapes the method consumes.  Each side
applies its own disk mask, units and physics.
"""
from __future__ import annotations

import numpy as np

# Permalloy-like material of the paper's simulations (Section III.A).
MATERIAL = dict(Ms=8.6e5, A=1.3e-11, gamma=1.76e11, a=2.0e-9)


def random_unit_vectors(D: int, seed: int = 0, batch: int | None = None) -> np.ndarray:
    """Isotropic random unit vectors on a D x D grid, shape (3, D, D) or
    (batch, 3, D, D), float64.  A white spectrum: the FFT's worst case."""
    rng = np.random.default_rng(seed)
    shape = (3, D, D) if batch is None else (batch, 3, D, D)
    v = rng.standard_normal(shape)
    ax = 0 if batch is None else 1
    return v / np.linalg.norm(v, axis=ax, keepdims=True)


def perturbed(m: np.ndarray, eps: float, seed: int = 1) -> np.ndarray:
    """m plus eps times an isotropic Gaussian perturbation (not renormalised)."""
    rng = np.random.default_rng(seed)
    return m + eps * rng.standard_normal(m.shape)


def seeds(n: int, start: int = 0) -> np.ndarray:
    """Per-replica noise seeds start..start+n-1 (uint64)."""
    return np.arange(start, start + n, dtype=np.uint64)


def uneven_disks(n: int, seed: int = 0, n_cold: int = 8):
    """A batch of n disks with R ~ U(20, 100) nm, L/R ~ U(0.05, 0.2) and
    T ~ U(0, 400) K; the first n_cold disks at T = 0."""
    rng = np.random.default_rng(seed)
    R = rng.uniform(20e-9, 100e-9, n)
    L = R * rng.uniform(0.05, 0.2, n)
    T = rng.uniform(0.0, 400.0, n)
    T[:n_cold] = 0.0
    return R, L, T


def sample_cells(D: int, k: int, seed: int = 0) -> np.ndarray:
    """k distinct flat cell indices in [0, D*D) (for sampled checks)."""
    rng = np.random.default_rng(seed)
    return rng.choice(D * D, size=k, replace=False)


def sample_indices(n: int, k: int, seed: int = 0) -> np.ndarray:
    """k distinct indices in [0, n)."""
    rng = np.random.default_rng(seed)
    return rng.choice(n, size=k, replace=False)
