"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds no arithmetic of the method: it only draws random numbers and lays them out.
Both sides receive the same arrays, so the choice of generator never affects parity.
"""
from __future__ import annotations

import numpy as np


def initial_density(n_nodes: int, amplitude: float, seed: int, rho0: float = 1.0) -> np.ndarray | None:
    """rho(n) = rho0 (1 + U(-amplitude, amplitude)) per node (node order x fastest); None if amplitude == 0."""
    if amplitude == 0.0:
        return None
    rng = np.random.Generator(np.random.PCG64(seed))
    return rho0 * (1.0 + rng.uniform(-amplitude, amplitude, size=n_nodes))


def kappa_sequence(T: int, n_nodes: int, d: int, scale: float, seed: int, shear: float = 0.0) -> np.ndarray:
    """Prescribed velocity-gradient history [T, n_nodes, d, d]: a constant simple shear `shear` e_xy plus
    a smooth random perturbation of size `scale` (a random walk in time, so kappa varies slowly like a
    flow that develops)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    steps = rng.normal(size=(T, n_nodes, d, d)) * (scale / np.sqrt(max(T, 1)))
    k = np.cumsum(steps, axis=0)
    k += rng.normal(size=(1, n_nodes, d, d)) * scale
    k[:, :, 0, 1] += shear
    return k


def channel_widths(n_channels: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Widths log-uniform in [lo, hi], rounded to even integers."""
    rng = np.random.Generator(np.random.PCG64(seed))
    w = np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_channels))
    return np.clip(2 * np.round(w / 2), lo, hi).astype(int)


def uniform_params(n: int, bounds: dict, seed: int) -> dict:
    """Independent uniform draws per key: bounds = {name: (lo, hi)}."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return {k: rng.uniform(lo, hi, size=n) for k, (lo, hi) in bounds.items()}


def perturbed(values, seed: int, frac: float = 0.1) -> np.ndarray:
    """values with each component scaled by (1 + frac) or (1 - frac), the signs drawn from `seed`."""
    rng = np.random.Generator(np.random.PCG64(seed))
    signs = rng.choice([-1.0, 1.0], size=len(values))
    return np.asarray(values, dtype=np.float64) * (1.0 + frac * signs)
