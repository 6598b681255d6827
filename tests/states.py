"""Seeded synthetic states for the tests (test code only).

The conserved vector of Eq. 2 (energy per unit volume, reading R2) is formed
here from primitive fields, so that the tests can build the same input for
the oracle and for the CUDA path.  Neither the product package nor the oracle
imports this module.
"""
from __future__ import annotations

import numpy as np


def smooth_field(shape, rng, modes: int = 3, amp: float = 1.0):
    """Sum of a few random periodic Fourier modes on an index-periodic box
    (shape = (nk, nj, ni))."""
    nk, nj, ni = shape
    k, j, i = np.meshgrid(np.arange(nk), np.arange(nj), np.arange(ni), indexing="ij")
    out = np.zeros(shape)
    for _ in range(modes):
        a, b, c = rng.integers(0, 3, size=3)
        ph = rng.uniform(0, 2 * np.pi)
        out += rng.uniform(-amp, amp) * np.cos(2 * np.pi * (a * i / ni + b * j / nj + c * k / nk) + ph)
    return out


def primitive_to_conserved(rho, u, v, w, p, gamma=1.4):
    """Conserved vector [rho, rho u, rho v, rho w, p/(gamma-1) + rho |u|^2 / 2]."""
    return np.stack([rho, rho * u, rho * v, rho * w, p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w)])


def random_state(shape, seed: int, noise: float = 0.02, gamma: float = 1.4, mach: float = 1.4):
    """Noisy jet-like state on an index-periodic box: smooth density,
    pressure and velocity fields plus white noise.  Returns (5, nk, nj, ni)."""
    rng = np.random.default_rng(seed)
    rho = 1.0 + 0.1 * smooth_field(shape, rng) + noise * rng.uniform(-1, 1, shape)
    p = (1.0 + 0.1 * smooth_field(shape, rng) + noise * rng.uniform(-1, 1, shape)) / gamma
    u = mach * (0.5 + 0.3 * smooth_field(shape, rng)) + noise * rng.uniform(-1, 1, shape)
    v = 0.2 * smooth_field(shape, rng) + noise * rng.uniform(-1, 1, shape)
    w = 0.2 * smooth_field(shape, rng) + noise * rng.uniform(-1, 1, shape)
    return primitive_to_conserved(rho, u, v, w, p, gamma)
