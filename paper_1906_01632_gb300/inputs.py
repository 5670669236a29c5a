"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds random draws only -- none of the method's arithmetic.  The
porosity formulas, Kozeny-Carman and everything downstream are computed
separately by the oracle and by the CUDA kernels from these draws.

* ``sobol_xi``: scrambled Sobol points mapped to [-1, 1]^3 (the stochastic
  parameters xi of the qMC sampling of Section 3 / Section 5.3; a scrambled
  Sobol sequence stands in for the paper's Halton points).
* ``halton_xi``: the paper's own Halton points on [-1, 1]^3 (Section 5.3).
* ``lognormal_z``: iid standard normals, one per cell, for a lognormal
  porosity field.
* ``fd_cells``: distinct cell indices for finite-difference checks.
"""
from __future__ import annotations

import numpy as np
import torch


def sobol_xi(n: int, seed: int = 0) -> np.ndarray:
    eng = torch.quasirandom.SobolEngine(3, scramble=True, seed=seed)
    u = eng.draw(n, dtype=torch.float64).numpy()
    return np.ascontiguousarray(2.0 * u - 1.0)


def _radical_inverse(i: int, base: int) -> float:
    f, r = 1.0, 0.0
    while i > 0:
        f /= base
        r += f * (i % base)
        i //= base
    return r


def halton_xi(n: int, skip: int = 1) -> np.ndarray:
    pts = np.array([[_radical_inverse(i + skip, b) for b in (2, 3, 5)] for i in range(n)])
    return np.ascontiguousarray(2.0 * pts - 1.0)


def lognormal_z(n_cells: int, seed: int = 1) -> np.ndarray:
    g = torch.Generator().manual_seed(seed)
    return torch.randn(n_cells, generator=g, dtype=torch.float64).numpy().copy()


def fd_cells(n_cells: int, count: int = 32, seed: int = 2) -> np.ndarray:
    g = torch.Generator().manual_seed(seed)
    return torch.randperm(n_cells, generator=g)[:count].numpy().copy()
