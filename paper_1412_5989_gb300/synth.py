"""Seeded synthetic inputs shared by the CUDA path, the oracle and the benchmark.

This module holds none of the method's arithmetic: it only draws numbers.
A two-body table is one float32 draw per packed table entry, in table order,
from numpy's PCG64 generator seeded with the set's seed; the table length is
supplied by the caller (each side derives it from its own layout).
"""
from __future__ import annotations

import numpy as np


def tbme_table(length: int, seed: int) -> np.ndarray:
    """One synthetic two-body table: ``length`` standard-normal float32 draws."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(length).astype(np.float32)


def tbme_tables(length: int, seeds) -> np.ndarray:
    """K tables, set-major, shape (K, length)."""
    seeds = list(seeds)
    out = np.empty((len(seeds), length), dtype=np.float32)
    for k, s in enumerate(seeds):
        out[k] = tbme_table(length, s)
    return out


def single_particle_energies(n: int, seed: int, scale: float = 10.0) -> np.ndarray:
    """Per-orbital one-body energies (float64), uniform in [0, scale)."""
    return np.random.Generator(np.random.PCG64(seed)).uniform(0.0, scale, n)


def onebody_table(length: int, seed: int) -> np.ndarray:
    """One synthetic one-body table: ``length`` standard-normal float64 draws,
    one per packed table entry in table order (the caller's layout)."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(length)
