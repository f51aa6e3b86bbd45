"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds no arithmetic of the transform itself: it only draws the
random coefficient sets and maps that both the CUDA path and the CPU oracle are
fed, and spells out the storage layout of a_lm.

Workload recipe (the paper transforms "a single set of standard Gaussian
coefficients", Sec. 3.2 / Table accuracy; the spectrum here follows the
benchmark configurations of this project): Re a_lm and Im a_lm are i.i.d.
N(0, C_l / 2) with C_l = 1/(l+1)^2, Im a_l0 = 0, drawn with numpy's
Generator(PCG64(seed + map_index)).
"""
from __future__ import annotations

import numpy as np


def nalm(lmax: int) -> int:
    """Stored coefficients per map: l = 0..L, m = 0..l, i.e. (L+1)(L+2)/2."""
    return (lmax + 1) * (lmax + 2) // 2


def alm_index(lmax: int, l, m):
    """Position of a_lm in the m-major layout (l = m..L contiguous per m)."""
    return m * (2 * lmax + 1 - m) // 2 + l


def l_of_index(lmax: int) -> np.ndarray:
    """l for every stored position."""
    return np.concatenate([np.arange(m, lmax + 1) for m in range(lmax + 1)])


def m_of_index(lmax: int) -> np.ndarray:
    """m for every stored position."""
    return np.concatenate([np.full(lmax + 1 - m, m) for m in range(lmax + 1)])


def gaussian_alm(lmax: int, nmaps: int = 1, seed: int = 0) -> np.ndarray:
    """complex128 [nmaps, nalm]: Re, Im ~ N(0, C_l/2), C_l = 1/(l+1)^2, Im a_l0 = 0."""
    l = l_of_index(lmax)
    m = m_of_index(lmax)
    sd = np.sqrt(0.5) / (l + 1.0)
    out = np.empty((nmaps, l.size), dtype=np.complex128)
    for b in range(nmaps):
        rng = np.random.Generator(np.random.PCG64(seed + b))
        re = rng.standard_normal(l.size) * sd
        im = rng.standard_normal(l.size) * sd
        im[m == 0] = 0.0
        out[b] = re + 1j * im
    return out


def gaussian_map(npix: int, nmaps: int = 1, seed: int = 0, sigma: float = 1.0) -> np.ndarray:
    """float64 [nmaps, npix] of i.i.d. N(0, sigma^2) pixels (white noise)."""
    out = np.empty((nmaps, npix))
    for b in range(nmaps):
        rng = np.random.Generator(np.random.PCG64(seed + b))
        out[b] = rng.standard_normal(npix) * sigma
    return out
