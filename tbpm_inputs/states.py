"""Random-phase initial states psi0 (the random-state trace estimate of TBPM, Sec. 3.2.3).

psi0_i = exp(2*pi*i*u_i) / sqrt(N) with u_i the SplitMix64 uniforms of stream
``seed``. State j of a block of B states uses seed ``seed0 + j``. The state is
generated here, on the host, and handed to both the oracle and the CUDA path.
"""
from __future__ import annotations

import numpy as np

from .rng import uniform01


def random_phase_state(n: int, seed: int) -> np.ndarray:
    """complex128[n], unit-modulus phases normalised to ||psi0|| = 1."""
    phi = 2.0 * np.pi * uniform01(seed, np.arange(n, dtype=np.uint64))
    return (np.cos(phi) + 1j * np.sin(phi)) / np.sqrt(n)


def random_phase_block(n: int, nstates: int, seed0: int = 0) -> np.ndarray:
    """complex128[n, nstates]: column j is ``random_phase_state(n, seed0 + j)``."""
    out = np.empty((n, nstates), dtype=np.complex128)
    for j in range(nstates):
        out[:, j] = random_phase_state(n, seed0 + j)
    return out


def site_state(n: int, site: int = 0) -> np.ndarray:
    """complex128[n] unit vector e_site."""
    v = np.zeros(n, dtype=np.complex128)
    v[site] = 1.0
    return v
