"""The uneven multi-lattice batch: 40 seeded lattices with N log-uniform in [1e4, 4e6].

Instance idx (0-based) draws u_N = U(seed 77, 2*idx) and u_W = U(seed 77, 2*idx+1)
from the SplitMix64 stream; log10 N = 4 + u_N*(log10(4e6) - 4). Even idx is a
monolayer with L = round(sqrt(N/2)), odd idx an AB bilayer with
L = round(sqrt(N/4)); W = 2*u_W eV, disorder seed 1000 + idx, and
rescale = max(9, 1.02 * Gershgorin bound) rounded to 1e-9 eV so that ||H~|| <= 1 for every
instance. These are input recipes only.
"""
from __future__ import annotations

from dataclasses import dataclass
import math

import numpy as np

from .lattice import (CSR, T_GRAPHENE, T_PERP_AB, anderson_onsite, bilayer_csr, graphene_csr,
                      gershgorin_bound)
from .rng import uniform01


@dataclass
class Instance:
    idx: int
    kind: str          # "monolayer" | "bilayer"
    l: int
    n: int
    w: float
    seed: int
    rescale: float
    csr: CSR | None = None


def batch_instances(count: int = 40, nmin: float = 1e4, nmax: float = 4e6,
                    build: bool = True, scale_n: float = 1.0) -> list[Instance]:
    """The batch recipe; ``scale_n`` < 1 shrinks every N for quick tests."""
    out = []
    for idx in range(count):
        u_n = float(uniform01(77, [2 * idx])[0])
        u_w = float(uniform01(77, [2 * idx + 1])[0])
        n_target = 10.0 ** (math.log10(nmin) + u_n * (math.log10(nmax) - math.log10(nmin)))
        n_target *= scale_n
        kind = "monolayer" if idx % 2 == 0 else "bilayer"
        per_cell = 2 if kind == "monolayer" else 4
        l = max(3, int(round(math.sqrt(n_target / per_cell))))
        n = per_cell * l * l
        w = 2.0 * u_w
        seed = 1000 + idx
        inst = Instance(idx, kind, l, n, w, seed, 0.0)
        eps = anderson_onsite(n, w, seed)
        if build:
            h = graphene_csr(l, l, onsite=eps) if kind == "monolayer" else bilayer_csr(l, l, onsite=eps)
            inst.csr = h
            bound = gershgorin_bound(h)
        else:
            # the same row sums without assembling the matrix
            row = np.full(n, 3 * abs(T_GRAPHENE)) + np.abs(eps)
            if kind == "bilayer":
                row[0::4] += abs(T_PERP_AB)
                row[3::4] += abs(T_PERP_AB)
            bound = float(row.max())
        inst.rescale = max(9.0, round(1.02 * bound, 9))
        out.append(inst)
    return out
