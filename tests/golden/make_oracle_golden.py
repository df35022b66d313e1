"""Writes the oracle's results for the full-size workloads to tests/golden/.

The GPU parity tests and the bench's accuracy fields compare against these
files instead of re-running the FP64 oracle for minutes on every call. Every
value here comes from the oracle (oracle/oracle.c: the forward Chebyshev
recurrence of Sec. 2.2.1 with separate arrays, a serial FP64 dot for C(t),
plain non-doubling KPM moments) on the seeded inputs of tbpm_inputs/; nothing
is taken from the CUDA path.

  python tests/golden/make_oracle_golden.py [name ...]    (default: all)

Workloads (graphene with Anderson disorder W = 1 eV from SplitMix64 seed 1,
rescale 9 eV, dt = pi/9, random-phase state seed 0 unless stated):
  graphene1024_dos2048   1024x1024 cells, C(t_n) for n = 0..2048
  graphene1024_kpm4096   1024x1024 cells, mu_m for m = 0..4095
  graphene2048_dos1024   2048x2048 cells, C(t_n) for n = 0..1024
  graphene4096_dos128    4096x4096 cells, C(t_n) for n = 0..128, states 0 and 15
"""
from __future__ import annotations

import math
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

RESCALE = 9.0
DT = math.pi / 9.0
W = 1.0

# name: (cells per side, kind, length, states)
WORKLOADS = {
    "graphene1024_dos2048": (1024, "dos", 2048, (0,)),
    "graphene1024_kpm4096": (1024, "kpm", 4096, (0,)),
    "graphene2048_dos1024": (2048, "dos", 1024, (0,)),
    "graphene4096_dos128": (4096, "dos", 128, (0, 15)),
}


def path(name: str, state: int = 0) -> str:
    return os.path.join(HERE, f"oracle_{name}_s{state}.txt")


def load(name: str, state: int = 0) -> np.ndarray:
    """The stored complex128 values of one workload and state."""
    a = np.loadtxt(path(name, state), comments="#")
    return a[:, 0] + 1j * a[:, 1]


def lattice(l: int):
    import tbpm_inputs as ti
    n = 2 * l * l
    return ti.graphene_csr(l, l, onsite=ti.anderson_onsite(n, W, 1))


def write(name: str) -> None:
    import oracle
    import tbpm_inputs as ti
    l, kind, length, states = WORKLOADS[name]
    h = lattice(l)
    for s in states:
        psi0 = ti.random_phase_state(h.n, s)
        t0 = time.perf_counter()
        if kind == "dos":
            vals = oracle.dos_corr(h, RESCALE, psi0, DT, length)
            what = f"C(t_n) = <psi0|psi(t_n)>, n = 0..{length}, dt = pi/9"
        else:
            vals = oracle.kpm_moments(h, RESCALE, psi0, length)
            what = f"mu_m = <psi0|T_m(H/rescale)|psi0>, m = 0..{length - 1}"
        el = time.perf_counter() - t0
        head = (f"oracle (oracle/oracle.c, FP64), {what}\n"
                f"graphene {l}x{l} cells (N = {h.n}), Anderson W = {W} eV (SplitMix64 seed 1), "
                f"t = -2.7 eV, rescale {RESCALE} eV, random-phase state seed {s}\n"
                f"written by tests/golden/make_oracle_golden.py {name} "
                f"({el:.0f} s on {oracle.get_threads()} threads)\n"
                f"columns: real imag")
        np.savetxt(path(name, s), np.stack([vals.real, vals.imag], axis=1), fmt="%.17e", header=head)
        print(f"{name} state {s}: {el:.1f} s", flush=True)


if __name__ == "__main__":
    for nm in sys.argv[1:] or list(WORKLOADS):
        write(nm)
