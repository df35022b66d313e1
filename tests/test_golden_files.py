"""The stored full-size oracle results (tests/golden/oracle_*.txt) against the
live oracle: the first steps or moments recomputed now must agree with the file,
so the files cannot drift from oracle.c or from the input recipes. The oracle's
results do not depend on its thread count (each row of a product is formed by
one thread in a fixed order; the dot is serial), so the agreement is to
rounding of the 17-digit text."""
import math
import os

import numpy as np
import pytest

import tbpm_inputs as ti

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
DT = math.pi / 9.0


def _lattice(l):
    n = 2 * l * l
    return ti.graphene_csr(l, l, onsite=ti.anderson_onsite(n, 1.0, 1))


@pytest.mark.parametrize("name,l,kind,prefix,length", [
    ("graphene1024_dos2048", 1024, "dos", 3, 2048),
    ("graphene1024_kpm4096", 1024, "kpm", 24, 4096),
    ("graphene2048_dos1024", 2048, "dos", 2, 1024),
])
def test_stored_results_match_the_oracle(orc, golden, name, l, kind, prefix, length):
    stored = golden(name)
    assert stored.size == (length + 1 if kind == "dos" else length)
    head = open(os.path.join(HERE, f"oracle_{name}_s0.txt")).read(600)
    assert f"graphene {l}x{l} cells" in head and "seed 0" in head
    h = _lattice(l)
    psi0 = ti.random_phase_state(h.n, 0)
    if kind == "dos":
        live = orc.dos_corr(h, 9.0, psi0, DT, prefix)
        assert np.max(np.abs(live - stored[:prefix + 1])) <= 1e-15
        assert abs(stored[0] - 1.0) <= 1e-14 and np.all(np.abs(stored) <= 1.0 + 1e-12)
    else:
        live = orc.kpm_moments(h, 9.0, psi0, prefix)
        assert np.max(np.abs(live - stored[:prefix])) <= 1e-15
        assert np.all(np.abs(stored.real) <= 1.0 + 1e-12)


def test_state_15_file_describes_its_state():
    head = open(os.path.join(HERE, "oracle_graphene4096_dos128_s15.txt")).read(600)
    assert "graphene 4096x4096 cells" in head and "state seed 15" in head
    a = np.loadtxt(os.path.join(HERE, "oracle_graphene4096_dos128_s15.txt"), comments="#")
    assert a.shape == (129, 2) and abs(a[0, 0] - 1.0) <= 1e-14 and abs(a[0, 1]) <= 1e-14
