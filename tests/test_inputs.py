"""Pins for the seeded input generators shared by the oracle and the CUDA path."""
import os

import numpy as np
import pytest

import tbpm_inputs as ti

GOLD = os.path.join(os.path.dirname(__file__), "golden", "splitmix64.txt")


def test_splitmix64_reference_vectors():
    rows = [l.split() for l in open(GOLD) if l.strip() and not l.startswith("#")]
    for r in rows:
        seed, want = int(r[0]), [int(v) for v in r[1:]]
        got = [int(v) for v in ti.splitmix64(seed, [0, 1, 2])]
        assert got == want


def test_uniform_range_and_mean():
    u = ti.uniform01(5, np.arange(200000, dtype=np.uint64))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 5e-3


def test_random_phase_state_unit():
    psi = ti.random_phase_state(1000, 3)
    assert np.allclose(np.abs(psi), 1 / np.sqrt(1000), atol=1e-15)
    assert abs(np.vdot(psi, psi) - 1) < 1e-13
    blk = ti.random_phase_block(100, 4, seed0=7)
    assert np.array_equal(blk[:, 2], ti.random_phase_state(100, 9))


@pytest.mark.parametrize("l1,l2", [(3, 3), (4, 7), (5, 2)])
def test_graphene_structure(l1, l2):
    h = ti.graphene_csr(l1, l2)
    d = h.to_dense()
    assert h.n == 2 * l1 * l2
    assert np.allclose(d, d.conj().T)
    assert np.all(np.diff(h.row_ptr) == 3)
    assert abs(ti.gershgorin_bound(h) - 8.1) < 1e-12
    # columns sorted within rows
    for i in range(h.n):
        c = h.col[h.row_ptr[i]:h.row_ptr[i + 1]]
        assert np.all(np.diff(c) > 0)


def test_graphene_bloch_spectrum():
    """Eigenvalues of the periodic sample = +-|t f(k)| on the L1 x L2 k grid."""
    l1, l2, t = 6, 5, -2.7
    ev = np.linalg.eigvalsh(ti.graphene_csr(l1, l2).to_dense())
    q1, q2 = np.meshgrid(np.arange(l1) / l1, np.arange(l2) / l2, indexing="ij")
    f = 1 + np.exp(2j * np.pi * q1) + np.exp(2j * np.pi * q2)
    want = np.sort(np.concatenate([abs(t * f).ravel(), -abs(t * f).ravel()]))
    assert np.allclose(ev, want, atol=1e-12)


def test_bilayer_bloch_spectrum():
    """AB bilayer: eigenvalues +-t_perp/2 +- sqrt(t_perp^2/4 + |t f(k)|^2)."""
    l, t, tp = 4, -2.7, 0.39
    h = ti.bilayer_csr(l, l)
    d = h.to_dense()
    assert np.allclose(d, d.conj().T)
    counts = np.diff(h.row_ptr).reshape(-1, 4)
    assert np.all(counts == np.array([4, 3, 3, 4]))
    ev = np.linalg.eigvalsh(d)
    q1, q2 = np.meshgrid(np.arange(l) / l, np.arange(l) / l, indexing="ij")
    g = abs(t * (1 + np.exp(2j * np.pi * q1) + np.exp(2j * np.pi * q2))).ravel()
    r = np.sqrt(tp ** 2 / 4 + g ** 2)
    want = np.sort(np.concatenate([tp / 2 + r, tp / 2 - r, -tp / 2 + r, -tp / 2 - r]))
    assert np.allclose(ev, want, atol=1e-12)
    assert abs(ti.gershgorin_bound(h) - (8.1 + 0.39)) < 1e-12


def test_disorder_and_phases():
    eps = ti.anderson_onsite(50, 1.0, 1)
    assert eps.min() >= -0.5 and eps.max() < 0.5
    h = ti.graphene_csr(5, 5, onsite=eps, bond_phases=[0.2, 1.1, -0.7])
    d = h.to_dense()
    assert np.all(np.diff(h.row_ptr) == 4)
    assert np.allclose(np.diag(d).real, eps) and np.allclose(d, d.conj().T)
    assert not np.allclose(d, d.T)


def test_tiny_torus_merges_duplicates():
    h = ti.graphene_csr(1, 1)
    assert h.nnz == 2 and np.allclose(h.val, -8.1)


def test_random_hermitian():
    h = ti.random_hermitian_csr(40, 3, seed=11)
    d = h.to_dense()
    assert np.allclose(d, d.conj().T)
    assert np.all(np.imag(np.diag(d)) == 0)


def test_batch_recipe():
    b = ti.batch_instances(build=False)
    assert len(b) == 40
    assert all(1e4 * 0.5 <= i.n <= 4e6 * 1.05 for i in b)
    assert [i.kind for i in b[:4]] == ["monolayer", "bilayer", "monolayer", "bilayer"]
    assert all(i.rescale >= 9.0 for i in b)
