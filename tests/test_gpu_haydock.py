"""Haydock recursion and continued-fraction LDOS on the GPU against the oracle.

Bars: FP64 chain coefficients, LDOS and correlations within 1e-10 of the oracle
(measured on GB300: <= 1.2e-13 over 120 levels); FP32 coefficients within 1e-5
(measured 4.8e-7: FP32 rounding of the stored vectors, 2^-24 per sweep, grows along
the recursion), FP32 correlations within 3e-5 as in the FP32 tests."""
import numpy as np
import pytest

import tbpm_inputs as ti
import paper_2509_26309_gb300 as tb

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec,tol", [(tb.TBPM_FP64, 1e-10), (tb.TBPM_FP32, 1e-5)])
def test_haydock_coefficients(orc, prec, tol):
    h = ti.graphene_csr(40, 30, onsite=ti.anderson_onsite(2400, 1.0, 3), bond_phases=[0.2, 0.5, -0.3])
    ctx = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, 9.0, tb.make_opts(precision=prec))
    for psi0 in (ti.site_state(h.n, 77), ti.random_phase_state(h.n, 4)):
        a, b = tb.tbpm_haydock(ctx, psi0, 120)
        ra, rb = orc.haydock(h, psi0, 120)
        assert np.max(np.abs(a - ra)) <= tol and np.max(np.abs(b - rb)) <= tol


def test_haydock_1024x1024_and_ldos(orc):
    """Full 1024x1024 disordered graphene (the bench lattice), LDOS at one site."""
    n = 2 * 1024 * 1024
    h = ti.graphene_csr(1024, 1024, onsite=ti.anderson_onsite(n, 1.0, 1))
    ctx = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, 9.0)
    psi0 = ti.site_state(n, 123457)
    a, b = tb.tbpm_haydock(ctx, psi0, 60)
    ra, rb = orc.haydock(h, psi0, 60)
    assert np.max(np.abs(a - ra)) <= 1e-10 and np.max(np.abs(b - rb)) <= 1e-10
    E = np.linspace(-9, 9, 361)
    got = tb.tbpm_haydock_ldos(ctx, a, b, E, 0.1)
    ref = orc.haydock_ldos(ra, rb, E, 0.1)
    assert np.max(np.abs(got - ref)) <= 1e-10


def test_haydock_stencil_and_chain_stop(orc):
    eps = ti.anderson_onsite(2 * 12 * 10, 0.5, 5)
    h = ti.graphene_csr(12, 10, onsite=eps)
    ctx = tb.tbpm_create_lattice(tb.TBPM_LATTICE_GRAPHENE, 12, 10, -2.7, 0.0, eps, 9.0)
    psi0 = ti.site_state(h.n, 3)
    a, b = tb.tbpm_haydock(ctx, psi0, 80)
    ra, rb = orc.haydock(h, psi0, 80)
    assert np.max(np.abs(a - ra)) <= 1e-9 and np.max(np.abs(b - rb)) <= 1e-9
    # a 2-orbital system reaches an invariant subspace: later coefficients are 0
    h2 = ti.graphene_csr(1, 1)
    c2 = tb.tbpm_create(h2.n, h2.row_ptr, h2.col, h2.val, 9.0)
    a2, b2 = tb.tbpm_haydock(c2, ti.site_state(2, 0), 6)
    # (the GPU applies (rescale/2) * (2H/rescale), so the zero is exact only to rounding)
    assert abs(b2[0] - 8.1) < 1e-13 and np.all(b2[1:] == 0) and np.all(np.abs(a2) < 1e-12)
    # a long run past the end stays at exact zeros (no growth of the residual), FP64 and FP32
    for prec in (tb.TBPM_FP64, tb.TBPM_FP32):
        c3 = tb.tbpm_create(h2.n, h2.row_ptr, h2.col, h2.val, 9.0, tb.make_opts(precision=prec))
        a3, b3 = tb.tbpm_haydock(c3, ti.site_state(2, 0), 1500)
        assert np.all(np.isfinite(a3)) and np.all(np.isfinite(b3))
        assert np.all(b3[1:] == 0) and np.all(a3[2:] == 0) and abs(b3[0] - 8.1) < 1e-5


def test_haydock_deterministic_and_launch_order_neutral(orc):
    """Each pass's scalar is formed by whichever block finishes last, from the
    per-block sums added in block order: repeated calls, and plain stream order
    instead of programmatic launches, give the same bits."""
    n = 2 * 300 * 200
    h = ti.graphene_csr(300, 200, onsite=ti.anderson_onsite(n, 1.0, 8))
    psi0 = ti.random_phase_state(n, 9)
    runs = []
    for flags in (0, 0, tb.TBPM_F_NO_PDL):
        ctx = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, 9.0, tb.make_opts(flags=flags))
        runs.append(tb.tbpm_haydock(ctx, psi0, 200))
        tb.tbpm_destroy(ctx)
    for a, b in runs[1:]:
        assert np.array_equal(a, runs[0][0]) and np.array_equal(b, runs[0][1])
    ra, rb = orc.haydock(h, psi0, 200)
    assert np.max(np.abs(runs[0][0] - ra)) <= 1e-10 and np.max(np.abs(runs[0][1] - rb)) <= 1e-10


@pytest.mark.parametrize("prec,tol", [(tb.TBPM_FP64, 1e-10), (tb.TBPM_FP32, 1e-5)])
def test_quasi_eigenstates(orc, prec, tol):
    h = ti.graphene_csr(20, 16, onsite=ti.anderson_onsite(640, 1.0, 2), bond_phases=[0.3, -0.2, 0.9])
    psi0 = ti.random_phase_state(h.n, 3)
    dt = np.pi / 9
    E = np.array([-6.0, -2.5, 0.0, 0.7, 4.4])
    ctx = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, 9.0, tb.make_opts(precision=prec))
    got = tb.tbpm_quasi_eigenstates(ctx, psi0, dt, 150, E)
    ref = orc.quasi_eigenstates(h, 9.0, psi0, dt, 150, E)
    assert got.shape == (5, h.n)
    assert np.max(np.abs(got - ref)) <= tol
    # the ordinary correlation call still works on the same context afterwards
    c = tb.tbpm_dos_corr(ctx, psi0, dt, 20)
    assert np.max(np.abs(c - orc.dos_corr(h, 9.0, psi0, dt, 20))) <= (1e-10 if prec == tb.TBPM_FP64 else 3e-5)
    # the graphs of the first call serve a call with other energies of the same
    # count (read from device memory at run time); another dt or count rebuilds them
    E2 = E + 0.35
    got2 = tb.tbpm_quasi_eigenstates(ctx, psi0, dt, 150, E2)
    assert np.max(np.abs(got2 - orc.quasi_eigenstates(h, 9.0, psi0, dt, 150, E2))) <= tol
    got3 = tb.tbpm_quasi_eigenstates(ctx, psi0, 0.8 * dt, 40, E2[:3])
    assert np.max(np.abs(got3 - orc.quasi_eigenstates(h, 9.0, psi0, 0.8 * dt, 40, E2[:3]))) <= tol
    got4 = tb.tbpm_quasi_eigenstates(ctx, psi0, dt, 150, E)
    assert np.array_equal(got4, got)
