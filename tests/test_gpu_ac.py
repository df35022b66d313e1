"""AC conductivity on the GPU (Fermi-operator series, current operators, the
current-current correlation of three propagated states, the windowed
transform) against the FP64 oracle on the same seeded inputs."""
import math

import numpy as np
import pytest

import tbpm_inputs as ti
import paper_2509_26309_gb300 as tb

pytestmark = pytest.mark.gpu
TOL = 1e-10
KCAP = tb.TBPM_FERMI_MAX_TERMS


def make(case):
    if case == "graphene_8x8":
        n = 2 * 8 * 8
        return ti.graphene_csr(8, 8, onsite=ti.anderson_onsite(n, 1.0, 11)), ti.graphene_current(8, 8)
    if case == "bilayer_5x5":
        n = 4 * 5 * 5
        return ti.bilayer_csr(5, 5, onsite=ti.anderson_onsite(n, 2.0, 12)), ti.bilayer_current(5, 5)
    if case == "phases_6x7":
        ph = np.array([0.4, -0.9, 1.3])
        n = 2 * 6 * 7
        return (ti.graphene_csr(6, 7, onsite=ti.anderson_onsite(n, 0.5, 13), bond_phases=ph),
                ti.graphene_current(6, 7, bond_phases=ph))
    if case == "graphene_40x37":
        n = 2 * 40 * 37
        return ti.graphene_csr(40, 37, onsite=ti.anderson_onsite(n, 1.0, 14)), ti.graphene_current(40, 37)
    raise ValueError(case)


def ctx_for(h, cur, rescale, **kw):
    ctx = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, rescale, tb.make_opts(**kw))
    tb.tbpm_set_current(ctx, *cur.as_tuple())
    return ctx


@pytest.mark.parametrize("case,beta,mu,dt,steps", [
    ("graphene_8x8", 8.0, 0.3, math.pi / 9.0, 40),
    ("bilayer_5x5", 5.0, -0.6, 0.5, 33),
    ("phases_6x7", 12.0, 0.0, 0.35, 20),
    ("graphene_40x37", 10.0, 0.2, math.pi / 9.0, 24),
])
def test_ac_corr_matches_oracle(orc, case, beta, mu, dt, steps):
    h, cur = make(case)
    rescale = max(9.0, 1.02 * ti.gershgorin_bound(h))
    psi0 = ti.random_phase_state(h.n, 21)
    ctx = ctx_for(h, cur, rescale)
    c = tb.tbpm_ac_corr(ctx, psi0, beta, mu, dt, steps)
    kf, ref = orc.ac_corr(h, cur.as_tuple(), rescale, psi0, beta, mu, dt, steps, kcap=KCAP)
    assert c.shape == (4, steps + 1)
    assert np.max(np.abs(c - ref)) <= TOL, np.max(np.abs(c - ref))
    assert tb.tbpm_get_info(ctx)["fermi_terms"] == kf
    assert np.max(np.abs(ref)) > 1e-3
    # a second call reuses the cached Fermi series and the graphs: same result
    c2 = tb.tbpm_ac_corr(ctx, psi0, beta, mu, dt, steps)
    assert np.array_equal(c, c2)


def test_ac_room_temperature_series(orc):
    """beta = 1/(k_B 300 K) on rescale 9: a Fermi series of about 2.6k terms."""
    h, cur = make("graphene_8x8")
    psi0 = ti.random_phase_state(h.n, 3)
    beta = 1.0 / 0.025852
    ctx = ctx_for(h, cur, 9.0)
    c = tb.tbpm_ac_corr(ctx, psi0, beta, 0.1, math.pi / 9.0, 12)
    kf, ref = orc.ac_corr(h, cur.as_tuple(), 9.0, psi0, beta, 0.1, math.pi / 9.0, 12, kcap=KCAP)
    assert 2000 < kf < KCAP
    assert np.max(np.abs(c - ref)) <= TOL


def test_ac_device_buffers_and_stencil_path(orc):
    torch = pytest.importorskip("torch")
    l1, l2 = 9, 12
    n = 2 * l1 * l2
    eps = ti.anderson_onsite(n, 1.0, 5)
    h = ti.graphene_csr(l1, l2, onsite=eps)
    cur = ti.graphene_current(l1, l2)
    psi0 = ti.random_phase_state(n, 8)
    ctx = ctx_for(h, cur, 9.0)
    host = tb.tbpm_ac_corr(ctx, psi0, 6.0, 0.4, 0.3, 30)
    dev = tb.tbpm_ac_corr(ctx, torch.from_numpy(psi0).cuda(), 6.0, 0.4, 0.3, 30)
    assert dev.is_cuda
    assert np.array_equal(dev.cpu().numpy(), host)
    # the matrix-free lattice operator with the same current operators
    st = tb.tbpm_create_lattice(tb.TBPM_LATTICE_GRAPHENE, l1, l2, ti.T_GRAPHENE, 0.0, eps, 9.0,
                                tb.make_opts(path=tb.TBPM_PATH_STENCIL))
    tb.tbpm_set_current(st, *cur.as_tuple())
    cs = tb.tbpm_ac_corr(st, psi0, 6.0, 0.4, 0.3, 30)
    _, ref = orc.ac_corr(h, cur.as_tuple(), 9.0, psi0, 6.0, 0.4, 0.3, 30, kcap=KCAP)
    assert np.max(np.abs(cs - ref)) <= TOL
    assert np.max(np.abs(host - ref)) <= TOL


def test_ac_cond_matches_oracle(orc):
    h, cur = make("bilayer_5x5")
    rescale = max(9.0, 1.02 * ti.gershgorin_bound(h))
    psi0 = ti.random_phase_state(h.n, 4)
    ctx = ctx_for(h, cur, rescale)
    dt, beta = 0.4, 5.0
    c = tb.tbpm_ac_corr(ctx, psi0, beta, 0.0, dt, 256)
    w = np.linspace(0.0, 8.0, 161)
    area = ti.graphene_area_per_orbital() / 2
    sg = tb.tbpm_ac_cond(ctx, c, dt, beta, area, w)
    assert sg.shape == (4, w.size)
    for q in range(4):
        ref = orc.ac_cond(c[q], dt, beta, area, w)
        scale = np.max(np.abs(ref)) + 1e-300
        assert np.max(np.abs(sg[q] - ref)) <= 1e-12 * scale, q
    assert np.all(sg[:, 0] == 0.0)
    assert np.max(sg[0]) > 0                          # sigma_xx absorbs


def test_ac_errors():
    h, cur = make("graphene_8x8")
    psi0 = ti.random_phase_state(h.n, 1)
    ctx = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, 9.0)
    with pytest.raises(tb.TbpmError) as e:
        tb.tbpm_ac_corr(ctx, psi0, 5.0, 0.0, 0.3, 4)              # no current operators
    assert e.value.status == tb.TBPM_ERR_ARG
    assert "tbpm_set_current" in tb.tbpm_last_error(ctx)
    assert "no current operators" in str(e.value)                 # the detail rides on the exception
    tb.tbpm_set_current(ctx, *cur.as_tuple())
    with pytest.raises(tb.TbpmError) as e:
        tb.tbpm_ac_corr(ctx, psi0, 5000.0, 0.0, 0.3, 4)           # Fermi series too long
    assert e.value.status == tb.TBPM_ERR_ARG
    assert "TBPM_FERMI_MAX_TERMS" in tb.tbpm_last_error(ctx)
    bad = cur.jx.copy()
    bad[0] += 0.5                                                  # breaks J_x = J_x^dagger
    with pytest.raises(tb.TbpmError) as e:
        tb.tbpm_set_current(ctx, cur.row_ptr, cur.col, bad, cur.jy)
    assert e.value.status == tb.TBPM_ERR_NOT_HERMITIAN
    c32 = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, 9.0, tb.make_opts(precision=tb.TBPM_FP32))
    with pytest.raises(tb.TbpmError) as e:
        tb.tbpm_set_current(c32, *cur.as_tuple())
    assert e.value.status == tb.TBPM_ERR_UNSUPPORTED
    # the earlier current operators survive a rejected replacement
    c = tb.tbpm_ac_corr(ctx, psi0, 5.0, 0.0, 0.3, 4)
    assert np.all(np.isfinite(c))


def test_ac_zero_steps(orc):
    """n_steps = 0 gives C_ab(0) only: <phi|f J_a [1 - f] J_b|phi>."""
    h, cur = make("graphene_8x8")
    psi0 = ti.random_phase_state(h.n, 5)
    ctx = ctx_for(h, cur, 9.0)
    c = tb.tbpm_ac_corr(ctx, psi0, 7.0, -0.2, 0.3, 0)
    _, ref = orc.ac_corr(h, cur.as_tuple(), 9.0, psi0, 7.0, -0.2, 0.3, 0, kcap=KCAP)
    assert c.shape == (4, 1)
    assert np.max(np.abs(c - ref)) <= TOL
