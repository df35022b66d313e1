"""CUDA path vs the FP64 oracle on the same seeded inputs, through the C ABI.

Tolerance: |dC| <= 1e-10 and |dmu| <= 1e-10 for the FP64 path. Both sides use
the same truncated series; what differs is the summation (Clenshaw on the GPU,
forward recurrence in the oracle), the Bessel method (Miller's recurrence vs
the power series) and the rounding order of the sums, each of order 1e-16 per
operation, far below 1e-10 over 10^4 sweeps.
"""
import math

import numpy as np
import pytest

import tbpm_inputs as ti
import paper_2509_26309_gb300 as tb

pytestmark = pytest.mark.gpu
DT = math.pi / 9
TOL = 1e-10


def create(h, rescale=9.0, **kw):
    return tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, rescale, tb.make_opts(**kw))


def test_pristine_64x64_1024_steps(orc):
    """64x64 pristine graphene, psi0 seed 0, 1024 steps of pi/9, K = 18."""
    h = ti.graphene_csr(64, 64)
    psi0 = ti.random_phase_state(h.n, 0)
    ctx = create(h)
    c = tb.tbpm_dos_corr(ctx, psi0, DT, 1024)
    ref = orc.dos_corr(h, 9.0, psi0, DT, 1024)
    assert tb.tbpm_get_info(ctx)["num_terms"] == 18
    assert np.max(np.abs(c - ref)) <= TOL
    c2 = tb.tbpm_dos_corr(ctx, psi0, DT, 1024)
    assert np.array_equal(c, c2)                      # deterministic reductions


@pytest.mark.parametrize("maker,prec", [
    (lambda: ti.graphene_csr(64, 64), tb.TBPM_FP64),
    (lambda: ti.random_hermitian_csr(3000, 4, seed=4, scale=1.0), tb.TBPM_FP64),
    (lambda: ti.bilayer_csr(64, 64, onsite=ti.anderson_onsite(16384, 1.0, 2)), tb.TBPM_FP64),
    (lambda: ti.graphene_csr(100, 90, onsite=ti.anderson_onsite(18000, 1.0, 2)), tb.TBPM_FP32),
    # 4096 rows per CTA: the vectors fill shared memory, the matrix stays in global memory
    (lambda: ti.graphene_csr(160, 160, onsite=ti.anderson_onsite(51200, 1.0, 5)), tb.TBPM_FP64),
])
def test_cluster_path_matches_graph_path(orc, maker, prec):
    """Small systems run all steps in one launch of one thread-block cluster; the
    per-row arithmetic and the per-slice reduction are those of the graph path."""
    h = maker()
    rescale = max(9.0, 1.02 * ti.gershgorin_bound(h))
    dt = math.pi / rescale
    psi0 = ti.random_phase_state(h.n, 2)
    a = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, rescale, tb.make_opts(precision=prec))
    b = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, rescale,
                       tb.make_opts(precision=prec, flags=tb.TBPM_F_NO_CLUSTER))
    ca = tb.tbpm_dos_corr(a, psi0, dt, 300)
    la = tb.tbpm_get_info(a)["kernel_launches"]
    cb = tb.tbpm_dos_corr(b, psi0, dt, 300)
    lb = tb.tbpm_get_info(b)["kernel_launches"]
    assert la < 10 < lb                              # one cluster launch vs one per sweep
    assert np.max(np.abs(ca - cb)) <= (1e-13 if prec == tb.TBPM_FP64 else 1e-6)
    if prec == tb.TBPM_FP64:
        assert np.max(np.abs(ca - orc.dos_corr(h, rescale, psi0, dt, 300))) <= TOL


@pytest.mark.parametrize("n,steps", [(1, 5), (31, 40), (1000, 200), (4133, 64)])
def test_ragged_complex_hermitian(orc, n, steps):
    h = ti.random_hermitian_csr(n, 3, seed=n, scale=1.5) if n > 1 else ti.graphene_csr(1, 1)
    rescale = 1.05 * ti.gershgorin_bound(h) if n > 1 else 9.0
    dt = 2.7 / rescale
    psi0 = ti.random_phase_state(h.n, 3)
    ctx = create(h, rescale)
    assert tb.tbpm_get_info(ctx)["real_values"] == (0 if n > 1 else 1)
    c = tb.tbpm_dos_corr(ctx, psi0, dt, steps)
    ref = orc.dos_corr(h, rescale, psi0, dt, steps)
    assert np.max(np.abs(c - ref)) <= TOL


def test_bilayer_disorder_and_phases(orc):
    h = ti.bilayer_csr(20, 17, onsite=ti.anderson_onsite(4 * 340, 1.5, 9))
    psi0 = ti.random_phase_state(h.n, 1)
    rescale = 1.02 * ti.gershgorin_bound(h)
    ctx = create(h, rescale)
    c = tb.tbpm_dos_corr(ctx, psi0, math.pi / rescale, 300)
    ref = orc.dos_corr(h, rescale, psi0, math.pi / rescale, 300)
    assert np.max(np.abs(c - ref)) <= TOL
    hp = ti.graphene_csr(13, 11, onsite=ti.anderson_onsite(286, 1.0, 2), bond_phases=[0.7, -0.4, 1.9])
    ctx = create(hp)
    psi0 = ti.random_phase_state(hp.n, 2)
    c = tb.tbpm_dos_corr(ctx, psi0, DT, 256)
    assert np.max(np.abs(c - orc.dos_corr(hp, 9.0, psi0, DT, 256))) <= TOL


@pytest.mark.parametrize("dt", [1e-7, 1e-5, 2e-4, 2e-3, 0.05, -DT, 2 * DT, 30.0 / 9.0, 40.0 / 9.0])
def test_term_counts_and_signs(orc, dt):
    """Small x gives K = 3 or 4 (the short Clenshaw forms); negative dt runs backwards;
    x = 40 is the largest step the library accepts."""
    h = ti.graphene_csr(9, 7, onsite=ti.anderson_onsite(126, 1.0, 4))
    psi0 = ti.random_phase_state(h.n, 5)
    ctx = create(h)
    c = tb.tbpm_dos_corr(ctx, psi0, dt, 50)
    ref = orc.dos_corr(h, 9.0, psi0, dt, 50)
    K_orc = orc.cheb_num_terms(abs(dt) * 9.0)
    assert tb.tbpm_get_info(ctx)["num_terms"] == max(K_orc, 3)
    assert np.max(np.abs(c - ref)) <= TOL


def test_step_beyond_the_coefficient_table_is_rejected():
    """|dt * rescale| > 40 would need more terms than the device table holds."""
    h = ti.graphene_csr(9, 7)
    psi0 = ti.random_phase_state(h.n, 5)
    ctx = create(h)
    with pytest.raises(tb.TbpmError) as e:
        tb.tbpm_dos_corr(ctx, psi0, 41.0 / 9.0, 2)
    assert e.value.status == tb.TBPM_ERR_ARG
    assert np.all(np.isfinite(tb.tbpm_dos_corr(ctx, psi0, 40.0 / 9.0, 2)))


def test_zero_steps_and_multistate(orc):
    h = ti.graphene_csr(10, 10, onsite=ti.anderson_onsite(200, 1.0, 7))
    ctx = create(h)
    psi = ti.random_phase_block(h.n, 3, seed0=4).T.copy()       # (3, n)
    c0 = tb.tbpm_dos_corr(ctx, psi, DT, 0)
    assert c0.shape == (3, 1) and np.allclose(c0[:, 0], 1.0, atol=1e-14)
    c = tb.tbpm_dos_corr(ctx, psi, DT, 33)
    for j in range(3):
        assert np.max(np.abs(c[j] - orc.dos_corr(h, 9.0, psi[j], DT, 33))) <= TOL


def test_disordered_1024x1024_first_steps(orc):
    """1024x1024 graphene (N = 2,097,152), W = 1 eV seed 1, psi0 seed 0: the bench's
    matrix and launch configuration, checked over the first steps and moments."""
    n = 2 * 1024 * 1024
    h = ti.graphene_csr(1024, 1024, onsite=ti.anderson_onsite(n, 1.0, 1))
    psi0 = ti.random_phase_state(n, 0)
    ctx = create(h)
    c = tb.tbpm_dos_corr(ctx, psi0, DT, 4)
    assert np.max(np.abs(c - orc.dos_corr(h, 9.0, psi0, DT, 4))) <= TOL
    mu = tb.kpm_moments(ctx, psi0, 40)
    assert np.max(np.abs(mu - orc.kpm_moments(h, 9.0, psi0, 40))) <= TOL


@pytest.mark.parametrize("M", [1, 2, 3, 17, 512])
def test_kpm_moments(orc, M):
    h = ti.graphene_csr(24, 20, onsite=ti.anderson_onsite(960, 1.0, 3), bond_phases=[0.3, 0.1, 0.2])
    psi0 = ti.random_phase_state(h.n, 8)
    ctx = create(h)
    mu = tb.kpm_moments(ctx, psi0, M)
    ref = orc.kpm_moments(h, 9.0, psi0, M)
    assert mu.shape == (M,)
    assert np.max(np.abs(mu - ref)) <= TOL


def test_kpm_pristine_64x64_site_state(orc):
    h = ti.graphene_csr(64, 64)
    ctx = create(h)
    psi0 = ti.site_state(h.n, 0)
    mu = tb.kpm_moments(ctx, psi0, 4096)
    assert np.max(np.abs(mu - orc.kpm_moments(h, 9.0, psi0, 4096))) <= TOL


@pytest.mark.parametrize("kind,l1,l2,w", [(0, 7, 9, 1.0), (0, 64, 64, 0.0), (1, 5, 6, 2.0),
                                          (1, 33, 17, 0.5)])
def test_stencil_matches_oracle(orc, kind, l1, l2, w):
    per = 2 if kind == 0 else 4
    n = per * l1 * l2
    eps = ti.anderson_onsite(n, w, 11) if w > 0 else None
    h = ti.graphene_csr(l1, l2, onsite=eps) if kind == 0 else ti.bilayer_csr(l1, l2, onsite=eps)
    rescale = max(9.0, 1.02 * ti.gershgorin_bound(h))
    psi0 = ti.random_phase_state(n, 6)
    for path in (tb.TBPM_PATH_STENCIL, tb.TBPM_PATH_SELL):
        ctx = tb.tbpm_create_lattice(kind, l1, l2, -2.7, 0.39, eps, rescale, tb.make_opts(path=path))
        info = tb.tbpm_get_info(ctx)
        assert info["path"] == path
        c = tb.tbpm_dos_corr(ctx, psi0, math.pi / rescale, 120)
        ref = orc.dos_corr(h, rescale, psi0, math.pi / rescale, 120)
        assert np.max(np.abs(c - ref)) <= TOL
        mu = tb.kpm_moments(ctx, psi0, 200)
        assert np.max(np.abs(mu - orc.kpm_moments(h, rescale, psi0, 200))) <= TOL


@pytest.mark.parametrize("flags", [0, tb.TBPM_F_NO_CLUSTER])
def test_propagate_wavefunction(orc, flags):
    """psi(t_N) element by element (cluster path and graph path), with C(t_n)."""
    h = ti.graphene_csr(20, 18, onsite=ti.anderson_onsite(720, 1.0, 3), bond_phases=[0.2, 0.4, 0.6])
    psi0 = ti.random_phase_block(h.n, 2, seed0=5).T.copy()
    ctx = create(h, flags=flags)
    psi, corr = tb.tbpm_propagate(ctx, psi0, DT, 150, with_corr=True)
    for j in range(2):
        K, rc, rpsi = orc.propagate(h, 9.0, psi0[j], DT, 150, want_psi=True)
        assert np.max(np.abs(psi[j] - rpsi)) <= TOL
        assert np.max(np.abs(corr[j] - rc)) <= TOL


def test_propagate_fp32_renorm_and_batched(orc):
    h = ti.graphene_csr(30, 26, onsite=ti.anderson_onsite(1560, 1.0, 4))
    psi0 = ti.random_phase_block(h.n, 16, seed0=0).T.copy()
    for flags in (0, tb.TBPM_F_RENORM):
        ctx = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, 9.0,
                             tb.make_opts(precision=tb.TBPM_FP32, flags=flags))
        psi = tb.tbpm_propagate(ctx, psi0, DT, 400)
        norms = np.linalg.norm(psi, axis=1)
        if flags:
            assert np.max(np.abs(norms - 1)) < 1e-6
        _, _, rpsi = orc.propagate(h, 9.0, psi0[3], DT, 400, want_psi=True)
        assert np.max(np.abs(psi[3] - rpsi)) < 1e-4


def test_autotuned_grid(orc):
    """The autotuner picks a launch shape (block width, slices per warp, a grid
    of whole blocks per SM) once at create; results match the oracle and repeat
    bit for bit on the context."""
    h = ti.graphene_csr(128, 100, onsite=ti.anderson_onsite(25600, 1.0, 2))
    psi0 = ti.random_phase_state(h.n, 1)
    ctx = create(h, flags=tb.TBPM_F_AUTOTUNE | tb.TBPM_F_NO_CLUSTER)
    info = tb.tbpm_get_info(ctx)
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    assert info["tuned"] == 1 and info["grid_blocks"] % sms == 0
    assert info["block_threads"] in (128, 256, 512, 1024) and info["slices_per_warp"] in (1, 2, 4)
    assert info["tune_candidates"] >= 10
    assert 0 < info["tune_best_us"] <= info["tune_default_us"]
    c = tb.tbpm_dos_corr(ctx, psi0, DT, 40)
    assert np.max(np.abs(c - orc.dos_corr(h, 9.0, psi0, DT, 40))) <= TOL
    assert np.array_equal(c, tb.tbpm_dos_corr(ctx, psi0, DT, 40))
    mu = tb.kpm_moments(ctx, psi0, 100)
    assert np.max(np.abs(mu - orc.kpm_moments(h, 9.0, psi0, 100))) <= TOL


SHAPES = [(128, 1), (256, 1), (512, 1), (1024, 1), (128, 2), (256, 2), (512, 2), (128, 4), (256, 4), (512, 4)]


@pytest.mark.parametrize("bt,spw", SHAPES)
def test_sweep_launch_shapes(orc, bt, spw):
    """Every launch shape the autotuner can pick, on the stored-matrix path:
    graphene with real and with complex hoppings (uniform slice width 3, a
    ragged last group), a random Hermitian matrix with complex values (mixed
    slice widths), FP64 and FP32, against the oracle."""
    cases = [(ti.graphene_csr(37, 29, onsite=ti.anderson_onsite(2146, 1.0, 4)), tb.TBPM_FP64, TOL),
             (ti.graphene_csr(37, 29, onsite=ti.anderson_onsite(2146, 1.0, 4), bond_phases=[0.3, 0.1, 0.2]),
              tb.TBPM_FP64, TOL),
             (ti.random_hermitian_csr(2500, 4, seed=6, scale=1.0), tb.TBPM_FP64, TOL),
             (ti.graphene_csr(37, 29, onsite=ti.anderson_onsite(2146, 1.0, 4)), tb.TBPM_FP32, 3e-5)]
    for h, prec, tol in cases:
        rescale = max(9.0, 1.02 * ti.gershgorin_bound(h))
        dt = math.pi / rescale
        psi0 = ti.random_phase_state(h.n, 3)
        ctx = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, rescale,
                             tb.make_opts(precision=prec, flags=tb.TBPM_F_NO_CLUSTER, block_threads=bt,
                                          slices_per_warp=spw))
        info = tb.tbpm_get_info(ctx)
        assert (info["block_threads"], info["slices_per_warp"]) == (bt, spw)
        c = tb.tbpm_dos_corr(ctx, psi0, dt, 60)
        assert np.max(np.abs(c - orc.dos_corr(h, rescale, psi0, dt, 60))) <= tol, (bt, spw, prec)
        assert np.array_equal(c, tb.tbpm_dos_corr(ctx, psi0, dt, 60))


def test_stencil_rejects_stored_matrix_shapes():
    for bt, spw in ((1024, 1), (512, 2)):
        with pytest.raises(tb.TbpmError) as e:
            tb.tbpm_create_lattice(tb.TBPM_LATTICE_GRAPHENE, 8, 8, ti.T_GRAPHENE, 0.0, None, 9.0,
                                   tb.make_opts(path=tb.TBPM_PATH_STENCIL, block_threads=bt, slices_per_warp=spw))
        assert e.value.status == tb.TBPM_ERR_UNSUPPORTED


def test_fp64_peak_probe():
    """The FP64 probe: its rate lies within a factor of two of the unit count
    (2 FP64 lanes per clock per SM, 152 SMs, about 2 GHz on GB300) and above the
    rate a middle sweep reaches, which it bounds."""
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    tf, ms = tb.tbpm_fp64_peak(0, 2000, 1)
    unit = 2 * sms * 2.0e9 * 2 / 1e12
    assert 0.5 * unit < tf < 2.0 * unit and ms > 0
    h = ti.graphene_csr(512, 512, onsite=ti.anderson_onsite(2 * 512 * 512, 1.0, 1))
    ctx = create(h, flags=tb.TBPM_F_NO_CLUSTER)
    psi0 = ti.random_phase_state(h.n, 0)
    tb.tbpm_dos_corr(ctx, psi0, DT, 16)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    tb.tbpm_dos_corr(ctx, psi0, DT, 64)
    b.record()
    torch.cuda.synchronize()
    sweep_tf = 2.0 * h.n * 64 * 178 / (a.elapsed_time(b) / 1e3) / 1e12     # 178 FP64 operations per row and step
    assert sweep_tf < tf


def test_dos_transforms(orc):
    h = ti.graphene_csr(16, 16, onsite=ti.anderson_onsite(512, 1.0, 1))
    psi0 = ti.random_phase_state(h.n, 0)
    ctx = create(h)
    corr = orc.dos_corr(h, 9.0, psi0, DT, 256)
    e, d = tb.tbpm_dos_from_corr(ctx, corr, DT)
    er, dr, _ = orc.dos_hann(corr, DT)
    assert np.max(np.abs(e - er)) < 1e-12 and np.max(np.abs(d - dr)) < 1e-12
    mu = orc.kpm_moments(h, 9.0, psi0, 300)
    e, r = tb.kpm_dos_jackson(ctx, mu, 700)
    er, rr = orc.kpm_dos(mu, 9.0, 700)
    assert np.max(np.abs(e - er)) < 1e-12 and np.max(np.abs(r - rr)) < 1e-12


def test_torch_device_buffers(orc):
    torch = pytest.importorskip("torch")
    h = ti.graphene_csr(32, 16, onsite=ti.anderson_onsite(1024, 1.0, 5))
    psi0 = ti.random_phase_block(h.n, 2, seed0=1).T.copy()
    s = torch.cuda.current_stream()
    ctx = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, 9.0, tb.make_opts(stream=s.cuda_stream))
    dpsi = torch.from_numpy(psi0).cuda()
    dc = tb.tbpm_dos_corr(ctx, dpsi, DT, 40)
    dmu = tb.kpm_moments(ctx, dpsi, 64)
    torch.cuda.synchronize()
    assert dc.is_cuda and dmu.is_cuda
    hc = tb.tbpm_dos_corr(ctx, psi0, DT, 40)
    assert np.array_equal(dc.cpu().numpy(), hc)
    assert np.max(np.abs(dmu.cpu().numpy()[1] - orc.kpm_moments(h, 9.0, psi0[1], 64))) <= TOL
    e, d = tb.tbpm_dos_from_corr(ctx, dc[0], DT)
    torch.cuda.synchronize()
    er, dr, _ = orc.dos_hann(hc[0], DT)
    assert np.max(np.abs(d.cpu().numpy() - dr)) < 1e-12


@pytest.mark.parametrize("prec,flags,path", [
    (tb.TBPM_FP64, 0, tb.TBPM_PATH_AUTO),
    (tb.TBPM_FP32, tb.TBPM_F_RENORM, tb.TBPM_PATH_AUTO),
    (tb.TBPM_FP64, 0, tb.TBPM_PATH_STENCIL),
])
def test_programmatic_launch_changes_nothing(orc, prec, flags, path):
    """The single-state sweeps as programmatic dependent launches (the default)
    and in plain stream order: bit-identical correlations, moments, propagated
    states and quasi-eigenstates, and the FP64 results within the tolerance of
    the oracle."""
    l1, l2 = 96, 70
    n = 2 * l1 * l2
    eps = ti.anderson_onsite(n, 1.0, 6)
    h = ti.graphene_csr(l1, l2, onsite=eps)
    psi0 = ti.random_phase_state(n, 3)
    ctxs = []
    for extra in (0, tb.TBPM_F_NO_PDL):
        o = tb.make_opts(precision=prec, path=path, flags=flags | extra | tb.TBPM_F_NO_CLUSTER)
        if path == tb.TBPM_PATH_STENCIL:
            ctxs.append(tb.tbpm_create_lattice(tb.TBPM_LATTICE_GRAPHENE, l1, l2, ti.T_GRAPHENE, 0.0, eps, 9.0, o))
        else:
            ctxs.append(tb.tbpm_create(n, h.row_ptr, h.col, h.val, 9.0, o))
    res = []
    for c in ctxs:
        corr = tb.tbpm_dos_corr(c, psi0, DT, 40)
        mu = tb.kpm_moments(c, psi0, 64)
        psi = tb.tbpm_propagate(c, psi0, DT, 7)
        r = [corr, mu, psi]
        if flags == 0:
            r.append(tb.tbpm_quasi_eigenstates(c, psi0, DT, 5, np.array([-1.0, 0.3])))
        res.append(r)
    for x, y in zip(*res):
        assert np.array_equal(x, y)
    if prec == tb.TBPM_FP64:
        assert np.max(np.abs(res[0][0] - orc.dos_corr(h, 9.0, psi0, DT, 40))) <= TOL
        assert np.max(np.abs(res[0][1] - orc.kpm_moments(h, 9.0, psi0, 64))) <= TOL
