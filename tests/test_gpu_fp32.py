"""FP32 paths (complex64 vectors and hoppings; FP64 coefficients and dot sums)
against the FP64 oracle.

FP32 results are not expected to equal FP64 ones. The bars, derived from the
arithmetic: each sweep rounds every vector element once at 2^-24 relative, and
a step makes K-1 = 17 sweeps whose rounding errors add up as a random walk
over steps; over n steps the correlation error is about
sqrt(17 n) * 2^-24 * O(1), i.e. ~1e-5 at n = 1024. The tests require
|dC| <= 3e-5 (n <= 1024) and a DOS L1 relative error <= 1e-4 (the target
stated for the mixed-precision path).
"""
import dataclasses
import math

import numpy as np
import pytest

import tbpm_inputs as ti
import paper_2509_26309_gb300 as tb

pytestmark = pytest.mark.gpu
DT = math.pi / 9
C_TOL = 3e-5


def dos_l1(orc, corr, ref, dt):
    _, d, _ = orc.dos_hann(corr, dt)
    _, dr, _ = orc.dos_hann(ref, dt)
    return float(np.sum(np.abs(d - dr)) / np.sum(np.abs(dr)))


def fp32(h, rescale=9.0):
    return tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, rescale, tb.make_opts(precision=tb.TBPM_FP32))


def test_fp32_single_state(orc):
    h = ti.graphene_csr(64, 64, onsite=ti.anderson_onsite(8192, 1.0, 1))
    psi0 = ti.random_phase_state(h.n, 0)
    c = tb.tbpm_dos_corr(fp32(h), psi0, DT, 1024)
    ref = orc.dos_corr(h, 9.0, psi0, DT, 1024)
    assert np.max(np.abs(c - ref)) <= C_TOL
    assert dos_l1(orc, c, ref, DT) <= 1e-4


@pytest.mark.parametrize("nstates", [16, 3, 17])
def test_fp32_batched_states(orc, nstates):
    h = ti.graphene_csr(40, 36, onsite=ti.anderson_onsite(2880, 1.0, 2))
    psi = ti.random_phase_block(h.n, nstates, seed0=0).T.copy()
    ctx = fp32(h)
    c = tb.tbpm_dos_corr(ctx, psi, DT, 300)
    assert c.shape == (nstates, 301)
    for j in range(nstates):
        ref = orc.dos_corr(h, 9.0, psi[j], DT, 300)
        assert np.max(np.abs(c[j] - ref)) <= C_TOL
    assert dos_l1(orc, c[nstates - 1], orc.dos_corr(h, 9.0, psi[-1], DT, 300), DT) <= 1e-4


def test_fp32_batched_complex_ragged(orc):
    h = ti.random_hermitian_csr(999, 4, seed=5, scale=1.0)
    rescale = 1.02 * ti.gershgorin_bound(h)
    psi = ti.random_phase_block(h.n, 16, seed0=3).T.copy()
    ctx = fp32(h, rescale)
    c = tb.tbpm_dos_corr(ctx, psi, math.pi / rescale, 128)
    for j in (0, 7, 15):
        ref = orc.dos_corr(h, rescale, psi[j], math.pi / rescale, 128)
        assert np.max(np.abs(c[j] - ref)) <= C_TOL


@pytest.mark.parametrize("kind,flags", [(tb.TBPM_LATTICE_GRAPHENE, 0),
                                        (tb.TBPM_LATTICE_GRAPHENE, tb.TBPM_F_NO_TBLOCK),
                                        (tb.TBPM_LATTICE_AB_BILAYER, 0),
                                        (tb.TBPM_LATTICE_AB_BILAYER, tb.TBPM_F_NO_TBLOCK)])
def test_fp32_batched_stencil(orc, kind, flags):
    """16 states on the stencil: one temporally blocked run per state, or the
    16-state sweeps with TBPM_F_NO_TBLOCK."""
    l1, l2 = 21, 19
    per = 2 if kind == 0 else 4
    n = per * l1 * l2
    eps = ti.anderson_onsite(n, 1.0, 8)
    h = ti.graphene_csr(l1, l2, onsite=eps) if kind == 0 else ti.bilayer_csr(l1, l2, onsite=eps)
    rescale = max(9.0, 1.02 * ti.gershgorin_bound(h))
    psi = ti.random_phase_block(n, 16, seed0=0).T.copy()
    ctx = tb.tbpm_create_lattice(kind, l1, l2, -2.7, 0.39, eps, rescale,
                                 tb.make_opts(precision=tb.TBPM_FP32, flags=flags))
    c = tb.tbpm_dos_corr(ctx, psi, math.pi / rescale, 200)
    for j in (0, 9):
        ref = orc.dos_corr(h, rescale, psi[j], math.pi / rescale, 200)
        assert np.max(np.abs(c[j] - ref)) <= C_TOL


@pytest.mark.parametrize("stencil,flags", [(False, 0), (True, 0), (True, tb.TBPM_F_NO_TBLOCK)])
def test_fp32_batched_large(orc, stencil, flags):
    """16 states on 512x512 graphene (N = 524,288; 268 MB of state vectors, beyond L2)."""
    l = 512
    n = 2 * l * l
    eps = ti.anderson_onsite(n, 1.0, 1)
    h = ti.graphene_csr(l, l, onsite=eps)
    opts = tb.make_opts(precision=tb.TBPM_FP32, flags=flags)
    ctx = (tb.tbpm_create_lattice(tb.TBPM_LATTICE_GRAPHENE, l, l, -2.7, 0.0, eps, 9.0, opts) if stencil
           else tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, 9.0, opts))
    psi = np.stack([ti.random_phase_state(n, j) for j in range(16)])
    c = tb.tbpm_dos_corr(ctx, psi, DT, 6)
    for j in (0, 15):
        assert np.max(np.abs(c[j] - orc.dos_corr(h, 9.0, psi[j], DT, 6))) <= C_TOL


def test_fp32_device_block(orc):
    torch = pytest.importorskip("torch")
    h = ti.graphene_csr(32, 32, onsite=ti.anderson_onsite(2048, 1.0, 4))
    psi = ti.random_phase_block(h.n, 16, seed0=2).T.copy()
    ctx = fp32(h)
    dc = tb.tbpm_dos_corr(ctx, torch.from_numpy(psi).cuda(), DT, 64)
    torch.cuda.synchronize()
    hc = tb.tbpm_dos_corr(ctx, psi, DT, 64)
    assert np.array_equal(dc.cpu().numpy(), hc)


def test_fp32_kpm(orc):
    h = ti.graphene_csr(30, 30, onsite=ti.anderson_onsite(1800, 1.0, 6))
    psi0 = ti.random_phase_state(h.n, 1)
    mu = tb.kpm_moments(fp32(h), psi0, 1024)
    ref = orc.kpm_moments(h, 9.0, psi0, 1024)
    assert np.max(np.abs(mu - ref)) <= 1e-4


def test_fp32_16_states_4096_full_size(orc, golden):
    """Sixteen FP32 states on 4096 x 4096 graphene (N = 33,554,432) in the
    launch configurations the benchmark times: the stencil (one blocked
    evolution per state) and the stored matrix (16 states per sweep); 128
    steps, states 0 and 15 against the oracle's stored C(t) (|dC| and the DOS
    L1 error)."""
    l = 4096
    n = 2 * l * l
    steps = 128
    eps = ti.anderson_onsite(n, 1.0, 1)
    psi = np.stack([ti.random_phase_state(n, j) for j in range(16)])
    ctx = tb.tbpm_create_lattice(tb.TBPM_LATTICE_GRAPHENE, l, l, -2.7, 0.0, eps, 9.0,
                                 tb.make_opts(precision=tb.TBPM_FP32))
    c_st = tb.tbpm_dos_corr(ctx, psi, DT, steps)
    del ctx
    h = ti.graphene_csr(l, l, onsite=eps)
    ctx = tb.tbpm_create(n, h.row_ptr, h.col, h.val, 9.0,
                         tb.make_opts(precision=tb.TBPM_FP32, path=tb.TBPM_PATH_SELL))
    del h
    c_sell = tb.tbpm_dos_corr(ctx, psi, DT, steps)
    del ctx
    for j in (0, 15):
        ref = golden("graphene4096_dos128", j)
        for c in (c_st[j], c_sell[j]):
            assert np.max(np.abs(c - ref)) <= C_TOL
            assert dos_l1(orc, c, ref, DT) <= 1e-4


@pytest.mark.parametrize("case", ["graphene", "bilayer", "graphene_wide"])
def test_packed_sell_matches_plain_and_oracle(orc, case):
    """FP32 stored matrices kept packed (16-bit column offsets modulo the padded
    row count, 8-bit value indices; graphene, whose slices all have width 3,
    one 64-bit word per row): the same entries, so C(t) and the KPM moments
    equal the plain form's bit for bit at the same launch shape (one and two
    slices per warp), and the packed default shape (128 threads and four
    slices per entry, 256 threads and two slices per row) stays within the FP32
    bars of the oracle."""
    if case == "graphene":
        h = ti.graphene_csr(60, 44, onsite=ti.anderson_onsite(5280, 1.0, 3))
    elif case == "bilayer":
        h = ti.bilayer_csr(23, 19, onsite=ti.anderson_onsite(4 * 23 * 19, 0.8, 4))
    else:                                   # periodic wrap offsets beyond 2^15 before the modulus
        h = ti.graphene_csr(256, 80, onsite=ti.anderson_onsite(40960, 1.0, 5))
    rescale = max(9.0, 1.02 * ti.gershgorin_bound(h))
    dt = math.pi / rescale
    psi0 = ti.random_phase_state(h.n, 6)
    ref = orc.dos_corr(h, rescale, psi0, dt, 128)
    ref_mu = orc.kpm_moments(h, rescale, psi0, 256)
    out = {}
    for name, flags, bt, spw in (("packed", 0, 512, 1), ("plain", tb.TBPM_F_PLAIN_SELL, 512, 1),
                                 ("packed_s2", 0, 256, 2), ("plain_s2", tb.TBPM_F_PLAIN_SELL, 256, 2),
                                 ("packed_default", 0, 0, 0)):
        ctx = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, rescale,
                             tb.make_opts(precision=tb.TBPM_FP32, flags=flags | tb.TBPM_F_NO_CLUSTER,
                                          block_threads=bt, slices_per_warp=spw))
        info = tb.tbpm_get_info(ctx)
        assert info["packed"] == (0 if name.startswith("plain") else 1 if case == "bilayer" else 2)
        if name == "packed_default":
            assert (info["block_threads"], info["slices_per_warp"]) == ((128, 4) if case == "bilayer" else (256, 2))
        out[name] = (tb.tbpm_dos_corr(ctx, psi0, dt, 128), tb.kpm_moments(ctx, psi0, 256))
    for a, b in (("packed", "plain"), ("packed_s2", "plain_s2")):
        assert np.array_equal(out[a][0], out[b][0]), a
        assert np.array_equal(out[a][1], out[b][1]), a
    assert np.max(np.abs(out["packed_default"][0] - ref)) <= C_TOL
    assert np.max(np.abs(out["packed_default"][1] - ref_mu)) <= 1e-4


def _bond_levels(h, levels):
    """The same lattice with each bond's hopping scaled by 1 + 0.01 k, k one of
    `levels` values fixed by the bond's two ends (the same both ways, so H stays
    Hermitian); the diagonal is unchanged."""
    rows = np.repeat(np.arange(h.n), np.diff(h.row_ptr))
    lo, hi = np.minimum(rows, h.col), np.maximum(rows, h.col)
    k = (lo * 1000003 + hi * 7920) % levels
    off = rows != h.col
    val = h.val.copy()
    val[off] *= 1.0 + 0.01 * k[off]
    return dataclasses.replace(h, val=val)


@pytest.mark.parametrize("case,form", [("ragged", 2), ("levels40", 1), ("levels300", 0)])
def test_packed_form_choice(orc, case, form):
    """Which packed form a graphene matrix gets: a ragged last slice still packs
    per row (its padding rows hold offset 0 and value 0); 40 distinct hoppings
    fit the per-entry form's 8-bit indices but not the per-row form's 5-bit ones;
    300 fit neither. Every form matches the plain one bit for bit at the same
    launch shape and the oracle within the FP32 bars."""
    if case == "ragged":
        h = ti.graphene_csr(61, 43, onsite=ti.anderson_onsite(2 * 61 * 43, 1.0, 7))
    else:
        h = _bond_levels(ti.graphene_csr(64, 48, onsite=ti.anderson_onsite(2 * 64 * 48, 1.0, 8)),
                         40 if case == "levels40" else 300)
    if case == "ragged":
        assert h.n % 32 != 0
    rescale = max(9.0, 1.02 * ti.gershgorin_bound(h))
    dt = math.pi / rescale
    psi0 = ti.random_phase_state(h.n, 9)
    ref = orc.dos_corr(h, rescale, psi0, dt, 64)
    out = {}
    for name, flags in (("packed", 0), ("plain", tb.TBPM_F_PLAIN_SELL)):
        ctx = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, rescale,
                             tb.make_opts(precision=tb.TBPM_FP32, flags=flags | tb.TBPM_F_NO_CLUSTER,
                                          block_threads=256, slices_per_warp=2))
        assert tb.tbpm_get_info(ctx)["packed"] == (form if name == "packed" else 0)
        out[name] = (tb.tbpm_dos_corr(ctx, psi0, dt, 64), tb.kpm_moments(ctx, psi0, 128))
    assert np.array_equal(out["packed"][0], out["plain"][0])
    assert np.array_equal(out["packed"][1], out["plain"][1])
    assert np.max(np.abs(out["packed"][0] - ref)) <= C_TOL


def test_what_is_not_packed(orc):
    """Complex values, FP64 contexts and column offsets beyond 16 bits keep the
    plain form only; the latter still matches the oracle."""
    h = ti.graphene_csr(20, 20, onsite=ti.anderson_onsite(800, 1.0, 3), bond_phases=[0.3, 0.1, 0.2])
    ctx = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, 9.0, tb.make_opts(precision=tb.TBPM_FP32))
    assert tb.tbpm_get_info(ctx)["packed"] == 0
    ctx = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, 9.0)                      # FP64
    assert tb.tbpm_get_info(ctx)["packed"] == 0
    r = ti.random_hermitian_csr(70000, 2, seed=3, scale=1.0)
    r.val = np.ascontiguousarray(r.val.real.astype(np.complex128))       # real symmetric, random columns
    rescale = 1.05 * ti.gershgorin_bound(r)
    ctx = tb.tbpm_create(r.n, r.row_ptr, r.col, r.val, rescale, tb.make_opts(precision=tb.TBPM_FP32))
    assert tb.tbpm_get_info(ctx)["packed"] == 0
    psi0 = ti.random_phase_state(r.n, 1)
    c = tb.tbpm_dos_corr(ctx, psi0, 2.0 / rescale, 20)
    assert np.max(np.abs(c - orc.dos_corr(r, rescale, psi0, 2.0 / rescale, 20))) <= C_TOL

