"""Temporally blocked sweeps on the FP32 monolayer stencil (several Chebyshev
terms per pass over a lattice tile held in shared memory) against the FP64
oracle and against the one-launch-per-sweep FP32 path.

The FP32 bars are those of test_gpu_fp32.py: |dC| <= 3e-5 over up to 1024
steps (a random walk of 2^-24 roundings over 17 sweeps per step) and a DOS L1
relative error <= 1e-4; blocked and per-sweep FP32 results differ only by the
rounding order, well inside that."""
import math

import numpy as np
import pytest

import tbpm_inputs as ti
import paper_2509_26309_gb300 as tb

pytestmark = pytest.mark.gpu
DT = math.pi / 9
C_TOL = 3e-5


MONO, BI = tb.TBPM_LATTICE_GRAPHENE, tb.TBPM_LATTICE_AB_BILAYER


def lattice(l1, l2, w=1.0, seed=1, flags=0, kind=MONO):
    n = (2 if kind == MONO else 4) * l1 * l2
    eps = ti.anderson_onsite(n, w, seed)
    ctx = tb.tbpm_create_lattice(kind, l1, l2, ti.T_GRAPHENE, ti.T_PERP_AB if kind == BI else 0.0, eps, 9.0,
                                 tb.make_opts(precision=tb.TBPM_FP32, path=tb.TBPM_PATH_STENCIL, flags=flags))
    return ctx, eps


def csr(l1, l2, eps, kind):
    return ti.graphene_csr(l1, l2, onsite=eps) if kind == MONO else ti.bilayer_csr(l1, l2, onsite=eps)


@pytest.mark.parametrize("kind,l1,l2,dt,steps", [
    (MONO, 9, 12, DT, 37),      # one tile smaller than the region: the halo wraps the torus
    (MONO, 61, 70, DT, 64),     # ragged tiles
    (MONO, 150, 131, DT, 33),   # several tiles, odd step count (chunk copy-back)
    (MONO, 64, 64, 0.05, 20),   # K = 4..5: a single block holds every sweep
    (MONO, 40, 58, 1e-4, 9),    # K = 3
    (MONO, 100, 116, 3.0, 16),  # x = 27: K ~ 45, eight blocks per step
    (BI, 7, 9, DT, 21),         # AB bilayer: wrapped single tile
    (BI, 90, 61, DT, 33),       # ragged tiles, odd steps
    (BI, 45, 50, 3.0, 8),       # many blocks per step
])
def test_tblock_matches_oracle(orc, kind, l1, l2, dt, steps):
    ctx, eps = lattice(l1, l2, kind=kind)
    h = csr(l1, l2, eps, kind)
    psi0 = ti.random_phase_state(h.n, 5)
    c = tb.tbpm_dos_corr(ctx, psi0, dt, steps)
    ref = orc.dos_corr(h, 9.0, psi0, dt, steps)
    assert np.max(np.abs(c - ref)) <= C_TOL, np.max(np.abs(c - ref))
    # blocked launches: ceil((K-1)/6) per step instead of K-1
    info = tb.tbpm_get_info(ctx)
    K = info["num_terms"]
    assert info["kernel_launches"] <= 3 + steps * ((K - 2) // 6 + 1) + 2 * ((steps + 15) // 16)
    # the per-sweep path on the same FP32 inputs differs only by rounding order
    ctx2, _ = lattice(l1, l2, flags=tb.TBPM_F_NO_TBLOCK, kind=kind)
    c2 = tb.tbpm_dos_corr(ctx2, psi0, dt, steps)
    assert np.max(np.abs(c - c2)) <= 2e-6


def test_tblock_long_run_dos(orc):
    l1, l2 = 48, 47
    ctx, eps = lattice(l1, l2, w=1.0, seed=2)
    h = ti.graphene_csr(l1, l2, onsite=eps)
    psi0 = ti.random_phase_state(h.n, 0)
    c = tb.tbpm_dos_corr(ctx, psi0, DT, 1024)
    ref = orc.dos_corr(h, 9.0, psi0, DT, 1024)
    assert np.max(np.abs(c - ref)) <= C_TOL
    _, d, _ = orc.dos_hann(c, DT)
    _, dr, _ = orc.dos_hann(ref, DT)
    assert np.sum(np.abs(d - dr)) / np.sum(np.abs(dr)) <= 1e-4
    c2 = tb.tbpm_dos_corr(ctx, psi0, DT, 1024)
    assert np.array_equal(c, c2)                       # fixed tiles and reduction order


def test_tblock_final_state(orc):
    l1, l2 = 70, 61
    ctx, eps = lattice(l1, l2, seed=3)
    h = ti.graphene_csr(l1, l2, onsite=eps)
    psi0 = ti.random_phase_state(h.n, 9)
    for steps in (7, 16):
        psi = tb.tbpm_propagate(ctx, psi0, DT, steps)
        _, _, ref = orc.propagate(h, 9.0, psi0, DT, steps, want_corr=False, want_psi=True)
        assert np.max(np.abs(np.asarray(psi).reshape(-1) - ref)) <= 1e-5


def test_tblock_device_buffers_and_pristine(orc):
    torch = pytest.importorskip("torch")
    l1, l2 = 64, 64
    ctx = tb.tbpm_create_lattice(tb.TBPM_LATTICE_GRAPHENE, l1, l2, ti.T_GRAPHENE, 0.0, None, 9.0,
                                 tb.make_opts(precision=tb.TBPM_FP32, path=tb.TBPM_PATH_STENCIL))
    h = ti.graphene_csr(l1, l2)
    psi0 = ti.random_phase_state(h.n, 0)
    out = torch.empty((1, 129), dtype=torch.complex128, device="cuda")
    tb.tbpm_dos_corr(ctx, torch.from_numpy(psi0).cuda().reshape(1, -1), DT, 128, out=out)
    ref = orc.dos_corr(h, 9.0, psi0, DT, 128)
    assert np.max(np.abs(out[0].cpu().numpy() - ref)) <= C_TOL


@pytest.mark.parametrize("kind,l", [(MONO, 2048), (BI, 1448)])
def test_tblock_large(orc, kind, l):
    """About 8.4 M orbitals (the state vectors exceed L2): six steps against the oracle."""
    ctx, eps = lattice(l, l, seed=4, kind=kind)
    h = csr(l, l, eps, kind)
    psi0 = ti.random_phase_state(h.n, 0)
    c = tb.tbpm_dos_corr(ctx, psi0, DT, 6)
    ref = orc.dos_corr(h, 9.0, psi0, DT, 6)
    assert np.max(np.abs(c - ref)) <= C_TOL


@pytest.mark.parametrize("kind,l1,l2,M", [
    (MONO, 30, 30, 1024),       # one wrapped tile
    (MONO, 130, 61, 301),       # ragged tiles, odd M, a short last chunk
    (MONO, 47, 50, 2),          # only the first pass
    (BI, 33, 29, 512),
])
def test_tblock_kpm_matches_oracle(orc, kind, l1, l2, M):
    """KPM moments with blocked passes on the FP32 stencils: the FP32 bar of the
    one-pass kernel (|dmu| <= 1e-4 over 1024 moments), and close to the
    one-pass FP32 result."""
    ctx, eps = lattice(l1, l2, seed=6, kind=kind)
    h = csr(l1, l2, eps, kind)
    psi0 = ti.random_phase_state(h.n, 1)
    mu = tb.kpm_moments(ctx, psi0, M)
    ref = orc.kpm_moments(h, 9.0, psi0, M)
    assert np.max(np.abs(mu - ref)) <= 1e-4
    ctx2, _ = lattice(l1, l2, seed=6, kind=kind, flags=tb.TBPM_F_NO_TBLOCK)
    mu2 = tb.kpm_moments(ctx2, psi0, M)
    assert np.max(np.abs(mu - mu2)) <= 2e-5
    assert np.array_equal(mu, tb.kpm_moments(ctx, psi0, M))      # fixed reduction order


def test_tblock_kpm_large(orc):
    """Blocked KPM passes on 2048 x 2048 cells (state vectors beyond L2)."""
    l = 2048
    ctx, eps = lattice(l, l, seed=7)
    h = csr(l, l, eps, MONO)
    psi0 = ti.random_phase_state(h.n, 2)
    mu = tb.kpm_moments(ctx, psi0, 40)
    ref = orc.kpm_moments(h, 9.0, psi0, 40)
    assert np.max(np.abs(mu - ref)) <= 1e-5
