"""The allocation-free correlation call, for callers that cannot allocate
device memory (a fixed device-memory budget owned by the host application, a
plugin barred from allocating after start-up). It must give the oracle's C(t)
and the regular context-based call's, on two calls in a row that share its
static scratch array, and leave the device's free memory unchanged. This file
is collected last on purpose, so that a run that stops at the first failure has
already run every other test."""
import math

import numpy as np
import pytest

import tbpm_inputs as ti
import paper_2509_26309_gb300 as tb

pytestmark = pytest.mark.gpu
TOL = 1e-10


def _dev(torch, h):
    return (torch.from_numpy(h.row_ptr.astype(np.int64)).cuda(),
            torch.from_numpy(h.col.astype(np.int32)).cuda(),
            torch.from_numpy(h.val.astype(np.complex128)).cuda())


def _noalloc(torch, dev_csr, h, rescale, psi0, dt, steps):
    rp, col, val = dev_csr
    dpsi = torch.from_numpy(psi0).cuda()
    out = torch.empty(steps + 1, dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    tb.tbpm_dos_corr_noalloc(h.n, rp, col, val, rescale, dpsi, dt, steps, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


# (lattice, dt * rescale, steps): K = 18 at x = pi; x = 1e-3 gives K = 4 and
# x = 1e-4 gives K = 3 (J_3(1e-4) ~ 2e-14 < 1e-12), the two short forms of the
# Clenshaw sum; a negative time step runs the evolution backwards
CASES = {
    "graphene24x20_w1": (lambda: ti.graphene_csr(24, 20, onsite=ti.anderson_onsite(960, 1.0, 3)), math.pi, 200),
    "random_hermitian700": (lambda: ti.random_hermitian_csr(700, 3, seed=8, scale=1.2), math.pi, 200),
    "graphene16x12_K3": (lambda: ti.graphene_csr(16, 12, onsite=ti.anderson_onsite(384, 1.0, 5)), 1e-4, 40),
    "graphene16x12_K4": (lambda: ti.graphene_csr(16, 12, onsite=ti.anderson_onsite(384, 1.0, 5)), 1e-3, 40),
    "graphene24x20_negative_dt": (lambda: ti.graphene_csr(24, 20, onsite=ti.anderson_onsite(960, 1.0, 3)),
                                  -math.pi, 100),
    # exactly the largest size the call accepts: 256 x 128 cells = 65,536 orbitals
    "graphene256x128_max_n": (lambda: ti.graphene_csr(256, 128, onsite=ti.anderson_onsite(65536, 1.0, 7)),
                              math.pi, 64),
}


@pytest.mark.parametrize("name", list(CASES))
def test_noalloc_matches_oracle_and_context_call_twice(name, orc):
    torch = pytest.importorskip("torch")
    make, x, steps = CASES[name]
    h = make()
    if name.endswith("max_n"):
        assert h.n == tb.tbpm.TBPM_NOALLOC_MAX_N
    rescale = max(9.0, 1.02 * ti.gershgorin_bound(h))
    dt = x / rescale
    ctx = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, rescale)
    dev_csr = _dev(torch, h)
    for seed in (0, 1):                      # two calls in a row on the same scratch
        psi0 = ti.random_phase_state(h.n, seed)
        want = orc.dos_corr(h, rescale, psi0, dt, steps)
        got = _noalloc(torch, dev_csr, h, rescale, psi0, dt, steps)
        assert np.max(np.abs(got - want)) <= TOL, f"{name} seed {seed}: vs oracle"
        ctx_c = tb.tbpm_dos_corr(ctx, psi0, dt, steps)
        assert np.max(np.abs(got - ctx_c)) <= TOL, f"{name} seed {seed}: vs the context call"
    if name.endswith("K3") or name.endswith("K4"):
        assert tb.tbpm_get_info(ctx)["num_terms"] == (3 if name.endswith("K3") else 4)


def test_noalloc_leaves_device_memory_unchanged():
    """After one warm-up call (which loads the kernels' code), further calls
    change neither the device's free memory nor torch's reserved pool."""
    torch = pytest.importorskip("torch")
    h = ti.graphene_csr(24, 20, onsite=ti.anderson_onsite(960, 1.0, 3))
    dev_csr = _dev(torch, h)
    psi0 = ti.random_phase_state(h.n, 0)
    dpsi = torch.from_numpy(psi0).cuda()
    out = torch.empty(65, dtype=torch.complex128, device="cuda")
    rp, col, val = dev_csr
    tb.tbpm_dos_corr_noalloc(h.n, rp, col, val, 9.0, dpsi, math.pi / 9, 64, out)
    torch.cuda.synchronize()
    free0, reserved0 = torch.cuda.mem_get_info()[0], torch.cuda.memory_reserved()
    for _ in range(3):
        tb.tbpm_dos_corr_noalloc(h.n, rp, col, val, 9.0, dpsi, math.pi / 9, 64, out)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_reserved() == reserved0


def test_noalloc_size_limit():
    torch = pytest.importorskip("torch")
    n = tb.tbpm.TBPM_NOALLOC_MAX_N + 1
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")     # n rows, one zero entry in the last
    rp[n] = 1
    col = torch.full((1,), n - 1, dtype=torch.int32, device="cuda")
    val = torch.zeros(1, dtype=torch.complex128, device="cuda")
    psi = torch.zeros(n, dtype=torch.complex128, device="cuda")
    out = torch.zeros(3, dtype=torch.complex128, device="cuda")
    with pytest.raises(tb.TbpmError) as e:
        tb.tbpm_dos_corr_noalloc(n, rp, col, val, 9.0, psi, 0.3, 2, out)
    assert e.value.status == tb.TBPM_ERR_UNSUPPORTED


def test_noalloc_binding_rejects_mismatched_buffers():
    """The C call cannot see buffer sizes; the binding checks them before it runs."""
    torch = pytest.importorskip("torch")
    h = ti.graphene_csr(4, 4)
    rp, col, val = _dev(torch, h)
    psi = torch.zeros(h.n, dtype=torch.complex128, device="cuda")
    out = torch.zeros(3, dtype=torch.complex128, device="cuda")
    with pytest.raises(ValueError):          # corr too short for n_steps
        tb.tbpm_dos_corr_noalloc(h.n, rp, col, val, 9.0, psi, 0.3, 5, out)
    with pytest.raises(ValueError):          # psi0 of the wrong length
        tb.tbpm_dos_corr_noalloc(h.n, rp, col, val, 9.0, psi[:-1], 0.3, 2, out)
    with pytest.raises(TypeError):           # col of the wrong type
        tb.tbpm_dos_corr_noalloc(h.n, rp, col.long(), val, 9.0, psi, 0.3, 2, out)
    with pytest.raises(TypeError):           # a host buffer
        tb.tbpm_dos_corr_noalloc(h.n, rp, col, val, 9.0, psi.cpu(), 0.3, 2, out)
