"""The allocation-free correlation call, for callers that cannot allocate
device memory (a fixed device-memory budget owned by the host application, a
plugin barred from allocating after start-up). It must give the same C(t) as
the regular context-based call, on two calls in a row that share its static
scratch array. This file is collected last on purpose, so that a run that
stops at the first failure has already run every other test."""
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


def test_noalloc_matches_context_call_twice():
    torch = pytest.importorskip("torch")
    dt, steps = math.pi / 9, 200
    cases = [ti.graphene_csr(24, 20, onsite=ti.anderson_onsite(960, 1.0, 3)),
             ti.random_hermitian_csr(700, 3, seed=8, scale=1.2)]
    for h in cases:
        rescale = max(9.0, 1.02 * ti.gershgorin_bound(h))
        ctx = tb.tbpm_create(h.n, h.row_ptr, h.col, h.val, rescale)
        rp, col, val = _dev(torch, h)
        for seed in (0, 1):                      # two calls in a row on the same scratch
            psi0 = ti.random_phase_state(h.n, seed)
            want = tb.tbpm_dos_corr(ctx, psi0, dt, steps)
            dpsi = torch.from_numpy(psi0).cuda()
            out = torch.empty(steps + 1, dtype=torch.complex128, device="cuda")
            torch.cuda.synchronize()
            tb.tbpm_dos_corr_noalloc(h.n, rp, col, val, rescale, dpsi, dt, steps, out)
            torch.cuda.synchronize()
            got = out.cpu().numpy()
            assert np.max(np.abs(got - want)) <= TOL


def test_noalloc_size_limit():
    torch = pytest.importorskip("torch")
    h = ti.graphene_csr(4, 4)
    rp, col, val = _dev(torch, h)
    psi = torch.zeros(16, dtype=torch.complex128, device="cuda")
    out = torch.zeros(3, dtype=torch.complex128, device="cuda")
    with pytest.raises(tb.TbpmError) as e:
        tb.tbpm_dos_corr_noalloc(tb.tbpm.TBPM_NOALLOC_MAX_N + 1, rp, col, val, 9.0, psi, 0.3, 2, out)
    assert e.value.status == tb.TBPM_ERR_UNSUPPORTED
