"""The full-size workloads over their full horizons, in the launch
configuration the benchmark times, against the oracle's stored results
(tests/golden/oracle_*.txt, written by tests/golden/make_oracle_golden.py from
the FP64 oracle alone).

Graphene 1024 x 1024 (N = 2,097,152), W = 1 eV, FP64 stored matrix: all 2048
time steps and all 4096 KPM moments within 1e-10 of the oracle, with the DOS
error of both transforms. Graphene 2048 x 2048 (N = 8,388,608), FP32 vectors and
hoppings: 1024 steps, |dC| <= 3e-5 and a DOS L1 relative error <= 1e-4 against
the oracle's FP64 C(t) (the bars of the FP32 tests, derived there).
"""
import math

import numpy as np
import pytest

import tbpm_inputs as ti
import paper_2509_26309_gb300 as tb

pytestmark = pytest.mark.gpu
DT = math.pi / 9
TOL = 1e-10


def dos_l1(orc, corr, ref, dt):
    """L1 relative error of the Hann-windowed DOS of corr against that of ref
    (both transformed by the oracle)."""
    _, d, _ = orc.dos_hann(corr, dt)
    _, dr, _ = orc.dos_hann(ref, dt)
    return float(np.sum(np.abs(d - dr)) / np.sum(np.abs(dr)))


def test_graphene1024_fp64_full_horizon(orc, golden):
    torch = pytest.importorskip("torch")
    l = 1024
    n = 2 * l * l
    h = ti.graphene_csr(l, l, onsite=ti.anderson_onsite(n, 1.0, 1))
    stream = torch.cuda.Stream()
    ctx = tb.tbpm_create(n, h.row_ptr, h.col, h.val, 9.0, tb.make_opts(device=0, stream=stream.cuda_stream))
    del h
    dpsi = torch.from_numpy(ti.random_phase_state(n, 0).reshape(1, n)).cuda()
    dc = torch.empty((1, 2049), dtype=torch.complex128, device="cuda")
    dmu = torch.empty((1, 4096), dtype=torch.complex128, device="cuda")
    torch.cuda.synchronize()
    tb.tbpm_dos_corr(ctx, dpsi, DT, 2048, out=dc)
    tb.kpm_moments(ctx, dpsi, 4096, out=dmu)
    stream.synchronize()
    c, mu = dc[0].cpu().numpy(), dmu[0].cpu().numpy()
    ref_c = golden("graphene1024_dos2048")
    ref_mu = golden("graphene1024_kpm4096")
    assert tb.tbpm_get_info(ctx)["num_terms"] == 18
    err_c = np.max(np.abs(c - ref_c))
    err_mu = np.max(np.abs(mu - ref_mu))
    assert err_c <= TOL, err_c
    assert err_mu <= TOL, err_mu
    # the DOS of both routes: Hann transform of C(t) and the Jackson KPM DOS
    assert dos_l1(orc, c, ref_c, DT) <= 1e-9
    _, rho = tb.kpm_dos_jackson(ctx, mu, 4096)
    _, rho_ref = orc.kpm_dos(ref_mu, 9.0, 4096)
    assert np.sum(np.abs(rho - rho_ref)) / np.sum(np.abs(rho_ref)) <= 1e-9


def test_graphene2048_fp32_full_horizon(orc, golden):
    l = 2048
    n = 2 * l * l
    h = ti.graphene_csr(l, l, onsite=ti.anderson_onsite(n, 1.0, 1))
    ref = golden("graphene2048_dos1024")
    for flags in (0, tb.TBPM_F_RENORM):
        ctx = tb.tbpm_create(n, h.row_ptr, h.col, h.val, 9.0, tb.make_opts(precision=tb.TBPM_FP32, flags=flags))
        c = tb.tbpm_dos_corr(ctx, ti.random_phase_state(n, 0), DT, 1024)
        del ctx
        err = np.max(np.abs(c - ref))
        l1 = dos_l1(orc, c, ref, DT)
        assert err <= 3e-5, (flags, err)
        assert l1 <= 1e-4, (flags, l1)
