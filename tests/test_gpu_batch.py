"""The uneven multi-lattice batch (one block-diagonal operator, per-instance
rescale, coefficients, state and correlation) against the FP64 oracle run on
each instance alone."""
import math

import numpy as np
import pytest

import tbpm_inputs as ti
import paper_2509_26309_gb300 as tb

pytestmark = pytest.mark.gpu
TOL = 1e-10


def concat_states(insts, seed0=0):
    return np.concatenate([ti.random_phase_state(i.csr.n, seed0 + k) for k, i in enumerate(insts)])


def split(v, insts):
    out, o = [], 0
    for i in insts:
        out.append(v[o:o + i.csr.n])
        o += i.csr.n
    return out


def test_small_uneven_batch_fp64(orc):
    insts = ti.batch_instances(count=7, scale_n=0.004)
    ctx = tb.tbpm_create_batch([(i.csr, i.rescale) for i in insts])
    psi = concat_states(insts)
    dts = [math.pi / i.rescale for i in insts]
    c = tb.tbpm_batch_dos_corr(ctx, psi, dts, 96)
    assert c.shape == (7, 97)
    for g, (i, p) in enumerate(zip(insts, split(psi, insts))):
        ref = orc.dos_corr(i.csr, i.rescale, p, dts[g], 96)
        assert np.max(np.abs(c[g] - ref)) <= TOL, g
    c2 = tb.tbpm_batch_dos_corr(ctx, psi, dts, 96)
    assert np.array_equal(c, c2)


def test_batch_launch_shapes_and_autotuner(orc):
    """The batch's sweeps at every launch shape against the oracle (each row's
    arithmetic is the same for every shape; the grouping of the dot partials
    follows the grid), each repeating itself bit for bit; the autotuned context
    too."""
    insts = ti.batch_instances(count=6, scale_n=0.004)
    psi = concat_states(insts, 3)
    dts = [math.pi / i.rescale for i in insts]
    parts = split(psi, insts)
    refs = [orc.dos_corr(i.csr, i.rescale, p, dts[g], 48) for g, (i, p) in enumerate(zip(insts, parts))]
    for bt, spw, flags in ((512, 1, 0), (128, 1, 0), (1024, 1, 0), (256, 2, 0), (512, 4, 0),
                           (0, 0, tb.TBPM_F_AUTOTUNE)):
        ctx = tb.tbpm_create_batch([(i.csr, i.rescale) for i in insts],
                                   tb.make_opts(block_threads=bt, slices_per_warp=spw, flags=flags))
        c = tb.tbpm_batch_dos_corr(ctx, psi, dts, 48)
        for g in range(len(insts)):
            assert np.max(np.abs(c[g] - refs[g])) <= TOL, (bt, spw, g)
        assert np.array_equal(c, tb.tbpm_batch_dos_corr(ctx, psi, dts, 48)), (bt, spw)
        if flags:
            info = tb.tbpm_get_info(ctx)
            assert info["tuned"] == 1 and info["tune_best_us"] <= info["tune_default_us"]


def test_batch_mixed_term_counts(orc):
    """Instances with different x = dt * rescale need different K; the batch runs
    the largest K with the shorter series zero-padded."""
    hs = [ti.graphene_csr(5, 7, onsite=ti.anderson_onsite(70, 1.0, 1)),
          ti.random_hermitian_csr(45, 3, seed=2, scale=1.0),
          ti.bilayer_csr(4, 4, onsite=ti.anderson_onsite(64, 0.5, 3))]
    rs = [9.0, 1.05 * ti.gershgorin_bound(hs[1]), 9.5]
    dts = [0.01, 2.0 / rs[1], 12.0 / rs[2]]
    ctx = tb.tbpm_create_batch(list(zip(hs, rs)))
    psis = [ti.random_phase_state(h.n, 4 + k) for k, h in enumerate(hs)]
    c = tb.tbpm_batch_dos_corr(ctx, np.concatenate(psis), dts, 40)
    for g in range(3):
        ref = orc.dos_corr(hs[g], rs[g], psis[g], dts[g], 40)
        assert np.max(np.abs(c[g] - ref)) <= TOL, g
    assert tb.tbpm_get_info(ctx)["num_terms"] == max(orc.cheb_num_terms(d * r) for d, r in zip(dts, rs))


@pytest.mark.parametrize("bt,spw", [(512, 1), (256, 2)])
def test_batch_fp32_renorm(orc, bt, spw):
    """FP32 batch with and without renormalisation (the final sweep's norm
    partials per instance run), at the default and a two-slice shape."""
    insts = ti.batch_instances(count=5, scale_n=0.003)
    psi = concat_states(insts, 10)
    dts = [math.pi / i.rescale for i in insts]
    for flags in (0, tb.TBPM_F_RENORM):
        ctx = tb.tbpm_create_batch([(i.csr, i.rescale) for i in insts],
                                   tb.make_opts(precision=tb.TBPM_FP32, flags=flags, block_threads=bt,
                                                slices_per_warp=spw))
        c = tb.tbpm_batch_dos_corr(ctx, psi, dts, 128)
        for g, (i, p) in enumerate(zip(insts, split(psi, insts))):
            ref = orc.dos_corr(i.csr, i.rescale, p, dts[g], 128)
            assert np.max(np.abs(c[g] - ref)) <= 3e-5


def test_batch_rejects_single_calls_and_bad_dt():
    h = ti.graphene_csr(4, 4)
    ctx = tb.tbpm_create_batch([(h, 9.0), (h, 9.0)])
    with pytest.raises(tb.TbpmError) as e:
        tb.tbpm_dos_corr(ctx, ti.random_phase_state(64, 0), 0.3, 2)
    assert e.value.status == tb.TBPM_ERR_UNSUPPORTED
    with pytest.raises(tb.TbpmError) as e:
        tb.tbpm_batch_dos_corr(ctx, np.zeros(64, complex), [0.3, 0.0], 2)
    assert e.value.status == tb.TBPM_ERR_ARG


def test_full_batch_first_steps(orc):
    """The 40-instance batch at full size (sum N ~ 1.9e7), two steps, three
    instances checked against the oracle."""
    insts = ti.batch_instances()
    ctx = tb.tbpm_create_batch([(i.csr, i.rescale) for i in insts])
    psi = concat_states(insts)
    dts = [math.pi / i.rescale for i in insts]
    c = tb.tbpm_batch_dos_corr(ctx, psi, dts, 2)
    parts = split(psi, insts)
    for g in (0, 17, 39):
        ref = orc.dos_corr(insts[g].csr, insts[g].rescale, parts[g], dts[g], 2)
        assert np.max(np.abs(c[g] - ref)) <= TOL, g
