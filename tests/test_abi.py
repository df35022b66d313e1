"""The C ABI without a GPU: the library builds for sm_103a, loads, exports every
declared entry point, and rejects bad input with the documented statuses
before any GPU work. Valid input on a machine without a GPU fails loudly."""
import ctypes as C
import os
import re

import numpy as np
import pytest

import tbpm_inputs as ti
import paper_2509_26309_gb300 as tb
from paper_2509_26309_gb300 import tbpm as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if not h.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", h)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(",
                            text, flags=re.M)
    return sorted(set(n for n in names if n not in ("defined",)))


def test_every_declared_symbol_is_exported():
    names = declared_functions()
    assert "tbpm_dos_corr" in names and "kpm_moments" in names and "tbpm_create" in names
    lib = C.CDLL(B.lib().__dict__["_name"])
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(B.SIGNATURES)


def test_statuses_have_names():
    for s in range(0, -10, -1):
        assert tb.tbpm_strerror(s) != "unknown status"
    assert tb.tbpm_strerror(-99) == "unknown status"
    assert B.lib().tbpm_last_error(None) == b""


def _h():
    return ti.graphene_csr(4, 4)


def _create(h, rescale=9.0, opts=None, row_ptr=None, col=None, val=None):
    rp = h.row_ptr if row_ptr is None else row_ptr
    try:
        tb.tbpm_create(h.n, rp, h.col if col is None else col, h.val if val is None else val,
                       rescale, opts)
    except tb.TbpmError as e:
        return e.status
    return 0


def test_rejects_bad_csr():
    h = _h()
    rp = h.row_ptr.copy(); rp[3], rp[4] = rp[4], rp[3]
    assert _create(h, row_ptr=rp) == tb.TBPM_ERR_CSR
    col = h.col.copy(); col[5] = h.n
    assert _create(h, col=col) == tb.TBPM_ERR_CSR
    col = h.col.copy(); col[0] = -1
    assert _create(h, col=col) == tb.TBPM_ERR_CSR
    rp = h.row_ptr.copy(); rp[0] = 1
    assert _create(h, row_ptr=rp) == tb.TBPM_ERR_CSR


def test_rejects_non_hermitian():
    h = _h()
    val = h.val.copy(); val[0] = -2.0
    assert _create(h, val=val) == tb.TBPM_ERR_NOT_HERMITIAN
    hd = ti.graphene_csr(4, 4, onsite=np.zeros(32))
    val = hd.val.copy()
    diag = np.where(hd.col == np.repeat(np.arange(32), 4))[0]
    val[diag[0]] = 0.1j
    assert _create(hd, val=val) == tb.TBPM_ERR_NOT_HERMITIAN
    # with the check disabled the structural transposition is not looked at,
    # but a complex diagonal is still rejected
    o = tb.make_opts(flags=tb.TBPM_F_NO_HERMITIAN_CHECK)
    assert _create(hd, val=val, opts=o) == tb.TBPM_ERR_NOT_HERMITIAN


def test_rejects_small_rescale_and_bad_args():
    h = _h()
    assert _create(h, rescale=8.0) == tb.TBPM_ERR_RESCALE
    assert _create(h, rescale=-1.0) == tb.TBPM_ERR_ARG
    assert _create(h, rescale=float("nan")) == tb.TBPM_ERR_ARG
    assert _create(h, opts=tb.make_opts(precision=7)) == tb.TBPM_ERR_ARG
    assert _create(h, opts=tb.make_opts(path=tb.TBPM_PATH_STENCIL)) == tb.TBPM_ERR_ARG
    assert _create(h, opts=tb.make_opts(flags=0x200)) == tb.TBPM_ERR_ARG
    assert _create(h, opts=tb.make_opts(flags=0x100)) == tb.TBPM_ERR_ARG    # the first undefined bit
    every = (tb.TBPM_F_NO_HERMITIAN_CHECK | tb.TBPM_F_FORCE_RESCALE | tb.TBPM_F_RENORM | tb.TBPM_F_NO_CLUSTER
             | tb.TBPM_F_AUTOTUNE | tb.TBPM_F_NO_TBLOCK | tb.TBPM_F_NO_PDL | tb.TBPM_F_PLAIN_SELL)
    assert _create(h, opts=tb.make_opts(flags=every)) != tb.TBPM_ERR_ARG
    val = h.val.copy(); val[2] = np.nan
    assert _create(h, val=val) == tb.TBPM_ERR_ARG
    # launch shapes: block widths 128..1024, 1, 2 or 4 slices per warp
    for bt, spw in ((64, 1), (384, 1), (2048, 1), (512, 3), (512, 8), (-1, 1), (512, -2)):
        assert _create(h, opts=tb.make_opts(block_threads=bt, slices_per_warp=spw)) == tb.TBPM_ERR_ARG, (bt, spw)
    for bt, spw in ((128, 1), (256, 2), (512, 4), (1024, 1), (0, 0)):
        assert _create(h, opts=tb.make_opts(block_threads=bt, slices_per_warp=spw)) != tb.TBPM_ERR_ARG, (bt, spw)
    l = B.lib()
    out = C.c_void_p()
    assert l.tbpm_create(C.byref(out), 0, None, None, None, 9.0, None) == tb.TBPM_ERR_ARG
    assert l.tbpm_create(None, 4, None, None, None, 9.0, None) == tb.TBPM_ERR_ARG
    assert l.tbpm_dos_corr(None, None, 1, 0.3, 4, None) == tb.TBPM_ERR_ARG
    assert l.kpm_moments(None, None, 1, 4, None) == tb.TBPM_ERR_ARG
    assert l.tbpm_dos_from_corr(None, None, 4, 0.3, None, None) == tb.TBPM_ERR_ARG
    assert l.kpm_dos_jackson(None, None, 4, 4, None, None) == tb.TBPM_ERR_ARG
    assert l.tbpm_get_info(None, None) == tb.TBPM_ERR_ARG
    assert l.tbpm_default_opts(None) == tb.TBPM_ERR_ARG
    tf = C.c_double()
    assert l.tbpm_fp64_peak(0, 0, 1, C.byref(tf), None) == tb.TBPM_ERR_ARG
    assert l.tbpm_fp64_peak(0, 100, 0, C.byref(tf), None) == tb.TBPM_ERR_ARG
    assert l.tbpm_fp64_peak(0, 100, 1, None, None) == tb.TBPM_ERR_ARG
    l.tbpm_destroy(None)


def test_lattice_validation():
    def st(**kw):
        args = dict(kind=tb.TBPM_LATTICE_GRAPHENE, l1=4, l2=4, t=-2.7, t_perp=0.0, onsite=None,
                    rescale=9.0)
        args.update(kw)
        try:
            tb.tbpm_create_lattice(**args)
        except tb.TbpmError as e:
            return e.status
        return 0
    assert st(kind=5) == tb.TBPM_ERR_ARG
    assert st(l1=2) == tb.TBPM_ERR_ARG
    assert st(rescale=8.0) == tb.TBPM_ERR_RESCALE
    assert st(kind=tb.TBPM_LATTICE_AB_BILAYER, t_perp=0.39, rescale=8.2) == tb.TBPM_ERR_RESCALE
    assert st(onsite=np.full(32, 1.5)) == tb.TBPM_ERR_RESCALE


@pytest.mark.skipif(os.path.exists("/dev/nvidia0"), reason="checks the no-GPU behaviour")
def test_valid_input_without_gpu_fails_loudly():
    assert _create(_h()) == tb.TBPM_ERR_NO_DEVICE
