"""GB300 (sm_103a) implementation of the TBPM hot path: Chebyshev time
evolution of random-phase states, the DOS correlation C(t_n) and KPM moments.

The compute runs in libtbpm.so (hand-written CUDA); this package only builds
it and marshals arguments through ctypes (``tbpm``).
"""
from .tbpm import (  # noqa: F401
    Ctx, TbpmError, make_opts, lib,
    tbpm_create, tbpm_create_lattice, tbpm_destroy, tbpm_dos_corr, kpm_moments,
    tbpm_dos_from_corr, kpm_dos_jackson, tbpm_get_info, tbpm_strerror,
    tbpm_create_batch, tbpm_batch_dos_corr, tbpm_propagate, tbpm_dos_corr_noalloc,
    tbpm_haydock, tbpm_haydock_ldos, tbpm_quasi_eigenstates,
    tbpm_set_current, tbpm_ac_corr, tbpm_ac_cond, TBPM_FERMI_MAX_TERMS, tbpm_last_error, tbpm_fp64_peak,
    TBPM_OK, TBPM_ERR_ARG, TBPM_ERR_CSR, TBPM_ERR_NOT_HERMITIAN, TBPM_ERR_RESCALE,
    TBPM_ERR_OOM, TBPM_ERR_CUDA, TBPM_ERR_TIMEOUT, TBPM_ERR_NO_DEVICE, TBPM_ERR_UNSUPPORTED,
    TBPM_FP64, TBPM_FP32, TBPM_PATH_AUTO, TBPM_PATH_SELL, TBPM_PATH_STENCIL,
    TBPM_F_NO_HERMITIAN_CHECK, TBPM_F_FORCE_RESCALE, TBPM_F_RENORM, TBPM_F_NO_CLUSTER, TBPM_F_AUTOTUNE, TBPM_F_NO_TBLOCK, TBPM_F_NO_PDL, TBPM_F_PLAIN_SELL,
    TBPM_LATTICE_GRAPHENE, TBPM_LATTICE_AB_BILAYER,
)
