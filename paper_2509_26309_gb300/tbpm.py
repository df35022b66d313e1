"""ctypes binding of libtbpm.so: the C calls of include/tbpm.h under the same names.

Argument marshalling only: every step of the propagation runs in the CUDA
library. Arrays may be numpy arrays (host memory) or torch tensors (host or
the context's GPU); complex arrays are complex128 (two interleaved doubles).
Outputs follow the input: a CUDA tensor in gives CUDA tensors out (the call is
then asynchronous on the context's stream), anything else gives numpy arrays.
If the library cannot be loaded the import fails; there is no fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from .build import LIB, build as _build

TBPM_OK = 0
TBPM_ERR_ARG = -1
TBPM_ERR_CSR = -2
TBPM_ERR_NOT_HERMITIAN = -3
TBPM_ERR_RESCALE = -4
TBPM_ERR_OOM = -5
TBPM_ERR_CUDA = -6
TBPM_ERR_TIMEOUT = -7
TBPM_ERR_NO_DEVICE = -8
TBPM_ERR_UNSUPPORTED = -9

TBPM_FP64 = 0
TBPM_FP32 = 1
TBPM_PATH_AUTO = 0
TBPM_PATH_SELL = 1
TBPM_PATH_STENCIL = 2
TBPM_F_NO_HERMITIAN_CHECK = 0x1
TBPM_F_FORCE_RESCALE = 0x2
TBPM_F_RENORM = 0x4
TBPM_F_NO_CLUSTER = 0x8
TBPM_F_AUTOTUNE = 0x10
TBPM_F_NO_TBLOCK = 0x20
TBPM_F_NO_PDL = 0x40
TBPM_F_PLAIN_SELL = 0x80
TBPM_LATTICE_GRAPHENE = 0
TBPM_LATTICE_AB_BILAYER = 1


class tbpm_opts(C.Structure):
    _fields_ = [("precision", C.c_int), ("path", C.c_int), ("flags", C.c_uint),
                ("device", C.c_int), ("stream", C.c_void_p), ("bessel_tol", C.c_double),
                ("block_threads", C.c_int), ("slices_per_warp", C.c_int)]


class tbpm_lattice(C.Structure):
    _fields_ = [("kind", C.c_int), ("l1", C.c_int64), ("l2", C.c_int64), ("t", C.c_double),
                ("t_perp", C.c_double), ("onsite", C.c_void_p)]


class tbpm_info(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("path", C.c_int), ("precision", C.c_int),
                ("real_values", C.c_int), ("num_terms", C.c_int), ("passes", C.c_int64),
                ("kernel_launches", C.c_int64), ("gershgorin", C.c_double), ("rescale", C.c_double),
                ("grid_blocks", C.c_int), ("tuned", C.c_int), ("fermi_terms", C.c_int),
                ("block_threads", C.c_int), ("slices_per_warp", C.c_int), ("tune_candidates", C.c_int),
                ("tune_default_us", C.c_double), ("tune_best_us", C.c_double), ("packed", C.c_int)]


class TbpmError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__(f"{what}: {tbpm_strerror(status)} ({status})")
        self.status = status


_lib = None

# name: (restype, argtypes) for every entry point the header declares
SIGNATURES = {
    "tbpm_default_opts": (C.c_int, [C.c_void_p]),
    "tbpm_create": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_double, C.c_void_p]),
    "tbpm_create_lattice": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]),
    "tbpm_destroy": (None, [C.c_void_p]),
    "tbpm_dos_corr": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_void_p]),
    "kpm_moments": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p]),
    "tbpm_dos_from_corr": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_void_p,
                                     C.c_void_p]),
    "kpm_dos_jackson": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "tbpm_get_info": (C.c_int, [C.c_void_p, C.c_void_p]),
    "tbpm_strerror": (C.c_char_p, [C.c_int]),
    "tbpm_last_error": (C.c_char_p, [C.c_void_p]),
    "tbpm_propagate": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_void_p,
                                 C.c_void_p]),
    "tbpm_haydock": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "tbpm_quasi_eigenstates": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_void_p, C.c_int,
                                         C.c_void_p]),
    "tbpm_haydock_ldos": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_int,
                                    C.c_double, C.c_void_p]),
    "tbpm_create_batch": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    "tbpm_batch_dos_corr": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p]),
    "tbpm_dos_corr_noalloc": (C.c_int, [C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p, C.c_double,
                                        C.c_void_p, C.c_double, C.c_int, C.c_void_p, C.c_void_p]),
    "tbpm_fp64_peak": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p]),
    "tbpm_set_current": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "tbpm_ac_corr": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_int,
                               C.c_void_p]),
    "tbpm_ac_cond": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_double, C.c_double,
                               C.c_void_p, C.c_int, C.c_void_p]),
}

TBPM_NOALLOC_MAX_N = 65536
TBPM_FERMI_MAX_TERMS = 8192


class tbpm_instance(C.Structure):
    _fields_ = [("n", C.c_int64), ("row_ptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
                ("rescale", C.c_double)]


def lib(build_if_missing: bool = True) -> C.CDLL:
    """The loaded libtbpm.so (built in-tree on first use when missing)."""
    global _lib
    if _lib is None:
        path = _build() if build_if_missing else LIB
        if not os.path.exists(path):
            raise ImportError(f"libtbpm.so not found at {path}")
        l = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(l, name)
            f.restype = res
            f.argtypes = args
        _lib = l
    return _lib


def tbpm_strerror(status: int) -> str:
    return lib().tbpm_strerror(int(status)).decode()


def _check(status: int, what: str, ctx: "Ctx | None" = None):
    if status != TBPM_OK:
        detail = lib().tbpm_last_error(ctx.handle).decode() if ctx is not None and ctx.handle else ""
        raise TbpmError(status, f"{what} [{detail}]" if detail else what)


# ------------------------------------------------------------ marshalling

def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a):
    """Address of a contiguous numpy array or torch tensor."""
    if _is_torch(a):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(a.data_ptr())
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data_as(C.c_void_p)


def _complex_in(a, n: int):
    """Returns (array, nstates, on_cuda) for a complex128 (n,) or (nstates, n) input."""
    if _is_torch(a):
        import torch
        if a.dtype != torch.complex128:
            raise TypeError("psi0 must be complex128")
        a = a.contiguous()
        on_cuda = a.is_cuda
    else:
        a = np.ascontiguousarray(a, dtype=np.complex128)
        on_cuda = False
    if a.ndim == 1:
        ns = 1
    elif a.ndim == 2:
        ns = a.shape[0]
    else:
        raise ValueError("psi0 must be 1-D or 2-D (nstates, n)")
    if a.shape[-1] != n:
        raise ValueError(f"psi0 has {a.shape[-1]} orbitals, the context {n}")
    return a, ns, on_cuda


def _alloc(shape, dtype, like_cuda: bool, device=None):
    if like_cuda:
        import torch
        td = {np.complex128: torch.complex128, np.float64: torch.float64}[dtype]
        return torch.empty(shape, dtype=td, device=device)
    return np.empty(shape, dtype=dtype)


class Ctx:
    """An owned tbpm_ctx handle; freed by tbpm_destroy or when collected."""

    def __init__(self, handle: C.c_void_p, n: int, device: int):
        self.handle = handle
        self.n = n
        self.device = device

    def __del__(self):
        try:
            tbpm_destroy(self)
        except Exception:
            pass


def make_opts(precision: int = TBPM_FP64, path: int = TBPM_PATH_AUTO, flags: int = 0,
              device: int = -1, stream=None, bessel_tol: float = 0.0, block_threads: int = 0,
              slices_per_warp: int = 0) -> tbpm_opts:
    o = tbpm_opts()
    _check(lib().tbpm_default_opts(C.byref(o)), "tbpm_default_opts")
    o.precision, o.path, o.flags, o.device = precision, path, flags, device
    o.stream = stream if stream is None else C.c_void_p(int(stream))
    o.bessel_tol = bessel_tol
    o.block_threads, o.slices_per_warp = block_threads, slices_per_warp
    return o


def tbpm_create(n: int, row_ptr, col, val, rescale: float, opts: tbpm_opts | None = None) -> Ctx:
    """Solver context for a CSR Hamiltonian (host arrays: int64, int32, complex128)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    val = np.ascontiguousarray(val, dtype=np.complex128)
    if row_ptr.shape != (n + 1,):
        raise ValueError("row_ptr must have n + 1 entries")
    h = C.c_void_p()
    _check(lib().tbpm_create(C.byref(h), int(n), _ptr(row_ptr), _ptr(col), _ptr(val),
                             float(rescale), C.byref(opts) if opts is not None else None),
           "tbpm_create")
    return Ctx(h, int(n), opts.device if opts is not None else -1)


def tbpm_create_lattice(kind: int, l1: int, l2: int, t: float, t_perp: float = 0.0,
                        onsite=None, rescale: float = 9.0, opts: tbpm_opts | None = None) -> Ctx:
    """Solver context for a periodic graphene (kind 0) or AB-bilayer (kind 1) supercell."""
    per = 2 if kind == TBPM_LATTICE_GRAPHENE else 4
    n = per * l1 * l2
    lat = tbpm_lattice(kind, l1, l2, t, t_perp, None)
    if onsite is not None:
        onsite = np.ascontiguousarray(onsite, dtype=np.float64)
        if onsite.shape != (n,):
            raise ValueError("onsite must have one entry per orbital")
        lat.onsite = onsite.ctypes.data_as(C.c_void_p)
    h = C.c_void_p()
    _check(lib().tbpm_create_lattice(C.byref(h), C.byref(lat), float(rescale),
                                     C.byref(opts) if opts is not None else None),
           "tbpm_create_lattice")
    return Ctx(h, n, opts.device if opts is not None else -1)


def tbpm_create_batch(instances, opts: tbpm_opts | None = None) -> Ctx:
    """One context for a list of (csr, rescale) instances; csr has n, row_ptr, col, val."""
    keep = []
    arr = (tbpm_instance * len(instances))()
    for g, (h, rescale) in enumerate(instances):
        rp = np.ascontiguousarray(h.row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(h.col, dtype=np.int32)
        val = np.ascontiguousarray(h.val, dtype=np.complex128)
        keep += [rp, col, val]
        arr[g] = tbpm_instance(int(h.n), rp.ctypes.data, col.ctypes.data, val.ctypes.data, float(rescale))
    hnd = C.c_void_p()
    _check(lib().tbpm_create_batch(C.byref(hnd), len(instances), arr,
                                   C.byref(opts) if opts is not None else None), "tbpm_create_batch")
    ctx = Ctx(hnd, int(sum(h.n for h, _ in instances)), opts.device if opts is not None else -1)
    ctx.inst_n = [int(h.n) for h, _ in instances]
    return ctx


def tbpm_batch_dos_corr(ctx: Ctx, psi0, dt, n_steps: int, out=None):
    """C_g(t_n) for every instance g: shape (ninst, n_steps+1). psi0 is the
    concatenation of the instances' states (complex128, sum n_g entries)."""
    a, ns, cuda = _complex_in(psi0, ctx.n)
    g = len(ctx.inst_n)
    dt = np.ascontiguousarray(np.broadcast_to(np.asarray(dt, dtype=np.float64), (g,)))
    if out is None:
        out = _alloc((g, n_steps + 1), np.complex128, cuda, a.device if cuda else None)
    _check(lib().tbpm_batch_dos_corr(ctx.handle, _ptr(a), dt.ctypes.data_as(C.c_void_p), int(n_steps),
                                     _ptr(out)), "tbpm_batch_dos_corr", ctx)
    return out


def tbpm_dos_corr_noalloc(n: int, row_ptr, col, val, rescale: float, psi0, dt: float,
                          n_steps: int, corr, stream=None) -> None:
    """The allocation-free correlation call. Every array is a caller-owned,
    contiguous CUDA tensor on one device: int64 row_ptr[n+1], int32 col[nnz],
    complex128 val[nnz] (nnz = row_ptr[n]), psi0[n] and corr[>= n_steps+1].
    The C call reads these buffers on the device only and cannot check their
    sizes, so they are checked here before it runs (on psi0's device). The
    call allocates nothing and leaves corr to be read after the stream
    synchronises."""
    import torch
    want = (("row_ptr", row_ptr, torch.int64), ("col", col, torch.int32), ("val", val, torch.complex128),
            ("psi0", psi0, torch.complex128), ("corr", corr, torch.complex128))
    for name, t, dtype in want:
        if not (_is_torch(t) and t.is_cuda and t.is_contiguous()):
            raise TypeError(f"tbpm_dos_corr_noalloc: {name} must be a contiguous CUDA tensor")
        if t.dtype != dtype:
            raise TypeError(f"tbpm_dos_corr_noalloc: {name} must be {dtype}, not {t.dtype}")
    for name, t, _ in want:
        if t.device != psi0.device:
            raise ValueError(f"tbpm_dos_corr_noalloc: {name} is on {t.device}, psi0 on {psi0.device}")
    n, n_steps = int(n), int(n_steps)
    if n >= 1:
        if row_ptr.numel() != n + 1:
            raise ValueError(f"tbpm_dos_corr_noalloc: row_ptr has {row_ptr.numel()} entries, not n + 1 = {n + 1}")
        if psi0.numel() != n:
            raise ValueError(f"tbpm_dos_corr_noalloc: psi0 has {psi0.numel()} entries, not n = {n}")
        if n_steps >= 0 and corr.numel() < n_steps + 1:
            raise ValueError(f"tbpm_dos_corr_noalloc: corr has {corr.numel()} entries, needs {n_steps + 1}")
        if n <= TBPM_NOALLOC_MAX_N:
            # the structure must lie inside col and val: row_ptr[0] = 0 and
            # row_ptr[n] = nnz (two 8-byte reads into host scalars, no device
            # allocation; monotonicity is the caller's)
            r0, rn = int(row_ptr[0].item()), int(row_ptr[n].item())
            if r0 != 0 or rn != col.numel() or col.numel() != val.numel():
                raise ValueError("tbpm_dos_corr_noalloc: row_ptr[0] must be 0 and row_ptr[n] = col.numel() "
                                 "= val.numel()")
    s = None if stream is None else C.c_void_p(int(stream))
    with torch.cuda.device(psi0.device):
        _check(lib().tbpm_dos_corr_noalloc(n, _ptr(row_ptr), _ptr(col), _ptr(val), float(rescale),
                                           _ptr(psi0), float(dt), n_steps, _ptr(corr), s),
               "tbpm_dos_corr_noalloc")


def tbpm_fp64_peak(device: int = -1, iters: int = 20000, reps: int = 3) -> tuple[float, float]:
    """(FP64 TFLOP/s, ms per launch) of an FMA-only kernel on the device: the
    measured ceiling of the FP64 sweeps."""
    tf, ms = C.c_double(), C.c_double()
    _check(lib().tbpm_fp64_peak(int(device), int(iters), int(reps), C.byref(tf), C.byref(ms)), "tbpm_fp64_peak")
    return tf.value, ms.value


def tbpm_destroy(ctx: Ctx) -> None:
    if ctx.handle:
        lib().tbpm_destroy(ctx.handle)
        ctx.handle = None


def tbpm_dos_corr(ctx: Ctx, psi0, dt: float, n_steps: int, out=None):
    """C(t_n) = <psi0|psi(t_n)>, n = 0..n_steps: shape (n_steps+1,) or (nstates, n_steps+1)."""
    a, ns, cuda = _complex_in(psi0, ctx.n)
    if out is None:
        out = _alloc((ns, n_steps + 1), np.complex128, cuda, a.device if cuda else None)
    _check(lib().tbpm_dos_corr(ctx.handle, _ptr(a), ns, float(dt), int(n_steps), _ptr(out)),
           "tbpm_dos_corr", ctx)
    return out[0] if (a.ndim == 1 and out.shape[0] == 1) else out


def tbpm_propagate(ctx: Ctx, psi0, dt: float, n_steps: int, with_corr: bool = False):
    """psi(t_{n_steps}) (same shape as psi0), and C(t_n) too when with_corr."""
    a, ns, cuda = _complex_in(psi0, ctx.n)
    dev = a.device if cuda else None
    psi = _alloc((ns, ctx.n), np.complex128, cuda, dev)
    corr = _alloc((ns, n_steps + 1), np.complex128, cuda, dev) if with_corr else None
    _check(lib().tbpm_propagate(ctx.handle, _ptr(a), ns, float(dt), int(n_steps), _ptr(psi),
                                _ptr(corr) if corr is not None else None), "tbpm_propagate", ctx)
    if a.ndim == 1:
        psi = psi[0]
        corr = corr[0] if corr is not None else None
    return (psi, corr) if with_corr else psi


def kpm_moments(ctx: Ctx, psi0, M: int, out=None):
    """mu_m = <psi0|T_m(H~)|psi0>, m = 0..M-1 (complex): shape (M,) or (nstates, M)."""
    a, ns, cuda = _complex_in(psi0, ctx.n)
    if out is None:
        out = _alloc((ns, M), np.complex128, cuda, a.device if cuda else None)
    _check(lib().kpm_moments(ctx.handle, _ptr(a), ns, int(M), _ptr(out)), "kpm_moments", ctx)
    return out[0] if (a.ndim == 1 and out.shape[0] == 1) else out


def tbpm_quasi_eigenstates(ctx: Ctx, psi0, dt: float, n_steps: int, energies):
    """Psi(E_e) for each energy: complex128 (n_e, n)."""
    a, ns, cuda = _complex_in(psi0, ctx.n)
    if ns != 1:
        raise ValueError("tbpm_quasi_eigenstates takes one state")
    if not _is_torch(energies):
        energies = np.ascontiguousarray(energies, dtype=np.float64)
    n_e = int(energies.shape[0])
    out = _alloc((n_e, ctx.n), np.complex128, cuda, a.device if cuda else None)
    _check(lib().tbpm_quasi_eigenstates(ctx.handle, _ptr(a), float(dt), int(n_steps), _ptr(energies), n_e,
                                        _ptr(out)), "tbpm_quasi_eigenstates", ctx)
    return out


def tbpm_haydock(ctx: Ctx, psi0, M: int):
    """Haydock recursion coefficients (a[M], b[M]) from psi0, b[n] = b_{n+1}."""
    a_, ns, cuda = _complex_in(psi0, ctx.n)
    if ns != 1:
        raise ValueError("tbpm_haydock takes one start state")
    dev = a_.device if cuda else None
    a = _alloc((M,), np.float64, cuda, dev)
    b = _alloc((M,), np.float64, cuda, dev)
    _check(lib().tbpm_haydock(ctx.handle, _ptr(a_), int(M), _ptr(a), _ptr(b)), "tbpm_haydock", ctx)
    return a, b


def tbpm_haydock_ldos(ctx: Ctx, a, b, energies, eta: float):
    """LDOS -Im G(E + i eta)/pi from the recursion coefficients (numpy or torch)."""
    cuda = _is_torch(a) and a.is_cuda
    if not _is_torch(a):
        a = np.ascontiguousarray(a, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        energies = np.ascontiguousarray(energies, dtype=np.float64)
    out = _alloc((energies.shape[0],), np.float64, cuda, a.device if cuda else None)
    _check(lib().tbpm_haydock_ldos(ctx.handle, _ptr(a), _ptr(b), int(a.shape[0]), _ptr(energies),
                                   int(energies.shape[0]), float(eta), _ptr(out)), "tbpm_haydock_ldos", ctx)
    return out


def tbpm_dos_from_corr(ctx: Ctx, corr, dt: float):
    """(energies[2N], dos[2N]) of the Hann-windowed transform of corr[N+1]."""
    cuda = _is_torch(corr) and corr.is_cuda
    if not _is_torch(corr):
        corr = np.ascontiguousarray(corr, dtype=np.complex128)
    n_steps = corr.shape[-1] - 1
    dev = corr.device if cuda else None
    e = _alloc((2 * n_steps,), np.float64, cuda, dev)
    d = _alloc((2 * n_steps,), np.float64, cuda, dev)
    _check(lib().tbpm_dos_from_corr(ctx.handle, _ptr(corr), int(n_steps), float(dt), _ptr(e), _ptr(d)),
           "tbpm_dos_from_corr", ctx)
    return e, d


def kpm_dos_jackson(ctx: Ctx, mu, n_e: int):
    """(energies[n_e], rho[n_e]) of the Jackson-kernel KPM DOS on Chebyshev nodes."""
    cuda = _is_torch(mu) and mu.is_cuda
    if not _is_torch(mu):
        mu = np.ascontiguousarray(mu, dtype=np.complex128)
    dev = mu.device if cuda else None
    e = _alloc((n_e,), np.float64, cuda, dev)
    r = _alloc((n_e,), np.float64, cuda, dev)
    _check(lib().kpm_dos_jackson(ctx.handle, _ptr(mu), int(mu.shape[-1]), int(n_e), _ptr(e), _ptr(r)),
           "kpm_dos_jackson", ctx)
    return e, r


def tbpm_set_current(ctx: Ctx, row_ptr, col, jx, jy) -> None:
    """Current operators J_x, J_y on one CSR pattern (host arrays: int64, int32,
    complex128, complex128)."""
    row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    jx = np.ascontiguousarray(jx, dtype=np.complex128)
    jy = np.ascontiguousarray(jy, dtype=np.complex128)
    if row_ptr.shape != (ctx.n + 1,):
        raise ValueError("row_ptr must have n + 1 entries")
    nnz = int(row_ptr[-1])
    if col.shape != (nnz,) or jx.shape != (nnz,) or jy.shape != (nnz,):
        raise ValueError("col, jx and jy must have row_ptr[n] entries")
    _check(lib().tbpm_set_current(ctx.handle, _ptr(row_ptr), _ptr(col), _ptr(jx), _ptr(jy)), "tbpm_set_current",
           ctx)


def tbpm_ac_corr(ctx: Ctx, psi0, beta: float, mu: float, dt: float, n_steps: int, out=None):
    """C_ab(t_n) for ab = xx, xy, yx, yy: complex128 (4, n_steps + 1)."""
    a, ns, cuda = _complex_in(psi0, ctx.n)
    if ns != 1:
        raise ValueError("tbpm_ac_corr takes one state")
    if out is None:
        out = _alloc((4, n_steps + 1), np.complex128, cuda, a.device if cuda else None)
    _check(lib().tbpm_ac_corr(ctx.handle, _ptr(a), float(beta), float(mu), float(dt), int(n_steps), _ptr(out)),
           "tbpm_ac_corr", ctx)
    return out


def tbpm_ac_cond(ctx: Ctx, corr, dt: float, beta: float, area: float, omegas):
    """Re sigma_ab(w) for the four rows of corr (4, n_steps + 1): float64 (4, n_w)."""
    cuda = _is_torch(corr) and corr.is_cuda
    if not _is_torch(corr):
        corr = np.ascontiguousarray(corr, dtype=np.complex128)
    if not _is_torch(omegas):
        omegas = np.ascontiguousarray(omegas, dtype=np.float64)
    if tuple(corr.shape[:1]) != (4,):
        raise ValueError("corr must have 4 rows")
    n_steps = int(corr.shape[-1]) - 1
    n_w = int(omegas.shape[0])
    out = _alloc((4, n_w), np.float64, cuda, corr.device if cuda else None)
    _check(lib().tbpm_ac_cond(ctx.handle, _ptr(corr), n_steps, float(dt), float(beta), float(area), _ptr(omegas),
                              n_w, _ptr(out)), "tbpm_ac_cond", ctx)
    return out


def tbpm_last_error(ctx: Ctx) -> str:
    """The detail of the context's last failure ("" if none)."""
    return lib().tbpm_last_error(ctx.handle).decode()


def tbpm_get_info(ctx: Ctx) -> dict:
    info = tbpm_info()
    _check(lib().tbpm_get_info(ctx.handle, C.byref(info)), "tbpm_get_info", ctx)
    return {name: getattr(info, name) for name, _ in tbpm_info._fields_}
