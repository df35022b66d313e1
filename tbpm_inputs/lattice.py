"""Synthetic lattice Hamiltonians in CSR form (the model-building step of Sec. 3.2.1).

Monolayer graphene follows the primitive cell printed in Sec. 3.2.1: two pz
orbitals (A at 0, B at (1/3, 1/3) in lattice units), hopping t = -2.7 eV, and
the three hopping terms <A,0|H|B,0> = t, <B,0|H|A,a1> = t, <B,0|H|A,a2> = t,
completed by H_ij(R) = H_ji(-R)^*. A periodic L1 x L2 supercell orders its
orbitals as i = 2*(m1*L2 + m2) + s (s = 0 for A, 1 for B).

The AB (Bernal) bilayer stacks a second, identical honeycomb layer shifted so
that its B site sits over the A site of layer 1. Its orbitals are ordered as
i = 4*(m1*L2 + m2) + o with o = 0 (A1), 1 (B1), 2 (A2), 3 (B2); the dimer pair
A1(m), B2(m) is coupled by t_perp = 0.39 eV.

Anderson disorder puts eps_i = W*(u_i - 1/2) on every orbital, u_i from the
SplitMix64 stream ``seed``. These builders only assemble inputs: they perform
no step of the propagation method.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from .rng import uniform01

T_GRAPHENE = -2.7
T_PERP_AB = 0.39


@dataclass
class CSR:
    """Hermitian sparse matrix: row_ptr int64[n+1], col int32[nnz], val complex128[nnz]."""

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    val: np.ndarray

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def to_dense(self) -> np.ndarray:
        d = np.zeros((self.n, self.n), dtype=np.complex128)
        rows = np.repeat(np.arange(self.n), np.diff(self.row_ptr))
        np.add.at(d, (rows, self.col.astype(np.int64)), self.val)
        return d


def anderson_onsite(n: int, w: float, seed: int) -> np.ndarray:
    """float64[n] on-site energies uniform in [-W/2, W/2)."""
    return w * (uniform01(seed, np.arange(n, dtype=np.uint64)) - 0.5)


def _assemble(n: int, cols: np.ndarray, vals: np.ndarray, valid: np.ndarray) -> CSR:
    """Rows given as padded [n, d] blocks; sort each row by column, merge duplicates."""
    big = np.int64(np.iinfo(np.int64).max)
    c = np.where(valid, cols, big)
    order = np.argsort(c, axis=1, kind="stable")
    c = np.take_along_axis(c, order, axis=1)
    v = np.take_along_axis(np.where(valid, vals, 0), order, axis=1)
    keep = c != big
    # merge duplicate columns inside a row (only possible on tiny tori)
    dup = np.zeros_like(keep)
    dup[:, 1:] = keep[:, 1:] & (c[:, 1:] == c[:, :-1])
    if dup.any():
        for j in range(c.shape[1] - 1, 0, -1):
            m = dup[:, j]
            v[m, j - 1] += v[m, j]
        keep &= ~dup
    counts = keep.sum(axis=1)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=row_ptr[1:])
    return CSR(n, row_ptr, c[keep].astype(np.int32), v[keep].astype(np.complex128))


def graphene_csr(l1: int, l2: int, t: complex = T_GRAPHENE, onsite: np.ndarray | None = None,
                 bond_phases: np.ndarray | None = None) -> CSR:
    """Periodic L1 x L2 monolayer graphene.

    ``onsite`` (float64[2*L1*L2]) adds the diagonal; without it the diagonal is
    absent (nnz = 3N). ``bond_phases`` (float64[3]) multiplies the three bond
    types (A-B in the cell, B-A along a1, B-A along a2) by exp(i*theta), which
    gives a Hermitian H with H^T != H for transposition tests.
    """
    if l1 < 1 or l2 < 1:
        raise ValueError("lattice dimensions must be positive")
    ncell = l1 * l2
    n = 2 * ncell
    th = np.zeros(3) if bond_phases is None else np.asarray(bond_phases, dtype=np.float64)
    t0, t1, t2 = (complex(t) * np.exp(1j * th[b]) for b in range(3))
    m1, m2 = np.divmod(np.arange(ncell, dtype=np.int64), l2)

    def cell(a, b):
        return (a % l1) * l2 + (b % l2)

    d = 4 if onsite is not None else 3
    cols = np.zeros((n, d), dtype=np.int64)
    vals = np.zeros((n, d), dtype=np.complex128)
    ia = 2 * cell(m1, m2)
    ib = ia + 1
    # row A(m): B(m) [t0], B(m - a1) [conj t1], B(m - a2) [conj t2]
    cols[ia, 0], vals[ia, 0] = ib, t0
    cols[ia, 1], vals[ia, 1] = 2 * cell(m1 - 1, m2) + 1, np.conj(t1)
    cols[ia, 2], vals[ia, 2] = 2 * cell(m1, m2 - 1) + 1, np.conj(t2)
    # row B(m): A(m) [conj t0], A(m + a1) [t1], A(m + a2) [t2]
    cols[ib, 0], vals[ib, 0] = ia, np.conj(t0)
    cols[ib, 1], vals[ib, 1] = 2 * cell(m1 + 1, m2), t1
    cols[ib, 2], vals[ib, 2] = 2 * cell(m1, m2 + 1), t2
    if onsite is not None:
        onsite = np.asarray(onsite, dtype=np.float64)
        if onsite.shape != (n,):
            raise ValueError("onsite must have one entry per orbital")
        cols[:, 3] = np.arange(n)
        vals[:, 3] = onsite
    return _assemble(n, cols, vals, np.ones((n, d), dtype=bool))


def bilayer_csr(l1: int, l2: int, t: float = T_GRAPHENE, t_perp: float = T_PERP_AB,
                onsite: np.ndarray | None = None) -> CSR:
    """Periodic L1 x L2 AB-stacked bilayer graphene (4 orbitals per cell)."""
    if l1 < 1 or l2 < 1:
        raise ValueError("lattice dimensions must be positive")
    ncell = l1 * l2
    n = 4 * ncell
    m1, m2 = np.divmod(np.arange(ncell, dtype=np.int64), l2)

    def cell(a, b):
        return (a % l1) * l2 + (b % l2)

    d = 5
    cols = np.zeros((n, d), dtype=np.int64)
    vals = np.zeros((n, d), dtype=np.complex128)
    valid = np.zeros((n, d), dtype=bool)
    base = 4 * cell(m1, m2)
    for layer in (0, 1):
        ia = base + 2 * layer
        ib = ia + 1
        cols[ia, 0], vals[ia, 0] = ib, t
        cols[ia, 1], vals[ia, 1] = 4 * cell(m1 - 1, m2) + 2 * layer + 1, np.conj(t)
        cols[ia, 2], vals[ia, 2] = 4 * cell(m1, m2 - 1) + 2 * layer + 1, np.conj(t)
        cols[ib, 0], vals[ib, 0] = ia, np.conj(t)
        cols[ib, 1], vals[ib, 1] = 4 * cell(m1 + 1, m2) + 2 * layer, t
        cols[ib, 2], vals[ib, 2] = 4 * cell(m1, m2 + 1) + 2 * layer, t
        valid[ia, :3] = True
        valid[ib, :3] = True
    a1, b2 = base, base + 3
    cols[a1, 3], vals[a1, 3] = b2, t_perp
    cols[b2, 3], vals[b2, 3] = a1, np.conj(t_perp)
    valid[a1, 3] = True
    valid[b2, 3] = True
    if onsite is not None:
        onsite = np.asarray(onsite, dtype=np.float64)
        if onsite.shape != (n,):
            raise ValueError("onsite must have one entry per orbital")
        cols[:, 4] = np.arange(n)
        vals[:, 4] = onsite
        valid[:, 4] = True
    return _assemble(n, cols, vals, valid)


def random_hermitian_csr(n: int, offdiag_per_row: int, seed: int, scale: float = 1.0) -> CSR:
    """Random sparse complex Hermitian matrix with a real diagonal (tests only)."""
    from .rng import splitmix64
    m = n * offdiag_per_row
    idx = np.arange(m, dtype=np.uint64)
    r = (splitmix64(seed, idx) % np.uint64(n)).astype(np.int64)
    c = (splitmix64(seed + 1, idx) % np.uint64(n)).astype(np.int64)
    re = uniform01(seed + 2, idx) - 0.5
    im = uniform01(seed + 3, idx) - 0.5
    keep = r != c
    r, c, v = r[keep], c[keep], scale * (re[keep] + 1j * im[keep])
    diag = scale * (uniform01(seed + 4, np.arange(n, dtype=np.uint64)) - 0.5)
    rows = np.concatenate([r, c, np.arange(n)])
    cols = np.concatenate([c, r, np.arange(n)])
    vals = np.concatenate([v, np.conj(v), diag.astype(np.complex128)])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    first = np.ones(rows.size, dtype=bool)
    first[1:] = (rows[1:] != rows[:-1]) | (cols[1:] != cols[:-1])
    grp = np.cumsum(first) - 1
    merged = np.zeros(int(first.sum()), dtype=np.complex128)
    np.add.at(merged, grp, vals)
    rows, cols = rows[first], cols[first]
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=n), out=row_ptr[1:])
    return CSR(n, row_ptr, cols.astype(np.int32), merged)


def gershgorin_bound(h: CSR) -> float:
    """max_i sum_j |H_ij|, an upper bound on the spectral radius."""
    rows = np.repeat(np.arange(h.n), np.diff(h.row_ptr))
    s = np.bincount(rows, weights=np.abs(h.val), minlength=h.n)
    return float(s.max()) if h.n else 0.0


# ------------------------------------------------------------ current operators

A_LATTICE = 0.246          # graphene lattice constant, nm (bond length a / sqrt(3) = 0.142 nm)


@dataclass
class Current:
    """Current operators J_x, J_y on one CSR pattern (row_ptr int64[n+1],
    col int32[nnz]) with complex128 values jx, jy."""

    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    jx: np.ndarray
    jy: np.ndarray

    def as_tuple(self):
        return self.row_ptr, self.col, self.jx, self.jy

    def to_dense(self):
        out = []
        for v in (self.jx, self.jy):
            out.append(CSR(self.n, self.row_ptr, self.col, v).to_dense())
        return out


def graphene_geometry(a: float = A_LATTICE):
    """Lattice vectors a1, a2 and the A, B positions (nm) of the primitive cell."""
    a1 = np.array([a, 0.0])
    a2 = np.array([0.5 * a, 0.5 * np.sqrt(3.0) * a])
    return a1, a2, np.zeros(2), (a1 + a2) / 3.0


def _current_from_bonds(n, cols, hvals, disp, valid) -> Current:
    """J_a with (J_a)_ij = i (r_j - r_i)_a H_ij per bond, r_j - r_i the bond
    vector (not the wrapped coordinate difference); duplicates summed."""
    jx = _assemble(n, cols, 1j * disp[..., 0] * hvals, valid)
    jy = _assemble(n, cols, 1j * disp[..., 1] * hvals, valid)
    return Current(n, jx.row_ptr, jx.col, jx.val, jy.val)


def graphene_current(l1: int, l2: int, t: complex = T_GRAPHENE, bond_phases: np.ndarray | None = None,
                     a: float = A_LATTICE) -> Current:
    """Current operators of graphene_csr(l1, l2, t, bond_phases=...)."""
    ncell = l1 * l2
    n = 2 * ncell
    th = np.zeros(3) if bond_phases is None else np.asarray(bond_phases, dtype=np.float64)
    t0, t1, t2 = (complex(t) * np.exp(1j * th[b]) for b in range(3))
    a1, a2, ra, rb = graphene_geometry(a)
    m1, m2 = np.divmod(np.arange(ncell, dtype=np.int64), l2)

    def cell(p, q):
        return (p % l1) * l2 + (q % l2)

    cols = np.zeros((n, 3), dtype=np.int64)
    vals = np.zeros((n, 3), dtype=np.complex128)
    disp = np.zeros((n, 3, 2))
    ia = 2 * cell(m1, m2)
    ib = ia + 1
    cols[ia, 0], vals[ia, 0], disp[ia, 0] = ib, t0, rb - ra
    cols[ia, 1], vals[ia, 1], disp[ia, 1] = 2 * cell(m1 - 1, m2) + 1, np.conj(t1), rb - a1 - ra
    cols[ia, 2], vals[ia, 2], disp[ia, 2] = 2 * cell(m1, m2 - 1) + 1, np.conj(t2), rb - a2 - ra
    cols[ib, 0], vals[ib, 0], disp[ib, 0] = ia, np.conj(t0), ra - rb
    cols[ib, 1], vals[ib, 1], disp[ib, 1] = 2 * cell(m1 + 1, m2), t1, ra + a1 - rb
    cols[ib, 2], vals[ib, 2], disp[ib, 2] = 2 * cell(m1, m2 + 1), t2, ra + a2 - rb
    return _current_from_bonds(n, cols, vals, disp, np.ones((n, 3), dtype=bool))


def bilayer_current(l1: int, l2: int, t: float = T_GRAPHENE, t_perp: float = T_PERP_AB,
                    a: float = A_LATTICE) -> Current:
    """Current operators of bilayer_csr(l1, l2, t, t_perp): in-plane bonds as in
    each layer, the vertical dimer bond carries no in-plane current (its
    entries are kept, with value 0)."""
    ncell = l1 * l2
    n = 4 * ncell
    a1, a2, ra, rb = graphene_geometry(a)
    m1, m2 = np.divmod(np.arange(ncell, dtype=np.int64), l2)

    def cell(p, q):
        return (p % l1) * l2 + (q % l2)

    cols = np.zeros((n, 4), dtype=np.int64)
    vals = np.zeros((n, 4), dtype=np.complex128)
    disp = np.zeros((n, 4, 2))
    valid = np.zeros((n, 4), dtype=bool)
    base = 4 * cell(m1, m2)
    for layer in (0, 1):
        ia = base + 2 * layer
        ib = ia + 1
        cols[ia, 0], vals[ia, 0], disp[ia, 0] = ib, t, rb - ra
        cols[ia, 1], vals[ia, 1], disp[ia, 1] = 4 * cell(m1 - 1, m2) + 2 * layer + 1, t, rb - a1 - ra
        cols[ia, 2], vals[ia, 2], disp[ia, 2] = 4 * cell(m1, m2 - 1) + 2 * layer + 1, t, rb - a2 - ra
        cols[ib, 0], vals[ib, 0], disp[ib, 0] = ia, t, ra - rb
        cols[ib, 1], vals[ib, 1], disp[ib, 1] = 4 * cell(m1 + 1, m2) + 2 * layer, t, ra + a1 - rb
        cols[ib, 2], vals[ib, 2], disp[ib, 2] = 4 * cell(m1, m2 + 1) + 2 * layer, t, ra + a2 - rb
        valid[ia, :3] = True
        valid[ib, :3] = True
    a1r, b2r = base, base + 3
    cols[a1r, 3], vals[a1r, 3] = b2r, t_perp
    cols[b2r, 3], vals[b2r, 3] = a1r, t_perp
    valid[a1r, 3] = True
    valid[b2r, 3] = True
    return _current_from_bonds(n, cols, vals, disp, valid)


def graphene_positions(l1: int, l2: int, a: float = A_LATTICE) -> np.ndarray:
    """float64[n, 2] orbital positions (nm) of the graphene supercell, unwrapped."""
    a1, a2, ra, rb = graphene_geometry(a)
    m1, m2 = np.divmod(np.arange(l1 * l2, dtype=np.int64), l2)
    base = m1[:, None] * a1 + m2[:, None] * a2
    out = np.zeros((2 * l1 * l2, 2))
    out[0::2] = base + ra
    out[1::2] = base + rb
    return out


def graphene_area_per_orbital(a: float = A_LATTICE) -> float:
    """Cell area |a1 x a2| / 2 orbitals, nm^2."""
    return 0.5 * (np.sqrt(3.0) / 2.0) * a * a
