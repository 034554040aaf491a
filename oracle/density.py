"""Electronic density rho(r) = sum_ab phi_a(r) K^ab phi_b(r) on the fine grid (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Sec. II.A, Eq. density (the density from the support functions and the density
kernel K^ab); App. D (the charge density is computed like the scalar products, pair by
pair over overlapping support functions).  The reading taken here:

* the value of phi_a at the fine point x_j = j h/2 is the real-space value the
  Hamiltonian's potential step uses: u_a = M W L phi_a (uncompress, one-level
  synthesis, magic filter, the same passes as ``hamiltonian.apply_hamiltonian``), on
  the real-space block of the locreg's coarse bounding box, zero outside;
* rho_j = sum over pattern entries (a, b) of K_ab u_a(j) u_b(j), with K given as values
  on the CSR pattern of H and S (entries outside the pattern are zero).  rho_j is the
  electron count carried by point j (u_j carries the factor (h/2)^(3/2) of the
  orthonormal basis), so rho(x_j) = rho_j / (h/2)^3 and sum_j V_j rho_j =
  sum_ab K_ab <phi_a|V|phi_b> with the potential matrix of the Hamiltonian;
* the grid is the caller's fine-index block [lo, lo + dims), stored [z][y][x]
  (x fastest), like the potential.

Every pair is accumulated as its own array product on the overlap of the two blocks:
no blocking, no symmetry folding.  ``absolute=True`` runs the same steps with |K|,
|phi| and the absolute filter taps: the result bounds |rho_j| term by term and is the
scale of the rounding error of any evaluation order.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from . import filters as _filters
from . import hamiltonian as _H


def abs_filters(F):
    """The filter set with every tap replaced by its absolute value."""
    return dataclasses.replace(F, h=np.abs(F.h), g=np.abs(F.g), magic=np.abs(F.magic))


def realspace_block(c, lo, F):
    """u = M W c for dense type arrays c[t, x, y, z] on the coarse block at ``lo``.

    Returns (u indexed [x, y, z], global fine index of u[0, 0, 0])."""
    cf, st = _H.synthesis3d(c, lo, F)
    return _H.magic3d(cf, st, F)


def realspace(geo, f, phi_f, F):
    """Real-space values of support function f on its block (Sec. II.B, Eq. phi)."""
    a = geo.sf_atom[f]
    L = geo.L[a]
    shape = tuple(L.hi - L.lo + 1)
    c = _H.uncompress(geo.desc.N, L, np.asarray(phi_f, np.float64), L.lo, shape)
    return realspace_block(c, list(L.lo), F)


def accumulate(fields, entries, grid_lo, grid_dims):
    """rho[z, y, x] = sum over (a, b, k) in ``entries`` of k u_a u_b.

    ``fields`` maps a function to (u [x, y, z], global start); each product is taken on
    the overlap of the two blocks and added where it lies on the grid block."""
    rho = np.zeros(tuple(int(grid_dims[d]) for d in (2, 1, 0)))
    for a, b, k in entries:
        if k == 0.0:
            continue
        ua, sa = fields[a]
        ub, sb = fields[b]
        lo = [max(sa[d], sb[d], grid_lo[d]) for d in range(3)]
        hi = [min(sa[d] + ua.shape[d], sb[d] + ub.shape[d], grid_lo[d] + grid_dims[d]) for d in range(3)]
        if any(hi[d] <= lo[d] for d in range(3)):
            continue
        pa = ua[tuple(slice(lo[d] - sa[d], hi[d] - sa[d]) for d in range(3))]
        pb = ub[tuple(slice(lo[d] - sb[d], hi[d] - sb[d]) for d in range(3))]
        prod = k * pa * pb                                   # [x, y, z]
        rho[tuple(slice(lo[d] - grid_lo[d], hi[d] - grid_lo[d]) for d in (2, 1, 0))] += prod.transpose(2, 1, 0)
    return rho


def pattern_entries(row_ptr, col, K):
    """(a, b, K_ab) for every stored entry of the CSR pattern."""
    out = []
    for a in range(len(row_ptr) - 1):
        for k in range(row_ptr[a], row_ptr[a + 1]):
            out.append((a, int(col[k]), float(K[k])))
    return out


def density(geo, phi, K, grid_lo, grid_dims, F=None, absolute=False):
    """rho_j = sum_ab K_ab u_a(j) u_b(j) on the grid block (Eq. density).

    ``phi`` maps function -> compressed vector on L; ``K`` holds values on the pattern
    (geo.row_ptr, geo.col).  Returns rho indexed [z, y, x]."""
    F = F or _filters.load()
    Kv = np.asarray(K, np.float64)
    if absolute:
        F = abs_filters(F)
        Kv = np.abs(Kv)
    entries = pattern_entries(geo.row_ptr, geo.col, Kv)
    need = sorted({a for a, _, _ in entries} | {b for _, b, _ in entries})
    fields = {}
    for f in need:
        v = np.asarray(phi[f], np.float64)
        fields[f] = realspace(geo, f, np.abs(v) if absolute else v, F)
    return accumulate(fields, entries, grid_lo, grid_dims)


def density_points(geo, phi, K, points, F=None, absolute=False):
    """rho_j at the listed fine points only: at each point, the sum over the pattern
    entries (a, b) of K_ab u_a(j) u_b(j) for the functions a, b whose blocks contain it
    (taken row by row of the pattern; same steps as ``density`` otherwise).

    ``points``: (n, 3) global fine indices (x, y, z).  ``phi`` maps function -> vector
    for at least the functions whose blocks contain a point.  Returns (n,) values."""
    F = F or _filters.load()
    Kv = np.asarray(K, np.float64)
    if absolute:
        F = abs_filters(F)
        Kv = np.abs(Kv)
    pts = np.asarray(points, np.int64).reshape(-1, 3)
    rp, col = geo.row_ptr, geo.col
    # real-space block of every function: fine points [2 lo - 14, 2 hi + 16]
    blo = np.array([2 * np.asarray(geo.L[a].lo) - 14 for a in geo.sf_atom], np.int64).reshape(-1, 3)
    bhi = np.array([2 * np.asarray(geo.L[a].hi) + 16 for a in geo.sf_atom], np.int64).reshape(-1, 3)
    covers = [np.nonzero(np.all((blo <= p) & (p <= bhi), axis=1))[0] for p in pts]
    fields = {}
    for f in sorted(set(int(f) for c in covers for f in c)):
        v = np.asarray(phi[f], np.float64)
        fields[f] = realspace(geo, f, np.abs(v) if absolute else v, F)
    out = np.zeros(len(pts))
    for i, p in enumerate(pts):
        C = covers[i]
        if len(C) == 0:
            continue
        uval = np.empty(len(C))
        for j, f in enumerate(C):
            u, st = fields[int(f)]
            uval[j] = u[p[0] - st[0], p[1] - st[1], p[2] - st[2]]
        acc = 0.0
        for ia, a in enumerate(C):
            cols = col[rp[a]:rp[a + 1]]
            sel = np.isin(cols, C)
            ub = uval[np.searchsorted(C, cols[sel])]
            acc += uval[ia] * float(np.dot(Kv[rp[a]:rp[a + 1]][sel], ub))
        out[i] = acc
    return out
