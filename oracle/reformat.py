"""Reuse of support functions on a shifted geometry (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: section "Flexibility of the minimal basis formalism", subsection "Geometry
optimization": the optimized support functions of the previous geometry step are moved
with the atoms (by an interpolation scheme the paper does not specify).  Reading taken:
integer grid shifts only.  Atom a moved by shift[a] grid points; for every function f
of atom a and every member p of its new locreg, the new coefficient is the old one at
p - shift[a] if that point was a member of the old locreg (coarse part for s, fine part
for d^1..d^7), else 0.  Plain dictionary lookups, function by function.
"""
from __future__ import annotations

import numpy as np

from .geometry import gcoords, gindex


def _lookup(N, g_new, shift, g_old):
    """Index into g_old of each point g_new - shift (-1 where absent or off the box)."""
    i1, i2, i3 = gcoords(N, g_new)
    j1, j2, j3 = i1 - shift[0], i2 - shift[1], i3 - shift[2]
    inside = (j1 >= 0) & (j2 >= 0) & (j3 >= 0) & (j1 < N[0]) & (j2 < N[1]) & (j3 < N[2])
    pos = {int(g): k for k, g in enumerate(g_old)}
    src = gindex(N, j1, j2, j3)
    return np.array([pos.get(int(s), -1) if ok else -1 for s, ok in zip(src, inside)], dtype=np.int64)


def reformat(geo_dst, geo_src, shift, f, phi_src):
    """Compressed coefficients of function f on geo_dst from phi_src on geo_src."""
    N = geo_dst.desc.N
    a = geo_dst.sf_atom[f]
    Ld, Ls = geo_dst.L[a], geo_src.L[a]
    sh = np.asarray(shift[a], np.int64)
    ncd, nfd = len(Ld.coarse.g), len(Ld.fine.g)
    ncs, nfs = len(Ls.coarse.g), len(Ls.fine.g)
    out = np.zeros(ncd + 7 * nfd)
    ic = _lookup(N, Ld.coarse.g, sh, Ls.coarse.g)
    ok = ic >= 0
    out[:ncd][ok] = phi_src[ic[ok]]
    jf = _lookup(N, Ld.fine.g, sh, Ls.fine.g)
    ok = jf >= 0
    for t in range(7):
        out[ncd + t * nfd: ncd + (t + 1) * nfd][ok] = phi_src[ncs + t * nfs + jf[ok]]
    return out
