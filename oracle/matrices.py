"""Sparse overlap and Hamiltonian matrices on the pair pattern (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Sec. II.A, S_ab = <phi_a|phi_b> and H_ab = <phi_a|H_KS|phi_b>; Sec. IV.A
("Suitability of the methods": sparse matrices in compressed form with the pattern
given by the localization regions); App. D (scalar products between overlapping
support functions).  In the orthonormal Daubechies basis a scalar product is the dot
product of the expansion coefficients of the basis functions both vectors carry:

  S_ab = sum_{p in L(a) n L(b)} s_a(p) s_b(p) + sum_{p in F(a) n F(b)} sum_l d_a^l(p) d_b^l(p)
  H_ab = the same over L(a) n L'(b) with H phi_b        (raw, not symmetrized)

Both are evaluated directly from the member lists, pair by pair.
"""
from __future__ import annotations

import numpy as np


def _dot(Ra, xa, Rb, xb) -> float:
    """Coefficient dot product of two compressed vectors over their common points."""
    nca, nfa = len(Ra.coarse.g), len(Ra.fine.g)
    ncb, nfb = len(Rb.coarse.g), len(Rb.fine.g)
    _, ia, ib = np.intersect1d(Ra.coarse.g, Rb.coarse.g, assume_unique=True, return_indices=True)
    acc = float(np.dot(xa[ia], xb[ib]))
    _, ja, jb = np.intersect1d(Ra.fine.g, Rb.fine.g, assume_unique=True, return_indices=True)
    for t in range(7):
        acc += float(np.dot(xa[nca + t * nfa + ja], xb[ncb + t * nfb + jb]))
    return acc


def overlap_entry(geo, a, b, phi_a, phi_b) -> float:
    A, B = geo.sf_atom[a], geo.sf_atom[b]
    return _dot(geo.L[A], phi_a, geo.L[B], phi_b)


def hamiltonian_entry(geo, a, b, phi_a, hphi_b) -> float:
    A, B = geo.sf_atom[a], geo.sf_atom[b]
    return _dot(geo.L[A], phi_a, geo.Lp[B], hphi_b)


def build_matrices(geo, phi, hphi, rows=None):
    """CSR values (H, S) over the pattern; ``phi``/``hphi`` map function -> vector.

    With ``rows`` given, only those rows are filled (the rest stay NaN)."""
    rp, col = geo.row_ptr, geo.col
    H = np.full(len(col), np.nan)
    S = np.full(len(col), np.nan)
    rows = range(len(rp) - 1) if rows is None else rows
    for a in rows:
        for k in range(rp[a], rp[a + 1]):
            b = int(col[k])
            S[k] = overlap_entry(geo, a, b, phi[a], phi[b])
            H[k] = hamiltonian_entry(geo, a, b, phi[a], hphi[b])
    return H, S
