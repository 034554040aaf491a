"""Sparse combinations of support functions and the Loewdin step (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Sec. "Orthogonalization" (the adaptively contracted basis is re-orthonormalized
after each update by the Loewdin procedure, with S^-1/2 replaced by its first-order
Taylor approximation since the functions are close to orthonormal) and Sec. "Gradient
and preconditioning" (Eq. gradient: sums sum_beta M_alpha,beta |phi_beta> over
overlapping functions, then localized, |g_alpha> <- L^(alpha) |g_alpha>).

Readings taken where the paper is silent:

* the primitive is (M Phi)_alpha = P_L(alpha) sum_beta M_alpha,beta phi_beta for a matrix
  M given as values on the CSR pattern of H and S (row alpha, column beta): each phi_beta
  is placed on the global two-level grid (its coefficients at its own members), and the
  sum is read back at the members of L(alpha) (coarse s, fine d^1..d^7), i.e. the
  localization projector applied to the exact sum;
* first-order Taylor approximation of S^-1/2 around the identity: (3 I - S) / 2, so the
  Loewdin step is phi'_alpha = P_L(alpha) sum_beta (3 delta - S)_alpha,beta / 2 phi_beta
  with S on the pattern.
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian as _H


def combine(geo, M, phi, rows=None):
    """{alpha: P_L(alpha) sum_beta M[alpha, beta] phi_beta} over the rows of the pattern.

    ``M`` holds values on (geo.row_ptr, geo.col); ``phi`` maps function -> compressed
    vector on L.  Every term is added on a dense block covering the box of L(alpha),
    then the result is compressed on L(alpha)."""
    N = geo.desc.N
    rp, col = geo.row_ptr, geo.col
    rows = range(len(rp) - 1) if rows is None else rows
    out = {}
    for a in rows:
        La = geo.L[geo.sf_atom[a]]
        lo = list(La.lo)
        shape = tuple(La.hi - La.lo + 1)
        acc = np.zeros((8,) + shape)
        for k in range(rp[a], rp[a + 1]):
            b = int(col[k])
            if M[k] == 0.0:
                continue
            Lb = geo.L[geo.sf_atom[b]]
            cb = _H.uncompress(N, Lb, np.asarray(phi[b], np.float64), Lb.lo, tuple(Lb.hi - Lb.lo + 1))
            _H._place(acc, lo, M[k] * cb, list(Lb.lo))
        out[a] = _H.compress(N, La, acc, lo)
    return out


def lowdin_taylor(geo, S, phi, rows=None):
    """phi'_alpha = P_L(alpha) sum_beta (3 delta_alpha,beta - S_alpha,beta) / 2 phi_beta."""
    rp, col = geo.row_ptr, geo.col
    T = np.empty(len(col))
    for a in range(len(rp) - 1):
        for k in range(rp[a], rp[a + 1]):
            T[k] = (3.0 * (int(col[k]) == a) - S[k]) / 2.0
    return combine(geo, T, phi, rows)
