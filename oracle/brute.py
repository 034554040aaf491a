"""Explicit dense matrices of the localized Hamiltonian on tiny boxes (oracle pin).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The separable oracle (``hamiltonian.py``) applies W, M, diag(V), M^T, W^T and the
kinetic blocks as 1D passes.  This module instead builds, entry by entry from the
filter definitions (Sec. II.B, Eq. phi; Sec. III.B), the 1D matrices

  S[k, (b, i)] = X_b[k - 2i]          synthesis, X_0 = h, X_1 = g
  M[j, k]      = w[j - k]             magic filter
  K[(b, i), (b', i')] = T_{b b'}(i' - i)   kinetic Galerkin block

and forms the full matrix over every basis function (b, i) of an N^3 box:

  H = -1/(2h^2) (K x I x I + I x K x I + I x I x K)
      + (MS x MS x MS)^T diag(V) (MS x MS x MS)

with one einsum contraction over the real-space grid.  A locreg result is then
P_{L'} H P_L phi.  Memory grows as (2N)^6, so N <= 6.
"""
from __future__ import annotations

import numpy as np

from . import filters as _filters
from .geometry import gcoords


def synthesis_matrix(N, F):
    """Rows: fine k = -7 .. 2N+6; columns (b, i) -> b*N + i."""
    k_lo = 2 * 0 + F.h_lo
    k_hi = 2 * (N - 1) + F.h_lo + len(F.h) - 1
    S = np.zeros((k_hi - k_lo + 1, 2 * N))
    for b, X in enumerate((F.h, F.g)):
        for i in range(N):
            for k in range(k_lo, k_hi + 1):
                m = k - 2 * i
                if F.h_lo <= m < F.h_lo + len(X):
                    S[k - k_lo, b * N + i] = X[m - F.h_lo]
    return S, k_lo


def magic_matrix(k_lo, nk, F):
    j_lo = k_lo + F.magic_lo
    nj = nk + len(F.magic) - 1
    M = np.zeros((nj, nk))
    for j in range(nj):
        for k in range(nk):
            m = (j + j_lo) - (k + k_lo)
            if F.magic_lo <= m < F.magic_lo + len(F.magic):
                M[j, k] = F.magic[m - F.magic_lo]
    return M, j_lo


def kinetic_matrix(N, F):
    K = np.zeros((2 * N, 2 * N))
    names = "hg"
    for b in range(2):
        for bp in range(2):
            T = F.kin[names[b] + names[bp]]
            for i in range(N):
                for ip in range(N):
                    l = ip - i
                    if -len(T) // 2 < l <= len(T) // 2:
                        K[b * N + i, bp * N + ip] = T[l - F.kin_lo]
    return K


def full_hamiltonian(N, h, V, V_lo, F=None):
    """Dense H over all (b1 i1, b2 i2, b3 i3) of an N^3 box; V stored [jz, jy, jx]."""
    F = F or _filters.load()
    S, k_lo = synthesis_matrix(N, F)
    M, j_lo = magic_matrix(k_lo, S.shape[0], F)
    A = M @ S
    nj = A.shape[0]
    off = [j_lo - V_lo[d] for d in range(3)]
    Vb = np.asarray(V)[off[2]:off[2] + nj, off[1]:off[1] + nj, off[0]:off[0] + nj]
    Vx = Vb.transpose(2, 1, 0)
    n = 2 * N
    Hp = np.einsum("pqr,pa,pA,qb,qB,rc,rC->abcABC", Vx, A, A, A, A, A, A, optimize=True)
    Hp = Hp.reshape(n ** 3, n ** 3)
    K = kinetic_matrix(N, F)
    I = np.eye(n)
    Kt = np.kron(np.kron(K, I), I) + np.kron(np.kron(I, K), I) + np.kron(np.kron(I, I), K)
    return Hp - Kt / (2.0 * h * h)


def basis_index(N, g, t):
    """Row of the dense matrix for type t at grid index g (cubic box N = (n, n, n))."""
    i1, i2, i3 = gcoords(N, g)
    b1, b2, b3 = t & 1, (t >> 1) & 1, (t >> 2) & 1
    m = N[0]
    n = 2 * m
    return ((b1 * m + i1) * n + (b2 * m + i2)) * n + (b3 * m + i3)


def region_rows(N, loc):
    rows = [basis_index(N, loc.coarse.g, 0)]
    for t in range(1, 8):
        rows.append(basis_index(N, loc.fine.g, t))
    return np.concatenate(rows)


def apply_dense(H, N, Lin, Lout, phi):
    """P_{L'} H P_L phi in the compressed layouts of Lin and Lout."""
    rin = region_rows(N, Lin)
    rout = region_rows(N, Lout)
    return H[np.ix_(rout, rin)] @ np.asarray(phi, np.float64)
