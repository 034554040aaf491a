"""Gradient of the band-structure energy with respect to the support functions (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Sec. "Gradient and preconditioning", Eq. gradient:
  |g_alpha> = sum_beta S_alpha,beta dOmega/d<phi_beta|
              - 1/2 sum_beta [S^-1 (Lambda + Lambda^T)]_alpha,beta |phi_beta>,
  Lambda_alpha,beta = <phi_alpha | sum_gamma S_beta,gamma dOmega/d<phi_gamma| >,
then localized, |g_alpha> <- L^(alpha) |g_alpha>.

Readings taken where the paper is silent:

* energy mode: Omega = Tr(K H) with H_alpha,beta = <phi_alpha|H|phi_beta> and K fixed and
  symmetric, so dOmega/d<phi_beta| = sum_alpha K_beta,alpha H|phi_alpha>;
* every intermediate is kept exact (no localization) and only the final gradient is
  projected on L(alpha); functions are held as dense two-level arrays over the whole box
  (small systems only);
* S^-1 is exact ("exact") or its first-order Taylor form 2 I - S ("taylor"); K, S are
  dense matrices over all functions.
"""
from __future__ import annotations

import numpy as np

from . import hamiltonian as _H


def to_box(geo, region, vec):
    """Dense [8, N1, N2, N3] array of a compressed vector on ``region`` (a Locreg)."""
    N = geo.desc.N
    return _H.uncompress(N, region, np.asarray(vec, np.float64), [0, 0, 0], tuple(N))


def from_box(geo, region, arr):
    return _H.compress(geo.desc.N, region, arr, [0, 0, 0])


def energy_gradient(geo, phi, hphi, K, S, sinv="exact"):
    """{alpha: g_alpha on L(alpha)} by Eq. gradient; ``phi`` on L, ``hphi`` on L'.

    K, S: dense symmetric matrices (n_sf x n_sf)."""
    n = len(geo.sf_atom)
    Phi = np.stack([to_box(geo, geo.L[geo.sf_atom[f]], phi[f]) for f in range(n)])
    HPhi = np.stack([to_box(geo, geo.Lp[geo.sf_atom[f]], hphi[f]) for f in range(n)])
    K = np.asarray(K, np.float64)
    S = np.asarray(S, np.float64)
    # dOmega/d<phi_beta| = sum_alpha K_beta,alpha H phi_alpha
    D = np.tensordot(K, HPhi, axes=([1], [0]))
    # chi_alpha = sum_beta S_alpha,beta dOmega/d<phi_beta|
    Chi = np.tensordot(S, D, axes=([1], [0]))
    # Lambda_alpha,beta = <phi_alpha | chi_beta>
    Lam = np.array([[float(np.sum(Phi[a] * Chi[b])) for b in range(n)] for a in range(n)])
    Sinv = np.linalg.inv(S) if sinv == "exact" else 2.0 * np.eye(n) - S
    M = 0.5 * Sinv @ (Lam + Lam.T)
    G = Chi - np.tensordot(M, Phi, axes=([1], [0]))
    return {f: from_box(geo, geo.L[geo.sf_atom[f]], G[f]) for f in range(n)}
