"""Fermi operator expansion of the density kernel (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Sec. "Density kernel optimization" (K = f(H) evaluated as a Chebyshev polynomial
of the Hamiltonian matrix) and App. "Fermi operator expansion":
  H~ = sigma (H - tau S), sigma = 2 / (e_max - e_min), tau = (e_min + e_max) / 2
  (e_min, e_max the extreme eigenvalues of H c = e S c);
  H~' = S^-1/2 H~ S^-1/2, S^-1/2 by its first-order Taylor expansion;
  K' = c_0/2 I + sum_{i=1}^{n_pl} c_i T_i(H~'), the c_i the Chebyshev coefficients of
  f(e) = 1/2 [1 - erf((e - mu) / de)] on [-1, 1] (in the scaled variable);
  columns by the recursion t^0 = e_l, t^1 = H~' e_l, t^{j+1} = 2 H~' t^j - t^{j-1};
  mu adjusted until Tr(K') equals the number of electrons;
  K = S^-1/2 K' S^-1/2, E_BS = Tr(K H~) / sigma + tau Tr(K S).

Readings taken where the paper is silent:

* the Chebyshev coefficients are those of the interpolating polynomial at the n_pl + 1
  Chebyshev nodes x_k = cos(pi (k + 1/2) / (n_pl + 1)):
  c_j = 2 / (n_pl + 1) sum_k f(x_k) T_j(x_k);
* mu and de are given in the units of the Hamiltonian; the target of Tr(K') is the
  number of occupied orbitals (occupations in [0, 1]);
* mu is found by bisection on [e_min, e_max] until |Tr(K') - n_el| <= tol;
* the matrices are dense by default; "taylor" (the paper's choice) or "exact" S^-1/2
  selects the transform;
* sparse form (``pattern``, a boolean n x n mask of the kernel's pattern, symmetric,
  diagonal included): H~' is kept on the mask and every Chebyshev column t_l^j is cut
  to the mask's column l after each product, as a linear-scaling evaluation must; with
  a complete mask the result equals the dense one.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.linalg import eigh
from scipy.special import erf


def fermi_erf(e, mu, de):
    """f(e) = 1/2 [1 - erf((e - mu) / de)] (App. FOE)."""
    return 0.5 * (1.0 - erf((np.asarray(e, np.float64) - mu) / de))


def chebyshev_coefficients(f, n_pl):
    """c_j, j = 0..n_pl, of the polynomial interpolating f at the n_pl + 1 Chebyshev nodes
    (with the c_0 / 2 convention of the expansion)."""
    N = n_pl + 1
    k = np.arange(N)
    theta = math.pi * (k + 0.5) / N
    fx = f(np.cos(theta))
    return np.array([2.0 / N * float(np.sum(fx * np.cos(j * theta))) for j in range(N)])


def chebyshev_value(c, x):
    """p(x) = c_0/2 + sum_j c_j T_j(x) by the three-term recursion."""
    x = np.asarray(x, np.float64)
    t0, t1 = np.ones_like(x), x
    p = 0.5 * c[0] * t0 + (c[1] * t1 if len(c) > 1 else 0.0)
    for j in range(2, len(c)):
        t0, t1 = t1, 2.0 * x * t1 - t0
        p = p + c[j] * t1
    return p


def s_inv_half(S, mode):
    if mode == "taylor":
        return 0.5 * (3.0 * np.eye(len(S)) - S)
    w, V = np.linalg.eigh(S)
    return (V / np.sqrt(w)) @ V.T


def spectrum_bounds(H, S):
    e = eigh(H, S, eigvals_only=True)
    return float(e[0]), float(e[-1])


def kernel_prime(Ht, c, pattern=None):
    """K' = c_0/2 I + sum c_i T_i(Ht), column by column with the Chebyshev recursion;
    with ``pattern`` every column is cut to the mask after each product."""
    n = len(Ht)
    K = np.zeros((n, n))
    for l in range(n):
        keep = np.ones(n) if pattern is None else pattern[:, l].astype(np.float64)
        t_prev = np.zeros(n)
        t_prev[l] = 1.0
        k = 0.5 * c[0] * t_prev
        if len(c) > 1:
            t = (Ht @ t_prev) * keep
            k = k + c[1] * t
            for j in range(2, len(c)):
                t_prev, t = t, (2.0 * (Ht @ t) - t_prev) * keep
                k = k + c[j] * t
        K[:, l] = k
    return K


def foe(H, S, n_el, n_pl, de, sinv="taylor", bounds=None, tol=1e-10, max_bisect=200, pattern=None):
    """Density kernel by FOE.  Returns dict(K, Kp, mu, sigma, tau, c, E_BS, bounds)."""
    H = np.asarray(H, np.float64)
    S = np.asarray(S, np.float64)
    e_min, e_max = bounds if bounds is not None else spectrum_bounds(H, S)
    sigma = 2.0 / (e_max - e_min)
    tau = 0.5 * (e_min + e_max)
    Ht = sigma * (H - tau * S)
    X = s_inv_half(S, sinv)
    Htp = X @ Ht @ X
    if pattern is not None:
        Htp = np.where(pattern, Htp, 0.0)
    lo, hi = e_min, e_max
    for _ in range(max_bisect):
        mu = 0.5 * (lo + hi)
        c = chebyshev_coefficients(lambda x: fermi_erf(x, sigma * (mu - tau), sigma * de), n_pl)
        Kp = kernel_prime(Htp, c, pattern)
        tr = float(np.trace(Kp))
        if abs(tr - n_el) <= tol:
            break
        if tr < n_el:
            lo = mu
        else:
            hi = mu
    K = X @ Kp @ X
    E = float(np.trace(K @ Ht)) / sigma + tau * float(np.trace(K @ S))
    return dict(K=K, Kp=Kp, mu=mu, sigma=sigma, tau=tau, c=c, E_BS=E, bounds=(e_min, e_max), trace=tr)
