"""Pins of the oracle's Fermi operator expansion (Sec. "Density kernel optimization", App.
"Fermi operator expansion"): Chebyshev interpolation and evaluation, the density kernel
against exact generalized diagonalization, the electron count, the band-structure
energy, the second-order error of the Taylor S^-1/2 and idempotency at low smearing."""
import math

import numpy as np
from scipy.linalg import eigh
from scipy.optimize import brentq

from oracle import foe as Fo


def test_chebyshev_interpolation_and_evaluation():
    f = lambda x: np.exp(np.sin(3 * x))          # noqa: E731
    n = 20
    c = Fo.chebyshev_coefficients(f, n)
    nodes = np.cos(math.pi * (np.arange(n + 1) + 0.5) / (n + 1))
    assert np.max(np.abs(Fo.chebyshev_value(c, nodes) - f(nodes))) <= 1e-13
    x = np.linspace(-1, 1, 101)
    cc = np.array(c, dtype=float)
    cc[0] *= 0.5
    assert np.max(np.abs(Fo.chebyshev_value(c, x) - np.polynomial.chebyshev.chebval(x, cc))) <= 1e-13
    # x^3 = (3 T_1 + T_3) / 4
    c3 = Fo.chebyshev_coefficients(lambda x: x ** 3, 5)
    assert np.max(np.abs(c3 - np.array([0, 0.75, 0, 0.25, 0, 0]))) <= 1e-15


def _system(n, eta, seed, gap=False):
    rng = np.random.default_rng(seed)
    if gap:
        ev = np.concatenate([rng.uniform(-2.0, -1.0, n // 2), rng.uniform(1.0, 2.0, n - n // 2)])
        Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
        H = (Q * ev) @ Q.T
    else:
        A = rng.standard_normal((n, n))
        H = 0.5 * (A + A.T)
    E0 = rng.standard_normal((n, n))
    E0 = 0.5 * (E0 + E0.T)
    E0 /= np.max(np.abs(np.linalg.eigvalsh(E0)))
    S = np.eye(n) + eta * E0
    return H, S


def _exact(H, S, n_el, de):
    e, C = eigh(H, S)
    mu = brentq(lambda m: float(np.sum(Fo.fermi_erf(e, m, de))) - n_el, e[0] - 10, e[-1] + 10, xtol=1e-14)
    f = Fo.fermi_erf(e, mu, de)
    return (C * f) @ C.T, float(np.sum(f * e)), mu


def test_kernel_equals_exact_diagonalization():
    H, S = _system(12, 0.08, 3)
    n_el, de = 5.0, 0.3
    r = Fo.foe(H, S, n_el, 400, de, sinv="exact", tol=1e-12)
    K, E, mu = _exact(H, S, n_el, de)
    # the polynomial's own error on [-1, 1] bounds the kernel's (with |S^-1/2|^2 <= 1/0.92)
    c = r["c"]
    x = np.linspace(-1, 1, 4001)
    perr = np.max(np.abs(Fo.chebyshev_value(c, x) - Fo.fermi_erf(x, r["sigma"] * (r["mu"] - r["tau"]), r["sigma"] * de)))
    assert perr < 1e-9
    assert np.max(np.abs(r["K"] - K)) <= 1e-8
    assert abs(r["E_BS"] - E) <= 1e-8 * max(1.0, abs(E))
    assert abs(r["mu"] - mu) <= 1e-8
    assert abs(float(np.trace(r["K"] @ S)) - n_el) <= 1e-9           # Tr(K S) = Tr(K')
    e = eigh(H, S, eigvals_only=True)
    assert r["bounds"] == (e[0], e[-1])


def test_taylor_inverse_square_root_error_is_second_order():
    n_el, de = 4.0, 0.3
    errs = []
    for eta in (0.04, 0.02, 0.01):
        H, S = _system(10, eta, 5)
        K, _, _ = _exact(H, S, n_el, de)
        r = Fo.foe(H, S, n_el, 300, de, sinv="taylor", tol=1e-12)
        errs.append(np.max(np.abs(r["K"] - K)))
    for k in range(2):
        assert 3.0 <= errs[k] / errs[k + 1] <= 5.0, errs


def test_low_smearing_kernel_is_a_projector():
    # spectrum with a gap around 0 and smearing far below it: K' S-orthogonally projects
    # on the occupied states, K' K' = K'
    H, S = _system(12, 0.0, 7, gap=True)
    r = Fo.foe(H, S, 6.0, 300, 0.1, sinv="exact", tol=1e-12)
    Kp = r["Kp"]
    assert np.max(np.abs(Kp @ Kp - Kp)) <= 1e-8
    assert abs(float(np.trace(Kp)) - 6.0) <= 1e-10


def _chain(n, t=1.0, gap=3.0):
    """Tight-binding chain with alternating on-site energies (+-gap/2): a gapped,
    nearsighted Hamiltonian (density matrix decays exponentially with distance)."""
    H = np.diag(np.where(np.arange(n) % 2 == 0, gap / 2, -gap / 2)) - t * (np.eye(n, k=1) + np.eye(n, k=-1))
    return H, np.eye(n)


def test_complete_pattern_equals_the_dense_expansion():
    H, S = _system(10, 0.05, 2)
    full = np.ones((10, 10), bool)
    a = Fo.foe(H, S, 4.0, 120, 0.3, sinv="taylor", tol=1e-12)
    b = Fo.foe(H, S, 4.0, 120, 0.3, sinv="taylor", tol=1e-12, pattern=full)
    assert np.array_equal(a["K"], b["K"])


def test_truncated_kernel_error_decays_with_the_pattern_radius():
    # nearsightedness: cutting the Chebyshev columns to |i - j| <= r loses less as r grows
    n = 40
    H, S = _chain(n)
    ref = Fo.foe(H, S, n / 2, 200, 0.2, sinv="exact", tol=1e-11)["K"]
    errs = []
    for r in (2, 4, 6, 8, 12):
        mask = np.abs(np.subtract.outer(np.arange(n), np.arange(n))) <= r
        K = Fo.foe(H, S, n / 2, 200, 0.2, sinv="exact", tol=1e-11, pattern=mask)["K"]
        errs.append(float(np.max(np.abs(K - ref))))
    assert all(errs[k + 1] < 0.5 * errs[k] for k in range(len(errs) - 1)), errs
    assert errs[-1] < 1e-4 * np.max(np.abs(ref))
