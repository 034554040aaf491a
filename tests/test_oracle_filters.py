"""Pins of the oracle's filter table against what the mathematics fixes (Sec. II.B)."""
import math

import numpy as np
import pytest

from oracle import filters as F

FT = F.load()
H = FT.h
G = FT.g
J = np.arange(-7, 9)


def shifted_dot(a, b, k):
    """sum_j a_j b_{j+k} for filters on the same index range."""
    n = len(a)
    if k >= 0:
        return float(np.dot(a[:n - k], b[k:]))
    return float(np.dot(a[-k:], b[:n + k]))


def test_orthonormal_shifts():
    # sum_j h_j h_{j+2k} = delta_k0, same for g, and h _|_ g at all even shifts
    for k in range(-7, 8):
        assert abs(shifted_dot(H, H, 2 * k) - (k == 0)) < 4e-16
        assert abs(shifted_dot(G, G, 2 * k) - (k == 0)) < 4e-16
        assert abs(shifted_dot(H, G, 2 * k)) < 4e-16


def test_sum_and_vanishing_moments():
    assert abs(H.sum() - math.sqrt(2)) < 4e-16
    assert abs(G.sum()) < 4e-16
    # psi has m = 8 vanishing moments: sum_j j^p g_j = 0, p = 0..7 (scaled by sum |j^p g_j|)
    for p in range(8):
        terms = (J.astype(float) ** p) * G
        assert abs(terms.sum()) <= 1e-13 * np.abs(terms).sum(), p
    # ... and no ninth: the p = 8 moment is far from zero
    terms = (J.astype(float) ** 8) * G
    assert abs(terms.sum()) > 1e-3 * np.abs(terms).sum()


def _integer_values(h):
    """phi(k), k = -7..8: eigenvector of sqrt2 h_{2k-m} for eigenvalue 1, sum = 1."""
    A = np.zeros((16, 16))
    for a, k in enumerate(J):
        for b, m in enumerate(J):
            j = 2 * k - m
            if -7 <= j <= 8:
                A[a, b] = math.sqrt(2) * h[j + 7]
    w, v = np.linalg.eig(A)
    phi = np.real(v[:, np.argmin(abs(w - 1))])
    return phi / phi.sum()


def _cascade(h, levels):
    """phi on the dyadic grid x = m / 2^levels (support [-7, 8])."""
    s = 2 ** levels
    grid = {int(k) * s: v for k, v in zip(J, _integer_values(h))}
    for lev in range(1, levels + 1):
        step = 2 ** (levels - lev)
        for m in range(-7 * s + step, 8 * s, 2 * step):
            acc = 0.0
            for j in range(-7, 9):
                idx = 2 * m - j * s
                if idx in grid:
                    acc += math.sqrt(2) * h[j + 7] * grid[idx]
            grid[m] = acc
    xs = np.array(sorted(grid))
    return xs / s, np.array([grid[x] for x in xs])


def test_moments_exact_low_orders():
    # Poisson summation: sum_k k^p phi(k) = int x^p phi for p < m = 8 (phi^ vanishes
    # to order 8 at 2 pi n, n != 0); phi(k) from the refinement eigenproblem.
    phik = _integer_values(H)
    for p in range(8):
        disc = float(np.sum((J.astype(float) ** p) * phik))
        assert abs(disc - FT.moments[p]) <= 1e-12 * max(1.0, abs(FT.moments[p])), p
    assert FT.moments[0] == 1.0


def test_moments_by_cascade_quadrature():
    x, y = _cascade(H, 10)
    dx = x[1] - x[0]
    for p in range(16):
        q = float(np.sum(x ** p * y) * dx)
        assert abs(q - FT.moments[p]) <= 2e-5 * max(1.0, abs(FT.moments[p])), p


def test_least_asymmetric_by_time_domain_measure():
    # the factor picked by the phase criterion must also minimise, over all 16 real
    # spectral factors, the mirror asymmetry of phi: min_c int (phi(c+x)-phi(c-x))^2
    pytest.importorskip("mpmath")
    cands = F.daubechies_candidates(30)
    scores = []
    for dev, m1, h in cands:
        x, y = _cascade(np.array([float(v) for v in h]), 6)
        best = np.inf
        for c in np.linspace(-2.0, 3.0, 201):
            yr = np.interp(2 * c - x, x, y, left=0.0, right=0.0)
            best = min(best, float(np.sum((y - yr) ** 2) / np.sum(y * y)))
        scores.append((best, float(m1), np.array([float(v) for v in h])))
    best = min(s[0] for s in scores)
    winners = [s for s in scores if s[0] < best + 1e-9]
    assert len(winners) == 2  # a factor and its mirror image
    chosen = [s for s in winners if s[1] <= 0.5][0]
    assert np.allclose(chosen[2], H, atol=1e-15)


def test_table_matches_multiprecision_derivation():
    mp = pytest.importorskip("mpmath")
    tab = F.derive(50)
    disk = F.read_table()
    for name, (lo, vals) in tab.items():
        assert disk[name][0] == lo
        ref = np.array([float(v) for v in vals])
        assert np.array_equal(disk[name][1], ref), name


def _poly_coeffs(q, k):
    """c_k = int x^q phi(x - k) dx = sum_i C(q,i) k^(q-i) M_i (coefficients of x^q)."""
    return sum(math.comb(q, i) * (k.astype(float) ** (q - i)) * FT.moments[i] for i in range(q + 1))


@pytest.mark.parametrize("q", range(16))
def test_magic_filter_reproduces_point_values(q):
    # u_j = sum_k w_{j-k} c_k returns x^q at the grid points for q <= 15: needs both
    # the moment match of w and the vanishing moments of the autocorrelation of phi.
    k = np.arange(-40, 41)
    c = _poly_coeffs(q, k)
    js = np.arange(-20, 21)
    u = np.array([sum(FT.magic[l + 7] * c[(j - l) + 40] for l in range(-7, 9)) for j in js])
    exact = js.astype(float) ** q
    scale = max(1.0, float(np.max(np.abs(exact))))
    assert np.max(np.abs(u - exact)) <= 1e-9 * scale * 10 ** (0.6 * max(0, q - 8))


def test_magic_filter_is_not_trivial():
    assert FT.magic.argmax() == 7 and 0.9 < FT.magic[7] < 1.0


def test_connection_coefficients_basic():
    r = FT.kin_r
    l = np.arange(-14, 15).astype(float)
    assert np.allclose(r, r[::-1], atol=0, rtol=0) or np.max(np.abs(r - r[::-1])) < 1e-15
    assert abs(r.sum()) < 1e-14                # annihilates constants
    assert abs(np.sum(l * l * r) - 2.0) < 1e-13  # d^2/dx^2 x^2 = 2
    assert r[14] < 0                           # <phi|phi''> = -|phi'|^2
    assert np.array_equal(FT.kin["hh"], r) or np.max(np.abs(FT.kin["hh"] - r)) < 1e-15


def test_connection_coefficients_two_scale_relation():
    r = {l: FT.kin_r[l + 14] for l in range(-14, 15)}
    for l in range(-14, 15):
        s = 0.0
        for i in range(16):
            for j in range(16):
                s += H[i] * H[j] * r.get(2 * l + j - i, 0.0)
        assert abs(4 * s - r[l]) < 1e-14


@pytest.mark.parametrize("q", range(8))
def test_kinetic_exact_on_polynomials(q):
    # sum_k r_{k-i} c_k(x^q) = c_i(q (q-1) x^(q-2)) for degree q <= 7 (polynomials in
    # the span of the integer translates of phi)
    k = np.arange(-60, 61)
    c = _poly_coeffs(q, k)
    i = np.arange(-30, 31)
    lhs = np.array([sum(FT.kin_r[l + 14] * c[ii + l + 60] for l in range(-14, 15)) for ii in i])
    rhs = q * (q - 1) * _poly_coeffs(q - 2, i) if q >= 2 else np.zeros(len(i))
    scale = max(1.0, float(np.max(np.abs(c))))
    assert np.max(np.abs(lhs - rhs)) <= 1e-12 * scale


def test_kinetic_by_fourier_integral():
    # independent route: r_l = -(1/2pi) int w^2 |phi^(w)|^2 cos(w l) dw with
    # |phi^(w)|^2 = prod_k |H(w/2^k)|^2 / 2 (infinite product, truncated)
    w = np.linspace(0.0, 80.0 * np.pi, 400001)
    dw = w[1] - w[0]
    prod = np.ones_like(w)
    for k in range(1, 40):
        z = np.exp(-1j * np.outer(w / 2 ** k, J))
        Hw = z @ H
        prod *= np.abs(Hw) ** 2 / 2.0
    for l in range(0, 4):
        f = w ** 2 * prod * np.cos(w * l)
        integral = (np.sum(f) - 0.5 * (f[0] + f[-1])) * dw * 2.0  # even integrand
        assert abs(-integral / (2 * np.pi) - FT.kin_r[l + 14]) < 2e-4 * abs(FT.kin_r[14])


def test_kinetic_operator_negative_semidefinite():
    # <f|d^2|f> <= 0 on any finite set of the 2-level basis: the block matrix
    # [[T_hh, T_hg], [T_gh, T_gg]] restricted to n points is negative semidefinite
    n = 40
    K = np.zeros((2 * n, 2 * n))
    names = "hg"
    for b in range(2):
        for bp in range(2):
            T = FT.kin[names[b] + names[bp]]
            for i in range(n):
                for ip in range(n):
                    if abs(ip - i) <= 14:
                        K[b * n + i, bp * n + ip] = T[ip - i + 14]
    assert np.max(np.abs(K - K.T)) < 1e-14
    ev = np.linalg.eigvalsh(K)
    assert ev.max() < 1e-13
    assert ev.min() < -1.0


def test_kinetic_blocks_two_routes():
    # T_XY(l) = <X_0|d^2|Y_l> must equal the h/2-level Galerkin matrix 4 r sandwiched
    # between the synthesis rows: sum_{k,k'} X_k (4 r_{k'-k}) Y_{k'-2l}
    r = {l: FT.kin_r[l + 14] for l in range(-14, 15)}
    names = {"h": H, "g": G}
    for key, T in FT.kin.items():
        X, Y = names[key[0]], names[key[1]]
        for l in range(-14, 15):
            s = 0.0
            for a in range(-7, 9):
                for b in range(-7, 9):
                    k, kp = a, b + 2 * l
                    s += X[a + 7] * 4.0 * r.get(kp - k, 0.0) * Y[b + 7]
            assert abs(s - T[l + 14]) < 1e-13
