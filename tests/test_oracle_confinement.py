"""Pins of the oracle's quartic confining potential and preconditioning equation (Sec.
"Support function optimization", Eq. precond): identities and quadrature of the moment
overlaps, Gaussian closed forms in 1D and 3D, the 3D assembly against Kronecker
products, and the preconditioning operator against the explicit kinetic matrices."""
import math

import numpy as np
import pytest

from oracle import brute as B
from oracle import confinement as Cf
from oracle import filters as F
from oracle import geometry as G
from oracle import matrices as Mx
from tests.oracle_support import desc_of, phi_all, tiny_workload
from tests.test_oracle_filters import _cascade
from tests.test_oracle_operator import _gauss_1d_coeffs, _gauss_3d

FT = F.load()
LS = np.arange(-14, 15)


def test_moment_overlaps_identities():
    # F^0(l) = delta_l0 (orthonormal translates); sum_l F^p(l) = M_p (the translates sum to
    # one); F^p(-l) = sum_q C(p,q) (-l)^(p-q) F^q(l) (substitution x -> x + l)
    assert np.array_equal(FT.movl[0], (LS == 0).astype(float))
    for p in range(5):
        assert abs(FT.movl[p].sum() - FT.moments[p]) <= 1e-14 * max(1.0, abs(FT.moments[p])), p
        for l in LS:
            lhs = FT.movl[p][-l + 14]
            rhs = sum(math.comb(p, q) * float(-l) ** (p - q) * FT.movl[q][l + 14] for q in range(p + 1))
            assert abs(lhs - rhs) <= 1e-12 * max(1.0, float(np.max(np.abs(FT.movl[p])))) * (1 + abs(l)) ** p, (p, l)


def test_moment_overlaps_by_cascade_quadrature():
    x, y = _cascade(FT.h, 10)
    dx = x[1] - x[0]
    s = 2 ** 10
    for p in range(5):
        for l in LS:
            yl = np.zeros_like(y)                                  # phi(x - l) on the same grid
            if l >= 0:
                yl[l * s:] = y[:len(y) - l * s]
            else:
                yl[:len(y) + l * s] = y[-l * s:]
            q = float(np.sum(x ** p * y * yl) * dx)
            assert abs(q - FT.movl[p][l + 14]) <= 3e-5 * max(1.0, abs(FT.movl[p][l + 14])), (p, l)


def test_quartic_blocks_by_cascade_quadrature():
    # <chi^b(. - i)|(x - c)^m|chi^b'(. - j)> at unit spacing by sums over the dyadic grid
    # 2^-10 of phi from the refinement eigenproblem and psi = sqrt2 sum_k g_k phi(2x - k):
    # every type pair, including the scaling <-> wavelet blocks
    s = 2 ** 10
    x, y = _cascade(FT.h, 10)
    m0 = int(round(x[0] * s))
    span = np.arange(-30 * s, 31 * s)
    phi = np.zeros(len(span))
    phi[m0 + 30 * s:m0 + 30 * s + len(y)] = y

    def at(idx):                       # phi at grid indices idx (0 outside the support)
        k = idx + 30 * s
        ok = (k >= 0) & (k < len(phi))
        return np.where(ok, phi[np.clip(k, 0, len(phi) - 1)], 0.0)

    grid = np.arange(-12 * s, 13 * s)
    psi = sum(math.sqrt(2) * gk * at(2 * grid - k * s) for k, gk in zip(range(-7, 9), FT.g))
    chi = {0: at(grid), 1: psi}

    def shifted(b, i):
        out = np.zeros(len(grid))
        if i >= 0:
            out[i * s:] = chi[b][:len(grid) - i * s]
        else:
            out[:len(grid) + i * s] = chi[b][-i * s:]
        return out

    c = 1.3
    idx = np.arange(-2, 3)
    xx = grid / s
    for m in (1, 2, 4):
        for b in (0, 1):
            for bp in (0, 1):
                Bq = np.array([[float(np.sum(shifted(b, i) * (xx - c) ** m * shifted(bp, j))) / s for j in idx]
                               for i in idx])
                Bo = Cf.quartic_block_1d(m, b, bp, idx, idx, c, 1.0, FT)
                assert np.max(np.abs(Bq - Bo)) <= 1e-12 * np.max(np.abs(Bo)), (m, b, bp)


@pytest.mark.parametrize("m", [1, 2, 3, 4])
def test_quartic_block_gaussian_moments_1d(m):
    # <f|(x - R)^m|f> for f^2 normal with variance s = sigma^2/2 centred at c:
    # E[(x - R)^m] with d = c - R
    sigma, h, n = 2.0, 0.45, 46
    cx = 0.37 + 22 * h
    s_, d_ = _gauss_1d_coeffs(sigma, cx, h, 0, n)
    R = cx + 0.7
    idx = np.arange(n)
    e = 0.0
    for b, cb in ((0, s_), (1, d_)):
        for bp, cbp in ((0, s_), (1, d_)):
            e += cb @ Cf.quartic_block_1d(m, b, bp, idx, idx, R / h, h, FT) @ cbp
    s, d = sigma ** 2 / 2, cx - R
    ref = {1: d, 2: s + d * d, 3: 3 * s * d + d ** 3, 4: 3 * s * s + 6 * s * d * d + d ** 4}[m]
    assert abs(e - ref) <= 1e-9 * max(1.0, abs(ref))


def test_confinement_gaussian_closed_form_3d():
    # <f|a|r - R|^4|f> = a (15 s^2 + 10 s |d|^2 + |d|^4), s = sigma^2/2, d = c - R
    sigma, h, n = 2.0, 0.45, 46
    centre = [0.37 + 22 * h, 0.11 + 22 * h, 0.29 + 22 * h]
    c = _gauss_3d(sigma, centre, h, [0, 0, 0], n)
    R = [centre[0] + 0.8, centre[1] - 0.5, centre[2] + 0.3]
    q, qlo = Cf.confine3d(c, [0, 0, 0], R, 0.7, h, FT)
    assert qlo == [-14, -14, -14]
    e = float(np.sum(c * q[:, 14:14 + n, 14:14 + n, 14:14 + n]))
    s, dd = sigma ** 2 / 2, 0.8 ** 2 + 0.5 ** 2 + 0.3 ** 2
    ref = 0.7 * (15 * s * s + 10 * s * dd + dd * dd)
    assert abs(e - ref) <= 1e-9 * ref


def _dense_quartic(N, R, h):
    """Q over every (b1 i1, b2 i2, b3 i3) of an N^3 box from Kronecker products of the
    1D blocks (layout of oracle/brute.py: row (b m + i) per dimension)."""
    idx = np.arange(N)
    mats = {}
    for d in range(3):
        for m in (2, 4):
            M = np.zeros((2 * N, 2 * N))
            for b in (0, 1):
                for bp in (0, 1):
                    M[b * N:(b + 1) * N, bp * N:(bp + 1) * N] = Cf.quartic_block_1d(m, b, bp, idx, idx, R[d] / h, h, FT)
            mats[d, m] = M
    Id = np.eye(2 * N)

    def kron3(A0, A1, A2):
        return np.kron(np.kron(A0, A1), A2)

    Q = kron3(mats[0, 4], Id, Id) + kron3(Id, mats[1, 4], Id) + kron3(Id, Id, mats[2, 4])
    Q += 2 * (kron3(mats[0, 2], mats[1, 2], Id) + kron3(mats[0, 2], Id, mats[2, 2]) + kron3(Id, mats[1, 2], mats[2, 2]))
    return Q


def test_confinement_assembly_against_kronecker_products():
    N, h = 5, 0.45
    R = [1.1, 0.7, 1.6]
    Q = _dense_quartic(N, R, h)
    assert np.max(np.abs(Q - Q.T)) <= 1e-13 * np.max(np.abs(Q))
    assert np.linalg.eigvalsh(Q).min() >= -1e-12 * np.max(np.abs(Q))   # (r - R)^4 >= 0
    rng = np.random.default_rng(4)
    c = rng.standard_normal((8, N, N, N))
    q, _ = Cf.confine3d(c, [0, 0, 0], R, 1.0, h, FT)
    # dense vector in brute.py's layout: index ((b1 N + i1) 2N + (b2 N + i2)) 2N + (b3 N + i3)
    v = np.zeros((2 * N,) * 3)
    out = np.zeros((2 * N,) * 3)
    for t in range(8):
        b1, b2, b3 = t & 1, (t >> 1) & 1, (t >> 2) & 1
        v[b1 * N:(b1 + 1) * N, b2 * N:(b2 + 1) * N, b3 * N:(b3 + 1) * N] = c[t]
        out[b1 * N:(b1 + 1) * N, b2 * N:(b2 + 1) * N, b3 * N:(b3 + 1) * N] = q[t, 14:14 + N, 14:14 + N, 14:14 + N]
    ref = (Q @ v.reshape(-1)).reshape(out.shape)
    assert np.max(np.abs(out - ref)) <= 1e-12 * np.max(np.abs(ref))


def _dense_operator(geo, f, a, eps):
    L = geo.L[geo.sf_atom[f]]
    n = L.n_coef
    A = np.zeros((n, n))
    for k in range(n):
        e = np.zeros(n)
        e[k] = 1.0
        A[:, k] = Cf.precond_operator(geo, f, e, a, eps, FT)
    return A


def test_precond_operator_against_explicit_matrices():
    # A = P_L (T + Q - eps) P_L: its kinetic part against oracle/brute.py's kinetic matrix
    # (Kronecker sum of the 1D Galerkin blocks), its confinement against the Kronecker
    # products of the quartic blocks, restricted to the members of L
    wl = tiny_workload(n=6, seed=5, n_atoms=1, r_loc=1.2, r_fine=0.6)
    geo = G.build(desc_of(wl))
    N, h = 6, wl.h
    rows = B.region_rows(wl.N, geo.L[0])
    K = B.kinetic_matrix(N, FT)
    Id = np.eye(2 * N)
    Kt = -(np.kron(np.kron(K, Id), Id) + np.kron(np.kron(Id, K), Id) + np.kron(np.kron(Id, Id), K)) / (2 * h * h)
    Q = _dense_quartic(N, wl.pos[0], h)
    a, eps = 0.3, -0.5
    A = _dense_operator(geo, 0, a, eps)
    ref = Kt[np.ix_(rows, rows)] + a * Q[np.ix_(rows, rows)] - eps * np.eye(len(rows))
    assert np.max(np.abs(A - ref)) <= 1e-12 * np.max(np.abs(ref))
    assert np.linalg.eigvalsh(0.5 * (A + A.T)).min() > 0                   # eps < 0: positive definite


def test_conjugate_gradients_converge_to_the_solution():
    wl = tiny_workload(n=6, seed=7, n_atoms=1, r_loc=1.3, r_fine=0.7)
    geo = G.build(desc_of(wl))
    g = phi_all(wl, geo)[0]
    a, eps = 0.2, -0.4
    A = _dense_operator(geo, 0, a, eps)
    x_ref = np.linalg.solve(A, -g)
    errs = []
    for it in (1, 2, 4, 8, 16):
        x, res = Cf.precondition(geo, 0, g, a, eps, it, FT)
        e = x - x_ref
        errs.append(float(e @ A @ e))
    assert all(errs[k + 1] <= errs[k] * (1 + 1e-12) for k in range(len(errs) - 1))   # A-norm error falls
    x, res = Cf.precondition(geo, 0, g, a, eps, 90, FT)
    assert np.linalg.norm(x - x_ref) <= 1e-8 * np.linalg.norm(x_ref)
    assert res[-1] <= 1e-10 * np.linalg.norm(g)


def test_confined_energy_of_a_support_function():
    # <phi|Q phi> from the compressed action on L' equals the block energy, and is positive
    wl = tiny_workload(n=7, seed=21, n_atoms=2, r_loc=1.3, r_fine=0.7, margin=40.0)
    geo = G.build(desc_of(wl))
    phi = phi_all(wl, geo)
    for f in range(len(geo.sf_atom)):
        qphi, e = Cf.confinement_energy_and_action(geo, f, phi[f], 0.5, FT)
        A = geo.sf_atom[f]
        dot = Mx._dot(geo.L[A], phi[f], geo.Lp[A], qphi)
        assert abs(dot - e) <= 1e-12 * abs(e)
        assert e > 0
