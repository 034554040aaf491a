"""Pins of the oracle's density rho_j = sum_ab K_ab u_a(j) u_b(j) (Sec. II.A, Eq. density):
closed forms for Gaussians, explicit dense matrices on tiny boxes, the trace identity
with the potential matrix of the Hamiltonian, and positivity for a positive kernel."""
import math

import numpy as np
import pytest

from oracle import brute as B
from oracle import density as Dn
from oracle import filters as F
from oracle import geometry as G
from oracle import hamiltonian as Hm
from oracle import matrices as Mx
from paper_1401_7441_gb300 import inputs as I
from tests.oracle_support import desc_of, phi_all, tiny_workload
from tests.test_oracle_operator import _gauss_3d

FT = F.load()


def _gauss_values(sigma, c, h, lo, dims):
    """(pi sigma^2)^(-3/4) exp(-|x - c|^2 / (2 sigma^2)) at x_j = j h/2, array [z, y, x]."""
    x = [(np.arange(dims[d]) + lo[d]) * (h / 2) for d in range(3)]
    e = [np.exp(-((x[d] - c[d]) ** 2) / (2 * sigma * sigma)) for d in range(3)]
    return (math.pi * sigma * sigma) ** -0.75 * np.einsum("i,j,k->kji", *e)


def test_density_of_two_gaussians_closed_form():
    # two normalized Gaussians on different coarse blocks: rho(x_j) = (h/2)^-3 rho_j must be
    # sum_ab K_ab g_a(x_j) g_b(x_j) at every point, and sum_j rho_j = sum_ab K_ab S_ab with
    # S_ab = exp(-D^2 / (4 sigma^2))
    sigma, h, n = 2.0, 0.45, 46
    ca = [0.37 + 22 * h, 0.11 + 22 * h, 0.29 + 22 * h]
    cb = [ca[0] + 1.3, ca[1] - 0.9, ca[2] + 0.6]
    lob = [2, 1, 3]
    fa = Dn.realspace_block(_gauss_3d(sigma, ca, h, [0, 0, 0], n), [0, 0, 0], FT)
    fb = Dn.realspace_block(_gauss_3d(sigma, cb, h, lob, n), lob, FT)
    K = {(0, 0): 0.8, (0, 1): 0.3, (1, 0): 0.25, (1, 1): 1.1}
    glo, gd = [-20, -20, -20], [140, 140, 140]
    rho = Dn.accumulate({0: fa, 1: fb}, [(a, b, k) for (a, b), k in K.items()], glo, gd)
    ga = _gauss_values(sigma, ca, h, glo, gd)
    gb = _gauss_values(sigma, cb, h, glo, gd)
    ref = K[0, 0] * ga * ga + (K[0, 1] + K[1, 0]) * ga * gb + K[1, 1] * gb * gb
    assert np.max(np.abs(rho / (h / 2) ** 3 - ref)) <= 1e-8 * np.max(ref)
    S_ab = math.exp(-(1.3 ** 2 + 0.9 ** 2 + 0.6 ** 2) / (4 * sigma * sigma))
    assert abs(rho.sum() - (K[0, 0] + K[1, 1] + (K[0, 1] + K[1, 0]) * S_ab)) <= 1e-8


def _dense_realspace(N, F_, loc, phi):
    """u = (A x A x A) P_L phi with A = M S built entry by entry (oracle/brute.py)."""
    S, k_lo = B.synthesis_matrix(N, F_)
    M, j_lo = B.magic_matrix(k_lo, S.shape[0], F_)
    A = M @ S
    n = 2 * N
    v = np.zeros(n ** 3)
    v[B.region_rows((N, N, N), loc)] = phi
    u = np.einsum("pa,qb,rc,abc->pqr", A, A, A, v.reshape(n, n, n), optimize=True)
    return u, j_lo


@pytest.mark.parametrize("seed,n,r_loc,r_fine", [(5, 6, 1.2, 0.6), (13, 5, 1.0, 0.7)])
def test_density_equals_dense_matrices(seed, n, r_loc, r_fine):
    wl = tiny_workload(n=n, seed=seed, n_atoms=3, r_loc=r_loc, r_fine=r_fine)
    geo = G.build(desc_of(wl))
    phi = phi_all(wl, geo)
    nsf = len(geo.sf_atom)
    rng = np.random.default_rng(seed)
    Kd = rng.uniform(-1.0, 1.0, (nsf, nsf))                # not symmetric on purpose
    K = np.array([Kd[a, geo.col[k]] for a in range(nsf) for k in range(geo.row_ptr[a], geo.row_ptr[a + 1])])
    us = {}
    for f in range(nsf):
        us[f], j_lo = _dense_realspace(n, FT, geo.L[geo.sf_atom[f]], phi[f])
    nj = us[0].shape[0]
    ref = np.zeros((nj, nj, nj))
    for a in range(nsf):
        for k in range(geo.row_ptr[a], geo.row_ptr[a + 1]):
            ref += K[k] * us[a] * us[int(geo.col[k])]
    rho = Dn.density(geo, phi, K, [j_lo] * 3, [nj] * 3)
    assert np.max(np.abs(rho - ref.transpose(2, 1, 0))) <= 1e-14 * np.max(np.abs(ref))


def test_density_trace_identity_with_potential_matrix():
    # sum_j V_j rho_j = sum_ab K_ab <phi_a | W^T M^T V M W phi_b>: the potential part of the
    # Hamiltonian (magic transpose, analysis, compress on L') against point products
    # (L' spans the whole box here, so nothing is truncated)
    wl = tiny_workload(n=7, seed=21, n_atoms=3, r_loc=1.3, r_fine=0.7, margin=40.0)
    geo = G.build(desc_of(wl))
    phi = phi_all(wl, geo)
    V = I.potential(wl)
    nsf = len(geo.sf_atom)
    K = I.density_kernel(wl, geo.sf_atom, geo.row_ptr, geo.col)
    pot = {b: Hm.apply_hamiltonian(geo, b, phi[b], V, wl.V_lo, parts=True)[0] for b in range(nsf)}
    lhs = 0.0
    for a in range(nsf):
        for k in range(geo.row_ptr[a], geo.row_ptr[a + 1]):
            b = int(geo.col[k])
            lhs += K[k] * Mx._dot(geo.L[geo.sf_atom[a]], phi[a], geo.Lp[geo.sf_atom[b]], pot[b])
    rho = Dn.density(geo, phi, K, wl.V_lo, wl.V_shape)
    rhs = float(np.sum(V * rho))
    scale = float(np.sum(np.abs(V) * Dn.density(geo, phi, K, wl.V_lo, wl.V_shape, absolute=True)))
    assert abs(lhs - rhs) <= 1e-13 * scale
    assert abs(lhs) > 1e-3 * scale                            # the identity is not vacuous


def test_density_positive_kernel_gives_nonnegative_density():
    # K = C C^T (occupations f_i >= 0 folded into C): rho_j = sum_i (sum_a C_ai u_a(j))^2 >= 0
    wl = tiny_workload(n=7, seed=3, n_atoms=4, r_loc=1.3, r_fine=0.7)
    geo = G.build(desc_of(wl))
    phi = phi_all(wl, geo)
    nsf = len(geo.sf_atom)
    assert len(geo.col) == nsf * nsf                         # complete pattern
    C = np.random.default_rng(1).standard_normal((nsf, 2))
    Kd = C @ C.T
    K = np.array([Kd[a, geo.col[k]] for a in range(nsf) for k in range(geo.row_ptr[a], geo.row_ptr[a + 1])])
    rho = Dn.density(geo, phi, K, wl.V_lo, wl.V_shape)
    rho_abs = Dn.density(geo, phi, K, wl.V_lo, wl.V_shape, absolute=True)
    assert rho.min() >= -1e-15 * rho_abs.max()
    assert np.all(np.abs(rho) <= rho_abs * (1 + 1e-14) + 1e-300)
    assert rho.max() > 1e-6 * rho_abs.max()


def test_density_points_equal_the_grid_values():
    # the point-sampled form used at sizes where the whole grid is out of reach
    wl = tiny_workload(n=7, seed=21, n_atoms=3, r_loc=1.3, r_fine=0.7)
    geo = G.build(desc_of(wl))
    phi = phi_all(wl, geo)
    K = I.density_kernel(wl, geo.sf_atom, geo.row_ptr, geo.col)
    rho = Dn.density(geo, phi, K, wl.V_lo, wl.V_shape)
    rng = np.random.default_rng(2)
    pts = np.stack([rng.integers(wl.V_lo[d], wl.V_lo[d] + wl.V_shape[d], 40) for d in range(3)], axis=1)
    pts[0] = np.unravel_index(np.argmax(rho), rho.shape)[::-1] + np.asarray(wl.V_lo)
    got = Dn.density_points(geo, phi, K, pts)
    ref = rho[pts[:, 2] - wl.V_lo[2], pts[:, 1] - wl.V_lo[1], pts[:, 0] - wl.V_lo[0]]
    assert np.max(np.abs(got - ref)) <= 1e-14 * np.max(np.abs(rho))
    assert got[0] == pytest.approx(rho.max(), rel=1e-13)
