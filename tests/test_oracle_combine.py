"""Pins of the oracle's sparse combination (M Phi)_alpha = P_L(alpha) sum_beta M_ab phi_beta
and of the first-order Taylor Loewdin step (Sec. "Orthogonalization", Sec. "Gradient and
preconditioning"): duality with the overlap scalar products, identities, plain matrix
products on whole-box regions, exact Loewdin with S^-1/2, and the quadratic law of the
Taylor step."""
import numpy as np
import pytest

from oracle import combine as Cb
from oracle import geometry as G
from oracle import matrices as Mx
from tests.oracle_support import desc_of, phi_all, tiny_workload


def _pattern_values(geo, Md):
    rp, col = geo.row_ptr, geo.col
    return np.array([Md[a, col[k]] for a in range(len(rp) - 1) for k in range(rp[a], rp[a + 1])])


@pytest.mark.parametrize("seed,n_atoms,r_loc", [(5, 3, 1.3), (9, 4, 1.1)])
def test_combination_is_the_adjoint_of_the_scalar_products(seed, n_atoms, r_loc):
    # sum_alpha <chi_alpha|(M Phi)_alpha> = sum_ab M_ab <chi_alpha|phi_beta> over L(a) n L(b),
    # the right side by the overlap oracle (member-set intersections), row by row
    wl = tiny_workload(n=7, seed=seed, n_atoms=n_atoms, r_loc=r_loc, r_fine=0.7)
    geo = G.build(desc_of(wl))
    phi = phi_all(wl, geo)
    nsf = len(geo.sf_atom)
    rng = np.random.default_rng(seed)
    M = _pattern_values(geo, rng.uniform(-1, 1, (nsf, nsf)))          # not symmetric
    chi = {a: rng.standard_normal(len(phi[a])) for a in range(nsf)}
    out = Cb.combine(geo, M, phi)
    for a in range(nsf):
        lhs = float(np.dot(chi[a], out[a]))
        rhs = sum(M[k] * Mx.overlap_entry(geo, a, int(geo.col[k]), chi[a], phi[int(geo.col[k])])
                  for k in range(geo.row_ptr[a], geo.row_ptr[a + 1]))
        assert abs(lhs - rhs) <= 1e-13 * (1 + abs(rhs)), a
    # some rows really mix functions of different regions
    assert any(len(phi[a]) != len(phi[b]) for a in range(nsf) for b in range(nsf))


def test_identity_returns_each_function():
    wl = tiny_workload(n=7, seed=5, n_atoms=3, r_loc=1.3, r_fine=0.7)
    geo = G.build(desc_of(wl))
    phi = phi_all(wl, geo)
    nsf = len(geo.sf_atom)
    out = Cb.combine(geo, _pattern_values(geo, np.eye(nsf)), phi)
    for a in range(nsf):
        assert np.array_equal(out[a], phi[a])


def _whole_box(n_atoms, seed, n=5):
    # every locreg is the whole box: the projector is the identity and every function has
    # the same layout, so M Phi is a plain matrix product of coefficient vectors
    return tiny_workload(n=n, seed=seed, n_atoms=n_atoms, r_loc=100.0, r_fine=100.0)


def test_whole_box_regions_give_the_matrix_product():
    wl = _whole_box(3, 2)
    geo = G.build(desc_of(wl))
    phi = phi_all(wl, geo)
    nsf = len(geo.sf_atom)
    Md = np.random.default_rng(3).standard_normal((nsf, nsf))
    out = Cb.combine(geo, _pattern_values(geo, Md), phi)
    P = np.stack([phi[b] for b in range(nsf)])
    ref = Md @ P
    for a in range(nsf):
        assert np.max(np.abs(out[a] - ref[a])) <= 1e-14 * np.max(np.abs(ref))


def _near_orthonormal(geo, eps, seed):
    nsf = len(geo.sf_atom)
    n = geo.L[0].n_coef
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, nsf)))
    Rp = rng.standard_normal((n, nsf)) / np.sqrt(n)       # columns of norm about 1
    return {a: Q[:, a] + eps * Rp[:, a] for a in range(nsf)}


def _overlap(phi, nsf):
    return np.array([[float(np.dot(phi[a], phi[b])) for b in range(nsf)] for a in range(nsf)])


def test_exact_loewdin_orthonormalizes():
    wl = _whole_box(3, 4)
    geo = G.build(desc_of(wl))
    nsf = len(geo.sf_atom)
    phi = _near_orthonormal(geo, 0.05, 1)
    S = _overlap(phi, nsf)
    w, V = np.linalg.eigh(S)
    Sm12 = (V / np.sqrt(w)) @ V.T
    out = Cb.combine(geo, _pattern_values(geo, Sm12), phi)
    assert np.max(np.abs(_overlap(out, nsf) - np.eye(nsf))) <= 1e-13


def test_taylor_loewdin_error_is_second_order():
    # with S = I + E and no truncation, the step T = (3I - S)/2 = I - E/2 gives exactly
    # S' = T S T = I - 3/4 E^2 + 1/4 E^3: second order, and halving the perturbation
    # divides the deviation by about four
    wl = _whole_box(3, 4)
    geo = G.build(desc_of(wl))
    nsf = len(geo.sf_atom)
    dev = []
    for eps in (0.04, 0.02, 0.01):
        phi = _near_orthonormal(geo, eps, 2)
        S = _overlap(phi, nsf)
        E = S - np.eye(nsf)
        out = Cb.lowdin_taylor(geo, _pattern_values(geo, S), phi)
        Sp = _overlap(out, nsf)
        assert np.max(np.abs(Sp - (np.eye(nsf) - 0.75 * E @ E + 0.25 * E @ E @ E))) <= 1e-15
        dev.append(np.max(np.abs(Sp - np.eye(nsf))))
    for k in range(2):
        assert 3.2 <= dev[k] / dev[k + 1] <= 4.8, dev
