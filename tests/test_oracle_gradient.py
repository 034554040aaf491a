"""Pins of the oracle's support-function gradient (Sec. "Gradient and preconditioning",
Eq. gradient) at orthonormal support functions: the gradient is tangent to the
orthonormality constraint (Phi^T g antisymmetric), and it is the derivative of the
band-structure energy Tr(K H) along every tangent direction, the energy taken from the
explicit dense Hamiltonian of oracle/brute.py."""
import numpy as np
import pytest

from oracle import brute as B
from oracle import geometry as G
from oracle import gradient as Gr
from oracle import hamiltonian as Hm
from paper_1401_7441_gb300 import inputs as I
from tests.oracle_support import desc_of, tiny_workload


def _setup(seed=3, n=5, n_atoms=3):
    # every region is the whole box (all functions share one layout) and every point is
    # fine: the compressed vectors are full coefficient vectors of the box
    wl = tiny_workload(n=n, seed=seed, n_atoms=n_atoms, r_loc=100.0, r_fine=100.0, margin=0.0)
    geo = G.build(desc_of(wl))
    V = I.potential(wl)
    Hd = B.full_hamiltonian(n, wl.h, V, wl.V_lo)
    rows = B.region_rows(wl.N, geo.L[0])
    Hc = Hd[np.ix_(rows, rows)]                                   # H in the compressed layout
    rng = np.random.default_rng(seed)
    m = len(rows)
    Phi, _ = np.linalg.qr(rng.standard_normal((m, n_atoms)))     # orthonormal columns
    A = rng.standard_normal((n_atoms, n_atoms))
    K = 0.5 * (A + A.T)
    return wl, geo, V, Hc, Phi, K


def _gradient(wl, geo, V, Phi, K, sinv="exact"):
    n = Phi.shape[1]
    phi = {f: Phi[:, f] for f in range(n)}
    hphi = {f: Hm.apply_hamiltonian(geo, f, phi[f], V, wl.V_lo)[0] for f in range(n)}
    S = Phi.T @ Phi
    g = Gr.energy_gradient(geo, phi, hphi, K, S, sinv)
    return np.stack([g[f] for f in range(n)], axis=1)


def test_gradient_is_tangent_to_the_orthonormality_constraint():
    wl, geo, V, Hc, Phi, K = _setup()
    Gm = _gradient(wl, geo, V, Phi, K)
    X = Phi.T @ Gm
    assert np.max(np.abs(X + X.T)) <= 1e-12 * np.max(np.abs(Gm))
    assert np.max(np.abs(X)) > 1e-6                                 # not trivially zero
    # at S = I the Taylor form of S^-1 is exact
    assert np.max(np.abs(_gradient(wl, geo, V, Phi, K, "taylor") - Gm)) <= 1e-14 * np.max(np.abs(Gm))


@pytest.mark.parametrize("seed", [3, 8])
def test_gradient_is_the_derivative_along_tangent_directions(seed):
    # Omega(Phi) = Tr(K Phi^T H Phi) is quadratic, so the central difference is exact:
    # dOmega = 2 <dPhi, g> for dPhi = (I - Phi Phi^T) R + Phi A, A antisymmetric
    wl, geo, V, Hc, Phi, K = _setup(seed)
    Gm = _gradient(wl, geo, V, Phi, K)
    rng = np.random.default_rng(seed + 100)
    R = rng.standard_normal(Phi.shape)
    Aa = rng.standard_normal((Phi.shape[1],) * 2)
    dPhi = R - Phi @ (Phi.T @ R) + Phi @ (Aa - Aa.T)

    def omega(P):
        return float(np.trace(K @ (P.T @ Hc @ P)))

    t = 1e-3
    fd = (omega(Phi + t * dPhi) - omega(Phi - t * dPhi)) / (2 * t)
    assert abs(fd - 2.0 * float(np.sum(dPhi * Gm))) <= 1e-9 * abs(fd)
