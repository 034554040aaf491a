"""Pins of the oracle's Hamiltonian application and matrices (Sec. II.A, II.B, III.B):
explicit dense matrices, closed forms for Gaussians, identities of the wavelet
transform, and the structural statements of the paper."""
import math

import numpy as np
import pytest

from oracle import brute as B
from oracle import filters as F
from oracle import geometry as G
from oracle import hamiltonian as Hm
from oracle import matrices as Mx
from paper_1401_7441_gb300 import inputs as I
from tests.oracle_support import desc_of, phi_all, tiny_workload

FT = F.load()


@pytest.mark.parametrize("seed,n,r_loc,r_fine", [(5, 6, 1.2, 0.6), (7, 6, 1.5, 0.9), (11, 5, 0.9, 0.5)])
def test_separable_oracle_equals_dense_matrices(seed, n, r_loc, r_fine):
    wl = tiny_workload(n=n, seed=seed, n_atoms=2, r_loc=r_loc, r_fine=r_fine)
    geo = G.build(desc_of(wl))
    V = I.potential(wl)
    Hd = B.full_hamiltonian(n, wl.h, V, wl.V_lo)
    assert np.max(np.abs(Hd - Hd.T)) <= 1e-13 * np.max(np.abs(Hd))
    for f in range(2):
        a = geo.sf_atom[f]
        phi = I.phi_values(wl, f, a, geo.L[a].coarse.g, geo.L[a].fine.g)
        hp, ek, ep = Hm.apply_hamiltonian(geo, f, phi, V, wl.V_lo)
        ref = B.apply_dense(Hd, wl.N, geo.L[a], geo.Lp[a], phi)
        assert np.max(np.abs(hp - ref)) <= 1e-13 * np.max(np.abs(ref))
        # E_kin + E_pot = <phi|H phi> (phi lives on L, inside L')
        full = B.apply_dense(Hd, wl.N, geo.L[a], geo.L[a], phi)
        assert abs((ek + ep) - float(np.dot(phi, full))) <= 1e-13 * abs(ek)


def test_analysis_inverts_synthesis_and_keeps_norm():
    rng = np.random.default_rng(0)
    c = rng.standard_normal((8, 5, 6, 4))
    cf, st = Hm.synthesis3d(c, [3, 2, 7], FT)
    assert abs(np.sum(cf * cf) - np.sum(c * c)) <= 1e-13 * np.sum(c * c)
    back, bst = Hm.analysis3d(cf, st, FT)
    lo = [3 - bst[0], 2 - bst[1], 7 - bst[2]]
    inner = back[:, lo[0]:lo[0] + 5, lo[1]:lo[1] + 6, lo[2]:lo[2] + 4]
    assert np.max(np.abs(inner - c)) < 1e-14
    mask = np.ones(back.shape, bool)
    mask[:, lo[0]:lo[0] + 5, lo[1]:lo[1] + 6, lo[2]:lo[2] + 4] = False
    assert np.max(np.abs(back[mask])) < 1e-14


def _gauss_1d_coeffs(sigma, centre, h, i_lo, n, levels=6):
    """Two-level coefficients (s_i, d_i), i = i_lo..i_lo+n-1, of
    (pi sigma^2)^(-1/4) exp(-(x-c)^2/(2 sigma^2)): magic-filter quadrature at spacing
    h/2^levels, then ``levels`` analysis steps (finer wavelets dropped)."""
    J = levels
    dx = h / 2 ** J
    k_lo = (i_lo - 20) * 2 ** J
    k_hi = (i_lo + n + 20) * 2 ** J
    k = np.arange(k_lo, k_hi + 1)
    lgrid = np.arange(-7, 9)
    x = (k[:, None] + lgrid[None, :]) * dx
    f = (math.pi * sigma * sigma) ** -0.25 * np.exp(-((x - centre) ** 2) / (2 * sigma * sigma))
    c = math.sqrt(dx) * (f @ FT.magic)
    start = k_lo
    for lev in range(J):
        s, i0 = Hm.downsample(c, start, FT.h, -7, 0)
        if lev == J - 1:
            d, _ = Hm.downsample(c, start, FT.g, -7, 0)
        c, start = s, i0
    a = i_lo - start
    return c[a:a + n], d[a:a + n]


def _gauss_3d(sigma, centre, h, lo, n):
    cs = [_gauss_1d_coeffs(sigma, centre[d], h, lo[d], n) for d in range(3)]
    c = np.zeros((8, n, n, n))
    for t in range(8):
        bx, by, bz = t & 1, (t >> 1) & 1, (t >> 2) & 1
        c[t] = np.einsum("i,j,k->ijk", cs[0][bx], cs[1][by], cs[2][bz])
    return c


def test_gaussian_kinetic_energy():
    # normalized Gaussian: <-1/2 nabla^2> = 3 / (4 sigma^2)
    sigma, h = 2.0, 0.45
    n = 46
    centre = [0.37 + 22 * h, 0.11 + 22 * h, 0.29 + 22 * h]
    c = _gauss_3d(sigma, centre, h, [0, 0, 0], n)
    norm = float(np.sum(c * c))
    assert abs(norm - 1.0) < 1e-9
    kin = Hm.kinetic3d(c, h, FT)
    ek = float(np.sum(c * kin[:, 14:14 + n, 14:14 + n, 14:14 + n]))
    assert abs(ek / norm - 3.0 / (4 * sigma * sigma)) < 1e-8 * 3.0 / (4 * sigma * sigma)


def test_gaussian_kinetic_offdiagonal():
    # two same-sigma Gaussians at distance D: T_ab = S_ab (3 - D^2/(2 sigma^2)) / (4 sigma^2),
    # S_ab = exp(-D^2 / (4 sigma^2))
    sigma, h, n = 1.0, 0.45, 34
    ca = [0.21 + 15 * h, 0.13 + 17 * h, 0.3 + 16 * h]
    cb = [ca[0] + 1.1, ca[1] - 0.4, ca[2] + 0.7]
    Dd2 = 1.1 ** 2 + 0.4 ** 2 + 0.7 ** 2
    a = _gauss_3d(sigma, ca, h, [0, 0, 0], n)
    b = _gauss_3d(sigma, cb, h, [0, 0, 0], n)
    S = float(np.sum(a * b))
    kin = Hm.kinetic3d(b, h, FT)
    T = float(np.sum(a * kin[:, 14:14 + n, 14:14 + n, 14:14 + n]))
    S_ref = math.exp(-Dd2 / (4 * sigma ** 2))
    T_ref = S_ref * (3 - Dd2 / (2 * sigma ** 2)) / (4 * sigma ** 2)
    assert abs(S - S_ref) < 1e-9
    assert abs(T - T_ref) < 1e-8


def test_gaussian_potential_closed_form():
    # <f|V|f> with V = -D exp(-|r-c'|^2/(2w^2)) and |f|^2 a Gaussian of variance sigma^2/2:
    # -D (w^2/(w^2+sigma^2/2))^(3/2) exp(-|c-c'|^2 / (2 (w^2 + sigma^2/2)))
    sigma, h, n = 2.0, 0.45, 46
    centre = [0.37 + 22 * h, 0.11 + 22 * h, 0.29 + 22 * h]
    c = _gauss_3d(sigma, centre, h, [0, 0, 0], n)
    cw = [centre[0] + 0.8, centre[1] - 0.5, centre[2] + 0.3]
    Dw, w = 2.0, 1.0
    cf, st = Hm.synthesis3d(c, [0, 0, 0], FT)
    u, ust = Hm.magic3d(cf, st, FT)
    x = [(np.arange(u.shape[d]) + ust[d]) * (h / 2) for d in range(3)]
    V = -Dw * np.einsum("i,j,k->ijk", *[np.exp(-((x[d] - cw[d]) ** 2) / (2 * w * w)) for d in range(3)])
    e = float(np.sum(V * u * u))
    dd2 = 0.8 ** 2 + 0.5 ** 2 + 0.3 ** 2
    ref = -Dw * (w * w / (w * w + sigma ** 2 / 2)) ** 1.5 * math.exp(-dd2 / (2 * (w * w + sigma ** 2 / 2)))
    assert abs(e - ref) <= 1e-8 * abs(ref)


def test_matrices_structure_atoms64_subset():
    wl = I.atoms64()
    geo = G.build(desc_of(wl))
    V = I.potential(wl)
    rows = [0, 17, 100]
    need = set(rows)
    for a in rows:
        need |= set(int(b) for b in geo.col[geo.row_ptr[a]:geo.row_ptr[a + 1]])
    phi = phi_all(wl, geo, sorted(need))
    hphi, ek, ep = {}, {}, {}
    for f in sorted(need):
        hphi[f], ek[f], ep[f] = Hm.apply_hamiltonian(geo, f, phi[f], V, wl.V_lo)
    Hv, Sv = Mx.build_matrices(geo, phi, hphi, rows=rows)
    for a in rows:
        for k in range(geo.row_ptr[a], geo.row_ptr[a + 1]):
            b = int(geo.col[k])
            if b == a:
                assert abs(Sv[k] - 1.0) < 1e-14            # S_aa = |phi_a|^2 = 1
                assert abs(Hv[k] - (ek[a] + ep[a])) < 1e-12 * abs(ek[a])
            # symmetry of S by the other order of the dot product
            assert abs(Sv[k] - Mx.overlap_entry(geo, b, a, phi[b], phi[a])) < 1e-15


def test_hamiltonian_symmetric_with_full_reach_margin():
    # with L' wide enough to hold every point H reaches (15 coarse points per axis,
    # i.e. 15 sqrt(3) < 27 in radius), H_ab = <phi_a|H phi_b> is exactly symmetric
    wl = I.scaled("atoms64", 6, seed=3)
    wl.r_loc[:] = 3.0
    wl.r_fine[:] = 1.0
    wl.lprime_margin = 27.0
    geo = G.build(desc_of(wl))
    V = I.potential(wl)
    fs = range(min(6, len(geo.sf_atom)))
    phi = phi_all(wl, geo, fs)
    hphi = {f: Hm.apply_hamiltonian(geo, f, phi[f], V, wl.V_lo)[0] for f in fs}
    for a in fs:
        for b in fs:
            hab = Mx.hamiltonian_entry(geo, a, b, phi[a], hphi[b])
            hba = Mx.hamiltonian_entry(geo, b, a, phi[b], hphi[a])
            scale = math.sqrt(np.dot(hphi[a], hphi[a]) * np.dot(hphi[b], hphi[b]))
            assert abs(hab - hba) <= 1e-13 * scale


@pytest.mark.parametrize("seed,n,r_loc,r_fine", [(5, 6, 1.2, 0.6), (11, 5, 0.9, 0.5)])
def test_hphi_abs_bound_equals_dense_absolute_matrices(seed, n, r_loc, r_fine):
    # The absolute-term bound of every H phi element (the per-element scale of the GPU
    # parity tests) against explicit dense matrices built entry by entry with absolute
    # taps: |P_L'| (|K|/(2h^2) + |MS|^T |V| |MS|) |P_L| |phi|, kinetic and potential
    # parts kept apart so that neither cancels the other.
    import dataclasses
    wl = tiny_workload(n=n, seed=seed, n_atoms=2, r_loc=r_loc, r_fine=r_fine)
    geo = G.build(desc_of(wl))
    V = I.potential(wl)
    Fa = dataclasses.replace(FT, h=np.abs(FT.h), g=np.abs(FT.g), magic=np.abs(FT.magic),
                             kin={k: np.abs(v) for k, v in FT.kin.items()})
    F0 = dataclasses.replace(Fa, kin={k: np.zeros_like(v) for k, v in FT.kin.items()})
    pot = B.full_hamiltonian(n, wl.h, np.abs(V), wl.V_lo, F0)
    K = B.kinetic_matrix(n, Fa)
    Id = np.eye(2 * n)
    kin = (np.kron(np.kron(K, Id), Id) + np.kron(np.kron(Id, K), Id) + np.kron(np.kron(Id, Id), K)) / (2 * wl.h ** 2)
    for f in range(2):
        a = geo.sf_atom[f]
        phi = I.phi_values(wl, f, a, geo.L[a].coarse.g, geo.L[a].fine.g)
        bound = Hm.hphi_abs_bound(geo, f, phi, V, wl.V_lo)
        ref = B.apply_dense(pot + kin, wl.N, geo.L[a], geo.Lp[a], np.abs(phi))
        assert np.max(np.abs(bound - ref)) <= 1e-13 * np.max(ref)
        hp, _, _ = Hm.apply_hamiltonian(geo, f, phi, V, wl.V_lo)
        assert np.all(np.abs(hp) <= bound * (1 + 1e-12))
        assert np.max(np.abs(hp) / np.maximum(bound, 1e-300)) > 0.3     # not a loose bound
