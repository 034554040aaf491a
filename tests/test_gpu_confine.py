"""GPU parity of the quartic confinement and the preconditioning solve (Sec. "Support
function optimization", Eq. precond) through the C ABI against the oracle
(oracle/confinement.py).

* a Q phi on L' and <phi|a Q|phi>: every element against the oracle's value, at the
  precision's tolerance of the largest element of the function (FP64 1e-12, FP32 1e-5);
* the conjugate-gradient solve: after k iterations the iterate and the residual norms
  against the oracle's own CG.  CG iterates are not backward stable as a sequence, so the
  tolerance grows with the iterations: FP64 1e-10 after 6 iterations (relative, 2-norm),
  FP32 2e-4 after 3 (the condition number of A, about 100 here, times FP32 rounding
  times the iterations).
"""
import numpy as np
import pytest

from oracle import confinement as Q
from oracle import geometry as G
from paper_1401_7441_gb300 import inputs as I
from paper_1401_7441_gb300 import lsw
from tests.lib_support import ensure_built, keys_to_g
from tests.oracle_support import desc_of

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()


def _setup(prec, n_atoms=6, seed=5):
    import torch
    wl = I.scaled("atoms64", n_atoms, seed=seed)
    S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   wl.lprime_margin, 0, prec, device=0, stream=torch.cuda.current_stream().cuda_stream)
    phi = np.zeros(S.total_L)
    for f in range(S.n_sf):
        a = int(S.sf_atom[f])
        v = I.phi_values(wl, f, a, keys_to_g(S.keys(a, 0, 0)), keys_to_g(S.keys(a, 0, 1)))
        phi[S.off_L[f]:S.off_L[f] + len(v)] = v
    geo = G.build(desc_of(wl))
    return wl, S, geo, phi


@pytest.mark.parametrize("prec", [lsw.LSW_FP64, lsw.LSW_FP32])
def test_confinement_action_and_energy(prec):
    import torch
    wl, S, geo, phi_h = _setup(prec)
    try:
        dt = torch.float64 if prec == lsw.LSW_FP64 else torch.float32
        tol = 1e-12 if prec == lsw.LSW_FP64 else 1e-5
        rng = np.random.default_rng(4)
        a_h = rng.uniform(0.001, 0.01, S.n_sf)
        phi = torch.tensor(phi_h, dtype=dt, device="cuda")
        hphi = torch.full((S.total_Lp,), 0.0, dtype=dt, device="cuda")
        e = torch.zeros(S.n_sf, dtype=torch.float64, device="cuda")
        a = torch.tensor(a_h, device="cuda")
        lsw.lsw_add_confinement(S.sys, a, phi, hphi, e)
        lsw.lsw_sync(S.sys, 120.0)
        got = hphi.double().cpu().numpy()
        eg = e.cpu().numpy()
        pin = phi.double().cpu().numpy()
        for f in range(S.n_sf):
            L = geo.L[geo.sf_atom[f]]
            pf = pin[S.off_L[f]:S.off_L[f] + L.n_coef]
            ref, e_ref = Q.confinement_energy_and_action(geo, f, pf, a_h[f])
            g = got[S.off_Lp[f]:S.off_Lp[f] + len(ref)]
            assert np.max(np.abs(g - ref)) <= tol * np.max(np.abs(ref)), f
            assert abs(eg[f] - e_ref) <= tol * abs(e_ref), (f, eg[f], e_ref)
        # adding to an existing H phi: the two calls add up
        lsw.lsw_add_confinement(S.sys, a, phi, hphi, e)
        lsw.lsw_sync(S.sys, 120.0)
        assert np.allclose(hphi.double().cpu().numpy(), 2 * got, rtol=0, atol=tol * 4 * np.max(np.abs(got)))
    finally:
        S.close()


@pytest.mark.parametrize("prec,iters,tol", [(lsw.LSW_FP64, 6, 1e-10), (lsw.LSW_FP32, 3, 2e-4)])
def test_precondition_cg_matches_oracle(prec, iters, tol):
    import torch
    wl, S, geo, phi_h = _setup(prec, n_atoms=4, seed=9)
    try:
        dt = torch.float64 if prec == lsw.LSW_FP64 else torch.float32
        rng = np.random.default_rng(8)
        a_h = rng.uniform(0.001, 0.01, S.n_sf)
        eps_h = -rng.uniform(0.3, 1.0, S.n_sf)
        g = torch.tensor(phi_h, dtype=dt, device="cuda")          # a smooth right-hand side
        gp = torch.full((S.total_L,), float("nan"), dtype=dt, device="cuda")
        res = torch.zeros((iters, S.n_sf), dtype=torch.float64, device="cuda")
        lsw.lsw_precondition(S.sys, torch.tensor(a_h, device="cuda"), torch.tensor(eps_h, device="cuda"), g, gp, iters, res)
        lsw.lsw_sync(S.sys, 120.0)
        got = gp.double().cpu().numpy()
        rs = res.cpu().numpy()
        gin = g.double().cpu().numpy()
        for f in range(S.n_sf):
            L = geo.L[geo.sf_atom[f]]
            gf = gin[S.off_L[f]:S.off_L[f] + L.n_coef]
            x, r = Q.precondition(geo, f, gf, a_h[f], eps_h[f], iters)
            xg = got[S.off_L[f]:S.off_L[f] + L.n_coef]
            assert np.linalg.norm(xg - x) <= tol * np.linalg.norm(x), f
            assert np.allclose(rs[:len(r), f], r, rtol=10 * tol, atol=0), (f, rs[:, f], r)
            assert r[-1] < r[0]                                     # the residual falls
            assert np.all(np.isnan(got[S.off_L[f] + L.n_coef:S.off_L[f + 1]]))   # gaps untouched
    finally:
        S.close()
