"""GPU parity of the sparse combination (M Phi)_a = L(a) sum_b M_ab phi_b and of the
first-order Taylor Loewdin step (Sec. "Orthogonalization", Sec. "Gradient and
preconditioning"), through the C ABI, against the oracle (oracle/combine.py).

Every member of every output function is checked against the oracle's absolute-term
bound of that element (the same combination taken with |M| and |phi|), at the
tolerance of the precision, on small systems (every function, several tile edges and
slab budgets) and on sampled rows of the 1,200-atom workload."""
import numpy as np
import pytest

from oracle import combine as Cb
from oracle import geometry as G
from paper_1401_7441_gb300 import inputs as I
from paper_1401_7441_gb300 import lsw
from tests.lib_support import ensure_built, keys_to_g
from tests.oracle_support import desc_of

pytestmark = pytest.mark.gpu

TOL = {lsw.LSW_FP64: 1e-12, lsw.LSW_FP32: 1e-5, lsw.LSW_FP32_BF16X: 1e-5}
FLOOR = {lsw.LSW_FP64: 0.0, lsw.LSW_FP32: 1e-36, lsw.LSW_FP32_BF16X: 1e-36}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()


def _system(wl, prec, options=None):
    import torch
    S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   wl.lprime_margin, 0, prec, device=0, stream=torch.cuda.current_stream().cuda_stream)
    for k, v in (options or {}).items():
        lsw.lsw_set_option(S.sys, k, v)
    return S


def _phi(wl, S, fs=None):
    phi = np.zeros(S.total_L)
    for f in (range(S.n_sf) if fs is None else fs):
        a = int(S.sf_atom[f])
        v = I.phi_values(wl, f, a, keys_to_g(S.keys(a, 0, 0)), keys_to_g(S.keys(a, 0, 1)))
        phi[S.off_L[f]:S.off_L[f] + len(v)] = v
    return phi


def _run(S, prec, phi_h, M_h, op="combine"):
    import torch
    dt = torch.float64 if prec == lsw.LSW_FP64 else torch.float32
    phi = torch.tensor(phi_h, dtype=dt, device="cuda")
    M = torch.tensor(M_h, dtype=torch.float64, device="cuda")
    out = torch.full((S.total_L,), float("nan"), dtype=dt, device="cuda")
    if op == "combine":
        lsw.lsw_combine(S.sys, M, phi, out)
    else:
        lsw.lsw_lowdin_taylor(S.sys, M, phi, out)
    lsw.lsw_sync(S.sys, 120.0)
    return out.double().cpu().numpy(), phi.double().cpu().numpy()


def _check(S, geo, got, M, phi_in, rows, prec):
    phi = {f: phi_in[S.off_L[f]:S.off_L[f + 1]][:geo.L[geo.sf_atom[f]].n_coef] for f in range(S.n_sf)}
    ref = Cb.combine(geo, M, phi, rows)
    bnd = Cb.combine(geo, np.abs(M), {f: np.abs(v) for f, v in phi.items()}, rows)
    worst = 0.0
    for a in rows:
        g = got[S.off_L[a]:S.off_L[a] + len(ref[a])]
        assert np.all(np.isfinite(g)), a                 # every member written
        err = np.abs(g - ref[a])
        bad = err > TOL[prec] * bnd[a] + FLOOR[prec]
        assert not bad.any(), (a, int(bad.sum()), float(np.max(err / np.maximum(bnd[a], 1e-300))))
        worst = max(worst, float(np.max(err / np.maximum(bnd[a], 1e-300))))
    # the alignment gaps between functions are not written
    for a in rows:
        n = len(ref[a])
        assert np.all(np.isnan(got[S.off_L[a] + n:S.off_L[a + 1]]))
    return worst


@pytest.mark.parametrize("prec", [lsw.LSW_FP64, lsw.LSW_FP32, lsw.LSW_FP32_BF16X])
@pytest.mark.parametrize("options", [{}, {"tile": 3}, {"tile": 5, "slab_mb": 1}])
def test_combine_small_system_every_function(prec, options):
    wl = I.scaled("atoms64", 8, seed=5)
    geo = G.build(desc_of(wl))
    S = _system(wl, prec, options)
    try:
        rng = np.random.default_rng(3)
        M = rng.uniform(-1.0, 1.0, len(S.col))           # not symmetric
        got, phi_in = _run(S, prec, _phi(wl, S), M)
        _check(S, geo, got, M, phi_in, range(S.n_sf), prec)
    finally:
        S.close()


@pytest.mark.parametrize("prec", [lsw.LSW_FP64, lsw.LSW_FP32])
def test_lowdin_taylor_step(prec):
    # phi' = L sum_b (3 delta - S)/2 phi_b with S from the library's own H/S build
    import torch
    wl = I.scaled("atoms64", 8, seed=7)
    geo = G.build(desc_of(wl))
    S = _system(wl, prec)
    try:
        dt = torch.float64 if prec == lsw.LSW_FP64 else torch.float32
        phi_h = _phi(wl, S)
        phi = torch.tensor(phi_h, dtype=dt, device="cuda")
        V = torch.tensor(I.potential(wl), dtype=dt, device="cuda")
        lsw.lsw_set_potential(S.sys, V, wl.V_lo, wl.V_shape)
        hphi = torch.zeros(S.total_Lp, dtype=dt, device="cuda")
        lsw.lsw_apply_hamiltonian(S.sys, phi, hphi)
        Hm = torch.zeros(len(S.col), dtype=torch.float64, device="cuda")
        Sm = torch.zeros_like(Hm)
        lsw.lsw_build_matrices(S.sys, phi, hphi, Hm, Sm)
        lsw.lsw_sync(S.sys, 120.0)
        Sv = Sm.cpu().numpy()
        got, phi_in = _run(S, prec, phi_h, Sv, op="lowdin")
        rp, col = S.row_ptr, S.col
        T = np.array([(3.0 * (int(col[k]) == a) - Sv[k]) / 2.0 for a in range(S.n_sf) for k in range(rp[a], rp[a + 1])])
        _check(S, geo, got, T, phi_in, range(S.n_sf), prec)
        # the oracle's own Loewdin step from the same S agrees with the combination form
        phid = {f: phi_in[S.off_L[f]:S.off_L[f] + geo.L[geo.sf_atom[f]].n_coef] for f in range(S.n_sf)}
        ref = Cb.lowdin_taylor(geo, Sv, phid, [0, S.n_sf - 1])
        for a in (0, S.n_sf - 1):
            g = got[S.off_L[a]:S.off_L[a] + len(ref[a])]
            assert np.max(np.abs(g - ref[a])) <= 10 * TOL[prec] * np.max(np.abs(ref[a]))
    finally:
        S.close()


def test_combine_atoms1200_sampled_rows_fp32():
    # the full 1,200-atom workload (radii 5-8 bohr), several slabs; rows checked against
    # the oracle restricted to them (their pattern partners' functions generated)
    wl = I.atoms1200()
    S = _system(wl, lsw.LSW_FP32, {"slab_mb": 256})
    try:
        rows = [0, 1, 2047, 4095]
        need = set(rows)
        for a in rows:
            need |= set(int(b) for b in S.col[S.row_ptr[a]:S.row_ptr[a + 1]])
        atoms = sorted(set(int(S.sf_atom[f]) for f in need))
        geo = G.build(desc_of(wl), atoms=atoms)
        rng = np.random.default_rng(11)
        M = rng.uniform(-1.0, 1.0, len(S.col))
        phi_h = _phi(wl, S)
        got, phi_in = _run(S, lsw.LSW_FP32, phi_h, M)
        phi = {f: phi_in[S.off_L[f]:S.off_L[f] + geo.L[geo.sf_atom[f]].n_coef] for f in sorted(need)}
        ref = Cb.combine(geo, M, phi, rows)
        bnd = Cb.combine(geo, np.abs(M), {f: np.abs(v) for f, v in phi.items()}, rows)
        for a in rows:
            g = got[S.off_L[a]:S.off_L[a] + len(ref[a])]
            assert np.all(np.abs(g - ref[a]) <= 1e-5 * bnd[a] + 1e-36), a
    finally:
        S.close()
