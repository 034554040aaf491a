"""GPU parity of the Fermi operator expansion (App. "Fermi operator expansion") through
the C ABI against the oracle (oracle/foe.py, sparse form on the kernel's pattern).

H and S come from the library's own H/S build of a seeded workload (symmetrized: the
expansion is defined for the symmetric pair), the spectrum bounds from the oracle's
generalized eigensolver, and both sides run the same expansion: Taylor S^-1/2,
Chebyshev columns cut to the pattern after every product, bisection on mu.  Tolerance:
the recursion's rounding grows with the number of terms and the row length, so K' and K
are compared at 1e-11 of their largest entry (FP64), mu and the trace exactly up to the
bisection's own tolerance."""
import numpy as np
import pytest

from oracle import foe as F
from paper_1401_7441_gb300 import inputs as I
from paper_1401_7441_gb300 import lsw
from tests.lib_support import ensure_built, keys_to_g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()


def _hs(wl):
    """The system, and symmetrized H, S on its pattern from the library."""
    import torch
    S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   wl.lprime_margin, 0, lsw.LSW_FP64, device=0, stream=torch.cuda.current_stream().cuda_stream)
    phi_h = np.zeros(S.total_L)
    for f in range(S.n_sf):
        a = int(S.sf_atom[f])
        v = I.phi_values(wl, f, a, keys_to_g(S.keys(a, 0, 0)), keys_to_g(S.keys(a, 0, 1)))
        phi_h[S.off_L[f]:S.off_L[f] + len(v)] = v
    phi = torch.tensor(phi_h, device="cuda")
    V = torch.tensor(I.potential(wl), device="cuda")
    lsw.lsw_set_potential(S.sys, V, wl.V_lo, wl.V_shape)
    hphi = torch.zeros(S.total_Lp, dtype=torch.float64, device="cuda")
    lsw.lsw_apply_hamiltonian(S.sys, phi, hphi)
    Hm = torch.zeros(len(S.col), dtype=torch.float64, device="cuda")
    Sm = torch.zeros_like(Hm)
    lsw.lsw_build_matrices(S.sys, phi, hphi, Hm, Sm)
    lsw.lsw_sync(S.sys, 120.0)
    n = S.n_sf
    rows = np.repeat(np.arange(n), np.diff(S.row_ptr))
    Hd = np.zeros((n, n))
    Sd = np.zeros((n, n))
    Hd[rows, S.col] = Hm.cpu().numpy()
    Sd[rows, S.col] = Sm.cpu().numpy()
    Hd = 0.5 * (Hd + Hd.T)
    Sd = 0.5 * (Sd + Sd.T)
    mask = np.zeros((n, n), bool)
    mask[rows, S.col] = True
    return S, Hd, Sd, mask, rows


@pytest.mark.parametrize("n_pl,de", [(30, 0.1), (60, 0.05)])
def test_foe_matches_oracle_on_the_pattern(n_pl, de):
    import torch
    wl = I.scaled("atoms64", 24, seed=21)
    S, Hd, Sd, mask, rows = _hs(wl)
    try:
        n = S.n_sf
        bounds = F.spectrum_bounds(Hd, Sd)
        n_el = float(n // 2)
        ref = F.foe(Hd, Sd, n_el, n_pl, de, sinv="taylor", bounds=bounds, pattern=mask)
        Hv = torch.tensor(Hd[rows, S.col], device="cuda")
        Sv = torch.tensor(Sd[rows, S.col], device="cuda")
        Kp = torch.zeros(len(S.col), dtype=torch.float64, device="cuda")
        K = torch.zeros_like(Kp)
        mu, ebs, tr = lsw.lsw_foe(S.sys, Hv, Sv, bounds[0], bounds[1], n_el, n_pl, de, Kp, K)
        assert mu == pytest.approx(ref["mu"], abs=1e-12 * (bounds[1] - bounds[0]))
        assert abs(tr - ref["trace"]) <= 1e-9
        kp_ref = ref["Kp"][rows, S.col]
        k_ref = ref["K"][rows, S.col]
        assert np.max(np.abs(Kp.cpu().numpy() - kp_ref)) <= 1e-11 * np.max(np.abs(kp_ref))
        assert np.max(np.abs(K.cpu().numpy() - k_ref)) <= 1e-11 * np.max(np.abs(k_ref))
        # E_BS from the kernel on the pattern equals the oracle's trace form
        assert ebs == pytest.approx(ref["E_BS"], rel=1e-11, abs=1e-11)
        # the expansion is nontrivial: partly occupied, K' off-diagonal entries present
        assert 0.05 < np.max(np.abs(kp_ref[rows != S.col])) or np.max(np.abs(kp_ref)) > 0.05
    finally:
        S.close()


def test_foe_argument_errors():
    import torch
    wl = I.scaled("atoms64", 4, seed=3)
    S, Hd, Sd, mask, rows = _hs(wl)
    try:
        Hv = torch.tensor(Hd[rows, S.col], device="cuda")
        Sv = torch.tensor(Sd[rows, S.col], device="cuda")
        Kp = torch.zeros(len(S.col), dtype=torch.float64, device="cuda")
        with pytest.raises(lsw.LswError) as e:
            lsw.lsw_foe(S.sys, Hv, Sv, 1.0, 1.0, 1.0, 10, 0.1, Kp, Kp.clone())
        assert e.value.status == lsw.LSW_ERR_ARG
        with pytest.raises(lsw.LswError):
            lsw.lsw_foe(S.sys, Hv, Sv, -1.0, 1.0, 1.0, 0, 0.1, Kp, Kp.clone())
    finally:
        S.close()
