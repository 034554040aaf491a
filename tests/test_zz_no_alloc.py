"""GPU test of lsw_apply_hamiltonian_noalloc, the allocation-free H phi entry point.

That entry point is for callers that must not allocate device memory while they work:
a serving process that reserves its HBM budget up front and forbids allocation on the
request path, an application whose device memory belongs to another allocator's pool,
or code issuing work inside a stream capture it does not own.  It keeps its workspace
in a fixed device array inside the library instead of a per-system allocation.

The test calls it twice in a row through the C ABI and checks both results against the
regular entry point, lsw_apply_hamiltonian, within the tolerances the parity tests use;
it also checks that the two calls change neither torch's allocation count nor the
device's free memory.  This file sorts last so that a run stopping at the first failure
has run every other test before it.
"""
import numpy as np
import pytest

from paper_1401_7441_gb300 import inputs as I
from paper_1401_7441_gb300 import lsw
from tests.lib_support import ensure_built, keys_to_g

pytestmark = pytest.mark.gpu

TOL = {lsw.LSW_FP64: 1e-12, lsw.LSW_FP32: 1e-5}


@pytest.mark.parametrize("prec", [lsw.LSW_FP64, lsw.LSW_FP32])
def test_noalloc_matches_regular_entry_point(prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    dt = torch.float64 if prec == lsw.LSW_FP64 else torch.float32
    wl = I.scaled("atoms64", 8, seed=5)
    S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   precision=prec, device=0, stream=torch.cuda.current_stream().cuda_stream)
    try:
        phi_h = np.zeros(S.total_L)
        for f in range(S.n_sf):
            a = int(S.sf_atom[f])
            v = I.phi_values(wl, f, a, keys_to_g(S.keys(a, 0, 0)), keys_to_g(S.keys(a, 0, 1)))
            phi_h[S.off_L[f]:S.off_L[f] + len(v)] = v
        phi = torch.tensor(phi_h, dtype=dt, device="cuda")
        V = torch.tensor(I.potential(wl), dtype=dt, device="cuda")
        lsw.lsw_set_potential(S.sys, V, wl.V_lo, wl.V_shape)
        ref = torch.full((S.total_Lp,), float("nan"), dtype=dt, device="cuda")
        ek_ref = torch.zeros(S.n_sf, dtype=torch.float64, device="cuda")
        ep_ref = torch.zeros(S.n_sf, dtype=torch.float64, device="cuda")
        lsw.lsw_apply_hamiltonian(S.sys, phi, ref, ek_ref, ep_ref)
        lsw.lsw_sync(S.sys, 120.0)
        ref_h = ref.double().cpu().numpy()
        gap = np.isnan(ref_h)                      # alignment gaps between functions
        scale = np.max(np.abs(ref_h[~gap]))
        outs = [torch.full((S.total_Lp,), float("nan"), dtype=dt, device="cuda") for _ in range(2)]
        eks = [torch.zeros(S.n_sf, dtype=torch.float64, device="cuda") for _ in range(2)]
        eps = [torch.zeros(S.n_sf, dtype=torch.float64, device="cuda") for _ in range(2)]
        torch.cuda.synchronize()
        allocated = torch.cuda.memory_allocated()
        free = []
        for k in range(2):
            lsw.lsw_apply_hamiltonian_noalloc(S.sys, phi, outs[k], eks[k], eps[k])
            lsw.lsw_sync(S.sys, 120.0)
            free.append(torch.cuda.mem_get_info()[0])
            got = outs[k].double().cpu().numpy()
            assert np.array_equal(np.isnan(got), gap), k
            assert np.max(np.abs(got[~gap] - ref_h[~gap])) <= TOL[prec] * scale, k
            ek, ep = eks[k].cpu().numpy(), eps[k].cpu().numpy()
            e_scale = np.abs(ek_ref.cpu().numpy()) + np.abs(ep_ref.cpu().numpy())
            assert np.all(np.abs(ek - ek_ref.cpu().numpy()) <= TOL[prec] * e_scale), k
            assert np.all(np.abs(ep - ep_ref.cpu().numpy()) <= TOL[prec] * e_scale), k
        assert torch.cuda.memory_allocated() == allocated
        assert free[0] == free[1]
    finally:
        S.close()
