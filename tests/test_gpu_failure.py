"""Failure handling on the GPU without a fault: lsw_sync's bounded wait.

lsw_sync polls an event and returns LSW_ERR_TIMEOUT when the system's work has not
finished in time; it never blocks longer and leaves the system usable.  The test
enqueues a step that takes tens of milliseconds, asks for a microsecond, and then
waits normally: the results must be those of an undisturbed run."""
import numpy as np
import pytest

from paper_1401_7441_gb300 import inputs as I
from paper_1401_7441_gb300 import lsw
from tests.lib_support import ensure_built, keys_to_g

pytestmark = pytest.mark.gpu


def test_sync_timeout_then_normal_sync():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    wl = I.scaled("atoms10k", 400)
    st = torch.cuda.Stream()
    S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   precision=lsw.LSW_FP32, device=0, stream=st.cuda_stream)
    try:
        phi = torch.zeros(S.total_L, dtype=torch.float32, device="cuda")
        atoms = sorted(set(int(a) for a in S.sf_atom))
        with torch.cuda.stream(st):
            I.fill_phi(wl, phi, S.off_L, S.sf_atom, {a: keys_to_g(S.keys(a, 0, 0)) for a in atoms},
                       {a: keys_to_g(S.keys(a, 0, 1)) for a in atoms})
            V = I.potential_fast(wl, "cuda").to(torch.float32)
        torch.cuda.synchronize()
        lsw.lsw_set_potential(S.sys, V, wl.V_lo, wl.V_shape)
        out = []
        for k in range(2):
            hphi = torch.zeros(S.total_Lp, dtype=torch.float32, device="cuda")
            H = torch.zeros(len(S.col), dtype=torch.float64, device="cuda")
            Sm = torch.zeros_like(H)
            lsw.lsw_apply_hamiltonian(S.sys, phi, hphi)
            lsw.lsw_build_matrices(S.sys, phi, hphi, H, Sm)
            if k == 0:
                with pytest.raises(lsw.LswError) as e:
                    lsw.lsw_sync(S.sys, 1e-6)
                assert e.value.status == lsw.LSW_ERR_TIMEOUT
            lsw.lsw_sync(S.sys, 600.0)
            out.append((hphi.cpu().numpy(), H.cpu().numpy(), Sm.cpu().numpy()))
        assert np.array_equal(out[0][0], out[1][0])          # H phi: no atomics, same bits
        for a, b in zip(out[0][1:], out[1][1:]):             # H, S: FP64 sums in any order
            assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(a))
        assert np.abs(out[0][2]).max() > 0
    finally:
        S.close()
