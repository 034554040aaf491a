"""GPU parity of lsw_reformat (support-function reuse on a displaced geometry) against
the oracle: pure data movement, compared bit for bit."""
import copy

import numpy as np
import pytest

from oracle import geometry as G
from oracle import reformat as R
from paper_1401_7441_gb300 import inputs as I
from paper_1401_7441_gb300 import lsw
from tests.lib_support import ensure_built, keys_to_g
from tests.oracle_support import desc_of

pytestmark = pytest.mark.gpu


def _displaced(wl, seed, sigma=0.05):
    w2 = copy.deepcopy(wl)
    rng = np.random.default_rng(seed)
    w2.pos = wl.pos + rng.normal(0.0, sigma, size=wl.pos.shape) * 10.0   # large enough to change grid points
    return w2


@pytest.mark.parametrize("prec", [lsw.LSW_FP64, lsw.LSW_FP32])
def test_reformat_matches_oracle(prec):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    dt = torch.float64 if prec == lsw.LSW_FP64 else torch.float32
    wl = I.scaled("atoms64", 8, seed=5)
    w2 = _displaced(wl, 11)
    shift = (np.rint(w2.pos / wl.h) - np.rint(wl.pos / wl.h)).astype(np.int32)
    assert np.any(shift != 0)
    st = torch.cuda.current_stream().cuda_stream
    mk = lambda w: lsw.System(w.N, w.h, w.pos, w.r_loc, w.r_fine, w.nsf, w.pair_cutoff, w.pair_mode,
                              precision=prec, device=0, stream=st)
    A, B = mk(wl), mk(w2)
    try:
        phi_h = np.zeros(A.total_L)
        for f in range(A.n_sf):
            a = int(A.sf_atom[f])
            v = I.phi_values(wl, f, a, keys_to_g(A.keys(a, 0, 0)), keys_to_g(A.keys(a, 0, 1)))
            phi_h[A.off_L[f]:A.off_L[f] + len(v)] = v
        src = torch.tensor(phi_h, dtype=dt, device="cuda")
        dst = torch.full((B.total_L,), float("nan"), dtype=dt, device="cuda")
        lsw.lsw_reformat(B.sys, A.sys, shift, src, dst)
        lsw.lsw_sync(B.sys, 60.0)
        got = dst.double().cpu().numpy()
        g1, g2 = G.build(desc_of(wl)), G.build(desc_of(w2))
        src_r = src.double().cpu().numpy()          # the values actually stored (FP32 rounded)
        for f in range(B.n_sf):
            ref = R.reformat(g2, g1, shift, f, src_r[A.off_L[f]:A.off_L[f + 1]])
            assert np.array_equal(got[B.off_L[f]:B.off_L[f] + len(ref)], ref), f
    finally:
        A.close()
        B.close()
