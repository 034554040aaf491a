"""Checkpoint through the C ABI: a system saved with its support functions and loaded
on a new context gives the same H phi bit for bit (same keys, same kernels) and the
same energies, H and S up to the order of their sums (FP64 atomics; in FP32 the
per-thread energy partials follow a task order built with shared-memory atomics)."""
import numpy as np
import pytest

from paper_1401_7441_gb300 import inputs as I
from paper_1401_7441_gb300 import lsw
from tests.lib_support import ensure_built, keys_to_g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def run(sys_handle, phi, wl, dt):
    import torch
    n_sf, total_L, total_Lp, off_L, off_Lp, sf_atom = lsw.lsw_system_layout(sys_handle)
    rp, col = lsw.lsw_pattern(sys_handle)
    V = torch.tensor(I.potential(wl), dtype=dt, device="cuda")
    lsw.lsw_set_potential(sys_handle, V, wl.V_lo, wl.V_shape)
    hphi = torch.zeros(total_Lp, dtype=dt, device="cuda")
    ek = torch.zeros(n_sf, dtype=torch.float64, device="cuda")
    ep = torch.zeros(n_sf, dtype=torch.float64, device="cuda")
    H = torch.zeros(len(col), dtype=torch.float64, device="cuda")
    S = torch.zeros(len(col), dtype=torch.float64, device="cuda")
    lsw.lsw_apply_hamiltonian(sys_handle, phi, hphi, ek, ep)
    lsw.lsw_build_matrices(sys_handle, phi, hphi, H, S)
    lsw.lsw_sync(sys_handle, 120.0)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in (hphi, ek, ep, H, S)]


@pytest.mark.parametrize("prec", [lsw.LSW_FP64, lsw.LSW_FP32_BF16X])
def test_save_load_same_results(prec, tmp_path):
    import torch
    ensure_built()
    wl = I.scaled("atoms64", 7, seed=21)
    dt = torch.float64 if prec == lsw.LSW_FP64 else torch.float32
    stream = torch.cuda.current_stream().cuda_stream
    A = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   precision=prec, device=0, stream=stream)
    ctx2 = lsw.lsw_ctx_create(0, stream)
    path = str(tmp_path / "ckpt.lsw")
    try:
        if prec == lsw.LSW_FP32_BF16X:
            lsw.lsw_set_option(A.sys, "zsplit", 3)
        phi_h = np.zeros(A.total_L)
        for f in range(A.n_sf):
            a = int(A.sf_atom[f])
            v = I.phi_values(wl, f, a, keys_to_g(A.keys(a, 0, 0)), keys_to_g(A.keys(a, 0, 1)))
            phi_h[A.off_L[f]:A.off_L[f] + len(v)] = v
        phi = torch.tensor(phi_h, dtype=dt, device="cuda")
        ref = run(A.sys, phi, wl, dt)
        lsw.lsw_save(A.sys, phi, path)
        B = lsw.lsw_load(ctx2, path)
        try:
            lay = lsw.lsw_system_layout(B)
            phi2 = torch.full((lay[1],), float("nan"), dtype=dt, device="cuda")
            lsw.lsw_load_phi(B, path, phi2)
            assert torch.equal(phi2, phi)
            got = run(B, phi2, wl, dt)
            assert np.array_equal(ref[0], got[0])            # H phi: no atomics
            tol = 1e-13 if prec == lsw.LSW_FP64 else 1e-6
            for x, y in zip(ref[1:], got[1:]):               # order of the sums
                assert np.max(np.abs(x - y)) <= tol * np.max(np.abs(x))
        finally:
            lsw.lsw_system_destroy(B)
        C2 = lsw.lsw_load(ctx2, path, torch.zeros(A.total_L, dtype=dt, device="cuda"))
        lsw.lsw_system_destroy(C2)
    finally:
        A.close()
        lsw.lsw_ctx_destroy(ctx2)


def test_measured_peaks_are_plausible():
    # roofline denominators from the library's own FMA loops and streaming copy
    ensure_built()
    import torch
    ctx = lsw.lsw_ctx_create(0, torch.cuda.current_stream().cuda_stream)
    try:
        f32, f64, copy = lsw.lsw_measure_peaks(ctx)
    finally:
        lsw.lsw_ctx_destroy(ctx)
    assert 10.0 < f32 < 200.0          # TFLOP/s
    assert 0.05 < f64 < 20.0
    assert 500.0 < copy < 20000.0      # GB/s
