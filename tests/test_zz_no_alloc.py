"""GPU tests of lsw_apply_hamiltonian_noalloc, the allocation-free H phi entry point.

That entry point is for callers that must not allocate device memory while they work:
a serving process that reserves its HBM budget up front and forbids allocation on the
request path, or an application whose device memory belongs to another allocator's
pool.  It keeps its workspace in a fixed device array inside the library instead of a
per-system allocation.

The first test calls it twice in a row through the C ABI, in every precision (FP64,
FP32 and the split-bfloat16 tensor-core z stage), on a system whose functions need
several batches of the fixed array, and checks both results against the regular entry
point, lsw_apply_hamiltonian, within the tolerances the parity tests use; it also checks
that the two calls change neither torch's allocation count nor the device's free
memory.  The second checks that a function too large for the array is refused before
anything is enqueued.  This file sorts last so that a run stopping at the first failure
has run every other test before it.
"""
import numpy as np
import pytest

from paper_1401_7441_gb300 import inputs as I
from paper_1401_7441_gb300 import lsw
from tests.lib_support import ensure_built, keys_to_g

pytestmark = pytest.mark.gpu

TOL = {lsw.LSW_FP64: 1e-12, lsw.LSW_FP32: 1e-5, lsw.LSW_FP32_BF16X: 1e-5}
SCRATCH_BYTES = 32 << 20          # the library's fixed array (lsw.h)


def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()
    return torch


def _workspace_elems(n, npr):
    """Elements of one function's workspace in the fixed array: dense 8-type L box, the
    two z-stage intermediates, the dense 8-type L' box and the z-arm flags (64-aligned)."""
    al = lambda x: (x + 63) // 64 * 64   # noqa: E731
    X, Y = 2 * n[0] + 29, 2 * n[1] + 29
    return (al(8 * n[0] * n[1] * n[2]) + al(2 * n[2] * Y * X) + al(2 * npr[2] * Y * X)
            + al(8 * npr[0] * npr[1] * npr[2]))


def _box(keys, N):
    g0, g1 = keys[:, 0], keys[:, 1]
    lo = np.array([(g0 % N[0]).min(), ((g0 // N[0]) % N[1]).min(), (g0 // (N[0] * N[1])).min()])
    hi = np.array([(g1 % N[0]).max(), ((g1 // N[0]) % N[1]).max(), (g1 // (N[0] * N[1])).max()])
    return hi - lo + 1


@pytest.mark.parametrize("prec", [lsw.LSW_FP64, lsw.LSW_FP32, lsw.LSW_FP32_BF16X])
def test_noalloc_matches_regular_entry_point(prec):
    torch = _cuda()
    dt = torch.float64 if prec == lsw.LSW_FP64 else torch.float32
    wl = I.scaled("atoms64", 8, seed=5)
    S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   precision=prec, device=0, stream=torch.cuda.current_stream().cuda_stream)
    try:
        # the functions need several batches of the fixed array, so later batches
        # overwrite the records and workspace of earlier ones
        es = 8 if prec == lsw.LSW_FP64 else 4
        ws = sum(_workspace_elems(_box(S.keys(int(a), 0, 0), wl.N), _box(S.keys(int(a), 1, 0), wl.N))
                 for a in S.sf_atom) * es
        assert ws > 2 * SCRATCH_BYTES
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


def test_noalloc_refuses_a_function_larger_than_the_array_before_any_work():
    """One FP32 function of locreg radius 12.5 bohr: the regular entry point serves it
    (its own workspace), but its workspace exceeds the fixed array, so the allocation-
    free call returns LSW_ERR_UNSUPPORTED and leaves every output as it was (the energy
    arrays are not even cleared)."""
    torch = _cuda()
    h, R = 0.45, 12.5
    n = 70
    c = (n // 2) * h
    S = lsw.System((n, n, n), h, np.array([[c, c, c]]), np.array([R]), np.array([2.0]), np.array([1], np.int32),
                   1.0, lsw.LSW_PAIR_CUTOFF, precision=lsw.LSW_FP32, device=0,
                   stream=torch.cuda.current_stream().cuda_stream)
    try:
        ws = _workspace_elems(_box(S.keys(0, 0, 0), (n, n, n)), _box(S.keys(0, 1, 0), (n, n, n))) * 4
        assert ws > SCRATCH_BYTES
        lo, shape = [-14] * 3, [2 * n + 29] * 3
        V = torch.zeros(int(np.prod(shape)), dtype=torch.float32, device="cuda")
        lsw.lsw_set_potential(S.sys, V, lo, shape)
        phi = torch.ones(S.total_L, dtype=torch.float32, device="cuda")
        hphi = torch.full((S.total_Lp,), 7.0, dtype=torch.float32, device="cuda")
        ek = torch.full((1,), 3.0, dtype=torch.float64, device="cuda")
        ep = torch.full((1,), 5.0, dtype=torch.float64, device="cuda")
        with pytest.raises(lsw.LswError) as e:
            lsw.lsw_apply_hamiltonian_noalloc(S.sys, phi, hphi, ek, ep)
        assert e.value.status == lsw.LSW_ERR_UNSUPPORTED
        lsw.lsw_sync(S.sys, 60.0)
        assert torch.all(hphi == 7.0).item()
        assert ek.item() == 3.0 and ep.item() == 5.0
        lsw.lsw_apply_hamiltonian(S.sys, phi, hphi, ek, ep)     # the regular path serves it
        lsw.lsw_sync(S.sys, 60.0)
        assert ek.item() > 0.0
    finally:
        S.close()
