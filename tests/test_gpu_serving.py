"""Serving form: every request's H and S are the same whether it runs alone or mixed
with other requests in flight (continuous batching over CUDA streams), within the
reduced-precision tolerance; reused systems (perturbed geometry, charged variant) go
through lsw_reformat and the resident support functions."""
import numpy as np
import pytest

from paper_1401_7441_gb300 import lsw

pytestmark = pytest.mark.gpu


def _stream():
    from paper_1401_7441_gb300 import serving as SV
    reqs = SV.request_stream(10, rate=200.0, atoms=(40, 160), reuse_frac=0.5, seed=77)
    assert {r.kind for r in reqs} >= {"new"}
    return SV, reqs


def test_each_result_same_alone_and_in_the_mix():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    SV, reqs = _stream()
    srv = SV.Server(budget_bytes=8e9, streams=4, host_threads=4)
    try:
        mixed = {r.rid: r for r in srv.run(reqs, realtime=True)}
    finally:
        srv.close()
    alone = {}
    for r in reqs:
        sub = [r]
        if r.parent is not None:            # a reuse needs its parent resident first
            sub = [q for q in reqs if q.rid == r.parent] + [r]
        srv = SV.Server(budget_bytes=8e9, streams=1, host_threads=1)
        try:
            out = {x.rid: x for x in srv.run(sub, realtime=False, max_inflight=1)}
        finally:
            srv.close()
        alone[r.rid] = out[r.rid]
    assert len(mixed) == len(reqs)
    for rid, a in alone.items():
        m = mixed[rid]
        assert m.n_sf == a.n_sf and len(m.S) == len(a.S)
        d = np.sqrt(np.maximum(a.S[np.isclose(a.S, a.S)], 0))
        scale_s = max(1.0, float(np.max(np.abs(a.S))))
        scale_h = max(1.0, float(np.max(np.abs(a.H))))
        assert np.max(np.abs(m.S - a.S)) <= 1e-5 * scale_s, rid
        assert np.max(np.abs(m.H - a.H)) <= 1e-5 * scale_h, rid
        assert np.max(np.abs(m.e_kin - a.e_kin)) <= 1e-5 * np.max(np.abs(a.e_kin)), rid
        _ = d
    kinds = {r.kind for r in mixed.values()}
    assert "new" in kinds


def test_budget_evicts_and_still_serves():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    SV, reqs = _stream()
    srv = SV.Server(budget_bytes=1.5e9, streams=2, host_threads=2)   # room for few residents
    try:
        res = srv.run(reqs, realtime=False)
        assert len(res) == len(reqs)
        assert srv.used <= srv.budget + 1
        s = SV.summarize(res)
        assert s["p99_latency_s"] >= s["p50_latency_s"] > 0
    finally:
        srv.close()


def test_workspace_bytes_count_the_panels_before_the_first_run():
    # the H/S panel buffers are allocated by the first lsw_build_matrices; the bytes a
    # request loop budgets for a system (lsw_workspace_bytes) are the same before and after
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1401_7441_gb300 import inputs as I
    from tests.lib_support import ensure_built
    ensure_built()
    wl = I.scaled("atoms64", 10, seed=3)
    S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   wl.lprime_margin, 0, lsw.LSW_FP32, device=0, stream=torch.cuda.current_stream().cuda_stream)
    try:
        before = lsw.lsw_workspace_bytes(S.sys)
        lsw.lsw_set_option(S.sys, "slab_mb", 64)           # re-planned, still not allocated
        planned = lsw.lsw_workspace_bytes(S.sys)
        phi = torch.zeros(S.total_L, device="cuda")
        V = torch.tensor(I.potential(wl), dtype=torch.float32, device="cuda")
        lsw.lsw_set_potential(S.sys, V, wl.V_lo, wl.V_shape)
        hphi = torch.zeros(S.total_Lp, device="cuda")
        H = torch.zeros(len(S.col), dtype=torch.float64, device="cuda")
        Sm = torch.zeros_like(H)
        lsw.lsw_apply_hamiltonian(S.sys, phi, hphi)
        lsw.lsw_build_matrices(S.sys, phi, hphi, H, Sm)
        lsw.lsw_sync(S.sys, 60.0)
        assert before > 0 and planned > 0
        assert lsw.lsw_workspace_bytes(S.sys) == planned
    finally:
        S.close()
