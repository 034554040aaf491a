"""Test helpers that drive the library through its binding (no method arithmetic)."""
import numpy as np

from paper_1401_7441_gb300 import build as B
from paper_1401_7441_gb300 import inputs as I
from paper_1401_7441_gb300 import lsw


def ensure_built():
    B.build()
    return lsw.lib()


def host_system(wl, ctx, **kw):
    return lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                      kw.get("lprime_margin", wl.lprime_margin),
                      lsw.LSW_FINE_UNION if kw.get("fine_mode", wl.fine_mode) == "union" else lsw.LSW_FINE_OWN,
                      kw.get("precision", lsw.LSW_FP64), ctx=ctx)


def gpu_run(wl, phi_of, precision=lsw.LSW_FP64, options=None, fine_mode=None, lprime_margin=None,
            repeat=1):
    """Run H phi and H/S on cuda:0.  ``phi_of(f, coarse_g, fine_g)`` -> compressed values."""
    import torch
    ensure_built()
    dt = torch.float64 if precision == lsw.LSW_FP64 else torch.float32
    stream = torch.cuda.current_stream().cuda_stream
    fm = fine_mode or wl.fine_mode
    S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   wl.lprime_margin if lprime_margin is None else lprime_margin,
                   lsw.LSW_FINE_UNION if fm == "union" else lsw.LSW_FINE_OWN, precision,
                   device=0, stream=stream)
    try:
        for k, v in (options or {}).items():
            lsw.lsw_set_option(S.sys, k, v)
        phi_h = np.zeros(S.total_L)
        for f in range(S.n_sf):
            a = int(S.sf_atom[f])
            gc = keys_to_g(S.keys(a, lsw.LSW_REGION_L, lsw.LSW_PART_COARSE))
            gf = keys_to_g(S.keys(a, lsw.LSW_REGION_L, lsw.LSW_PART_FINE))
            v = phi_of(f, a, gc, gf)
            phi_h[S.off_L[f]:S.off_L[f] + len(v)] = v
        phi = torch.tensor(phi_h, dtype=dt, device="cuda")
        V = torch.tensor(I.potential(wl), dtype=dt, device="cuda")
        lsw.lsw_set_potential(S.sys, V, wl.V_lo, wl.V_shape)
        hphi = torch.full((S.total_Lp,), float("nan"), dtype=dt, device="cuda")
        ek = torch.zeros(S.n_sf, dtype=torch.float64, device="cuda")
        ep = torch.zeros(S.n_sf, dtype=torch.float64, device="cuda")
        Hm = torch.zeros(len(S.col), dtype=torch.float64, device="cuda")
        Sm = torch.zeros(len(S.col), dtype=torch.float64, device="cuda")
        for _ in range(repeat):
            lsw.lsw_apply_hamiltonian(S.sys, phi, hphi, ek, ep)
            lsw.lsw_build_matrices(S.sys, phi, hphi, Hm, Sm)
        lsw.lsw_sync(S.sys, 120.0)
        torch.cuda.synchronize()
        out = dict(phi=phi_h, phi_dev=phi.double().cpu().numpy(), hphi=hphi.double().cpu().numpy(),
                   ek=ek.cpu().numpy(), ep=ep.cpu().numpy(), H=Hm.cpu().numpy(), S=Sm.cpu().numpy(),
                   off_L=S.off_L, off_Lp=S.off_Lp, sf_atom=S.sf_atom, row_ptr=S.row_ptr, col=S.col)
        return out
    finally:
        S.close()


def keys_to_g(keys):
    if len(keys) == 0:
        return np.zeros(0, np.int64)
    return np.concatenate([np.arange(s, e + 1, dtype=np.int64) for s, e, _ in keys])


def gpu_density(wl, precision=lsw.LSW_FP64, kernel=None, grid=None, repeat=1, options=None):
    """Run lsw_build_density on cuda:0 with the workload's support functions.

    ``kernel(row_ptr, col, sf_atom)`` -> K values on the pattern (default: the seeded
    density kernel); ``grid`` = (fine_lo, fine_dims), default the potential's grid.
    Returns the density [z, y, x] of every repetition, K and the pattern.  Runs on a
    stream of its own, so that the library captures and replays a CUDA graph."""
    import torch
    ensure_built()
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        return _gpu_density(wl, precision, kernel, grid, repeat, options, st)


def _gpu_density(wl, precision, kernel, grid, repeat, options, st):
    import torch
    dt = torch.float64 if precision == lsw.LSW_FP64 else torch.float32
    stream = st.cuda_stream
    S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   wl.lprime_margin, lsw.LSW_FINE_UNION if wl.fine_mode == "union" else lsw.LSW_FINE_OWN,
                   precision, device=0, stream=stream)
    try:
        for k, v in (options or {}).items():
            lsw.lsw_set_option(S.sys, k, v)
        phi_h = np.zeros(S.total_L)
        for f in range(S.n_sf):
            a = int(S.sf_atom[f])
            gc = keys_to_g(S.keys(a, lsw.LSW_REGION_L, lsw.LSW_PART_COARSE))
            gf = keys_to_g(S.keys(a, lsw.LSW_REGION_L, lsw.LSW_PART_FINE))
            v = I.phi_values(wl, f, a, gc, gf)
            phi_h[S.off_L[f]:S.off_L[f] + len(v)] = v
        phi = torch.tensor(phi_h, dtype=dt, device="cuda")
        if kernel is None:
            Kh = I.density_kernel(wl, S.sf_atom, S.row_ptr, S.col)
        else:
            Kh = np.asarray(kernel(S.row_ptr, S.col, S.sf_atom), np.float64)
        K = torch.tensor(Kh, dtype=torch.float64, device="cuda")
        lo, dims = grid if grid is not None else (wl.V_lo, wl.V_shape)
        out = []
        for _ in range(repeat):
            rho = torch.full((dims[2], dims[1], dims[0]), float("nan"), dtype=torch.float64, device="cuda")
            lsw.lsw_build_density(S.sys, phi, K, rho, lo, dims)
            lsw.lsw_sync(S.sys, 120.0)
            out.append(rho.cpu().numpy())
        torch.cuda.synchronize()
        return dict(rho=out, K=Kh, row_ptr=S.row_ptr, col=S.col, sf_atom=S.sf_atom,
                    workspace=lsw.lsw_workspace_bytes(S.sys))
    finally:
        S.close()
