"""GPU parity: the sm_103a path through the C ABI against the FP64 oracle, element by
element (tolerances of the method's reading: FP64 path 1e-12, FP32 path 1e-5).  Every
element of H phi on L' is checked against the oracle's absolute-term bound of that
element (the sum of the magnitudes of its terms, which scales the rounding of any
evaluation order), and per function in the 2-norm; energies and H/S entries are scaled
by their Cauchy-Schwarz bounds."""
import math

import numpy as np
import pytest

from oracle import geometry as G
from oracle import hamiltonian as Hm
from oracle import matrices as Mx
from paper_1401_7441_gb300 import inputs as I
from paper_1401_7441_gb300 import lsw
from tests.lib_support import gpu_run
from tests.oracle_support import desc_of

pytestmark = pytest.mark.gpu

TOL = {lsw.LSW_FP64: 1e-12, lsw.LSW_FP32: 1e-5, lsw.LSW_FP32_BF16X: 1e-5}
# absolute floor of the per-element check: FP32 flushes results below 2^-126 to zero
FLOOR = {lsw.LSW_FP64: 0.0, lsw.LSW_FP32: 1e-36, lsw.LSW_FP32_BF16X: 1e-36}


def check_elements(g, h, bound, tol, floor, tag):
    """|H phi_gpu - H phi| <= tol * (absolute-term bound) + floor at every L' element."""
    err = np.abs(g - h)
    bad = err > tol * bound + floor
    assert not bad.any(), (tag, int(bad.sum()), float(np.max(err / np.maximum(bound, 1e-300))))
    return float(np.max(err / np.maximum(bound, 1e-300)))


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def phi_fn(wl):
    return lambda f, a, gc, gf: I.phi_values(wl, f, a, gc, gf)


def oracle_hphi(wl, geo, fs, V):
    out = {}
    for f in fs:
        a = geo.sf_atom[f]
        phi = I.phi_values(wl, f, a, geo.L[a].coarse.g, geo.L[a].fine.g)
        h, ek, ep = Hm.apply_hamiltonian(geo, f, phi, V, wl.V_lo)
        out[f] = (phi, h, ek, ep, Hm.hphi_abs_bound(geo, f, phi, V, wl.V_lo))
    return out


def check_functions(wl, geo, gpu, ref, tol):
    worst = 0.0
    floor = 0.0 if tol <= 1e-12 else 1e-36
    for f, (phi, h, ek, ep, bound) in ref.items():
        o = gpu["off_Lp"][f]
        gh = gpu["hphi"][o:o + len(h)]
        assert np.all(np.isfinite(gh)), f          # every member of L' was written
        check_elements(gh, h, bound, tol, floor, f)
        err = np.linalg.norm(gh - h) / np.linalg.norm(h)
        worst = max(worst, err)
        assert err <= tol, (f, err)
        scale = np.linalg.norm(phi) * np.linalg.norm(h)
        assert abs(gpu["ek"][f] - ek) <= tol * scale, (f, gpu["ek"][f], ek)
        assert abs(gpu["ep"][f] - ep) <= tol * scale, (f, gpu["ep"][f], ep)
    return worst


def check_rows(wl, geo, gpu, ref, rows, tol, h_cols=None):
    rp, col = gpu["row_ptr"], gpu["col"]
    for a in rows:
        phi_a = ref[a][0]
        for k in range(rp[a], rp[a + 1]):
            b = int(col[k])
            phi_b = ref[b][0] if b in ref else I.phi_values(
                wl, b, geo.sf_atom[b], geo.L[geo.sf_atom[b]].coarse.g, geo.L[geo.sf_atom[b]].fine.g)
            s_ref = Mx.overlap_entry(geo, a, b, phi_a, phi_b)
            assert abs(gpu["S"][k] - s_ref) <= tol * np.linalg.norm(phi_a) * np.linalg.norm(phi_b), (a, b)
            if h_cols is None or b in h_cols:
                hb = ref[b][1]
                h_ref = Mx.hamiltonian_entry(geo, a, b, phi_a, hb)
                assert abs(gpu["H"][k] - h_ref) <= tol * np.linalg.norm(phi_a) * np.linalg.norm(hb), (a, b)


@pytest.mark.parametrize("prec", [lsw.LSW_FP64, lsw.LSW_FP32, lsw.LSW_FP32_BF16X])
def test_single_function_box(prec):
    wl = I.single_sf_24()
    geo = G.build(desc_of(wl))
    V = I.potential(wl)
    ref = oracle_hphi(wl, geo, [0], V)
    gpu = gpu_run(wl, phi_fn(wl), prec)
    check_functions(wl, geo, gpu, ref, TOL[prec])
    check_rows(wl, geo, gpu, ref, [0], TOL[prec])
    # H_aa = E_kin + E_pot, S_aa = |phi|^2 = 1
    assert abs(gpu["S"][0] - 1.0) <= TOL[prec]
    assert abs(gpu["H"][0] - (gpu["ek"][0] + gpu["ep"][0])) <= TOL[prec] * abs(gpu["ek"][0])


@pytest.mark.parametrize("prec", [lsw.LSW_FP64, lsw.LSW_FP32, lsw.LSW_FP32_BF16X])
def test_small_system_every_function_and_entry(prec):
    wl = I.scaled("atoms64", 8, seed=5)
    geo = G.build(desc_of(wl))
    V = I.potential(wl)
    n = len(geo.sf_atom)
    ref = oracle_hphi(wl, geo, range(n), V)
    gpu = gpu_run(wl, phi_fn(wl), prec)
    check_functions(wl, geo, gpu, ref, TOL[prec])
    check_rows(wl, geo, gpu, ref, range(n), TOL[prec])


@pytest.mark.parametrize("variant", ["own", "margin3", "margin0", "clipped"])
def test_region_variants(variant):
    wl = I.scaled("atoms64", 5, seed=8)
    fm = "union"
    margin = None
    if variant == "own":
        fm = "own"
        wl.fine_mode = "own"
    elif variant == "margin3":
        margin = 3.0
        wl.lprime_margin = 3.0
    elif variant == "margin0":
        margin = 0.0
        wl.lprime_margin = 0.0
    elif variant == "clipped":
        wl.pos[0] = [0.2, 0.3, 0.1]          # locreg clipped by the box corner
        wl.pos[1] = [wl.N[0] * wl.h - 0.5, 3.0, wl.N[2] * wl.h - 0.7]
    geo = G.build(desc_of(wl))
    V = I.potential(wl)
    n = len(geo.sf_atom)
    ref = oracle_hphi(wl, geo, range(n), V)
    gpu = gpu_run(wl, phi_fn(wl), lsw.LSW_FP64, fine_mode=fm, lprime_margin=margin)
    check_functions(wl, geo, gpu, ref, 1e-12)
    check_rows(wl, geo, gpu, ref, range(n), 1e-12)


def test_options_do_not_change_results():
    wl = I.scaled("atoms64", 8, seed=6)
    base = gpu_run(wl, phi_fn(wl), lsw.LSW_FP64)
    # the alignment gaps between functions are never written (NaN from the fill)
    gap = np.isnan(base["hphi"])
    for opts in ({"batch": 1}, {"batch": 7, "graph": 0}, {"tile": 3}, {"tile": 4}, {"tile": 5, "batch": 64},
                 {"tile": 8, "batch": 512}):
        o = gpu_run(wl, phi_fn(wl), lsw.LSW_FP64, options=opts, repeat=2)
        assert np.array_equal(np.isnan(o["hphi"]), gap), opts
        d = np.abs(o["hphi"][~gap] - base["hphi"][~gap])
        assert np.max(d) <= 1e-13 * np.max(np.abs(base["hphi"][~gap])), opts
        assert np.max(np.abs(o["S"] - base["S"])) <= 1e-13, opts
        assert np.max(np.abs(o["H"] - base["H"])) <= 1e-12 * np.max(np.abs(base["H"])), opts


@pytest.mark.parametrize("prec", [lsw.LSW_FP64, lsw.LSW_FP32, lsw.LSW_FP32_BF16X])
def test_persistent_plane_kernels_same_bits(prec):
    # option "persistent" (3: both FMA plane kernels) loops over the batch's planes,
    # largest first, from a queue; 0: one CTA per grid slot.  Option "fwd_list" (default
    # 1): the forward x pass computes only the blocks whose input window meets the row's
    # members and zeroes the rest (0: every block; an all-zero window gives +0 either way).
    # H phi is the same bits; uneven radii (5-8 bohr) and several batches (the queue is
    # reset before each).  Against the oracle as well.
    wl = I.scaled("atoms1200", 14, seed=21)
    geo = G.build(desc_of(wl))
    V = I.potential(wl)
    n = len(geo.sf_atom)
    assert len(set(np.round(wl.r_loc, 3))) > 1                 # uneven radii
    runs = {}
    for pers in (0, 1):
        runs[pers] = gpu_run(wl, phi_fn(wl), prec, options={"persistent": 3 * pers, "fwd_list": pers, "batch": 5},
                             repeat=2)
    a, b = runs[0], runs[1]
    gap = np.isnan(a["hphi"])
    assert np.array_equal(np.isnan(b["hphi"]), gap)
    assert np.array_equal(a["hphi"][~gap], b["hphi"][~gap])
    # energies: FP64 sums of per-thread partial sums, in FP32 for the FP32 forms; the
    # kinetic task lists are built with shared-memory atomics, so which thread sums which
    # products varies from run to run (FP32 rounding of the partial sums)
    etol = 1e-12 if prec == lsw.LSW_FP64 else 1e-6
    for k in ("ek", "ep"):
        assert np.allclose(a[k], b[k], rtol=etol, atol=0), k
    assert np.max(np.abs(a["S"] - b["S"])) <= 1e-13 * max(1.0, np.max(np.abs(a["S"])))
    assert np.max(np.abs(a["H"] - b["H"])) <= 1e-12 * np.max(np.abs(a["H"]))
    first = np.searchsorted(geo.sf_atom, np.arange(6))        # one function of each of six atoms
    ref = oracle_hphi(wl, geo, [int(f) for f in first if f < n], V)
    check_functions(wl, geo, b, ref, 1e-12 if prec == lsw.LSW_FP64 else 1e-5)


def test_autotuner_choices_keep_the_results():
    # the autotuner sweeps batch, xy_tc, persistent, fwd_list and tile; whatever it picks,
    # H phi is the same bits as the default form's, and H/S agree within the reduced
    # precision's tolerance (another tile edge regroups the FP32 per-tile sums)
    import torch
    from paper_1401_7441_gb300 import autotune
    wl = I.scaled("atoms1200", 10, seed=5)
    base = gpu_run(wl, phi_fn(wl), lsw.LSW_FP32)
    S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   wl.lprime_margin, 0, lsw.LSW_FP32, device=0, stream=torch.cuda.current_stream().cuda_stream)
    try:
        phi = torch.tensor(base["phi"], dtype=torch.float32, device="cuda")
        V = torch.tensor(I.potential(wl), dtype=torch.float32, device="cuda")
        lsw.lsw_set_potential(S.sys, V, wl.V_lo, wl.V_shape)
        hphi = torch.full((S.total_Lp,), float("nan"), dtype=torch.float32, device="cuda")
        ek = torch.zeros(S.n_sf, dtype=torch.float64, device="cuda")
        ep = torch.zeros_like(ek)
        H = torch.zeros(len(S.col), dtype=torch.float64, device="cuda")
        Sm = torch.zeros_like(H)
        rep = autotune.autotune(S, phi, hphi, H, Sm, ek, ep, torch.cuda.current_stream(),
                                batches=(4, 16, 64), tiles=(4, 6))
        assert set(rep["chosen"]) >= {"batch", "tile", "xy_tc", "persistent", "fwd_list"}
        H.zero_()
        Sm.zero_()
        lsw.lsw_apply_hamiltonian(S.sys, phi, hphi, ek, ep)
        lsw.lsw_build_matrices(S.sys, phi, hphi, H, Sm)
        lsw.lsw_sync(S.sys, 120.0)
        got = hphi.double().cpu().numpy()
        gap = np.isnan(base["hphi"])
        assert np.array_equal(got[~gap], base["hphi"][~gap])
        assert np.max(np.abs(Sm.cpu().numpy() - base["S"])) <= 1e-5 * max(1.0, np.max(np.abs(base["S"])))
        assert np.max(np.abs(H.cpu().numpy() - base["H"])) <= 1e-5 * np.max(np.abs(base["H"]))
    finally:
        S.close()


@pytest.mark.parametrize("prec", [lsw.LSW_FP64, lsw.LSW_FP32, lsw.LSW_FP32_BF16X])
def test_atoms64_full_size_sampled(prec):
    wl = I.atoms64()
    geo = G.build(desc_of(wl))
    V = I.potential(wl)
    gpu = gpu_run(wl, phi_fn(wl), prec)
    rows = [0, 101]
    need = set(rows)
    for a in rows:
        need |= set(int(b) for b in gpu["col"][gpu["row_ptr"][a]:gpu["row_ptr"][a + 1]])
    need |= {57, 207}
    ref = oracle_hphi(wl, geo, sorted(need), V)
    check_functions(wl, geo, gpu, ref, TOL[prec])
    check_rows(wl, geo, gpu, ref, rows, TOL[prec])


def test_step_host_equals_device_calls():
    import torch
    from tests.lib_support import ensure_built, keys_to_g
    ensure_built()
    wl = I.scaled("atoms64", 6, seed=9)
    dev = gpu_run(wl, phi_fn(wl), lsw.LSW_FP64)
    S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   precision=lsw.LSW_FP64, device=0, stream=torch.cuda.current_stream().cuda_stream)
    try:
        # several batches: Phi goes up and H phi comes back batch by batch on copy streams
        lsw.lsw_set_option(S.sys, "batch", 4)
        V = torch.tensor(I.potential(wl), dtype=torch.float64, device="cuda")
        lsw.lsw_set_potential(S.sys, V, wl.V_lo, wl.V_shape)
        gap = np.isnan(dev["hphi"])                 # alignment gaps: never written
        for _ in range(2):                          # the second call reuses the copy streams
            H = np.zeros(len(S.col))
            Sm = np.zeros(len(S.col))
            hphi = np.zeros(S.total_Lp)
            ek = np.zeros(S.n_sf)
            ep = np.zeros(S.n_sf)
            lsw.lsw_step_host(S.sys, dev["phi"], hphi, H, Sm, ek, ep)
            assert np.max(np.abs(hphi[~gap] - dev["hphi"][~gap])) <= 1e-13 * np.max(np.abs(dev["hphi"][~gap]))
            assert np.max(np.abs(H - dev["H"])) <= 1e-12 * np.max(np.abs(dev["H"]))
            assert np.max(np.abs(Sm - dev["S"])) <= 1e-13
            assert np.allclose(ek, dev["ek"], rtol=1e-12, atol=0) and np.allclose(ep, dev["ep"], rtol=1e-12, atol=0)
    finally:
        S.close()


@pytest.mark.parametrize("prec", [lsw.LSW_FP64, lsw.LSW_FP32, lsw.LSW_FP32_BF16X])
def test_graph_path_on_created_stream(prec):
    # on a created (non-default) stream the library replays captured CUDA graphs
    import torch
    wl = I.scaled("atoms64", 8, seed=5)
    geo = G.build(desc_of(wl))
    V = I.potential(wl)
    n = len(geo.sf_atom)
    ref = oracle_hphi(wl, geo, range(n), V)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        gpu = gpu_run(wl, phi_fn(wl), prec, repeat=3)
    check_functions(wl, geo, gpu, ref, TOL[prec])
    check_rows(wl, geo, gpu, ref, range(n), TOL[prec])


def test_split_bf16_parts_against_fp32_and_oracle():
    # Tensor-core z stage (split bfloat16, FP32 accumulation): 2 parts (3 products)
    # are within the reduced-precision tolerance of the oracle; 3 parts (6 products)
    # sit at the FP32 rounding level, far closer to the FP32 FMA path than 2 parts.
    wl = I.scaled("atoms64", 6, seed=12)
    geo = G.build(desc_of(wl))
    V = I.potential(wl)
    n = len(geo.sf_atom)
    ref = oracle_hphi(wl, geo, range(n), V)
    f32 = gpu_run(wl, phi_fn(wl), lsw.LSW_FP32)
    errs = {}
    for parts in (2, 3):
        g = gpu_run(wl, phi_fn(wl), lsw.LSW_FP32_BF16X, options={"zsplit": parts})
        errs[parts] = check_functions(wl, geo, g, ref, 1e-5)
        check_rows(wl, geo, g, ref, range(n), 1e-5)
        gap = np.isnan(f32["hphi"])
        assert np.array_equal(np.isnan(g["hphi"]), gap)
        d = np.linalg.norm(g["hphi"][~gap] - f32["hphi"][~gap]) / np.linalg.norm(f32["hphi"][~gap])
        errs[(parts, "f32")] = d
    assert errs[(3, "f32")] <= 2e-7, errs
    assert errs[(3, "f32")] < errs[(2, "f32")], errs
    f32_err = check_functions(wl, geo, f32, ref, 1e-5)
    assert errs[3] <= 3 * f32_err + 1e-7, errs


def test_split_bf16_option_errors():
    import torch
    from tests.lib_support import ensure_built
    ensure_built()
    wl = I.scaled("atoms64", 3, seed=2)
    S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   precision=lsw.LSW_FP32, device=0, stream=torch.cuda.current_stream().cuda_stream)
    try:
        with pytest.raises(lsw.LswError):
            lsw.lsw_set_option(S.sys, "zsplit", 3)       # not a split-bfloat16 system
    finally:
        S.close()
    S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   precision=lsw.LSW_FP32_BF16X, device=0, stream=torch.cuda.current_stream().cuda_stream)
    try:
        with pytest.raises(lsw.LswError):
            lsw.lsw_set_option(S.sys, "zsplit", 4)
        lsw.lsw_set_option(S.sys, "zsplit", 3)
        lsw.lsw_set_option(S.sys, "zsplit", 2)
    finally:
        S.close()


@pytest.mark.parametrize("parts", [2, 3])
def test_tensor_core_plane_kernels_option(parts):
    # option "xy_tc": the x and y passes of the plane kernels on the tensor cores too
    wl = I.scaled("atoms64", 6, seed=13)
    geo = G.build(desc_of(wl))
    V = I.potential(wl)
    n = len(geo.sf_atom)
    ref = oracle_hphi(wl, geo, range(n), V)
    g = gpu_run(wl, phi_fn(wl), lsw.LSW_FP32_BF16X, options={"zsplit": parts, "xy_tc": 1})
    err = check_functions(wl, geo, g, ref, 1e-5)
    check_rows(wl, geo, g, ref, range(n), 1e-5)
    if parts == 3:
        assert err <= 1e-6


def _full_size_sampled(wl, prec, options, fs, rows, tol):
    # the bench's launch configuration on the full workload; sampled functions and rows
    # against the oracle (each function's H phi from its own locreg, V from the same
    # sum of wells)
    import torch
    from tests.lib_support import ensure_built, keys_to_g
    ensure_built()
    geo = G.build(desc_of(wl), atoms=sorted(set(int(a) for a in np.repeat(np.arange(len(wl.nsf)), wl.nsf)[fs])),
                  pattern=False)
    dt = torch.float64 if prec == lsw.LSW_FP64 else torch.float32
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                       wl.lprime_margin, 0, prec, device=0, stream=st.cuda_stream)
        try:
            for k, v in options.items():
                lsw.lsw_set_option(S.sys, k, v)
            phi = torch.zeros(S.total_L, dtype=dt, device="cuda")
            atoms = sorted(set(int(a) for a in S.sf_atom))
            I.fill_phi(wl, phi, S.off_L, S.sf_atom, {a: keys_to_g(S.keys(a, 0, 0)) for a in atoms},
                       {a: keys_to_g(S.keys(a, 0, 1)) for a in atoms})
            V = I.potential_fast(wl, "cuda").to(dt)
            lsw.lsw_set_potential(S.sys, V, wl.V_lo, wl.V_shape)
            hphi = torch.zeros(S.total_Lp, dtype=dt, device="cuda")
            ek = torch.zeros(S.n_sf, dtype=torch.float64, device="cuda")
            ep = torch.zeros_like(ek)
            H = torch.zeros(len(S.col), dtype=torch.float64, device="cuda")
            Sm = torch.zeros_like(H)
            lsw.lsw_apply_hamiltonian(S.sys, phi, hphi, ek, ep)
            lsw.lsw_build_matrices(S.sys, phi, hphi, H, Sm)
            lsw.lsw_sync(S.sys, 600.0)
            torch.cuda.synchronize()
            hp, phd = hphi.double().cpu().numpy(), phi.double().cpu().numpy()
            Hh, Sh, ekh, eph = H.cpu().numpy(), Sm.cpu().numpy(), ek.cpu().numpy(), ep.cpu().numpy()
            off_L, off_Lp, rp, col = S.off_L, S.off_Lp, S.row_ptr, S.col
        finally:
            S.close()
    ref = {}
    for f in fs:
        a = geo.sf_atom[f]
        L = geo.L[a]
        phi_f = I.phi_values(wl, f, a, L.coarse.g, L.fine.g)
        assert np.allclose(phd[off_L[f]:off_L[f] + len(phi_f)], phi_f, rtol=1e-6, atol=1e-7)
        lo = [2 * int(L.lo[d]) - 14 for d in range(3)]
        shape = [2 * int(L.hi[d] - L.lo[d] + 1) + 29 for d in range(3)]
        Vb = I.potential_block(wl, lo, shape)
        h, e_k, e_p = Hm.apply_hamiltonian(geo, f, phi_f, Vb, lo)
        ref[f] = (phi_f, h)
        g = hp[off_Lp[f]:off_Lp[f] + len(h)]
        assert np.all(np.isfinite(g)), f
        check_elements(g, h, Hm.hphi_abs_bound(geo, f, phi_f, Vb, lo), tol, 0.0 if tol <= 1e-12 else 1e-36, f)
        assert np.linalg.norm(g - h) / np.linalg.norm(h) <= tol, f
        scale = np.linalg.norm(phi_f) * np.linalg.norm(h)
        assert abs(ekh[f] - e_k) <= tol * scale and abs(eph[f] - e_p) <= tol * scale, f
    for a in rows:
        for k in range(rp[a], rp[a + 1]):
            b = int(col[k])
            if b not in ref:
                continue
            pa, pb, hb = ref[a][0], ref[b][0], ref[b][1]
            s_ref = Mx.overlap_entry(geo, a, b, pa, pb)
            h_ref = Mx.hamiltonian_entry(geo, a, b, pa, hb)
            assert abs(Sh[k] - s_ref) <= tol * np.linalg.norm(pa) * np.linalg.norm(pb), (a, b)
            assert abs(Hh[k] - h_ref) <= tol * np.linalg.norm(pa) * np.linalg.norm(hb), (a, b)


def test_atoms10k_full_size_sampled_split_bf16():
    # 28,000 functions at the launch shape the benchmark's autotuner picks on a GB300
    # (batch 4096, tile edge 6, the persistent backward plane kernel and the forward
    # member block lists, both defaults); every L' element of the sampled functions
    # checked, in the first, a middle and the last batch
    wl = I.atoms10k()
    fs = [0, 1, 2, 3, 4, 5, 6, 7, 13999, 27999]
    _full_size_sampled(wl, lsw.LSW_FP32_BF16X, {"batch": 4096, "tile": 6}, fs, [0, 1, 2], 1e-5)


def test_atoms1200_full_size_sampled_fp32():
    # 4,096 functions on radii 5-8 bohr, all in one batch (one launch per stage) at the
    # benchmark's autotuned tile edge 8
    wl = I.atoms1200()
    fs = list(range(12)) + [2047, 4095]
    _full_size_sampled(wl, lsw.LSW_FP32, {"batch": 4096, "tile": 8}, fs, [0, 1, 4], 1e-5)


def test_fp64_largest_locregs_plane_kernel_without_staging():
    # FP64 locregs of 8 bohr leave no shared-memory room for staging the z-arm plane in
    # the backward plane kernel; the host then has it read from global memory
    wl = I.scaled("atoms1200", 40, seed=31)
    big = [i for i in range(len(wl.r_loc)) if wl.r_loc[i] >= 8.0 and wl.nsf[i] > 0]
    assert big, "the scaled workload has an 8-bohr locreg"
    first = np.concatenate([[0], np.cumsum(wl.nsf)])
    fs = sorted({int(first[big[0]]), int(first[big[-1]]), 0})
    _full_size_sampled(wl, lsw.LSW_FP64, {"batch": 8}, fs, fs[:1], 1e-12)


@pytest.mark.parametrize("prec", [lsw.LSW_FP32, lsw.LSW_FP32_BF16X])
def test_hs_tensor_core_products_against_fma_and_oracle(prec):
    # the per-tile H/S products on the tensor cores (split bfloat16, 3 parts, 6 products)
    # and on the FMA units: both within the tolerance of the oracle, and close to each
    # other (FP32 rounding of the per-tile sums), for tile edges 4 and 6
    wl = I.scaled("atoms64", 8, seed=5)
    geo = G.build(desc_of(wl))
    V = I.potential(wl)
    n = len(geo.sf_atom)
    ref = oracle_hphi(wl, geo, range(n), V)
    for tile in (4, 6):
        g_tc = gpu_run(wl, phi_fn(wl), prec, options={"tile": tile, "hs_tc": 1})
        g_fma = gpu_run(wl, phi_fn(wl), prec, options={"tile": tile, "hs_tc": 0})
        check_rows(wl, geo, g_tc, ref, range(n), 1e-5)
        check_rows(wl, geo, g_fma, ref, range(n), 1e-5)
        sd = np.sqrt(np.abs(g_fma["S"][g_fma["row_ptr"][:-1] + np.array(
            [np.searchsorted(g_fma["col"][g_fma["row_ptr"][i]:g_fma["row_ptr"][i + 1]], i) for i in range(n)])]))
        rows = np.repeat(np.arange(n), np.diff(g_fma["row_ptr"]))
        scale = sd[rows] * sd[g_fma["col"]]
        assert np.max(np.abs(g_tc["S"] - g_fma["S"]) / scale) <= 1e-6, tile
        hn = np.array([np.linalg.norm(g_fma["hphi"][g_fma["off_Lp"][f]:g_fma["off_Lp"][f + 1]][
            ~np.isnan(g_fma["hphi"][g_fma["off_Lp"][f]:g_fma["off_Lp"][f + 1]])]) for f in range(n)])
        assert np.max(np.abs(g_tc["H"] - g_fma["H"]) / (sd[rows] * hn[g_fma["col"]])) <= 1e-6, tile
