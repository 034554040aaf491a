"""GPU parity of the density rho_j = sum_ab K_ab u_a(j) u_b(j) (Sec. II.A, Eq. density)
through the C ABI against the FP64 oracle, point by point.

Tolerance: |rho_gpu - rho| <= tau * rho_abs at every point, where rho_abs is the same
sum taken with |K|, |phi| and the absolute filter taps (a bound of every term, hence
the scale of the rounding error of any summation order); tau = 1e-12 for the FP64
path, 1e-5 for the FP32 ones (the tolerances of H phi).  The FP32 paths also get an
absolute floor of 1e-34: far out in the tails of the blocks the products u_a u_b fall
below FP32's smallest normal number (2^-126, about 1.2e-38) and keep only an absolute
accuracy of that order times the number of terms."""
import numpy as np
import pytest

from oracle import density as Dn
from oracle import geometry as G
from paper_1401_7441_gb300 import inputs as I
from paper_1401_7441_gb300 import lsw
from tests.lib_support import gpu_density
from tests.oracle_support import desc_of, phi_all

pytestmark = pytest.mark.gpu

TOL = {lsw.LSW_FP64: 1e-12, lsw.LSW_FP32: 1e-5, lsw.LSW_FP32_BF16X: 1e-5}
FLOOR = {lsw.LSW_FP64: 0.0, lsw.LSW_FP32: 1e-34, lsw.LSW_FP32_BF16X: 1e-34}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def oracle_density(wl, K, lo, dims):
    geo = G.build(desc_of(wl))
    phi = phi_all(wl, geo)
    rho = Dn.density(geo, phi, K, lo, dims)
    rho_abs = Dn.density(geo, phi, K, lo, dims, absolute=True)
    return geo, rho, rho_abs


def check(gpu_rho, rho, rho_abs, tol, floor=0.0):
    assert np.all(np.isfinite(gpu_rho))                      # every point written
    err = np.abs(gpu_rho - rho)
    bad = err > tol * rho_abs + floor
    assert not bad.any(), (int(bad.sum()), float(err[bad].max()), float(rho_abs[bad].max()))
    assert np.all(gpu_rho[rho_abs == 0] == 0)


def max_cover(wl, geo):
    """Largest number of real-space blocks covering one fine point (chunks of the kernel)."""
    lo, dims = wl.V_lo, wl.V_shape
    cnt = np.zeros(tuple(dims[::-1]), np.int32)
    for f in range(len(geo.sf_atom)):
        L = geo.L[geo.sf_atom[f]]
        o = [2 * L.lo[d] - 14 - lo[d] for d in range(3)]
        n = [2 * (L.hi[d] - L.lo[d] + 1) + 29 for d in range(3)]
        cnt[o[2]:o[2] + n[2], o[1]:o[1] + n[1], o[0]:o[0] + n[0]] += 1
    return int(cnt.max())


@pytest.mark.parametrize("prec", [lsw.LSW_FP64, lsw.LSW_FP32, lsw.LSW_FP32_BF16X])
def test_density_small_system(prec):
    wl = I.scaled("atoms64", 8, seed=5)
    gpu = gpu_density(wl, prec)
    _, rho, rho_abs = oracle_density(wl, gpu["K"], wl.V_lo, wl.V_shape)
    check(gpu["rho"][0], rho, rho_abs, TOL[prec], FLOOR[prec])
    assert rho.max() > 0


def test_density_several_chunks_nonsymmetric_kernel():
    # more than 32 functions over the central points (several 32-function chunks, the
    # K_ab + K_ba blocks), a kernel that is not symmetric, and signs of both kinds
    wl = I.scaled("atoms64", 12, seed=6)
    geo = G.build(desc_of(wl))
    assert max_cover(wl, geo) > 32

    def kernel(row_ptr, col, sf_atom):
        rng = np.random.default_rng(7)
        return rng.uniform(-1.0, 1.0, len(col))

    gpu = gpu_density(wl, lsw.LSW_FP64, kernel=kernel)
    K = gpu["K"]
    rp, col = gpu["row_ptr"], gpu["col"]
    Kd = {}
    for a in range(len(rp) - 1):
        for k in range(rp[a], rp[a + 1]):
            Kd[a, int(col[k])] = K[k]
    assert any(abs(Kd[a, b] - Kd.get((b, a), 0.0)) > 0.1 for a, b in Kd)
    _, rho, rho_abs = oracle_density(wl, K, wl.V_lo, wl.V_shape)
    check(gpu["rho"][0], rho, rho_abs, TOL[lsw.LSW_FP64])


def test_density_single_function_offset_grid_and_repeat():
    # one function (K = [0.7]): rho = 0.7 u^2; a grid wider than needed, starting off the
    # potential's origin, with ragged tiles on every side; a second call (graph replay)
    # gives the same bits; a zero kernel gives zero
    wl = I.single_sf_24()
    lo = [wl.V_lo[0] - 3, wl.V_lo[1] - 5, wl.V_lo[2] - 1]
    dims = [wl.V_shape[0] + 7, wl.V_shape[1] + 9, wl.V_shape[2] + 2]
    gpu = gpu_density(wl, lsw.LSW_FP64, kernel=lambda rp, c, sa: np.full(len(c), 0.7), grid=(lo, dims), repeat=2)
    _, rho, rho_abs = oracle_density(wl, gpu["K"], lo, dims)
    check(gpu["rho"][0], rho, rho_abs, TOL[lsw.LSW_FP64])
    assert np.array_equal(gpu["rho"][0], gpu["rho"][1])
    assert np.all(gpu["rho"][0] >= 0)
    zero = gpu_density(wl, lsw.LSW_FP32, kernel=lambda rp, c, sa: np.zeros(len(c)), grid=(lo, dims))
    assert np.all(zero["rho"][0] == 0)


def test_density_grid_must_cover_every_block():
    torch = pytest.importorskip("torch")
    wl = I.single_sf_24()
    lo = [wl.V_lo[0] + 1, wl.V_lo[1], wl.V_lo[2]]
    with pytest.raises(lsw.LswError) as e:
        gpu_density(wl, lsw.LSW_FP64, grid=(lo, wl.V_shape))
    assert e.value.status == lsw.LSW_ERR_ARG
    torch.cuda.synchronize()


def test_density_trace_matches_potential_energy_matrix():
    # sum_j V_j rho_j = sum_ab K_ab <phi_a|V|phi_b>; with K = identity this is the sum of
    # the potential energies E_pot,a the Hamiltonian path reports
    import torch
    from tests.lib_support import gpu_run
    wl = I.scaled("atoms64", 6, seed=9)
    ident = lambda rp, col, sa: np.array([1.0 if col[k] == a else 0.0
                                          for a in range(len(rp) - 1) for k in range(rp[a], rp[a + 1])])
    dens = gpu_density(wl, lsw.LSW_FP64, kernel=ident)
    ham = gpu_run(wl, lambda f, a, gc, gf: I.phi_values(wl, f, a, gc, gf), lsw.LSW_FP64)
    V = I.potential(wl)
    tr = float(np.sum(V * dens["rho"][0]))
    assert abs(tr - float(np.sum(ham["ep"]))) <= 1e-11 * float(np.sum(np.abs(ham["ep"])))


class _LazyPhi(dict):
    """Compressed vectors from the input generator, made on first use."""

    def __init__(self, wl, geo):
        super().__init__()
        self.wl, self.geo = wl, geo

    def __missing__(self, f):
        a = self.geo.sf_atom[f]
        L = self.geo.L[a]
        v = I.phi_values(self.wl, f, a, L.coarse.g, L.fine.g)
        self[f] = v
        return v


def test_density_atoms1200_full_size_sampled_fp32():
    # the whole 1,200-atom workload (4,096 functions, real-space store of several GB,
    # int64 offsets), every grid point written; a cluster of points at the centre of the
    # atom cube plus scattered points against the oracle evaluated point by point
    import torch
    from tests.lib_support import ensure_built, keys_to_g
    ensure_built()
    wl = I.atoms1200()
    geo = G.build(desc_of(wl))
    vol = sum(int(np.prod(2 * (geo.L[a].hi - geo.L[a].lo + 1) + 29)) for a in geo.sf_atom)
    assert vol > 1 << 31                     # store offsets beyond 2^31 elements
    K = I.density_kernel(wl, geo.sf_atom, geo.row_ptr, geo.col)
    c = int(round(2 * (8.0 + 30.0) / wl.h))
    rng = np.random.default_rng(11)
    pts = [[c, c, c], [c + 7, c, c + 3], [c, c + 7, c + 7], [c + 5, c + 6, c]]
    pts += [list(rng.integers(wl.V_lo[0], wl.V_lo[0] + wl.V_shape[0], 3))]
    pts = np.asarray(pts, np.int64)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                       wl.lprime_margin, 0, lsw.LSW_FP32, device=0, stream=st.cuda_stream)
        try:
            assert np.array_equal(S.row_ptr, geo.row_ptr) and np.array_equal(S.col, geo.col)
            phi = torch.zeros(S.total_L, dtype=torch.float32, device="cuda")
            atoms = sorted(set(int(a) for a in S.sf_atom))
            I.fill_phi(wl, phi, S.off_L, S.sf_atom, {a: keys_to_g(S.keys(a, 0, 0)) for a in atoms},
                       {a: keys_to_g(S.keys(a, 0, 1)) for a in atoms})
            Kd = torch.tensor(K, dtype=torch.float64, device="cuda")
            d = wl.V_shape
            rho = torch.full((d[2], d[1], d[0]), float("nan"), dtype=torch.float64, device="cuda")
            lsw.lsw_build_density(S.sys, phi, Kd, rho, wl.V_lo, wl.V_shape)
            lsw.lsw_sync(S.sys, 600.0)
            torch.cuda.synchronize()
            assert bool(torch.isfinite(rho).all())
            q = torch.as_tensor(pts - np.asarray(wl.V_lo), device="cuda")
            got = rho[q[:, 2], q[:, 1], q[:, 0]].cpu().numpy()
        finally:
            S.close()
    phi_o = _LazyPhi(wl, geo)
    ref = Dn.density_points(geo, phi_o, K, pts)
    ref_abs = Dn.density_points(geo, phi_o, K, pts, absolute=True)
    assert np.all(np.abs(got - ref) <= TOL[lsw.LSW_FP32] * ref_abs + FLOOR[lsw.LSW_FP32]), (got, ref)
    assert np.all(ref_abs[:4] > 0)
