"""The sharded form on one GPU: every rank's sub-system through the library in turn.

Each rank (x slabs of the atoms, balanced by support functions) builds its sub-system
(own atoms first, then the halo whose functions its rows reach, then ghost atoms that
keep the fine region), applies H to its own functions only (option "hphi_limit"), takes
H phi of its halo functions from their owners (the exchange, done here by copying
between the ranks' buffers on the device; across GPUs it is the grouped NCCL send and
receive of shard.exchange_local, tested with gloo ranks on the CPU), and builds H and S.
Every row a rank owns must equal the whole system's row: H phi of own functions bit for
bit, the matrix entries within FP64 rounding of the sums' order."""
import numpy as np
import pytest

from paper_1401_7441_gb300 import inputs as I
from paper_1401_7441_gb300 import lsw
from paper_1401_7441_gb300 import shard
from tests.lib_support import ensure_built, keys_to_g

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ensure_built()


def _system(wl, prec):
    import torch
    return lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                      wl.lprime_margin, 0, prec, device=0, stream=torch.cuda.current_stream().cuda_stream)


def _phi(wl_glob, S, fn_map, atom_map):
    """Compressed phi of a (sub-)system: each function's content is that of its global
    function on its global atom."""
    import torch
    phi = np.zeros(S.total_L)
    for f in range(S.n_sf):
        a = int(S.sf_atom[f])
        v = I.phi_values(wl_glob, int(fn_map[f]), int(atom_map[a]), keys_to_g(S.keys(a, 0, 0)), keys_to_g(S.keys(a, 0, 1)))
        phi[S.off_L[f]:S.off_L[f] + len(v)] = v
    return phi


@pytest.mark.parametrize("world,prec", [(2, lsw.LSW_FP64), (3, lsw.LSW_FP64), (3, lsw.LSW_FP32_BF16X)])
def test_each_rank_owned_rows_equal_whole_system(world, prec):
    import torch
    wl = I.atoms64()
    dt = torch.float64 if prec == lsw.LSW_FP64 else torch.float32
    V = torch.tensor(I.potential(wl), dtype=dt, device="cuda")
    W = _system(wl, prec)
    ranks = []
    try:
        n = W.n_sf
        phi = torch.tensor(_phi(wl, W, np.arange(n), np.arange(len(wl.pos))), dtype=dt, device="cuda")
        lsw.lsw_set_potential(W.sys, V, wl.V_lo, wl.V_shape)
        hphi = torch.zeros(W.total_Lp, dtype=dt, device="cuda")
        Hw = torch.zeros(len(W.col), dtype=torch.float64, device="cuda")
        Sw = torch.zeros_like(Hw)
        lsw.lsw_apply_hamiltonian(W.sys, phi, hphi)
        lsw.lsw_build_matrices(W.sys, phi, hphi, Hw, Sw)
        lsw.lsw_sync(W.sys, 120.0)
        hphi_w, Hw, Sw = hphi.cpu().numpy(), Hw.cpu().numpy(), Sw.cpu().numpy()
        owner = shard.partition_atoms(wl.pos, wl.nsf, world)
        fown = owner[W.sf_atom]
        # phase 1: each rank, its own functions
        for r in range(world):
            w, amap, fmap = shard.subsystem(wl, owner, r, W.sf_atom, W.row_ptr, W.col, own_first=True)
            R = _system(w, prec)
            n_own = int(np.sum(fown == r))
            assert np.all(fown[fmap[:n_own]] == r) and np.all(fown[fmap[n_own:]] != r)
            lsw.lsw_set_option(R.sys, "hphi_limit", n_own)
            ph = torch.tensor(_phi(wl, R, fmap, amap), dtype=dt, device="cuda")
            lsw.lsw_set_potential(R.sys, V, wl.V_lo, wl.V_shape)
            hp = torch.full((R.total_Lp,), float("nan"), dtype=dt, device="cuda")
            lsw.lsw_apply_hamiltonian(R.sys, ph, hp)
            lsw.lsw_sync(R.sys, 120.0)
            ranks.append(dict(R=R, fmap=fmap, n_own=n_own, phi=ph, hphi=hp))
        # the exchange: halo H phi from the owner's buffer, at this rank's offsets
        g2l = [{int(g): k for k, g in enumerate(d["fmap"])} for d in ranks]
        for r, d in enumerate(ranks):
            for k in range(d["n_own"], len(d["fmap"])):
                g = int(d["fmap"][k])
                q = int(fown[g])
                src = ranks[q]
                kq = g2l[q][g]
                a0, a1 = int(src["R"].off_Lp[kq]), int(src["R"].off_Lp[kq + 1])
                b0, b1 = int(d["R"].off_Lp[k]), int(d["R"].off_Lp[k + 1])
                assert a1 - a0 == b1 - b0
                d["hphi"][b0:b1] = src["hphi"][a0:a1]
        # phase 2: each rank's matrices; its own rows against the whole system's
        for r, d in enumerate(ranks):
            R = d["R"]
            Hr = torch.zeros(len(R.col), dtype=torch.float64, device="cuda")
            Sr = torch.zeros_like(Hr)
            lsw.lsw_build_matrices(R.sys, d["phi"], d["hphi"], Hr, Sr)
            lsw.lsw_sync(R.sys, 120.0)
            Hr, Sr, hp = Hr.cpu().numpy(), Sr.cpu().numpy(), d["hphi"].cpu().numpy()
            fmap = d["fmap"]
            for k in range(d["n_own"]):
                g = int(fmap[k])
                # H phi of an own function: the same bits as the whole system's
                a0, a1 = int(R.off_Lp[k]), int(R.off_Lp[k + 1])
                w0 = int(W.off_Lp[g])
                ok = ~np.isnan(hp[a0:a1])
                assert np.array_equal(hp[a0:a1][ok], hphi_w[w0:w0 + (a1 - a0)][ok]), (r, g)
                # the row: same columns, same values
                cols = fmap[R.col[R.row_ptr[k]:R.row_ptr[k + 1]]]
                wcols = W.col[W.row_ptr[g]:W.row_ptr[g + 1]]
                assert np.array_equal(np.sort(cols), wcols), (r, g)
                order = np.argsort(cols)
                hs = Hr[R.row_ptr[k]:R.row_ptr[k + 1]][order]
                ss = Sr[R.row_ptr[k]:R.row_ptr[k + 1]][order]
                hw = Hw[W.row_ptr[g]:W.row_ptr[g + 1]]
                sw = Sw[W.row_ptr[g]:W.row_ptr[g + 1]]
                assert np.max(np.abs(ss - sw)) <= 1e-12 * max(1.0, np.max(np.abs(sw))), (r, g)
                assert np.max(np.abs(hs - hw)) <= 1e-12 * max(1.0, np.max(np.abs(hw))), (r, g)
        # every function is owned exactly once
        assert sorted(int(g) for d in ranks for g in d["fmap"][:d["n_own"]]) == list(range(n))
    finally:
        for d in ranks:
            d["R"].close()
        W.close()
