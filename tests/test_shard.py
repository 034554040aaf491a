"""Sharding over ranks with one halo exchange (host logic, CPU): partition balance, the
symmetry of the halo plan, and world_size-2 gloo ranks that each apply H to their own
functions, exchange phi and H phi of the halo, and form their own rows of H and S,
identical to the single-process result."""
import datetime
import os
import socket
import sys

import numpy as np
import pytest

from paper_1401_7441_gb300 import inputs as I
from paper_1401_7441_gb300 import lsw
from paper_1401_7441_gb300 import shard
from tests.lib_support import ensure_built, host_system

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def test_partition_balances_support_functions():
    wl = I.atoms64()
    for world in (2, 3, 4, 8):
        owner = shard.partition_atoms(wl.pos, wl.nsf, world)
        assert owner.min() >= 0 and owner.max() == world - 1
        counts = np.bincount(owner, weights=wl.nsf, minlength=world)
        assert counts.max() - counts.min() <= 2 * wl.nsf.max(), counts
        # slabs: x order is rank order
        order = np.argsort(wl.pos[:, 0], kind="stable")
        assert np.all(np.diff(owner[order]) >= 0)


def test_halo_plan_is_symmetric_and_complete():
    ensure_built()
    wl = I.atoms64()
    ctx = lsw.lsw_ctx_create(lsw.LSW_HOST_ONLY)
    S = host_system(wl, ctx)
    try:
        world = 3
        owner = shard.partition_atoms(wl.pos, wl.nsf, world)
        plans = [shard.halo_plan(S.row_ptr, S.col, S.sf_atom, owner, r) for r in range(world)]
        fown = owner[S.sf_atom]
        for q in range(world):
            send, recv = plans[q]
            for r in range(world):
                assert send.get(r, []) == plans[r][1].get(q, [])     # q -> r equals r <- q
            # every column of an owned row is owned here or received
            have = set(np.nonzero(fown == q)[0].tolist()) | set(f for v in recv.values() for f in v)
            for a in np.nonzero(fown == q)[0]:
                assert set(S.col[S.row_ptr[a]:S.row_ptr[a + 1]].tolist()) <= have
            assert all(int(fown[f]) == r for r, v in recv.items() for f in v)
        assert any(plans[0][1])                                  # a real halo
    finally:
        S.close()
        lsw.lsw_ctx_destroy(ctx)


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from oracle import geometry as G
    from oracle import hamiltonian as Hm
    from oracle import matrices as Mx
    from paper_1401_7441_gb300 import inputs as I_
    from paper_1401_7441_gb300 import lsw as L_
    from paper_1401_7441_gb300 import shard as SH
    from tests.lib_support import host_system as hs
    from tests.oracle_support import desc_of
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    try:
        wl = I_.scaled("atoms64", 8, seed=5)
        ctx = L_.lsw_ctx_create(L_.LSW_HOST_ONLY)
        S = hs(wl, ctx)
        owner = SH.partition_atoms(wl.pos, wl.nsf, world)
        plan = SH.halo_plan(S.row_ptr, S.col, S.sf_atom, owner, rank)
        geo = G.build(desc_of(wl))
        V = I_.potential(wl)
        fown = owner[S.sf_atom]
        phi = torch.full((S.total_L,), float("nan"), dtype=torch.float64)
        hphi = torch.full((S.total_Lp,), float("nan"), dtype=torch.float64)
        ref = {}
        for f in range(S.n_sf):
            a = geo.sf_atom[f]
            p = I_.phi_values(wl, f, a, geo.L[a].coarse.g, geo.L[a].fine.g)
            ref[f] = p
            if fown[f] == rank:                                   # own functions only
                phi[S.off_L[f]:S.off_L[f] + len(p)] = torch.from_numpy(p)
                h = Hm.apply_hamiltonian(geo, f, p, V, wl.V_lo)[0]
                hphi[S.off_Lp[f]:S.off_Lp[f] + len(h)] = torch.from_numpy(h)
        SH.exchange([phi, hphi], [S.off_L, S.off_Lp], plan)
        rows = {}
        for a in np.nonzero(fown == rank)[0]:
            na = len(ref[a])
            pa = phi[S.off_L[a]:S.off_L[a] + na].numpy()
            vals = []
            for k in range(S.row_ptr[a], S.row_ptr[a + 1]):
                b = int(S.col[k])
                pb = phi[S.off_L[b]:S.off_L[b] + len(ref[b])].numpy()
                hlen = geo.Lp[geo.sf_atom[b]].n_coef
                hb = hphi[S.off_Lp[b]:S.off_Lp[b] + hlen].numpy()
                assert np.all(np.isfinite(pb)) and np.all(np.isfinite(hb)), (rank, a, b)
                vals.append((Mx.overlap_entry(geo, a, b, pa, pb), Mx.hamiltonian_entry(geo, a, b, pa, hb)))
            rows[int(a)] = vals
        n_halo = sum(len(v) for v in plan[1].values())
        q.put(("ok", rank, rows, n_halo))
        S.close()
        L_.lsw_ctx_destroy(ctx)
    except Exception as e:                     # report instead of leaving the parent waiting
        q.put(("error", rank, repr(e), 0))
        raise
    finally:
        dist.destroy_process_group()


def test_sharded_rows_equal_single_process_gloo():
    import torch.multiprocessing as mp
    from oracle import geometry as G
    from oracle import hamiltonian as Hm
    from oracle import matrices as Mx
    from tests.oracle_support import desc_of, phi_all
    ensure_built()
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, qu)) for r in range(2)]
    for p in procs:
        p.start()
    res = [qu.get(timeout=600) for _ in range(2)]
    for p in procs:
        p.join(120)
    assert all(r[0] == "ok" for r in res), res
    assert all(p.exitcode == 0 for p in procs)
    res = [r[1:] for r in res]
    wl = I.scaled("atoms64", 8, seed=5)
    geo = G.build(desc_of(wl))
    V = I.potential(wl)
    phi = phi_all(wl, geo)
    hphi = {f: Hm.apply_hamiltonian(geo, f, phi[f], V, wl.V_lo)[0] for f in phi}
    H, Sm = Mx.build_matrices(geo, phi, hphi)
    seen = set()
    for rank, rows, n_halo in res:
        assert n_halo > 0
        for a, vals in rows.items():
            assert a not in seen
            seen.add(a)
            for j, k in enumerate(range(geo.row_ptr[a], geo.row_ptr[a + 1])):
                assert vals[j][0] == Sm[k] and vals[j][1] == H[k], (a, k)
    assert seen == set(range(len(geo.sf_atom)))                   # every row owned once


@pytest.mark.parametrize("name,world", [("atoms64", 2), ("atoms64", 3), ("atoms1200_small", 2),
                                        ("atoms64_cutoff8", 2)])
def test_subsystem_reproduces_the_owned_functions(name, world):
    # through the library (host-only): in each rank's sub-system every own and halo
    # function has the same L and L' keys and lengths as in the whole system, and every
    # own function's pattern row maps onto the whole system's row.  With an 8 bohr pair cutoff the halo alone misses atoms
    # whose fine spheres reach L' (R + 8h + r_f = 11.6 bohr): the ghost atoms keep those
    # fine points (without them 82 fine key sets of own functions differ)
    ensure_built()
    wl = I.scaled("atoms1200", 150, seed=4) if name == "atoms1200_small" else I.atoms64()
    if name == "atoms64_cutoff8":
        wl.pair_cutoff = 8.0
    ctx = lsw.lsw_ctx_create(lsw.LSW_HOST_ONLY)
    S = host_system(wl, ctx)
    try:
        owner = shard.partition_atoms(wl.pos, wl.nsf, world)
        fown = owner[S.sf_atom]
        covered = set()
        for r in range(world):
            sw, amap, fmap = shard.subsystem(wl, owner, r, S.sf_atom, S.row_ptr, S.col)
            T = host_system(sw, ctx)
            try:
                assert T.n_sf == len(fmap)
                for fs in range(T.n_sf):
                    f = int(fmap[fs])
                    a, asub = int(S.sf_atom[f]), int(T.sf_atom[fs])
                    assert amap[asub] == a
                    # own and halo functions alike: the whole system's regions and lengths
                    # (the halo's phi and H phi arrive in the owner's layout)
                    for region in (lsw.LSW_REGION_L, lsw.LSW_REGION_LP):
                        for part in (lsw.LSW_PART_COARSE, lsw.LSW_PART_FINE):
                            assert np.array_equal(S.keys(a, region, part), T.keys(asub, region, part)), (f, region, part)
                    assert S.off_L[f + 1] - S.off_L[f] == T.off_L[fs + 1] - T.off_L[fs]
                    assert S.off_Lp[f + 1] - S.off_Lp[f] == T.off_Lp[fs + 1] - T.off_Lp[fs]
                    if fown[f] != r:
                        continue
                    covered.add(f)
                    row = fmap[T.col[T.row_ptr[fs]:T.row_ptr[fs + 1]]]
                    assert np.array_equal(np.sort(row), S.col[S.row_ptr[f]:S.row_ptr[f + 1]])
            finally:
                T.close()
        assert covered == set(range(S.n_sf))
    finally:
        S.close()
        lsw.lsw_ctx_destroy(ctx)


def test_cell_weights_count_the_blocks_touching_each_point():
    # two blocks on a 6 x 1 x 1 line: points 0-1 in one, 2-3 in both, 4-5 in the other
    lo = np.array([[0, 0, 0], [2, 0, 0]])
    hi = np.array([[3, 0, 0], [5, 0, 0]])
    assert np.array_equal(shard.cell_weights(lo, hi, [6, 1, 1]), [1, 1, 3, 3, 1, 1])       # m(m+1)/2
    assert np.array_equal(shard.cell_weights(lo, hi, [6, 1, 1], symmetric=False), [1, 1, 4, 4, 1, 1])


def test_cell_partition_is_as_even_as_planes_allow():
    rng = np.random.default_rng(0)
    for world in (2, 3, 4, 7):
        w = rng.uniform(0, 10, 97) ** 2
        b = shard.cell_partition(w, world)
        assert b[0] == 0 and b[-1] == len(w) and np.all(np.diff(b) >= 1)
        loads = np.array([w[b[r]:b[r + 1]].sum() for r in range(world)])
        # each cut is within one plane of its ideal position
        assert np.max(np.abs(np.cumsum(loads)[:-1] - w.sum() * np.arange(1, world) / world)) <= w.max()
    # uniform weights split exactly; one plane per slab at the limit; more slabs than planes
    assert np.array_equal(shard.cell_partition(np.ones(12), 4), [0, 3, 6, 9, 12])
    assert np.array_equal(shard.cell_partition(np.array([5.0, 0.0, 0.0]), 3), [0, 1, 2, 3])
    with pytest.raises(ValueError):
        shard.cell_partition(np.ones(2), 3)


def test_cell_partition_balances_the_density_work_of_a_workload():
    # the real-space blocks of atoms64: slabs by weight carry about equal m(m+1)/2 totals,
    # unlike equal-width slabs (the centre of the cell is denser than its edges)
    ensure_built()
    wl = I.atoms64()
    ctx = lsw.lsw_ctx_create(lsw.LSW_HOST_ONLY)
    S = host_system(wl, ctx)
    try:
        boxes = []
        for f in range(S.n_sf):
            k = S.keys(int(S.sf_atom[f]), lsw.LSW_REGION_L, lsw.LSW_PART_COARSE)
            g0, g1 = k[:, 0], k[:, 1]
            N = wl.N
            lo = np.array([(g0 % N[0]).min(), ((g0 // N[0]) % N[1]).min(), (g0 // (N[0] * N[1])).min()])
            hi = np.array([(g1 % N[0]).max(), ((g1 // N[0]) % N[1]).max(), (g1 // (N[0] * N[1])).max()])
            boxes.append((2 * lo - 14 - np.array(wl.V_lo), 2 * hi + 16 - np.array(wl.V_lo)))
        w = shard.cell_weights([b[0] for b in boxes], [b[1] for b in boxes], wl.V_shape)
        world = 4
        b = shard.cell_partition(w, world)
        loads = np.array([w[b[r]:b[r + 1]].sum() for r in range(world)])
        eq = np.linspace(0, len(w), world + 1).astype(int)
        eq_loads = np.array([w[eq[r]:eq[r + 1]].sum() for r in range(world)])
        assert loads.max() / loads.mean() < 1.02
        assert eq_loads.max() / eq_loads.mean() > loads.max() / loads.mean()
    finally:
        S.close()
        lsw.lsw_ctx_destroy(ctx)


def _worker_local(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1401_7441_gb300 import inputs as I_
    from paper_1401_7441_gb300 import lsw as L_
    from paper_1401_7441_gb300 import shard as SH
    from tests.lib_support import host_system as hs
    from tests.lib_support import keys_to_g
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=120))
    try:
        wl = I_.scaled("atoms64", 10, seed=6)
        ctx = L_.lsw_ctx_create(L_.LSW_HOST_ONLY)
        W = hs(wl, ctx)
        owner = SH.partition_atoms(wl.pos, wl.nsf, world)
        plan = SH.halo_plan(W.row_ptr, W.col, W.sf_atom, owner, rank)
        w, amap, fmap = SH.subsystem(wl, owner, rank, W.sf_atom, W.row_ptr, W.col, own_first=True)
        R = hs(w, ctx)
        n_own = int(np.sum(owner[W.sf_atom] == rank))
        g2l = {int(g): k for k, g in enumerate(fmap)}
        phi = torch.full((R.total_L,), float("nan"), dtype=torch.float64)
        for k in range(n_own):                                 # own functions only
            a = int(R.sf_atom[k])
            v = I_.phi_values(wl, int(fmap[k]), int(amap[a]), keys_to_g(R.keys(a, 0, 0)), keys_to_g(R.keys(a, 0, 1)))
            phi[R.off_L[k]:R.off_L[k] + len(v)] = torch.from_numpy(v)
        SH.exchange_local([phi], [R.off_L], g2l, plan)
        bad = 0
        for k in range(n_own, R.n_sf):                         # the halo arrived at this rank's offsets
            a = int(R.sf_atom[k])
            v = I_.phi_values(wl, int(fmap[k]), int(amap[a]), keys_to_g(R.keys(a, 0, 0)), keys_to_g(R.keys(a, 0, 1)))
            if not np.array_equal(phi[R.off_L[k]:R.off_L[k] + len(v)].numpy(), v):
                bad += 1
        q.put(("ok", rank, bad, R.n_sf - n_own))
        R.close()
        W.close()
        L_.lsw_ctx_destroy(ctx)
    except Exception as e:
        q.put(("error", rank, repr(e), 0))
        raise
    finally:
        dist.destroy_process_group()


def test_exchange_between_subsystem_layouts_gloo():
    # the exchange of the sharded benchmark: each rank holds its own sub-system layout
    # (own functions first); halo functions arrive from their owners at the local offsets
    import torch.multiprocessing as mp
    ensure_built()
    ctx = mp.get_context("spawn")
    qu = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker_local, args=(r, 2, port, qu)) for r in range(2)]
    for p in procs:
        p.start()
    res = [qu.get(timeout=600) for _ in range(2)]
    for p in procs:
        p.join(120)
    assert all(r[0] == "ok" for r in res), res
    assert all(p.exitcode == 0 for p in procs)
    for _, rank, bad, n_halo in res:
        assert n_halo > 0 and bad == 0, (rank, bad, n_halo)
