"""Spatial sharding of a locreg system over ranks, with one halo exchange.

The H phi step has independent units (one support function each, given V); the H/S
build needs, for the rows of a rank's own functions, phi and H phi of every column of
those rows.  Sharding therefore takes one exchange step (the paper distributes its
support functions over MPI tasks and forms the matrices in a redistributed layout,
App. D): atoms are cut into slabs along x, each rank applies H to the functions of its
own atoms, then receives phi and H phi of the functions its rows reach on other ranks
(its halo) and sends those of its own functions that other ranks' rows reach.  After
the exchange every owned row of H and S is complete locally: no reduction of matrices.

Everything here is host logic over the library's pattern and layout (no method
arithmetic); the exchange runs on ``torch.distributed`` (NCCL on GPUs, gloo on CPUs)
as grouped point-to-point sends and receives.
"""
from __future__ import annotations

import numpy as np


def partition_atoms(pos, nsf, world):
    """owner[atom]: slabs along x, cut so that each rank holds about the same number of
    support functions (atoms in x order, ties by index)."""
    pos = np.asarray(pos, np.float64)
    nsf = np.asarray(nsf, np.int64)
    order = np.lexsort((np.arange(len(pos)), pos[:, 0]))
    csum = np.cumsum(nsf[order])
    total = max(1, int(csum[-1])) if len(csum) else 1
    owner = np.empty(len(pos), np.int64)
    # the atom whose functions end at csum belongs to the rank of its first function
    first = csum - nsf[order]
    owner[order] = np.minimum(first * world // total, world - 1)
    return owner


def halo_plan(row_ptr, col, sf_atom, owner, rank):
    """(send, recv): for every other rank r, the functions this rank sends to r (its own
    functions that appear in rows owned by r) and receives from r (functions of r that
    appear in this rank's rows), ascending.  The pattern is symmetric, so rank q's send
    list to r is rank r's receive list from q."""
    row_ptr = np.asarray(row_ptr, np.int64)
    col = np.asarray(col, np.int64)
    fown = np.asarray(owner, np.int64)[np.asarray(sf_atom, np.int64)]     # owner of each function
    send, recv = {}, {}
    for a in np.nonzero(fown == rank)[0]:
        for b in col[row_ptr[a]:row_ptr[a + 1]]:
            r = int(fown[b])
            if r != rank:
                recv.setdefault(r, set()).add(int(b))
                send.setdefault(r, set()).add(int(a))
    return ({r: sorted(v) for r, v in sorted(send.items())}, {r: sorted(v) for r, v in sorted(recv.items())})


def _ranges(off, fs):
    return [(int(off[f]), int(off[f + 1])) for f in fs]


def exchange(buffers, offsets, plan, group=None):
    """Grouped point-to-point halo exchange.

    ``buffers``: list of 1D tensors in the global compressed layout (e.g. phi with the
    offsets of L and H phi with those of L'), each holding this rank's own functions;
    ``offsets``: the matching offset arrays (n_sf + 1).  After the call the halo
    functions' ranges hold the values of their owners.  Every receive is posted before
    the sends; one message per (peer, buffer)."""
    import torch
    import torch.distributed as dist
    send, recv = plan
    reqs, inbox = [], []
    for r, fs in recv.items():
        for bi, (buf, off) in enumerate(zip(buffers, offsets)):
            rg = _ranges(off, fs)
            n = sum(e - s for s, e in rg)
            t = torch.empty(n, dtype=buf.dtype, device=buf.device)
            reqs.append(dist.irecv(t, src=r, group=group, tag=bi))
            inbox.append((buf, rg, t))
    for r, fs in send.items():
        for bi, (buf, off) in enumerate(zip(buffers, offsets)):
            rg = _ranges(off, fs)
            t = torch.cat([buf[s:e] for s, e in rg]) if rg else buf[:0].clone()
            reqs.append(dist.isend(t.contiguous(), dst=r, group=group, tag=bi))
    for q in reqs:
        q.wait()
    for buf, rg, t in inbox:
        p = 0
        for s, e in rg:
            buf[s:e] = t[p:p + (e - s)]
            p += e - s


def subsystem(wl, owner, rank, sf_atom, row_ptr, col, own_first=False):
    """The atoms a rank hands to the library for its share of a sharded run.

    Its own atoms, the atoms of the functions its rows reach (the halo), and ghost atoms
    (no support functions) whose fine spheres can reach the L' region of an own or halo
    atom, so that the fine region -- the union of every atom's fine sphere -- is the same
    as the whole system's wherever a function of the sub-system lives (its keys, layout
    and results are the whole system's).  The grid, the potential's wells and
    every radius are the whole system's.  With ``own_first`` the own atoms come first (so
    the own functions are the sub-system's first functions, the ones the library's
    "hphi_limit" option selects), then the others, each group in global order.  Returns
    (workload, global atom of each sub-system atom, global function of each sub-system
    function)."""
    import copy
    pos = np.asarray(wl.pos, np.float64)
    owner = np.asarray(owner, np.int64)
    sf_atom = np.asarray(sf_atom, np.int64)
    row_ptr = np.asarray(row_ptr, np.int64)
    col = np.asarray(col, np.int64)
    own_atoms = np.nonzero(owner == rank)[0]
    halo_atoms = set()
    for a in np.nonzero(owner[sf_atom] == rank)[0]:
        halo_atoms.update(int(sf_atom[b]) for b in col[row_ptr[a]:row_ptr[a + 1]])
    # L' radius plus the largest fine radius, with a grid diagonal of slack, around every
    # atom with functions here (own and halo): the regions of the halo functions are then
    # the whole system's too, so their phi and H phi have the owner's layout; an extra
    # ghost only repeats fine points the whole system has anyway
    fn_atoms = np.array(sorted(set(own_atoms.tolist()) | halo_atoms), np.int64)
    reach = np.asarray(wl.r_loc)[fn_atoms] + wl.lprime_margin * wl.h + np.max(wl.r_fine) + 2.0 * wl.h
    d2 = np.sum((pos[None, :, :] - pos[fn_atoms][:, None, :]) ** 2, axis=2)
    ghosts = set(np.nonzero(np.any(d2 <= (reach[:, None]) ** 2, axis=0))[0].tolist())
    keep = sorted(set(own_atoms.tolist()) | halo_atoms | ghosts)
    if own_first:
        own_set = set(own_atoms.tolist())
        keep = sorted(own_set) + [a for a in keep if a not in own_set]
    with_fns = set(own_atoms.tolist()) | halo_atoms
    nsf = np.asarray(wl.nsf, np.int64)
    sub_nsf = np.array([nsf[a] if a in with_fns else 0 for a in keep], np.int64)
    first = np.concatenate([[0], np.cumsum(nsf)])
    fn_map = np.concatenate([np.arange(first[a], first[a] + sub_nsf[k]) for k, a in enumerate(keep)]) \
        if keep else np.zeros(0, np.int64)
    w = copy.copy(wl)
    w.name = "%s_rank%d" % (wl.name, rank)
    w.pos = pos[keep]
    w.r_loc = np.asarray(wl.r_loc)[keep]
    w.r_fine = np.asarray(wl.r_fine)[keep]
    w.nsf = sub_nsf
    return w, np.asarray(keep, np.int64), fn_map.astype(np.int64)


def exchange_local(buffers, offsets, g2l, plan, group=None):
    """The halo exchange of ``exchange`` between ranks whose buffers use their own
    sub-system layouts: ``offsets`` (per buffer, n_local + 1) and ``g2l`` (dict: global
    function -> local function) of this rank.  Function f occupies the same number of
    elements on every rank that holds it (its keys are the same), so each range is sent
    from the owner's layout and written at the receiver's."""
    import torch
    import torch.distributed as dist
    send, recv = plan
    reqs, inbox = [], []
    for r, fs in recv.items():
        for bi, (buf, off) in enumerate(zip(buffers, offsets)):
            rg = [(int(off[g2l[f]]), int(off[g2l[f] + 1])) for f in fs]
            t = torch.empty(sum(e - b for b, e in rg), dtype=buf.dtype, device=buf.device)
            reqs.append(dist.irecv(t, src=r, group=group, tag=bi))
            inbox.append((buf, rg, t))
    for r, fs in send.items():
        for bi, (buf, off) in enumerate(zip(buffers, offsets)):
            rg = [(int(off[g2l[f]]), int(off[g2l[f] + 1])) for f in fs]
            t = torch.cat([buf[b:e] for b, e in rg]) if rg else buf[:0].clone()
            reqs.append(dist.isend(t.contiguous(), dst=r, group=group, tag=bi))
    for q in reqs:
        q.wait()
    for buf, rg, t in inbox:
        p = 0
        for b, e in rg:
            buf[b:e] = t[p:p + (e - b)]
            p += e - b


def cell_weights(blocks_lo, blocks_hi, dims, symmetric=True):
    """Per grid plane along x, the total App. D weight of its points: m(m + 1)/2 per point
    (m^2 without symmetry), m the number of blocks [lo, hi] (inclusive, grid indices) that
    contain the point.  Returns an array of length dims[0]."""
    cnt = np.zeros(tuple(int(d) for d in dims[::-1]), np.int32)        # [z][y][x]
    for lo, hi in zip(np.asarray(blocks_lo), np.asarray(blocks_hi)):
        lo = np.maximum(lo, 0)
        hi = np.minimum(hi, np.asarray(dims) - 1)
        if np.any(hi < lo):
            continue
        cnt[lo[2]:hi[2] + 1, lo[1]:hi[1] + 1, lo[0]:hi[0] + 1] += 1
    m = cnt.astype(np.float64)
    w = m * (m + 1) / 2 if symmetric else m * m
    return w.sum(axis=(0, 1))


def cell_partition(plane_weights, world):
    """Cut the cell into ``world`` slabs of consecutive x planes whose weights are as even
    as a plane-granular cut allows (App. D: the total weight divided among the tasks).
    Returns the first plane of each slab and the end: bounds[r] .. bounds[r + 1] - 1.

    Cut r is placed at the plane where the running total first reaches r / world of the
    total, moved back by one plane when that leaves the slab closer to its share."""
    w = np.asarray(plane_weights, np.float64)
    n = len(w)
    if not 1 <= world <= n:
        raise ValueError("cell_partition: %d slabs of %d planes" % (world, n))
    total = float(w.sum())
    csum = np.concatenate([[0.0], np.cumsum(w)])
    bounds = [0]
    for r in range(1, world):
        target = total * r / world
        k = int(np.searchsorted(csum, target, side="left"))
        k = min(max(k, bounds[-1] + 1), n - (world - r))
        if k - 1 > bounds[-1] and abs(csum[k - 1] - target) < abs(csum[k] - target):
            k -= 1
        bounds.append(k)
    bounds.append(n)
    return np.asarray(bounds, np.int64)
