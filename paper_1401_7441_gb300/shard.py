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
