"""Algorithmic work of one H phi + H/S step, counted from the library's segment keys.

This is the numerator of the roofline figures: the arithmetic the method itself needs,
not what a kernel happens to execute.  For each support function (the count depends
only on its atom's regions, so it is taken per atom and weighted by the atom's
functions) every separable pass is followed through the nonzero support of its data:

* forward passes (synthesis + magic filter, the combined 31-tap filters (w*h), (w*g),
  Sec. II.B Eq. phi): 2 flop for each of the 31 outputs of every nonzero input - the
  eight coefficient types on their members of L (scaling at the coarse members, the
  seven wavelets at the fine ones), then the nonzero rows of each intermediate;
* potential (Sec. III.B): 3 flop per nonzero real-space value (v = V u, E_pot += v u);
* backward passes (the transposed filters onto L', Sec. III.B): 2 flop per tap that
  meets a nonzero input, for every value the compressed result on L' needs (its
  members, then the rows the later passes read);
* kinetic arms (the 29-tap Galerkin blocks of the two-level basis, one axis each):
  2 flop per tap that meets a member of L, for every member of L' and type;
* H/S (Sec. II.A, App. D): one multiply-add per coefficient of L(a) n L(b) (S_ab) and
  of L(a) n L'(b) (H_ab) for every pattern entry (a, b).

The counts are grouped by the kernel that does the work (``fwd_xy``: forward x, y;
``z_stage``: forward z, potential, backward z; ``kinetic``: kinetic z arm; ``bwd_xy``:
backward y, x and the kinetic x, y arms; ``hs_tiles``: the H/S products).  A workload
with more than ``max_atoms`` atoms is counted exactly on a seeded random sample of its
atoms and scaled by functions (the estimate's standard error is reported); the H/S
count always comes from a seeded sample of pattern entries.
"""
from __future__ import annotations

import numpy as np

KINDS = ("fwd_xy", "z_stage", "kinetic", "bwd_xy")


def _mask(keys, lo, n, N):
    """[z][y][x] boolean member mask of one region part on the box lo .. lo + n - 1."""
    m = np.zeros((n[2], n[1], n[0] + 1), np.int32)
    if len(keys):
        g0, g1 = keys[:, 0], keys[:, 1]
        x0 = g0 % N[0] - lo[0]
        x1 = g1 % N[0] - lo[0]
        y = (g0 // N[0]) % N[1] - lo[1]
        z = g0 // (N[0] * N[1]) - lo[2]
        np.add.at(m, (z, y, x0), 1)
        np.add.at(m, (z, y, x1 + 1), -1)
    return np.cumsum(m, axis=2)[:, :, :n[0]] > 0


def _box(keys, N):
    g0, g1 = keys[:, 0], keys[:, 1]
    lo = np.array([(g0 % N[0]).min(), ((g0 // N[0]) % N[1]).min(), (g0 // (N[0] * N[1])).min()])
    hi = np.array([(g1 % N[0]).max(), ((g1 // N[0]) % N[1]).max(), (g1 // (N[0] * N[1])).max()])
    return lo, hi - lo + 1


def _window_count(a, axis, lo_off, hi_off):
    """c[i] = sum of a[i + lo_off .. i + hi_off] along ``axis`` (zero outside)."""
    a = np.moveaxis(a.astype(np.int32), axis, -1)
    n = a.shape[-1]
    cs = np.concatenate([np.zeros(a.shape[:-1] + (1,), np.int32), np.cumsum(a, axis=-1)], axis=-1)
    i = np.arange(n)
    lo = np.clip(i + lo_off, 0, n)
    hi = np.clip(i + hi_off + 1, 0, n)
    return np.moveaxis(cs[..., hi] - cs[..., lo], -1, axis)


def _up(a, axis):
    """Support of a forward (upsampling) pass along ``axis``: out[o] nonzero iff some
    nonzero input q has 0 <= o - 2 q <= 30; length 2 n + 29."""
    a = np.moveaxis(a, axis, -1)
    n = a.shape[-1]
    u = np.zeros(a.shape[:-1] + (2 * n + 29,), np.int32)
    u[..., 0:2 * n:2] = a
    out = _window_count(u, -1, -30, 0) > 0
    return np.moveaxis(out, -1, axis)


def _down_needed(a, axis, off, n_in):
    """Inputs a backward (decimating) pass reads for the needed outputs ``a`` along
    ``axis``: input o is read by output b iff 0 <= o - 2 (b + off) <= 30, o in [0, n_in)."""
    a = np.moveaxis(a, axis, -1)
    nb = a.shape[-1]
    out = np.zeros(a.shape[:-1] + (n_in,), bool)
    for b in range(nb):
        col = a[..., b]
        if not col.any():
            continue
        o0 = max(0, 2 * (b + off))
        o1 = min(n_in, 2 * (b + off) + 31)
        if o0 < o1:
            out[..., o0:o1] |= col[..., None]
    return np.moveaxis(out, -1, axis)


def _down_taps(needed, src, axis, off):
    """For every needed output b along ``axis``, the number of nonzero inputs of ``src``
    among o = 2 (b + off) + m, m = 0..30; returns (sum over needed outputs, computed
    support = needed outputs with at least one nonzero tap)."""
    s = np.moveaxis(src.astype(np.int32), axis, -1)
    nd = np.moveaxis(needed, axis, -1)
    n_in, nb = s.shape[-1], nd.shape[-1]
    cs = np.concatenate([np.zeros(s.shape[:-1] + (1,), np.int32), np.cumsum(s, axis=-1)], axis=-1)
    b = np.arange(nb)
    lo = np.clip(2 * (b + off), 0, n_in)
    hi = np.clip(2 * (b + off) + 31, 0, n_in)
    cnt = cs[..., hi] - cs[..., lo]
    cnt = np.where(nd, cnt, 0)
    return int(cnt.sum()), np.moveaxis(cnt > 0, -1, axis)


def atom_work(keys_L, keys_Lp, N):
    """Flop of every kernel kind for one function of an atom, from the atom's keys:
    keys_L = (coarse, fine) of L, keys_Lp = (coarse, fine) of L' (int64 (n, 3) arrays)."""
    lo, n = _box(keys_L[0], N)
    lop, npr = _box(keys_Lp[0], N)
    # coefficient masks [t] on the L box and the L' box, t = bx + 2 by + 4 bz
    cL = _mask(keys_L[0], lo, n, N)
    fL = _mask(keys_L[1], lo, n, N) if len(keys_L[1]) else np.zeros_like(cL)
    cP = _mask(keys_Lp[0], lop, npr, N)
    fP = _mask(keys_Lp[1], lop, npr, N) if len(keys_Lp[1]) else np.zeros_like(cP)
    D = [cL] + [fL] * 7
    G = [cP] + [fP] * 7
    w = {k: 0.0 for k in KINDS}
    # forward x: row type r = (by, bz) from input types 2r (bx = 0) and 2r + 1 (bx = 1)
    w["fwd_xy"] += 62.0 * sum(int(D[t].sum()) for t in range(8))
    Ax = [_up(D[2 * r] | D[2 * r + 1], 2) for r in range(4)]            # [z][y][x']
    # forward y: type bz from row types (0, bz), (1, bz)
    w["fwd_xy"] += 62.0 * sum(int(Ax[r].sum()) for r in range(4))
    Ay = [_up(Ax[2 * bz] | Ax[2 * bz + 1], 1) for bz in range(2)]       # [z][y'][x']
    w["z_stage"] += 62.0 * sum(int(Ay[bz].sum()) for bz in range(2))
    U = _up(Ay[0] | Ay[1], 0)                                            # [z'][y'][x']
    w["z_stage"] += 3.0 * int(U.sum())
    Z, Y, X = U.shape
    d = lop - lo
    # backward: values the compressed result on L' needs, last pass first
    Nx = [_down_needed(G[2 * r] | G[2 * r + 1], 2, d[0], X) for r in range(4)]      # [z''][y''][x']
    Ny = [_down_needed(Nx[2 * bz] | Nx[2 * bz + 1], 1, d[1], Y) for bz in range(2)]  # [z''][y'][x']
    cz, Cz = 0, []
    for bz in range(2):
        c, s = _down_taps(Ny[bz], U, 0, d[2])
        cz += c
        Cz.append(s)
    w["z_stage"] += 2.0 * cz
    cy, Cy = 0, []
    for r in range(4):
        c, s = _down_taps(Nx[r], Cz[r >> 1], 1, d[1])
        cy += c
        Cy.append(s)
    w["bwd_xy"] += 2.0 * cy
    cx = 0
    for t in range(8):
        c, _ = _down_taps(G[t], Cy[t >> 1], 2, d[0])
        cx += c
    w["bwd_xy"] += 2.0 * cx
    # kinetic arms on the L' box: inputs (members of L) placed at their L' box positions
    e0 = lo - lop

    def embed(m):
        e = np.zeros((npr[2], npr[1], npr[0]), bool)
        e[e0[2]:e0[2] + n[2], e0[1]:e0[1] + n[1], e0[0]:e0[0] + n[0]] = m
        return e
    DE = [embed(D[0]), embed(D[1])]                                      # coarse, fine
    for dim, kind in ((0, "bwd_xy"), (1, "bwd_xy"), (2, "kinetic")):
        ax = 2 - dim
        W = [_window_count(DE[0], ax, -14, 14), _window_count(DE[1], ax, -14, 14)]
        tot = 0
        for t in range(8):
            # inputs: types t with bit dim = 0 and = 1 (the scaling type 0 is coarse)
            t0, t1 = t & ~(1 << dim), t | (1 << dim)
            s = (W[0] if t0 == 0 else W[1]) + W[1]
            tot += int(s[G[t]].sum())
            _ = t1
        w[kind] += 2.0 * tot
    return w


def _atom_job(args):
    keys_L, keys_Lp, N = args
    return atom_work(keys_L, keys_Lp, N)


def hphi_work(S, N, max_atoms=1500, sample=512, seed=7, pool=None):
    """Flop per kernel kind of one H phi over every function of system ``S`` (an
    lsw.System); returns (dict kind -> flop, dict of notes)."""
    nsf_of = np.bincount(np.asarray(S.sf_atom), minlength=0)
    atoms = np.nonzero(nsf_of)[0]
    exact = len(atoms) <= max_atoms
    if not exact:
        rng = np.random.default_rng(seed)
        atoms = np.sort(rng.choice(atoms, size=sample, replace=False))
    jobs = [((S.keys(int(a), 0, 0), S.keys(int(a), 0, 1)), (S.keys(int(a), 1, 0), S.keys(int(a), 1, 1)), tuple(N))
            for a in atoms]
    res = list(pool.map(_atom_job, jobs, chunksize=8)) if pool is not None else [_atom_job(j) for j in jobs]
    wts = nsf_of[atoms].astype(np.float64)
    tot = {}
    note = {"atoms_counted": int(len(atoms)), "exact": bool(exact)}
    for k in KINDS:
        v = np.array([r[k] for r in res])
        if exact:
            tot[k] = float(np.sum(v * wts))
        else:
            per_fn = v                                    # flop per function of a sampled atom
            mean = float(np.sum(per_fn * wts) / np.sum(wts))
            tot[k] = mean * S.n_sf
            sd = float(np.sqrt(np.sum(wts * (per_fn - mean) ** 2) / np.sum(wts)))
            note["rel_se_" + k] = sd / mean / np.sqrt(len(atoms)) if mean > 0 else 0.0
    return tot, note


def _g(keys):
    if len(keys) == 0:
        return np.zeros(0, np.int64)
    lens = keys[:, 1] - keys[:, 0] + 1
    starts = np.repeat(keys[:, 0] - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
    return starts + np.arange(int(lens.sum()), dtype=np.int64)


def hs_work(S, sample=3000, seed=11):
    """Multiply-adds of the H/S build over the whole pattern, estimated from a seeded
    uniform sample of pattern entries: per entry (a, b), |L(a) n L(b)| (S) and
    |L(a) n L'(b)| (H), each counted over the scaling part and 7x over the wavelet part.
    Returns (MAC, relative standard error)."""
    nnz = len(S.col)
    if nnz == 0:
        return 0.0, 0.0
    rng = np.random.default_rng(seed)
    k = rng.integers(0, nnz, size=min(sample, nnz))
    rows = np.searchsorted(S.row_ptr, k, side="right") - 1
    cache = {}

    def sets(a):
        if a not in cache:
            cache[a] = (_g(S.keys(a, 0, 0)), _g(S.keys(a, 0, 1)), _g(S.keys(a, 1, 0)), _g(S.keys(a, 1, 1)))
        return cache[a]
    vals = []
    for kk, r in zip(k, rows):
        fa, fb = int(S.sf_atom[r]), int(S.sf_atom[S.col[kk]])
        A, B = sets(fa), sets(fb)
        s = len(np.intersect1d(A[0], B[0], assume_unique=True)) + 7 * len(np.intersect1d(A[1], B[1], assume_unique=True))
        h = len(np.intersect1d(A[0], B[2], assume_unique=True)) + 7 * len(np.intersect1d(A[1], B[3], assume_unique=True))
        vals.append(s + h)
    v = np.asarray(vals, np.float64)
    mean = float(v.mean())
    return mean * nnz, float(v.std() / mean / np.sqrt(len(v))) if mean > 0 else 0.0
