"""Seeded synthetic workloads: atoms, radii, potential V(r) and support-function content.

This module is shared by the tests, the benchmark and the oracle's callers; it holds
none of the method's arithmetic (no membership test, no key, no filter, no operator).
Every random number comes from a counter-based generator (a 32-bit integer mixer,
then Box-Muller), so any coefficient can be regenerated on its own from
(seed, function, type, grid index) on the CPU (numpy) or on a GPU (torch).

Workloads (the paper's shapes: 1 support function per H atom and 4 per heavy atom;
grid spacing h = 0.45 bohr; locreg radii 5-8 bohr; atoms up to 10,000):

* ``single_sf_24``   1 function, 24^3 box, fine sphere of radius 6 grid points at
                     the centre, 4 Gaussian wells, every point in the locreg.
* ``atoms64``        64 atoms (16 H-like + 48 heavy, 208 functions) in a 30 bohr cube,
                     min separation 1.8 bohr, R = 6, r_f = 2, pairs within 12 bohr.
* ``atoms1200``      1,200 atoms in a 60 bohr cube, R in {5,6,7,8}, r_f = 0.3 R,
                     4,096 functions, pairs with |R_a - R_b| <= r_a + r_b.
* ``atoms10k``       10,000 atoms (40 % H-like) in a 110 bohr cube, R = 7, r_f = 2.1,
                     28,000 functions, pairs within 14 bohr.
* ``atomsN``         any of the above shrunk/grown: ``scaled(name, n_atoms)``.

Box: the atom cube padded by R_max on every side; N = ceil(extent / h) + 1.
Potential: one Gaussian well per atom, depth D ~ U[1, 3] Ha, width w ~ U[0.5, 1.5]
bohr (``single_sf_24``: 4 wells uniform in the central half of the box), sampled at
x_j = j h / 2 on fine indices j in [-14, 2N + 14] (every point the magic filter can
reach), each well cut off beyond 6 w along each axis.
Support-function content: coefficient = z * exp(-|r_p - R_atom|^2 / (2 sigma^2)),
z ~ N(0, 1) per (seed, function, type, point), sigma = 2 bohr; then scaled to unit
norm (sum of squares over the compressed vector = 1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

V_PAD = 14   # fine points the magic filter reaches beyond 2*i on each side


@dataclass
class Workload:
    name: str
    N: tuple
    h: float
    pos: np.ndarray
    r_loc: np.ndarray
    r_fine: np.ndarray
    nsf: np.ndarray
    pair_cutoff: float
    pair_mode: int              # 0: fixed cutoff, 1: r_a + r_b
    wells: np.ndarray           # (n_wells, 5): cx, cy, cz, depth D, width w
    seed: int
    lprime_margin: float = 8.0
    fine_mode: str = "union"
    sigma: float = 2.0
    precision: str = "fp64"
    extra: dict = field(default_factory=dict)

    @property
    def n_sf(self) -> int:
        return int(np.sum(self.nsf))

    @property
    def V_lo(self):
        return (-V_PAD, -V_PAD, -V_PAD)

    @property
    def V_shape(self):
        return tuple(2 * n + 2 * V_PAD + 1 for n in self.N)


# ----------------------------------------------------------------- counters

_M32 = 0xFFFFFFFF


def _mul32(x, c, xp):
    """(x * c) mod 2^32 for 0 <= x < 2^32 held in int64, without int64 overflow."""
    c_lo, c_hi = c & 0xFFFF, c >> 16
    return ((x * c_lo) + (((x * c_hi) & 0xFFFF) << 16)) & _M32


def mix32(x, xp=np):
    """32-bit integer mixer (xor-shift / multiply, constants 0x7feb352d, 0x846ca68b)."""
    x = x & _M32
    x = x ^ (x >> 16)
    x = _mul32(x, 0x7FEB352D, xp)
    x = x ^ (x >> 15)
    x = _mul32(x, 0x846CA68B, xp)
    x = x ^ (x >> 16)
    return x


def counter_normal(seed, f, t, g, xp=np):
    """N(0,1) deviate for each (seed, function f, type t, grid index g); numpy or torch."""
    k = mix32(g & _M32, xp)
    k = mix32(k ^ ((g >> 32) & _M32) ^ (t * 0x9E3779B1 & _M32), xp)
    k = mix32(k ^ (f & _M32), xp)
    k = mix32(k ^ (seed & _M32), xp)
    a = mix32(k ^ 0x68E31DA4, xp)
    b = mix32(k ^ 0xB5297A4D, xp)
    if xp is np:
        u1 = (a.astype(np.float64) + 0.5) * (1.0 / 4294967296.0)
        u2 = (b.astype(np.float64) + 0.5) * (1.0 / 4294967296.0)
        return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    u1 = (a.to(xp.float64) + 0.5) * (1.0 / 4294967296.0)
    u2 = (b.to(xp.float64) + 0.5) * (1.0 / 4294967296.0)
    return xp.sqrt(-2.0 * xp.log(u1)) * xp.cos(2.0 * math.pi * u2)


def uniform(seed, stream, n):
    """n uniforms in [0,1) from the counter generator (used for geometry)."""
    i = np.arange(n, dtype=np.int64)
    k = mix32(mix32(i ^ (stream * 0x27D4EB2F & _M32)) ^ (seed & _M32))
    return (k.astype(np.float64) + 0.5) / 4294967296.0


# ----------------------------------------------------------------- workloads

def _place_atoms(seed, n_atoms, cube, pad, min_sep):
    pts = []
    draw = 0
    cand = uniform(seed, 1, 3 * 64 * n_atoms).reshape(-1, 3)
    cell = {}
    cs = min_sep
    for p in cand:
        draw += 1
        q = pad + p * cube
        key = tuple((q // cs).astype(int))
        ok = True
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    for r in cell.get((key[0] + dx, key[1] + dy, key[2] + dz), ()):
                        if np.sum((q - r) ** 2) < min_sep * min_sep:
                            ok = False
                            break
                    if not ok:
                        break
                if not ok:
                    break
            if not ok:
                break
        if ok:
            pts.append(q)
            cell.setdefault(key, []).append(q)
            if len(pts) == n_atoms:
                break
    if len(pts) < n_atoms:
        raise RuntimeError("could not place atoms")
    return np.array(pts, dtype=np.float64)


def _wells_per_atom(seed, pos):
    u = uniform(seed, 2, 2 * len(pos)).reshape(-1, 2)
    D = 1.0 + 2.0 * u[:, 0]
    w = 0.5 + u[:, 1]
    return np.column_stack([pos, D, w])


def single_sf_24(seed: int = 1001) -> Workload:
    n = 24
    h = 0.45
    c = np.array([[12 * h, 12 * h, 12 * h]])
    u = uniform(seed, 3, 4 * 5).reshape(4, 5)
    ext = (n - 1) * h
    centres = ext * (0.25 + 0.5 * u[:, :3])
    wells = np.column_stack([centres, 1.0 + 2.0 * u[:, 3], 0.5 + u[:, 4]])
    return Workload("single_sf_24", (n, n, n), h, c, np.array([100.0]),
                    np.array([6.0 * h * (1 + 1e-9)]), np.array([1]), 12.0, 0, wells, seed)


def atoms_cube(name, seed, n_atoms, cube, radii_choices, fine_of_r, frac_h, cutoff,
               pair_mode=0, n_sf_total=None, precision="fp64", h=0.45) -> Workload:
    rmax = max(radii_choices)
    pos = _place_atoms(seed, n_atoms, cube, rmax, 1.8)
    u = uniform(seed, 4, 2 * n_atoms).reshape(-1, 2)
    n_h = int(round(frac_h * n_atoms))
    is_h = np.zeros(n_atoms, dtype=bool)
    is_h[np.argsort(u[:, 0], kind="stable")[:n_h]] = True
    nsf = np.where(is_h, 1, 4).astype(np.int64)
    if n_sf_total is not None:
        extra = int(nsf.sum()) - n_sf_total
        k = n_atoms - 1
        while extra > 0:
            if nsf[k] > 1:
                take = min(extra, int(nsf[k]) - 1)
                nsf[k] -= take
                extra -= take
            k -= 1
    rc = np.asarray(radii_choices, dtype=np.float64)
    r_loc = rc[np.minimum((u[:, 1] * len(rc)).astype(int), len(rc) - 1)]
    r_fine = np.array([fine_of_r(r) for r in r_loc])
    ext = cube + 2 * rmax
    N = int(math.ceil(ext / h)) + 1
    return Workload(name, (N, N, N), h, pos, r_loc, r_fine, nsf, cutoff, pair_mode,
                    _wells_per_atom(seed, pos), seed, precision=precision)


def atoms64(seed: int = 1002) -> Workload:
    return atoms_cube("atoms64", seed, 64, 30.0, [6.0], lambda r: 2.0, 16 / 64, 12.0)


def atoms1200(seed: int = 1003) -> Workload:
    return atoms_cube("atoms1200", seed, 1200, 60.0, [5.0, 6.0, 7.0, 8.0],
                      lambda r: 0.3 * r, 234 / 1200, 0.0, pair_mode=1, n_sf_total=4096,
                      precision="fp32")


def atoms10k(seed: int = 1004) -> Workload:
    # the 10,000-atom configuration runs the z-direction magic filter (with synthesis,
    # and its transpose) as split-bfloat16 tensor-core products, the rest in FP32
    return atoms_cube("atoms10k", seed, 10000, 110.0, [7.0], lambda r: 2.1, 0.4, 14.0,
                      precision="bf16x")


def scaled(base: str, n_atoms: int, seed: int = 77) -> Workload:
    """Same density and radii as ``base`` with ``n_atoms`` atoms (cube rescaled)."""
    ref = {"atoms64": (64, 30.0, [6.0], lambda r: 2.0, 0.25, 12.0, 0),
           "atoms1200": (1200, 60.0, [5.0, 6.0, 7.0, 8.0], lambda r: 0.3 * r, 0.195, 0.0, 1),
           "atoms10k": (10000, 110.0, [7.0], lambda r: 2.1, 0.4, 14.0, 0)}[base]
    n0, cube0, rc, fr, fh, cut, mode = ref
    cube = cube0 * (n_atoms / n0) ** (1.0 / 3.0)
    return atoms_cube("%s_n%d" % (base, n_atoms), seed, n_atoms, cube, rc, fr, fh, cut,
                      pair_mode=mode)


WORKLOADS = {"single_sf_24": single_sf_24, "atoms64": atoms64, "atoms1200": atoms1200,
             "atoms10k": atoms10k}


# ----------------------------------------------------------------- potential

def potential_block(wl: Workload, lo, shape, xp=np, device=None):
    """V on fine indices [lo, lo + shape) (x fastest in memory: array [z, y, x])."""
    h2 = wl.h / 2.0
    if xp is np:
        V = np.zeros(tuple(shape[::-1]))
    else:
        V = xp.zeros(tuple(shape[::-1]), dtype=xp.float64, device=device)
    for cx, cy, cz, D, w in wl.wells:
        cut = 6.0 * w
        sl = []
        e = []
        for d, c in enumerate((cx, cy, cz)):
            j0 = max(lo[d], int(math.floor((c - cut) / h2)))
            j1 = min(lo[d] + shape[d] - 1, int(math.ceil((c + cut) / h2)))
            if j1 < j0:
                break
            x = np.arange(j0, j1 + 1, dtype=np.float64) * h2
            ev = np.exp(-((x - c) ** 2) / (2.0 * w * w))
            e.append(ev if xp is np else xp.as_tensor(ev, device=device))
            sl.append(slice(j0 - lo[d], j1 + 1 - lo[d]))
        if len(sl) < 3:
            continue
        blk = (-D) * e[2][:, None, None] * e[1][None, :, None] * e[0][None, None, :]
        V[sl[2], sl[1], sl[0]] += blk
    return V


def potential_fast(wl: Workload, device, chunk=64):
    """The same V as ``potential`` (up to the order of the additions), built on a torch
    device with one scatter-add per chunk of wells instead of one per well."""
    import torch
    lo = np.asarray(wl.V_lo, np.int64)
    shape = np.asarray(wl.V_shape, np.int64)
    V = torch.zeros(int(np.prod(shape)), dtype=torch.float64, device=device)
    h2 = wl.h / 2.0
    wells = np.asarray(wl.wells, np.float64)
    wmax = float(wells[:, 4].max()) if len(wells) else 1.0
    W = int(math.ceil(2 * 6.0 * wmax / h2)) + 3               # padded block edge (fine points)
    ar = torch.arange(W, device=device, dtype=torch.int64)
    for c0 in range(0, len(wells), chunk):
        wc = torch.as_tensor(wells[c0:c0 + chunk], device=device)
        n = wc.shape[0]
        cut = 6.0 * wc[:, 4]
        E, I0 = [], []
        for d in range(3):
            j0 = torch.clamp(torch.floor((wc[:, d] - cut) / h2).to(torch.int64), min=int(lo[d]))
            j1 = torch.clamp(torch.ceil((wc[:, d] + cut) / h2).to(torch.int64), max=int(lo[d] + shape[d] - 1))
            j = j0[:, None] + ar[None, :]                      # (n, W) fine indices
            ok = j <= j1[:, None]
            x = j.to(torch.float64) * h2
            e = torch.exp(-((x - wc[:, d:d + 1]) ** 2) / (2.0 * wc[:, 4:5] ** 2))
            E.append(torch.where(ok, e, torch.zeros_like(e)))
            I0.append(torch.clamp(j - int(lo[d]), 0, int(shape[d] - 1)))
        blk = (-wc[:, 3])[:, None, None, None] * E[2][:, :, None, None] * E[1][:, None, :, None] \
            * E[0][:, None, None, :]
        idx = (I0[2][:, :, None, None] * shape[1] + I0[1][:, None, :, None]) * shape[0] + I0[0][:, None, None, :]
        V.index_add_(0, idx.reshape(-1), blk.reshape(-1))
    return V.reshape(int(shape[2]), int(shape[1]), int(shape[0]))


def potential(wl: Workload, xp=np, device=None):
    """V on the whole fine grid the method can touch, array [z, y, x] from index -14."""
    return potential_block(wl, wl.V_lo, wl.V_shape, xp, device)


# ----------------------------------------------------------------- support functions

def phi_values(wl: Workload, f: int, atom: int, g_coarse, g_fine, xp=np, device=None):
    """Compressed coefficients of function ``f`` (centred on ``atom``) given the grid
    indices of its coarse and fine members in layout order (s, then d^1..d^7)."""
    N = wl.N
    h = wl.h
    c = wl.pos[atom]

    def env(g):
        if xp is np:
            g = np.asarray(g, np.int64)
            x = (g % N[0]).astype(np.float64) * h - c[0]
            y = ((g // N[0]) % N[1]).astype(np.float64) * h - c[1]
            z = (g // (N[0] * N[1])).astype(np.float64) * h - c[2]
            return np.exp(-(x * x + y * y + z * z) / (2.0 * wl.sigma ** 2))
        x = (g % N[0]).to(xp.float64) * h - c[0]
        y = ((g // N[0]) % N[1]).to(xp.float64) * h - c[1]
        z = (g // (N[0] * N[1])).to(xp.float64) * h - c[2]
        return xp.exp(-(x * x + y * y + z * z) / (2.0 * wl.sigma ** 2))

    if xp is np:
        gc = np.asarray(g_coarse, np.int64)
        gf = np.asarray(g_fine, np.int64)
        parts = [counter_normal(wl.seed, f, 0, gc) * env(gc)]
        ef = env(gf)
        for t in range(1, 8):
            parts.append(counter_normal(wl.seed, f, t, gf) * ef)
        v = np.concatenate(parts)
        return v / np.sqrt(np.sum(v * v))
    gc = xp.as_tensor(g_coarse, dtype=xp.int64, device=device)
    gf = xp.as_tensor(g_fine, dtype=xp.int64, device=device)
    parts = [counter_normal(wl.seed, f, 0, gc, xp) * env(gc)]
    ef = env(gf)
    for t in range(1, 8):
        parts.append(counter_normal(wl.seed, f, t, gf, xp) * ef)
    v = xp.cat(parts)
    return v / xp.sqrt(xp.sum(v * v))


def fill_phi(wl: Workload, phi, off_L, sf_atom, coarse_g, fine_g, chunk_coefs=1 << 25, fn_ids=None):
    """Write every support function's compressed coefficients into the torch tensor
    ``phi`` (layout ``off_L``) in a few large vectorized passes, with the same values
    as ``phi_values`` for each function.  ``coarse_g[a]`` / ``fine_g[a]`` are the grid
    indices of atom a's coarse and fine members (layout order).  ``fn_ids`` (optional):
    the workload's function number of each entry (a sub-system's functions keep the
    content of their function in the whole system; ``sf_atom`` then holds the whole
    system's atoms)."""
    import torch
    dev = phi.device
    N = wl.N
    h = wl.h
    n_sf = len(sf_atom)
    nc = np.array([len(coarse_g[int(a)]) for a in sf_atom], dtype=np.int64)
    nf = np.array([len(fine_g[int(a)]) for a in sf_atom], dtype=np.int64)
    ncoef = nc + 7 * nf
    # per-atom concatenated g lists on the device
    atoms = sorted(set(int(a) for a in sf_atom))
    gc_off, gf_off = {}, {}
    gcs, gfs = [], []
    oc = of = 0
    for a in atoms:
        gc_off[a] = oc
        gf_off[a] = of
        gcs.append(np.asarray(coarse_g[a], np.int64))
        gfs.append(np.asarray(fine_g[a], np.int64))
        oc += len(gcs[-1])
        of += len(gfs[-1])
    GC = torch.as_tensor(np.concatenate(gcs), device=dev)
    GF = torch.as_tensor(np.concatenate(gfs) if of else np.zeros(0, np.int64), device=dev)
    pos = torch.as_tensor(np.asarray(wl.pos, np.float64), device=dev)
    f = 0
    while f < n_sf:
        f1 = f
        tot = 0
        while f1 < n_sf and (f1 == f or tot + ncoef[f1] <= chunk_coefs):
            tot += ncoef[f1]
            f1 += 1
        fs = np.arange(f, f1)
        cnt = torch.as_tensor(ncoef[fs], device=dev)
        fid = torch.repeat_interleave(torch.as_tensor(fs, device=dev), cnt)        # function of each coef
        start = torch.cumsum(cnt, 0) - cnt
        k = torch.arange(int(tot), device=dev) - torch.repeat_interleave(start, cnt)  # index within function
        ncf = torch.as_tensor(nc[fs], device=dev)
        nff = torch.as_tensor(nf[fs], device=dev)
        ncr = torch.repeat_interleave(ncf, cnt)
        nfr = torch.repeat_interleave(nff, cnt)
        is_c = k < ncr
        kf = torch.where(is_c, torch.zeros_like(k), k - ncr)
        t = torch.where(is_c, torch.zeros_like(k), kf // torch.clamp(nfr, min=1) + 1)
        j = torch.where(is_c, k, kf - (t - 1) * nfr)
        atom = torch.as_tensor(np.asarray(sf_atom)[fs], device=dev)
        atom_r = torch.repeat_interleave(atom, cnt)
        oc_a = torch.as_tensor(np.array([gc_off[int(a)] for a in np.asarray(sf_atom)[fs]]), device=dev)
        of_a = torch.as_tensor(np.array([gf_off[int(a)] for a in np.asarray(sf_atom)[fs]]), device=dev)
        gidx = torch.where(is_c, torch.repeat_interleave(oc_a, cnt) + j, torch.repeat_interleave(of_a, cnt) + j)
        g = torch.where(is_c, GC[torch.clamp(gidx, max=max(0, GC.numel() - 1))],
                        GF[torch.clamp(gidx, max=max(0, GF.numel() - 1))] if GF.numel() else torch.zeros_like(gidx))
        fg_ = fid if fn_ids is None else torch.as_tensor(np.asarray(fn_ids, np.int64), device=dev)[fid]
        z = counter_normal(wl.seed, fg_, t, g, xp=torch)
        c = pos[atom_r]
        x = (g % N[0]).to(torch.float64) * h - c[:, 0]
        y = ((g // N[0]) % N[1]).to(torch.float64) * h - c[:, 1]
        zz = (g // (N[0] * N[1])).to(torch.float64) * h - c[:, 2]
        v = z * torch.exp(-(x * x + y * y + zz * zz) / (2.0 * wl.sigma ** 2))
        nrm = torch.zeros(len(fs), dtype=torch.float64, device=dev).index_add_(0, fid - f, v * v)
        v = v / torch.sqrt(nrm)[fid - f]
        dest = torch.as_tensor(np.asarray(off_L)[fs], device=dev)
        phi[torch.repeat_interleave(dest, cnt) + k] = v.to(phi.dtype)
        f = f1


# ----------------------------------------------------------------- density kernel

def density_kernel(wl: Workload, sf_atom, row_ptr, col, scale: float = 3.0):
    """Seeded symmetric density kernel K on a CSR pattern (values in pattern order).

    K_ab = (0.5 + xi) exp(-|R_A - R_B|^2 / (2 scale^2)), A, B the atoms of a and b, with
    xi ~ U[0, 1) drawn once per unordered pair {a, b}: K_ab = K_ba whenever both entries
    are stored.  A stand-in for a converged kernel: positive, decaying with distance."""
    sf_atom = np.asarray(sf_atom, np.int64)
    row_ptr = np.asarray(row_ptr, np.int64)
    col = np.asarray(col, np.int64)
    n = len(row_ptr) - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(row_ptr))
    lo = np.minimum(rows, col)
    hi = np.maximum(rows, col)
    key = lo * n + hi
    k = mix32(mix32((key & _M32) ^ (0x5BD1E995 & _M32)) ^ ((key >> 32) & _M32) ^ (wl.seed & _M32))
    xi = (k.astype(np.float64) + 0.5) / 4294967296.0
    pos = np.asarray(wl.pos, np.float64)
    d = pos[sf_atom[rows]] - pos[sf_atom[col]]
    d2 = np.sum(d * d, axis=1)
    return (0.5 + xi) * np.exp(-d2 / (2.0 * scale * scale))
