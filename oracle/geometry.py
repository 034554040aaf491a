"""Grid, fine region, localization regions L and L', segment keys, compressed layout
and pair pattern (oracle).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Paper: Sec. II.B (coarse/fine/empty regions; rectangular box with its origin at a
corner, positive grid coordinates), Sec. III Eq. loccon (the projector L^(alpha) keeps
the basis functions centred within R_cut of R_alpha), Sec. III.B (L' with
R'_cut = R_cut + 8 grid points), Sec. II.A (H_ab, S_ab sparse with the overlap pattern).

Readings taken where the paper is silent:

* coarse point (i1, i2, i3) sits at (i1 h, i2 h, i3 h); 0 <= i_d < N_d (free boundary).
* membership is inclusive, d^2 <= R^2, with d^2 evaluated in FP64 as
  ((x-X)*(x-X) + (y-Y)*(y-Y)) + (z-Z)*(z-Z), x = i*h, each operation rounded once
  (numpy evaluates these element-wise, never fused).
* fine region = union over atoms of their fine spheres (default, "union"); the
  alternative "own" keeps only the locreg's own atom's fine sphere.
* L' radius R + margin*h with margin = 8 (Sec. III.B); its fine points are the fine
  region's points inside L'.
* a segment is a maximal run of members along i1 at fixed (i2, i3); segments are
  sorted by g = i1 + N1 (i2 + N2 i3); key = (start g, end g inclusive, coefficient
  offset).  Compressed vector of one function: s over coarse members in key order,
  then 7 planes d^1..d^7 over fine members in key order.
* functions are numbered atom by atom; function f starts at element offset off[f],
  off[f+1] = off[f] + ceil(N_coef(f) / 64) * 64.
* pattern: (a, b) is kept iff the distance between their atoms' centres is <= cutoff
  (same FP64 arithmetic; cutoff fixed, or r_a + r_b in pair mode 1); rows a,
  columns b ascending; a = b included.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ALIGN = 64


@dataclass
class SystemDesc:
    N: tuple              # (N1, N2, N3) coarse grid points
    h: float              # grid spacing (bohr)
    pos: np.ndarray       # (n_atoms, 3) bohr, box coordinates
    r_loc: np.ndarray     # (n_atoms,) locreg radius R_cut (bohr)
    r_fine: np.ndarray    # (n_atoms,) fine-sphere radius (bohr)
    nsf: np.ndarray       # (n_atoms,) support functions per atom
    pair_cutoff: float    # bohr
    pair_mode: int = 0    # 0: fixed cutoff; 1: cutoff = r_loc(a) + r_loc(b)
    lprime_margin: float = 8.0   # grid points
    fine_mode: str = "union"     # "union" | "own"


@dataclass
class Region:
    """Member set of one region (coarse or fine part) with its keys."""
    g: np.ndarray          # int64 global indices, ascending (= key order)
    keys: np.ndarray       # (nseg, 3) int64: start g, end g (inclusive), coefficient offset


@dataclass
class Locreg:
    coarse: Region
    fine: Region
    lo: np.ndarray         # bounding box of the coarse members (inclusive)
    hi: np.ndarray

    @property
    def n_coef(self) -> int:
        return len(self.coarse.g) + 7 * len(self.fine.g)


@dataclass
class Geometry:
    desc: SystemDesc
    fine_mask: np.ndarray          # bool (N1, N2, N3), indexed [i1, i2, i3]
    L: list                        # per atom
    Lp: list                       # per atom
    sf_atom: np.ndarray            # function -> atom
    off_L: np.ndarray              # (n_sf + 1,) element offsets
    off_Lp: np.ndarray
    row_ptr: np.ndarray = field(default=None)
    col: np.ndarray = field(default=None)


def dist2(px, py, pz, X, Y, Z):
    """((x-X)*(x-X) + (y-Y)*(y-Y)) + (z-Z)*(z-Z), every step rounded once in FP64."""
    dx = np.subtract(px, X)
    dy = np.subtract(py, Y)
    dz = np.subtract(pz, Z)
    return np.add(np.add(np.multiply(dx, dx), np.multiply(dy, dy)), np.multiply(dz, dz))


def sphere_points(N, h, c, R):
    """Coarse points of the box with dist2 <= R*R (Eq. loccon, inclusive).

    Returns a bool array over the bounding block [lo, hi] (inclusive) and lo."""
    h = float(h)
    R = float(R)
    lo = np.zeros(3, dtype=np.int64)
    hi = np.zeros(3, dtype=np.int64)
    for d in range(3):
        lo[d] = max(0, int(np.floor((c[d] - R) / h)) - 1)
        hi[d] = min(N[d] - 1, int(np.ceil((c[d] + R) / h)) + 1)
    if np.any(hi < lo):
        return np.zeros((0, 0, 0), dtype=bool), lo
    ax = [np.arange(lo[d], hi[d] + 1, dtype=np.int64) * h for d in range(3)]
    x = ax[0][:, None, None]
    y = ax[1][None, :, None]
    z = ax[2][None, None, :]
    d2 = dist2(x, y, z, c[0], c[1], c[2])
    return d2 <= np.multiply(R, R), lo


def fine_region(desc: SystemDesc) -> np.ndarray:
    """Global fine region: union of the atoms' fine spheres inside the box (Sec. II.B)."""
    N = desc.N
    mask = np.zeros(N, dtype=bool)
    for a in range(len(desc.pos)):
        blk, lo = sphere_points(N, desc.h, desc.pos[a], desc.r_fine[a])
        if blk.size:
            s = blk.shape
            mask[lo[0]:lo[0] + s[0], lo[1]:lo[1] + s[1], lo[2]:lo[2] + s[2]] |= blk
    return mask


def gindex(N, i1, i2, i3):
    return np.asarray(i1, np.int64) + N[0] * (np.asarray(i2, np.int64) + N[1] * np.asarray(i3, np.int64))


def gcoords(N, g):
    g = np.asarray(g, np.int64)
    i1 = g % N[0]
    i2 = (g // N[0]) % N[1]
    i3 = g // (N[0] * N[1])
    return i1, i2, i3


def make_keys(N, g_sorted: np.ndarray) -> np.ndarray:
    """Segments = maximal runs of consecutive i1 at fixed (i2, i3) (reading A9)."""
    if len(g_sorted) == 0:
        return np.zeros((0, 3), dtype=np.int64)
    g = g_sorted
    i1 = g % N[0]
    row = g // N[0]
    brk = np.ones(len(g), dtype=bool)
    brk[1:] = (row[1:] != row[:-1]) | (i1[1:] != i1[:-1] + 1)
    starts = np.nonzero(brk)[0]
    ends = np.append(starts[1:], len(g)) - 1
    return np.stack([g[starts], g[ends], starts.astype(np.int64)], axis=1)


def _region_from_block(N, blk, lo) -> np.ndarray:
    idx = np.nonzero(blk)
    g = gindex(N, idx[0] + lo[0], idx[1] + lo[1], idx[2] + lo[2])
    return np.sort(g)


def make_locreg(desc: SystemDesc, fine_mask, a: int, R: float) -> Locreg:
    N = desc.N
    blk, lo = sphere_points(N, desc.h, desc.pos[a], R)
    gc = _region_from_block(N, blk, lo)
    i1, i2, i3 = gcoords(N, gc)
    if desc.fine_mode == "union":
        gf = gc[fine_mask[i1, i2, i3]]
    elif desc.fine_mode == "own":
        fblk, flo = sphere_points(N, desc.h, desc.pos[a], desc.r_fine[a])
        own = _region_from_block(N, fblk, flo)
        gf = np.intersect1d(gc, own, assume_unique=True)
    else:
        raise ValueError(desc.fine_mode)
    if len(gc):
        blo = np.array([i1.min(), i2.min(), i3.min()])
        bhi = np.array([i1.max(), i2.max(), i3.max()])
    else:
        blo = np.zeros(3, np.int64)
        bhi = -np.ones(3, np.int64)
    return Locreg(Region(gc, make_keys(N, gc)), Region(gf, make_keys(N, gf)), blo, bhi)


def lprime_radius(desc: SystemDesc, a: int) -> float:
    """R' = R_cut + margin * h (Sec. III.B), FP64: r + (margin * h)."""
    return float(np.add(desc.r_loc[a], np.multiply(desc.lprime_margin, desc.h)))


def layout(n_coef: np.ndarray) -> np.ndarray:
    off = np.zeros(len(n_coef) + 1, dtype=np.int64)
    off[1:] = np.cumsum((np.asarray(n_coef, np.int64) + ALIGN - 1) // ALIGN * ALIGN)
    return off


def pair_pattern(desc: SystemDesc, sf_atom: np.ndarray):
    """CSR of the pairs (a, b) with |R_atom(a) - R_atom(b)| <= cutoff (Sec. II.A)."""
    pos = np.asarray(desc.pos, np.float64)
    nat = len(pos)
    first = np.zeros(nat + 1, dtype=np.int64)
    first[1:] = np.cumsum(desc.nsf)
    nb = []
    for a in range(nat):
        d2 = dist2(pos[:, 0], pos[:, 1], pos[:, 2], pos[a, 0], pos[a, 1], pos[a, 2])
        if desc.pair_mode == 1:
            c = np.add(np.asarray(desc.r_loc, np.float64), desc.r_loc[a])
        else:
            c = np.float64(desc.pair_cutoff)
        nb.append(np.nonzero(d2 <= np.multiply(c, c))[0])
    rows = []
    for f in range(len(sf_atom)):
        a = sf_atom[f]
        cols = np.concatenate([np.arange(first[b], first[b + 1]) for b in nb[a]])
        rows.append(np.sort(cols))
    row_ptr = np.zeros(len(rows) + 1, dtype=np.int64)
    row_ptr[1:] = np.cumsum([len(r) for r in rows])
    col = np.concatenate(rows).astype(np.int32) if rows else np.zeros(0, np.int32)
    return row_ptr, col


def build(desc: SystemDesc, atoms=None, pattern: bool = True) -> Geometry:
    """Locregs of every atom (or of the listed atoms only) plus layout and pattern."""
    fm = fine_region(desc)
    nat = len(desc.pos)
    want = range(nat) if atoms is None else sorted(set(int(a) for a in atoms))
    L = [None] * nat
    Lp = [None] * nat
    for a in want:
        L[a] = make_locreg(desc, fm, a, float(desc.r_loc[a]))
        Lp[a] = make_locreg(desc, fm, a, lprime_radius(desc, a))
    sf_atom = np.repeat(np.arange(nat), desc.nsf)
    geo = Geometry(desc, fm, L, Lp, sf_atom, None, None)
    if atoms is None:
        geo.off_L = layout([L[a].n_coef for a in sf_atom])
        geo.off_Lp = layout([Lp[a].n_coef for a in sf_atom])
    if pattern:
        geo.row_ptr, geo.col = pair_pattern(desc, sf_atom)
    return geo
