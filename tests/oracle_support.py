"""Test helpers: turn a seeded workload into oracle inputs (no method arithmetic here)."""
import numpy as np

from oracle import geometry as G
from paper_1401_7441_gb300 import inputs as I


def desc_of(wl: I.Workload, **kw) -> G.SystemDesc:
    d = dict(N=tuple(wl.N), h=wl.h, pos=np.asarray(wl.pos, np.float64),
             r_loc=np.asarray(wl.r_loc, np.float64), r_fine=np.asarray(wl.r_fine, np.float64),
             nsf=np.asarray(wl.nsf, np.int64), pair_cutoff=float(wl.pair_cutoff),
             pair_mode=int(wl.pair_mode), lprime_margin=float(wl.lprime_margin),
             fine_mode=wl.fine_mode)
    d.update(kw)
    return G.SystemDesc(**d)


def phi_all(wl, geo, fs=None):
    fs = range(len(geo.sf_atom)) if fs is None else fs
    out = {}
    for f in fs:
        a = geo.sf_atom[f]
        out[f] = I.phi_values(wl, f, a, geo.L[a].coarse.g, geo.L[a].fine.g)
    return out


def tiny_workload(n=7, seed=5, n_atoms=2, r_loc=1.3, r_fine=0.7, margin=8.0, h=0.45):
    """A small box with a few atoms at seeded off-grid positions."""
    u = I.uniform(seed, 9, 3 * n_atoms + 2 * n_atoms).reshape(-1)
    pos = (1.0 + u[:3 * n_atoms].reshape(n_atoms, 3) * (n - 3)) * h
    wells = np.column_stack([pos, 1.0 + 2.0 * u[3 * n_atoms:4 * n_atoms],
                             0.5 + u[4 * n_atoms:5 * n_atoms]])
    return I.Workload("tiny", (n, n, n), h, pos, np.full(n_atoms, r_loc),
                      np.full(n_atoms, r_fine), np.ones(n_atoms, np.int64), 100.0, 0,
                      wells, seed, lprime_margin=margin)
