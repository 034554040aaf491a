"""Pins of the oracle's support-function reuse (integer grid shifts; section "Geometry
optimization" of the paper): identity, lattice-translation covariance of H phi."""
import numpy as np

from oracle import geometry as G
from oracle import hamiltonian as Hm
from oracle import reformat as R
from paper_1401_7441_gb300 import inputs as I
from tests.oracle_support import desc_of


def _shifted(wl, shift_pts):
    import copy
    w2 = copy.deepcopy(wl)
    w2.pos = wl.pos + np.asarray(shift_pts, float)[None, :] * wl.h
    w2.wells = wl.wells.copy()
    w2.wells[:, :3] += np.asarray(shift_pts, float)[None, :] * wl.h
    return w2


def test_zero_shift_is_identity():
    wl = I.scaled("atoms64", 6, seed=2)
    geo = G.build(desc_of(wl))
    for f in range(len(geo.sf_atom)):
        a = geo.sf_atom[f]
        phi = I.phi_values(wl, f, a, geo.L[a].coarse.g, geo.L[a].fine.g)
        out = R.reformat(geo, geo, np.zeros((len(wl.pos), 3), int), f, phi)
        assert np.array_equal(out, phi)


def test_lattice_translation_moves_values_and_commutes_with_H():
    # translate every atom and well by whole grid points: the reused functions are the
    # old ones moved, and H phi on the new geometry is the old H phi moved (to rounding)
    wl = I.scaled("atoms64", 5, seed=7)
    sh = (2, -1, 1)
    w2 = _shifted(wl, sh)
    g1 = G.build(desc_of(wl))
    g2 = G.build(desc_of(w2))
    V1 = I.potential(wl)
    V2 = I.potential(w2)
    shift = np.tile(np.array(sh), (len(wl.pos), 1))
    for f in range(len(g1.sf_atom)):
        a = g1.sf_atom[f]
        # nothing is clipped by the box here, so membership moves exactly
        assert len(g1.L[a].coarse.g) == len(g2.L[a].coarse.g)
        phi1 = I.phi_values(wl, f, a, g1.L[a].coarse.g, g1.L[a].fine.g)
        phi2 = R.reformat(g2, g1, shift, f, phi1)
        assert np.array_equal(phi2, phi1)               # same key order after a translation
        h1, ek1, ep1 = Hm.apply_hamiltonian(g1, f, phi1, V1, wl.V_lo)
        h2, ek2, ep2 = Hm.apply_hamiltonian(g2, f, phi2, V2, w2.V_lo)
        # L' may be clipped differently by the box: compare H phi on the points of L
        # (inside the box in both geometries), s part and the 7 wavelet parts
        for part in ("coarse", "fine"):
            r1, r2 = getattr(g1.Lp[a], part), getattr(g2.Lp[a], part)
            p1 = {int(g): k for k, g in enumerate(r1.g)}
            p2 = {int(g): k for k, g in enumerate(r2.g)}
            pts = getattr(g1.L[a], part).g
            i1, i2, i3 = G.gcoords(wl.N, pts)
            moved = G.gindex(wl.N, i1 + sh[0], i2 + sh[1], i3 + sh[2])
            k1 = np.array([p1[int(g)] for g in pts])
            k2 = np.array([p2[int(g)] for g in moved])
            n1, n2 = len(g1.Lp[a].coarse.g), len(g2.Lp[a].coarse.g)
            planes = [0] if part == "coarse" else range(7)
            for t in planes:
                if part == "coarse":
                    v1, v2 = h1[k1], h2[k2]
                else:
                    f1, f2 = len(r1.g), len(r2.g)
                    v1, v2 = h1[n1 + t * f1 + k1], h2[n2 + t * f2 + k2]
                assert np.max(np.abs(v2 - v1)) <= 1e-12 * np.max(np.abs(h1))
        assert abs(ek2 - ek1) <= 1e-12 * abs(ek1) and abs(ep2 - ep1) <= 1e-11 * abs(ek1)


def test_partial_overlap_drops_and_zero_fills():
    wl = I.scaled("atoms64", 4, seed=3)
    g1 = G.build(desc_of(wl))
    shift = np.zeros((len(wl.pos), 3), int)
    shift[0] = (3, 0, 0)                                 # atom 0 moves by 3 grid points
    f = 0
    a = g1.sf_atom[f]
    phi = I.phi_values(wl, f, a, g1.L[a].coarse.g, g1.L[a].fine.g)
    out = R.reformat(g1, g1, shift, f, phi)             # same locreg, shifted content
    nc = len(g1.L[a].coarse.g)
    i1, i2, i3 = G.gcoords(wl.N, g1.L[a].coarse.g)
    src = G.gindex(wl.N, i1 - 3, i2, i3)
    pos = {int(g): k for k, g in enumerate(g1.L[a].coarse.g)}
    for k in range(nc):
        j = pos.get(int(src[k]), -1)
        assert out[k] == (phi[j] if j >= 0 else 0.0)
