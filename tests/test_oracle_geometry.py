"""Pins of the oracle's locreg geometry, keys, layout and pattern against brute force
(Sec. II.B regions; Sec. III Eq. loccon; Sec. III.B L'; Sec. II.A pattern)."""
import numpy as np
import pytest

from oracle import geometry as G
from paper_1401_7441_gb300 import inputs as I
from tests.oracle_support import desc_of, tiny_workload


def brute_members(N, h, c, R):
    """Every box point tested one by one with Python floats (IEEE, never fused)."""
    out = []
    R2 = R * R
    for k in range(N[2]):
        for j in range(N[1]):
            for i in range(N[0]):
                dx, dy, dz = i * h - c[0], j * h - c[1], k * h - c[2]
                if (dx * dx + dy * dy) + dz * dz <= R2:
                    out.append(i + N[0] * (j + N[1] * k))
    return np.array(out, dtype=np.int64)


def test_single_function_box_counts():
    wl = I.single_sf_24()
    geo = G.build(desc_of(wl))
    L = geo.L[0]
    assert len(L.coarse.g) == 24 ** 3          # every point carries a scaling function
    assert len(L.fine.g) == 925                # lattice points with i^2+j^2+k^2 <= 36
    assert L.n_coef == 24 ** 3 + 7 * 925
    cnt = sum(1 for a in range(-6, 7) for b in range(-6, 7) for c in range(-6, 7)
              if a * a + b * b + c * c <= 36)
    assert cnt == 925


@pytest.mark.parametrize("seed", [3, 4, 5])
def test_membership_and_keys_brute_force(seed):
    wl = tiny_workload(n=11, seed=seed, n_atoms=3, r_loc=1.6, r_fine=0.8)
    d = desc_of(wl)
    geo = G.build(d)
    N = d.N
    fine = np.zeros(N[0] * N[1] * N[2], dtype=bool)
    for a in range(len(d.pos)):
        fine[brute_members(N, d.h, d.pos[a], d.r_fine[a])] = True
    for a in range(len(d.pos)):
        for loc, R in ((geo.L[a], d.r_loc[a]), (geo.Lp[a], d.r_loc[a] + 8.0 * d.h)):
            gc = brute_members(N, d.h, d.pos[a], R)
            assert np.array_equal(loc.coarse.g, gc)
            assert np.array_equal(loc.fine.g, gc[fine[gc]])
            for reg in (loc.coarse, loc.fine):
                # segments: maximal runs along i1, cover exactly the member set
                cover = []
                for s, e, off in reg.keys:
                    assert e // N[0] == s // N[0] and e >= s
                    assert off == len(cover)
                    cover += list(range(s, e + 1))
                assert np.array_equal(np.array(cover, dtype=np.int64), reg.g)
                for (s0, e0, _), (s1, e1, _) in zip(reg.keys[:-1], reg.keys[1:]):
                    assert s1 > e0 + 1 or s1 // N[0] != e0 // N[0]


def test_clipped_locreg_at_box_corner():
    wl = tiny_workload(n=9, seed=2, n_atoms=1, r_loc=2.0, r_fine=0.9)
    wl.pos[:] = [[0.1, 0.2, 0.05]]
    geo = G.build(desc_of(wl))
    L = geo.L[0]
    assert L.lo.tolist() == [0, 0, 0]
    ref = brute_members(wl.N, wl.h, wl.pos[0], 2.0)
    assert np.array_equal(L.coarse.g, ref)


def test_layout_alignment():
    wl = I.atoms64()
    geo = G.build(desc_of(wl))
    off = geo.off_L
    assert off[0] == 0 and np.all(off % 64 == 0)
    n = np.array([geo.L[a].n_coef for a in geo.sf_atom])
    assert np.all(off[1:] - off[:-1] >= n) and np.all(off[1:] - off[:-1] < n + 64)
    assert len(geo.sf_atom) == 208


def test_pattern_brute_force():
    wl = I.atoms64()
    d = desc_of(wl)
    geo = G.build(d)
    nsf = d.nsf
    atom = np.repeat(np.arange(len(nsf)), nsf)
    nnz = 0
    for a in range(len(atom)):
        cols = []
        for b in range(len(atom)):
            p, q = d.pos[atom[a]], d.pos[atom[b]]
            dx, dy, dz = p[0] - q[0], p[1] - q[1], p[2] - q[2]
            if (dx * dx + dy * dy) + dz * dz <= d.pair_cutoff * d.pair_cutoff:
                cols.append(b)
        assert geo.col[geo.row_ptr[a]:geo.row_ptr[a + 1]].tolist() == cols
        nnz += len(cols)
    assert nnz == geo.row_ptr[-1]


def test_pattern_sum_of_radii_mode():
    wl = I.scaled("atoms1200", 60)
    d = desc_of(wl)
    geo = G.build(d, pattern=True)
    atom = np.repeat(np.arange(len(d.nsf)), d.nsf)
    for a in range(0, len(atom), 7):
        cols = []
        for b in range(len(atom)):
            p, q = d.pos[atom[a]], d.pos[atom[b]]
            c = d.r_loc[atom[a]] + d.r_loc[atom[b]]
            dx, dy, dz = p[0] - q[0], p[1] - q[1], p[2] - q[2]
            if (dx * dx + dy * dy) + dz * dz <= c * c:
                cols.append(b)
        assert geo.col[geo.row_ptr[a]:geo.row_ptr[a + 1]].tolist() == cols
