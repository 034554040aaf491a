"""The C-ABI library without a GPU: it loads, exports every declared symbol, and its
host-side filter derivation, locreg keys, layout and pattern equal the oracle's
bit for bit (independent implementations of Sec. II.B, Eq. loccon, Sec. III.B)."""
import os
import re

import numpy as np
import pytest

from oracle import filters as F
from oracle import geometry as G
from paper_1401_7441_gb300 import inputs as I
from paper_1401_7441_gb300 import lsw
from tests.lib_support import ensure_built, host_system
from tests.oracle_support import desc_of

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def ctx():
    ensure_built()
    c = lsw.lsw_ctx_create(lsw.LSW_HOST_ONLY)
    yield c
    lsw.lsw_ctx_destroy(c)


def declared_symbols():
    txt = open(os.path.join(ROOT, "include", "lsw.h")).read()
    return sorted(set(re.findall(r"^\S.*?\b(lsw_[a-z_]+)\s*\(", txt, flags=re.M)))


def test_library_exports_every_declared_symbol():
    lib = ensure_built()
    names = declared_symbols()
    assert len(names) >= 16
    for n in names:
        assert hasattr(lib, n), n


def test_filters_equal_oracle_table(ctx):
    tab = F.read_table()
    for name in ("h", "g", "moments", "magic", "kin_r", "kin_hh", "kin_hg", "kin_gh", "kin_gg"):
        lo, vals = lsw.lsw_filter_table(ctx, name)
        assert lo == tab[name][0]
        assert np.array_equal(vals, tab[name][1]), name
    # moment overlaps of the confinement: the library's double-double solve against the
    # oracle's 50-digit one, each rounded once to FP64
    for p in range(5):
        lo, vals = lsw.lsw_filter_table(ctx, "movl_%d" % p)
        ref = tab["movl_%d" % p]
        assert lo == ref[0]
        assert np.max(np.abs(vals - ref[1])) <= 2e-16 * max(1.0, np.max(np.abs(ref[1]))), p


def test_forward_filters_are_the_convolution(ctx):
    ft = F.load()
    for key, X in (("fwd_h", ft.h), ("fwd_g", ft.g)):
        lo, v = lsw.lsw_filter_table(ctx, key)
        ref = np.convolve(ft.magic, X)
        assert lo == -14 and np.max(np.abs(v - ref)) < 4e-16  # FP64 convolution rounding


@pytest.mark.parametrize("name,kw", [("atoms64", {}), ("atoms64", {"fine_mode": "own"}),
                                     ("atoms64", {"lprime_margin": 3.0}),
                                     ("single_sf_24", {}), ("atoms1200_small", {})])
def test_keys_layout_pattern_bit_exact(ctx, name, kw):
    wl = I.scaled("atoms1200", 90, seed=11) if name == "atoms1200_small" else I.WORKLOADS[name]()
    if "fine_mode" in kw:
        wl.fine_mode = kw["fine_mode"]
    if "lprime_margin" in kw:
        wl.lprime_margin = kw["lprime_margin"]
    S = host_system(wl, ctx, fine_mode=wl.fine_mode, lprime_margin=wl.lprime_margin)
    geo = G.build(desc_of(wl))
    try:
        for a in range(len(wl.pos)):
            for reg, locs in ((lsw.LSW_REGION_L, geo.L), (lsw.LSW_REGION_LP, geo.Lp)):
                assert np.array_equal(S.keys(a, reg, lsw.LSW_PART_COARSE), locs[a].coarse.keys)
                assert np.array_equal(S.keys(a, reg, lsw.LSW_PART_FINE), locs[a].fine.keys)
        assert np.array_equal(S.off_L, geo.off_L)
        assert np.array_equal(S.off_Lp, geo.off_Lp)
        assert np.array_equal(S.row_ptr, geo.row_ptr)
        assert np.array_equal(S.col, geo.col)
        assert np.array_equal(S.sf_atom, geo.sf_atom)
    finally:
        S.close()


def test_argument_errors(ctx):
    wl = I.single_sf_24()
    with pytest.raises(lsw.LswError) as e:
        lsw.System((0, 4, 4), wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, 1.0, ctx=ctx)
    assert e.value.status == lsw.LSW_ERR_ARG
    with pytest.raises(lsw.LswError):
        lsw.System(wl.N, -1.0, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, 1.0, ctx=ctx)
    with pytest.raises(lsw.LswError):
        lsw.System(wl.N, wl.h, wl.pos, np.array([0.0]), wl.r_fine, wl.nsf, 1.0, ctx=ctx)
    with pytest.raises(lsw.LswError):
        lsw.lsw_filter_table(ctx, 99)
    S = host_system(wl, ctx)
    try:
        with pytest.raises(lsw.LswError) as e:
            lsw.lsw_system_keys(S.sys, 5, 0, 0)
        assert e.value.status == lsw.LSW_ERR_ARG
        with pytest.raises(lsw.LswError) as e:
            lsw.lsw_apply_hamiltonian(S.sys, 16, 32)
        assert e.value.status == lsw.LSW_ERR_STATE   # host-only context: no device work
        with pytest.raises(lsw.LswError) as e:
            lsw.lsw_build_density(S.sys, 16, 32, 48, wl.V_lo, wl.V_shape)
        assert e.value.status == lsw.LSW_ERR_STATE
        with pytest.raises(lsw.LswError):
            lsw.lsw_set_option(S.sys, "nonsense", 1)
    finally:
        S.close()


def test_atom_without_functions_and_empty_rows(ctx):
    wl = I.scaled("atoms64", 10, seed=4)
    wl.nsf[3] = 0
    S = host_system(wl, ctx)
    geo = G.build(desc_of(wl))
    try:
        assert S.n_sf == int(wl.nsf.sum())
        assert np.array_equal(S.row_ptr, geo.row_ptr) and np.array_equal(S.col, geo.col)
    finally:
        S.close()


def test_checkpoint_description_roundtrip(ctx, tmp_path):
    # lsw_save without support functions writes the description; lsw_load rebuilds a
    # system with the same keys, layout and pattern (same host arithmetic).
    wl = I.scaled("atoms64", 9, seed=3)
    S = host_system(wl, ctx, precision=lsw.LSW_FP32_BF16X)
    path = str(tmp_path / "sys.lsw")
    try:
        lsw.lsw_save(S.sys, None, path)
        T = lsw.lsw_load(ctx, path)
        try:
            lay_s = lsw.lsw_system_layout(S.sys)
            lay_t = lsw.lsw_system_layout(T)
            for x, y in zip(lay_s, lay_t):
                assert np.array_equal(np.asarray(x), np.asarray(y))
            rs, cs = lsw.lsw_pattern(S.sys)
            rt, ct = lsw.lsw_pattern(T)
            assert np.array_equal(rs, rt) and np.array_equal(cs, ct)
            for a in range(len(wl.pos)):
                for region in (lsw.LSW_REGION_L, lsw.LSW_REGION_LP):
                    for part in (lsw.LSW_PART_COARSE, lsw.LSW_PART_FINE):
                        assert np.array_equal(lsw.lsw_system_keys(S.sys, a, region, part),
                                              lsw.lsw_system_keys(T, a, region, part))
            with pytest.raises(lsw.LswError) as e:
                lsw.lsw_load_phi(T, path, 64)               # no support functions saved
            assert e.value.status == lsw.LSW_ERR_STATE
        finally:
            lsw.lsw_system_destroy(T)
    finally:
        S.close()
    bad = tmp_path / "bad.lsw"
    bad.write_bytes(b"not a checkpoint")
    with pytest.raises(lsw.LswError) as e:
        lsw.lsw_load(ctx, str(bad))
    assert e.value.status == lsw.LSW_ERR_IO
    with pytest.raises(lsw.LswError) as e:
        lsw.lsw_load(ctx, str(tmp_path / "missing.lsw"))
    assert e.value.status == lsw.LSW_ERR_IO


def test_confinement_rows_equal_oracle_blocks(ctx):
    # the library's 1D operator entries of (x - R)^m (m = 2, 4) between scaling and
    # wavelet functions, from its own moment overlaps, against the oracle's blocks
    from oracle import confinement as Q
    wl = I.scaled("atoms64", 4, seed=3)
    S = host_system(wl, ctx)
    ft = F.load()
    cols = np.arange(-4, 60)
    for atom in range(2):
        for dim in range(3):
            c = wl.pos[atom][dim] / wl.h
            for m in (2, 4):
                for b in (0, 1):
                    for bp in (0, 1):
                        idx = np.arange(10, 40, 3)
                        ref = Q.quartic_block_1d(m, b, bp, idx, cols, c, wl.h, ft)
                        for ii, i in enumerate(idx):
                            row = lsw.lsw_confinement_row(S.sys, atom, dim, m, b, bp, int(i))
                            r2 = ref[ii, np.searchsorted(cols, i + np.arange(-14, 15))]
                            assert np.max(np.abs(row - r2)) <= 1e-13 * np.max(np.abs(r2)), (atom, dim, m, b, bp, i)
    S.close()
