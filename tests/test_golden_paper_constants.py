"""The values the paper prints for the operators on this path (tests/golden/
paper_constants.txt, each line citing its passage) against the oracle and the library."""
import inspect
import os

import numpy as np

from oracle import filters as F
from oracle import geometry as G
from paper_1401_7441_gb300 import inputs as I
from paper_1401_7441_gb300 import lsw
from paper_1401_7441_gb300 import shard
from tests.lib_support import ensure_built

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_constants.txt")


def _constants():
    out = {}
    for ln in open(GOLDEN):
        ln = ln.split("#", 1)[0].strip()
        if ln:
            k, *v = ln.split()
            out[k] = v
    return out


def test_filter_order_support_and_exactness():
    c = _constants()
    FT = F.load()
    order = int(c["filter_order"][0])
    lo, hi = (int(x) for x in c["support"])
    m = order // 2
    assert (lo, hi) == (1 - m, m)
    assert len(FT.h) == order and len(FT.g) == order and FT.h_lo == lo
    # exact representation of polynomials of degree < m: the wavelet has m vanishing moments
    j = np.arange(lo, hi + 1)
    for p in range(int(c["polynomial_order"][0])):
        t = (j.astype(float) ** p) * FT.g
        assert abs(t.sum()) <= 1e-13 * np.abs(t).sum()
    ensure_built()
    ctx = lsw.lsw_ctx_create(lsw.LSW_HOST_ONLY)
    try:
        first, vals = lsw.lsw_filter_table(ctx, "h")
        assert first == lo and len(vals) == order
    finally:
        lsw.lsw_ctx_destroy(ctx)


def test_lprime_margin_and_types():
    c = _constants()
    assert float(c["lprime_margin"][0]) == G.SystemDesc.__dataclass_fields__["lprime_margin"].default
    assert float(c["lprime_margin"][0]) == I.Workload.__dataclass_fields__["lprime_margin"].default
    assert float(c["lprime_margin"][0]) == inspect.signature(lsw.System).parameters["lprime_margin"].default
    # compressed layout: s on coarse points, then 7 wavelet planes on fine points
    wl = I.single_sf_24()
    geo = G.build(G.SystemDesc(tuple(wl.N), wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff))
    L = geo.L[0]
    assert L.n_coef == len(L.coarse.g) + int(c["wavelets_per_fine_point"][0]) * len(L.fine.g)


def test_cell_weights_follow_the_appendix():
    c = _constants()
    assert c["cell_weight_symmetric"] == ["m(m+1)/2"] and c["cell_weight_plain"] == ["m^2"]
    lo = np.array([[0, 0, 0], [0, 0, 0], [1, 0, 0]])
    hi = np.array([[1, 0, 0], [1, 0, 0], [1, 0, 0]])           # point 0: m = 2, point 1: m = 3
    assert np.array_equal(shard.cell_weights(lo, hi, [2, 1, 1]), [2 * 3 / 2, 3 * 4 / 2])
    assert np.array_equal(shard.cell_weights(lo, hi, [2, 1, 1], symmetric=False), [4, 9])
