"""JSON system specs (host logic, CPU): round trips through explicit and generator specs
give the same system (layout and pattern bit for bit, through the library's host-only
context), and malformed specs are rejected with a message."""
import json

import numpy as np
import pytest

from paper_1401_7441_gb300 import inputs as I
from paper_1401_7441_gb300 import lsw
from paper_1401_7441_gb300 import spec as SP
from tests.lib_support import ensure_built, host_system


def _same_system(a, b):
    ensure_built()
    ctx = lsw.lsw_ctx_create(lsw.LSW_HOST_ONLY)
    Sa, Sb = host_system(a, ctx), host_system(b, ctx)
    try:
        assert Sa.n_sf == Sb.n_sf
        assert np.array_equal(Sa.off_L, Sb.off_L) and np.array_equal(Sa.off_Lp, Sb.off_Lp)
        assert np.array_equal(Sa.row_ptr, Sb.row_ptr) and np.array_equal(Sa.col, Sb.col)
    finally:
        Sa.close()
        Sb.close()
        lsw.lsw_ctx_destroy(ctx)


@pytest.mark.parametrize("name", ["atoms64", "single_sf_24"])
def test_explicit_spec_round_trip(name, tmp_path):
    w = I.WORKLOADS[name]()
    p = tmp_path / "sys.json"
    SP.dump(w, p)
    v = SP.load(p)
    assert v.N == tuple(w.N) and v.h == w.h and v.seed == w.seed
    assert np.array_equal(v.pos, w.pos) and np.array_equal(v.nsf, w.nsf)
    assert np.array_equal(v.r_loc, w.r_loc) and np.array_equal(v.r_fine, w.r_fine)
    assert np.array_equal(v.wells, w.wells)
    assert np.array_equal(I.potential(v), I.potential(w))          # same synthetic V
    _same_system(v, w)


def test_sum_of_radii_pattern_and_precision_round_trip():
    w = I.scaled("atoms64", 10)
    w.pair_mode, w.pair_cutoff, w.precision = 1, 0.0, "bf16x"
    v = SP.from_dict(json.loads(json.dumps(SP.to_dict(w))))
    assert v.pair_mode == 1 and v.precision == "bf16x"
    _same_system(v, w)


def test_generator_spec():
    v = SP.from_dict({"generator": "scaled", "base": "atoms64", "n_atoms": 20, "seed": 3, "precision": "fp32"})
    w = I.scaled("atoms64", 20, seed=3)
    assert np.array_equal(v.pos, w.pos) and v.precision == "fp32"
    assert SP.from_dict({"generator": "atoms64"}).name == "atoms64"


def test_derived_grid_covers_the_atoms():
    v = SP.from_dict({"h": 0.5, "pair_cutoff": 10.0,
                      "atoms": [{"pos": [6.0, 6.0, 6.0], "r_loc": 5.0, "r_fine": 1.5, "n_sf": 4},
                                {"pos": [9.0, 7.5, 6.5], "r_loc": 5.0, "r_fine": 1.5, "n_sf": 1}]})
    assert v.N == (29, 29, 29)                                   # ceil((9 + 5) / 0.5) + 1
    assert v.n_sf == 5 and v.pair_mode == 0


@pytest.mark.parametrize("bad, msg", [
    ({"atoms": [{"pos": [1, 1, 1], "r_loc": 5, "r_fine": 1, "n_sf": 1}], "pair_cutoff": 5}, "missing 'h'"),
    ({"h": 0.45, "atoms": [], "pair_cutoff": 5}, "non-empty"),
    ({"h": 0.45, "atoms": [{"pos": [1, 1], "r_loc": 5, "r_fine": 1, "n_sf": 1}], "pair_cutoff": 5}, "three numbers"),
    ({"h": 0.45, "atoms": [{"pos": [-1, 1, 1], "r_loc": 5, "r_fine": 1, "n_sf": 1}], "pair_cutoff": 5}, ">= 0"),
    ({"h": 0.45, "atoms": [{"pos": [1, 1, 1], "r_loc": 5, "r_fine": 1, "n_sf": 1}], "pair_cutoff": 5,
      "precision": "fp16"}, "precision"),
    ({"generator": "nope"}, "unknown generator"),
    ([1, 2], "JSON object"),
])
def test_malformed_specs_are_rejected(bad, msg):
    with pytest.raises(SP.SpecError, match=msg):
        SP.from_dict(bad)


def test_invalid_json_file(tmp_path):
    p = tmp_path / "bad.json"
    p.write_text("{not json")
    with pytest.raises(SP.SpecError, match="not valid JSON"):
        SP.load(p)
