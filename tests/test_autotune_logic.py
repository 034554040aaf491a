"""The autotuner's selection logic (host, CPU): with the library calls and the timer
replaced by fakes whose timings depend on the options set, every knob keeps its fastest
candidate, candidates over the workspace budget are skipped, the tensor-core plane
kernels are only tried on split-bfloat16 systems, and the system is left on the chosen
values."""
from types import SimpleNamespace

import pytest

from paper_1401_7441_gb300 import autotune as AT
from paper_1401_7441_gb300 import lsw


class _FakeLib:
    """Options of one fake system; the "time" of a call is a function of them."""

    def __init__(self, xy_tc_error=False):
        self.opts = {"batch": 32, "tile": 4, "xy_tc": 0, "persistent": 1, "fwd_list": 1, "slab_mb": 8192}
        self.xy_tc_error = xy_tc_error
        self.last = None

    def set_option(self, sys, name, value):
        if name == "xy_tc" and value == 1 and self.xy_tc_error:
            raise lsw.LswError(lsw.LSW_ERR_UNSUPPORTED, "too large")
        self.opts[name] = value

    def workspace_bytes(self, sys):
        return 1000 * self.opts["batch"] + 10 * self.opts["slab_mb"]

    def apply(self, *a):
        o = self.opts
        # fastest at batch 512, xy_tc off, persistent 3, fwd_list 0
        self.last = (abs(o["batch"] - 512) / 100.0 + 5.0 * o["xy_tc"] + {0: 3, 1: 2, 2: 4, 3: 1}[o["persistent"]]
                     + 0.5 * o["fwd_list"])

    def build(self, *a):
        self.last = abs(self.opts["tile"] - 6) + 1.0 + (0.1 if self.opts["slab_mb"] < 65536 else 0.0)


@pytest.fixture
def fake(monkeypatch):
    def make(**kw):
        f = _FakeLib(**kw)
        monkeypatch.setattr(AT.lsw, "lsw_set_option", f.set_option)
        monkeypatch.setattr(AT.lsw, "lsw_workspace_bytes", f.workspace_bytes)
        monkeypatch.setattr(AT.lsw, "lsw_apply_hamiltonian", f.apply)
        monkeypatch.setattr(AT.lsw, "lsw_build_matrices", f.build)

        def timed(fn, stream, reps):
            fn()
            return f.last

        monkeypatch.setattr(AT, "_time", timed)
        return f
    return make


def _system(prec, n_sf=10000):
    return SimpleNamespace(sys=object(), n_sf=n_sf, precision=prec)


def test_each_knob_keeps_its_fastest_candidate(fake):
    f = fake()
    rep = AT.autotune(_system(lsw.LSW_FP32_BF16X), None, None, None, None, None, None, None)
    assert rep["chosen"] == {"batch": 512, "tile": 6, "xy_tc": 0, "persistent": 3, "fwd_list": 0, "slab_mb": 65536}
    assert {k: f.opts[k] for k in rep["chosen"]} == rep["chosen"]          # left on the choice
    assert set(rep["batch"]) == set(AT.BATCH_CANDIDATES)
    assert set(rep["persistent"]) == set(AT.PERSISTENT_CANDIDATES)
    assert set(rep["tile"]) == set(AT.TILE_CANDIDATES)


def test_budget_skips_large_batches_and_fp32_skips_the_tensor_core_planes(fake):
    f = fake()
    rep = AT.autotune(_system(lsw.LSW_FP32), None, None, None, None, None, None, None,
                      budget_bytes=1000 * 256 + 10 * 8192)
    assert max(rep["batch"]) == 256 and rep["chosen"]["batch"] == 256
    assert list(rep["slab_mb"]) == [8192] and rep["chosen"]["slab_mb"] == 8192    # the larger slab does not fit
    assert "xy_tc" not in rep and rep["chosen"]["xy_tc"] == 0
    assert f.opts["batch"] == 256


def test_tensor_core_planes_that_do_not_fit_are_skipped(fake):
    f = fake(xy_tc_error=True)
    rep = AT.autotune(_system(lsw.LSW_FP32_BF16X), None, None, None, None, None, None, None)
    assert rep["xy_tc"] == {0: rep["batch"][rep["chosen"]["batch"]]} and rep["chosen"]["xy_tc"] == 0
    assert rep["chosen"]["persistent"] == 3 and f.opts["xy_tc"] == 0


def test_small_systems_skip_batches_far_above_their_size(fake):
    fake()
    rep = AT.autotune(_system(lsw.LSW_FP64, n_sf=20), None, None, None, None, None, None, None)
    assert max(rep["batch"]) <= 20 and rep["chosen"]["batch"] in rep["batch"]
