"""Autotuner for the library's launch shapes: functions per H phi batch ("batch"), the
plane kernels of split-bfloat16 systems on the FMA units or the tensor cores ("xy_tc"),
persistent grids for the FMA plane kernels ("persistent": bit 0 backward, bit 1 forward)
and the forward member block lists ("fwd_list"), the H/S tile edge ("tile") and the H/S
panel budget per slab ("slab_mb": fewer, larger slabs repack fewer atoms at slab edges
but hold more device memory).

Each candidate is set through lsw_set_option, warmed once, then timed with CUDA events
on the system's stream; the fastest is kept.  Everything runs in the library's kernels;
this module only picks knob values.  Run it before a timed region (setting "batch"
rebuilds the batch plans and reallocates the workspace).
"""
from __future__ import annotations

from . import lsw

BATCH_CANDIDATES = (16, 32, 64, 128, 256, 512, 1024, 2048, 4096)
TILE_CANDIDATES = (3, 4, 5, 6, 7, 8)
PERSISTENT_CANDIDATES = (1, 0, 3, 2)
SLAB_CANDIDATES = (8192, 65536)


def _time(fn, stream, reps):
    import torch
    fn()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune(system, phi, hphi, H, S, e_kin, e_pot, stream, batches=BATCH_CANDIDATES,
             tiles=TILE_CANDIDATES, reps=2, budget_bytes=None, slabs=SLAB_CANDIDATES):
    """Pick "batch" and "tile" for ``system`` (an lsw.System); returns a report dict.

    ``budget_bytes`` caps the workspace a batch may take (None: no cap)."""
    report = {"batch": {}, "tile": {}}
    n_sf = system.n_sf
    best_b, best_t = None, None
    for b in batches:
        if b > max(8, n_sf):
            continue
        lsw.lsw_set_option(system.sys, "batch", b)
        ws = lsw.lsw_workspace_bytes(system.sys)
        if budget_bytes is not None and ws > budget_bytes:
            continue
        ms = _time(lambda: lsw.lsw_apply_hamiltonian(system.sys, phi, hphi, e_kin, e_pot), stream, reps)
        report["batch"][b] = ms
        if best_b is None or ms < report["batch"][best_b]:
            best_b = b
    lsw.lsw_set_option(system.sys, "batch", best_b)
    best_x = 0
    if system.precision == lsw.LSW_FP32_BF16X:
        report["xy_tc"] = {0: report["batch"][best_b]}
        try:
            lsw.lsw_set_option(system.sys, "xy_tc", 1)
            report["xy_tc"][1] = _time(lambda: lsw.lsw_apply_hamiltonian(system.sys, phi, hphi, e_kin, e_pot),
                                       stream, reps)
            best_x = 1 if report["xy_tc"][1] < report["xy_tc"][0] else 0
        except lsw.LswError:              # locregs too large for the tensor-core plane tiles
            pass
        lsw.lsw_set_option(system.sys, "xy_tc", best_x)
    hphi_ms = lambda: _time(lambda: lsw.lsw_apply_hamiltonian(system.sys, phi, hphi, e_kin, e_pot), stream, reps)
    best_p, best_l = 1, 1
    if not best_x:                      # the FMA plane kernels run: their grid forms and work lists
        report["persistent"] = {}
        for pv in PERSISTENT_CANDIDATES:
            lsw.lsw_set_option(system.sys, "persistent", pv)
            report["persistent"][pv] = hphi_ms()
        best_p = min(report["persistent"], key=report["persistent"].get)
        lsw.lsw_set_option(system.sys, "persistent", best_p)
        report["fwd_list"] = {1: report["persistent"][best_p]}
        lsw.lsw_set_option(system.sys, "fwd_list", 0)
        report["fwd_list"][0] = hphi_ms()
        best_l = min(report["fwd_list"], key=report["fwd_list"].get)
        lsw.lsw_set_option(system.sys, "fwd_list", best_l)
    lsw.lsw_apply_hamiltonian(system.sys, phi, hphi, e_kin, e_pot)
    for t in tiles:
        lsw.lsw_set_option(system.sys, "tile", t)
        ms = _time(lambda: lsw.lsw_build_matrices(system.sys, phi, hphi, H, S), stream, reps)
        report["tile"][t] = ms
        if best_t is None or ms < report["tile"][best_t]:
            best_t = t
    lsw.lsw_set_option(system.sys, "tile", best_t)
    report["slab_mb"] = {}
    best_s = None
    for sm in slabs:
        lsw.lsw_set_option(system.sys, "slab_mb", sm)
        if budget_bytes is not None and lsw.lsw_workspace_bytes(system.sys) > budget_bytes:
            continue
        report["slab_mb"][sm] = _time(lambda: lsw.lsw_build_matrices(system.sys, phi, hphi, H, S), stream, reps)
        if best_s is None or report["slab_mb"][sm] < report["slab_mb"][best_s]:
            best_s = sm
    best_s = best_s if best_s is not None else min(slabs)
    lsw.lsw_set_option(system.sys, "slab_mb", best_s)
    report["chosen"] = {"batch": best_b, "tile": best_t, "xy_tc": best_x, "persistent": best_p, "fwd_list": best_l,
                        "slab_mb": best_s}
    return report
