"""Benchmark: H phi for every support function + sparse H_ab / S_ab, on synthetic
locreg workloads shaped like the paper's (arXiv 1401.7441), on one or more GPUs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME]
                  [--precision fp32|fp64|bf16x] [--impl ours|reference]

One step = lsw_apply_hamiltonian (every support function) + lsw_build_matrices (the
whole CSR pattern) on inputs resident in HBM.  The L2 is flushed (a 512 MB write)
before every timed step; each step is bracketed by CUDA events on the library's
stream.  value = support functions per second (whole job; N > 1 runs N independent
replicas, one per rank, no collective: "replicas only", weak scaling).

Extra keys: e2e (the same metric through lsw_step_host with pinned host buffers:
phi host->device, H and S device->host inside the timed region), roofline (the
dominant kernel, from the library's per-launch device trace over the timed steps),
cpu_baseline (the oracle on a bounded sample, host cores), clocks (nvidia-smi sampled
during the timed steps), gpu_launches (kernels enqueued per timed step x steps).

--impl reference runs the oracle (the plain FP64 CPU implementation written from the
paper) on a bounded sample of the same workload: it is the only reference there is.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1401_7441_gb300 import inputs as I  # noqa: E402

METRIC = "H-phi support functions/s incl. sparse H,S build"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
# Nominal CUDA-core peaks (context beside the measured ones): FP32 152 SMs x 128 lanes x
# 2 flop x 2.07 GHz; FP64 the nominal GB300 figure.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
FP64_PEAK_TFLOPS = 1.25


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--workload", default=None, help="default atoms10k (atoms1200 for --mode density)")
    p.add_argument("--precision", default=None, choices=[None, "fp32", "fp64", "bf16x"])
    p.add_argument("--impl", default="ours", choices=["ours", "reference"])
    p.add_argument("--mode", default="step", choices=["step", "serving", "density", "compare", "foe"],
                   help="serving: Poisson request stream through the continuous-batching server; "
                        "density: rho = sum_ab K_ab phi_a phi_b on the fine grid (default workload atoms1200); "
                        "compare: the served form (split-bf16, batched) against the plain per-locreg FP64 GPU "
                        "form on the same system, errors of both against each other and the oracle; "
                        "foe: the Fermi operator expansion on the system's H, S (default workload atoms1200)")
    p.add_argument("--requests", type=int, default=60)
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu", action="store_true")
    p.add_argument("--batch", type=int, default=0)
    p.add_argument("--tile", type=int, default=0)
    p.add_argument("--no-autotune", action="store_true")
    p.add_argument("--set", action="append", default=[], metavar="NAME=VALUE",
                   help="library option (lsw_set_option), applied after the autotuner; repeatable")
    p.add_argument("--record-traffic", default=None, metavar="CSV",
                   help="write profiles/roofline_traffic.json from an ncu launch list (dram bytes) of a run with "
                        "the given --workload/--precision/--batch, then exit")
    p.add_argument("--replicas", action="store_true",
                   help="N > 1: N independent replicas of the whole workload instead of the sharded form")
    p.add_argument("--oracle-functions", type=int, default=512,
                   help="functions of the oracle sample (CPU baseline and errors)")
    p.add_argument("--sync-each", action="store_true",
                   help="warm-up only: wait for the device and check its status after every call")
    return p.parse_args()


def workload(name):
    if name in I.WORKLOADS:
        return I.WORKLOADS[name]()
    if name.startswith("atoms10k_n"):
        return I.scaled("atoms10k", int(name.split("_n")[1]))
    if name.startswith("atoms64_n"):
        return I.scaled("atoms64", int(name.split("_n")[1]))
    if name.endswith(".json"):                      # a JSON system spec (spec.py)
        from paper_1401_7441_gb300 import spec
        return spec.load(name)
    raise SystemExit("unknown workload " + name)


def kernels_source_hash():
    """SHA-256 over the CUDA sources (every .cu file and the internal header, in name
    order): ties a stored ncu traffic figure to the kernels it was measured on."""
    import hashlib
    d = os.path.join(ROOT, "paper_1401_7441_gb300", "csrc")
    hs = hashlib.sha256()
    for name in sorted(os.listdir(d)):
        if name.endswith(".cu") or name == "lsw_internal.h":
            hs.update(name.encode())
            hs.update(open(os.path.join(d, name), "rb").read())
    return hs.hexdigest()


def stored_traffic(kernel, prec, fns_per_launch):
    """(DRAM bytes per launch of ``kernel``, note) from profiles/roofline_traffic.json, if
    that file was written from an ncu capture of the current kernel sources (else (None,
    reason)).  The capture stores bytes per support function of a launch (the kernels'
    traffic grows with the functions they process); they are scaled to this launch's
    functions."""
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    try:
        rec = json.load(open(path))
    except Exception:
        return None, "no stored capture"
    if rec.get("kernels_sha256") != kernels_source_hash():
        return None, "stored capture is of another kernel source"
    ent = rec.get("kernels", {}).get(kernel)
    if not ent or ent.get("precision") != prec or not fns_per_launch:
        return None, "no stored capture for this kernel and precision"
    per_fn = ent["dram_bytes_per_function"]
    return per_fn * fns_per_launch, ("ncu capture (%s: %d functions per launch) scaled to %d functions per launch"
                                     % (rec.get("workload", "?"), ent.get("functions_per_launch", 0), fns_per_launch))


KERNEL_KIND = {"k_uncompress": "uncompress", "k_fwd_xy": "fwd_xy", "k_fwd_xy_tc": "fwd_xy", "k_z": "z_stage",
               "k_z_tc": "z_stage", "k_kin_z": "kinetic", "k_bwd_xy": "bwd_xy", "k_pack": "hs_pack",
               "k_panel_hs": "hs_tiles", "k_panel_hs_tc": "hs_tiles"}


def record_traffic(csv_path, wl, prec, batch, n_slab_launches=1):
    """Write profiles/roofline_traffic.json from an ncu launch list with
    dram__bytes_read.sum and dram__bytes_write.sum (CSV) of a run of this benchmark:
    DRAM bytes per support function of a launch, per kernel kind (H phi kernels: the
    launch's batch; H/S kernels: the system's functions over its slab launches), tied to
    the SHA-256 of the kernel sources."""
    import csv
    import io
    txt = open(csv_path).read()
    rows = list(csv.DictReader(io.StringIO(txt[txt.index('"ID"'):])))
    per = {}
    for r in rows:
        name = r["Kernel Name"].split("(")[0].split("<")[0].replace("void ", "").strip()
        kind = KERNEL_KIND.get(name)
        if kind is None or r["Metric Name"] not in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            continue
        v = float(r["Metric Value"].replace(",", ""))
        unit = r.get("Metric Unit", "byte")
        v *= {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9}.get(unit, 1)
        per.setdefault(kind, {}).setdefault(r["ID"], 0.0)
        per[kind][r["ID"]] += v
    n_sf = int(np.sum(wl.nsf))
    # functions of the j-th launch of an H phi kernel in a step: the batches in order
    sizes = [min(batch, n_sf - b0) for b0 in range(0, n_sf, batch)]
    out = {"kernels_sha256": kernels_source_hash(), "workload": wl.name, "kernels": {}}
    for kind, launches in per.items():
        ids = sorted(launches, key=int)
        vals = [launches[i] for i in ids]
        if kind.startswith("hs_"):
            fns = [n_sf / n_slab_launches] * len(vals)
        else:
            fns = [sizes[j % len(sizes)] for j in range(len(vals))]
        out["kernels"][kind] = {"precision": prec, "functions_per_launch": int(round(np.mean(fns))),
                                "launches_captured": len(vals), "dram_bytes_per_launch": float(np.mean(vals)),
                                "dram_bytes_per_function": float(np.sum(vals) / np.sum(fns))}
    path = os.path.join(ROOT, "profiles", "roofline_traffic.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    return path


def keys_to_g(keys):
    if len(keys) == 0:
        return np.zeros(0, np.int64)
    lens = keys[:, 1] - keys[:, 0] + 1
    starts = np.repeat(keys[:, 0] - np.concatenate([[0], np.cumsum(lens)[:-1]]), lens)
    return starts + np.arange(int(lens.sum()), dtype=np.int64)


# ---------------------------------------------------------------- oracle (CPU) leg
#
# The oracle (plain FP64 numpy, written from the paper) timed on the host cores: H phi of
# a bounded sample of functions, spread over a pool of worker processes (spawned, so no
# process inherits a CUDA context), then S/H entries of pattern pairs among them.

_ORC = {}


def _orc_desc(wl):
    from oracle import geometry as G
    return G.SystemDesc(tuple(wl.N), wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff,
                        wl.pair_mode, wl.lprime_margin, wl.fine_mode)


def _orc_init(wl_name, atoms):
    from oracle import geometry as G
    wl = workload(wl_name)
    _ORC["wl"] = wl
    _ORC["geo"] = G.build(_orc_desc(wl), atoms=atoms, pattern=False)


def _orc_hphi(fs):
    """H phi, E_kin, E_pot of the functions ``fs`` by the oracle (in a worker)."""
    from oracle import hamiltonian as Hm
    wl, geo = _ORC["wl"], _ORC["geo"]
    out = []
    for f in fs:
        a = int(geo.sf_atom[f])
        L = geo.L[a]
        phi = I.phi_values(wl, f, a, L.coarse.g, L.fine.g)
        lo = [2 * int(L.lo[d]) - 14 for d in range(3)]
        shape = [2 * int(L.hi[d] - L.lo[d] + 1) + 29 for d in range(3)]
        Vb = I.potential_block(wl, lo, shape)
        h, ek, ep = Hm.apply_hamiltonian(geo, f, phi, Vb, lo)
        out.append((f, phi, h, ek, ep))
    return out


def cpu_model():
    try:
        for ln in open("/proc/cpuinfo"):
            k = ln.split(":")[0].strip().lower()
            if k in ("model name", "cpu model", "hardware"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


class OraclePool:
    """Worker processes (spawn) holding the oracle's geometry of a sample of atoms."""

    def __init__(self, wl_name, atoms, cores):
        import concurrent.futures as cf
        import multiprocessing as mp
        self.cores = max(1, int(cores))
        old = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
        for k in old:
            os.environ[k] = "1"                      # one thread per worker process
        try:
            self.ex = cf.ProcessPoolExecutor(self.cores, mp_context=mp.get_context("spawn"),
                                             initializer=_orc_init, initargs=(wl_name, atoms))
            list(self.ex.map(int, range(self.cores)))   # start every worker now
            _orc_init(wl_name, atoms)                    # this process: the entries
        finally:
            for k, v in old.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v

    def hphi(self, fs):
        chunks = [fs[i::self.cores] for i in range(self.cores) if fs[i::self.cores]]
        out = []
        for part in self.ex.map(_orc_hphi, chunks):
            out.extend(part)
        return out

    def close(self):
        self.ex.shutdown()


def sample_functions(wl, n_fn):
    """The n_fn functions whose atoms are nearest the cell's centre (so that many of their
    pattern partners are in the sample), and their atoms."""
    pos = np.asarray(wl.pos)
    c = pos.mean(axis=0)
    order = np.argsort(np.sum((pos - c) ** 2, axis=1), kind="stable")
    first = np.concatenate([[0], np.cumsum(wl.nsf)])
    fs, atoms = [], []
    for a in order:
        if len(fs) >= n_fn:
            break
        if wl.nsf[a] == 0:
            continue
        atoms.append(int(a))
        fs.extend(range(int(first[a]), int(first[a + 1])))
    return sorted(fs[:n_fn]), sorted(atoms)


def oracle_entries(geo, done, row_ptr, col, max_entries, seed=3):
    """Pattern entries (a, b) with both functions in ``done`` (seeded subsample of at most
    max_entries): {(a, b): (S_ab, H_ab)} by the oracle, and the time it took."""
    from oracle import matrices as Mx
    have = set(done["phi"].keys())
    pairs = [(a, int(col[k])) for a in sorted(have) for k in range(row_ptr[a], row_ptr[a + 1]) if int(col[k]) in have]
    if len(pairs) > max_entries:
        rng = np.random.default_rng(seed)
        pairs = [pairs[i] for i in sorted(rng.choice(len(pairs), size=max_entries, replace=False))]
    t0 = time.perf_counter()
    ents = {(a, b): (Mx.overlap_entry(geo, a, b, done["phi"][a], done["phi"][b]),
                     Mx.hamiltonian_entry(geo, a, b, done["phi"][a], done["hphi"][b])) for a, b in pairs}
    return ents, time.perf_counter() - t0


def oracle_run(wl, pool, fs, row_ptr, col, max_entries):
    """The oracle on functions ``fs`` (pool) and the entries among them (this process,
    whose geometry the pool set up).
    Returns (results dict, seconds for H phi, seconds per entry)."""
    t0 = time.perf_counter()
    res = pool.hphi(fs)
    t_h = time.perf_counter() - t0
    done = {"phi": {f: p for f, p, _, _, _ in res}, "hphi": {f: h for f, _, h, _, _ in res},
            "energies": {f: (ek, ep) for f, _, _, ek, ep in res}}
    ents, t_e = oracle_entries(_ORC["geo"], done, row_ptr, col, max_entries)
    done["entries"] = ents
    return done, t_h, (t_e / len(ents) if ents else 0.0)


def cpu_baseline_of(wl, n_fn, nnz_per_fn, t_h, t_entry, cores, n_entries):
    """Oracle support functions/s for H phi plus the function's row of S and H: H phi
    time per function (measured on ``cores`` processes) plus the measured time per entry
    times the mean pattern entries per function (extrapolated)."""
    per_fn = t_h / n_fn + t_entry * nnz_per_fn / cores
    sample = ("oracle (numpy FP64) on %d host cores (%d in the machine, %s): H phi of the %d support functions "
              "nearest the cell centre in %.1f s, then %d S/H entries among them at %.2f ms each (one process); "
              "per function: H phi time + %.0f entries (the mean pattern row) at that rate / %d cores, extrapolated"
              % (cores, os.cpu_count() or 1, cpu_model(), n_fn, t_h, n_entries, 1e3 * t_entry, nnz_per_fn, cores))
    return {"value": 1.0 / per_fn, "unit": "support_functions/s", "cores": cores, "kind": "oracle",
            "sample": sample}


def error_report(ref, S, hphi_dev, ek_dev, ep_dev, H_dev, S_dev, tag="FP64 CPU oracle"):
    """Errors of the GPU results against a reference sample: H phi normwise per function
    and element by element (each element against tau-free scale |H phi|_max of its
    function), energies and H/S entries by Cauchy-Schwarz bounds."""
    done = sorted(ref["hphi"].keys())
    hp = hphi_dev.double().cpu().numpy() if hasattr(hphi_dev, "cpu") else hphi_dev
    ek = ek_dev.cpu().numpy() if hasattr(ek_dev, "cpu") else ek_dev
    ep = ep_dev.cpu().numpy() if hasattr(ep_dev, "cpu") else ep_dev
    e_h, e_el, e_en = [], [], []
    for f in done:
        h = ref["hphi"][f]
        o = int(S.off_Lp[f])
        g = hp[o:o + len(h)]
        e_h.append(float(np.linalg.norm(g - h) / np.linalg.norm(h)))
        e_el.append(float(np.max(np.abs(g - h)) / np.max(np.abs(h))))
        scale = np.linalg.norm(ref["phi"][f]) * np.linalg.norm(h)
        rk, rp_ = ref["energies"][f]
        e_en.append(float(max(abs(ek[f] - rk), abs(ep[f] - rp_)) / scale))
    Hh = H_dev.cpu().numpy() if hasattr(H_dev, "cpu") else H_dev
    Sh = S_dev.cpu().numpy() if hasattr(S_dev, "cpu") else S_dev
    e_s, e_hh = [], []
    for (a, b), (sv, hv) in ref.get("entries", {}).items():
        row = S.col[S.row_ptr[a]:S.row_ptr[a + 1]]
        k = np.searchsorted(row, b)
        if k < len(row) and row[k] == b:
            kk = int(S.row_ptr[a] + k)
            e_s.append(abs(Sh[kk] - sv) / (np.linalg.norm(ref["phi"][a]) * np.linalg.norm(ref["phi"][b])))
            e_hh.append(abs(Hh[kk] - hv) / (np.linalg.norm(ref["phi"][a]) * np.linalg.norm(ref["hphi"][b])))
    return {"against": tag, "functions": len(done), "entries": len(e_s),
            "hphi_rel_max": max(e_h), "hphi_rel_mean": float(np.mean(e_h)),
            "hphi_elem_rel_max": max(e_el),
            "energy_scaled_max": max(e_en),
            "S_scaled_max": float(max(e_s)) if e_s else None, "H_scaled_max": float(max(e_hh)) if e_hh else None}


def canonical_config(wl, prec, n_sf):
    """The workload's identity, the same in both arms of the benchmark."""
    return {"workload": wl.name, "atoms": int(len(wl.pos)), "support_functions": int(n_sf),
            "grid": [int(x) for x in wl.N], "h_bohr": wl.h, "precision": prec,
            "l2": "flushed (512 MB write) before every timed step"}


def reference_main(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    wl = workload(args.workload or "atoms10k")
    prec = args.precision or wl.precision
    cores = os.cpu_count() or 1
    from oracle import geometry as G
    row_ptr, col = G.pair_pattern(_orc_desc(wl), np.repeat(np.arange(len(wl.nsf)), wl.nsf))
    nnz_per_fn = len(col) / max(1, wl.n_sf)
    # one step = H phi of 2 functions per core + their row entries (extrapolated), so the
    # whole --steps/--warmup run ends within a few minutes
    n_step = 2 * cores
    fs_all, atoms = sample_functions(wl, n_step * (args.steps + args.warmup))
    pool = OraclePool(args.workload or "atoms10k", atoms, cores)
    vals, samples = [], []
    try:
        for i in range(args.warmup + args.steps):
            fs = fs_all[i * n_step:(i + 1) * n_step] or fs_all[:n_step]
            done, t_h, t_e = oracle_run(wl, pool, fs, row_ptr, col, max_entries=64)
            cb = cpu_baseline_of(wl, len(fs), nnz_per_fn, t_h, t_e, cores, len(done["entries"]))
            if i >= args.warmup:
                vals.append(cb["value"])
                samples.append(cb["sample"])
    finally:
        pool.close()
    val = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "support_functions/s",
            "n_gpus": 0, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * n_step / val,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": canonical_config(wl, prec, wl.n_sf),
            "cpu_baseline": {"value": val, "unit": "support_functions/s", "cores": cores,
                             "kind": "oracle", "sample": "per step: " + samples[-1]},
            "e2e": {"value": val, "unit": "support_functions/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------- multi-process aggregation

def aggregate(local_value, world, device=None, op="max"):
    """Max (or sum) of a per-rank scalar over all ranks; the identity on one rank.

    Replicas run the same workload on every rank without any data-path collective;
    this is the only collective of the benchmark (timing), as the contract asks:
    the job time is the slowest rank's."""
    if world <= 1:
        return float(local_value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def job_value(n_sf, steps, world, max_ms):
    """Support functions per second of the whole job: every rank processes n_sf per step."""
    return world * n_sf * steps / (max_ms / 1000.0)


# ---------------------------------------------------------------- GPU leg

class ClockSampler:
    def __init__(self, path):
        self.path = path
        self.proc = None

    def __enter__(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                          "-lms", "100"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self, dev_index):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": []}
        try:
            rows = [ln.split(",") for ln in open(self.path) if ln.strip()]
        except Exception:
            return out
        rows = [[x.strip() for x in r] for r in rows if r and r[0].strip() == str(dev_index)]
        if not rows:
            return out
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        out["sm_mhz"] = statistics.median(sm) if sm else None
        out["sm_max_mhz"] = max(mx) if mx else None
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        out["reasons"] = sorted(reasons)
        out["samples"] = len(rows)
        return out


def kernel_work(S, wl, prec):
    """Algorithmic FLOPs per kernel kind for one full step: the in-range taps of each
    separable filter (zero padding and out-of-box taps are not counted),
    and the compulsory bytes of a step (phi in, H phi out, H and S values out)."""
    es = 8 if prec == "fp64" else 4
    fl = {"fwd_xy": 0.0, "z_stage": 0.0, "bwd_xy": 0.0, "kinetic": 0.0}

    def up_taps(nout, nin):
        # sum over fine outputs o of #{coarse q in [0, nin): 0 <= o - 2q <= 30}
        o = np.arange(nout)[:, None]
        q = np.arange(nin)[None, :]
        return int(np.sum((o - 2 * q >= 0) & (o - 2 * q <= 30)))

    def down_taps(nout, off, nin):
        # sum over coarse outputs b (L' box, offset off) of #{fine o in [0, nin): 0 <= o - 2(b+off) <= 30}
        b = np.arange(nout)[:, None] + off
        o = np.arange(nin)[None, :]
        return int(np.sum((o - 2 * b >= 0) & (o - 2 * b <= 30)))

    def kin_taps(nout, off, nin):
        # sum over L' outputs of #{l in [-14, 14]: 0 <= out + off + l < nin}
        o = np.arange(nout)[:, None] + off
        l = np.arange(-14, 15)[None, :]
        return int(np.sum((o + l >= 0) & (o + l < nin)))

    def box(k, N):
        g0, g1 = k[:, 0], k[:, 1]
        x0, x1 = g0 % N[0], g1 % N[0]
        y = (g0 // N[0]) % N[1]
        z = g0 // (N[0] * N[1])
        lo = np.array([x0.min(), y.min(), z.min()])
        hi = np.array([x1.max(), y.max(), z.max()])
        return lo, hi - lo + 1

    cache = {}
    for f in range(S.n_sf):
        a = int(S.sf_atom[f])
        if a not in cache:
            lo, n = box(S.keys(a, 0, 0), wl.N)
            lop, npp = box(S.keys(a, 1, 0), wl.N)
            X, Y, Z = (2 * n + 29)
            d = lop - lo
            fx = 4 * n[1] * n[2] * 2 * up_taps(X, n[0])       # 4 (by, bz) rows x 2 input types
            fy = 2 * n[2] * X * 2 * up_taps(Y, n[1])
            fz = X * Y * 2 * up_taps(Z, n[2])
            bz = X * Y * 2 * down_taps(npp[2], d[2], Z)        # 2 output types
            by = npp[2] * 2 * X * 2 * down_taps(npp[1], d[1], Y)
            bx = npp[2] * 4 * npp[1] * 2 * down_taps(npp[0], d[0], X)
            # kinetic arms: per output point and output type, 2 input types x in-range taps
            kx = 8 * n[2] * n[1] * 2 * kin_taps(npp[0], d[0], n[0])
            ky = 8 * n[2] * n[0] * 2 * kin_taps(npp[1], d[1], n[1])
            kz = 8 * n[1] * n[0] * 2 * kin_taps(npp[2], d[2], n[2])
            cache[a] = (2.0 * (fx + fy), 2.0 * (fz + bz), 2.0 * (by + bx + kx + ky), 2.0 * kz)
        c = cache[a]
        fl["fwd_xy"] += c[0]
        fl["z_stage"] += c[1]
        fl["bwd_xy"] += c[2]
        fl["kinetic"] += c[3]
    comp_bytes = es * (S.total_L + S.total_Lp) + 16.0 * len(S.col)
    return fl, comp_bytes


def gpu_main(args):
    import torch
    import torch.distributed as dist

    from paper_1401_7441_gb300 import build as B
    from paper_1401_7441_gb300 import lsw

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    B.build()
    wl = workload(args.workload or "atoms10k")
    prec = args.precision or wl.precision
    P = {"fp64": lsw.LSW_FP64, "fp32": lsw.LSW_FP32, "bf16x": lsw.LSW_FP32_BF16X}[prec]
    dt = torch.float64 if prec == "fp64" else torch.float32
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    t_setup = time.perf_counter()
    sharded = world > 1 and not args.replicas
    n_sf_job = int(np.sum(wl.nsf))
    wl_glob = wl
    if sharded:
        # this rank's sub-system: own atoms (x slabs balanced by functions) first, then the
        # halo its rows reach and the ghosts that keep the fine region; H phi only for the
        # own functions; halo phi and H phi arrive by the grouped NCCL exchange each step
        from paper_1401_7441_gb300 import shard
        hctx = lsw.lsw_ctx_create(lsw.LSW_HOST_ONLY)
        Wh = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                        wl.lprime_margin, 0, P, ctx=hctx)
        owner = shard.partition_atoms(wl.pos, wl.nsf, world)
        wsub, amap, fmap = shard.subsystem(wl, owner, rank, Wh.sf_atom, Wh.row_ptr, Wh.col, own_first=True)
        plan = shard.halo_plan(Wh.row_ptr, Wh.col, Wh.sf_atom, owner, rank)
        n_own = int(np.sum(owner[Wh.sf_atom] == rank))
        Wh.close()
        lsw.lsw_ctx_destroy(hctx)
        wl = wsub
    S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   wl.lprime_margin, 0, P, device=local, stream=stream.cuda_stream)
    if sharded:
        lsw.lsw_set_option(S.sys, "hphi_limit", n_own)
        g2l = {int(g): k for k, g in enumerate(fmap)}
    if args.batch:
        lsw.lsw_set_option(S.sys, "batch", args.batch)
    if args.tile:
        lsw.lsw_set_option(S.sys, "tile", args.tile)
    # inputs on the device: phi from the counter generator, V sampled on the fine grid
    phi = torch.zeros(S.total_L, dtype=dt, device="cuda")
    atoms = sorted(set(int(a) for a in S.sf_atom))
    cg = {a: keys_to_g(S.keys(a, 0, 0)) for a in atoms}
    fg = {a: keys_to_g(S.keys(a, 0, 1)) for a in atoms}
    if sharded:
        I.fill_phi(wl_glob, phi, S.off_L, amap[np.asarray(S.sf_atom)],
                   {int(amap[a]): cg[a] for a in atoms}, {int(amap[a]): fg[a] for a in atoms}, fn_ids=fmap)
    else:
        I.fill_phi(wl, phi, S.off_L, S.sf_atom, cg, fg)
    V = I.potential_fast(wl_glob, "cuda").to(dt)
    lsw.lsw_set_potential(S.sys, V, wl.V_lo, wl.V_shape)
    hphi = torch.zeros(S.total_Lp, dtype=dt, device="cuda")
    ek = torch.zeros(S.n_sf, dtype=torch.float64, device="cuda")
    ep = torch.zeros(S.n_sf, dtype=torch.float64, device="cuda")
    nnz = len(S.col)
    Hm = torch.zeros(max(1, nnz), dtype=torch.float64, device="cuda")
    Sm = torch.zeros(max(1, nnz), dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup

    def step():
        lsw.lsw_apply_hamiltonian(S.sys, phi, hphi, ek, ep)
        if sharded:
            shard.exchange_local([phi, hphi], [S.off_L, S.off_Lp], g2l, plan)
        lsw.lsw_build_matrices(S.sys, phi, hphi, Hm, Sm)

    # roofline denominators measured on this GPU (FMA loops, streaming copy)
    peaks = dict(zip(("fp32_fma_tflops", "fp64_fma_tflops", "copy_gbs"), lsw.lsw_measure_peaks(S.ctx)))
    try:   # the pool's own copy / bf16 GEMM measurements, as context beside these
        pool = json.load(open(PEAKS_PATH))
        peaks["pool_hbm_gbs"] = pool.get("hbm_gbs")
        peaks["pool_bf16_tflops"] = pool.get("bf16_tflops")
    except Exception:
        pass
    tune = None
    if not args.no_autotune and not args.batch and not args.tile:
        from paper_1401_7441_gb300 import autotune
        tune = autotune.autotune(S, phi, hphi, Hm, Sm, ek, ep, stream)
    set_opts = {}
    for kv in args.set:
        k, v = kv.split("=", 1)
        lsw.lsw_set_option(S.sys, k, int(v))
        set_opts[k] = int(v)

    for _ in range(args.warmup):
        if args.sync_each:
            lsw.lsw_apply_hamiltonian(S.sys, phi, hphi, ek, ep)
            lsw.lsw_sync(S.sys, 600.0)
            lsw.lsw_build_matrices(S.sys, phi, hphi, Hm, Sm)
            lsw.lsw_sync(S.sys, 600.0)
        else:
            step()
    torch.cuda.synchronize()
    lsw.lsw_profile(S.sys, 1)
    step()                      # capture the traced graphs outside the timed region
    lsw.lsw_profile_read(S.sys)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    prof = {}
    clk_path = os.path.join(tempfile.gettempdir(), "lsw_clocks_%d.csv" % os.getpid())
    with ClockSampler(clk_path) as clk:
        time.sleep(0.3)
        for i in range(args.steps):
            flush.fill_(float(i))
            if world > 1:
                dist.barrier()
            torch.cuda.synchronize()
            ev0[i].record(stream)
            step()
            ev1[i].record(stream)
            torch.cuda.synchronize()
            for k, (ms, n) in lsw.lsw_profile_read(S.sys).items():
                a, b = prof.get(k, (0.0, 0))
                prof[k] = (a + ms, b + n)
    step_ms = [ev0[i].elapsed_time(ev1[i]) for i in range(args.steps)]
    total_ms = aggregate(sum(step_ms), world, device="cuda")
    lsw.lsw_profile(S.sys, 0)
    clocks = clk.summary(local)
    # the whole job's functions per second: replicas each process the whole workload,
    # sharded ranks together process it once
    value = (n_sf_job * args.steps / (total_ms / 1000.0)) if sharded else job_value(S.n_sf, args.steps, world, total_ms)

    # end to end through the host API (pinned host buffers): phi host -> device, the
    # step, H and S device -> host; and the same with H phi copied back too
    e2e = e2e_h = None
    if not args.no_e2e:
        phi_h = phi.cpu().pin_memory()
        hphi_h = torch.empty(S.total_Lp, dtype=dt).pin_memory()
        H_h = torch.empty(max(1, nnz), dtype=torch.float64).pin_memory()
        S_h = torch.empty(max(1, nnz), dtype=torch.float64).pin_memory()
        k2 = max(1, min(args.steps, 3))

        def host_step(with_h):
            if not sharded:
                lsw.lsw_step_host(S.sys, phi_h, hphi_h if with_h else None, H_h, S_h)
                return
            # the sharded step through the same calls: phi in, H phi, the exchange, H/S out
            phi.copy_(phi_h, non_blocking=True)
            step()
            if with_h:
                hphi_h.copy_(hphi, non_blocking=True)
            H_h.copy_(Hm, non_blocking=True)
            S_h.copy_(Sm, non_blocking=True)
            torch.cuda.synchronize()
        for with_h in (False, True):
            host_step(with_h)
            if world > 1:
                dist.barrier()
            t0 = time.perf_counter()
            for _ in range(k2):
                host_step(with_h)
            el = aggregate(time.perf_counter() - t0, world, device="cuda")
            rec = {"value": (n_sf_job * k2 / el) if sharded else job_value(S.n_sf, k2, world, 1000.0 * el),
                   "unit": "support_functions/s",
                   "h2d_bytes_per_step": int(phi_h.numel() * phi_h.element_size()),
                   "d2h_bytes_per_step": int(2 * nnz * 8 + (hphi_h.numel() * hphi_h.element_size() if with_h else 0)),
                   "steps": k2}
            if with_h:
                e2e_h = rec
            else:
                e2e = rec

    # roofline: the method's own work per kernel (workcount) over the kernels' device time
    from paper_1401_7441_gb300 import workcount as WC
    import concurrent.futures as cf
    import multiprocessing as mp
    with cf.ProcessPoolExecutor(min(16, os.cpu_count() or 1), mp_context=mp.get_context("spawn")) as wpool:
        flops, wnote = WC.hphi_work(S, wl.N, pool=wpool)
    hs_mac, hs_se = WC.hs_work(S)
    flops["hs_tiles"] = 2.0 * hs_mac
    wnote["hs_rel_se"] = hs_se
    dense, comp_bytes = kernel_work(S, wl, prec)
    peak_alu = FP64_PEAK_TFLOPS if prec == "fp64" else FP32_PEAK_TFLOPS
    peak_meas = peaks["fp64_fma_tflops"] if prec == "fp64" else peaks["fp32_fma_tflops"]
    hbm_peak = None
    try:
        hbm_peak = json.load(open(PEAKS_PATH)).get("hbm_gbs")
    except Exception:
        pass
    hbm_peak = hbm_peak or 6800.0
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    batch_now = args.batch or (tune or {}).get("chosen", {}).get("batch") or None
    per_kernel = {}
    for k, (ms_tot, n_l) in kinds.items():
        ms_step, l_step = ms_tot / args.steps, n_l / args.steps
        ent = {"ms_per_step": ms_step, "launches_per_step": l_step}
        if k in flops:
            ent["method_tflop_per_step"] = flops[k] / 1e12
            ent["method_tflops"] = flops[k] / (ms_step / 1e3) / 1e12
            ent["alu_frac"] = ent["method_tflops"] / peak_alu
        if k in dense:
            ent["dense_box_tflops"] = dense[k] / (ms_step / 1e3) / 1e12
        fpl = S.n_sf / l_step if l_step else None
        tr, _ = stored_traffic(k, prec, fpl)
        if tr is not None:
            ent["dram_gb_per_launch"] = tr / 1e9
            ent["dram_gbs"] = tr / (ms_tot / n_l / 1e3) / 1e9
            ent["hbm_frac"] = ent["dram_gbs"] / hbm_peak
        per_kernel[k] = ent
    dom = max(kinds, key=lambda k: kinds[k][0]) if kinds else None
    roof = None
    if dom is not None:
        ms_tot, n_launch = kinds[dom]
        per_launch_ms = ms_tot / n_launch
        fpl = S.n_sf / (n_launch / args.steps)
        traffic, traffic_note = stored_traffic(dom, prec, fpl)
        if dom in flops:
            work_per_launch = flops[dom] / (n_launch / args.steps)
            ach = work_per_launch / (per_launch_ms / 1000.0) / 1e12
            roof = {"kernel": dom, "bound": "alu", "achieved": ach, "peak": peak_alu, "unit": "TFLOP/s",
                    "frac": ach / peak_alu, "traffic": traffic, "traffic_note": traffic_note,
                    "work": "method flop per launch %.4g (workcount: in-range taps over the nonzero support of each "
                            "pass, %s)" % (work_per_launch, "exact" if wnote.get("exact") else
                                           "exact on %d sampled atoms" % wnote.get("atoms_counted", 0)),
                    "peak_source": "%s: 152 SMs x %s x 2 flop x 2.07 GHz (recipe unit counts and clock); the FMA "
                                   "loop of lsw_measure_peaks reaches %.1f on this GPU"
                                   % ("FP64 nominal" if prec == "fp64" else "FP32 nominal",
                                      "FP64 units" if prec == "fp64" else "128 lanes", peak_meas)}
    kshare = {k: round(v[0] / sum(x[0] for x in kinds.values()), 4) for k, v in kinds.items()} if kinds else {}
    launches_per_step = int(sum(v[1] for v in kinds.values()) / args.steps) if kinds else None

    cpu = err = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cores = os.cpu_count() or 1
        n_fn = min(S.n_sf, args.oracle_functions)
        fs, atoms = sample_functions(wl, n_fn)
        pool = OraclePool(args.workload or "atoms10k", atoms, cores)
        try:
            ref, t_h, t_e = oracle_run(wl, pool, fs, S.row_ptr, S.col, max_entries=400)
        finally:
            pool.close()
        cpu = cpu_baseline_of(wl, len(fs), nnz / S.n_sf, t_h, t_e, cores, len(ref["entries"]))
        step()
        torch.cuda.synchronize()
        err = error_report(ref, S, hphi, ek, ep, Hm, Sm)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "support_functions/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
                "higher_is_better": True, "scaling": "strong" if sharded else "weak", "vs_baseline": None,
                "dtype": {"fp64": "f64", "fp32": "f32", "bf16x": "f32+bf16x3"}[prec], "data": "synthetic",
                "config": canonical_config(wl_glob, prec, n_sf_job),
                "e2e": e2e, "e2e_with_hphi": e2e_h, "roofline": roof, "cpu_baseline": cpu,
                "error_vs_oracle": err, "clocks": clocks,
                "gpu_launches": (launches_per_step * args.steps) if launches_per_step else None,
                "parallelism": ("sharded: x slabs, halo exchange of phi and H phi by NCCL send/recv" if sharded
                                else "replicas" if world > 1 else "single"),
                "pattern_nnz": nnz,
                "tuning": {"options": {**(tune or {}).get("chosen", {"batch": args.batch or None,
                                                                       "tile": args.tile or None}), **set_opts},
                           "autotune_ms": {k: v for k, v in (tune or {}).items() if k != "chosen"}},
                "kernels": per_kernel, "kernel_share": kshare, "work_count": wnote,
                "dense_box_tflop_per_step": {k: v / 1e12 for k, v in dense.items()},
                "compulsory_gb_per_step": comp_bytes / 1e9,
                "compulsory_hbm_frac": comp_bytes / (total_ms / args.steps / 1e3) / 1e9 / hbm_peak,
                "peaks_measured": peaks, "setup_s": t_setup, "step_ms": step_ms}
        print(json.dumps(line))
    S.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


def serving_main(args):
    """p50/p99 latency and support functions/s of the served form (split-bfloat16 z stage,
    FP32 elsewhere, batched, graphs, one stream per request in flight) on a Poisson
    stream of 50-5,000-atom systems with 30 % reuse: at the offered 20 req/s, and at a
    rate the GPU sustains (0.8 x the throughput the first run measured, in requests/s of
    the same size mix), where the latency is the server's and not the queue's.  Against
    the same requests, each run alone on the plain form (FP64, one function per batch,
    no graphs), one after another."""
    import torch
    from paper_1401_7441_gb300 import serving as SV
    from paper_1401_7441_gb300 import lsw
    runs = {}
    clk = None
    for tag, rate in (("offered_20_per_s", 20.0), ("sustained", None)):
        if rate is None:
            first = runs["offered_20_per_s"]
            mean_sf = first["support_functions"] / max(1, first["requests"])
            rate = 0.8 * first["support_functions_per_s"] / max(mean_sf, 1.0)
        reqs = SV.request_stream(args.requests, rate=rate, atoms=(50, 5000), reuse_frac=0.3, seed=5005)
        srv = SV.Server(budget_bytes=150e9, precision=lsw.LSW_FP32_BF16X, streams=4, host_threads=8)
        t0 = time.perf_counter()
        with ClockSampler(os.path.join(tempfile.gettempdir(), "lsw_clk_srv_%d.csv" % os.getpid())) as c:
            res = srv.run(reqs, realtime=True)
        wall = time.perf_counter() - t0
        srv.close()
        runs[tag] = dict(SV.summarize(res), rate_per_s=rate, wall_s=wall)
        clk = clk or c.summary(0)
    # the plain form on the same requests (the sustained run's stream), each alone
    reqs = SV.request_stream(args.requests, rate=runs["sustained"]["rate_per_s"], atoms=(50, 5000),
                             reuse_frac=0.3, seed=5005)
    lat, nsf = [], 0
    t1 = time.perf_counter()
    for r in reqs:
        sub = [r] if r.parent is None else [q for q in reqs if q.rid == r.parent] + [r]
        p = SV.Server(budget_bytes=150e9, precision=lsw.LSW_FP64, streams=1, host_threads=1, graphs=False)
        out = {x.rid: x for x in p.run(sub, realtime=False, max_inflight=1)}
        p.close()
        lat.append(out[r.rid].t_done - out[r.rid].t_admit)
        nsf += out[r.rid].n_sf
    plain_s = time.perf_counter() - t1
    served = runs["sustained"]
    line = {"metric": METRIC + " (serving)", "value": served["support_functions_per_s"],
            "unit": "support_functions/s", "n_gpus": 1, "steps": served["requests"], "warmup": 0,
            "ms_per_step": 1000.0 * served["span_s"] / max(1, served["requests"]), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16x3", "data": "synthetic",
            "config": {"workload": "serving: Poisson stream, 50-5,000 atoms log-uniform, 30% reuse",
                       "requests": served["requests"], "budget_gb": 150},
            "serving": runs,
            "plain_alone": {"requests": len(reqs), "support_functions_per_s": nsf / plain_s,
                            "p50_latency_s": float(np.percentile(lat, 50)),
                            "p99_latency_s": float(np.percentile(lat, 99)),
                            "note": "the same requests, FP64, one function per batch, no graphs, one at a time"},
            "clocks": clk}
    print(json.dumps(line))
    return 0


def density_work(wl, geo_boxes, row_ptr, col):
    """Algorithmic work of one density build.  The quadratic form at a point needs, with
    K's symmetry, one multiply-add per unordered pattern pair (a <= b) whose real-space
    blocks both contain the point, and one per function there (the outer product):
    FMAs = sum over pattern pairs a <= b of |B_a n B_b| + sum_a |B_a|."""
    lo, hi = geo_boxes                     # (n_sf, 3) inclusive fine-index blocks
    n = len(row_ptr) - 1
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    cols = np.asarray(col, np.int64)
    keep = rows <= cols
    a, b = rows[keep], cols[keep]
    ext = np.clip(np.minimum(hi[a], hi[b]) - np.maximum(lo[a], lo[b]) + 1, 0, None)
    pair_pts = float(np.sum(np.prod(ext.astype(np.float64), axis=1)))
    own = float(np.sum(np.prod((hi - lo + 1).astype(np.float64), axis=1)))
    return pair_pts + own


def density_main(args):
    """Throughput of lsw_build_density (Eq. density) on a locreg workload: support
    functions per second for the real-space values of every function plus the density
    on the whole fine grid, inputs resident in HBM, L2 flushed before every step."""
    import torch
    from paper_1401_7441_gb300 import build as B
    from paper_1401_7441_gb300 import lsw
    torch.cuda.set_device(0)
    B.build()
    wl = workload(args.workload or "atoms1200")
    prec = args.precision or ("fp64" if wl.precision == "fp64" else "fp32")
    P = {"fp64": lsw.LSW_FP64, "fp32": lsw.LSW_FP32, "bf16x": lsw.LSW_FP32_BF16X}[prec]
    dt = torch.float64 if prec == "fp64" else torch.float32
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    t_setup = time.perf_counter()
    S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   wl.lprime_margin, 0, P, device=0, stream=stream.cuda_stream)
    phi = torch.zeros(S.total_L, dtype=dt, device="cuda")
    atoms = sorted(set(int(a) for a in S.sf_atom))
    cg = {a: keys_to_g(S.keys(a, 0, 0)) for a in atoms}
    fg = {a: keys_to_g(S.keys(a, 0, 1)) for a in atoms}
    I.fill_phi(wl, phi, S.off_L, S.sf_atom, cg, fg)
    Kh = I.density_kernel(wl, S.sf_atom, S.row_ptr, S.col)
    K = torch.tensor(Kh, dtype=torch.float64, device="cuda")
    dims = wl.V_shape
    rho = torch.empty((dims[2], dims[1], dims[0]), dtype=torch.float64, device="cuda")
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def box(k):
        g0, g1 = k[:, 0], k[:, 1]
        return (np.array([(g0 % wl.N[0]).min(), ((g0 // wl.N[0]) % wl.N[1]).min(), (g0 // (wl.N[0] * wl.N[1])).min()]),
                np.array([(g1 % wl.N[0]).max(), ((g1 // wl.N[0]) % wl.N[1]).max(), (g1 // (wl.N[0] * wl.N[1])).max()]))
    bx = {a: box(S.keys(a, 0, 0)) for a in atoms}
    blo = np.array([2 * bx[int(a)][0] - 14 for a in S.sf_atom])
    bhi = np.array([2 * bx[int(a)][1] + 16 for a in S.sf_atom])
    fma = density_work(wl, (blo, bhi), S.row_ptr, S.col)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t_setup

    def step():
        lsw.lsw_build_density(S.sys, phi, K, rho, wl.V_lo, dims)

    peaks = dict(zip(("fp32_fma_tflops", "fp64_fma_tflops", "copy_gbs"), lsw.lsw_measure_peaks(S.ctx)))
    for _ in range(max(1, args.warmup)):
        step()
    lsw.lsw_sync(S.sys, 600.0)
    lsw.lsw_profile(S.sys, 1)
    step()
    lsw.lsw_profile_read(S.sys)
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    prof = {}
    with ClockSampler(os.path.join(tempfile.gettempdir(), "lsw_clk_dens_%d.csv" % os.getpid())) as clk:
        time.sleep(0.3)
        for i in range(args.steps):
            flush.fill_(float(i))
            torch.cuda.synchronize()
            ev0[i].record(stream)
            step()
            ev1[i].record(stream)
            torch.cuda.synchronize()
            for k, (ms, n) in lsw.lsw_profile_read(S.sys).items():
                a, b = prof.get(k, (0.0, 0))
                prof[k] = (a + ms, b + n)
    lsw.lsw_profile(S.sys, 0)
    lsw.lsw_sync(S.sys, 60.0)
    step_ms = [ev0[i].elapsed_time(ev1[i]) for i in range(args.steps)]
    total_ms = sum(step_ms)
    kinds = {k: v for k, v in prof.items() if v[1] > 0}
    roof = None
    if "dens_products" in kinds:
        ms_tot, n_launch = kinds["dens_products"]
        ach = 2.0 * fma / (ms_tot / n_launch / 1000.0) / 1e12
        peak = peaks["fp64_fma_tflops"] if prec == "fp64" else peaks["fp32_fma_tflops"]
        roof = {"kernel": "dens_products", "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None,
                "work": "2 x (sum over pattern pairs a <= b of the points both real-space blocks contain "
                        "+ sum of block sizes) = %.3e flop per launch" % (2.0 * fma),
                "peak_source": "measured on this GPU: %s FMA loop over every SM (lsw_measure_peaks)"
                               % ("FP64" if prec == "fp64" else "FP32")}
    cpu = None
    if not args.no_cpu:
        from oracle import density as Dn
        from oracle import filters as OF
        from oracle import geometry as G
        c = np.asarray(wl.pos).mean(axis=0)
        near = set(np.nonzero(np.sum((np.asarray(wl.pos) - c) ** 2, axis=1) <= 8.0 ** 2)[0].tolist())
        sel = [f for f in range(S.n_sf) if int(S.sf_atom[f]) in near]
        t0 = time.perf_counter()
        desc = G.SystemDesc(tuple(wl.N), wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff,
                            wl.pair_mode, wl.lprime_margin, wl.fine_mode)
        geo = G.build(desc, atoms=sorted(near), pattern=False)
        FO = OF.load()
        fields = {}
        for f in sel:
            L = geo.L[int(S.sf_atom[f])]
            fields[f] = Dn.realspace(geo, f, I.phi_values(wl, f, int(S.sf_atom[f]), L.coarse.g, L.fine.g), FO)
        ents = [(a, int(S.col[k]), float(Kh[k])) for a in sel for k in range(S.row_ptr[a], S.row_ptr[a + 1])
                if int(S.col[k]) in fields]
        Dn.accumulate(fields, ents, wl.V_lo, dims)
        el = time.perf_counter() - t0
        cpu = {"value": len(sel) / el, "unit": "support_functions/s", "cores": 1, "kind": "oracle",
               "sample": "oracle (numpy FP64, 1 thread of %d host cores): real-space values of the %d functions "
                         "on the atoms within 8 bohr of the centre and the density of the %d pattern entries "
                         "among them on the whole grid; %.1f s" % (os.cpu_count() or 1, len(sel), len(ents), el)}
    line = {"metric": "density build: support functions/s (real-space values + rho on the fine grid)",
            "value": S.n_sf * args.steps / (total_ms / 1000.0), "unit": "support_functions/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "bf16x": "f32"}[prec] + " (FP64 sums per point)",
            "data": "synthetic",
            "config": {"workload": wl.name, "atoms": len(wl.pos), "support_functions": S.n_sf,
                       "pattern_nnz": len(S.col), "grid_points": int(np.prod(dims)), "precision": prec,
                       "l2": "flushed (512 MB write) before every timed step"},
            "roofline": roof, "cpu_baseline": cpu, "peaks_measured": peaks, "clocks": clk.summary(0),
            "gpu_launches": int(sum(v[1] for v in kinds.values())) if kinds else None,
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in kinds.items()},
            "algorithmic_gflop_per_step": 2.0 * fma / 1e9,
            "workspace_gb": lsw.lsw_workspace_bytes(S.sys) / 1e9, "setup_s": t_setup, "step_ms": step_ms}
    print(json.dumps(line))
    S.close()
    return 0


def _make_system(lsw, torch, wl, P, stream, options=None):
    dt = torch.float64 if P == lsw.LSW_FP64 else torch.float32
    S = lsw.System(wl.N, wl.h, wl.pos, wl.r_loc, wl.r_fine, wl.nsf, wl.pair_cutoff, wl.pair_mode,
                   wl.lprime_margin, 0, P, device=0, stream=stream.cuda_stream)
    for k, v in (options or {}).items():
        lsw.lsw_set_option(S.sys, k, v)
    phi = torch.zeros(S.total_L, dtype=dt, device="cuda")
    atoms = sorted(set(int(a) for a in S.sf_atom))
    I.fill_phi(wl, phi, S.off_L, S.sf_atom, {a: keys_to_g(S.keys(a, 0, 0)) for a in atoms},
               {a: keys_to_g(S.keys(a, 0, 1)) for a in atoms})
    V = I.potential_fast(wl, "cuda").to(dt)
    lsw.lsw_set_potential(S.sys, V, wl.V_lo, wl.V_shape)
    nnz = len(S.col)
    bufs = dict(phi=phi, V=V, hphi=torch.zeros(S.total_Lp, dtype=dt, device="cuda"),
                ek=torch.zeros(S.n_sf, dtype=torch.float64, device="cuda"),
                ep=torch.zeros(S.n_sf, dtype=torch.float64, device="cuda"),
                H=torch.zeros(max(1, nnz), dtype=torch.float64, device="cuda"),
                S=torch.zeros(max(1, nnz), dtype=torch.float64, device="cuda"))
    return S, bufs


def _timed_steps(lsw, torch, S, b, stream, steps, flush):
    ts = []
    for i in range(steps):
        flush.fill_(float(i))
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        lsw.lsw_apply_hamiltonian(S.sys, b["phi"], b["hphi"], b["ek"], b["ep"])
        lsw.lsw_build_matrices(S.sys, b["phi"], b["hphi"], b["H"], b["S"])
        e1.record(stream)
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    return ts


def compare_main(args):
    """Served form against the plain form on one system: the served form (split-bfloat16 z stage,
    FP32 elsewhere, batched, graphs, autotuned) against the plain per-locreg FP64 GPU form
    (FP64, one function per batch, no graphs), both through the library; every H phi
    element and every H/S entry of the served form against the FP64 form, and both
    against the oracle on a sample of functions."""
    import torch
    from paper_1401_7441_gb300 import build as B
    from paper_1401_7441_gb300 import lsw
    torch.cuda.set_device(0)
    B.build()
    wl = workload(args.workload or "atoms10k")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    # plain FP64 form: one function per batch, no graph
    S64, b64 = _make_system(lsw, torch, wl, lsw.LSW_FP64, stream, {"batch": 1, "graph": 0})
    _timed_steps(lsw, torch, S64, b64, stream, 1, flush)
    t64 = _timed_steps(lsw, torch, S64, b64, stream, max(1, min(args.steps, 2)), flush)
    hp64 = b64["hphi"].cpu().numpy()
    H64, S64v = b64["H"].cpu().numpy(), b64["S"].cpu().numpy()
    ek64, ep64 = b64["ek"].cpu().numpy(), b64["ep"].cpu().numpy()
    off_Lp, row_ptr, col = S64.off_Lp, S64.row_ptr, S64.col
    phi64 = b64["phi"].cpu().numpy()
    S64.close()
    del b64
    torch.cuda.empty_cache()
    # served form
    Ssv, bsv = _make_system(lsw, torch, wl, lsw.LSW_FP32_BF16X, stream,
                            {"batch": args.batch or 512, "tile": args.tile or 5})
    _timed_steps(lsw, torch, Ssv, bsv, stream, max(3, args.warmup), flush)
    tsv = _timed_steps(lsw, torch, Ssv, bsv, stream, args.steps, flush)
    hpsv = bsv["hphi"].double().cpu().numpy()
    Hsv, Ssvv = bsv["H"].cpu().numpy(), bsv["S"].cpu().numpy()
    # served against FP64 GPU: every function, element by element and normwise
    n = Ssv.n_sf
    el, nw = [], []
    for f in range(n):
        a, b = int(off_Lp[f]), int(off_Lp[f + 1])
        ref = hp64[a:b]
        g = hpsv[a:b]
        m = np.max(np.abs(ref))
        el.append(float(np.max(np.abs(g - ref)) / m) if m > 0 else 0.0)
        nw.append(float(np.linalg.norm(g - ref) / max(np.linalg.norm(ref), 1e-300)))
    rows = np.repeat(np.arange(n), np.diff(row_ptr))
    sd = np.sqrt(np.abs(S64v[row_ptr[:-1] + np.array([np.searchsorted(col[row_ptr[i]:row_ptr[i + 1]], i)
                                                       for i in range(n)])]))
    hn = np.array([np.linalg.norm(hp64[off_Lp[f]:off_Lp[f + 1]]) for f in range(n)])
    s_err = np.abs(Ssvv - S64v) / (sd[rows] * sd[col])
    h_err = np.abs(Hsv - H64) / (sd[rows] * hn[col])
    vs64 = {"functions": n, "entries": int(len(col)), "hphi_elem_rel_max": max(el), "hphi_rel_max": max(nw),
            "S_scaled_max": float(np.max(s_err)), "H_scaled_max": float(np.max(h_err)),
            "note": "element errors relative to the largest |H phi| of the function; entries Cauchy-Schwarz scaled"}
    # both against the oracle on a sample
    cpu = err_sv = err_64 = None
    if not args.no_cpu:
        cores = os.cpu_count() or 1
        fs, atoms = sample_functions(wl, min(n, args.oracle_functions))
        pool = OraclePool(args.workload or "atoms10k", atoms, cores)
        try:
            ref, t_h, t_e = oracle_run(wl, pool, fs, Ssv.row_ptr, Ssv.col, max_entries=400)
        finally:
            pool.close()
        cpu = cpu_baseline_of(wl, len(fs), len(col) / n, t_h, t_e, cores, len(ref["entries"]))
        err_sv = error_report(ref, Ssv, bsv["hphi"], bsv["ek"], bsv["ep"], bsv["H"], bsv["S"])
        err_64 = error_report(ref, Ssv, hp64, ek64, ep64, H64, S64v, tag="FP64 CPU oracle (plain FP64 GPU form)")
    _ = phi64
    v64 = n / (statistics.median(t64) / 1000.0)
    vsv = n / (statistics.median(tsv) / 1000.0)
    line = {"metric": METRIC + " (served vs plain FP64 form)", "value": vsv, "unit": "support_functions/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(tsv),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16x3",
            "data": "synthetic", "config": canonical_config(wl, "bf16x", n),
            "plain_fp64": {"value": v64, "ms_per_step": statistics.median(t64),
                           "form": "FP64, one function per batch, no CUDA graph"},
            "speedup_vs_plain_fp64": vsv / v64, "served_vs_fp64_gpu": vs64,
            "served_vs_oracle": err_sv, "fp64_gpu_vs_oracle": err_64, "cpu_baseline": cpu}
    print(json.dumps(line))
    Ssv.close()
    return 0


def foe_main(args):
    """The Fermi operator expansion (lsw_foe) on the H and S the library builds for a
    workload (symmetrized on the pattern).  Spectrum bounds: the Gershgorin discs of H,
    widened by 10 % (S is close to the identity here).  Reports the time of one expansion
    (both passes of the Chebyshev recursion, the triple products, the host search of mu)
    and the work of the recursion: per step one multiply-add per (pattern entry, common
    index) pair."""
    import torch
    from paper_1401_7441_gb300 import build as B
    from paper_1401_7441_gb300 import lsw
    torch.cuda.set_device(0)
    B.build()
    wl = workload(args.workload or "atoms1200")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    S, b = _make_system(lsw, torch, wl, lsw.LSW_FP64, stream, {})
    _timed_steps(lsw, torch, S, b, stream, 1, flush)
    n = S.n_sf
    rp, col = S.row_ptr, S.col
    rows = np.repeat(np.arange(n), np.diff(rp))
    # symmetrize on the pattern (the transposed position of every entry)
    key = rows.astype(np.int64) * n + col
    tkey = col.astype(np.int64) * n + rows
    tpos = np.searchsorted(key, tkey)
    Hh, Sh = b["H"].cpu().numpy(), b["S"].cpu().numpy()
    Hs, Ss = 0.5 * (Hh + Hh[tpos]), 0.5 * (Sh + Sh[tpos])
    # spectrum bounds: Gershgorin discs of H with the S-weighting ignored, widened by 10 %
    diag = Hs[key == rows.astype(np.int64) * (n + 1)]
    radius = np.bincount(rows, weights=np.abs(Hs), minlength=n) - np.abs(diag)
    e_min, e_max = float(np.min(diag - radius)), float(np.max(diag + radius))
    span = e_max - e_min
    e_min, e_max = e_min - 0.1 * span, e_max + 0.1 * span
    n_pl = 100
    Hd, Sd = torch.tensor(Hs, device="cuda"), torch.tensor(Ss, device="cuda")
    Kp, K = torch.zeros_like(Hd), torch.zeros_like(Hd)
    lsw.lsw_foe(S.sys, Hd, Sd, e_min, e_max, n / 2.0, n_pl, 0.05 * span, Kp, K)     # warm-up
    ts = []
    for _ in range(max(1, args.steps)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        mu, ebs, tr = lsw.lsw_foe(S.sys, Hd, Sd, e_min, e_max, n / 2.0, n_pl, 0.05 * span, Kp, K)
        ts.append(time.perf_counter() - t0)
    # work of one Chebyshev step: sum over pattern entries (i, l) of |row_i n row_l|
    import scipy.sparse as sp
    P = sp.csr_matrix((np.ones(len(col)), col, rp), shape=(n, n))
    PP = (P @ P).tocsr()
    common = float(np.asarray(PP[rows, col]).sum())
    flops = 2.0 * common * (2 * n_pl)          # two passes of n_pl steps
    t = statistics.median(ts)
    line = {"metric": "Fermi operator expansion: seconds per density kernel (n_pl = %d, 2 passes)" % n_pl,
            "value": t, "unit": "s", "n_gpus": 1, "steps": len(ts), "warmup": 1, "ms_per_step": 1000.0 * t,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": wl.name, "support_functions": n, "pattern_nnz": int(len(col))},
            "mu": mu, "E_BS": ebs, "trace": tr, "n_el": n / 2.0,
            "algorithmic_gflop": flops / 1e9, "achieved_tflops": flops / t / 1e12,
            "roofline": {"bound": "alu", "achieved": flops / t / 1e12, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                         "frac": flops / t / 1e12 / FP64_PEAK_TFLOPS,
                         "note": "Chebyshev products only (2 x n_pl steps); the triple products and the host "
                                 "search of mu are in the time but not in the flop count"}}
    print(json.dumps(line))
    S.close()
    return 0


def main():
    args = parse()
    if args.record_traffic:
        wl = workload(args.workload or "atoms10k")
        print(record_traffic(args.record_traffic, wl, args.precision or wl.precision, args.batch or 512))
        return 0
    if args.impl == "reference":
        return reference_main(args)
    if args.mode == "serving":
        return serving_main(args)
    if args.mode == "density":
        return density_main(args)
    if args.mode == "compare":
        return compare_main(args)
    if args.mode == "foe":
        return foe_main(args)
    return gpu_main(args)


if __name__ == "__main__":
    sys.exit(main())
